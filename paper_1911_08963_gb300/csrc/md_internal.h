// md_internal.h -- types shared by the host planner, the CUDA kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "md.h"

namespace mdl {

constexpr int kMaxN = MD_MAX_N;
constexpr int kMaxWords = kMaxN / 32;         // 32-bit words of a packed row
constexpr int kMaxG = 64;                     // deepest stage g handled
#ifndef MD_UPPERS_PER_LANE
#define MD_UPPERS_PER_LANE 2
#endif
constexpr int kUppersPerLane = MD_UPPERS_PER_LANE;  // upper parts a lane walks at once
constexpr int kMaxLevels = MD_MAX_LEVELS;
constexpr int kRankBits = 55;                 // level key = weight << 55 | colex rank
constexpr uint64_t kRankLimit = 1ull << kRankBits;
constexpr uint64_t kNoKey = ~0ull;
constexpr int MD_EAGAIN_INTERNAL = 100;       // engine: the run needs stages past its plan
constexpr uint64_t kBatchHeavyDefault = 1ull << 34;   // md_batch: single-code runs from this estimated work

// -------------------------------------------------------------------- host side ---

// One systematic matrix Gamma_j (Section 2.1).  Full-rank (k_j = k): the k columns of
// S_j hold an identity, so the weight of a sum of g rows is g plus the weight of the
// sum over the other n - k columns, and only those columns are packed.  Rank-deficient
// (the leftover columns, Gamma_m = [[I, A], [0, B]]): every column is packed and the
// weight is the popcount of the packed row alone.
struct Gamma {
    int rank = 0;                   // k_j
    std::vector<int> order;         // reduction order: the set's columns, then the rest
    std::vector<uint64_t> rows;     // k x nw64 full rows in the original column order
    std::vector<int> packed_cols;   // original column of each packed bit
    int W = 0;                      // 32-bit words holding the packed columns
    int WP = 0;                     // row stride in words on the device (1, 2, 4 or 8)
    int weight_base_is_g = 0;       // 1 for full rank: weight = g + popcount(packed)
    std::vector<uint32_t> packed;   // k x WP words
    unsigned long long fmax8 = 0;   // filter thresholds for the default mode (see plan_level)
};

struct Code {
    int n = 0, k = 0, nw64 = 0;
    std::vector<uint64_t> G;        // in the processing column order (see perm)
    std::vector<Gamma> gam;
    std::vector<int> perm;          // processing position -> caller's column (empty: identity)
};

// Validate, check rank, find the information sets and build every Gamma_j.
int build_code(const uint64_t *G, int n, int k, Code *out);

// As build_code, after choosing a column order (Section 2.2: random column permutations, the
// one with the most full-rank information sets and then the largest rank of the last set).
// trials <= 1: the caller's order.  Trial 0 is the caller's order; trial t >= 1 is a
// Fisher-Yates shuffle driven by SplitMix64(seed) (one stream for all trials: for i = n-1
// down to 1, swap position i with position next() mod (i+1)).  Ties keep the earlier trial.
int build_code_permuted(const uint64_t *G, int n, int k, int trials, uint64_t seed, Code *out);

// A row in the processing order -> the caller's column order.
void to_caller_order(const Code &c, const uint64_t *row, uint64_t *out);

uint64_t binom(int a, int b);                   // saturating at UINT64_MAX
void colex_unrank(uint64_t r, int g, int k, int *c);
int popcount_row(const uint64_t *row, int nw);

// Lower bound after stage g (Alg. 1): L(g) = sum_j max(0, g + 1 - (k - k_j)).
int lower_bound_after(const Code &c, int g);

// Work plan of one level (g, j).  A combination c_1 < ... < c_g splits into a head
// (c_1..c_P), the pivot element M = c_{P+1} and an upper part (c_{P+2}..c_g) of v
// elements.  Work items group the upper parts that share M: a warp gives each lane its
// own run of upper parts and walks all heads below M in lockstep.
struct MEntry {
    uint64_t chunk_begin;   // first work item of this M
    uint64_t uppers;        // number of upper parts covered (C(k - 1 - M, v) for a level)
    uint64_t upper_base;    // colex index of the first covered upper part
    uint32_t M;
    uint32_t per_lane;      // upper parts per lane in one work item
};

enum KernelKind : int { KIND_SIMPLE = 0, KIND_SPLIT2 = 2, KIND_SPLIT3 = 3, KIND_TC = 4 };

struct LevelPlan {
    int g = 0, j = 0;
    int kind = KIND_SIMPLE;         // 0 = per-lane rank ranges; 2, 3 = head size P
    int v = 0;                      // upper elements per lane (kinds 2, 3)
    int base = 0;                   // weight base (g or 0)
    int L_after = -1;               // lower bound once this level is complete (-1: unchanged)
    int L_first = 0;                // 1: raise L before the check after this level (rule 1)
    // filter thresholds: byte f-1 holds 1 + the largest packed-weight threshold at which the
    // popcount of the OR of the first f words still rejects almost every codeword (0 = never)
    unsigned long long fmax8 = 0;
    uint64_t count = 0;             // C(k, g)
    uint64_t nchunks = 0;
    uint64_t per_chunk = 0;         // kind 0: ranks per lane
    std::vector<MEntry> mtab;       // kinds 2, 3
    int tc_q = 0;                   // kind 4: head size q (tail = the other g - q elements)
    int tc_smin = 0;                // kind 4: combinations with c_{q+1} < tc_smin use (q+1)-heads
    unsigned long long tc_words8 = 0;   // kind 4: word counts of the product (tc_word_thresholds)
};

struct PlanOptions {
    int stop_rule = 0;              // 0: Alg. 1 stage bound; 1: per-matrix bound
    int perm_trials = 0;            // column orders tried (build_code_permuted)
    uint64_t perm_seed = 0;
    int chunk_log2 = 20;
    int filter = 1;                 // 0 = never, 1 = when it pays, 2 = always
    int tensor = 0;                 // 0 = never, 1 = large levels, 2 = every level it can run
    int tensor_head = 0;            // q for the tensor-core levels (0 = automatic)
};

// ---- tensor-core levels (md_tc.cu) ----
size_t tc_tables_bytes(int k, int q, int W);  // head table of one matrix
int tc_smem_bytes(int k, int W, int optin, int *with_bsub);

// Raise a kernel's dynamic shared-memory limit to the most the current device allows, once per
// kernel and device (thread-safe).  The limit is an attribute of the kernel for the whole
// process: set per launch to that launch's size, two threads launching the same kernel with
// different sizes (distinct handles, batch workers) could lower it under each other's launch.
// The occupancy of a launch still follows the size it requests.  Returns a cudaError_t value.
int allow_full_smem(const void *kernel);
uint64_t tc_level_items(int k, int g, int q, int smin, int W);
int tc_split_point(int k, int q);   // s_min of the two-phase split (see md_tc.cu)
size_t tc_heads_bytes(uint64_t nheads, int W);
int tc_auto_head(int k, int W);     // q used when PlanOptions::tensor_head is 0
int tc_max_upper();                 // largest g - q - 1 the tensor-core kernel handles

LevelPlan plan_level(const Code &c, int g, int j, const PlanOptions &o);

// Largest threshold t with P(popcount(OR of the first f packed words) <= t) below 1e-5 for
// uniformly random packed rows (-1 if none): above it the filter would rarely reject.
int filter_threshold(const Gamma &gm, int f, double pmax);
unsigned long long filter_thresholds(const Gamma &gm, int mode);
unsigned long long tc_word_thresholds(const Gamma &gm, int mode);

// -------------------------------------------------------------------- device side ---

// Device-resident state of one code run.
struct DevState {
    unsigned int U;                 // least weight found (n + 1 = none yet)
    int L;                          // current lower bound
    int stop;                       // set once L >= U
    int error;                      // device-side error code (0 = none)
    int last_level;                 // last level finalised
    int pad;
    unsigned long long skipped;     // work left out by the mid-level stop
    unsigned int u_in[kMaxLevels];  // U when each level started
    unsigned long long key[kMaxLevels];   // per-level least (weight << 55 | first rank)
    unsigned long long ctr[kMaxLevels];   // per-level work-item counters
};

// Kernel arguments of one level.
struct LevelArgs {
    const uint32_t *rows;           // k x WP
    const uint32_t *h2;             // C(k, 2) x WP, pair sums in colex order
    const unsigned long long *binom;// (k + 1) x (k + 1): C(a, b) at a * (k + 1) + b
    const MEntry *mtab;
    DevState *st;
    unsigned long long nchunks;
    unsigned long long count;       // kind 0: end of the rank range (C(k, g) for a level)
    unsigned long long r_begin;     // kind 0: start of the rank range (0 for a level)
    unsigned long long per_chunk;
    int n_m;
    int k, g, v, base, level;
    unsigned long long fmax8;
    int h2_in_smem;
    int m_total;                    // number of Gamma matrices
    int j;
    int L_after;
    int L_first;
    int check_stop;                 // 0 for md_scan_range (no stop logic)
    const volatile int *cancel;     // non-zero: stop before the next work item (null: none)
};

// ---- many codes: the engine behind md_batch and the server (md_engine.cu) ----
constexpr int kWClasses = 9;                // index by W = 1..8

// One level of one code.
struct BLevel {
    const uint32_t *rows;           // Gamma_j packed rows (k x WP), global memory
    const uint32_t *h2;             // Gamma_j pair table
    const MEntry *mtab;
    unsigned long long nchunks, count, per_chunk;
    unsigned long long fmax8;
    unsigned long long quota;       // work items per tick (0 = the whole level)
    int n_m, g, v, base, kind, L_after, j, W, WP, L_first;
};

// A slot of the engine: one resident code (written by the host on admission).
struct BCode {
    const BLevel *levels;           // nlev levels, level l = (g - 1) * m + j
    unsigned long long *keys;       // per-level least (weight << 55 | first rank)
    int k, m, nlev, live;
};

// Device-side state of a slot: Alg. 1's bounds plus the level cursor.
struct BState {
    unsigned int U;                 // least weight found (n + 1 = none yet)
    int L, stop, last_level;
    int cur;                        // level being enumerated
    int pad;
    unsigned long long next_item;   // first work item of `cur` not yet handed out
    unsigned long long tick_items;  // items of `cur` handed out in the current tick (0 = idle)
};

struct EngineArgs {
    const BCode *codes;
    BState *states;
    int nslots;
    int *act_slots;                 // [kWClasses][nslots]: slots running in this tick, per row width
    unsigned long long *act_prefix; // inclusive prefix of their items
    int *act_count;                 // [kWClasses]
    unsigned long long *act_total;  // [kWClasses]
    unsigned long long *tick_ctr;   // [kWClasses] work-item tickets of the current tick
    const unsigned long long *binom;// 257 x 257
};

int launch_engine_prepare(const EngineArgs &a, void *stream);
int launch_engine_round(const EngineArgs &a, int W, int blocks, int threads, void *stream);
int launch_engine_post(const EngineArgs &a, void *stream);
int engine_blocks_per_sm(int W, int threads);
int launch_h2_build_many(const uint32_t *const *rows, uint32_t *const *h2, const int *k, const int *WP, int count,
                         void *stream);

// Estimated combinations until L >= U for a random code with these parameters (the
// expected weight distribution C(n, w) / 2^(n-k) gives d_est; g_stop is the first stage with
// L(g) >= d_est).  Used for budgets and admission.
double estimate_work(const Code &c, int *d_est, int *g_stop);

// Launchers (md_kernels.cu).  Return cudaError_t as int.
int launch_h2_build(const uint32_t *rows, uint32_t *h2, int k, int WP, void *stream);
// Tables of Gamma_j for its tensor-core levels (tc_tables_bytes(k, q, W) bytes, 16-byte aligned).
int launch_tc_tables(const uint32_t *rows, const unsigned long long *binom_d, int k, int q, int W, int WP,
                     uint64_t nheads, unsigned char *tables, void *stream);
// One tensor-core level: `blocks` persistent blocks (one per SM), work items from st->ctr[level].
// words8: the product's word counts per threshold (LevelPlan::tc_words8).
int launch_tc_level(const unsigned char *tables, const unsigned char *tables2, int smin, const uint32_t *rows,
                    const unsigned long long *binom_d, DevState *st, int k, int g, int q, int base, int level, int W,
                    int WP, int check_stop, int blocks, int stall, unsigned long long words8,
                    const volatile int *cancel, void *stream);
int launch_level(const LevelArgs &a, int kind, int W, int WP, int blocks, int threads, size_t smem,
                 void *stream);
int launch_finalize(const LevelArgs &a, void *stream);
int launch_state_init(DevState *st, unsigned int u0, void *stream);
int level_smem_bytes(int k, int WP, bool h2_in_smem);
int level_blocks_per_sm(int kind, int W, bool h2_in_smem, int threads, size_t smem);
int max_smem_per_block();
int sm_count();

// Range checks of the debug build (-DMD_DEBUG_BOUNDS): each CUDA source's first failing check
// site (0 = none), read and optionally cleared; the normal build reports 0.
int bounds_site_kernels(unsigned *site, int reset);
int bounds_site_tc(unsigned *site, int reset);
int bounds_site_engine(unsigned *site, int reset);
int bounds_site_noalloc(unsigned *site, int reset);
// MD_EINTERNAL if a range check of the debug build failed since the last call (clears the
// sites), else MD_OK; always MD_OK in the normal build.
int bounds_status();

}  // namespace mdl
