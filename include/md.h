/*
 * md.h -- C ABI of the GB300 minimum-distance library.
 *
 * The library computes the minimum distance d of a binary linear code [n, k] and a
 * codeword of weight d, with the Brouwer-Zimmermann algorithm as described in Section 2.1
 * (Alg. 1) of Quintana-Orti, Hernando and Igual, "Parallel implementations for computing
 * the minimum distance of a random linear code on multicomputers":
 *
 *   - disjoint information sets S_1..S_m of G and the systematic matrices
 *     Gamma_j = (I_k | A_j), plus Gamma_m = [[I_{k_m}, A], [0, B]] for the leftover columns
 *     (Section 2.1), are built on the host by elimination over F2;
 *   - for g = 1, 2, ... and each Gamma_j, every sum of g rows of Gamma_j is formed on the
 *     GPU and its weight tightens the upper bound U (Alg. 1, the U update);
 *   - after each Gamma matrix the bounds are compared (Section 2.2) and after each stage
 *     the lower bound becomes L(g) = sum_j max(0, g + 1 - (k - k_j)) (Alg. 1, the L
 *     update); the run stops once L >= U and returns d = U.
 *
 * Conventions shared by every entry point:
 *   - Matrices are bit-packed rows of uint64 words: row i of a k x n matrix occupies
 *     words [i * ceil(n/64), (i + 1) * ceil(n/64)); bit t of word w is column 64w + t.
 *     Bits beyond column n - 1 must be zero.
 *   - Every call returns an int status (MD_OK or an MD_E* code) and never aborts the
 *     process.  Output arguments are written only when the call returns MD_OK.
 *   - Input buffers are host memory, read during the call and not retained (the library
 *     copies what it needs).  Output buffers are caller-owned host memory.
 *   - A handle may be used by one thread at a time; distinct handles are independent.
 *   - The witness is canonical: among all codewords of weight d that the run enumerates,
 *     the first in (stage g, matrix j, colexicographic rank of the row combination) order.
 *     The colex rank of rows c_1 < ... < c_g (0-based) is sum_i C(c_i, i).
 */
#ifndef MD_H
#define MD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
enum {
    MD_OK = 0,
    MD_EINVAL = 1,        /* bad argument: n < 1, k < 1, k > n, NULL pointer, padding bits set */
    MD_ERANK = 2,         /* G is not of full row rank k */
    MD_EUNSUPPORTED = 3,  /* n > MD_MAX_N, or a level with C(k, g) >= 2^55 combinations */
    MD_ENOMEM = 4,        /* host or device allocation failed */
    MD_ECUDA = 5,         /* a CUDA runtime call failed, or no usable GPU */
    MD_EBUDGET = 6,       /* the work would exceed md_options.work_budget combinations */
    MD_ECANCELED = 7,     /* the run was cancelled through md_options.cancel_flag */
    MD_ETIMEOUT = 8,      /* a bounded device-side wait gave up */
    MD_EBUSY = 9,         /* server: the request is still pending */
    MD_EINTERNAL = 10     /* an internal consistency check failed */
};

#define MD_MAX_N 256      /* longest code supported */
#define MD_MAX_GAMMA 256  /* at most n information sets */
#define MD_MAX_LEVELS 1024

/* Opaque handle of one code: built by md_create, released by md_destroy. */
typedef struct md_ctx *md_handle;

/* Options.  Zero-initialise, or call md_options_init, then set fields. */
typedef struct md_options {
    uint64_t work_budget;     /* max combinations to enumerate; 0 = unlimited.  Exceeding it
                                 (estimated before a stage starts) returns MD_EBUDGET */
    int max_stage;            /* stop after this stage g even if L < U; 0 = run to the end.
                                 The result is then the best weight found (an upper bound)
                                 and md_info reports complete = 0 */
    int chunk_log2;           /* log2 of the combinations per work item; 0 = default (20) */
    int threads_per_block;    /* 0 = default (512) */
    int blocks_per_sm;        /* 0 = default (occupancy-derived) */
    int filter;               /* 1 (default) = reject codewords with a one-popcount lower
                                 bound (popcount of the OR of the fewest packed words that
                                 still proves wt > U for almost all of them); 0 = exact
                                 weight of every codeword; 2 = also filter with all words
                                 when no word count qualifies; 3 = always filter with one
                                 word (a test setting).  Results are identical for all. */
    void *stream;             /* cudaStream_t to run on; NULL = the library's own stream */
    volatile int *cancel_flag;/* optional host flag (ordinary or pinned memory): set non-zero,
                                 from any thread, to cancel a running md_compute, which then
                                 returns MD_ECANCELED.  While the device works the calling
                                 thread polls it (every ~0.1 ms) and passes it on to the
                                 kernels, which check it before each work item; the handle
                                 stays usable and the next md_compute starts afresh */
    int batch_mode;           /* md_batch only: 0 (default) = all codes in one persistent
                                 round schedule; 1 = one md_compute per code, in order */
    int use_graph;            /* md_batch only: 1 (default) = capture the round schedule in a
                                 CUDA graph and launch it once; 0 = plain stream launches */
    int plan_horizon;         /* md_batch only: stages planned past each code's estimated
                                 stopping stage (0 = default 3); a code that needs more is
                                 finished by a single-code run, with the same result */
    int stop_rule;            /* 0 (default) = Alg. 1: after each Gamma matrix compare U with
                                 the L of the last complete stage; 1 = per-matrix bound: after
                                 matrix j of stage g, L = sum_{i<=j} b_i(g) + sum_{i>j} b_i(g-1)
                                 with b_i(g) = max(0, g+1-(k-k_i)).  Both give the same d and
                                 witness; rule 1 can stop inside the last stage */
    int perm_trials;          /* column orders tried before the information sets are chosen
                                 (Section 2.2): trial 0 is the given order, trials 1.. are
                                 Fisher-Yates shuffles driven by SplitMix64(perm_seed); the
                                 order with the most full-rank sets, then the largest rank of
                                 the last set, wins (earlier trial on ties).  0 or 1 = the given
                                 order.  Outputs stay in the caller's column order. */
    uint64_t perm_seed;
    int tensor;               /* md_compute: 1 (default) = run large levels on the tensor cores
                                 (tcgen05 MMA over +-1 encodings of the packed rows, exact
                                 integer results); 0 = never; 2 = every level with g >= q + 1
                                 (a test setting).  Results are identical for all. */
    int tensor_head;          /* head size q of the tensor-core split (2 to 5); 0 = automatic: the
                                 widest of 5, 4, 3 whose head table (C(k, q) rows of the packed
                                 width) fits in 1 GiB, else 2 */
    int test_stall;           /* test hook, 0 in normal use.  1 = in every tensor-core level the
                                 tail producers never signal their first tile set, so the
                                 MMA issuers' bounded wait (4 s) runs out: each block frees
                                 its tensor memory and returns, the run stops, and
                                 md_compute returns MD_ETIMEOUT with the context intact */
    /* Optional device allocator for the library's device buffers (md_compute's per-handle
       buffer, md_scan_task's work table, md_batch's engine tables and code arena), for
       callers whose device memory belongs to another allocator.  dev_alloc returns device
       memory of at least `bytes` bytes aligned to 256 bytes, or NULL on failure (the call
       then returns MD_ENOMEM); dev_free releases it.  Both are called from the thread that
       calls the library, with alloc_ctx.  NULL = cudaMalloc / cudaFree.  Memory is released
       by md_destroy (md_compute) or before the call returns (md_scan_task, md_batch); the
       caller keeps the allocator valid until then. */
    void *(*dev_alloc)(size_t bytes, void *alloc_ctx);
    void (*dev_free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    uint64_t batch_heavy;     /* md_batch: codes whose estimated work (combinations until L >= U
                                 for a random code of that shape) reaches this run as
                                 single-code computations, with the tensor-core levels (such a
                                 code fills the GPU by itself; see batch_workers), while the
                                 others share rounds; 0 = default 2^34, UINT64_MAX = none */
    int autotune;             /* md_batch: 1 = first pick chunk_log2, blocks_per_sm and batch_heavy
                                 with md_batch_tune (cached in tune_cache when set) */
    const char *tune_cache;   /* md_batch_tune's JSON cache file (NULL = no cache) */
    int batch_workers;        /* md_batch: threads that run the single-code computations side by
                                 side, each on a stream of its own, largest estimated work first,
                                 beside the shared rounds (0 = default 2).  With dev_alloc set
                                 they run one by one on the calling thread, the only thread the
                                 allocator is called from. */
} md_options;

/* Result details of the last md_compute on a handle. */
typedef struct md_info {
    int n, k;
    int m;                         /* number of Gamma matrices */
    int ranks[MD_MAX_GAMMA];       /* k_j of each Gamma_j (k for a full information set) */
    int d;                         /* minimum distance (or best weight if incomplete) */
    int complete;                  /* 1 if L >= U was reached (d exact) */
    int lower_bound;               /* L when the run stopped */
    int key_g, key_j;              /* canonical witness key: stage, matrix (0-based) */
    uint64_t key_rank;             /* ... and colex rank */
    int stop_g, stop_j;            /* last level processed */
    int nlevels;                   /* levels processed */
    uint64_t codewords;            /* combinations enumerated (sum of C(k, g) over levels) */
    double seconds_total;          /* wall time of md_compute */
    double seconds_device;         /* device time of the enumeration kernels */
    int gpu_launches;              /* kernels launched by the last md_compute */
    uint64_t h2d_bytes;            /* host-to-device bytes copied by the last md_compute */
    uint64_t d2h_bytes;            /* device-to-host bytes copied by the last md_compute */
    uint64_t skipped_work;         /* work units left out by the mid-level stop: once U <= L
                                      during a level, work ranked after the level's best
                                      codeword is skipped (it cannot change d or the witness);
                                      codewords above still counts those levels in full */
} md_info;

/* One processed level: stage g, matrix j, and the least weight of that level with its
   first colex rank.  weight = -1 when the level's least weight exceeds the bound U held
   before the level (the level cannot change U or the witness); the kernels only resolve
   weights up to that bound. */
typedef struct md_level {
    int g, j;
    int weight;
    int words;                     /* tensor-core levels: packed 32-bit words in each product at
                                      the level's start (a bound over fewer words than the row
                                      holds filters codewords, see md_options.filter); 0 for
                                      the popcount kernels */
    uint64_t first_rank;
    uint64_t count;                /* C(k, g) */
    double seconds;                /* device time of the level's enumeration kernel */
} md_level;

/* Fill *opt with defaults.  Always MD_OK (MD_EINVAL for NULL). */
int md_options_init(md_options *opt);

/* Build a handle for the code generated by the k x n matrix G (copied).
   Validates G (MD_EINVAL, MD_EUNSUPPORTED for n > MD_MAX_N), checks full row rank
   (MD_ERANK), finds the information sets and the Gamma_j on the host.  No device work. */
int md_create(const uint64_t *G, int n, int k, md_handle *out);
int md_create_ex(const uint64_t *G, int n, int k, const md_options *opt, md_handle *out);

/* Run Brouwer-Zimmermann on the GPU.  *d receives the minimum distance; witness
   (ceil(n/64) caller-owned words, may be NULL) receives the canonical codeword of weight
   d.  Device buffers are allocated on the first call and reused. */
int md_compute(md_handle h, int *d, uint64_t *witness);

/* Checkpoint and resume (the paper has no counterpart; a run's state is small: the bounds and
   one record per level).  md_checkpoint, after an md_compute that stopped early -- cancelled
   (MD_ECANCELED), over budget (MD_EBUDGET) or at md_options.max_stage -- or that finished,
   writes that run's state at its last completed level into buf: the bounds L and U (U taken
   from the completed levels' records, so a level the run did not complete leaves no trace),
   and each completed level's record.  *size receives the bytes needed; with cap below that,
   nothing is written and MD_EINVAL is returned (call with buf = NULL to ask for the size).
   MD_EINVAL also when the handle has run no md_compute.  md_resume loads such a buffer into a
   handle made from the same G, n, k, stop rule and column-order options (checked; MD_EINVAL
   otherwise); its next md_compute starts at the level after the checkpoint and returns the d,
   witness and level records of an uninterrupted run, whatever else the options say (a larger
   max_stage, another stream, ...).  The buffer is plain bytes, caller-owned, valid across
   processes on machines of the same byte order. */
int md_checkpoint(md_handle h, void *buf, size_t cap, size_t *size);
int md_resume(md_handle h, const void *buf, size_t size);

/* Details of the last md_compute (md_create alone fills n, k, m, ranks). */
int md_info_get(md_handle h, md_info *info);

/* Per-level records of the last md_compute: up to max entries, *count = levels written. */
int md_levels(md_handle h, md_level *levels, int max, int *count);

/* Gamma_j as built on the host (k x n, full rows in the original column order) and the
   column order of its reduction (information set first); either pointer may be NULL. */
int md_gamma(md_handle h, int j, uint64_t *gamma, int *order);

/* Least weight over the colex ranks [r0, r1) of the g-row combinations of Gamma_j,
   computed on the GPU with the enumeration kernel, and the first rank reaching it.
   With bound >= 0 only weights <= bound are resolved (*weight = -1 if none);
   bound < 0 resolves the exact least weight.  The whole level is r0 = 0, r1 = C(k, g). */
int md_scan_range(md_handle h, int g, int j, uint64_t r0, uint64_t r1, int bound,
                  int *weight, uint64_t *first_rank);

/* Least weight over one task of level (g, j), g >= 5, computed by the production
   enumeration kernel: all combinations c_1 < ... < c_g whose element c_{P+1} equals M and
   whose upper elements (c_{P+2}, ..., c_g), as a subset of {M+1, ..., k-1}, have colex
   index in [u0, u1).  P = 2 for g = 5 and P = 3 for g >= 6; the heads (c_1..c_P) range
   over every P-subset of {0..M-1}.  This is the analogue of the paper's prefix task
   (Section 3.1, Process_prefix) for the colex-ordered decomposition the kernels use.
   bound as in md_scan_range.  MD_EINVAL if M is outside [P, k - 1 - (g - P - 1)]. */
int md_scan_task(md_handle h, int g, int j, int M, uint64_t u0, uint64_t u1, int bound,
                 int *weight, uint64_t *first_rank);

/* The work decomposition of level (g, j) that md_compute uses under the handle's options
   (host-only, no device work).  *kind: 0 = per-lane colex rank ranges (small levels), 2 or
   3 = the head size P of the split enumeration, 4 = the tensor-core product (heads of q
   elements, q = md_options.tensor_head or the automatic choice, and for small c_{q+1} of q + 1
   elements).
   For kind 2/3 each entry i describes the tasks with c_{P+1} = M: tasks[i] = {M, number
   of upper parts, upper parts per lane, first work item}; *count receives the number of
   entries (at most max written); for kinds 0 and 4, *count = 0.  *work_items receives the
   number of work items of the level (kind 4: groups of up to 16 slices of 256 heads times
   runs of up to 128 T tails, T = 8, 4, 2, 1 for packed widths W <= 2, 4, 6, 8). */
typedef struct md_task_info {
    uint32_t M;
    uint32_t per_lane;
    uint64_t uppers;
    uint64_t first_item;
} md_task_info;

int md_level_plan(md_handle h, int g, int j, int *kind, md_task_info *tasks, int max, int *count,
                  uint64_t *work_items);

void md_destroy(md_handle h);

/* Measurement utility (no counterpart in the paper): the POPC throughput of the current GPU in
   popc lane-operations per SM per clock, from a kernel whose 16 independent popc/add chains
   per thread keep the POPC pipe the limit (one block of 1024 threads per SM, clock64 cycles,
   median over SMs).  The popcount kernels' roofline is this rate x SMs x the SM clock. */
int md_popc_rate(double *per_sm_per_clk);

/* Measurement utility (no counterpart in the paper): the dense fp8 (e4m3) throughput of the
   current GPU's tensor pipe in flops per SM per clock.  In one block per SM, two threads issue
   tcgen05.mma kind::f8f6f4 (M = 128, N = 256, K = 32, +-1 operands) back to back into two
   accumulators, as the tensor-core level kernel's two issuers do; clock64 cycles, median over
   SMs.  This rate x SMs x the SM clock is the fp8 peak at that clock, a denominator for the
   tensor-core kernel's roofline beside the cuBLAS-derived one.  Returns MD_ETIMEOUT if a chain
   did not complete within the kernel's time bound, MD_ECUDA on a failed CUDA call. */
int md_mma_rate(double *flops_per_sm_per_clk);

/* The range-checked build (compiled with -DMD_DEBUG_BOUNDS; paper_1911_08963_gb300.build
   builds it as libmd_debug.so): every index into the shared-memory rows and pair tables, the
   binomial tables, the work tables, and the tensor-core kernel's tables, tiles and head slices
   is checked; an index out of range records the check's site and is replaced by a safe one (no
   trap, no access out of bounds), and the call that launched the kernel returns MD_EINTERNAL.
   md_debug_bounds gives the last failing site (0 = none): MD_OK in the range-checked build,
   MD_EUNSUPPORTED (site 0) in the normal one. */
int md_debug_bounds(unsigned *site);

/* Static text for a status code. */
const char *md_strerror(int code);

/* ---- rank-range scan without device allocation --------------------------------------
 * md_scan_range_noalloc computes what md_scan_range computes -- the least weight over the
 * colex ranks [r0, r1) of the g-row combinations of a matrix, and the first rank reaching
 * it -- but makes no device allocation and no heap allocation of its own.  It is meant for
 * callers that cannot allocate: real-time loops that forbid allocation after start-up (a
 * cudaMalloc may wait for the whole device and take an unbounded time), and programs whose
 * device memory belongs to another allocator (a framework's caching pool that already holds
 * the free memory, or a fixed budget that an outside allocation would break).
 * The paper has no counterpart to this entry point.
 *
 *   rows         device pointer, 16-byte aligned, owned by the caller: k packed rows of
 *                `words` 32-bit words each (bit t of word w = packed column 32w + t), stored
 *                with a row stride of 1, 2, 4, 4, 8, 8, 8, 8 words for words = 1..8; unused
 *                words and bits must be zero.  Read only.
 *   weight_base  added to every popcount (g for the non-pivot columns of a full-rank
 *                Gamma_j, 0 when every column is packed).
 *   bound        as in md_scan_range (< 0: exact least weight).
 *   stream       cudaStream_t or NULL; the call synchronises it before returning.
 *   weight, first_rank  host outputs, as md_scan_range.
 *
 * Its device scratch is one fixed array of MD_NOALLOC_SCRATCH_BYTES inside the library;
 * every GPU that loads the library holds it until the process exits.  The first call on a
 * device looks the array up and fills its binomial table (make that first call before any
 * stream capture).  Every call resets the scratch before use, and all calls share it: calls
 * that overlap on the GPU (from several threads or streams) race and give wrong results.
 * k > MD_NOALLOC_MAX_K, or more than 2^55 combinations, returns MD_EUNSUPPORTED; a bad
 * pointer alignment or argument returns MD_EINVAL; a failed CUDA call (including the device
 * queries of the first call) returns MD_ECUDA. */
#define MD_NOALLOC_MAX_K 128
#define MD_NOALLOC_SCRATCH_BYTES 139264
int md_scan_range_noalloc(const uint32_t *rows, int k, int words, int weight_base, int g, uint64_t r0,
                          uint64_t r1, int bound, void *stream, int *weight, uint64_t *first_rank);

/* ---- batched codes ------------------------------------------------------------------
 * md_batch runs many codes of uneven n, k to completion in one schedule: each code keeps
 * its own U, L, stage and level records on the device (its own Alg. 1 state machine);
 * round r enumerates level r of every code still running, with the work items of all
 * codes pooled behind shared atomic tickets, so idle warps take work from any code.  The
 * rounds are captured in a CUDA graph (md_options.use_graph) and launched at once.
 * codes[i].G follows the packing rule above.  d[i] and status[i] are written per code;
 * witness (may be NULL) receives code i's witness at word offset sum_{t<i} ceil(n_t/64).
 * Results are identical to md_compute on each code.  Per-code status: MD_OK (d exact),
 * MD_EINVAL / MD_ERANK / MD_EUNSUPPORTED for that code's G, MD_EBUDGET if its estimated
 * work exceeds opt->work_budget (not run; d = -1) or if opt->max_stage stopped it early
 * (d = the best weight found).  Returns MD_OK if the batch ran, or an error for the whole
 * call (MD_EINVAL for NULL arguments, MD_ECUDA, MD_ENOMEM). */
typedef struct md_code {
    const uint64_t *G;
    int n, k;
} md_code;

int md_batch(const md_code *codes, int count, const md_options *opt,
             int *d, uint64_t *witness, int *status);

/* ---- autotuning of md_batch ----------------------------------------------------------
 * md_batch_tune picks md_batch's schedule options for batches shaped like codes[0..count) on
 * the current GPU: the combinations per work item (chunk_log2 in {16, 18, 20}), the blocks per
 * SM of the shared rounds ({occupancy, 2, 4}), and the single-code threshold (batch_heavy in
 * {2^30, 2^32, ..., 2^38}).  It times md_batch on deterministic samples of the batch (every
 * i-th code): up to 384 codes of estimated work below 2^34 for the first two, then those
 * together with up to 24 codes between 2^30 and 2^38 for the threshold, and writes into *tuned
 * a copy of *base (defaults if NULL) with the fastest values.  With cache_path, the choice is
 * stored in that JSON file under the key md_batch_tune_key(...) + " | budget " + the work
 * budget + " | " + the GPU's name, and a later call with the same key reads it back without
 * timing anything.  Codes over base->work_budget
 * are left out of the samples.  Returns MD_OK, MD_EINVAL (bad arguments, unwritable cache),
 * MD_ECUDA (no GPU) or the error of a timing run.  The paper's own tuning is the choice of
 * prefix size and threads per process (Section 4); these knobs are this library's analogue.
 */
int md_batch_tune(const md_code *codes, int count, const md_options *base, const char *cache_path,
                  md_options *tuned);

/* The batch-shape part of the tuning key: "n<lo>-<hi> k<lo>-<hi> c2^<e>" with n rounded out to
   multiples of 16, k to multiples of 8, and count to the next power of two.  Host only. */
int md_batch_tune_key(const md_code *codes, int count, char *key, size_t len);

/* ---- continuous-batching server -------------------------------------------------------
 * A server owns a device region for resident codes and a host thread that admits
 * submitted codes into free slots while others run, by memory and by estimated work.
 * Results are identical to md_compute on the same code. */
typedef struct md_server md_server;

typedef struct md_server_opts {
    int slots;                  /* codes resident on the device at once (0 = default 64) */
    uint64_t work_budget;       /* per-request estimated combinations; larger requests are
                                   rejected with MD_EBUDGET (0 = unlimited) */
    size_t device_bytes;        /* device memory for resident codes (0 = default 256 MiB) */
    void *stream;               /* cudaStream_t or NULL */
    int stop_rule;              /* as md_options.stop_rule */
    uint64_t heavy;             /* requests whose estimated work reaches this run one at a time
                                   as single-code computations with the tensor-core levels, on a
                                   second worker thread and a stream of the server's own (their
                                   device memory is their own, outside device_bytes), while
                                   lighter requests share the ticks of the resident slots;
                                   0 = default 2^30, UINT64_MAX = every request in the slots */
} md_server_opts;

int md_server_create(const md_server_opts *opts, md_server **out);
/* Copies G; returns a ticket.  MD_EINVAL / MD_ERANK / MD_EUNSUPPORTED / MD_EBUDGET are
   reported here, before the request is queued. */
int md_server_submit(md_server *s, const uint64_t *G, int n, int k, uint64_t *ticket);
/* MD_OK with *d, witness (ceil(n/64) words, may be NULL) and *status filled when done;
   MD_EBUSY while pending; MD_EINVAL for an unknown ticket.  A finished ticket is
   released by the poll that returns it.  After a failed CUDA call the server takes no more
   work: a request still waiting then completes with *status = that error (MD_ECUDA) and
   *d = -1, so no caller polls MD_EBUSY forever. */
int md_server_poll(md_server *s, uint64_t ticket, int *d, uint64_t *witness, int *status);
void md_server_destroy(md_server *s);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
