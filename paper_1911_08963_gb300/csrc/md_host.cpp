// md_host.cpp -- host-side preparation of a code (Section 2.1 of the paper):
// validation, rank, disjoint information sets, the systematic matrices Gamma_j, the
// packing of each Gamma_j for the device, and the per-level work plans.
//
// Each information set comes from one Gauss-Jordan pass over the still-unused columns: the
// pass that finds k pivots leaves Gamma_j = G[:, S_j]^-1 G in its rows, and for the leftover
// columns the pass continues into the other columns to give the reduced form
// [[I, A], [0, B]].
#include <algorithm>
#include <utility>
#include <cmath>
#include <cstring>

#include "md_internal.h"

namespace mdl {

namespace {

// Pascal's triangle with saturating addition, rows 0..256.
struct BinomTable {
    std::vector<uint64_t> t;  // 257 x 257
    BinomTable() : t(257 * 257, 0) {
        for (int a = 0; a <= 256; a++) {
            t[a * 257] = 1;
            for (int b = 1; b <= a; b++) {
                uint64_t x = t[(a - 1) * 257 + b - 1], y = t[(a - 1) * 257 + b];
                t[a * 257 + b] = (x > UINT64_MAX - y) ? UINT64_MAX : x + y;
            }
        }
    }
};

const BinomTable &table() {
    static BinomTable tb;
    return tb;
}

}  // namespace

uint64_t binom(int a, int b) {
    if (a < 0 || b < 0 || b > a) return 0;
    if (a > 256) return UINT64_MAX;
    return table().t[a * 257 + b];
}

// Colex unranking by binary search on C(x, i) (positions i = g..1).
void colex_unrank(uint64_t r, int g, int k, int *c) {
    int hi = k - 1;
    for (int i = g; i >= 1; i--) {
        int lo = i - 1, h = hi;          // largest x in [lo, h] with C(x, i) <= r
        while (lo < h) {
            int mid = (lo + h + 1) / 2;
            if (binom(mid, i) <= r) lo = mid; else h = mid - 1;
        }
        c[i - 1] = lo;
        r -= binom(lo, i);
        hi = lo - 1;
    }
}

int popcount_row(const uint64_t *row, int nw) {
    int s = 0;
    for (int i = 0; i < nw; i++) s += __builtin_popcountll(row[i]);
    return s;
}

int lower_bound_after(const Code &c, int g) {
    int L = 0;
    for (const Gamma &gm : c.gam) L += std::max(0, g + 1 - (c.k - gm.rank));
    return L;
}

namespace {

void pack_gamma(Gamma &gm, int n, int k, int nw) {
    std::vector<char> in_set(n, 0);
    if (gm.rank == k)
        for (int t = 0; t < k; t++) in_set[gm.order[t]] = 1;
    gm.packed_cols.clear();
    for (int c = 0; c < n; c++)
        if (!in_set[c]) gm.packed_cols.push_back(c);
    gm.weight_base_is_g = (gm.rank == k) ? 1 : 0;
    int bits = (int)gm.packed_cols.size();
    gm.W = std::max(1, (bits + 31) / 32);
    gm.WP = gm.W == 1 ? 1 : gm.W == 2 ? 2 : gm.W <= 4 ? 4 : 8;
    gm.packed.assign((size_t)k * gm.WP, 0);
    std::vector<int> pos(n, -1);                    // column -> packed bit
    for (int b = 0; b < bits; b++) pos[gm.packed_cols[b]] = b;
    for (int i = 0; i < k; i++)
        for (int w = 0; w < nw; w++) {
            uint64_t x = gm.rows[(size_t)i * nw + w];
            while (x) {
                const int b = pos[64 * w + __builtin_ctzll(x)];
                x &= x - 1;
                if (b >= 0) gm.packed[(size_t)i * gm.WP + b / 32] |= 1u << (b % 32);
            }
        }
}

}  // namespace

namespace {

// Gauss-Jordan over the columns in `order`, stopping once k pivots are found.  Returns
// the pivot columns in the order they were found; `rows` receives the reduced matrix with
// row i holding the i-th pivot (the reduced row echelon form for this column order).
std::vector<int> reduce_in_order(const std::vector<uint64_t> &G, int nw, int k, const std::vector<int> &order,
                                 std::vector<uint64_t> *rows) {
    std::vector<uint64_t> A(G);
    std::vector<int> piv_row;                       // row index of each pivot found so far
    std::vector<char> used(k, 0);
    std::vector<int> cols;
    for (int col : order) {
        if ((int)cols.size() == k) break;
        const int w = col / 64;
        const uint64_t bit = 1ull << (col % 64);
        int p = -1;
        for (int i = 0; i < k; i++)
            if (!used[i] && (A[(size_t)i * nw + w] & bit)) { p = i; break; }
        if (p < 0) continue;
        used[p] = 1;
        const uint64_t *pr = &A[(size_t)p * nw];
        for (int i = 0; i < k; i++)
            if (i != p && (A[(size_t)i * nw + w] & bit)) {
                uint64_t *ri = &A[(size_t)i * nw];
                for (int t = 0; t < nw; t++) ri[t] ^= pr[t];
            }
        piv_row.push_back(p);
        cols.push_back(col);
    }
    if (rows) {
        rows->assign((size_t)k * nw, 0);
        for (size_t i = 0; i < piv_row.size(); i++)
            std::memcpy(rows->data() + i * nw, &A[(size_t)piv_row[i] * nw], nw * 8);
    }
    return cols;
}

}  // namespace

int build_code(const uint64_t *G, int n, int k, Code *out) {
    if (!G || !out || n < 1 || k < 1 || k > n) return MD_EINVAL;
    if (n > kMaxN) return MD_EUNSUPPORTED;
    const int nw = (n + 63) / 64;
    for (int i = 0; i < k; i++) {
        uint64_t last = G[(size_t)i * nw + nw - 1];
        if (n % 64 && (last >> (n % 64))) return MD_EINVAL;   // padding bits must be zero
    }
    Code c;
    c.n = n; c.k = k; c.nw64 = nw;
    c.G.assign(G, G + (size_t)k * nw);

    // greedy disjoint information sets over the unused columns, ascending; the first pass
    // over all columns also decides the rank
    std::vector<char> used(n, 0);
    for (;;) {
        std::vector<int> remaining;
        for (int col = 0; col < n; col++)
            if (!used[col]) remaining.push_back(col);
        if (remaining.empty()) break;
        Gamma gm;
        std::vector<int> kept = reduce_in_order(c.G, nw, k, remaining, &gm.rows);
        if (c.gam.empty() && (int)kept.size() < k) return MD_ERANK;
        if ((int)kept.size() == k) {
            // the pass stopped at k pivots, all inside S_j, each cleared from every other
            // row: the rows are G[:, S_j]^-1 G with row i holding the i-th column of S_j
            gm.rank = k;
            std::vector<char> in(n, 0);
            for (int col : kept) { gm.order.push_back(col); in[col] = 1; used[col] = 1; }
            for (int col = 0; col < n; col++)
                if (!in[col]) gm.order.push_back(col);
            c.gam.push_back(std::move(gm));
            continue;
        }
        if (!kept.empty()) {
            gm.rank = (int)kept.size();
            std::vector<char> in(n, 0);
            for (int col : remaining) { gm.order.push_back(col); in[col] = 1; }
            for (int col = 0; col < n; col++)
                if (!in[col]) gm.order.push_back(col);
            reduce_in_order(c.G, nw, k, gm.order, &gm.rows);
            c.gam.push_back(std::move(gm));
        }
        break;
    }
    if ((int)c.gam.size() > MD_MAX_GAMMA) return MD_EUNSUPPORTED;
    // the default filter thresholds depend only on the number of packed columns
    thread_local unsigned long long fmax_cache[kMaxN + 1];
    thread_local bool fmax_known[kMaxN + 1] = {false};
    for (Gamma &gm : c.gam) {
        pack_gamma(gm, n, k, nw);
        const int bits = (int)gm.packed_cols.size();
        if (!fmax_known[bits]) {
            fmax_cache[bits] = filter_thresholds(gm, 1);
            fmax_known[bits] = true;
        }
        gm.fmax8 = fmax_cache[bits];
    }
    *out = std::move(c);
    return MD_OK;
}

namespace {

struct SplitMix64 {
    uint64_t state;
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// The columns of G (k x n, nw words per row) taken in `order`.
std::vector<uint64_t> permute_columns(const uint64_t *G, int n, int k, const std::vector<int> &order) {
    const int nw = (n + 63) / 64;
    std::vector<uint64_t> out((size_t)k * nw, 0);
    for (int i = 0; i < k; i++)
        for (int p = 0; p < n; p++) {
            const int c = order[p];
            if ((G[(size_t)i * nw + c / 64] >> (c % 64)) & 1u) out[(size_t)i * nw + p / 64] |= 1ull << (p % 64);
        }
    return out;
}

// (number of full-rank information sets, rank of the last set) for the greedy sets taken
// in the given column order.
std::pair<int, int> set_profile(const std::vector<uint64_t> &G, int n, int k) {
    const int nw = (n + 63) / 64;
    std::vector<char> used(n, 0);
    int full = 0, last = 0;
    for (;;) {
        std::vector<int> remaining;
        for (int col = 0; col < n; col++)
            if (!used[col]) remaining.push_back(col);
        if (remaining.empty()) break;
        std::vector<int> kept = reduce_in_order(G, nw, k, remaining, nullptr);
        if ((int)kept.size() == k) {
            full++;
            for (int col : kept) used[col] = 1;
            continue;
        }
        last = (int)kept.size();
        break;
    }
    return {full, last};
}

}  // namespace

int build_code_permuted(const uint64_t *G, int n, int k, int trials, uint64_t seed, Code *out) {
    if (trials <= 1) return build_code(G, n, k, out);
    if (!G || !out || n < 1 || k < 1 || k > n) return MD_EINVAL;
    if (n > kMaxN) return MD_EUNSUPPORTED;
    std::vector<int> order(n), best;
    for (int i = 0; i < n; i++) order[i] = i;
    SplitMix64 rng{seed};
    std::pair<int, int> best_score{-1, -1};
    for (int t = 0; t < trials; t++) {
        if (t > 0)
            for (int i = n - 1; i >= 1; i--) std::swap(order[i], order[(int)(rng.next() % (uint64_t)(i + 1))]);
        const std::pair<int, int> sc = set_profile(permute_columns(G, n, k, order), n, k);
        if (sc > best_score) { best_score = sc; best = order; }
    }
    std::vector<uint64_t> Gp = permute_columns(G, n, k, best);
    int rc = build_code(Gp.data(), n, k, out);
    if (rc != MD_OK) return rc;
    bool identity = true;
    for (int i = 0; i < n; i++) identity &= best[i] == i;
    if (!identity) out->perm = best;
    return MD_OK;
}

void to_caller_order(const Code &c, const uint64_t *row, uint64_t *out) {
    if (c.perm.empty()) {
        std::memcpy(out, row, (size_t)c.nw64 * 8);
        return;
    }
    std::vector<uint64_t> tmp((size_t)c.nw64, 0);
    for (int p = 0; p < c.n; p++)
        if ((row[p / 64] >> (p % 64)) & 1u) tmp[c.perm[p] / 64] |= 1ull << (c.perm[p] % 64);
    std::memcpy(out, tmp.data(), (size_t)c.nw64 * 8);
}

double estimate_work(const Code &c, int *d_est, int *g_stop) {
    // expected number of codewords of weight <= w in a random [n, k] code
    double acc = 0.0;
    int d = c.n - c.k + 1;
    for (int w = 1; w <= c.n; w++) {
        acc += std::exp(std::lgamma(c.n + 1.0) - std::lgamma(w + 1.0) - std::lgamma(c.n - w + 1.0) -
                        (c.n - c.k) * std::log(2.0));
        if (acc >= 0.5) { d = w; break; }
    }
    d = std::min(d, c.n - c.k + 1);
    int gs = c.k;
    for (int g = 1; g <= c.k; g++)
        if (lower_bound_after(c, g) >= d) { gs = g; break; }
    double work = 0.0;
    for (int g = 1; g <= gs; g++) work += (double)c.gam.size() * std::exp(std::lgamma(c.k + 1.0) - std::lgamma(g + 1.0) - std::lgamma(c.k - g + 1.0));
    if (d_est) *d_est = d;
    if (g_stop) *g_stop = gs;
    return work;
}

int filter_threshold(const Gamma &gm, int f, double pmax) {
    const int bits = (int)gm.packed_cols.size();
    // per bit position b of a 32-bit word: how many of the first f words have a column there
    double dist[33] = {1.0};
    for (int b = 0; b < 32; b++) {
        int nb = 0;
        for (int w = 0; w < f && w < gm.W; w++)
            if (32 * w + b < bits) nb++;
        double p = nb ? 1.0 - std::ldexp(1.0, -nb) : 0.0;
        for (int t = b + 1; t >= 1; t--) dist[t] = dist[t] * (1 - p) + dist[t - 1] * p;
        dist[0] *= (1 - p);
    }
    double cdf = 0.0;
    int best = -1;
    for (int t = 0; t <= 32; t++) {
        cdf += dist[t];
        if (cdf < pmax) best = t; else break;
    }
    return best;
}

// mode 0: never filter; 1: every word count whose threshold allows it; 2: also always with
// all words; 3: always with one word (a test setting that sends many codewords down the
// exact path).
unsigned long long filter_thresholds(const Gamma &gm, int mode) {
    unsigned long long out = 0;
    if (mode == 0) return 0;
    for (int f = 1; f <= gm.W && f <= 8; f++) {
        int t = filter_threshold(gm, f, 1e-5);
        if (mode == 2 && f == gm.W) t = 254;
        if (mode == 3) t = (f == 1) ? 254 : -1;
        const unsigned long long byte = (unsigned long long)(t < 0 ? 0 : std::min(255, t + 1));
        out |= byte << (8 * (f - 1));
    }
    return out;
}

// Word counts of the tensor-core product.  A product over the first f packed words gives the
// weight of those words only, a lower bound of the weight; byte f-1 holds 1 + the largest
// packed-weight threshold at which that bound rejects all but a fraction 1e-7 of random
// codewords (0 = never), and the last word count, the exact product, is always usable (255).
// mode 0: always every word; 3: always one word (a test setting: most products then send
// rows to the exact check); otherwise adaptive.
#ifndef MD_TC_WORD_PMAX
#define MD_TC_WORD_PMAX 1e-7
#endif
unsigned long long tc_word_thresholds(const Gamma &gm, int mode) {
    unsigned long long out = 0;
    for (int f = 1; f <= gm.W && f <= 8; f++) {
        int t = f == gm.W ? 254 : (mode == 0 ? -1 : filter_threshold(gm, f, MD_TC_WORD_PMAX));
        if (mode == 3) t = f == 1 ? 254 : -1;
        const unsigned long long byte = (unsigned long long)(t < 0 ? 0 : std::min(255, t + 1));
        out |= byte << (8 * (f - 1));
    }
    return out;
}

LevelPlan plan_level(const Code &c, int g, int j, const PlanOptions &o) {
    LevelPlan p;
    const Gamma &gm = c.gam[j];
    const int k = c.k;
    p.g = g; p.j = j;
    p.count = binom(k, g);
    p.base = gm.weight_base_is_g ? g : 0;
    if (o.stop_rule == 1) {
        // matrices up to j have completed stage g, the later ones stage g - 1
        int L = 0;
        for (int i = 0; i < (int)c.gam.size(); i++)
            L += std::max(0, (i <= j ? g : g - 1) + 1 - (k - c.gam[i].rank));
        p.L_after = L;
        p.L_first = 1;
    } else {
        p.L_after = j == (int)c.gam.size() - 1 ? lower_bound_after(c, g) : -1;
    }
    p.fmax8 = o.filter == 1 ? gm.fmax8 : filter_thresholds(gm, o.filter);
    if (o.tensor && g <= kMaxG) {
        // tensor-core level: head (c_1..c_q) x tail products, see md_tc.cu
        const int q = o.tensor_head ? o.tensor_head : tc_auto_head(k, gm.W);
        const int v = g - q - 1;
        bool use = false;
        if (q >= 2 && q <= 5 && q < k && v >= 0 && v <= tc_max_upper())
            use = o.tensor == 2 || (v >= 1 && p.count >= (1ull << 28));
        if (use) {
            p.kind = KIND_TC;
            p.tc_q = q;
            p.v = v;
            p.tc_smin = g >= q + 2 ? tc_split_point(k, q) : q;
            p.nchunks = tc_level_items(k, g, q, p.tc_smin, gm.W);
            p.tc_words8 = tc_word_thresholds(gm, o.filter);
            return p;
        }
    }
    const uint64_t target_full = 1ull << std::max(8, std::min(30, o.chunk_log2));
    // keep at least ~64 work items per SM-sized slice of the level
    const uint64_t target = std::max<uint64_t>(1ull << 10, std::min<uint64_t>(target_full, p.count / (152ull * 64)));
    if (g <= 4 || p.count < (1ull << 18) || g > 64) {
        p.kind = KIND_SIMPLE;
        p.per_chunk = std::max<uint64_t>(1, target / 32);
        p.nchunks = (p.count + 32 * p.per_chunk - 1) / (32 * p.per_chunk);
        return p;
    }
    const int P = (g == 5) ? 2 : 3;
    p.kind = P == 2 ? KIND_SPLIT2 : KIND_SPLIT3;
    p.v = g - P - 1;
    uint64_t chunks = 0;
    for (int M = P; M <= k - 1 - p.v; M++) {
        MEntry e{};
        e.M = (uint32_t)M;
        e.uppers = binom(k - 1 - M, p.v);
        const uint64_t cost = binom(M, P) + 16;           // codewords + upper-part bookkeeping
        uint64_t per_lane = (target + 32 * cost - 1) / (32 * cost);
        per_lane = std::max<uint64_t>(1, std::min<uint64_t>(per_lane, 1u << 30));
        const uint64_t need = (e.uppers + 31) / 32;       // never more than the lanes can use
        per_lane = std::min(per_lane, std::max<uint64_t>(1, need));
        // lanes walk kUppersPerLane upper parts at once: whole groups avoid repeated work
        per_lane = (per_lane + kUppersPerLane - 1) / kUppersPerLane * kUppersPerLane;
        e.per_lane = (uint32_t)per_lane;
        e.chunk_begin = chunks;
        chunks += (e.uppers + 32 * per_lane - 1) / (32 * per_lane);
        p.mtab.push_back(e);
    }
    p.nchunks = chunks;
    return p;
}

}  // namespace mdl
