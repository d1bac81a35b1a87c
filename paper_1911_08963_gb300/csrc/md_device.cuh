// md_device.cuh -- device building blocks of the enumeration, shared by the single-code
// kernels (md_kernels.cu) and the multi-code engine (md_engine.cu).
//
// Every codeword is a sum of g rows of a systematic matrix Gamma_j (Section 2.1); its
// weight tightens U (Alg. 1).  A combination c_1 < ... < c_g with colex rank
// sum_i C(c_i, i) (the paper's "left-lexicographical" order, Section 3.1) is split into
// head (c_1..c_P), pivot M = c_{P+1} and an upper part (c_{P+2}..c_g): for a fixed M and
// upper part the heads occupy a contiguous run of C(M, P) ranks starting at
// C(M, P+1) + sum_{i>P+1} C(c_i, i).  Lanes hold distinct upper parts; the warp walks the
// heads in lockstep against pre-added pair sums (the right combinations of the paper's
// saved-additions composition, Section 2.2.1).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "md_internal.h"

namespace mdl {
namespace dev {

// ---- range checks of the debug build (-DMD_DEBUG_BOUNDS) ----
// MD_BOUND(idx, lim, site): in the debug build an index at or past its array's limit records
// `site` in this file's status word (the first failure wins) and is replaced by 0, so the
// kernel goes on without touching memory out of bounds; the library then reports
// MD_EINTERNAL and md_debug_bounds returns the site.  In the normal build it is the index.
#ifdef MD_DEBUG_BOUNDS
static __device__ unsigned int md_bounds_word;
static __device__ __noinline__ void md_bounds_fail(unsigned site) { atomicCAS(&md_bounds_word, 0u, site); }
template <class I>
__device__ __forceinline__ I md_bound(I idx, unsigned long long lim, unsigned site) {
    if ((unsigned long long)idx < lim) return idx;
    md_bounds_fail(site);
    return (I)0;
}
#define MD_BOUND(idx, lim, site) ::mdl::dev::md_bound((idx), (unsigned long long)(lim), (site))
// The host side of this file's status word: read it into *site and optionally clear it.
#define MD_BOUNDS_ACCESSOR(name)                                                                    \
    int name(unsigned *site, int reset) {                                                           \
        if (cudaMemcpyFromSymbol(site, ::mdl::dev::md_bounds_word, sizeof(unsigned)) != cudaSuccess) \
            return -1;                                                                              \
        const unsigned zero = 0;                                                                    \
        if (reset && cudaMemcpyToSymbol(::mdl::dev::md_bounds_word, &zero, sizeof(unsigned)) != cudaSuccess) \
            return -1;                                                                              \
        return 0;                                                                                   \
    }
#else
#define MD_BOUND(idx, lim, site) (idx)
#define MD_BOUNDS_ACCESSOR(name)                \
    int name(unsigned *site, int) {             \
        *site = 0;                              \
        return 0;                               \
    }
#endif
// Check sites (the value md_debug_bounds reports).
enum : unsigned {
    kSiteSmemRow = 1, kSiteGlobRow = 2, kSiteBinom = 3, kSiteMtab = 4, kSiteTcTable = 5, kSiteTcTile = 6,
    kSiteTcSlice = 7, kSiteTcBinom = 8, kSiteTcTail = 9, kSiteTcHead = 10, kSiteNoallocBinom = 11
};

constexpr unsigned kFull = 0xffffffffu;
constexpr int kInf = 0x3fffffff;
constexpr int kNU = kUppersPerLane;           // upper parts a lane walks against each loaded head

__device__ __forceinline__ unsigned long long binom_d(const unsigned long long *tb, int stride, int a, int b) {
    return (b < 0 || b > a) ? 0ull : __ldg(tb + MD_BOUND((size_t)a * stride + b, (size_t)stride * stride, kSiteBinom));
}

// Row sources: packed rows of WP words, W of them used (the rest are zero padding).
template <int W, int WP>
struct SmemSrc {           // rows in shared memory, read with explicit ld.shared
    uint32_t base;         // shared-window address of row 0
    uint32_t n = ~0u;      // rows held (checked in the debug build)
    __device__ __forceinline__ void load(int idx, uint32_t (&r)[W]) const {
        const uint32_t a = base + (uint32_t)MD_BOUND(idx, n, kSiteSmemRow) * (WP * 4);
        if constexpr (WP == 1) {
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r[0]) : "r"(a));
        } else if constexpr (WP == 2) {
            uint32_t x, y;
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(a));
            r[0] = x;
            if constexpr (W > 1) r[1] = y;
        } else {
            uint32_t x, y, z, w;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a));
            r[0] = x;
            if constexpr (W > 1) r[1] = y;
            if constexpr (W > 2) r[2] = z;
            if constexpr (W > 3) r[3] = w;
            if constexpr (WP == 8) {
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(x), "=r"(y), "=r"(z), "=r"(w) : "r"(a + 16));
                if constexpr (W > 4) r[4] = x;
                if constexpr (W > 5) r[5] = y;
                if constexpr (W > 6) r[6] = z;
                if constexpr (W > 7) r[7] = w;
            }
        }
    }
};

template <int W, int WP>
struct GlobSrc {           // rows in global memory (read-only path)
    const uint32_t *p;
    uint32_t n = ~0u;      // rows held (checked in the debug build)
    __device__ __forceinline__ void load(int idx, uint32_t (&r)[W]) const {
        const uint32_t *q = p + (size_t)MD_BOUND(idx, n, kSiteGlobRow) * WP;
        if constexpr (WP == 1) {
            r[0] = __ldg(q);
        } else if constexpr (WP == 2) {
            uint2 t = __ldg(reinterpret_cast<const uint2 *>(q));
            r[0] = t.x;
            if constexpr (W > 1) r[1] = t.y;
        } else {
            uint4 t = __ldg(reinterpret_cast<const uint4 *>(q));
            r[0] = t.x;
            if constexpr (W > 1) r[1] = t.y;
            if constexpr (W > 2) r[2] = t.z;
            if constexpr (W > 3) r[3] = t.w;
            if constexpr (WP == 8) {
                uint4 u = __ldg(reinterpret_cast<const uint4 *>(q + 4));
                if constexpr (W > 4) r[4] = u.x;
                if constexpr (W > 5) r[5] = u.y;
                if constexpr (W > 6) r[6] = u.z;
                if constexpr (W > 7) r[7] = u.w;
            }
        }
    }
};

template <int W>
__device__ __forceinline__ int weight_xor(const uint32_t (&T)[W], const uint32_t (&h)[W]) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < W; w++) s += __popc(T[w] ^ h[w]);
    return s;
}

// Lower bound of the weight: popc of the OR of the first F words (one POPC for F words;
// F = 0 means the exact weight).  Each bit position is counted at most once, so the bound
// never exceeds the weight.
template <int W, int F>
__device__ __forceinline__ int weight_lb(const uint32_t (&T)[W], const uint32_t (&h)[W]) {
    if constexpr (F == 0) {
        return weight_xor<W>(T, h);
    } else {
        uint32_t o = T[0] ^ h[0];
#pragma unroll
        for (int w = 1; w < F; w++) o |= T[w] ^ h[w];
        return __popc(o);
    }
}

__device__ __forceinline__ int min3(int a, int b, int c) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    return __vimin3_s32(a, b, c);
#else
    return min(min(a, b), c);
#endif
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(kFull, x, o);
        x = y < x ? y : x;
    }
    return x;
}

// A lane's running best inside one work item, as the 64-bit key (weight << 55 | colex rank):
// the smaller key is the better codeword, and among equal weights the earlier one.
struct LaneBest {
    unsigned long long key = kNoKey;
    __device__ __forceinline__ int w() const { return key == kNoKey ? kInf : (int)(key >> kRankBits); }
    __device__ __forceinline__ void offer(int weight, unsigned long long rank) {
        const unsigned long long k = ((unsigned long long)weight << kRankBits) | rank;
        if (k < key) key = k;
    }
};

// Walk pair-table entries [0, n2) against the NU lane sums T[q].  thr is the largest
// packed weight the lane still has to resolve, min(U, best) - base (-1: nothing); the
// exact weights of codewords that pass are offered to the lane's best with their ranks
// rbase[q] + i.  One loaded entry serves all NU sums (the unrolling of the paper's
// saved-additions engine, Section 2.2.1: several left combinations share each right one).
template <int W, int WP, int NU, int F, class H2Src>
__device__ __forceinline__ void walk_pairs(const H2Src &h2, const uint32_t (&T)[NU][W], int n2, int &thr, int base,
                                           LaneBest &best, const unsigned long long (&rbase)[NU]) {
    int i = 0;
    for (; i + 8 <= n2; i += 8) {
        int lbmin = kInf;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            uint32_t h[W];
            h2.load(i + u, h);
            if constexpr (NU == 2) {
                lbmin = min3(lbmin, weight_lb<W, F>(T[0], h), weight_lb<W, F>(T[1], h));
            } else {
#pragma unroll
                for (int q = 0; q < NU; q++) lbmin = min(lbmin, weight_lb<W, F>(T[q], h));
            }
        }
        if (__any_sync(kFull, lbmin <= thr)) {
            if (lbmin <= thr) {
#pragma unroll 1
                for (int u = 0; u < 8; u++) {
                    uint32_t h[W];
                    h2.load(i + u, h);
#pragma unroll
                    for (int q = 0; q < NU; q++) {
                        const int w = weight_xor<W>(T[q], h);
                        if (w <= thr) best.offer(w + base, rbase[q] + (unsigned long long)(i + u));
                    }
                    thr = min(thr, best.w() - base);
                }
            }
        }
    }
#pragma unroll 1
    for (; i < n2; i++) {
        uint32_t h[W];
        h2.load(i, h);
#pragma unroll
        for (int q = 0; q < NU; q++) {
            const int w = weight_xor<W>(T[q], h);
            if (w <= thr) best.offer(w + base, rbase[q] + (unsigned long long)i);
        }
        thr = min(thr, best.w() - base);
    }
}

// Run walk_pairs with F filter words (runtime value, 0..W).
template <int W, int WP, int NU, class H2Src>
__device__ __forceinline__ void walk_dispatch(int F, const H2Src &h2, const uint32_t (&T)[NU][W], int n2, int &thr,
                                              int base, LaneBest &best, const unsigned long long (&rbase)[NU]) {
    switch (F) {
        case 1: walk_pairs<W, WP, NU, 1>(h2, T, n2, thr, base, best, rbase); break;
        case 2: if constexpr (W >= 2) walk_pairs<W, WP, NU, 2>(h2, T, n2, thr, base, best, rbase); break;
        case 3: if constexpr (W >= 3) walk_pairs<W, WP, NU, 3>(h2, T, n2, thr, base, best, rbase); break;
        case 4: if constexpr (W >= 4) walk_pairs<W, WP, NU, 4>(h2, T, n2, thr, base, best, rbase); break;
        case 5: if constexpr (W >= 5) walk_pairs<W, WP, NU, 5>(h2, T, n2, thr, base, best, rbase); break;
        case 6: if constexpr (W >= 6) walk_pairs<W, WP, NU, 6>(h2, T, n2, thr, base, best, rbase); break;
        case 7: if constexpr (W >= 7) walk_pairs<W, WP, NU, 7>(h2, T, n2, thr, base, best, rbase); break;
        case 8: if constexpr (W >= 8) walk_pairs<W, WP, NU, 8>(h2, T, n2, thr, base, best, rbase); break;
        default: walk_pairs<W, WP, NU, 0>(h2, T, n2, thr, base, best, rbase); break;
    }
}

// Level-constant parameters of a chunk.
struct ChunkCtx {
    int k, g, v, base;
    unsigned long long fmax8;      // byte f-1: 1 + largest threshold for an f-word filter
    const unsigned long long *tb;
    int stride;
    // mid-level stop (may be null): the code's lower bound of completed stages and this
    // level's key; `skipped` counts upper parts (or rank runs) left out
    const int *L;
    const unsigned long long *key;
    unsigned long long *skipped;
};

// Once U <= L the minimum distance is U: no codeword lighter than U exists.  This level then
// holds the first codeword of weight U (it lowered U to L or below), and work whose ranks all
// exceed the level's best rank cannot change the result.  Returns that rank, or ~0.
__device__ __forceinline__ unsigned long long skip_above(const ChunkCtx &c, const unsigned int *U) {
    if (!c.L) return ~0ull;
    const int u = (int)*(volatile const unsigned int *)U;
    if (u > *(volatile const int *)c.L) return ~0ull;
    const unsigned long long key = *(volatile const unsigned long long *)c.key;
    if (key == kNoKey || (int)(key >> kRankBits) != u) return ~0ull;
    return key & (kRankLimit - 1);
}

// Colex state of a lane's next upper part (v elements of [0, K'), column M + 1 + element),
// its row sum and the rank of its first head.
template <int W, int P, class RowSrc>
struct UpperWalker {
    int el[kMaxG];
    uint32_t S[W];
    unsigned long long R;

    __device__ __forceinline__ void start(const ChunkCtx &c, const RowSrc &rows, int M, unsigned long long r) {
        const int v = c.v;
        int top = c.k - 1 - M - 1;
        for (int t = v; t >= 1; t--) {
            int l2 = t - 1, h = top;
            while (l2 < h) {
                const int mid = (l2 + h + 1) >> 1;
                if (binom_d(c.tb, c.stride, mid, t) <= r) l2 = mid; else h = mid - 1;
            }
            el[t - 1] = l2;
            r -= binom_d(c.tb, c.stride, l2, t);
            top = l2 - 1;
        }
        uint32_t rw[W];
        rows.load(M, rw);
#pragma unroll
        for (int w = 0; w < W; w++) S[w] = rw[w];
        R = binom_d(c.tb, c.stride, M, P + 1);
        for (int t = 0; t < v; t++) {
            const int col = M + 1 + el[t];
            rows.load(col, rw);
#pragma unroll
            for (int w = 0; w < W; w++) S[w] ^= rw[w];
            R += binom_d(c.tb, c.stride, col, P + 2 + t);
        }
    }

    // colex successor: the left-most element that can move up moves, those below it reset
    __device__ __forceinline__ void advance(const ChunkCtx &c, const RowSrc &rows, int M) {
        const int v = c.v;
        int t = 0;
        while (t < v - 1 && el[t] + 1 >= el[t + 1]) t++;
        uint32_t rw[W];
        for (int s = 0; s <= t; s++) {
            const int col = M + 1 + el[s];
            rows.load(col, rw);
#pragma unroll
            for (int w = 0; w < W; w++) S[w] ^= rw[w];
            R -= binom_d(c.tb, c.stride, col, P + 2 + s);
        }
        el[t] += 1;
        for (int s = 0; s < t; s++) el[s] = s;
        for (int s = 0; s <= t; s++) {
            const int col = M + 1 + el[s];
            rows.load(col, rw);
#pragma unroll
            for (int w = 0; w < W; w++) S[w] ^= rw[w];
            R += binom_d(c.tb, c.stride, col, P + 2 + s);
        }
    }
};

// One work item of a split level: the upper parts of one M entry assigned to this warp,
// NU of them per lane at a time.  U: the code's shared upper bound (read for thresholds,
// atomicMin'd on improvement).
template <int W, int WP, int P, int NU, class RowSrc, class H2Src>
__device__ __forceinline__ void split_chunk(const ChunkCtx &c, const MEntry &e, unsigned long long chunk,
                                            const RowSrc &rows, const H2Src &h2, unsigned int *U, int &Usnap,
                                            LaneBest &best) {
    const int lane = threadIdx.x & 31;
    const int M = (int)e.M;
    const unsigned long long per_lane = e.per_lane;
    const unsigned long long u0 = (chunk - e.chunk_begin) * 32ull * per_lane;
    const unsigned long long uend = min(u0 + 32ull * per_lane, (unsigned long long)e.uppers);
    const unsigned long long my_lo = u0 + (unsigned long long)lane * per_lane;
    const unsigned long long my_hi = min(my_lo + per_lane, uend);
    long long remaining = my_hi > my_lo ? (long long)(my_hi - my_lo) : 0;

    UpperWalker<W, P, RowSrc> up;
#pragma unroll
    for (int w = 0; w < W; w++) up.S[w] = 0;
    up.R = 0;
    if (remaining > 0) up.start(c, rows, M, e.upper_base + my_lo);
    // the completed stages' bound does not change during a level: the mid-level stop can only
    // apply once U has come down to it
    const int Lfix = c.L ? *(volatile const int *)c.L : -1;
    // U as last read; the read for the next head check is issued before each pair walk so its
    // latency hides behind the walk
    int Upre = Usnap;

    for (long long it = 0; it < (long long)per_lane; it += NU) {
        // a lane whose next upper part starts above the rank that settles the run stops
        if (remaining > 0 && min(Usnap, Upre) <= Lfix && up.R > skip_above(c, U)) {
            if (c.skipped) atomicAdd(c.skipped, (unsigned long long)remaining);
            remaining = 0;
        }
        const bool on = remaining > 0;
        if (!__any_sync(kFull, on)) break;
        // NU upper parts of this lane; past the lane's end the last one is repeated (a repeat
        // offers the same keys again and cannot change the minimum)
        uint32_t S[NU][W];
        unsigned long long R[NU];
#pragma unroll
        for (int q = 0; q < NU; q++) {
#pragma unroll
            for (int w = 0; w < W; w++) S[q][w] = up.S[w];
            R[q] = up.R;
            if (remaining > 0) {
                remaining--;
                if (remaining > 0) up.advance(c, rows, M);
            }
        }
        int thr = on ? min(Usnap, best.w()) - c.base : -1;
        // filter words: the fewest whose popcount-of-OR bound still rejects almost every
        // codeword at the warp's largest threshold (0 = exact weights)
        const int tmax = __reduce_max_sync(kFull, thr);
        int F = 0;
#pragma unroll
        for (int f = W; f >= 1; f--)
            if (tmax < (int)((c.fmax8 >> (8 * (f - 1))) & 0xff)) F = f;
        if constexpr (P == 2) {
            const int n2 = M * (M - 1) / 2;
            walk_dispatch<W, WP, NU>(F, h2, S, n2, thr, c.base, best, R);
        } else {
            for (int c3 = 2; c3 < M; c3++) {
                uint32_t T[NU][W], rw[W];
                unsigned long long rb[NU];
                rows.load(c3, rw);
                const unsigned long long h3 = (unsigned long long)c3 * (c3 - 1) * (c3 - 2) / 6;
                unsigned long long rmin = ~0ull;
#pragma unroll
                for (int q = 0; q < NU; q++) {
#pragma unroll
                    for (int w = 0; w < W; w++) T[q][w] = S[q][w] ^ rw[w];
                    rb[q] = R[q] + h3;
                    rmin = min(rmin, rb[q]);
                }
                // heads are walked in rank order: once every lane's next rank lies above the
                // rank that settles the run, the rest of this upper part's heads can go
                if (__any_sync(kFull, Upre <= Lfix) && __all_sync(kFull, !on || rmin > skip_above(c, U))) {
                    if (c.skipped && (threadIdx.x & 31) == 0) atomicAdd(c.skipped, 1ull);
                    break;
                }
                if (Lfix >= 0) Upre = (int)*(volatile const unsigned int *)U;
                const int n2 = c3 * (c3 - 1) / 2;
                walk_dispatch<W, WP, NU>(F, h2, T, n2, thr, c.base, best, rb);
            }
        }
        const int Ug = (int)*(volatile unsigned int *)U;
        Usnap = min(Usnap, Ug);
        if (best.w() < Usnap) {
            atomicMin(U, (unsigned int)best.w());
            Usnap = best.w();
        }
    }
}

// One work item of a small level: each lane walks its own run of colex ranks [lo, hi)
// with the colex successor, updating the row sum by the rows that leave and enter.
template <int W, int WP, class RowSrc>
__device__ __forceinline__ void simple_chunk(const ChunkCtx &c, unsigned long long lo, const unsigned long long hi,
                                             const RowSrc &rows, unsigned int *U, int &Usnap, LaneBest &best) {
    const int g = c.g;
    if (lo < hi && lo > skip_above(c, U)) {
        if (c.skipped) atomicAdd(c.skipped, 1ull);
        lo = hi;
    }
    if (lo < hi) {
        int cc[kMaxG];
        unsigned long long r = lo;
        int top = c.k - 1;
        for (int t = g; t >= 1; t--) {
            int l2 = t - 1, h = top;
            while (l2 < h) {
                const int mid = (l2 + h + 1) >> 1;
                if (binom_d(c.tb, c.stride, mid, t) <= r) l2 = mid; else h = mid - 1;
            }
            cc[t - 1] = l2;
            r -= binom_d(c.tb, c.stride, l2, t);
            top = l2 - 1;
        }
        uint32_t acc[W], rw[W];
#pragma unroll
        for (int w = 0; w < W; w++) acc[w] = 0;
        for (int t = 0; t < g; t++) {
            rows.load(cc[t], rw);
#pragma unroll
            for (int w = 0; w < W; w++) acc[w] ^= rw[w];
        }
        // ranks ascend within the lane: a strict improvement keeps the first rank
        int thr = min(Usnap, best.w()) - c.base;
        for (unsigned long long rank = lo; rank < hi; ++rank) {
            int s = 0;
#pragma unroll
            for (int w = 0; w < W; w++) s += __popc(acc[w]);
            if (s <= thr) {
                best.offer(s + c.base, rank);
                thr = s - 1;
            }
            if (rank + 1 < hi) {
                int t = 0;
                while (t < g - 1 && cc[t] + 1 >= cc[t + 1]) t++;
                for (int q = 0; q <= t; q++) {
                    rows.load(cc[q], rw);
#pragma unroll
                    for (int w = 0; w < W; w++) acc[w] ^= rw[w];
                }
                cc[t] += 1;
                for (int q = 0; q < t; q++) cc[q] = q;
                for (int q = 0; q <= t; q++) {
                    rows.load(cc[q], rw);
#pragma unroll
                    for (int w = 0; w < W; w++) acc[w] ^= rw[w];
                }
            }
        }
    }
    const int Ug = (int)*(volatile unsigned int *)U;
    Usnap = min(Usnap, Ug);
    if (best.w() < Usnap) {
        atomicMin(U, (unsigned int)best.w());
        Usnap = best.w();
    }
}

// Warp min of (weight << 55 | rank) and one atomicMin into the level key.
__device__ __forceinline__ void publish(unsigned long long *key, const LaneBest &best) {
    unsigned long long x = warp_min_u64(best.key);
    if ((threadIdx.x & 31) == 0 && x != kNoKey) atomicMin(key, x);
}

// Work item -> M entry (binary search on the first work item of each entry).
__device__ __forceinline__ int find_entry(const MEntry *mtab, int n_m, unsigned long long chunk) {
    int lo = 0, hi = n_m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&mtab[mid].chunk_begin) <= chunk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void stage_to_smem(uint32_t *dst, const uint32_t *src, int nwords) {
    const int n4 = nwords / 4;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = __ldg(s4 + i);
    for (int i = 4 * n4 + threadIdx.x; i < nwords; i += blockDim.x) dst[i] = __ldg(src + i);
}

}  // namespace dev
}  // namespace mdl
