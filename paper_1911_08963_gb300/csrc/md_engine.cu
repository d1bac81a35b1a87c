// md_engine.cu -- kernels of the multi-code engine (md_batch and the server).
//
// Every resident code keeps its own Alg. 1 state machine on the device: the bound U, the
// lower bound L, the stop flag and a level cursor.  The schedule advances in ticks.  A tick
// is three launches on one stream:
//   prepare  -- one block: every live code that has not stopped offers the next work
//               items of its current level (all of them, or a quota of about a fixed
//               number of combinations, for time slicing); the offers are compacted per row
//               width W with prefix sums;
//   round(W) -- persistent grid per row width present: warps take tickets from one
//               shared counter, so idle warps pick up items of any code (work stealing);
//   post     -- one block: codes whose level is now complete apply the bound check of
//               Section 2.2 (after every Gamma matrix) and Alg. 1 (L at the end of a stage)
//               and move their cursor to the next level.
// No kernel waits on another kernel; ticks are ordered by the stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "md_device.cuh"
#include "md_internal.h"

namespace mdl {

namespace {

using namespace dev;
constexpr int kEngineThreads = 256;
constexpr int kBinomStride = 257;

template <int W, int WP>
__global__ void __launch_bounds__(kEngineThreads) engine_round_kernel(const EngineArgs a, int Wc) {
    const unsigned long long total = *(volatile unsigned long long *)&a.act_total[Wc];
    if (total == 0) return;
    const int count = *(volatile int *)&a.act_count[Wc];
    const int *list = a.act_slots + (size_t)Wc * a.nslots;
    const unsigned long long *prefix = a.act_prefix + (size_t)Wc * a.nslots;
    unsigned long long *ctr = a.tick_ctr + Wc;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long ticket = 0;
        if (lane == 0) ticket = atomicAdd(ctr, 1ull);
        ticket = __shfl_sync(kFull, ticket, 0);
        if (ticket >= total) break;
        int lo = 0, hi = count - 1;          // first slot whose inclusive prefix exceeds the ticket
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(prefix + mid) > ticket) hi = mid; else lo = mid + 1;
        }
        const int slot = __ldg(list + lo);
        const BCode cd = a.codes[slot];
        const BState &stv = a.states[slot];
        const int cur = *(volatile const int *)&stv.cur;
        const unsigned long long item = *(volatile const unsigned long long *)&stv.next_item + ticket -
                                        (lo ? __ldg(prefix + lo - 1) : 0ull);
        const BLevel L = cd.levels[cur];
        const ChunkCtx c{cd.k, L.g, L.v, L.base, L.fmax8, a.binom, kBinomStride, &a.states[slot].L, &cd.keys[cur],
                         nullptr};
        unsigned int *U = &a.states[slot].U;
        int Usnap = (int)*(volatile unsigned int *)U;
        const GlobSrc<W, WP> rows{L.rows, (uint32_t)cd.k};
        LaneBest best;
        if (L.kind == KIND_SIMPLE) {
            const unsigned long long r0 = (item * 32ull + (unsigned long long)lane) * L.per_chunk;
            const unsigned long long r1 = min(r0 + L.per_chunk, L.count);
            simple_chunk<W, WP>(c, r0, r1, rows, U, Usnap, best);
        } else {
            const MEntry e = L.mtab[MD_BOUND(find_entry(L.mtab, L.n_m, item), L.n_m, kSiteMtab)];
            const GlobSrc<W, WP> h2{L.h2, (uint32_t)(cd.k * (cd.k - 1) / 2)};
            if (L.kind == KIND_SPLIT2) split_chunk<W, WP, 2, kNU>(c, e, item, rows, h2, U, Usnap, best);
            else split_chunk<W, WP, 3, kNU>(c, e, item, rows, h2, U, Usnap, best);
        }
        publish(&cd.keys[cur], best);
    }
}

// Block-wide inclusive scan of one value per thread (blockDim.x = 1024).
template <class T>
__device__ T block_inclusive_scan(T x, T *warp_tot, T &block_total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (wid > 0) x += warp_tot[wid - 1];
    block_total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return x;
}

__global__ void __launch_bounds__(1024) engine_prepare_kernel(const EngineArgs a) {
    __shared__ unsigned long long wt_u64[32];
    __shared__ int wt_int[32];
    __shared__ int run_count[kWClasses];
    __shared__ unsigned long long run_total[kWClasses];
    __shared__ unsigned int present;            // row widths offered in this tile
    if (threadIdx.x < kWClasses) {
        run_count[threadIdx.x] = 0;
        run_total[threadIdx.x] = 0;
        a.tick_ctr[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int base = 0; base < a.nslots; base += blockDim.x) {
        const int s = base + threadIdx.x;
        int wc = 0;
        unsigned long long items = 0;
        if (s < a.nslots) {
            const BCode cd = a.codes[s];
            BState &st = a.states[s];
            if (cd.live && !st.stop && st.cur < cd.nlev) {
                const BLevel &L = cd.levels[st.cur];
                items = L.nchunks - st.next_item;
                if (L.quota && items > L.quota) items = L.quota;
                wc = L.W;
            }
            st.tick_items = items;
        }
        if (threadIdx.x == 0) present = 0;
        __syncthreads();
        if (items > 0) atomicOr(&present, 1u << wc);
        __syncthreads();
        const unsigned int mask = present;
        for (int w = 1; w < kWClasses; w++) {
            if (!((mask >> w) & 1u)) continue;          // block-uniform: no slot of this width
            const int flag = (wc == w && items > 0) ? 1 : 0;
            int nflag = 0;
            unsigned long long ntot = 0;
            const int pos = block_inclusive_scan<int>(flag, wt_int, nflag) - flag;
            const unsigned long long pre = block_inclusive_scan<unsigned long long>(flag ? items : 0ull, wt_u64, ntot);
            if (flag) {
                a.act_slots[(size_t)w * a.nslots + run_count[w] + pos] = s;
                a.act_prefix[(size_t)w * a.nslots + run_count[w] + pos] = run_total[w] + pre;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                run_count[w] += nflag;
                run_total[w] += ntot;
            }
            __syncthreads();
        }
        __syncthreads();                            // every thread has read `present`
    }
    if (threadIdx.x < kWClasses) {
        a.act_count[threadIdx.x] = run_count[threadIdx.x];
        a.act_total[threadIdx.x] = run_total[threadIdx.x];
    }
}

__global__ void engine_post_kernel(const EngineArgs a) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nslots; s += gridDim.x * blockDim.x) {
        BState st = a.states[s];
        if (st.tick_items == 0) continue;
        const BCode cd = a.codes[s];
        const BLevel &L = cd.levels[st.cur];
        st.next_item += st.tick_items;
        st.tick_items = 0;
        if (st.next_item >= L.nchunks) {
            // level complete: the bound check after each Gamma matrix, L(g) after a stage
            st.last_level = st.cur;
            const int U = (int)st.U;
            if (L.L_first && L.L_after >= 0) st.L = max(st.L, L.L_after);   // per-matrix bound
            if (st.L >= U) {
                st.stop = 1;
            } else if (L.L_after >= 0) {
                st.L = max(st.L, L.L_after);
                if (st.L >= U) st.stop = 1;
            }
            st.cur += 1;
            st.next_item = 0;
        }
        a.states[s] = st;
    }
}

// Pair tables of many matrices: block b builds matrix b's table.
__global__ void h2_many_kernel(const uint32_t *const *rows, uint32_t *const *h2, const int *kk, const int *wp) {
    const int b = blockIdx.x;
    const uint32_t *R = rows[b];
    uint32_t *H = h2[b];
    const int k = kk[b], WP = wp[b];
    const long long npairs = (long long)k * (k - 1) / 2;
    for (long long idx = threadIdx.x; idx < npairs * WP; idx += blockDim.x) {
        const long long pr = idx / WP;
        const int w = (int)(idx % WP);
        int c2 = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) / 2.0);
        while ((long long)c2 * (c2 - 1) / 2 > pr) c2--;
        while ((long long)(c2 + 1) * c2 / 2 <= pr) c2++;
        const int c1 = (int)(pr - (long long)c2 * (c2 - 1) / 2);
        H[idx] = R[c1 * WP + w] ^ R[c2 * WP + w];
    }
}

template <int W, int WP>
cudaError_t launch_round_w(const EngineArgs &a, int blocks, int threads, cudaStream_t s) {
    engine_round_kernel<W, WP><<<blocks, threads, 0, s>>>(a, W);
    return cudaGetLastError();
}

template <int W, int WP>
int occ_w(int threads) {
    int nb = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, engine_round_kernel<W, WP>, threads, 0) == cudaSuccess
               ? nb : 0;
}

}  // namespace

int launch_engine_round(const EngineArgs &a, int W, int blocks, int threads, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (W) {
        case 1: return (int)launch_round_w<1, 1>(a, blocks, threads, s);
        case 2: return (int)launch_round_w<2, 2>(a, blocks, threads, s);
        case 3: return (int)launch_round_w<3, 4>(a, blocks, threads, s);
        case 4: return (int)launch_round_w<4, 4>(a, blocks, threads, s);
        case 5: return (int)launch_round_w<5, 8>(a, blocks, threads, s);
        case 6: return (int)launch_round_w<6, 8>(a, blocks, threads, s);
        case 7: return (int)launch_round_w<7, 8>(a, blocks, threads, s);
        case 8: return (int)launch_round_w<8, 8>(a, blocks, threads, s);
        default: return (int)cudaErrorInvalidValue;
    }
}

int engine_blocks_per_sm(int W, int threads) {
    switch (W) {
        case 1: return occ_w<1, 1>(threads);
        case 2: return occ_w<2, 2>(threads);
        case 3: return occ_w<3, 4>(threads);
        case 4: return occ_w<4, 4>(threads);
        case 5: return occ_w<5, 8>(threads);
        case 6: return occ_w<6, 8>(threads);
        case 7: return occ_w<7, 8>(threads);
        default: return occ_w<8, 8>(threads);
    }
}

int launch_engine_prepare(const EngineArgs &a, void *stream) {
    engine_prepare_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int launch_engine_post(const EngineArgs &a, void *stream) {
    const int blocks = (a.nslots + 255) / 256;
    engine_post_kernel<<<blocks > 0 ? blocks : 1, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int launch_h2_build_many(const uint32_t *const *rows, uint32_t *const *h2, const int *k, const int *WP, int count,
                         void *stream) {
    if (count <= 0) return 0;
    h2_many_kernel<<<count, 256, 0, (cudaStream_t)stream>>>(rows, h2, k, WP);
    return (int)cudaGetLastError();
}

MD_BOUNDS_ACCESSOR(bounds_site_engine)

}  // namespace mdl
