// md_kernels.cu -- sm_103a kernels of the Brouwer-Zimmermann enumeration.
//
// The hot loop of the paper (Section 2.2: "the generation of all the linear
// combinations ... is the most compute-intensive part"; Process_combination in Alg. 2)
// forms every sum of g rows of Gamma_j and takes its weight.  On the GPU:
//
//   * A combination c_1 < ... < c_g is split as head (c_1..c_P), pivot M = c_{P+1} and
//     an upper part (c_{P+2}..c_g).  Its colex rank (Section 3.1, left-lexicographical
//     order) is  sum_i C(c_i, i) = head index + C(M, P+1) + sum_{i>P+1} C(c_i, i),  so for
//     fixed M and upper part the heads occupy one contiguous run of ranks.
//   * A work item is a run of upper parts sharing M.  Each lane holds one upper part's
//     row sum S in registers (the "left combination" of the paper's saved-additions
//     scheme, Section 2.2.1); the warp walks all heads below M in lockstep, reading the
//     pre-added pair sums (the "right combinations") from shared memory as warp-wide
//     broadcasts.  Every codeword costs one XOR per 32-bit word.
//   * Weights: W words of popc.  When the current bound U is far below the typical weight,
//     the weight is first bounded below by popc(OR of the W words) -- one POPC instead
//     of W -- and only codewords that could reach U get their exact weight.
//   * Minimum tracking: each lane keeps its best (weight, rank); a warp min and one 64-bit
//     atomicMin per work item publish (weight << 55 | colex rank) per level, and an
//     atomicMin on U lets every warp tighten its threshold (the OpenMP reduction of
//     Section 2.2.2, with one global update per work item).
//   * Work items are taken from a per-level atomic counter (dynamic distribution, as the
//     paper's D-* family, Section 3.2, at warp granularity).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "md_device.cuh"
#include "md_internal.h"

namespace mdl {

namespace {

using namespace dev;
constexpr int kThreads = 512;

// The warp's next work item of the level (lane 0 takes a ticket, the warp shares it), or
// ~0 once the caller cancels the run: the cancel word (mapped host memory) is read before
// every ticket, and a cancelled run is stopped with MD_ECANCELED for the levels after it.
__device__ __forceinline__ unsigned long long next_item(const LevelArgs &a, int lane) {
    unsigned long long chunk = 0;
    if (lane == 0) {
        if (a.cancel && *a.cancel) {
            atomicExch(&a.st->error, MD_ECANCELED);
            atomicExch(&a.st->stop, 1);
            chunk = ~0ull;
        } else {
            chunk = atomicAdd(&a.st->ctr[a.level], 1ull);
        }
    }
    return __shfl_sync(kFull, chunk, 0);
}

// ---------------------------------------------------------------- split kernel ----
// One level (g, j) of one code.  The packed rows of Gamma_j are staged in shared memory
// once per block, with the pair table too when it fits (H2S); warps then take work items
// from the level's atomic counter until none is left.
template <int W, int WP, int P, bool H2S>
__global__ void __launch_bounds__(kThreads, 1) split_kernel(const LevelArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    DevState *st = a.st;
    if (a.check_stop && *(volatile int *)&st->stop) return;
    const int k = a.k;
    const int rows_words = (k * WP + 3) & ~3;
    stage_to_smem(smem, a.rows, k * WP);
    if constexpr (H2S) stage_to_smem(smem + rows_words, a.h2, (k * (k - 1) / 2) * WP);
    __syncthreads();

    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const SmemSrc<W, WP> rows{sbase, (uint32_t)k};
    const ChunkCtx c{k, a.g, a.v, a.base, a.fmax8, a.binom, k + 1,
                     a.check_stop ? &st->L : nullptr, &st->key[a.level], &st->skipped};
    const int lane = threadIdx.x & 31;
    int Usnap = (int)*(volatile unsigned int *)&st->U;

    for (;;) {
        const unsigned long long chunk = next_item(a, lane);
        if (chunk >= a.nchunks) break;
        const MEntry e = a.mtab[MD_BOUND(find_entry(a.mtab, a.n_m, chunk), a.n_m, kSiteMtab)];
        LaneBest best;
        if constexpr (H2S) {
            const SmemSrc<W, WP> h2{sbase + (uint32_t)rows_words * 4u, (uint32_t)(k * (k - 1) / 2)};
            split_chunk<W, WP, P, kNU>(c, e, chunk, rows, h2, &st->U, Usnap, best);
        } else {
            const GlobSrc<W, WP> h2{a.h2, (uint32_t)(k * (k - 1) / 2)};
            split_chunk<W, WP, P, kNU>(c, e, chunk, rows, h2, &st->U, Usnap, best);
        }
        publish(&st->key[a.level], best);
    }
}

// --------------------------------------------------------------- simple kernel ----
// Small levels (g <= 4 or few combinations) and colex rank ranges: each lane walks its own
// run of ranks [r_begin + (32 * item + lane) * per_chunk, ...).
template <int W, int WP>
__global__ void __launch_bounds__(kThreads, 1) simple_kernel(const LevelArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    DevState *st = a.st;
    if (a.check_stop && *(volatile int *)&st->stop) return;
    const int k = a.k;
    stage_to_smem(smem, a.rows, k * WP);
    __syncthreads();
    const SmemSrc<W, WP> rows{(uint32_t)__cvta_generic_to_shared(smem), (uint32_t)k};
    const ChunkCtx c{k, a.g, a.v, a.base, a.fmax8, a.binom, k + 1,
                     a.check_stop ? &st->L : nullptr, &st->key[a.level], &st->skipped};
    const int lane = threadIdx.x & 31;
    int Usnap = (int)*(volatile unsigned int *)&st->U;
    for (;;) {
        const unsigned long long chunk = next_item(a, lane);
        if (chunk >= a.nchunks) break;
        const unsigned long long lo = a.r_begin + (chunk * 32ull + (unsigned long long)lane) * a.per_chunk;
        const unsigned long long hi = min(lo + a.per_chunk, (unsigned long long)a.count);
        LaneBest best;
        simple_chunk<W, WP>(c, lo, hi, rows, &st->U, Usnap, best);
        publish(&st->key[a.level], best);
    }
}

// Pair table: H2[C(c2, 2) + c1] = row c1 ^ row c2 for c1 < c2 (colex order of pairs).
__global__ void h2_kernel(const uint32_t *rows, uint32_t *h2, int k, int WP) {
    const long long npairs = (long long)k * (k - 1) / 2;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < npairs * WP;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long pr = idx / WP;
        const int w = (int)(idx % WP);
        int c2 = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) / 2.0);
        while ((long long)c2 * (c2 - 1) / 2 > pr) c2--;
        while ((long long)(c2 + 1) * c2 / 2 <= pr) c2++;
        const int c1 = (int)(pr - (long long)c2 * (c2 - 1) / 2);
        h2[idx] = rows[c1 * WP + w] ^ rows[c2 * WP + w];
    }
}

// After level `a.level`: compare the bounds (Section 2.2: after each Gamma matrix) and,
// at the end of a stage, raise L to L(g) (Alg. 1).
__global__ void finalize_kernel(const LevelArgs a) {
    DevState *st = a.st;
    if (st->stop) return;
    st->last_level = a.level;
    const int U = (int)st->U;
    if (a.level + 1 < kMaxLevels) st->u_in[a.level + 1] = (unsigned int)U;
    if (a.L_first && a.L_after >= 0) st->L = max(st->L, a.L_after);   // per-matrix bound
    if (st->L >= U) { st->stop = 1; return; }
    if (a.L_after >= 0) {                       // the bound this level completes
        st->L = max(st->L, a.L_after);
        if (st->L >= U) st->stop = 1;
    }
}

__global__ void state_init_kernel(DevState *st, unsigned int u0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t; i < kMaxLevels; i += gridDim.x * blockDim.x) {
        st->key[i] = kNoKey;
        st->ctr[i] = 0;
        st->u_in[i] = u0;
    }
    if (t == 0) {
        st->U = u0;
        st->L = 1;
        st->stop = 0;
        st->error = 0;
        st->last_level = -1;
        st->skipped = 0;
    }
}

template <int W, int WP>
cudaError_t launch_kind(const LevelArgs &a, int kind, int blocks, int threads, size_t smem, cudaStream_t s) {
    if (kind == KIND_SIMPLE) {
        auto kern = simple_kernel<W, WP>;
        allow_full_smem((const void *)kern);
        kern<<<blocks, threads, smem, s>>>(a);
    } else if (kind == KIND_SPLIT2) {
        if (a.h2_in_smem) {
            auto kern = split_kernel<W, WP, 2, true>;
            allow_full_smem((const void *)kern);
            kern<<<blocks, threads, smem, s>>>(a);
        } else {
            auto kern = split_kernel<W, WP, 2, false>;
            allow_full_smem((const void *)kern);
            kern<<<blocks, threads, smem, s>>>(a);
        }
    } else {
        if (a.h2_in_smem) {
            auto kern = split_kernel<W, WP, 3, true>;
            allow_full_smem((const void *)kern);
            kern<<<blocks, threads, smem, s>>>(a);
        } else {
            auto kern = split_kernel<W, WP, 3, false>;
            allow_full_smem((const void *)kern);
            kern<<<blocks, threads, smem, s>>>(a);
        }
    }
    return cudaGetLastError();
}

}  // namespace

int launch_level(const LevelArgs &a, int kind, int W, int WP, int blocks, int threads, size_t smem, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (W) {
        case 1: e = launch_kind<1, 1>(a, kind, blocks, threads, smem, s); break;
        case 2: e = launch_kind<2, 2>(a, kind, blocks, threads, smem, s); break;
        case 3: e = launch_kind<3, 4>(a, kind, blocks, threads, smem, s); break;
        case 4: e = launch_kind<4, 4>(a, kind, blocks, threads, smem, s); break;
        case 5: e = launch_kind<5, 8>(a, kind, blocks, threads, smem, s); break;
        case 6: e = launch_kind<6, 8>(a, kind, blocks, threads, smem, s); break;
        case 7: e = launch_kind<7, 8>(a, kind, blocks, threads, smem, s); break;
        case 8: e = launch_kind<8, 8>(a, kind, blocks, threads, smem, s); break;
        default: return (int)cudaErrorInvalidValue;
    }
    (void)WP;
    return (int)e;
}

int launch_h2_build(const uint32_t *rows, uint32_t *h2, int k, int WP, void *stream) {
    const long long total = (long long)k * (k - 1) / 2 * WP;
    if (total == 0) return 0;
    int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    h2_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(rows, h2, k, WP);
    return (int)cudaGetLastError();
}

int launch_finalize(const LevelArgs &a, void *stream) {
    finalize_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int launch_state_init(DevState *st, unsigned int u0, void *stream) {
    state_init_kernel<<<8, 128, 0, (cudaStream_t)stream>>>(st, u0);
    return (int)cudaGetLastError();
}

int level_smem_bytes(int k, int WP, bool h2_in_smem) {
    const int rows_words = (k * WP + 3) & ~3;
    long long words = rows_words;
    if (h2_in_smem) words += (long long)k * (k - 1) / 2 * WP;
    return (int)(words * 4);
}

int allow_full_smem(const void *kernel) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, kernel})) return cudaSuccess;
    cudaFuncAttributes fa{};
    int optin = 0;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert({dev, kernel});
    else cudaGetLastError();
    return (int)e;
}

int level_blocks_per_sm(int kind, int W, bool h2s, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaSuccess;
#define MDL_OCC(KERN)                                                                          \
    do {                                                                                       \
        allow_full_smem((const void *)KERN);                                                  \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, KERN, threads, smem);           \
    } while (0)
#define MDL_OCC_W(WW, WPP)                                                                     \
    case WW:                                                                                   \
        if (kind == KIND_SIMPLE) MDL_OCC((simple_kernel<WW, WPP>));                            \
        else if (kind == KIND_SPLIT2 && h2s) MDL_OCC((split_kernel<WW, WPP, 2, true>));        \
        else if (kind == KIND_SPLIT2) MDL_OCC((split_kernel<WW, WPP, 2, false>));              \
        else if (h2s) MDL_OCC((split_kernel<WW, WPP, 3, true>));                               \
        else MDL_OCC((split_kernel<WW, WPP, 3, false>));                                       \
        break;
    switch (W) {
        MDL_OCC_W(1, 1) MDL_OCC_W(2, 2) MDL_OCC_W(3, 4) MDL_OCC_W(4, 4)
        MDL_OCC_W(5, 8) MDL_OCC_W(6, 8) MDL_OCC_W(7, 8) MDL_OCC_W(8, 8)
        default: return 0;
    }
#undef MDL_OCC_W
#undef MDL_OCC
    return e == cudaSuccess ? nb : 0;
}

// ------------------------------------------------------------- POPC throughput ----
// Every thread runs 16 independent popc -> add chains whose inputs change each iteration (one
// integer add feeds each popc), so the POPC pipe is the limit: 16 x 32 popc lane-operations per
// warp iteration against 2 x 16 x 32 integer adds.  One block per SM (the shared-memory request
// keeps a second one away); cycles by clock64 between two block barriers.
__global__ void __launch_bounds__(1024, 1) popc_probe_kernel(unsigned iters, unsigned seed, unsigned long long *cycles,
                                                            unsigned *sink) {
    uint32_t x[16], acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 16; j++) x[j] = seed * (threadIdx.x + 1u) + (uint32_t)j * 0x9E3779B9u;
    __syncthreads();
    const long long t0 = clock64();
    for (unsigned i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 16; j++) {
            x[j] += i;
            acc[j & 3] += (uint32_t)__popc(x[j]);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
    if ((acc[0] ^ acc[1] ^ acc[2] ^ acc[3]) == 0x9E3779B9u) sink[0] = 1u;   // keeps the work live
}

int max_smem_per_block() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

MD_BOUNDS_ACCESSOR(bounds_site_kernels)

int sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

}  // namespace mdl

// POPC lane-operations per SM per clock (median over one block per SM).
extern "C" int md_popc_rate(double *per_sm_per_clk) {
    using namespace mdl;
    if (!per_sm_per_clk) return MD_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    const int smem = 120 * 1024;
    unsigned long long *cyc = nullptr;
    unsigned *sink = nullptr;
    if (cudaFuncSetAttribute(popc_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(unsigned long long) * sms) != cudaSuccess || cudaMalloc(&sink, 4) != cudaSuccess) {
        cudaGetLastError();
        if (cyc) cudaFree(cyc);
        return MD_ECUDA;
    }
    const unsigned iters = 1u << 14;
    popc_probe_kernel<<<sms, 1024, smem>>>(256u, 7u, cyc, sink);                 // warm-up
    popc_probe_kernel<<<sms, 1024, smem>>>(iters, 7u, cyc, sink);
    std::vector<unsigned long long> h(sms);
    bool ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
              cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(cyc);
    cudaFree(sink);
    if (!ok) { cudaGetLastError(); return MD_ECUDA; }
    std::sort(h.begin(), h.end());
    const double med = (double)h[h.size() / 2];
    if (med <= 0) return MD_EINTERNAL;
    *per_sm_per_clk = 1024.0 * iters * 16.0 / med;
    return MD_OK;
}
