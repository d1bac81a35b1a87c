// md_noalloc.cu -- md_scan_range_noalloc: the rank-range scan for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time or embedded loops that forbid allocation
// after start-up (an allocation may wait for the whole device), and processes whose device
// memory is owned by another allocator (a framework's caching allocator) that this library
// must not bypass.  This entry point gives them the colex rank-range scan with no
// allocation: its device scratch (the bound U, the work-item counter, the result key and a
// binomial table) lives in one file-scope __device__ array of fixed size that every GPU
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "md_device.cuh"
#include "md_internal.h"

namespace mdl {
namespace {

using namespace dev;

constexpr int kNoAllocMaxK = MD_NOALLOC_MAX_K;
constexpr int kThreads = 256;

// Scratch layout: [0, 64) the run state, [256, ...) C(a, b) for a, b <= kNoAllocMaxK.
struct NoAllocState {
    unsigned int U;
    unsigned int pad;
    unsigned long long ctr;
    unsigned long long key;
};
constexpr size_t kBinomOffset = 256;
constexpr size_t kScratchBytes = kBinomOffset + (size_t)(kNoAllocMaxK + 1) * (kNoAllocMaxK + 1) * 8;
static_assert(kScratchBytes <= MD_NOALLOC_SCRATCH_BYTES, "scratch size");

static __device__ __align__(256) unsigned char md_noalloc_scratch[MD_NOALLOC_SCRATCH_BYTES];

// Host-side address of the scratch on each device, found once per device.
std::mutex g_mu;
void *g_ptr[64] = {nullptr};

__global__ void noalloc_reset_kernel(NoAllocState *st, unsigned int u0) {
    st->U = u0;
    st->ctr = 0ull;
    st->key = kNoKey;
}

// The per-lane colex walk of the rank-range scan (the small-level kernel of md_kernels.cu),
// with its state and binomial table taken from the scratch array.
template <int W, int WP>
__global__ void __launch_bounds__(kThreads) noalloc_scan_kernel(const uint32_t *rows_g, int k, int g, int base,
                                                                unsigned long long r_begin, unsigned long long r_end,
                                                                unsigned long long per_chunk,
                                                                unsigned long long nchunks, unsigned char *scratch) {
    extern __shared__ __align__(16) uint32_t smem[];
    NoAllocState *st = reinterpret_cast<NoAllocState *>(scratch);
    const unsigned long long *tb = reinterpret_cast<const unsigned long long *>(scratch + kBinomOffset);
    stage_to_smem(smem, rows_g, k * WP);
    __syncthreads();
    const SmemSrc<W, WP> rows{(uint32_t)__cvta_generic_to_shared(smem), (uint32_t)k};
    const ChunkCtx c{k, g, 0, base, 0ull, tb, kNoAllocMaxK + 1, nullptr, nullptr, nullptr};
    const int lane = threadIdx.x & 31;
    int Usnap = (int)*(volatile unsigned int *)&st->U;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(&st->ctr, 1ull);
        chunk = __shfl_sync(kFull, chunk, 0);
        if (chunk >= nchunks) break;
        const unsigned long long lo = r_begin + (chunk * 32ull + (unsigned long long)lane) * per_chunk;
        const unsigned long long hi = min(lo + per_chunk, r_end);
        LaneBest best;
        simple_chunk<W, WP>(c, lo, hi, rows, &st->U, Usnap, best);
        publish(&st->key, best);
    }
}

template <int W, int WP>
cudaError_t launch_scan(const uint32_t *rows, int k, int g, int base, unsigned long long r0, unsigned long long r1,
                        unsigned long long per_chunk, unsigned long long nchunks, unsigned char *scratch,
                        int blocks, cudaStream_t s) {
    const size_t smem = (size_t)((k * WP + 3) & ~3) * 4;
    noalloc_scan_kernel<W, WP><<<blocks, kThreads, smem, s>>>(rows, k, g, base, r0, r1, per_chunk, nchunks, scratch);
    return cudaGetLastError();
}

// Find the scratch address on the current device and fill its binomial table (first call
// on each device only).
int scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return MD_ECUDA; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, md_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return MD_ECUDA; }
        static unsigned long long tb[(kNoAllocMaxK + 1) * (kNoAllocMaxK + 1)];
        for (int a = 0; a <= kNoAllocMaxK; a++)
            for (int b = 0; b <= kNoAllocMaxK; b++) tb[a * (kNoAllocMaxK + 1) + b] = binom(a, b);
        if (cudaMemcpyToSymbol(md_noalloc_scratch, tb, sizeof(tb), kBinomOffset, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            cudaGetLastError();
            return MD_ECUDA;
        }
        g_ptr[dev] = p;
    }
    *out = (unsigned char *)g_ptr[dev];
    return MD_OK;
}

}  // namespace

MD_BOUNDS_ACCESSOR(bounds_site_noalloc)

}  // namespace mdl

using namespace mdl;

extern "C" int md_scan_range_noalloc(const uint32_t *rows, int k, int words, int weight_base, int g, uint64_t r0,
                                     uint64_t r1, int bound, void *stream, int *weight, uint64_t *first_rank) {
    if (!rows || !weight || !first_rank) return MD_EINVAL;
    if (k < 1 || g < 1 || g > k || words < 1 || words > 8 || weight_base < 0) return MD_EINVAL;
    if (((uintptr_t)rows & 15) != 0) return MD_EINVAL;
    if (k > kNoAllocMaxK) return MD_EUNSUPPORTED;          // beyond the scratch's binomial table
    const uint64_t total = binom(k, g);
    if (total >= kRankLimit) return MD_EUNSUPPORTED;
    if (r1 > total) r1 = total;
    if (r0 > r1) r0 = r1;
    unsigned char *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != MD_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t span = r1 - r0;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    unsigned long long per_chunk = span / (32ull * (unsigned long long)sms * 16);
    if (per_chunk < 1) per_chunk = 1;
    if (per_chunk > 4096) per_chunk = 4096;
    const unsigned long long nchunks = (span + 32 * per_chunk - 1) / (32 * per_chunk);
    const unsigned long long want = (unsigned long long)sms * 4;
    const int blocks = (int)(nchunks / (kThreads / 32) + 1 < want ? nchunks / (kThreads / 32) + 1 : want);
    const unsigned int u0 = bound >= 0 ? (unsigned int)bound : 0x7fffffffu;
    NoAllocState *st = reinterpret_cast<NoAllocState *>(scratch);
    noalloc_reset_kernel<<<1, 1, 0, s>>>(st, u0);               // every call starts from a clean state
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && span > 0) {
        switch (words) {
            case 1: e = launch_scan<1, 1>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            case 2: e = launch_scan<2, 2>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            case 3: e = launch_scan<3, 4>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            case 4: e = launch_scan<4, 4>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            case 5: e = launch_scan<5, 8>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            case 6: e = launch_scan<6, 8>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            case 7: e = launch_scan<7, 8>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
            default: e = launch_scan<8, 8>(rows, k, g, weight_base, r0, r1, per_chunk, nchunks, scratch, blocks, s); break;
        }
    }
    unsigned long long key = kNoKey;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&key, &st->key, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cudaGetLastError(); return MD_ECUDA; }
    if (bounds_status() != MD_OK) return MD_EINTERNAL;
    if (key == kNoKey) { *weight = -1; *first_rank = 0; }
    else { *weight = (int)(key >> kRankBits); *first_rank = key & (kRankLimit - 1); }
    return MD_OK;
}
