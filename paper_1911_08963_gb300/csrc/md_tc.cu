// md_tc.cu -- one level (g, j) of the enumeration on the fifth-generation tensor cores.
//
// The weight of a sum of g rows of Gamma_j is base + popcount(S), S the XOR of their packed
// rows.  Mapping every packed bit b to the sign (-1)^b turns the popcount into an inner
// product: for packed vectors x, y of K = 32 W bits,  <sign x, sign y> = K - 2 popcount(x ^ y).
//
// A combination c_1 < ... < c_g is split into a head (c_1..c_q) and a tail (c_{q+1}..c_g)
// with smallest tail element s = c_{q+1}.  For one s the admissible heads are exactly the
// q-subsets of [0, s), i.e. the first C(s, q) heads in colex order, and every (tail, head)
// pair of that s is a combination.  So the weights of all combinations with a given s form
// one dense product D = A B^T, A = signs of the tail sums, B = signs of the head sums: the
// left/right combination split of Section 2.2.1 taken all the way to a matrix product.  Its
// colex rank is (head index) + sum_{i > q} C(c_i, i), so within one tail the first column
// holding a row's best weight is that tail's smallest rank of it.
//
// Two phases cover a level: phase 0 takes the combinations with s = c_{q+1} >= s_min and the
// split above; phase 1 takes those with c_{q+1} < s_min and splits one element later: heads
// (c_1..c_{q+1}) with c_{q+1} < s_min (a colex prefix of the (q+1)-subsets) and tails
// (c_{q+2}..c_g).  For small s the q-heads are few, so a tail would serve only one or two
// head slices and cost more to produce than to multiply; the second phase gives every tail
// of those combinations C(min(s, s_min), q + 1) heads.
//
//   * Heads: a table of the C(k, q) head sums as e4m3 signs (+1.0 = 0x38, -1.0 = 0xB8), in
//     256-row slices of 8-row x 16-byte core matrices (the K-major operand layout without
//     swizzle), built once per matrix and copied slice by slice into shared memory with bulk
//     copies (cp.async.bulk, completion on an mbarrier).
//   * Tails: four producer warps (one per SM sub-partition, so their work spreads evenly
//     beside the epilogue warps), one tile row per thread; a thread unranks one tail per
//     item and walks its na consecutive tails in colex order (row p of each of the item's
//     tiles), keeping the tail sum in registers, and writes its e4m3 signs: two 16-byte
//     stores per packed word.  A colex step moves a run of consecutive elements
//     o0..o0+m: they leave, s+1..s+m and o0+m+1 enter, which prefix XORs of the rows give in
//     five lookups whatever m is (usually m = 0: one XOR with the difference of two adjacent
//     rows).  The rows, their adjacent differences and prefix XORs sit in shared memory
//     word-major, so the 32 lanes' reads spread over the banks.
//   * A work item is a block of up to 128 T tails (T tiles, kept in shared memory, two sets
//     so the producers fill one while the other is in use) times a group of up to 16 head
//     slices of the same s: every tail tile is multiplied with each slice of the group, so
//     generating it costs little per codeword, and each slice is fetched once for T tiles.
//   * Two threads issue tcgen05.mma kind::f8f6f4 (M = 128 tails, N <= 256 heads, one
//     instruction per 32 packed bits), each into its own accumulator: D accumulates in fp32
//     in tensor memory (exact, |D| <= 256), two accumulators of 256 columns.  The W MMAs of
//     one product form a dependent chain; issued from two threads, the chains of the two
//     accumulators interleave in the tensor pipe, which hides the latency between the MMAs
//     of a chain, while the epilogue drains whichever accumulator is done.
//   * Four epilogue warps (one per tensor-memory lane quarter) read D with tcgen05.ld.red,
//     which also returns each lane's maximum over the columns it loads, so no per-element
//     arithmetic is left: two round trips of two 64-column loads per accumulator.  (Two
//     warps of a sub-partition issuing tcgen05.ld.red while products run slowed the
//     turnaround of the accumulators, hence one warp per quarter.)  Per tile the common path
//     is one compare with a threshold kept per item and one warp vote, which also orders the
//     warp's loads before lane 0 frees the accumulator.  A row reaching
//     K - 2 (min(U, best) - base) takes an out-of-line path: it is resolved to (weight, first
//     rank) and published with atomicMin, as in the other level kernels.
//   * One scheduler thread takes work items (s, head slices, run of tails) from the level's
//     atomic counter, applies the mid-level stop, and passes them on through a ring in shared
//     memory.
// Every wait is bounded by the global timer; on expiry the block records MD_ETIMEOUT in the
// state, stops the run, waits (bounded) for its own tensor-core work, frees its tensor memory
// and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "md_device.cuh"
#include "md_internal.h"

namespace mdl {

namespace {

using namespace dev;

constexpr int kTcM = 128;                  // tails per tile (tensor-memory lanes)
constexpr int kTcN = 256;                  // heads per slice (accumulator columns)
// 11 warps: one SM sub-partition holds three of them, and its 16384 registers cap a thread at
// 170, so 168 with the allocation unit of 8; a launch above the cap fails for lack of
// registers, hence the explicit limit.  An epilogue warp keeps two 64-column loads (a
// 128-column half of an accumulator) in flight within it.
constexpr int kEpiWarps = 4;               // warps 0-3: one per tensor-memory lane quarter
constexpr int kProdWarp0 = 4;              // warps 4-7: one tile row per thread
constexpr int kProdWarps = 4;
constexpr int kProdRows = kTcM / (32 * kProdWarps);   // tile rows per producer thread
constexpr int kMmaWarp0 = 8;              // warps 8-9: one MMA issuer per accumulator
constexpr int kMmaWarps = 2;
constexpr int kSchedWarp = 10;
constexpr int kTcWarps = 11;
constexpr int kTcThreads = kTcWarps * 32;
constexpr int kTcMaxRegs = 168;
static_assert((kTcWarps + 3) / 4 * 32 * kTcMaxRegs <= 16384, "register cap above a sub-partition's file");
static_assert(kProdRows * 32 * kProdWarps == kTcM, "producer threads must cover the tile rows");
static_assert(kSchedWarp == kTcWarps - 1 && kMmaWarp0 == kProdWarp0 + kProdWarps, "warp roles overlap");
constexpr int kRing = 8;                   // work items between the scheduler and the others
constexpr int kItemReaders = kEpiWarps + kProdWarps + kMmaWarps;   // warps that take each ring entry
constexpr uint32_t kTmemCols = 512;
constexpr unsigned long long kWaitNs = 4000000000ull;
constexpr int kMaxV = 10;                  // upper elements of a tail (g - q - 1) handled

constexpr int kGroup = 16;                 // head slices per work item

// Tail tiles per set (two sets), as shared memory allows for the row width.
__host__ __device__ constexpr int tc_tiles_per_set(int W) { return W <= 2 ? 8 : W <= 4 ? 4 : W <= 6 ? 2 : 1; }

template <int W>
struct TcCfg {
    static constexpr int kTiles = tc_tiles_per_set(W);
    static constexpr int kATile = kTcM * 32 * W;           // bytes of one tail tile
    static constexpr int kBTile = kTcN * 32 * W;           // bytes of one head slice
    static constexpr int kSbo = 256 * W;                   // bytes per 8-row group
};

struct TcItem {
    unsigned long long t0;                 // first tail (colex index among the tails of s)
    int s;                                 // smallest tail element
    int sl0;                               // first head slice (heads sl0 * 256 ...)
    int nsl;                               // head slices in the item
    int nb;                                // heads of s: C(s, q)
    int nt;                                // tails in the item
    int na;                                // tail tiles: ceil(nt / 128); tile a row r = tail t0 + r na + a
    int u;                                 // U when the item was handed out
    int end;                               // 1: the level has no more items
    int ph;                                // phase: heads of q + ph elements
    int F;                                 // packed words in the product (1..W): see TcArgs::words8
};

// Heads of slice sl that belong to s (the MMA N covers them rounded up to 16).
__device__ __forceinline__ int slice_heads(const TcItem &it, int sl) { return min(kTcN, it.nb - sl * kTcN); }

struct TcShared {
    unsigned long long afull[2];           // producers -> MMA: tail set written (2 warp arrivals)
    unsigned long long afree[2];           // MMA -> producers: products reading the set done
    unsigned long long mdone[2];           // MMA -> epilogue: accumulator complete
    unsigned long long tfree[2];           // epilogue -> MMA: accumulator read (8 arrivals)
    unsigned long long bfull[2];           // head slice landed (transaction count)
    unsigned long long bfree[2];           // MMA -> MMA: products reading the slice complete
    unsigned long long ifull[kRing];       // scheduler -> readers
    unsigned long long ifree[kRing];       // readers -> scheduler (11 warp arrivals)
    TcItem ring[kRing];
    unsigned long long cum[2][kMaxN + 1];  // per phase: work items before s
    uint32_t taddr;
    int abort;
    int stop;
};

__host__ __device__ constexpr int align_up(int x, int a) { return (x + a - 1) / a * a; }
constexpr int kHdrBytes = align_up((int)sizeof(TcShared), 1024);

// ------------------------------------------------------------------ PTX wrappers ----
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One try_wait (the hardware may hold the thread for a short, system-defined time).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking: has the phase of parity `parity` completed?
__device__ __forceinline__ bool mbar_poll(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete.  False once the block aborts or the wait
// exceeds kWaitNs (which aborts the block).
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    const uint64_t t0 = gtimer();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            return false;
        }
    }
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    return mbar_test(bar, parity) || mbar_wait_slow(bar, parity, abort_flag);
}

// All lanes of a warp wait; the outcome is made warp-uniform (the warp's later
// .sync.aligned instructions need every lane).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    const bool ok = mbar_wait(bar, parity, abort_flag);
    return __all_sync(0xffffffffu, ok);
}

// The same without the abort flag (draining after an abort), bounded.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    while (!mbar_test(bar, parity) && gtimer() - t0 < kWaitNs) {
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory operand descriptor: K-major, no swizzle; lbo = byte step between core
// matrices along K, sbo = byte step between 8-row groups; bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor, kind::f8f6f4: fp32 accumulator, A and B e4m3, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_e4m3(int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes; the values are valid after a
// tmem_wait that takes them as operands (so no use moves above the wait).
#define MDL_R8(a, i) "=r"(a[i]), "=r"(a[i + 1]), "=r"(a[i + 2]), "=r"(a[i + 3]), "=r"(a[i + 4]), "=r"(a[i + 5]), \
                     "=r"(a[i + 6]), "=r"(a[i + 7])
#define MDL_P8(a, i) "+r"(a[i]), "+r"(a[i + 1]), "+r"(a[i + 2]), "+r"(a[i + 3]), "+r"(a[i + 4]), "+r"(a[i + 5]), \
                     "+r"(a[i + 6]), "+r"(a[i + 7])
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : MDL_R8(v, 0), MDL_R8(v, 8), MDL_R8(v, 16), MDL_R8(v, 24)
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : MDL_P8(v, 0), MDL_P8(v, 8), MDL_P8(v, 16), MDL_P8(v, 24)::"memory");
}
__device__ __forceinline__ void tmem_wait2(uint32_t (&v)[32], uint32_t (&u)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : MDL_P8(v, 0), MDL_P8(v, 8), MDL_P8(v, 16), MDL_P8(v, 24), MDL_P8(u, 0), MDL_P8(u, 8),
                   MDL_P8(u, 16), MDL_P8(u, 24)::"memory");
}
#define MDL_F8(a, i) "=f"(a[i]), "=f"(a[i + 1]), "=f"(a[i + 2]), "=f"(a[i + 3]), "=f"(a[i + 4]), "=f"(a[i + 5]), \
                     "=f"(a[i + 6]), "=f"(a[i + 7])
#define MDL_G8(a, i) "+f"(a[i]), "+f"(a[i + 1]), "+f"(a[i + 2]), "+f"(a[i + 3]), "+f"(a[i + 4]), "+f"(a[i + 5]), \
                     "+f"(a[i + 6]), "+f"(a[i + 7])
// As tmem_ld32, and `red` = the maximum of the 32 values (tcgen05.ld.red, sm_103a).
__device__ __forceinline__ void tmem_ldmax32(uint32_t taddr, float (&v)[32], float &red) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, %32, [%33];"
        : MDL_F8(v, 0), MDL_F8(v, 8), MDL_F8(v, 16), MDL_F8(v, 24), "=f"(red)
        : "r"(taddr));
}
// Wait for two reducing loads; every register they write is an operand, so none is reused
// before the data lands.
__device__ __forceinline__ void tmem_wait_red2(float (&v)[32], float &rv, float (&u)[32], float &ru) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : MDL_G8(v, 0), MDL_G8(v, 8), MDL_G8(v, 16), MDL_G8(v, 24), MDL_G8(u, 0), MDL_G8(u, 8),
                   MDL_G8(u, 16), MDL_G8(u, 24), "+f"(rv), "+f"(ru)::"memory");
}
#undef MDL_F8
#undef MDL_G8
#undef MDL_R8
#undef MDL_P8

// 64 consecutive accumulator columns and their maximum (tcgen05.ld.red, sm_103a)
__device__ __forceinline__ void tmem_ldmax64(uint32_t taddr, float (&v)[64], float &red) {
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x64.max.f32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, %64, [%65];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31]), "=f"(v[32]), "=f"(v[33]), "=f"(v[34]), "=f"(v[35]), "=f"(v[36]), "=f"(v[37]), "=f"(v[38]), "=f"(v[39]), "=f"(v[40]), "=f"(v[41]), "=f"(v[42]), "=f"(v[43]), "=f"(v[44]), "=f"(v[45]), "=f"(v[46]), "=f"(v[47]), "=f"(v[48]), "=f"(v[49]), "=f"(v[50]), "=f"(v[51]), "=f"(v[52]), "=f"(v[53]), "=f"(v[54]), "=f"(v[55]), "=f"(v[56]), "=f"(v[57]), "=f"(v[58]), "=f"(v[59]), "=f"(v[60]), "=f"(v[61]), "=f"(v[62]), "=f"(v[63]), "=f"(red) : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_red64(float (&v)[64], float &r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]), "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]), "+f"(v[22]), "+f"(v[23]), "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]), "+f"(v[29]), "+f"(v[30]), "+f"(v[31]), "+f"(v[32]), "+f"(v[33]), "+f"(v[34]), "+f"(v[35]), "+f"(v[36]), "+f"(v[37]), "+f"(v[38]), "+f"(v[39]), "+f"(v[40]), "+f"(v[41]), "+f"(v[42]), "+f"(v[43]), "+f"(v[44]), "+f"(v[45]), "+f"(v[46]), "+f"(v[47]), "+f"(v[48]), "+f"(v[49]), "+f"(v[50]), "+f"(v[51]), "+f"(v[52]), "+f"(v[53]), "+f"(v[54]), "+f"(v[55]), "+f"(v[56]), "+f"(v[57]), "+f"(v[58]), "+f"(v[59]), "+f"(v[60]), "+f"(v[61]), "+f"(v[62]), "+f"(v[63]), "+f"(r)::"memory");
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Maximum of the first `valid` (all 32 when valid >= 32) accumulator values of a chunk, as a
// shallow tree: four independent chains of three-input maxima.
__device__ __forceinline__ float chunk_max(const uint32_t (&v)[32], int valid) {
    if (valid >= 32) {
        float m[4];
#pragma unroll
        for (int j = 0; j < 4; j++) m[j] = fmaxf(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
#pragma unroll
        for (int i = 8; i < 32; i += 8)
#pragma unroll
            for (int j = 0; j < 4; j++) m[j] = fmax3(m[j], __uint_as_float(v[i + 2 * j]), __uint_as_float(v[i + 2 * j + 1]));
        return fmax3(m[0], m[1], fmaxf(m[2], m[3]));
    }
    float m = -1e30f;
#pragma unroll
    for (int i = 0; i < 32; i++)
        if (i < valid) m = fmaxf(m, __uint_as_float(v[i]));
    return m;
}

// ---------------------------------------------------------------- sign encoding ----
// The 32 sign bytes of packed word x (bit i -> byte i) as two 16-byte vectors: bit 7 of a
// byte is its bit (the product places bit i of a nibble at bit 7 + 8 i -- the partial
// products occupy disjoint bit positions, so there are no carries -- and the mask keeps
// those bits); the rest is `base`: 0x38383838 gives the e4m3 values 0x38 (+1.0) and 0xB8
// (-1.0), 0 only the sign bits (the part that is linear over XOR).
__device__ __forceinline__ void sign_word(uint32_t x, uint32_t base, uint4 &lo, uint4 &hi) {
    auto sb = [&](uint32_t nib) { return ((nib * 0x10204080u) & 0x80808080u) | base; };
    lo = make_uint4(sb(x & 15u), sb((x >> 4) & 15u), sb((x >> 8) & 15u), sb((x >> 12) & 15u));
    hi = make_uint4(sb((x >> 16) & 15u), sb((x >> 20) & 15u), sb((x >> 24) & 15u), sb(x >> 28));
}

// ------------------------------------------------------------------- tail walking ----
struct TcArgs {
    const unsigned char *heads[2];         // per phase: head slices (launch_tc_tables)
    const uint32_t *rows;                  // k x WP packed rows of Gamma_j
    const unsigned long long *binom;       // (k + 1) x (k + 1)
    DevState *st;
    int k, g, q, base, level, WP, tiles, check_stop;   // tiles: tail tiles per set
    int bsub;                              // 1: C(x, i), i <= kMaxV, staged in shared memory
    int smin;                              // phase split (q: no second phase)
    int stall;                             // test hook: the first tile set is never signalled
    // Products over the first F packed words only give the weight of those words, a lower bound
    // of the codeword's weight: byte f-1 = 1 + the largest packed-weight threshold U - base at
    // which f words still reject all but a tiny fraction of codewords (0 = never; the byte of
    // f = W, the exact product, is 255).  An item takes the fewest qualifying words.
    unsigned long long words8;
    const volatile int *cancel;            // non-zero: hand out no more items (null: none)
};

__device__ __forceinline__ unsigned long long C(const TcArgs &a, int n, int r) {
    return (r < 0 || n < r) ? 0ull
                            : __ldg(a.binom + MD_BOUND((size_t)n * (a.k + 1) + r, (size_t)(a.k + 1) * (a.k + 1), kSiteTcBinom));
}

// Largest x in [lo, hi] with C(x, i) <= t (C(lo, i) <= t holds).
__device__ __forceinline__ int colex_digit(const TcArgs &a, int lo, int hi, int i, unsigned long long t) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (C(a, mid, i) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Tail index t (colex among the v-subsets of [s + 1, k)) -> its elements o[0..v), in registers.
// bs: C(x, i) at bs[x * (kMaxV + 1) + i] in shared memory, or null for the global table.
// Each digit (the largest x with C(x, i) <= t) starts from C(x, i) ~ (x - (i-1)/2)^i / i!,
// i.e. x ~ (i! t)^(1/i) + (i-1)/2, and is then corrected with exact comparisons (one or two
// steps instead of a binary search).
__device__ __forceinline__ void tail_unrank(const TcArgs &a, const unsigned long long *bs, int s, int v,
                                            unsigned long long t, int (&o)[kMaxV]) {
    int top = a.k - 2 - s;
    float fact = 1.f;
    for (int i = 2; i <= v; i++) fact *= (float)i;
#pragma unroll
    for (int i = kMaxV; i >= 1; i--) {
        if (i <= v) {
            auto Cb = [&](int x) {
                return bs ? bs[MD_BOUND(x * (kMaxV + 1) + i, (a.k + 1) * (kMaxV + 1), kSiteTcBinom)] : C(a, x, i);
            };
            const int lo = i - 1, hi = top;
            int x;
            if (i == 1) {
                x = (int)min((unsigned long long)hi, t);
            } else {
                const float est = exp2f(__log2f(fmaxf((float)t, 1.f) * fact) / (float)i) + 0.5f * (float)(i - 1);
                x = max(lo, min(hi, (int)est));
                while (x < hi && Cb(x + 1) <= t) x++;
                while (x > lo && Cb(x) > t) x--;
            }
            o[i - 1] = x + s + 1;
            t -= Cb(x);
            top = x - 1;
            fact /= (float)i;
        }
    }
}

// Rank contribution of the tail with index t of phase ph (heads of q = a.q + ph elements):
// C(s, q + 1) + sum_i C(o_i, q + 2 + i).
__device__ __forceinline__ unsigned long long tail_rank_at(const TcArgs &a, int ph, int s, unsigned long long t) {
    const int q = a.q + ph, v = a.g - q - 1;
    int top = a.k - 2 - s;
    unsigned long long r = C(a, s, q + 1);
    for (int i = v; i >= 1; i--) {
        const int x = colex_digit(a, i - 1, top, i, t);
        t -= C(a, x, i);
        top = x - 1;
        r += C(a, x + s + 1, q + 1 + i);
    }
    return r;
}

// Heads of s in phase ph: C(s, q) in phase 0 (s >= s_min), C(min(s, s_min), q + 1) in phase 1.
__device__ __forceinline__ unsigned long long heads_of(const TcArgs &a, int ph, int s) {
    return ph ? C(a, min(s, a.smin), a.q + 1) : C(a, s, a.q);
}

// Items of s in phase ph: groups of up to kGroup head slices x runs of 128 * tiles tails.
__device__ __forceinline__ unsigned long long items_of(const TcArgs &a, int ph, int s) {
    const int q = a.q + ph, v = a.g - q - 1;
    if (v < 0 || s < (ph ? q : max(a.q, a.smin)) || s > a.k - 1 - v) return 0;
    const unsigned long long nb = heads_of(a, ph, s), nt = C(a, a.k - 1 - s, v);
    const unsigned long long per = (unsigned long long)kTcM * a.tiles;
    const unsigned long long nsl = (nb + kTcN - 1) / kTcN;
    return ((nsl + kGroup - 1) / kGroup) * ((nt + per - 1) / per);
}

// S ^= the packed words [w0, w0 + NW) of row x of a word-major table (k rows).
template <int NW>
__device__ __forceinline__ void xor_words(uint32_t (&S)[NW], const uint32_t *tab, int k, int x, int w0, int W) {
#pragma unroll
    for (int i = 0; i < NW; i++)
        if (w0 + i < W) S[i] ^= tab[(w0 + i) * k + MD_BOUND(x, k, kSiteTcTable)];
}

// The epilogue's rare path, for a warp in which some row's maximum reached the threshold
// (pass).  Out of line, so that the epilogue's common path is compiled without it (inlined,
// it cost a quarter of the kernel's throughput).  Returns the warp's best weight so far.
//   * F = W: the product is the exact weight.  The passing rows re-read their columns, take
//     the first one holding the maximum (the tail's smallest rank of that weight) and publish
//     (weight, rank).
//   * F < W: the product covered the first F packed words only, so D >= thrf marks codewords
//     whose weight over those words -- a lower bound of the weight -- can still reach
//     T = min(U, best).  Each such column's exact weight is counted from the rows: the tail
//     sum (its elements by unranking) XOR the head sum (the head's q + ph elements by colex
//     unranking of its index), over all W words.  The lightest one, first in column order,
//     is published if it reaches T.
template <int W>
__device__ __noinline__ int tc_publish(const TcArgs a, const uint32_t *rT, const unsigned long long *bs, uint32_t col0,
                                       int nchunk, int nvh, bool pass, float mx, float thrf, int F, int p0, int ph,
                                       int s, unsigned long long tail, int ubest, int u) {
    const int k = a.k;
    if (F == W) {
        int firstc = 0x7fffffff;
        for (int c = 0; c < nchunk; c++) {
            uint32_t vv[32];
            __syncwarp();
            tmem_ld32(col0 + 32u * c, vv);
            tmem_wait(vv);
#pragma unroll
            for (int i = 0; i < 32; i++) {
                const int col = 32 * c + i;
                if (pass && col < nvh && col < firstc && __uint_as_float(vv[i]) == mx) firstc = col;
            }
        }
        if (pass) {
            const int w = a.base + (32 * W - (int)mx) / 2;
            const unsigned long long rank = (unsigned long long)(p0 + firstc) + tail_rank_at(a, ph, s, tail);
            atomicMin(&a.st->key[a.level], ((unsigned long long)w << kRankBits) | rank);
            atomicMin(&a.st->U, (unsigned int)w);
            ubest = min(ubest, w);
        }
        return ubest;
    }
    const int qq = a.q + ph, v = a.g - qq - 1;
    uint32_t S[W];
#pragma unroll
    for (int w = 0; w < W; w++) S[w] = 0u;
    if (pass) {
        int o[kMaxV];
        tail_unrank(a, bs, s, v, tail, o);
#pragma unroll
        for (int w = 0; w < W; w++) {
            S[w] = rT[w * k + MD_BOUND(s, k, kSiteTcTail)];
            for (int i = 0; i < v; i++) S[w] ^= rT[w * k + MD_BOUND(o[i], k, kSiteTcTail)];
        }
    }
    int bw = 0x7fffffff, bc = -1;
    for (int c = 0; c < nchunk; c++) {
        uint32_t vv[32];
        __syncwarp();
        tmem_ld32(col0 + 32u * c, vv);
        tmem_wait(vv);
        if (!pass) continue;
        for (int i = 0; i < 32; i++) {
            const int col = 32 * c + i;
            if (col >= nvh || __uint_as_float(vv[i]) < thrf) continue;
            uint32_t H[W];
#pragma unroll
            for (int w = 0; w < W; w++) H[w] = S[w];
            unsigned long long t = (unsigned long long)(p0 + col);
            int hi = s - 1;                                  // the heads of s lie below s
            for (int e = qq; e >= 1; e--) {
                const int x = colex_digit(a, e - 1, hi, e, t);
                t -= C(a, x, e);
                hi = x - 1;
#pragma unroll
                for (int w = 0; w < W; w++) H[w] ^= rT[w * k + MD_BOUND(x, k, kSiteTcHead)];
            }
            int wt = a.base;
#pragma unroll
            for (int w = 0; w < W; w++) wt += __popc(H[w]);
            if (wt < bw) { bw = wt; bc = col; }
        }
    }
    if (pass && bc >= 0 && bw <= min(u, ubest)) {
        const unsigned long long rank = (unsigned long long)(p0 + bc) + tail_rank_at(a, ph, s, tail);
        atomicMin(&a.st->key[a.level], ((unsigned long long)bw << kRankBits) | rank);
        atomicMin(&a.st->U, (unsigned int)bw);
        ubest = min(ubest, bw);
    }
    return ubest;
}

// ------------------------------------------------------------------------ kernel ----
template <int W>
__global__ void __maxnreg__(kTcMaxRegs) tc_kernel(const TcArgs a) {
    using Cfg = TcCfg<W>;
    constexpr int T = Cfg::kTiles;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared &sh = *reinterpret_cast<TcShared *>(smem);
    // word-major tables: rT[w * k + x] = word w of row x, dT[w * k + x] = that of row x ^ row x+1,
    // pX[w * (k + 1) + x] = that of row 0 ^ ... ^ row x-1
    uint32_t *rT = reinterpret_cast<uint32_t *>(smem + kHdrBytes);
    uint32_t *dT = rT + W * a.k;
    uint32_t *pX = dT + W * a.k;
    unsigned char *Atile = smem + kHdrBytes + align_up((3 * a.k + 1) * W * 4, 1024);   // [2][T] tiles
    unsigned char *Btile = Atile + 2 * T * Cfg::kATile;                                // [2] slices
    unsigned long long *bsub = a.bsub ? reinterpret_cast<unsigned long long *>(Btile + 2 * Cfg::kBTile) : nullptr;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DevState *st = a.st;
    const int k = a.k;
    volatile int *abort_flag = &sh.abort;

    if (threadIdx.x == 0) {
        sh.abort = 0;
        sh.stop = a.check_stop ? *(volatile int *)&st->stop : 0;
        for (int i = 0; i < 2; i++) {
            mbar_init(saddr(&sh.afull[i]), kProdWarps);
            mbar_init(saddr(&sh.afree[i]), kMmaWarps);
            mbar_init(saddr(&sh.mdone[i]), 1);
            mbar_init(saddr(&sh.tfree[i]), kEpiWarps);
            mbar_init(saddr(&sh.bfull[i]), 1);
            mbar_init(saddr(&sh.bfree[i]), kMmaWarps);
        }
        for (int i = 0; i < kRing; i++) {
            mbar_init(saddr(&sh.ifull[i]), 1);
            mbar_init(saddr(&sh.ifree[i]), kItemReaders);
        }
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < k * W; i += blockDim.x) {
        const int w = i / k, x = i % k;
        const uint32_t y = __ldg(a.rows + x * a.WP + w);
        rT[i] = y;
        dT[i] = x + 1 < k ? y ^ __ldg(a.rows + (x + 1) * a.WP + w) : 0u;
    }
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        uint32_t acc = 0;
        for (int x = 0; x <= k; x++) {
            pX[w * (k + 1) + x] = acc;
            if (x < k) acc ^= __ldg(a.rows + x * a.WP + w);
        }
    }
    for (int i = threadIdx.x; i < 2 * k; i += blockDim.x) sh.cum[i / k][i % k + 1] = items_of(a, i / k, i % k);
    if (bsub)
        for (int i = threadIdx.x; i < (k + 1) * (kMaxV + 1); i += blockDim.x)
            bsub[i] = C(a, i / (kMaxV + 1), i % (kMaxV + 1));
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ph = 0; ph < 2; ph++) {
            sh.cum[ph][0] = 0;
            for (int s = 0; s < k; s++) sh.cum[ph][s + 1] += sh.cum[ph][s];
        }
    }
    __syncthreads();
    if (sh.stop) return;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&sh.taddr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = sh.taddr;

    if (warp == kSchedWarp) {
        // ------------------------------------------------------------ scheduler ----
        if (lane == 0) {
            const unsigned long long total0 = sh.cum[0][k], total = total0 + sh.cum[1][k];
            const unsigned long long per = (unsigned long long)kTcM * T;
            for (long long n = 0;; n++) {
                const int slot = (int)(n % kRing);
                const unsigned use = (unsigned)(n / kRing);
                if (use >= 1 && !mbar_wait(saddr(&sh.ifree[slot]), (use - 1) & 1, abort_flag)) break;
                TcItem it{};
                for (;;) {
                    if (a.cancel && *a.cancel) {                // the caller cancelled the run
                        atomicExch(&st->error, MD_ECANCELED);
                        atomicExch(&st->stop, 1);
                        it.end = 1;
                        break;
                    }
                    unsigned long long idx = atomicAdd(&st->ctr[a.level], 1ull);
                    if (idx >= total) { it.end = 1; break; }
                    const int ph = idx >= total0 ? 1 : 0;
                    if (ph) idx -= total0;
                    const unsigned long long *cum = sh.cum[ph];
                    int lo = 0, hi = k - 1;                    // last s with cum[s] <= idx
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (cum[mid] <= idx) lo = mid; else hi = mid - 1;
                    }
                    const int s = lo;
                    const unsigned long long local = idx - cum[s];
                    const unsigned long long nb = heads_of(a, ph, s);
                    const unsigned long long nsl = (nb + kTcN - 1) / kTcN;
                    // consecutive items share a group of head slices and take successive runs
                    // of tails: the blocks working at once read the same slices, which then stay
                    // in L2 even when the whole head table does not fit there
                    const unsigned long long ntails = C(a, k - 1 - s, a.g - a.q - ph - 1);
                    const unsigned long long ntb = (ntails + per - 1) / per;
                    const unsigned long long tblock = local % ntb, grp = local / ntb;
                    it.s = s;
                    it.ph = ph;
                    it.nb = (int)nb;
                    it.sl0 = (int)(grp * kGroup);
                    it.nsl = (int)min((unsigned long long)kGroup, nsl - grp * kGroup);
                    it.t0 = tblock * per;
                    it.nt = (int)min(per, ntails - it.t0);
                    it.na = (it.nt + kTcM - 1) / kTcM;
                    const int U = (int)*(volatile unsigned int *)&st->U;
                    it.u = U;
                    it.F = W;
                    for (int f = 1; f < W; f++)
                        if ((int)((a.words8 >> (8 * (f - 1))) & 255ull) > U - a.base) { it.F = f; break; }
                    // mid-level stop: once U <= L this level holds the answer's weight, and an
                    // item whose smallest rank lies above the best rank of that weight can go
                    if (a.check_stop && U <= *(volatile int *)&st->L) {
                        const unsigned long long key = *(volatile unsigned long long *)&st->key[a.level];
                        if (key != kNoKey && (int)(key >> kRankBits) == U &&
                            (unsigned long long)it.sl0 * kTcN + tail_rank_at(a, ph, s, it.t0) > (key & (kRankLimit - 1))) {
                            atomicAdd(&st->skipped, 1ull);
                            continue;
                        }
                    }
                    break;
                }
                sh.ring[slot] = it;
                mbar_arrive(saddr(&sh.ifull[slot]));
                if (it.end) break;
            }
        }
    } else if (warp >= kMmaWarp0 && warp < kMmaWarp0 + kMmaWarps) {
        // ------------------------------------------------- MMA issue and head slices ----
        // Two issuers walk the same items and slices; issuer `me` multiplies the tiles u with
        // u % 2 == me into accumulator me.  A product of K = 32 W is a chain of W dependent
        // MMAs; from two threads the tensor pipe interleaves the chains of both accumulators
        // and hides the latency between the MMAs of a chain.  Issuer 0 also fetches the head
        // slices; both release a slice buffer and a tail set (barriers of two arrivals).
        if (lane == 0) {
            const int me = warp - kMmaWarp0;
            long long n = 0;                               // ring entries taken
            bool ok = true;
            auto take = [&](TcItem &it) -> bool {
                const int slot = (int)(n % kRing);
                if (!mbar_wait(saddr(&sh.ifull[slot]), (unsigned)(n / kRing) & 1, abort_flag)) return false;
                it = sh.ring[slot];
                mbar_arrive(saddr(&sh.ifree[slot]));
                n++;
                return true;
            };
            int pend_buf = -1;                             // head slice copy not yet waited for
            unsigned pend_parity = 0;
            auto load_slice = [&](const TcItem &it, int sl, long long step) {
                const int buf = (int)(step & 1);
                const int npad = (slice_heads(it, sl) + 15) & ~15;
                const uint32_t bytes = (uint32_t)(npad / 8) * Cfg::kSbo;
#ifdef MD_DEBUG_BOUNDS
                // the table of phase ph holds C(k, q) (ph 0) or C(s_min, q + 1) (ph 1) heads in 256-row slices
                const unsigned long long nslices = ((it.ph ? C(a, a.smin, a.q + 1) : C(a, k, a.q)) + kTcN - 1) / kTcN;
#endif
                const unsigned char *src = a.heads[it.ph] + (size_t)MD_BOUND(sl, nslices, kSiteTcSlice) * Cfg::kBTile;
                mbar_expect_tx(saddr(&sh.bfull[buf]), bytes);
                bulk_g2s(saddr(Btile + buf * Cfg::kBTile), src, bytes, saddr(&sh.bfull[buf]));
                pend_buf = buf;
                pend_parity = (unsigned)(step >> 1) & 1;
            };
            TcItem cur{}, nxt{};
            unsigned u = 0;                                // accumulator uses
            long long step = 0;                            // head slices multiplied
            long long j = 0;                               // items
            int last_acc = -1;
            unsigned last_parity = 0;
            ok = take(cur);
            if (ok && !cur.end && me == 0) load_slice(cur, cur.sl0, 0);
            while (ok && !cur.end) {
                const int set = (int)(j & 1);
                if (!mbar_wait(saddr(&sh.afull[set]), (unsigned)(j >> 1) & 1, abort_flag)) { ok = false; break; }
                nxt.end = 1;
                for (int sl = 0; sl < cur.nsl && ok; sl++, step++) {
                    const int bb = (int)(step & 1);
                    if (!mbar_wait(saddr(&sh.bfull[bb]), (unsigned)(step >> 1) & 1, abort_flag)) { ok = false; break; }
                    if (pend_buf == bb) pend_buf = -1;
                    const uint32_t idesc = idesc_e4m3((slice_heads(cur, cur.sl0 + sl) + 15) & ~15);
                    const uint32_t bbase = saddr(Btile + bb * Cfg::kBTile);
                    // the next slice (of this item or the next) goes into the other buffer as
                    // soon as the products of the slice before this one are done with it
                    const TcItem *ni = &cur;
                    int nsl_idx = cur.sl0 + sl + 1;
                    if (sl + 1 == cur.nsl) {
                        if (!take(nxt)) { ok = false; break; }
                        ni = &nxt;
                        nsl_idx = nxt.sl0;
                    }
                    bool fetched = ni->end != 0 || me != 0;
                    const uint32_t prev_free = saddr(&sh.bfree[(step + 1) & 1]);
                    const unsigned prev_parity = (unsigned)((step - 1) >> 1) & 1;
                    for (int t = 0; t < cur.na; t++, u++) {
                        const int acc = (int)(u & 1);
                        if (acc != me) continue;
                        // descriptors before the wait: the step of 32 K bytes (256 B of core
                        // matrices) adds 256 >> 4 to the start-address field
                        const uint64_t adesc = smem_desc(saddr(Atile + (set * T + t) * Cfg::kATile), 128u, Cfg::kSbo);
                        const uint64_t bdesc = smem_desc(bbase, 128u, Cfg::kSbo);
                        const uint32_t d = tmem + (uint32_t)(acc * kTcN);
                        if (u >= 2 && !mbar_wait(saddr(&sh.tfree[acc]), ((u >> 1) - 1) & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_after();
#pragma unroll
                        for (int w = 0; w < W; w++)
                            if (w < cur.F)
                                mma_e4m3(d, adesc + (uint64_t)(16 * w), bdesc + (uint64_t)(16 * w), idesc, w > 0 ? 1u : 0u);
                        mma_commit(saddr(&sh.mdone[acc]));
                        last_acc = acc;
                        last_parity = (u >> 1) & 1;
                        if (!fetched && (step == 0 || mbar_poll(prev_free, prev_parity))) {
                            load_slice(*ni, nsl_idx, step + 1);
                            fetched = true;
                        }
                    }
                    if (!ok) break;
                    mma_commit(saddr(&sh.bfree[bb]));
                    if (!fetched) {
                        if (step >= 1 && !mbar_wait(prev_free, prev_parity, abort_flag)) {
                            ok = false;
                            break;
                        }
                        load_slice(*ni, nsl_idx, step + 1);
                    }
                }
                if (!ok) break;
                mma_commit(saddr(&sh.afree[set]));
                cur = nxt;
                j++;
            }
            if (!ok) {
                if (last_acc >= 0) mbar_drain(saddr(&sh.mdone[last_acc]), last_parity);
                if (pend_buf >= 0) mbar_drain(saddr(&sh.bfull[pend_buf]), pend_parity);
            }
        }
    } else if (warp >= kProdWarp0) {
        // ------------------------------------------------------------ producers ----
        constexpr int NW = W;
        const int w0 = 0;
        long long n = 0, j = 0;
        int o[kMaxV];                                      // upper elements of the current tail
#pragma unroll
        for (int i = 0; i < kMaxV; i++) o[i] = 0;
        uint32_t Sx[NW];                                   // the tail sum
        for (;;) {
            const int slot = (int)(n % kRing);
            if (!warp_wait(saddr(&sh.ifull[slot]), (unsigned)(n / kRing) & 1, abort_flag)) break;
            const TcItem it = sh.ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&sh.ifree[slot]));
            n++;
            if (it.end) break;
            const int set = (int)(j & 1);
            const int v = a.g - a.q - it.ph - 1;               // upper elements of this item's tails
            {
                // thread p walks tails [R na p, R na p + R na), R = kProdRows rows per thread:
                // the first na go to tile row p (tile t of each), the next na to row
                // p + 128 / R, and so on
                const int p = (warp - kProdWarp0) * 32 + lane;
                const int first = kProdRows * it.na * p;
                const int cnt = max(0, min(kProdRows * it.na, it.nt - first));
                // the first tail needs no tile memory: it is found while the set is still in use
#pragma unroll
                for (int i = 0; i < NW; i++) Sx[i] = 0;
                if (cnt > 0) {
                    tail_unrank(a, bsub, it.s, v, it.t0 + (unsigned long long)first, o);
                    xor_words<NW>(Sx, rT, k, it.s, w0, W);
#pragma unroll
                    for (int i = 0; i < kMaxV; i++)
                        if (i < v) xor_words<NW>(Sx, rT, k, o[i], w0, W);
                }
                if (j >= 2 && !warp_wait(saddr(&sh.afree[set]), (unsigned)((j >> 1) - 1) & 1, abort_flag)) break;
                for (int m = 0; m < kProdRows * it.na; m++) {
                    const int r = p + (kTcM / kProdRows) * (m / it.na);
                    const int t = m % it.na;
                    unsigned char *rowp =
                        Atile + MD_BOUND((set * T + t) * Cfg::kATile + (r >> 3) * Cfg::kSbo + (r & 7) * 16,
                                         2 * T * Cfg::kATile - (W - 1) * 256 - 143, kSiteTcTile);
                    const bool valid = m < cnt;
#pragma unroll
                    for (int i = 0; i < NW; i++) {
                        if (i >= it.F) continue;               // the item's products read F words
                        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
                        if (valid) sign_word(Sx[i], 0x38383838u, lo, hi);
                        *reinterpret_cast<uint4 *>(rowp + i * 256) = lo;
                        *reinterpret_cast<uint4 *>(rowp + i * 256 + 128) = hi;
                    }
                    // colex successor of the upper elements o[0..v) within (s, k): the lowest
                    // element that can move up moves; those below it restart at s + 1, s + 2, ...
                    const bool stepv = m + 1 < cnt;
                    const int o0 = o[0];
                    const int o1 = v >= 2 ? o[1] : k;
                    if (!__any_sync(kFull, stepv && o0 + 1 == o1)) {
                        if (stepv) {
                            xor_words<NW>(Sx, dT, k, o0, w0, W);
                            o[0] = o0 + 1;
                        }
                    } else if (stepv) {
                        // o[0..m] = o0, o0 + 1, ..., o0 + m and o[m] can move up
                        unsigned stop = 1u << (v - 1);
#pragma unroll
                        for (int i = 0; i < kMaxV - 1; i++)
                            if (i < v - 1 && o[i] + 1 != o[i + 1]) stop |= 1u << i;
                        const int mm = __ffs(stop) - 1;
                        const int sp = it.s + 1;
                        xor_words<NW>(Sx, pX, k + 1, o0, w0, W);
                        xor_words<NW>(Sx, pX, k + 1, o0 + mm + 1, w0, W);
                        xor_words<NW>(Sx, pX, k + 1, sp, w0, W);
                        xor_words<NW>(Sx, pX, k + 1, sp + mm, w0, W);
                        xor_words<NW>(Sx, rT, k, o0 + mm + 1, w0, W);
#pragma unroll
                        for (int i = 0; i < kMaxV; i++) o[i] = i < mm ? sp + i : (i == mm ? o[i] + 1 : o[i]);
                    }
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0 && !(a.stall && j == 0)) mbar_arrive(saddr(&sh.afull[set]));
            j++;
        }
    } else {
        // ------------------------------------------------------------- epilogue ----
        const int quarter = warp;
        const int r = quarter * 32 + lane;                 // tensor-memory lane = tile row
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        long long n = 0;
        unsigned u = 0;
        bool ok = true;
        int ubest = 0x7fffffff;
        while (ok) {
            const int slot = (int)(n % kRing);
            if (!warp_wait(saddr(&sh.ifull[slot]), (unsigned)(n / kRing) & 1, abort_flag)) break;
            const TcItem it = sh.ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&sh.ifree[slot]));
            n++;
            if (it.end) break;
            // the least accumulator value that can reach min(U, best): D >= K - 2 (min(U, best) -
            // base) with K = 32 F the product's bits (its weight is that of the first F words, a
            // lower bound when F < W); with a negative margin no row passes, since D <= K
            float thrf = (float)(32 * it.F - 2 * (min(it.u, ubest) - a.base));
            for (int sl = 0; sl < it.nsl && ok; sl++) {
                const int p0 = (it.sl0 + sl) * kTcN;
                const int nvh = slice_heads(it, it.sl0 + sl);                                   // columns here
                const int nchunk = (nvh + 31) >> 5;
                for (int t = 0; t < it.na; t++) {
                    const int acc = (int)(u & 1);
                    if (!warp_wait(saddr(&sh.mdone[acc]), (u >> 1) & 1, abort_flag)) { ok = false; break; }
                    tc_after();
                    const uint32_t col0 = lane_base + (uint32_t)(acc * kTcN);
                    float mx = -1e30f;
                    if (nvh == kTcN) {
                        // all eight chunks whole: two round trips of two 64-column loads
#pragma unroll 1
                        for (int h = 0; h < 2; h++) {
                            float v0[64], v1[64], r0, r1;
                            tmem_ldmax64(col0 + 128u * h, v0, r0);
                            tmem_ldmax64(col0 + 128u * h + 64u, v1, r1);
                            tmem_wait_red64(v0, r0);
                            tmem_wait_red64(v1, r1);
                            mx = fmax3(r0, r1, mx);
                        }
                    } else
                    for (int c = 0; c < nchunk; c += 2) {
                        const bool two = c + 1 < nchunk;
                        if (32 * (c + 2) <= nvh || (!two && 32 * (c + 1) <= nvh)) {
                            // whole chunks: the load returns each row's maximum
                            float va[32], vb[32], ra = -1e30f, rb = -1e30f;
                            tmem_ldmax32(col0 + 32u * c, va, ra);
                            if (two) tmem_ldmax32(col0 + 32u * (c + 1), vb, rb);
                            tmem_wait_red2(va, ra, vb, rb);
                            mx = fmax3(mx, ra, rb);
                        } else {
                            // a chunk holding columns past the slice's heads: mask them
                            uint32_t va[32], vb[32];
#pragma unroll
                            for (int i = 0; i < 32; i++) vb[i] = 0xff800000u;    // -inf where no second chunk
                            tmem_ld32(col0 + 32u * c, va);
                            if (two) tmem_ld32(col0 + 32u * (c + 1), vb);
                            tmem_wait2(va, vb);
                            mx = fmax3(mx, chunk_max(va, nvh - 32 * c), chunk_max(vb, two ? nvh - 32 * (c + 1) : 32));
                        }
                    }
                    // tail index within the item: row r of tile t is tail R na (r mod 128 / R) +
                    // na (r div 128 / R) + t, R = kProdRows (na r + t with one row per thread)
                    const int row = kProdRows * it.na * (r % (kTcM / kProdRows)) + it.na * (r / (kTcM / kProdRows)) + t;
                    const bool pass = mx >= thrf && row < it.nt;
                    tc_before();
                    // the vote also synchronises the warp before lane 0 releases the accumulator
                    // (each lane's loads are complete at its wait)
                    if (__any_sync(kFull, pass)) {
                        tc_after();
                        ubest = tc_publish<W>(a, rT, bsub, col0, nchunk, nvh, pass, mx, thrf, it.F, p0, it.ph,
                                              it.s, it.t0 + (unsigned long long)row, ubest, it.u);
                        thrf = (float)(32 * it.F - 2 * (min(it.u, ubest) - a.base));
                        tc_before();
                        __syncwarp();
                    }
                    if (lane == 0) mbar_arrive(saddr(&sh.tfree[acc]));
                    u++;
                }
            }
        }
    }

    if (sh.abort && threadIdx.x == 0) {
        // a wait ran out: record it and stop the run (the levels after this one return at once)
        atomicExch(&st->error, MD_ETIMEOUT);
        atomicExch(&st->stop, 1);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Head table of one matrix, one thread per (head, packed word): row p < C(k, q) = e4m3 signs
// of the sum of the rows of the p-th q-subset in colex order (rows up to the next multiple of
// 256 are zero); slice p / 256 starts at byte (p / 256) * 256 * 32 W, in the core-matrix
// layout of the tail tiles.
__global__ void tc_heads_kernel(const uint32_t *rows, const unsigned long long *binom, int k, int q, int W, int WP,
                                unsigned long long nheads, unsigned long long nrows, unsigned char *heads) {
    for (unsigned long long idx = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; idx < nrows * W;
         idx += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long p = idx / W;
        const int w = (int)(idx % W);
        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
        if (p < nheads) {
            uint32_t x = 0;
            unsigned long long t = p;
            int top = k - 1;
            for (int i = q; i >= 1; i--) {
                int l = i - 1, h = top;
                while (l < h) {
                    const int mid = (l + h + 1) >> 1;
                    if (binom[(size_t)mid * (k + 1) + i] <= t) l = mid; else h = mid - 1;
                }
                x ^= rows[l * WP + w];
                t -= binom[(size_t)l * (k + 1) + i];
                top = l - 1;
            }
            sign_word(x, 0x38383838u, lo, hi);
        }
        const unsigned long long slice = p / kTcN;
        const int rr = (int)(p % kTcN);
        unsigned char *row = heads + slice * (unsigned long long)(kTcN * 32 * W) + (rr >> 3) * (256 * W) + (rr & 7) * 16;
        *reinterpret_cast<uint4 *>(row + (2 * w) * 128) = lo;
        *reinterpret_cast<uint4 *>(row + (2 * w + 1) * 128) = hi;
    }
}

// Tensor-pipe probe: threads 0 and 32 (warps 0 and 1) each issue `iters` e4m3 MMAs (M = 128,
// N = 256, K = 32) back to back into an accumulator of their own, as the level kernel's two
// issuers do; operands are +-1 tiles in shared memory in the level kernel's layout.  cyc[b] =
// block b's clock64 cycles from the first issue to the completion of both chains; err = 1 if a
// chain did not complete within the time bound (the block then still waits for it, bounded,
// before freeing its tensor memory).  The dynamic shared memory asked for keeps one block per SM.
constexpr int kProbeThreads = 64;
__global__ void __launch_bounds__(kProbeThreads) mma_probe_kernel(unsigned iters, unsigned long long *cyc, int *err) {
    extern __shared__ __align__(1024) unsigned char probe_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(((uintptr_t)probe_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) unsigned long long done[2];
    __shared__ uint32_t taddr;
    __shared__ unsigned long long t0s[2], t1s[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kBytes = (kTcM + kTcN) * 32;           // one tail tile and one head slice, W = 1
    for (int i = threadIdx.x; i < kBytes / 4; i += blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B9u;
        h ^= h >> 15;
        uint32_t v = 0;
        for (int b = 0; b < 4; b++) v |= (((h >> b) & 1u) ? 0xB8u : 0x38u) << (8 * b);
        reinterpret_cast<uint32_t *>(tiles)[i] = v;
    }
    if (threadIdx.x == 0) {
        mbar_init(saddr(&done[0]), 1);
        mbar_init(saddr(&done[1]), 1);
        fence_mbar_init();
    }
    fence_async_smem();                                  // the tiles, for the tensor core's reads
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&taddr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = taddr;
    if (lane == 0) {
        const int me = warp;
        const uint64_t adesc = smem_desc(saddr(tiles), 128u, 256u);
        const uint64_t bdesc = smem_desc(saddr(tiles + kTcM * 32), 128u, 256u);
        const uint32_t idesc = idesc_e4m3(kTcN);
        const uint32_t d = tmem + (uint32_t)(me * kTcN);
        const unsigned long long t0 = clock64();
        for (unsigned i = 0; i < iters; i++) mma_e4m3(d, adesc, bdesc, idesc, i > 0 ? 1u : 0u);
        mma_commit(saddr(&done[me]));
        const uint64_t g0 = gtimer();
        bool ok = true;
        while (!mbar_test(saddr(&done[me]), 0))
            if (gtimer() - g0 > kWaitNs) { ok = false; break; }
        t0s[me] = t0;
        t1s[me] = clock64();
        if (!ok) {
            atomicExch(err, 1);
            mbar_drain(saddr(&done[me]), 0);
        }
    }
    tc_before();
    __syncthreads();
    if (threadIdx.x == 0) cyc[blockIdx.x] = max(t1s[0], t1s[1]) - min(t0s[0], t0s[1]);
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

template <int W>
cudaError_t launch_tc_w(const TcArgs &a, int blocks, size_t smem, cudaStream_t s) {
    auto kern = tc_kernel<W>;
    const cudaError_t e = (cudaError_t)allow_full_smem((const void *)kern);
    if (e != cudaSuccess) return e;
    kern<<<blocks, kTcThreads, smem, s>>>(a);
    return cudaGetLastError();
}

size_t head_bytes(int k, int q, int W) {
    const uint64_t nheads = binom(k, q);
    const uint64_t slices = (nheads + kTcN - 1) / kTcN;
    return (size_t)slices * kTcN * 32 * W;
}

}  // namespace

size_t tc_tables_bytes(int k, int q, int W) { return head_bytes(k, q, W); }

MD_BOUNDS_ACCESSOR(bounds_site_tc)

size_t tc_heads_bytes(uint64_t nheads, int W) { return (size_t)((nheads + kTcN - 1) / kTcN) * kTcN * 32 * W; }

#ifndef MD_TC_HEAD_TABLE_MAX
#define MD_TC_HEAD_TABLE_MAX (size_t(1) << 30)
#endif
int tc_auto_head(int k, int W) {
    // The head dimension of a product is C(s, q) for the tail's smallest element s, and s is
    // small for most combinations when g is a sizeable fraction of k (about q k / g): wider heads
    // give each tail tile more slices to be multiplied with.  The widest of 5, 4, 3 elements
    // whose table fits in 1 GiB (k = 100: q = 4, 1.05x over q = 3 on stage 10; k = 56..64:
    // q = 5, 1.4-2.2x on stages 11-13), pairs beyond.
    for (int q = 5; q >= 3; q--)
        if (k > q + 1 && head_bytes(k, q, W) <= MD_TC_HEAD_TABLE_MAX) return q;
    return 2;
}

int tc_max_upper() { return kMaxV; }

// Shared memory without / with the binomial sub-table of the producers.
int tc_smem_base(int k, int W) {
    return 1024 + kHdrBytes + align_up((3 * k + 1) * W * 4, 1024) + 2 * tc_tiles_per_set(W) * kTcM * 32 * W +
           2 * kTcN * 32 * W;
}
int tc_bsub_bytes(int k) { return (k + 1) * (kMaxV + 1) * 8; }

// Dynamic shared memory of a launch, with the binomial sub-table when it fits in `optin`;
// at least 116 KB, so that one block (holding all 512 tensor-memory columns) runs per SM.
int tc_smem_bytes(int k, int W, int optin, int *with_bsub) {
    int bytes = tc_smem_base(k, W);
    *with_bsub = bytes + tc_bsub_bytes(k) <= optin ? 1 : 0;
    if (*with_bsub) bytes += tc_bsub_bytes(k);
    return bytes < 116 * 1024 ? 116 * 1024 : bytes;
}

int tc_split_point(int k, int q) {
    // the smallest s whose q-heads fill seven slices: below it, tails of q-heads would serve
    // too few heads, and the second phase's (q+1)-heads take over
    int s = q;
    while (s < k && binom(s, q) < 7ull * kTcN) s++;
    return s;
}

uint64_t tc_level_items(int k, int g, int q, int smin, int W) {
    uint64_t total = 0;
    const uint64_t per = (uint64_t)kTcM * tc_tiles_per_set(W);
    for (int ph = 0; ph < 2; ph++) {
        const int qq = q + ph, v = g - qq - 1;
        if (v < 0) continue;
        for (int s = ph ? qq : std::max(q, smin); s <= k - 1 - v; s++) {
            const uint64_t nb = ph ? binom(std::min(s, smin), qq) : binom(s, qq), nt = binom(k - 1 - s, v);
            const uint64_t nsl = (nb + kTcN - 1) / kTcN;
            total += ((nsl + kGroup - 1) / kGroup) * ((nt + per - 1) / per);
        }
    }
    return total;
}

int launch_tc_tables(const uint32_t *rows, const unsigned long long *binom_d, int k, int q, int W, int WP,
                     uint64_t nheads, unsigned char *tables, void *stream) {
    const uint64_t nrows = (nheads + kTcN - 1) / kTcN * kTcN;
    if (nrows == 0) return 0;
    const uint64_t total = nrows * (uint64_t)W;
    const int blocks = (int)std::min<uint64_t>((total + 255) / 256, 8192);
    tc_heads_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(rows, binom_d, k, q, W, WP, nheads, nrows, tables);
    return (int)cudaGetLastError();
}

int launch_tc_level(const unsigned char *tables, const unsigned char *tables2, int smin, const uint32_t *rows,
                    const unsigned long long *binom_d, DevState *st, int k, int g, int q, int base, int level, int W,
                    int WP, int check_stop, int blocks, int stall, unsigned long long words8,
                    const volatile int *cancel, void *stream) {
    int dev = 0, optin = 0, with_bsub = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return (int)cudaErrorInvalidValue;
    const size_t smem = (size_t)tc_smem_bytes(k, W, optin, &with_bsub);
    TcArgs a{{tables, tables2}, rows, binom_d, st, k, g, q, base, level, WP, tc_tiles_per_set(W), check_stop,
             with_bsub, smin, stall, words8, cancel};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (W) {
        case 1: e = launch_tc_w<1>(a, blocks, smem, s); break;
        case 2: e = launch_tc_w<2>(a, blocks, smem, s); break;
        case 3: e = launch_tc_w<3>(a, blocks, smem, s); break;
        case 4: e = launch_tc_w<4>(a, blocks, smem, s); break;
        case 5: e = launch_tc_w<5>(a, blocks, smem, s); break;
        case 6: e = launch_tc_w<6>(a, blocks, smem, s); break;
        case 7: e = launch_tc_w<7>(a, blocks, smem, s); break;
        case 8: e = launch_tc_w<8>(a, blocks, smem, s); break;
        default: return (int)cudaErrorInvalidValue;
    }
    return (int)e;
}

}  // namespace mdl

// Dense e4m3 flops per SM per clock of the tensor pipe, measured (median over one block per SM).
extern "C" int md_mma_rate(double *flops_per_sm_per_clk) {
    using namespace mdl;
    if (!flops_per_sm_per_clk) return MD_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    const int smem = 150 * 1024;                        // more than half an SM's shared memory
    unsigned long long *cyc = nullptr;
    int *err = nullptr;
    if (cudaFuncSetAttribute(mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(unsigned long long) * sms) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (cyc) cudaFree(cyc);
        return MD_ECUDA;
    }
    const unsigned iters = 1u << 13;
    int herr = 0;
    bool ok = cudaMemset(err, 0, sizeof(int)) == cudaSuccess;
    if (ok) {
        mma_probe_kernel<<<sms, kProbeThreads, smem>>>(256u, cyc, err);          // warm-up
        mma_probe_kernel<<<sms, kProbeThreads, smem>>>(iters, cyc, err);
    }
    std::vector<unsigned long long> h(sms);
    ok = ok && cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
         cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost) == cudaSuccess &&
         cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(cyc);
    cudaFree(err);
    if (!ok) { cudaGetLastError(); return MD_ECUDA; }
    if (herr) return MD_ETIMEOUT;
    std::sort(h.begin(), h.end());
    const double med = (double)h[h.size() / 2];
    if (med <= 0) return MD_EINTERNAL;
    *flops_per_sm_per_clk = 2.0 * iters * (2.0 * kTcM * kTcN * 32) / med;
    return MD_OK;
}
