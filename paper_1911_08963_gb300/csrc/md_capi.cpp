// md_capi.cpp -- the C ABI (include/md.h): handles, device buffers and the stage loop of
// Alg. 1 (Brouwer-Zimmermann).  Every level (g, j) is one kernel launch followed by a
// one-thread finalize kernel that compares the bounds on the device, so consecutive
// levels are queued back to back without host round trips; the host only looks at the
// stop flag one stage behind the device.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "md_internal.h"

using namespace mdl;

namespace {

constexpr int kDefaultThreads = 512;

struct DevLayout {
    char *base = nullptr;
    size_t bytes = 0;
    std::vector<uint32_t *> rows, h2;
    std::vector<unsigned char *> heads;     // tensor-core head tables per matrix (null: none)
    std::vector<unsigned char *> heads2;    // second-phase (q+1)-head tables
    std::vector<int> tc_smin;
    unsigned long long *binom = nullptr;
    MEntry *mtab = nullptr;
    DevState *st = nullptr;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct md_ctx {
    Code code;
    md_options opt{};
    bool dev_ready = false;
    int device = -1;
    cudaStream_t own_stream = nullptr;
    DevLayout dev;
    std::vector<LevelPlan> plans;           // level index = (g - 1) * m + j
    std::vector<size_t> mtab_offset;        // per level, entries into dev.mtab
    int g_limit = 0;                        // deepest stage that can be planned
    DevState *host_state = nullptr;         // pinned copy of the device state
    struct Head { unsigned int U; int L, stop, error, last_level; };
    Head *heads = nullptr;                  // pinned, one per stage: the stop flag a stage behind
    std::vector<cudaEvent_t> lev_ev;        // timing events, two per level
    std::vector<cudaEvent_t> stage_ev;      // one per stage
    cudaEvent_t run_ev[2] = {nullptr, nullptr};
    md_info info{};
    std::vector<md_level> levels;
    int threads = kDefaultThreads;
    int sms = 0;
    int smem_optin = 0;
    int setup_launches = 0;                 // device setup work charged to the next compute
    uint64_t setup_h2d = 0;
    volatile int *cancel_host = nullptr;    // mapped pinned word the kernels poll per work item
    const volatile int *cancel_dev = nullptr;
    bool have_state = false;                // host_state holds the end of the last md_compute
    std::vector<char> resume;               // a checkpoint armed for the next md_compute
};

namespace {

cudaStream_t stream_of(md_ctx *h) {
    return h->opt.stream ? (cudaStream_t)h->opt.stream : h->own_stream;
}

// Device memory through the caller's allocator (md_options.dev_alloc), else cudaMalloc.
void *dev_malloc(const md_options &o, size_t bytes) {
    if (o.dev_alloc) return o.dev_alloc(bytes, o.alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return p;
}
void dev_release(const md_options &o, void *p) {
    if (!p) return;
    if (o.dev_free) o.dev_free(p, o.alloc_ctx);
    else cudaFree(p);
}

// Wait for an event.  With a cancel flag, poll instead of blocking and pass the flag on to the
// kernels, which stop before their next work item.
cudaError_t wait_event(md_ctx *h, cudaEvent_t e) {
    if (!h->opt.cancel_flag || !h->cancel_host) return cudaEventSynchronize(e);
    for (;;) {
        const cudaError_t q = cudaEventQuery(e);
        if (q != cudaErrorNotReady) return q;
        if (*h->opt.cancel_flag) *h->cancel_host = 1;
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

void fill_static_info(md_ctx *h) {
    std::memset(&h->info, 0, sizeof(h->info));
    h->info.n = h->code.n;
    h->info.k = h->code.k;
    h->info.m = (int)h->code.gam.size();
    for (int j = 0; j < h->info.m && j < MD_MAX_GAMMA; j++) h->info.ranks[j] = h->code.gam[j].rank;
    h->info.d = -1;
}

void free_device(md_ctx *h) {
    if (h->dev.base) {
        cudaStreamSynchronize(stream_of(h));        // a caller's free need not wait for our kernels
        dev_release(h->opt, h->dev.base);
    }
    h->dev = DevLayout();
    if (h->cancel_host) cudaFreeHost((void *)h->cancel_host);
    h->cancel_host = nullptr;
    h->cancel_dev = nullptr;
    if (h->host_state) cudaFreeHost(h->host_state);
    h->host_state = nullptr;
    if (h->heads) cudaFreeHost(h->heads);
    h->heads = nullptr;
    for (cudaEvent_t e : h->lev_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->stage_ev) cudaEventDestroy(e);
    h->lev_ev.clear();
    h->stage_ev.clear();
    for (cudaEvent_t &e : h->run_ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    h->own_stream = nullptr;
    h->dev_ready = false;
}

// Allocate and fill the device buffers: packed rows and pair tables of every Gamma_j,
// the binomial table, the work tables of every level that may run, and the state.
int setup_device(md_ctx *h) {
    if (h->dev_ready) return MD_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return MD_ECUDA;
    if (cudaGetDevice(&h->device) != cudaSuccess) return MD_ECUDA;
    if (!h->opt.stream && cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return MD_ECUDA;
    h->sms = sm_count();
    h->smem_optin = max_smem_per_block();
    h->threads = h->opt.threads_per_block > 0 ? std::min(1024, (h->opt.threads_per_block + 31) / 32 * 32)
                                              : kDefaultThreads;
    if (h->threads > 512) h->threads = 512;     // the kernels are bounded for 512 threads
    const Code &c = h->code;
    const int k = c.k, m = (int)c.gam.size();

    // plan every level up to the deepest stage with C(k, g) < 2^55
    PlanOptions po;
    po.chunk_log2 = h->opt.chunk_log2 > 0 ? h->opt.chunk_log2 : 20;
    po.filter = h->opt.filter;
    po.stop_rule = h->opt.stop_rule;
    po.tensor = h->opt.tensor;
    po.tensor_head = h->opt.tensor_head;
    h->g_limit = 0;
    for (int g = 1; g <= std::min(k, kMaxG); g++) {
        if (binom(k, g) >= kRankLimit) break;
        if ((size_t)g * m > (size_t)kMaxLevels) break;
        h->g_limit = g;
    }
    h->plans.clear();
    h->mtab_offset.clear();
    size_t mtab_entries = 0;
    for (int g = 1; g <= h->g_limit; g++)
        for (int j = 0; j < m; j++) {
            h->plans.push_back(plan_level(c, g, j, po));
            h->mtab_offset.push_back(mtab_entries);
            mtab_entries += h->plans.back().mtab.size();
        }

    // head size of each matrix's tensor-core levels (0: it has none)
    std::vector<int> tc_q(m, 0), tc_smin(m, 0);
    for (const LevelPlan &p : h->plans)
        if (p.kind == KIND_TC) {
            tc_q[p.j] = p.tc_q;
            tc_smin[p.j] = std::max(tc_smin[p.j], p.tc_smin);
        }
    size_t off = 0;
    std::vector<size_t> rows_off(m), h2_off(m), heads_off(m, 0), heads2_off(m, 0);
    for (int j = 0; j < m; j++) {
        rows_off[j] = off;
        off = align256(off + (size_t)k * c.gam[j].WP * 4);
        h2_off[j] = off;
        off = align256(off + (size_t)k * (k - 1) / 2 * c.gam[j].WP * 4 + 16);
        if (tc_q[j]) {
            heads_off[j] = off;
            off = align256(off + tc_tables_bytes(k, tc_q[j], c.gam[j].W));
            heads2_off[j] = off;      // (q+1)-heads of the second phase: the first C(s_min, q+1)
            off = align256(off + tc_heads_bytes(binom(tc_smin[j], tc_q[j] + 1), c.gam[j].W) + 256);
        }
    }
    const size_t binom_off = off;
    off = align256(off + (size_t)(k + 1) * (k + 1) * 8);
    const size_t mtab_off = off;
    off = align256(off + std::max<size_t>(1, mtab_entries) * sizeof(MEntry));
    const size_t st_off = off;
    off = align256(off + sizeof(DevState));

    h->dev.base = (char *)dev_malloc(h->opt, off);
    if (!h->dev.base) { free_device(h); return MD_ENOMEM; }
    if (((uintptr_t)h->dev.base & 255) != 0) { free_device(h); return MD_EINVAL; }   // the hook's alignment
    {
        // the cancel word: mapped pinned memory, read by the kernels through its device address
        void *cw = nullptr, *cwd = nullptr;
        if (cudaHostAlloc(&cw, 64, cudaHostAllocMapped) != cudaSuccess) { cudaGetLastError(); free_device(h); return MD_ENOMEM; }
        h->cancel_host = (volatile int *)cw;
        *h->cancel_host = 0;
        if (cudaHostGetDevicePointer(&cwd, cw, 0) != cudaSuccess) { cudaGetLastError(); free_device(h); return MD_ECUDA; }
        h->cancel_dev = (const volatile int *)cwd;
    }
    if (cudaMallocHost(&h->host_state, sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost(&h->heads, sizeof(md_ctx::Head) * std::max(1, h->g_limit)) != cudaSuccess) {
        cudaGetLastError();
        free_device(h);
        return MD_ENOMEM;
    }
    // events reused by every md_compute on this handle
    h->lev_ev.resize((size_t)2 * h->g_limit * m);
    h->stage_ev.resize(h->g_limit);
    for (cudaEvent_t &e : h->lev_ev) cudaEventCreate(&e);
    for (cudaEvent_t &e : h->stage_ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventCreate(&h->run_ev[0]);
    cudaEventCreate(&h->run_ev[1]);
    h->dev.bytes = off;
    h->dev.rows.resize(m);
    h->dev.h2.resize(m);
    h->dev.heads.assign(m, nullptr);
    h->dev.heads2.assign(m, nullptr);
    h->dev.tc_smin = tc_smin;
    for (int j = 0; j < m; j++) {
        h->dev.rows[j] = (uint32_t *)(h->dev.base + rows_off[j]);
        h->dev.h2[j] = (uint32_t *)(h->dev.base + h2_off[j]);
        if (tc_q[j]) {
            h->dev.heads[j] = (unsigned char *)(h->dev.base + heads_off[j]);
            h->dev.heads2[j] = (unsigned char *)(h->dev.base + heads2_off[j]);
        }
    }
    h->dev.binom = (unsigned long long *)(h->dev.base + binom_off);
    h->dev.mtab = (MEntry *)(h->dev.base + mtab_off);
    h->dev.st = (DevState *)(h->dev.base + st_off);

    cudaStream_t s = stream_of(h);
    std::vector<unsigned long long> tb((size_t)(k + 1) * (k + 1));
    for (int a = 0; a <= k; a++)
        for (int b = 0; b <= k; b++) tb[(size_t)a * (k + 1) + b] = binom(a, b);
    std::vector<MEntry> all;
    all.reserve(mtab_entries);
    for (const LevelPlan &p : h->plans) all.insert(all.end(), p.mtab.begin(), p.mtab.end());
    // synchronous uploads (pageable host memory), then the pair tables on the device
    bool ok = cudaMemcpy(h->dev.binom, tb.data(), tb.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !all.empty())
        ok = cudaMemcpy(h->dev.mtab, all.data(), all.size() * sizeof(MEntry), cudaMemcpyHostToDevice) == cudaSuccess;
    for (int j = 0; ok && j < m; j++) {
        ok = cudaMemcpy(h->dev.rows[j], c.gam[j].packed.data(), c.gam[j].packed.size() * 4, cudaMemcpyHostToDevice) ==
             cudaSuccess;
        if (ok) ok = launch_h2_build(h->dev.rows[j], h->dev.h2[j], k, c.gam[j].WP, s) == 0;
    }
    int head_tables = 0;
    for (int j = 0; ok && j < m; j++)
        if (tc_q[j]) {
            ok = launch_tc_tables(h->dev.rows[j], h->dev.binom, k, tc_q[j], c.gam[j].W, c.gam[j].WP,
                                  binom(k, tc_q[j]), h->dev.heads[j], s) == 0;
            const uint64_t n2 = binom(tc_smin[j], tc_q[j] + 1);
            if (ok && n2) ok = launch_tc_tables(h->dev.rows[j], h->dev.binom, k, tc_q[j] + 1, c.gam[j].W,
                                                c.gam[j].WP, n2, h->dev.heads2[j], s) == 0;
            head_tables += 2;
        }
    if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) { cudaGetLastError(); free_device(h); return MD_ECUDA; }
    h->setup_launches = m + head_tables;
    h->setup_h2d = tb.size() * 8 + all.size() * sizeof(MEntry);
    for (int j = 0; j < m; j++) h->setup_h2d += c.gam[j].packed.size() * 4;
    h->dev_ready = true;
    return MD_OK;
}

struct LaunchCfg {
    int blocks, threads;
    size_t smem;
    bool h2s;
};

LaunchCfg launch_cfg(md_ctx *h, const LevelPlan &p) {
    const Gamma &gm = h->code.gam[p.j];
    LaunchCfg L;
    L.threads = h->threads;
    const int with_h2 = level_smem_bytes(h->code.k, gm.WP, true);
    L.h2s = p.kind != KIND_SIMPLE && with_h2 <= h->smem_optin - 1024;
    L.smem = (size_t)level_smem_bytes(h->code.k, gm.WP, p.kind != KIND_SIMPLE && L.h2s);
    int per_sm = level_blocks_per_sm(p.kind, gm.W, L.h2s, L.threads, L.smem);
    if (h->opt.blocks_per_sm > 0) per_sm = std::min(std::max(1, per_sm), h->opt.blocks_per_sm);
    per_sm = std::max(1, per_sm);
    uint64_t want = (uint64_t)h->sms * per_sm;
    // no more blocks than 16-warp groups of work items
    const uint64_t warps_per_block = (uint64_t)L.threads / 32;
    const uint64_t need = (p.nchunks + warps_per_block - 1) / warps_per_block;
    L.blocks = (int)std::max<uint64_t>(1, std::min(want, need));
    return L;
}

LevelArgs level_args(md_ctx *h, const LevelPlan &p, int level, bool h2s) {
    const Gamma &gm = h->code.gam[p.j];
    LevelArgs a{};
    a.rows = h->dev.rows[p.j];
    a.h2 = h->dev.h2[p.j];
    a.binom = h->dev.binom;
    a.mtab = p.mtab.empty() ? nullptr : h->dev.mtab + h->mtab_offset[level];
    a.st = h->dev.st;
    a.nchunks = p.nchunks;
    a.count = p.count;
    a.r_begin = 0;
    a.per_chunk = p.per_chunk;
    a.n_m = (int)p.mtab.size();
    a.k = h->code.k;
    a.g = p.g;
    a.v = p.v;
    a.base = p.base;
    a.level = level;
    a.fmax8 = p.fmax8;
    a.h2_in_smem = h2s ? 1 : 0;
    a.m_total = (int)h->code.gam.size();
    a.j = p.j;
    a.L_after = p.L_after;
    a.L_first = p.L_first;
    a.check_stop = 1;
    a.cancel = h->cancel_dev;
    (void)gm;
    return a;
}

unsigned g_last_bounds_site = 0;    // the debug build's last failing check site

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// ---- checkpoints: a header, then the completed levels' records and the U each started with ----
constexpr uint64_t kCkptMagic = 0x3130545048434B4Dull;     // "MKCHPT01"
struct CkptHeader {
    uint64_t magic;
    uint64_t code_hash;     // the code in processing order and the stop rule (level order and bounds)
    int32_t n, k, m, nlev;  // nlev = completed levels: 0 .. nlev-1 in (g, j) order
    uint32_t U;             // least weight among the completed levels' records (n + 1: none)
    int32_t L;              // lower bound after the last completed level
    int32_t stop;           // L >= U: the run is complete
    int32_t pad;
};                          // then uint64 key[nlev], uint32 u_in[nlev]

uint64_t code_hash(const md_ctx *h) {
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t bytes) {
        for (size_t i = 0; i < bytes; i++) x = (x ^ ((const unsigned char *)p)[i]) * 1099511628211ull;
    };
    const Code &c = h->code;
    mix(&c.n, sizeof(c.n));
    mix(&c.k, sizeof(c.k));
    mix(&h->opt.stop_rule, sizeof(h->opt.stop_rule));
    mix(c.G.data(), c.G.size() * sizeof(uint64_t));
    mix(c.perm.data(), c.perm.size() * sizeof(int));
    return x;
}

// Validate a checkpoint image against the handle; MD_OK with *hdr filled.
int parse_checkpoint(const md_ctx *h, const void *buf, size_t size, CkptHeader *hdr) {
    if (!buf || size < sizeof(CkptHeader)) return MD_EINVAL;
    std::memcpy(hdr, buf, sizeof(CkptHeader));
    const int m = (int)h->code.gam.size();
    if (hdr->magic != kCkptMagic || hdr->code_hash != code_hash(h) || hdr->n != h->code.n || hdr->k != h->code.k ||
        hdr->m != m || hdr->nlev < 0 || hdr->nlev > std::min(h->code.k * m, kMaxLevels - 1) ||
        size != sizeof(CkptHeader) + (size_t)hdr->nlev * 12 || hdr->U > (uint32_t)h->code.n + 1)
        return MD_EINVAL;
    return MD_OK;
}

// Queue the device state of a checkpoint on stream s (after the state initialisation).
int restore_checkpoint(md_ctx *h, const std::vector<char> &img, cudaStream_t s, int *first_level) {
    CkptHeader hdr;
    if (parse_checkpoint(h, img.data(), img.size(), &hdr) != MD_OK) return MD_EINVAL;
    std::vector<unsigned char> raw(sizeof(DevState));
    DevState &st = *reinterpret_cast<DevState *>(raw.data());
    st.U = hdr.U;
    st.L = hdr.L;
    st.stop = hdr.stop;
    st.error = 0;
    st.last_level = hdr.nlev - 1;
    st.pad = 0;
    st.skipped = 0;
    const unsigned long long *keys = reinterpret_cast<const unsigned long long *>(img.data() + sizeof(CkptHeader));
    const uint32_t *u_in = reinterpret_cast<const uint32_t *>(img.data() + sizeof(CkptHeader) + (size_t)hdr.nlev * 8);
    for (int i = 0; i < kMaxLevels; i++) {
        st.key[i] = i < hdr.nlev ? keys[i] : kNoKey;
        st.u_in[i] = i < hdr.nlev ? u_in[i] : hdr.U;
        st.ctr[i] = 0;
    }
    if (cudaMemcpyAsync(h->dev.st, raw.data(), raw.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    *first_level = hdr.nlev;
    return MD_OK;
}

}  // namespace

namespace mdl {
int bounds_status() {
    unsigned s[4] = {0u, 0u, 0u, 0u};
    bounds_site_kernels(&s[0], 1);
    bounds_site_tc(&s[1], 1);
    bounds_site_engine(&s[2], 1);
    bounds_site_noalloc(&s[3], 1);
    for (unsigned v : s)
        if (v) {
            g_last_bounds_site = v;
            return MD_EINTERNAL;
        }
    return MD_OK;
}
}  // namespace mdl

extern "C" {

int md_debug_bounds(unsigned *site) {
    if (!site) return MD_EINVAL;
    *site = g_last_bounds_site;
#ifdef MD_DEBUG_BOUNDS
    return MD_OK;
#else
    return MD_EUNSUPPORTED;
#endif
}

int md_checkpoint(md_handle h, void *buf, size_t cap, size_t *size) {
    if (!h || !size || !h->have_state || !h->host_state) return MD_EINVAL;
    const DevState &st = *h->host_state;
    const int n = h->code.n;
    CkptHeader hdr{};
    hdr.magic = kCkptMagic;
    hdr.code_hash = code_hash(h);
    hdr.n = n;
    hdr.k = h->code.k;
    hdr.m = (int)h->code.gam.size();
    hdr.nlev = st.last_level + 1;
    // U from the completed levels only: a level cut short by a cancel may have lowered the
    // device's U with a codeword whose record was not kept
    unsigned U = (unsigned)n + 1;
    for (int i = 0; i < hdr.nlev; i++)
        if (st.key[i] != kNoKey) U = std::min(U, (unsigned)(st.key[i] >> kRankBits));
    hdr.U = U;
    hdr.L = st.L;
    hdr.stop = st.L >= (int)U ? 1 : 0;        // the stop of Alg. 1, whatever ended the run
    const size_t need = sizeof(CkptHeader) + (size_t)hdr.nlev * 12;
    *size = need;
    if (!buf) return MD_OK;
    if (cap < need) return MD_EINVAL;
    char *out = (char *)buf;
    std::memcpy(out, &hdr, sizeof(hdr));
    std::memcpy(out + sizeof(hdr), st.key, (size_t)hdr.nlev * 8);
    std::memcpy(out + sizeof(hdr) + (size_t)hdr.nlev * 8, st.u_in, (size_t)hdr.nlev * 4);
    return MD_OK;
}

int md_resume(md_handle h, const void *buf, size_t size) {
    if (!h) return MD_EINVAL;
    CkptHeader hdr;
    const int rc = parse_checkpoint(h, buf, size, &hdr);
    if (rc != MD_OK) return rc;
    h->resume.assign((const char *)buf, (const char *)buf + size);
    return MD_OK;
}

int md_options_init(md_options *opt) {
    if (!opt) return MD_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->chunk_log2 = 20;
    opt->filter = 1;
    opt->use_graph = 1;
    opt->tensor = 1;
    return MD_OK;
}

const char *md_strerror(int code) {
    switch (code) {
        case MD_OK: return "ok";
        case MD_EINVAL: return "invalid argument";
        case MD_ERANK: return "generator matrix is not of full row rank";
        case MD_EUNSUPPORTED: return "unsupported size (n > 256, or a level with C(k,g) >= 2^55)";
        case MD_ENOMEM: return "out of memory";
        case MD_ECUDA: return "CUDA error or no usable GPU";
        case MD_EBUDGET: return "work budget exceeded";
        case MD_ECANCELED: return "cancelled";
        case MD_ETIMEOUT: return "device-side wait timed out";
        case MD_EBUSY: return "request pending";
        case MD_EINTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int md_create_ex(const uint64_t *G, int n, int k, const md_options *opt, md_handle *out) {
    if (!G || !out) return MD_EINVAL;
    md_ctx *h = new (std::nothrow) md_ctx();
    if (!h) return MD_ENOMEM;
    if (opt) h->opt = *opt; else md_options_init(&h->opt);
    int rc = build_code_permuted(G, n, k, h->opt.perm_trials, h->opt.perm_seed, &h->code);
    if (rc != MD_OK) { delete h; return rc; }
    fill_static_info(h);
    *out = h;
    return MD_OK;
}

int md_create(const uint64_t *G, int n, int k, md_handle *out) { return md_create_ex(G, n, k, nullptr, out); }

void md_destroy(md_handle h) {
    if (!h) return;
    free_device(h);
    delete h;
}

int md_info_get(md_handle h, md_info *info) {
    if (!h || !info) return MD_EINVAL;
    *info = h->info;
    return MD_OK;
}

int md_levels(md_handle h, md_level *levels, int max, int *count) {
    if (!h || !count || (max > 0 && !levels)) return MD_EINVAL;
    int nl = std::min<int>(max, (int)h->levels.size());
    for (int i = 0; i < nl; i++) levels[i] = h->levels[i];
    *count = nl;
    return MD_OK;
}

int md_gamma(md_handle h, int j, uint64_t *gamma, int *order) {
    if (!h || j < 0 || j >= (int)h->code.gam.size()) return MD_EINVAL;
    const Code &c = h->code;
    const Gamma &gm = c.gam[j];
    if (gamma)
        for (int i = 0; i < c.k; i++) to_caller_order(c, &gm.rows[(size_t)i * c.nw64], gamma + (size_t)i * c.nw64);
    if (order)
        for (int p = 0; p < c.n; p++) order[p] = c.perm.empty() ? gm.order[p] : c.perm[gm.order[p]];
    return MD_OK;
}

int md_compute(md_handle h, int *d, uint64_t *witness) {
    if (!h || !d) return MD_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    int rc = setup_device(h);
    if (rc != MD_OK) return rc;
    cudaStream_t s = stream_of(h);
    const Code &c = h->code;
    const int n = c.n, k = c.k, m = (int)c.gam.size();
    fill_static_info(h);
    h->levels.clear();
    // NVTX ranges (no-ops unless a profiler is attached): the call, and the enqueue of each level
    char label[64];
    std::snprintf(label, sizeof(label), "md_compute [%d,%d]", c.n, c.k);
    nvtxRangePushA(label);
    struct RangePop {
        ~RangePop() { nvtxRangePop(); }
    } range_pop;

    cudaEvent_t ev0 = h->run_ev[0], ev1 = h->run_ev[1];
    using Head = md_ctx::Head;
    *h->cancel_host = 0;                  // a cancelled run left it set
    int nlev_ev = 0, nstages = 0;
    int launches = 0;
    uint64_t h2d = 0, d2h = 0;
    bool err = launch_state_init(h->dev.st, (unsigned)(n + 1), s) != 0;
    launches++;
    // a resumed run: the bounds and the completed levels' records of the checkpoint, and the
    // stage loop from the level after it
    int first_level = 0;
    if (!h->resume.empty()) {
        std::vector<char> img;
        img.swap(h->resume);
        if (!err) err = restore_checkpoint(h, img, s, &first_level) != MD_OK;
        h2d += img.size();
    }
    cudaEventRecord(ev0, s);
    uint64_t planned = 0;
    int status = MD_OK;
    bool stopped = false;
    std::vector<int> ev_level;              // the level timed by each pair of events
    int g = first_level / m + 1;
    for (; g <= k && !err; g++) {
        if (g > h->g_limit) { status = MD_EUNSUPPORTED; break; }
        if (h->opt.max_stage > 0 && g > h->opt.max_stage) break;
        if (h->opt.cancel_flag && *h->opt.cancel_flag) { status = MD_ECANCELED; break; }
        const uint64_t stage_work = (uint64_t)m * binom(k, g);
        if (h->opt.work_budget && planned + stage_work > h->opt.work_budget) {
            // the budget would be exceeded only if the run has not stopped already
            cudaStreamSynchronize(s);
            Head hd;
            cudaMemcpy(&hd, h->dev.st, sizeof(Head), cudaMemcpyDeviceToHost);
            d2h += sizeof(Head);
            if (!hd.stop) status = MD_EBUDGET;
            stopped = hd.stop != 0;
            break;
        }
        planned += stage_work;
        for (int j = (g - 1) * m < first_level ? first_level % m : 0; j < m && !err; j++) {
            const int level = (g - 1) * m + j;
            ev_level.push_back(level);
            const LevelPlan &p = h->plans[level];
            std::snprintf(label, sizeof(label), "level g=%d j=%d %s", p.g, p.j, p.kind == KIND_TC ? "tensor" : "popcount");
            nvtxRangePushA(label);
            cudaEventRecord(h->lev_ev[nlev_ev], s);
            LevelArgs a;
            if (p.kind == KIND_TC) {
                a = level_args(h, p, level, false);
                err |= launch_tc_level(h->dev.heads[p.j], h->dev.heads2[p.j], p.tc_smin, h->dev.rows[p.j],
                                       h->dev.binom, h->dev.st, k, p.g, p.tc_q, p.base, level, c.gam[p.j].W,
                                       c.gam[p.j].WP, 1, h->sms, h->opt.test_stall, p.tc_words8, h->cancel_dev,
                                       s) != 0;
            } else {
                LaunchCfg L = launch_cfg(h, p);
                a = level_args(h, p, level, L.h2s);
                err |= launch_level(a, p.kind, c.gam[p.j].W, c.gam[p.j].WP, L.blocks, L.threads, L.smem, s) != 0;
            }
            cudaEventRecord(h->lev_ev[nlev_ev + 1], s);
            nlev_ev += 2;
            err |= launch_finalize(a, s) != 0;
            launches += 2;
            nvtxRangePop();
        }
        Head *hd = h->heads + nstages;
        cudaMemcpyAsync(hd, h->dev.st, sizeof(Head), cudaMemcpyDeviceToHost, s);
        d2h += sizeof(Head);
        cudaEventRecord(h->stage_ev[nstages], s);
        nstages++;
        // look one stage behind: the device keeps working on the stage just queued
        if (nstages >= 2) {
            wait_event(h, h->stage_ev[nstages - 2]);
            if (h->heads[nstages - 2].stop) { stopped = true; break; }
        }
    }
    cudaEventRecord(ev1, s);
    if (wait_event(h, ev1) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) err = true;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    std::vector<double> lev_sec((size_t)h->g_limit * m, 0.0);      // per level index (0: not run in this call)
    for (int i = 0; i + 1 < nlev_ev; i += 2) {
        float lms = 0.f;
        if (cudaEventElapsedTime(&lms, h->lev_ev[i], h->lev_ev[i + 1]) == cudaSuccess) lev_sec[ev_level[i / 2]] = lms * 1e-3;
    }
    if (err) { cudaGetLastError(); return MD_ECUDA; }
    if (cudaMemcpy(h->host_state, h->dev.st, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) return MD_ECUDA;
    h->have_state = true;
    d2h += sizeof(DevState);
    const DevState &st = *h->host_state;
    if (st.error) return st.error == MD_ETIMEOUT || st.error == MD_ECANCELED ? st.error : MD_EINTERNAL;
    // complete: L >= U was reached, or every stage up to g = k ran (Alg. 1's loop bound)
    stopped = st.stop != 0 || (status == MD_OK && st.last_level == k * m - 1);

    // per-level records of the levels that ran
    const int last = st.last_level;
    uint64_t evaluated = 0;
    int key_level = -1;
    const int U = (int)st.U;
    for (int lv = 0; lv <= last; lv++) {
        const LevelPlan &p = h->plans[lv];
        md_level r{};
        r.g = p.g;
        r.j = p.j;
        r.count = p.count;
        const unsigned long long key = st.key[lv];
        if (key == kNoKey) {
            r.weight = -1;
            r.first_rank = 0;
        } else {
            r.weight = (int)(key >> kRankBits);
            r.first_rank = key & (kRankLimit - 1);
        }
        r.seconds = lv < (int)lev_sec.size() ? lev_sec[lv] : 0.0;
        if (p.kind == KIND_TC) {
            // the scheduler's word count for the U the level started with (U only drops later)
            const int W = c.gam[p.j].W, thr = (int)st.u_in[lv] - p.base;
            r.words = W;
            for (int f = 1; f < W; f++)
                if ((int)((p.tc_words8 >> (8 * (f - 1))) & 255ull) > thr) { r.words = f; break; }
        }
        if (key_level < 0 && r.weight == U) key_level = lv;
        evaluated += p.count;
        h->levels.push_back(r);
    }
    h->info.d = U <= n ? U : -1;
    h->info.complete = stopped ? 1 : 0;
    h->info.lower_bound = st.L;
    h->info.nlevels = last + 1;
    h->info.codewords = evaluated;
    h->info.stop_g = last >= 0 ? h->plans[last].g : 0;
    h->info.stop_j = last >= 0 ? h->plans[last].j : 0;
    h->info.seconds_device = ms * 1e-3;
    h->info.gpu_launches = launches + h->setup_launches;
    h->info.h2d_bytes = h2d + h->setup_h2d;
    h->info.skipped_work = st.skipped;
    h->info.d2h_bytes = d2h;
    h->setup_launches = 0;
    h->setup_h2d = 0;
    if (U > n || key_level < 0) {
        h->info.seconds_total = seconds_since(t0);
        return status != MD_OK ? status : MD_EINTERNAL;
    }
    const md_level &kr = h->levels[key_level];
    h->info.key_g = kr.g;
    h->info.key_j = kr.j;
    h->info.key_rank = kr.first_rank;
    // witness: the rows of Gamma_j at the key's combination, summed
    std::vector<int> comb(kr.g);
    colex_unrank(kr.first_rank, kr.g, k, comb.data());
    std::vector<uint64_t> wv(c.nw64, 0);
    const Gamma &gm = c.gam[kr.j];
    for (int i : comb)
        for (int w = 0; w < c.nw64; w++) wv[w] ^= gm.rows[(size_t)i * c.nw64 + w];
    if (popcount_row(wv.data(), c.nw64) != U) return MD_EINTERNAL;
    if (bounds_status() != MD_OK) return MD_EINTERNAL;          // the debug build's range checks
    h->info.seconds_total = seconds_since(t0);
    if (status != MD_OK) return status;
    *d = U;
    if (witness) to_caller_order(c, wv.data(), witness);
    return MD_OK;
}

int md_level_plan(md_handle h, int g, int j, int *kind, md_task_info *tasks, int max, int *count,
                  uint64_t *work_items) {
    if (!h || !kind || !count || !work_items || (max > 0 && !tasks)) return MD_EINVAL;
    const Code &c = h->code;
    if (j < 0 || j >= (int)c.gam.size() || g < 1 || g > c.k || g > kMaxG) return MD_EINVAL;
    if (binom(c.k, g) >= kRankLimit) return MD_EUNSUPPORTED;
    PlanOptions po;
    po.chunk_log2 = h->opt.chunk_log2 > 0 ? h->opt.chunk_log2 : 20;
    po.filter = h->opt.filter;
    po.stop_rule = h->opt.stop_rule;
    po.tensor = h->opt.tensor;
    po.tensor_head = h->opt.tensor_head;
    LevelPlan p = plan_level(c, g, j, po);
    *kind = p.kind;
    *work_items = p.nchunks;
    int nt = 0;
    for (const MEntry &e : p.mtab) {
        if (e.upper_base != 0) return MD_EINTERNAL;
        if (nt < max) {
            tasks[nt].M = e.M;
            tasks[nt].per_lane = e.per_lane;
            tasks[nt].uppers = e.uppers;
            tasks[nt].first_item = e.chunk_begin;
        }
        nt++;
    }
    *count = std::min(nt, max);
    return MD_OK;
}

// Least weight over colex ranks [r0, r1) of level (g, j), with the per-lane kernel.
int md_scan_range(md_handle h, int g, int j, uint64_t r0, uint64_t r1, int bound, int *weight,
                  uint64_t *first_rank) {
    if (!h || !weight || !first_rank) return MD_EINVAL;
    const Code &c = h->code;
    if (j < 0 || j >= (int)c.gam.size() || g < 1 || g > c.k || g > kMaxG) return MD_EINVAL;
    const uint64_t total = binom(c.k, g);
    if (total >= kRankLimit) return MD_EUNSUPPORTED;
    r1 = std::min<uint64_t>(r1, total);
    if (r0 > r1) r0 = r1;
    int rc = setup_device(h);
    if (rc != MD_OK) return rc;
    cudaStream_t s = stream_of(h);
    PlanOptions po;
    po.chunk_log2 = h->opt.chunk_log2 > 0 ? h->opt.chunk_log2 : 20;
    LevelPlan p = plan_level(c, g, j, po);
    p.kind = KIND_SIMPLE;
    p.mtab.clear();
    const uint64_t span = r1 - r0;
    p.per_chunk = std::max<uint64_t>(1, std::min<uint64_t>(p.per_chunk ? p.per_chunk : 1, span / (32ull * 152 * 16)));
    p.per_chunk = std::max<uint64_t>(p.per_chunk, 1);
    p.nchunks = (span + 32 * p.per_chunk - 1) / (32 * p.per_chunk);
    LaunchCfg L = launch_cfg(h, p);
    LevelArgs a = level_args(h, p, 0, false);
    a.r_begin = r0;
    a.count = r1;
    a.check_stop = 0;
    a.cancel = nullptr;                   // scans are not cancelled
    const unsigned u0 = bound >= 0 ? (unsigned)bound : (unsigned)(c.n + 1);
    bool err = launch_state_init(h->dev.st, u0, s) != 0;
    if (span > 0) err |= launch_level(a, p.kind, c.gam[j].W, c.gam[j].WP, L.blocks, L.threads, L.smem, s) != 0;
    unsigned long long key = kNoKey;
    if (!err) err = cudaMemcpyAsync(&key, &h->dev.st->key[0], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess;
    if (cudaStreamSynchronize(s) != cudaSuccess || err) { cudaGetLastError(); return MD_ECUDA; }
    if (bounds_status() != MD_OK) return MD_EINTERNAL;
    if (key == kNoKey) { *weight = -1; *first_rank = 0; }
    else { *weight = (int)(key >> kRankBits); *first_rank = key & (kRankLimit - 1); }
    return MD_OK;
}

// Least weight over the combinations of level (g, j) whose element M = c_{P+1} is fixed
// and whose upper part has colex index in [u0, u1), with the production split kernel.
int md_scan_task(md_handle h, int g, int j, int M, uint64_t u0, uint64_t u1, int bound, int *weight,
                 uint64_t *first_rank) {
    if (!h || !weight || !first_rank) return MD_EINVAL;
    const Code &c = h->code;
    if (j < 0 || j >= (int)c.gam.size() || g < 5 || g > c.k || g > kMaxG) return MD_EINVAL;
    if (binom(c.k, g) >= kRankLimit) return MD_EUNSUPPORTED;
    int rc = setup_device(h);
    if (rc != MD_OK) return rc;
    cudaStream_t s = stream_of(h);
    PlanOptions po;
    po.chunk_log2 = h->opt.chunk_log2 > 0 ? h->opt.chunk_log2 : 20;
    po.filter = h->opt.filter;
    po.stop_rule = h->opt.stop_rule;
    LevelPlan p = plan_level(c, g, j, po);
    if (p.kind == KIND_SIMPLE) p.kind = (g == 5) ? KIND_SPLIT2 : KIND_SPLIT3, p.v = g - p.kind - 1;
    const int P = p.kind;
    if (M < P || M > c.k - 1 - p.v) return MD_EINVAL;
    const uint64_t nup = binom(c.k - 1 - M, p.v);
    u1 = std::min<uint64_t>(u1, nup);
    if (u0 > u1) u0 = u1;
    MEntry e{};
    e.M = (uint32_t)M;
    e.upper_base = u0;
    e.uppers = u1 - u0;
    e.chunk_begin = 0;
    // the same per-lane run length as the level plan uses for this M
    uint32_t per_lane = 1;
    for (const MEntry &x : p.mtab)
        if ((int)x.M == M) per_lane = x.per_lane;
    e.per_lane = per_lane;
    p.mtab.assign(1, e);
    p.nchunks = (e.uppers + 32ull * per_lane - 1) / (32ull * per_lane);
    // the task's work table lives in the spare entry past the planned levels
    MEntry *dtab = (MEntry *)dev_malloc(h->opt, 256);
    if (!dtab) return MD_ENOMEM;
    bool err = cudaMemcpy(dtab, &e, sizeof(MEntry), cudaMemcpyHostToDevice) != cudaSuccess;
    LaunchCfg L = launch_cfg(h, p);
    LevelArgs a = level_args(h, p, 0, L.h2s);
    a.mtab = dtab;
    a.check_stop = 0;
    a.cancel = nullptr;
    const unsigned ub = bound >= 0 ? (unsigned)bound : (unsigned)(c.n + 1);
    err |= launch_state_init(h->dev.st, ub, s) != 0;
    if (p.nchunks > 0) err |= launch_level(a, p.kind, c.gam[j].W, c.gam[j].WP, L.blocks, L.threads, L.smem, s) != 0;
    unsigned long long key = kNoKey;
    if (!err) err = cudaMemcpyAsync(&key, &h->dev.st->key[0], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess;
    if (cudaStreamSynchronize(s) != cudaSuccess) err = true;
    dev_release(h->opt, dtab);
    if (err) { cudaGetLastError(); return MD_ECUDA; }
    if (bounds_status() != MD_OK) return MD_EINTERNAL;
    if (key == kNoKey) { *weight = -1; *first_rank = 0; }
    else { *weight = (int)(key >> kRankBits); *first_rank = key & (kRankLimit - 1); }
    return MD_OK;
}

}  // extern "C"
