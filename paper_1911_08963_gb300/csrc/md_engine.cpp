// md_engine.cpp -- host side of the multi-code engine and md_batch.
#include "md_engine.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>

namespace mdl {

namespace {

constexpr int kThreads = 256;
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int prepare_code(const uint64_t *G, int n, int k, const PlanOptions &po, int max_stage, uint64_t budget,
                 PreparedCode *out, int horizon) {
    PreparedCode p;
    int rc = build_code_permuted(G, n, k, po.perm_trials, po.perm_seed, &p.code);
    if (rc != MD_OK) return rc;
    int g_est = 0;
    const double work = estimate_work(p.code, nullptr, &g_est);
    if (budget && work > (double)budget) return MD_EBUDGET;
    p.est_work = work;
    const int m = (int)p.code.gam.size();
    for (int g = 1; g <= std::min(k, kMaxG); g++) {
        if (binom(k, g) >= kRankLimit) break;
        if (max_stage > 0 && g > max_stage) break;
        if ((size_t)g * m > (size_t)kMaxLevels) break;
        p.g_max = g;
    }
    // plans (and their device tables) only a few stages past the estimated stop; a code
    // that runs past them is finished by a single-code run
    p.g_limit = horizon > 0 ? std::min(p.g_max, g_est + horizon) : p.g_max;
    p.max_stage = max_stage;
    size_t nm = 0;
    for (int g = 1; g <= p.g_limit; g++)
        for (int j = 0; j < m; j++) {
            p.plans.push_back(plan_level(p.code, g, j, po));
            nm += p.plans.back().mtab.size();
        }
    size_t hb = 0, h2 = 0;
    for (const Gamma &gm : p.code.gam) {
        hb = align256(hb + (size_t)k * gm.WP * 4);
        h2 = align256(h2 + (size_t)k * (k - 1) / 2 * gm.WP * 4 + 16);
    }
    hb = align256(hb + p.plans.size() * sizeof(BLevel));
    hb = align256(hb + std::max<size_t>(1, nm) * sizeof(MEntry));
    hb = align256(hb + std::max<size_t>(1, p.plans.size()) * 8);
    p.header_bytes = hb;
    p.h2_bytes = h2;
    *out = std::move(p);
    return MD_OK;
}

void prepare_codes(const md_code *codes, int count, const PlanOptions &po, int max_stage, uint64_t budget,
                   std::vector<PreparedCode> &out, int *status, int horizon) {
    out.resize(count);
    const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), std::min(32, count / 8 + 1)));
    std::atomic<int> next{0};
    auto work = [&]() {
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            status[i] = prepare_code(codes[i].G, codes[i].n, codes[i].k, po, max_stage, budget, &out[i], horizon);
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
}

Engine::~Engine() { release_all(); }

void *Engine::dmalloc(size_t bytes) {
    if (alloc_) {
        void *p = alloc_(bytes, alloc_ctx_);
        return ((uintptr_t)p & 255) == 0 ? p : nullptr;     // the hook promises 256-byte alignment
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return p;
}

void Engine::dfree(void *p) {
    if (!p) return;
    if (free_) free_(p, alloc_ctx_);
    else cudaFree(p);
}

int Engine::init(int nslots, cudaStream_t stream, unsigned long long quota, int blocks_per_sm_cap) {
    stream_ = stream;
    nslots_ = nslots;
    cap_ = blocks_per_sm_cap;
    own_mem_.assign(nslots, nullptr);
    host_codes_.assign(nslots, BCode{});
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev);
    size_t off = 0;
    const size_t codes_off = off; off = align256(off + nslots * sizeof(BCode));
    const size_t st_off = off; off = align256(off + nslots * sizeof(BState));
    const size_t as_off = off; off = align256(off + (size_t)kWClasses * nslots * sizeof(int));
    const size_t ap_off = off; off = align256(off + (size_t)kWClasses * nslots * 8);
    const size_t cnt_off = off; off = align256(off + kWClasses * sizeof(int));
    const size_t tot_off = off; off = align256(off + kWClasses * 8);
    const size_t ctr_off = off; off = align256(off + kWClasses * 8);
    const size_t bin_off = off; off = align256(off + (size_t)257 * 257 * 8);
    tables_ = (char *)dmalloc(off);
    if (!tables_) return MD_ENOMEM;
    if (cudaMemsetAsync(tables_, 0, off, stream_) != cudaSuccess) return MD_ECUDA;
    std::vector<unsigned long long> tb((size_t)257 * 257);
    for (int a = 0; a <= 256; a++)
        for (int b = 0; b <= 256; b++) tb[(size_t)a * 257 + b] = binom(a, b);
    if (cudaMemcpyAsync(tables_ + bin_off, tb.data(), tb.size() * 8, cudaMemcpyHostToDevice, stream_) != cudaSuccess)
        return MD_ECUDA;
    if (cudaStreamSynchronize(stream_) != cudaSuccess) return MD_ECUDA;
    args_.codes = (const BCode *)(tables_ + codes_off);
    args_.states = (BState *)(tables_ + st_off);
    args_.nslots = nslots;
    args_.act_slots = (int *)(tables_ + as_off);
    args_.act_prefix = (unsigned long long *)(tables_ + ap_off);
    args_.act_count = (int *)(tables_ + cnt_off);
    args_.act_total = (unsigned long long *)(tables_ + tot_off);
    args_.tick_ctr = (unsigned long long *)(tables_ + ctr_off);
    args_.binom = (const unsigned long long *)(tables_ + bin_off);
    quota_cw_ = quota;
    for (int w = 1; w < kWClasses; w++) {
        int per = engine_blocks_per_sm(w, kThreads);
        if (cap_ > 0) per = std::min(std::max(1, per), cap_);
        blocks_[w] = sms_ * std::max(1, per);
    }
    return MD_OK;
}

// Lay out one code: header (rows, levels, work tables, keys) at `header`, pair tables at
// `h2`; the host image of the header goes to img[img_off ...].
int Engine::fill_code(PreparedCode &pc, char *header, char *h2, std::vector<char> &img, size_t img_off,
                      BCode *bc) {
    const Code &cd = pc.code;
    const int k = cd.k, m = (int)cd.gam.size();
    std::vector<size_t> rows_off(m), h2_off(m);
    size_t off = 0, hoff = 0;
    for (int j = 0; j < m; j++) {
        rows_off[j] = off;
        off = align256(off + (size_t)k * cd.gam[j].WP * 4);
        h2_off[j] = hoff;
        hoff = align256(hoff + (size_t)k * (k - 1) / 2 * cd.gam[j].WP * 4 + 16);
        std::memcpy(img.data() + img_off + rows_off[j], cd.gam[j].packed.data(), cd.gam[j].packed.size() * 4);
        wclass_[cd.gam[j].W] = true;
    }
    const size_t lev_off = off;
    off = align256(off + pc.plans.size() * sizeof(BLevel));
    const size_t mt_off = off;
    size_t nm = 0;
    for (const LevelPlan &p : pc.plans) nm += p.mtab.size();
    off = align256(off + std::max<size_t>(1, nm) * sizeof(MEntry));
    const size_t key_off = off;
    off = align256(off + std::max<size_t>(1, pc.plans.size()) * 8);
    if (off != pc.header_bytes) return MD_EINTERNAL;
    size_t mcount = 0;
    for (size_t l = 0; l < pc.plans.size(); l++) {
        const LevelPlan &p = pc.plans[l];
        BLevel L{};
        L.rows = (const uint32_t *)(header + rows_off[p.j]);
        L.h2 = (const uint32_t *)(h2 + h2_off[p.j]);
        L.mtab = p.mtab.empty() ? nullptr : (const MEntry *)(header + mt_off) + mcount;
        L.nchunks = p.nchunks;
        L.count = p.count;
        L.per_chunk = p.per_chunk;
        L.n_m = (int)p.mtab.size();
        L.g = p.g;
        L.v = p.v;
        L.base = p.base;
        L.kind = p.kind;
        L.fmax8 = p.fmax8;
        if (quota_cw_ && p.nchunks) {
            const unsigned long long per_item = std::max<unsigned long long>(1, p.count / p.nchunks);
            L.quota = std::max<unsigned long long>(1, quota_cw_ / per_item);
        }
        L.L_after = p.L_after;
        L.L_first = p.L_first;
        L.j = p.j;
        L.W = cd.gam[p.j].W;
        L.WP = cd.gam[p.j].WP;
        std::memcpy(img.data() + img_off + lev_off + l * sizeof(BLevel), &L, sizeof(BLevel));
        if (!p.mtab.empty())
            std::memcpy(img.data() + img_off + mt_off + mcount * sizeof(MEntry), p.mtab.data(),
                        p.mtab.size() * sizeof(MEntry));
        mcount += p.mtab.size();
    }
    std::memset(img.data() + img_off + key_off, 0xff, std::max<size_t>(1, pc.plans.size()) * 8);
    bc->levels = (const BLevel *)(header + lev_off);
    bc->keys = (unsigned long long *)(header + key_off);
    bc->k = k;
    bc->m = m;
    bc->nlev = (int)pc.plans.size();
    bc->live = 1;
    return MD_OK;
}

// Stream-ordered: the copies from pageable host memory are staged before the calls return,
// and the next tick on the same stream sees them.
int Engine::write_slot(int slot, const BCode &bc, const BState &bs) {
    host_codes_[slot] = bc;
    if (cudaMemcpyAsync((void *)(args_.codes + slot), &host_codes_[slot], sizeof(BCode), cudaMemcpyHostToDevice,
                        stream_) != cudaSuccess)
        return MD_ECUDA;
    if (cudaMemcpyAsync(args_.states + slot, &bs, sizeof(BState), cudaMemcpyHostToDevice, stream_) != cudaSuccess)
        return MD_ECUDA;
    return MD_OK;
}

// Build the pair tables of the given matrices (groups of up to 256 per launch).
static int build_pair_tables(const std::vector<const uint32_t *> &rp, const std::vector<uint32_t *> &hp,
                             const std::vector<int> &kk, const std::vector<int> &wp, cudaStream_t s, char *ptrs) {
    if (rp.empty()) return MD_OK;
    const size_t bytes = (size_t)2 * 256 * 8 + 2 * 256 * 4;
    int rc = MD_OK;
    for (size_t g0 = 0; g0 < rp.size() && rc == MD_OK; g0 += 256) {
        const int cnt = (int)std::min<size_t>(256, rp.size() - g0);
        std::vector<char> img(bytes, 0);
        std::memcpy(img.data(), rp.data() + g0, cnt * 8);
        std::memcpy(img.data() + 256 * 8, hp.data() + g0, cnt * 8);
        std::memcpy(img.data() + 512 * 8, kk.data() + g0, cnt * 4);
        std::memcpy(img.data() + 512 * 8 + 256 * 4, wp.data() + g0, cnt * 4);
        if (cudaMemcpy(ptrs, img.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = MD_ECUDA;
        else if (launch_h2_build_many((const uint32_t *const *)ptrs, (uint32_t *const *)(ptrs + 256 * 8),
                                      (const int *)(ptrs + 512 * 8), (const int *)(ptrs + 512 * 8 + 256 * 4), cnt,
                                      s) != 0)
            rc = MD_ECUDA;
        else if (cudaStreamSynchronize(s) != cudaSuccess)
            rc = MD_ECUDA;
    }
    return rc;
}

static void collect_pair_tables(const PreparedCode &pc, const BCode &bc, char *h2base,
                                std::vector<const uint32_t *> &rp, std::vector<uint32_t *> &hp,
                                std::vector<int> &kk, std::vector<int> &wp) {
    // the first level of each matrix j (g = 1) carries its row and pair-table pointers
    const int m = (int)pc.code.gam.size();
    size_t hoff = 0;
    for (int j = 0; j < m; j++) {
        const Gamma &gm = pc.code.gam[j];
        (void)bc;
        rp.push_back(nullptr);
        hp.push_back((uint32_t *)(h2base + hoff));
        kk.push_back(pc.code.k);
        wp.push_back(gm.WP);
        hoff = align256(hoff + (size_t)pc.code.k * (pc.code.k - 1) / 2 * gm.WP * 4 + 16);
    }
}

int Engine::load_many(const std::vector<PreparedCode *> &codes, const std::vector<int> &slots) {
    size_t hb = 0, h2b = 0;
    for (PreparedCode *p : codes) {
        hb += p->header_bytes;
        h2b += p->h2_bytes;
    }
    // one allocation: headers, pair tables, and the pointer block of the pair-table builds
    const size_t ptr_off = align256(hb + h2b);
    char *mem = (char *)dmalloc(ptr_off + (size_t)2 * 256 * 8 + 2 * 256 * 4);
    if (!mem) return MD_ENOMEM;
    shared_mem_.push_back(mem);
    std::vector<char> img(hb, 0);
    std::vector<BCode> bcs(codes.size());
    std::vector<const uint32_t *> rp;
    std::vector<uint32_t *> hp;
    std::vector<int> kk, wp;
    size_t hoff = 0, h2off = 0;
    for (size_t i = 0; i < codes.size(); i++) {
        PreparedCode &pc = *codes[i];
        int rc = fill_code(pc, mem + hoff, mem + hb + h2off, img, hoff, &bcs[i]);
        if (rc != MD_OK) return rc;
        collect_pair_tables(pc, bcs[i], mem + hb + h2off, rp, hp, kk, wp);
        // row pointers: the rows of matrix j start at the header's rows_off[j]
        size_t roff = 0;
        for (size_t j = 0; j < pc.code.gam.size(); j++) {
            rp[rp.size() - pc.code.gam.size() + j] = (const uint32_t *)(mem + hoff + roff);
            roff = align256(roff + (size_t)pc.code.k * pc.code.gam[j].WP * 4);
        }
        hoff += pc.header_bytes;
        h2off += pc.h2_bytes;
    }
    if (cudaMemcpyAsync(mem, img.data(), hb, cudaMemcpyHostToDevice, stream_) != cudaSuccess) return MD_ECUDA;
    int rc = build_pair_tables(rp, hp, kk, wp, stream_, mem + ptr_off);
    if (rc != MD_OK) return rc;
    std::vector<BState> bss(codes.size());
    for (size_t i = 0; i < codes.size(); i++) {
        bss[i] = BState{(unsigned)(codes[i]->code.n + 1), 1, 0, -1, 0, 0, 0ull, 0ull};
        host_codes_[slots[i]] = bcs[i];
    }
    // slots are contiguous in md_batch; copy them one by one in general
    for (size_t i = 0; i < codes.size(); i++) {
        if (cudaMemcpyAsync((void *)(args_.codes + slots[i]), &host_codes_[slots[i]], sizeof(BCode),
                            cudaMemcpyHostToDevice, stream_) != cudaSuccess ||
            cudaMemcpyAsync(args_.states + slots[i], &bss[i], sizeof(BState), cudaMemcpyHostToDevice, stream_) !=
                cudaSuccess)
            return MD_ECUDA;
    }
    return cudaStreamSynchronize(stream_) == cudaSuccess ? MD_OK : MD_ECUDA;
}

int Engine::load_one(PreparedCode &pc, int slot) {
    if (slot < 0 || slot >= nslots_) return MD_EINVAL;
    char *mem = nullptr;
    // stream-ordered allocation from the device's memory pool: no device-wide synchronisation
    if (cudaMallocAsync((void **)&mem, std::max<size_t>(256, pc.header_bytes + pc.h2_bytes), stream_) != cudaSuccess) {
        cudaGetLastError();
        return MD_ENOMEM;
    }
    std::vector<char> img(pc.header_bytes, 0);
    BCode bc{};
    int rc = fill_code(pc, mem, mem + pc.header_bytes, img, 0, &bc);
    if (rc != MD_OK) { cudaFreeAsync(mem, stream_); return rc; }
    if (cudaMemcpyAsync(mem, img.data(), img.size(), cudaMemcpyHostToDevice, stream_) != cudaSuccess) {
        cudaFreeAsync(mem, stream_);
        return MD_ECUDA;
    }
    size_t roff = 0, hoff = 0;
    for (const Gamma &gm : pc.code.gam) {
        if (launch_h2_build((const uint32_t *)(mem + roff), (uint32_t *)(mem + pc.header_bytes + hoff), pc.code.k,
                            gm.WP, stream_) != 0) {
            cudaFreeAsync(mem, stream_);
            return MD_ECUDA;
        }
        roff = align256(roff + (size_t)pc.code.k * gm.WP * 4);
        hoff = align256(hoff + (size_t)pc.code.k * (pc.code.k - 1) / 2 * gm.WP * 4 + 16);
    }
    own_mem_[slot] = mem;
    BState bs{(unsigned)(pc.code.n + 1), 1, 0, -1, 0, 0, 0ull, 0ull};
    return write_slot(slot, bc, bs);
}

int Engine::enqueue_ticks(int repeats) {
    bool ok = true;
    for (int r = 0; r < repeats; r++) {
        ok &= launch_engine_prepare(args_, stream_) == 0;
        launches_++;
        for (int w = 1; w < kWClasses; w++)
            if (wclass_[w]) {
                ok &= launch_engine_round(args_, w, blocks_[w], kThreads, stream_) == 0;
                launches_++;
            }
        ok &= launch_engine_post(args_, stream_) == 0;
        launches_++;
    }
    return ok ? MD_OK : MD_ECUDA;
}

int Engine::tick(int repeats, bool use_graph) {
    if (!use_graph) return enqueue_ticks(repeats);
    unsigned mask = 0;
    for (int w = 1; w < kWClasses; w++)
        if (wclass_[w]) mask |= 1u << w;
    if (!graph_ || mask != graph_mask_ || repeats != graph_repeats_) {
        if (graph_) { cudaGraphExecDestroy(graph_); graph_ = nullptr; }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MD_ECUDA;
        int rc = enqueue_ticks(repeats);
        if (cudaStreamEndCapture(stream_, &g) != cudaSuccess || rc != MD_OK) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return MD_ECUDA;
        }
        const bool ok = cudaGraphInstantiate(&graph_, g, 0) == cudaSuccess;
        cudaGraphDestroy(g);
        if (!ok) { cudaGetLastError(); graph_ = nullptr; return MD_ECUDA; }
        graph_mask_ = mask;
        graph_repeats_ = repeats;
    }
    return cudaGraphLaunch(graph_, stream_) == cudaSuccess ? MD_OK : MD_ECUDA;
}

int Engine::read_states(std::vector<BState> &out) {
    out.resize(nslots_);
    if (cudaMemcpyAsync(out.data(), args_.states, nslots_ * sizeof(BState), cudaMemcpyDeviceToHost, stream_) !=
        cudaSuccess)
        return MD_ECUDA;
    return cudaStreamSynchronize(stream_) == cudaSuccess ? MD_OK : MD_ECUDA;
}

int Engine::collect(int slot, const PreparedCode &pc, const BState &st, CodeResult *res) {
    const BCode &bc = host_codes_[slot];
    const Code &cd = pc.code;
    const int m = (int)cd.gam.size();
    std::vector<unsigned long long> keys(std::max(1, bc.nlev));
    if (cudaMemcpyAsync(keys.data(), bc.keys, keys.size() * 8, cudaMemcpyDeviceToHost, stream_) != cudaSuccess ||
        cudaStreamSynchronize(stream_) != cudaSuccess)
        return MD_ECUDA;
    res->complete = st.stop || st.last_level == cd.k * m - 1;
    const int U = (int)st.U;
    int key_level = -1;
    for (int lv = 0; lv <= st.last_level && lv < bc.nlev; lv++)
        if (keys[lv] != kNoKey && (int)(keys[lv] >> kRankBits) == U) { key_level = lv; break; }
    res->witness.assign(cd.nw64, 0);
    if (U > cd.n || key_level < 0) { res->status = MD_EINTERNAL; return MD_OK; }
    const LevelPlan &kp = pc.plans[key_level];
    std::vector<int> comb(kp.g);
    colex_unrank(keys[key_level] & (kRankLimit - 1), kp.g, cd.k, comb.data());
    for (int r : comb)
        for (int w = 0; w < cd.nw64; w++) res->witness[w] ^= cd.gam[kp.j].rows[(size_t)r * cd.nw64 + w];
    if (popcount_row(res->witness.data(), cd.nw64) != U) { res->status = MD_EINTERNAL; return MD_OK; }
    to_caller_order(cd, res->witness.data(), res->witness.data());
    res->d = U;
    res->status = MD_OK;
    if (!res->complete) {
        if (pc.g_limit < pc.g_max) res->status = MD_EAGAIN_INTERNAL;      // ran past the planned stages
        else if (pc.max_stage > 0 && pc.g_limit >= pc.max_stage) res->status = MD_EBUDGET;
        else res->status = MD_EUNSUPPORTED;
    }
    return MD_OK;
}

int Engine::release(int slot) {
    if (slot < 0 || slot >= nslots_) return MD_EINVAL;
    BCode off{};
    host_codes_[slot] = off;
    int rc = MD_OK;
    if (cudaMemcpyAsync((void *)(args_.codes + slot), &host_codes_[slot], sizeof(BCode), cudaMemcpyHostToDevice,
                        stream_) != cudaSuccess)
        rc = MD_ECUDA;
    if (own_mem_[slot]) {
        cudaFreeAsync(own_mem_[slot], stream_);      // after every kernel queued so far
        own_mem_[slot] = nullptr;
    }
    return rc;
}

void Engine::release_all() {
    if (graph_) { cudaGraphExecDestroy(graph_); graph_ = nullptr; }
    for (char *&p : own_mem_)
        if (p) { cudaFreeAsync(p, stream_); p = nullptr; }
    if (stream_) cudaStreamSynchronize(stream_);
    for (char *p : shared_mem_) dfree(p);
    shared_mem_.clear();
    dfree(tables_);
    tables_ = nullptr;
    stream_ = nullptr;                 // the stream belongs to the caller
}

}  // namespace mdl

using namespace mdl;

namespace {

// Reference schedule: one md_compute per code, in order, on the same stream.
int per_code_loop(const md_code *codes, int count, const md_options &o, int *d, uint64_t *witness, int *status) {
    size_t woff = 0;
    for (int i = 0; i < count; i++) {
        const int nw = codes[i].n > 0 ? (codes[i].n + 63) / 64 : 0;
        md_handle h = nullptr;
        md_options oi = o;
        oi.work_budget = 0;
        int rc = MD_OK;
        if (o.work_budget) {
            Code tmp;
            rc = build_code(codes[i].G, codes[i].n, codes[i].k, &tmp);
            if (rc == MD_OK && estimate_work(tmp, nullptr, nullptr) > (double)o.work_budget) rc = MD_EBUDGET;
        }
        if (rc == MD_OK) rc = md_create_ex(codes[i].G, codes[i].n, codes[i].k, &oi, &h);
        int di = -1;
        if (rc == MD_OK) {
            rc = md_compute(h, &di, witness ? witness + woff : nullptr);
            if (rc == MD_OK) {
                md_info inf;
                md_info_get(h, &inf);
                if (!inf.complete) rc = MD_EBUDGET;
            }
            md_destroy(h);
        }
        if (rc == MD_ECUDA || rc == MD_ENOMEM) return rc;
        d[i] = di;
        status[i] = rc;
        woff += nw;
    }
    return MD_OK;
}

// One code as a single-code computation (md_compute, with the tensor-core levels the options
// allow) on stream s: its status, d and witness.
int single_code_run(const md_code &c, const md_options &o, cudaStream_t s, int *d, uint64_t *witness) {
    md_options oi = o;
    oi.stream = s;
    oi.work_budget = 0;                      // the batch's budget was applied to the estimate
    md_handle h = nullptr;
    int di = -1;
    int rc = md_create_ex(c.G, c.n, c.k, &oi, &h);
    if (rc == MD_OK) rc = md_compute(h, &di, witness);
    if (rc == MD_OK) {
        md_info inf;
        md_info_get(h, &inf);
        if (!inf.complete) rc = MD_EBUDGET;    // stopped by max_stage: d is the best weight found
    }
    if (h) md_destroy(h);
    *d = rc == MD_OK || rc == MD_EBUDGET ? di : -1;
    return rc;
}

}  // namespace

extern "C" int md_batch(const md_code *codes, int count, const md_options *opt, int *d, uint64_t *witness,
                        int *status) {
    if (!codes || count < 0 || !d || !status) return MD_EINVAL;
    if (count == 0) return MD_OK;
    md_options o;
    if (opt) o = *opt; else md_options_init(&o);
    if (o.batch_mode == 1) return per_code_loop(codes, count, o, d, witness, status);
    if (o.autotune) {
        md_options base = o;
        base.autotune = 0;
        const int rc = md_batch_tune(codes, count, &base, o.tune_cache, &o);
        if (rc != MD_OK) return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) { cudaGetLastError(); return MD_ECUDA; }

    PlanOptions po;
    po.chunk_log2 = o.chunk_log2 > 0 ? o.chunk_log2 : 20;
    po.filter = o.filter;
    po.stop_rule = o.stop_rule;
    po.perm_trials = o.perm_trials;
    po.perm_seed = o.perm_seed;
    std::vector<PreparedCode> prep;
    std::vector<size_t> woffs(count);
    std::vector<PreparedCode *> ok_codes;
    std::vector<int> ok_index, heavy_index;
    std::vector<std::pair<double, int>> heavy_work;
    size_t wtot = 0;
    int rounds = 0;
    prepare_codes(codes, count, po, o.max_stage, o.work_budget, prep, status,
                  o.plan_horizon > 0 ? o.plan_horizon : 3);
    // codes whose estimated work reaches batch_heavy fill the GPU on their own: they run as
    // single-code computations (with the tensor-core levels) beside the shared schedule
    const double heavy = o.batch_heavy ? (double)o.batch_heavy : (double)kBatchHeavyDefault;
    for (int i = 0; i < count; i++) {
        woffs[i] = wtot;
        wtot += codes[i].n > 0 ? (size_t)(codes[i].n + 63) / 64 : 0;
        d[i] = -1;
        if (status[i] != MD_OK) continue;
        if (prep[i].est_work >= heavy) {
            heavy_work.emplace_back(-prep[i].est_work, i);
            prep[i] = PreparedCode();          // its plans are not needed
            continue;
        }
        ok_codes.push_back(&prep[i]);
        ok_index.push_back(i);
        rounds = std::max(rounds, (int)prep[i].plans.size());
    }
    // largest estimated work first, so that the workers finish together
    std::sort(heavy_work.begin(), heavy_work.end());
    for (const auto &hw : heavy_work) heavy_index.push_back(hw.second);
    const int nc = (int)ok_codes.size();
    if (nc == 0 && heavy_index.empty()) return MD_OK;
    // NVTX ranges (no-ops unless a profiler is attached): the batch, its shared rounds and
    // its single-code runs
    nvtxRangePushA("md_batch");
    struct RangePop {
        ~RangePop() { nvtxRangePop(); }
    } range_pop;
    cudaStream_t s = (cudaStream_t)o.stream;
    cudaStream_t own = nullptr;
    if (!s) {
        if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) return MD_ECUDA;
        s = own;
    }
    int rc = MD_OK;
    // Single-code runs on worker threads, each with a stream of its own, while this thread runs
    // the shared rounds: one code's host set-up, table builds and small levels then overlap
    // another's tensor-core levels.  With the caller's allocator they stay on this thread.
    const int nworkers = heavy_index.empty() || o.dev_alloc ? 0 : (o.batch_workers > 0 ? o.batch_workers : 2);
    std::atomic<size_t> next_heavy{0};
    std::atomic<int> heavy_rc{MD_OK};
    std::vector<std::thread> workers;
    int dev = 0;
    if (nworkers > 0 && cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); rc = MD_ECUDA; }
    for (int w = 0; rc == MD_OK && w < nworkers; w++)
        workers.emplace_back([&, dev] {
            cudaStream_t ws = nullptr;
            if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                int ok = MD_OK;
                heavy_rc.compare_exchange_strong(ok, MD_ECUDA);
                return;
            }
            nvtxRangePushA("md_batch single-code runs");
            for (;;) {
                if (heavy_rc.load() != MD_OK) break;
                const size_t h = next_heavy.fetch_add(1);
                if (h >= heavy_index.size()) break;
                const int i = heavy_index[h];
                status[i] = single_code_run(codes[i], o, ws, &d[i], witness ? witness + woffs[i] : nullptr);
                if (status[i] == MD_ECUDA || status[i] == MD_ENOMEM) {
                    int ok = MD_OK;
                    heavy_rc.compare_exchange_strong(ok, status[i]);
                }
            }
            nvtxRangePop();
            cudaStreamDestroy(ws);
        });
    if (nc > 0 && rc == MD_OK) {
        nvtxRangePushA("md_batch shared rounds");
        RangePop rounds_pop;
        Engine eng;
        eng.set_allocator(o.dev_alloc, o.dev_free, o.alloc_ctx);
        rc = eng.init(nc, s, 0, o.blocks_per_sm);
        std::vector<int> slots(nc);
        for (int i = 0; i < nc; i++) slots[i] = i;
        if (rc == MD_OK) rc = eng.load_many(ok_codes, slots);
        // one level of every code per tick: as many ticks as the longest plan
        if (rc == MD_OK && o.use_graph) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            for (int r = 0; ok && r < rounds; r++) ok = eng.tick() == MD_OK;
            if (cudaStreamEndCapture(s, &graph) != cudaSuccess) ok = false;
            if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
            if (ok) ok = cudaGraphLaunch(exec, s) == cudaSuccess;
            if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (!ok) { cudaGetLastError(); rc = MD_ECUDA; }
        } else if (rc == MD_OK) {
            for (int r = 0; rc == MD_OK && r < rounds; r++) rc = eng.tick();
            if (rc == MD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = MD_ECUDA;
        }
        std::vector<BState> st;
        if (rc == MD_OK) rc = eng.read_states(st);
        for (int c = 0; rc == MD_OK && c < nc; c++) {
            CodeResult res;
            rc = eng.collect(c, *ok_codes[c], st[c], &res);
            const int i = ok_index[c];
            if (res.status == MD_EAGAIN_INTERNAL) {
                // rare: the run went past the planned stages; finish it as a single code
                status[i] = single_code_run(codes[i], o, s, &d[i], witness ? witness + woffs[i] : nullptr);
                continue;
            }
            status[i] = res.status;
            if (res.status == MD_OK || res.status == MD_EBUDGET || res.status == MD_EUNSUPPORTED) {
                d[i] = res.d;
                if (witness) std::memcpy(witness + woffs[i], res.witness.data(), res.witness.size() * 8);
            }
        }
    }
    if (rc != MD_OK) {
        int ok = MD_OK;
        heavy_rc.compare_exchange_strong(ok, rc);             // the workers take no further code
    }
    for (std::thread &t : workers) t.join();
    if (rc == MD_OK) rc = heavy_rc.load();
    size_t ran = std::min(next_heavy.load(), heavy_index.size());     // single-code runs started
    if (nworkers == 0 && !heavy_index.empty()) {
        nvtxRangePushA("md_batch single-code runs");
        for (; rc == MD_OK && ran < heavy_index.size(); ran++) {
            const int i = heavy_index[ran];
            status[i] = single_code_run(codes[i], o, s, &d[i], witness ? witness + woffs[i] : nullptr);
            if (status[i] == MD_ECUDA || status[i] == MD_ENOMEM) rc = status[i];
        }
        nvtxRangePop();
    }
    // after a failure, the codes no run reached carry the batch's status
    for (; ran < heavy_index.size(); ran++) status[heavy_index[ran]] = rc;
    if (own) cudaStreamDestroy(own);
    if (rc == MD_OK && bounds_status() != MD_OK) rc = MD_EINTERNAL;      // the debug build's range checks
    return rc;
}
