// md_server.cpp -- continuous-batching server on the multi-code engine.
//
// Submissions are validated and planned on the caller's thread (so errors come back at
// once), then queued.  One worker thread owns the GPU stream: between ticks it admits
// queued codes into free slots while their estimated device memory fits the budget, runs
// eight ticks (in each, every resident code advances by up to ~2^28 combinations of its
// current level, and by at most one level),
// reads the slot states back, and retires codes whose run has finished.  Codes admitted in
// the middle of another code's run share every following tick with it, so their work
// overlaps on the device; results are identical to md_compute because every code's bounds,
// level order and records are its own.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <thread>

#include "md_engine.h"

using namespace mdl;

namespace {

struct Request {
    uint64_t ticket = 0;
    std::unique_ptr<PreparedCode> code;
    size_t bytes = 0;
};

struct Done {
    int status = MD_OK;
    int d = -1;
    std::vector<uint64_t> witness;
};

}  // namespace

constexpr int kTicksPerRound = 8;

struct md_server {
    md_server_opts opts{};
    Engine eng;
    cudaStream_t own = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    std::map<int, Request> resident;          // slot -> request
    std::map<uint64_t, Done> done;
    std::set<uint64_t> live;                  // submitted and not yet returned by a poll
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0;
    int fatal = MD_OK;
    PlanOptions po;

    void run();
};

void md_server::run() {
    std::vector<BState> st;
    std::vector<int> free_slots;
    for (int s = opts.slots - 1; s >= 0; s--) free_slots.push_back(s);
    while (!stop.load()) {
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (resident.empty() && pending.empty()) {
                cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            // admission: free slot and memory budget (a code that fits alone is always admitted
            // when nothing else is resident)
            while (!pending.empty() && admit.size() < free_slots.size()) {
                Request &r = pending.front();
                if (bytes_in_use + r.bytes > opts.device_bytes && !(resident.empty() && admit.empty())) break;
                bytes_in_use += r.bytes;
                admit.push_back(std::move(r));
                pending.pop_front();
            }
        }
        for (Request &r : admit) {
            const int slot = free_slots.back();
            free_slots.pop_back();
            int rc = eng.load_one(*r.code, slot);
            if (rc != MD_OK) {
                std::lock_guard<std::mutex> lk(mu);
                Done d;
                d.status = rc;
                done[r.ticket] = std::move(d);
                bytes_in_use -= r.bytes;
                free_slots.push_back(slot);
                if (rc == MD_ECUDA) fatal = rc;
                continue;
            }
            std::lock_guard<std::mutex> lk(mu);
            resident[slot] = std::move(r);
        }
        if (resident.empty()) continue;
        // eight ticks per host round trip, one graph launch: a code with small levels moves
        // through up to eight levels between two looks from the host
        if (eng.tick(kTicksPerRound, true) != MD_OK || eng.read_states(st) != MD_OK) {
            std::lock_guard<std::mutex> lk(mu);
            fatal = MD_ECUDA;
            for (auto &kv : resident) { Done d; d.status = MD_ECUDA; done[kv.second.ticket] = std::move(d); }
            resident.clear();
            return;
        }
        std::vector<int> finished;
        for (auto &kv : resident) {
            const int s = kv.first;
            const PreparedCode &pc = *kv.second.code;
            if (st[s].stop || st[s].cur >= (int)pc.plans.size()) finished.push_back(s);
        }
        for (int s : finished) {
            // only this thread modifies `resident`, so reading it without the lock is safe
            const Request &r = resident[s];
            CodeResult res;
            int rc = eng.collect(s, *r.code, st[s], &res);
            eng.release(s);
            if (rc == MD_OK && res.status == MD_EAGAIN_INTERNAL) {
                // rare: the run went past the planned stages; finish it as a single code
                const Code &cd = r.code->code;
                md_options oi;
                md_options_init(&oi);
                oi.stream = eng.stream();
                md_handle h = nullptr;
                int di = -1;
                res.witness.assign(cd.nw64, 0);
                int r2 = md_create_ex(cd.G.data(), cd.n, cd.k, &oi, &h);
                if (r2 == MD_OK) r2 = md_compute(h, &di, res.witness.data());
                if (h) md_destroy(h);
                res.status = r2;
                res.d = r2 == MD_OK ? di : -1;
            }
            free_slots.push_back(s);
            Done d;
            d.status = rc != MD_OK ? rc : res.status;
            d.d = res.d;
            d.witness = std::move(res.witness);
            std::lock_guard<std::mutex> lk(mu);
            bytes_in_use -= r.bytes;
            done[r.ticket] = std::move(d);
            resident.erase(s);
        }
    }
}

extern "C" {

int md_server_create(const md_server_opts *opts, md_server **out) {
    if (!out) return MD_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) { cudaGetLastError(); return MD_ECUDA; }
    md_server *s = new (std::nothrow) md_server();
    if (!s) return MD_ENOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.slots <= 0) s->opts.slots = 64;
    if (s->opts.device_bytes == 0) s->opts.device_bytes = (size_t)256 << 20;
    cudaStream_t stream = (cudaStream_t)s->opts.stream;
    if (!stream) {
        if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess) { delete s; return MD_ECUDA; }
        stream = s->own;
    }
    // small work items keep the idle tail at the end of every tick short
    s->po.chunk_log2 = 16;
    s->po.stop_rule = s->opts.stop_rule;
    // time slice: about 2^28 combinations of each resident code per tick (a fraction of a
    // millisecond of the whole GPU per code), so codes that arrive wait at most a few ticks
    int rc = s->eng.init(s->opts.slots, stream, 1ull << 28, 0);
    if (rc != MD_OK) {
        if (s->own) cudaStreamDestroy(s->own);
        delete s;
        return rc;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return MD_OK;
}

int md_server_submit(md_server *s, const uint64_t *G, int n, int k, uint64_t *ticket) {
    if (!s || !G || !ticket) return MD_EINVAL;
    Request r;
    r.code.reset(new (std::nothrow) PreparedCode());
    if (!r.code) return MD_ENOMEM;
    int rc = prepare_code(G, n, k, s->po, 0, s->opts.work_budget, r.code.get());
    if (rc != MD_OK) return rc;
    r.bytes = r.code->header_bytes + r.code->h2_bytes;
    if (r.bytes > s->opts.device_bytes) return MD_ENOMEM;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != MD_OK) return s->fatal;
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    s->live.insert(r.ticket);
    s->pending.push_back(std::move(r));
    s->cv.notify_one();
    return MD_OK;
}

int md_server_poll(md_server *s, uint64_t ticket, int *d, uint64_t *witness, int *status) {
    if (!s || !d || !status) return MD_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return s->live.count(ticket) ? MD_EBUSY : MD_EINVAL;
    *d = it->second.d;
    *status = it->second.status;
    if (witness) std::memcpy(witness, it->second.witness.data(), it->second.witness.size() * 8);
    s->done.erase(it);
    s->live.erase(ticket);
    return MD_OK;
}

void md_server_destroy(md_server *s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    s->eng.release_all();
    if (s->own) cudaStreamDestroy(s->own);
    delete s;
}

}  // extern "C"
