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
//
// Requests whose estimated work reaches the heavy threshold do not enter the slots: a second
// worker thread runs them one at a time as single-code computations (md_compute, whose large
// levels run on the tensor cores) on a stream of the server's own, so their levels neither
// stretch the shared ticks nor wait behind them.  A slot code that runs past its planned
// stages is handed to the same thread.
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
    std::unique_ptr<PreparedCode> code;   // slot requests only
    size_t bytes = 0;
    std::vector<uint64_t> G;              // the caller's rows, for a single-code run
    int n = 0, k = 0;
};

struct Done {
    int status = MD_OK;
    int d = -1;
    std::vector<uint64_t> witness;
};

}  // namespace

constexpr int kTicksPerRound = 8;
// Default heavy threshold: from about 10^9 estimated combinations a code fills the GPU on its
// own for long enough that running it alone is quicker than sharing ticks; on a Poisson
// stream of codes n = 64..200 it gave the lowest latencies of 10^8..3*10^9 (the spread was
// a few percent).
constexpr uint64_t kServeHeavyDefault = 1ull << 30;

struct md_server {
    md_server_opts opts{};
    Engine eng;
    cudaStream_t own = nullptr;
    cudaStream_t heavy_stream = nullptr;
    int device = 0;                           // the creating thread's device, made current in both workers
    std::thread worker, heavy_worker;
    std::mutex mu;
    std::condition_variable cv, heavy_cv;
    std::deque<Request> pending;
    std::deque<Request> heavy_queue;          // single-code runs, in submission order
    volatile int heavy_cancel = 0;            // set by md_server_destroy: ends a running one
    std::map<int, Request> resident;          // slot -> request
    std::map<uint64_t, Done> done;
    std::set<uint64_t> live;                  // submitted and not yet returned by a poll
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0;
    int fatal = MD_OK;
    PlanOptions po;

    void run();
    void run_heavy();
    void to_heavy(Request &&r);
};

// One request as a single-code computation on stream `st`.
static Done single_code(const Request &r, cudaStream_t st, int stop_rule, volatile int *cancel) {
    md_options oi;
    md_options_init(&oi);
    oi.stream = st;
    oi.stop_rule = stop_rule;
    oi.cancel_flag = cancel;
    Done d;
    d.witness.assign((size_t)(r.n + 63) / 64, 0);
    md_handle h = nullptr;
    int di = -1;
    int rc = md_create_ex(r.G.data(), r.n, r.k, &oi, &h);
    if (rc == MD_OK) rc = md_compute(h, &di, d.witness.data());
    if (h) md_destroy(h);
    d.status = rc;
    d.d = rc == MD_OK ? di : -1;
    return d;
}

void md_server::to_heavy(Request &&r) {
    std::lock_guard<std::mutex> lk(mu);
    heavy_queue.push_back(std::move(r));
    heavy_cv.notify_one();
}

void md_server::run_heavy() {
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(mu);
        fatal = MD_ECUDA;
        return;
    }
    for (;;) {
        Request r;
        {
            std::unique_lock<std::mutex> lk(mu);
            heavy_cv.wait(lk, [&] { return stop.load() || fatal != MD_OK || !heavy_queue.empty(); });
            if (stop.load() || fatal != MD_OK) return;     // after a failed CUDA call: no more work
            r = std::move(heavy_queue.front());
            heavy_queue.pop_front();
        }
        Done d = single_code(r, heavy_stream, opts.stop_rule, &heavy_cancel);
        std::lock_guard<std::mutex> lk(mu);
        if (d.status == MD_ECUDA) {
            fatal = MD_ECUDA;
            cv.notify_all();
        }
        done[r.ticket] = std::move(d);
    }
}

void md_server::run() {
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(mu);
        fatal = MD_ECUDA;
        return;
    }
    std::vector<BState> st;
    std::vector<int> free_slots;
    for (int s = opts.slots - 1; s >= 0; s--) free_slots.push_back(s);
    while (!stop.load()) {
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (fatal != MD_OK) {
                // a CUDA call failed (in either worker): finish what is resident with that error
                for (auto &kv : resident) { Done d; d.status = fatal; done[kv.second.ticket] = std::move(d); }
                resident.clear();
                return;
            }
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
                if (rc == MD_ECUDA) {
                    fatal = rc;
                    heavy_cv.notify_all();
                }
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
            heavy_cv.notify_all();
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
            Request &r = resident[s];
            CodeResult res;
            int rc = eng.collect(s, *r.code, st[s], &res);
            eng.release(s);
            free_slots.push_back(s);
            if (rc == MD_OK && res.status == MD_EAGAIN_INTERNAL) {
                // rare: the run went past the planned stages; it is finished as a single code
                Request h;
                h.ticket = r.ticket;
                h.G = std::move(r.G);
                h.n = r.n;
                h.k = r.k;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    bytes_in_use -= r.bytes;
                    resident.erase(s);
                }
                to_heavy(std::move(h));
                continue;
            }
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
    if (cudaGetDevice(&s->device) != cudaSuccess) { cudaGetLastError(); delete s; return MD_ECUDA; }
    if (s->opts.slots <= 0) s->opts.slots = 64;
    if (s->opts.device_bytes == 0) s->opts.device_bytes = (size_t)256 << 20;
    cudaStream_t stream = (cudaStream_t)s->opts.stream;
    if (!stream) {
        if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess) { delete s; return MD_ECUDA; }
        stream = s->own;
    }
    s->opts.heavy = s->opts.heavy ? s->opts.heavy : kServeHeavyDefault;
    if (cudaStreamCreateWithFlags(&s->heavy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        if (s->own) cudaStreamDestroy(s->own);
        delete s;
        return MD_ECUDA;
    }
    // small work items keep the idle tail at the end of every tick short
    s->po.chunk_log2 = 16;
    s->po.stop_rule = s->opts.stop_rule;
    // time slice: about 2^28 combinations of each resident code per tick (a fraction of a
    // millisecond of the whole GPU per code), so codes that arrive wait at most a few ticks
    int rc = s->eng.init(s->opts.slots, stream, 1ull << 28, 0);
    if (rc != MD_OK) {
        if (s->own) cudaStreamDestroy(s->own);
        cudaStreamDestroy(s->heavy_stream);
        delete s;
        return rc;
    }
    s->worker = std::thread([s] { s->run(); });
    s->heavy_worker = std::thread([s] { s->run_heavy(); });
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
    r.n = n;
    r.k = k;
    r.G.assign(G, G + (size_t)k * ((n + 63) / 64));
    const bool heavy = s->opts.heavy != UINT64_MAX && r.code->est_work >= (double)s->opts.heavy;
    if (heavy) {
        r.code.reset();
    } else {
        r.bytes = r.code->header_bytes + r.code->h2_bytes;
        if (r.bytes > s->opts.device_bytes) return MD_ENOMEM;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != MD_OK) return s->fatal;
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    s->live.insert(r.ticket);
    if (heavy) {
        s->heavy_queue.push_back(std::move(r));
        s->heavy_cv.notify_one();
    } else {
        s->pending.push_back(std::move(r));
        s->cv.notify_one();
    }
    return MD_OK;
}

int md_server_poll(md_server *s, uint64_t ticket, int *d, uint64_t *witness, int *status) {
    if (!s || !d || !status) return MD_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (!s->live.count(ticket)) return MD_EINVAL;
        if (s->fatal == MD_OK) return MD_EBUSY;
        // the workers stopped taking work after a failed CUDA call: report it for this ticket
        *d = -1;
        *status = s->fatal;
        s->live.erase(ticket);
        return MD_OK;
    }
    *d = it->second.d;
    *status = it->second.status;
    if (witness) std::memcpy(witness, it->second.witness.data(), it->second.witness.size() * 8);
    s->done.erase(it);
    s->live.erase(ticket);
    return MD_OK;
}

void md_server_destroy(md_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
        s->heavy_cancel = 1;                  // a running single-code computation ends early
    }
    s->cv.notify_all();
    s->heavy_cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->heavy_worker.joinable()) s->heavy_worker.join();
    s->eng.release_all();
    if (s->own) cudaStreamDestroy(s->own);
    if (s->heavy_stream) cudaStreamDestroy(s->heavy_stream);
    delete s;
}

}  // extern "C"
