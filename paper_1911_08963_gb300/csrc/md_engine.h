// md_engine.h -- host side of the multi-code engine shared by md_batch and the server.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "md_internal.h"

namespace mdl {

// A code ready for the engine: Gamma matrices and the plans of every level it may run.
struct PreparedCode {
    Code code;
    std::vector<LevelPlan> plans;   // level l = (g - 1) * m + j
    int g_limit = 0;                // stages planned
    int g_max = 0;                  // deepest stage that could be planned (C(k, g) < 2^55)
    int max_stage = 0;
    size_t header_bytes = 0;        // rows, level table, work tables, keys
    size_t h2_bytes = 0;            // pair tables
    double est_work = 0.0;          // estimated combinations until L >= U (estimate_work)
};

// Validate G, build the Gamma_j, check the work budget (estimated combinations) and plan
// the levels up to `horizon` stages past the estimated stopping stage (0 = every stage that
// can be planned).  Returns an MD_* status for this code.
int prepare_code(const uint64_t *G, int n, int k, const PlanOptions &po, int max_stage, uint64_t budget,
                 PreparedCode *out, int horizon = 3);

// Prepare many codes on all host cores.
void prepare_codes(const md_code *codes, int count, const PlanOptions &po, int max_stage, uint64_t budget,
                   std::vector<PreparedCode> &out, int *status, int horizon = 3);

// Per-code outcome read back from the engine.
struct CodeResult {
    int status = MD_OK;
    int d = -1;
    bool complete = false;
    std::vector<uint64_t> witness;
};

class Engine {
  public:
    Engine() = default;
    ~Engine();
    Engine(const Engine &) = delete;
    Engine &operator=(const Engine &) = delete;

    // Slot tables for up to nslots resident codes; quota = combinations a code may enumerate
    // per tick, rounded to whole work items (0 = a whole level per tick).
    int init(int nslots, cudaStream_t stream, unsigned long long quota, int blocks_per_sm_cap);

    // Place codes in slots with one device allocation for all of them (owned by the
    // engine until release_all).  Uploads rows and tables, builds pair tables.
    int load_many(const std::vector<PreparedCode *> &codes, const std::vector<int> &slots);
    // Place one code in a slot with its own device allocation (released by release).
    int load_one(PreparedCode &code, int slot);

    // Enqueue `repeats` ticks (prepare, one round per row width present, post), as one
    // captured CUDA graph when use_graph is set (re-captured when the set of row widths
    // present changes).
    int tick(int repeats = 1, bool use_graph = false);
    // Copy the slot states to the host (synchronises the stream).
    int read_states(std::vector<BState> &out);
    // Result of the code in `slot` (its keys are read back); state from read_states.
    int collect(int slot, const PreparedCode &code, const BState &st, CodeResult *res);
    // Free a slot (and its own allocation, if load_one placed it).
    int release(int slot);
    void release_all();

    // Device allocations of init and load_many through the caller's allocator (md_options
    // dev_alloc / dev_free); set before init.  Unset: cudaMalloc / cudaFree.
    void set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx) {
        alloc_ = alloc;
        free_ = release;
        alloc_ctx_ = ctx;
    }

    int nslots() const { return nslots_; }
    cudaStream_t stream() const { return stream_; }
    int launches() const { return launches_; }
    void set_wclass(int W) { wclass_[W] = true; }

  private:
    int write_slot(int slot, const BCode &bc, const BState &bs);
    int fill_code(PreparedCode &pc, char *header, char *h2, std::vector<char> &img, size_t img_off,
                  BCode *bc);
    cudaStream_t stream_ = nullptr;
    int nslots_ = 0;
    char *tables_ = nullptr;
    EngineArgs args_{};
    std::vector<char *> own_mem_;   // per slot, allocations made by load_one
    std::vector<char *> shared_mem_;
    bool wclass_[kWClasses] = {false};
    int blocks_[kWClasses] = {0};
    int launches_ = 0;
    int sms_ = 0;
    int cap_ = 0;
    unsigned long long quota_cw_ = 0;
    cudaGraphExec_t graph_ = nullptr;
    unsigned graph_mask_ = 0;
    int graph_repeats_ = 0;
    int enqueue_ticks(int repeats);
    void *dmalloc(size_t bytes);
    void dfree(void *p);
    std::vector<BCode> host_codes_;
    void *(*alloc_)(size_t, void *) = nullptr;
    void (*free_)(void *, void *) = nullptr;
    void *alloc_ctx_ = nullptr;
};

}  // namespace mdl
