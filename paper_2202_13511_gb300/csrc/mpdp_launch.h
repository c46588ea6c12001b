// Host-side view of the device workspace and the launch sequence of one query.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>

#include "mpdp_device.cuh"

namespace mpdp {

// Device buffers of one query slot.  All pointers are device memory.
struct Workspace {
    int n_cap = 0;                 // largest n the buffers were sized for
    int memo_kind = MPDP_MEMO_DENSE;
    StagedQuery* staged = nullptr;
    DevQuery* query = nullptr;
    DevCounters* counters = nullptr;
    DevResult* result = nullptr;
    uint32_t* lists = nullptr;     // per level k: C(n,k) slots (connected k-sets)
    uint32_t* heavy = nullptr;     // per level k: C(n,k) slots (heavy k-sets)
    double* dcost = nullptr;       // dense memo: cost[S], S < 2^n
    uint32_t* dleft = nullptr;     // dense memo: left[S]
    HashSlot* arena = nullptr;     // hash memo slots
    unsigned long long arena_slots = 0;
    HashLayout* layout = nullptr;
};

struct PipelineCfg {
    int n = 0;
    int enumeration = MPDP_ENUM_TREE;  // resolved: TREE or BLOCKS
    int memo_kind = MPDP_MEMO_DENSE;
    int heavy_threshold = 64;
    int use_ccc = 1;
    int run_length = 32;
    int num_sms = 152;
    int blocks_per_sm = 4;
};

// Parameters of the unrank + filter launch (passed by value).
struct FilterParams {
    int n;
    int run;                              // consecutive ranks per lane (<= 32)
    uint32_t nranks[kLevels];             // C(n, k)
    uint32_t warp_begin[kLevels + 1];     // first warp of level k
    uint32_t list_off[kLevels];           // level k's region in the list buffer
};

// Hook around every kernel launch (profiling mode): begin/end are called on
// the host right before and after the launch of a kernel of class `cls`.
struct LaunchHook {
    virtual ~LaunchHook() {}
    virtual void begin(int cls, cudaStream_t st) = 0;
    virtual void end(int cls, cudaStream_t st) = 0;
};

void level_layout(int n, uint32_t* list_off);
size_t list_entries(int n);
size_t hash_arena_slots(int n);

cudaError_t enqueue_pipeline(const Workspace& ws, const PipelineCfg& pc, cudaStream_t st,
                             int* launches, LaunchHook* hook = nullptr);
cudaError_t enqueue_stage_device(const double* card, const mpdp_edge* edges, int n, int m,
                                 int cost_model, StagedQuery* staged, cudaStream_t st,
                                 LaunchHook* hook = nullptr);
cudaError_t enqueue_publish(const Workspace& ws, mpdp_plan_node* nodes, double* cost,
                            int32_t* status, cudaStream_t st, LaunchHook* hook = nullptr);
cudaError_t enqueue_memo_lookup(const Workspace& ws, int memo_kind, const uint32_t* d_sets,
                                int count, double* d_costs, uint32_t* d_lefts, cudaStream_t st);

}  // namespace mpdp
