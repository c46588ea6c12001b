// Host-side view of a batch launch: plan (grid sizes) and launch sequence.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>

#include "mpdp_device.cuh"

namespace mpdp {

// Grid sizing of one batch, computed on the host from the queries' sizes.
// One evaluated CCP pair of the unfused ablation path: (x, left) as the
// fused kernels fold them (x = bit pattern of cost(S_l) + cost(S_r)).
struct PairRec {
    unsigned long long x;
    uint32_t left;
    uint32_t pad;
};

struct BatchPlan {
    int num_sms = 152;
    int blocks_per_sm = 8;  // eval grids: 8 x 256 threads = a full SM's worth of warps
    uint32_t filter_blocks = 0;     // bitmap / unrank filter blocks
    uint32_t connected_blocks = 0;  // k_filter_connected grid (tree queries in mode CONNECTED)
    uint32_t group_threads = 1u << 18;  // tree levels: groups of lanes while sets x G <= this (0: never)
    PairRec* pairs = nullptr;  // non-null: tree levels run unfused (evaluate, then prune + scatter)
    uint32_t* level_pref = nullptr;  // [2][kLevels][kMaxBatch + 1]: per-level tile prefix, tree then block mode
    bool block_lists = false;  // some block-mode query of the lane has block CCP lists
    unsigned long long tree_tiles[kLevels] = {};   // upper bound of level-k tiles, tree queries
    unsigned long long block_tiles[kLevels] = {};  // same, block-mode queries
    unsigned long long block_sets[kLevels] = {};   // upper bound of level-k heavy tiles (8 chunks), block-mode queries
};

// Hook around every kernel launch (profiling mode): begin/end are called on
// the host right before and after the launch of a kernel of class `cls`.
struct LaunchHook {
    virtual ~LaunchHook() {}
    virtual void begin(int cls, cudaStream_t st) = 0;
    virtual void end(int cls, cudaStream_t st) = 0;
};

unsigned long long binom_host(int n, int k);
// Pair records the unfused tree path needs for a plan: the largest level's
// tiles x 256 sets x (k - 1) pairs.
unsigned long long unfused_pair_records(const BatchPlan& bp);
size_t list_entries(int n);
// words of a block-mode query's connectivity bitmap (2^n bits, at least one word)
size_t conn_words(int n);
// Per-kernel attributes set once per context (the shared-memory carveout of
// the tree evaluate); no device-wide setting is touched.
cudaError_t configure_kernels();
// List words of a query's block CCP lists (0 when it has none).
size_t block_list_words(int n, int enumeration);
// Find-Blocks cache words of a query (block mode; after the block CCP lists).
size_t fb_cache_words(int n, int enumeration);
size_t hash_arena_slots(int n);
// Per-level list offsets and filter warp ranges of one query; returns the
// query's filter block count in filter_blocks.
void fill_levels(QDesc& d, int run, int filter_mode, uint32_t& filter_blocks);

cudaError_t enqueue_pipeline(const BatchArgs& a, const BatchPlan& bp, int memo_kind, cudaStream_t st,
                             int* launches, LaunchHook* hook = nullptr);
cudaError_t enqueue_stage_device(const BatchArgs& a, const double* card, const mpdp_edge* edges,
                                 cudaStream_t st, LaunchHook* hook = nullptr);
cudaError_t enqueue_publish(const BatchArgs& a, mpdp_plan_node* nodes, double* cost, int32_t* status,
                            cudaStream_t st, LaunchHook* hook = nullptr);
cudaError_t enqueue_memo_lookup(const BatchArgs& a, int memo_kind, int qi, const uint32_t* d_sets,
                                int count, double* d_costs, uint32_t* d_lefts, cudaStream_t st);

// Ingest and the bitmap filter only (validation, tables, the connected sets
// of every level): the structure any arithmetic can then evaluate.
cudaError_t enqueue_structure(const BatchArgs& a, const BatchPlan& bp, cudaStream_t st);

// Device workspace (bytes) a context needs for one batch of these queries
// under configuration cfg; defined with the context code.
size_t batch_workspace_bytes(const int* n, const int* m, int count, const mpdp_config& cfg);
// The host-side checks mpdp_optimize_batch applies to each query (exact mode).
int validate_host_query(const mpdp_query* q);

}  // namespace mpdp
