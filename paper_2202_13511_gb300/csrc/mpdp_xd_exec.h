// Host interface of the extended-range (XD) exact DP over heuristic
// sub-problems: a batch of sub-problems in, the chosen plan of each out.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "mpdp_device.cuh"
#include "mpdp_xd.cuh"

namespace mpdp {

constexpr int kXdMaxRels = 25;                    // relations of one sub-problem
constexpr size_t kXdBatchMemoBytes = (size_t)8 << 30;  // XD memo bytes of one device batch

// Per query, device side: cards and neighbour selectivities in XD (the
// nsel layout of DevQuery).
struct XdExtra {
    XD card[kMaxRels];
    XD nsel[2 * kMaxEdges];
};

// Per query, the plan read back: nodes in breadth-first order from the full
// set (children of node i at left[i], right[i]; -1 for a relation).
struct XdPlanOut {
    XD cost;
    int32_t status;
    int32_t n_nodes;
    uint32_t set[kPlanNodes];
    int32_t left[kPlanNodes];
    int32_t right[kPlanNodes];
};

// One sub-problem: n relations with XD cards, edges u < v with XD sels.
struct XdSubQuery {
    int n = 0;
    std::vector<XD> card;
    std::vector<int32_t> eu, ev;
    std::vector<XD> sel;
};

struct XdSubPlan {
    XD cost;
    std::vector<uint32_t> set;
    std::vector<int32_t> left, right;
};

// Device buffers kept across calls (grown on demand).
class XdExecutor {
public:
    ~XdExecutor();
    // Solve every sub-problem; plans come back in input order.
    int run(const std::vector<XdSubQuery>& qs, std::vector<XdSubPlan>& out, cudaStream_t st, int num_sms);

private:
    int run_batch(const std::vector<XdSubQuery>& qs, size_t b0, size_t b1, std::vector<XdSubPlan>& out,
                  cudaStream_t st, int num_sms);
    void* fixed_ = nullptr;
    void* host_ = nullptr;
    void* var_ = nullptr;
    size_t var_bytes_ = 0;
};

}  // namespace mpdp
