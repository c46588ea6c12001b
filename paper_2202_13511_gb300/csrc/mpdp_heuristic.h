// Host interface of the heuristic modes (IDP2, UnionDP; Sec. 4).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/mpdp.h"
#include "mpdp_xd.cuh"

namespace mpdp {

class XdExecutor;

struct HeuristicQuery {
    int n = 0;
    int mode = MPDP_MODE_IDP2;
    int k = 25;  // sub-problem size (IDP2: k <= 1 gives GOO's plan)
    int t = 0;   // UnionDP partition threshold (0: k)
    const double* card = nullptr;
    std::vector<int> eu, ev;
    std::vector<double> sel;
};

struct HeuristicResult {
    std::vector<mpdp_plan_node> nodes;  // breadth-first, node 0 = root
    XD cost;
    int subproblems = 0;                // exact sub-problems solved on the device
};

int run_heuristic(const HeuristicQuery& q, XdExecutor& ex, cudaStream_t st, int num_sms, HeuristicResult& res);

}  // namespace mpdp
