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
    mpdp_mlp* model = nullptr;  // learned proposal (UnionDP edge order); nullptr: plain
};

// Features of every edge (i, j) of a graph for the learned proposal, in edge
// order, kEdgeFeatures floats each.  lcard: log2 card of each node; lsel:
// log2 sel of each edge.
constexpr int kEdgeFeatures = 12;
double xd_log2(XD x);
void edge_features(int n, const std::vector<double>& lcard, const std::vector<int>& eu, const std::vector<int>& ev,
                   const std::vector<double>& lsel, std::vector<float>& out);

struct HeuristicResult {
    std::vector<mpdp_plan_node> nodes;  // breadth-first, node 0 = root
    XD cost;
    int subproblems = 0;                // exact sub-problems solved on the device
    bool learned_won = false;           // UnionDP-learned: the learned plan beat the plain one
};

int run_heuristic(const HeuristicQuery& q, XdExecutor& ex, cudaStream_t st, int num_sms, HeuristicResult& res);

}  // namespace mpdp
