// Allocation-free exact optimization of one small query (n <= 16).
//
// The whole DP of one query runs in one kernel of one block: ingest and
// validation, base fill, levels 2..n (a block barrier between levels is the
// level barrier of Sec. 2.1.1), and the plan fetch.  Each level scans every
// bitmap, keeps the connected k-subsets, and evaluates each one with a warp:
// Find-Blocks, the unordered block bipartitions of Algorithm 4, the CCP test,
// grow, and the (x, left) prune of the batched kernels, so the results are
// bit-identical to theirs.  The dense memo lives in a fixed device array of
// this file; the library allocates nothing for it.  Calls whose kernels can
// overlap on the GPU (other streams, unordered host threads) share that
// array and race: order them on one stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "mpdp_device.cuh"

namespace mpdp {
namespace {

constexpr int kNoAllocRels = MPDP_NOALLOC_MAX_RELS;
constexpr uint32_t kNoAllocSets = 1u << kNoAllocRels;
constexpr int kNoAllocThreads = 512;
constexpr int kNoAllocWarps = kNoAllocThreads / 32;
constexpr size_t kNoAllocCcBytes = sizeof(double2) * kNoAllocSets;                // {cost, card}[S]
constexpr size_t kNoAllocBytes = kNoAllocCcBytes + sizeof(uint32_t) * kNoAllocSets;  // + left[S]
static_assert(kNoAllocBytes == MPDP_NOALLOC_SCRATCH_BYTES, "scratch size in the header");

// The memo: {cost, card} of S at entry S, then left(S) at entry S.  Nothing
// in it has to start at zero: a call writes the base entries first, and
// every set it reads was written earlier in the same call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Dense memo over the scratch with plain (coherent) loads: the entries are
// written and read by the same block within one kernel, ordered by its
// barriers, so the read-only data path may not be used.
struct ScratchMemo {
    double2* cc;
    uint32_t* left;

    __device__ __forceinline__ double get_cost(uint32_t s, DevCounters*) const { return cc[s].x; }
    __device__ __forceinline__ double get_card(uint32_t s, DevCounters*) const { return cc[s].y; }
    __device__ __forceinline__ void get(uint32_t s, double& c, double& cd, uint32_t& l, DevCounters*) const
    {
        const double2 v = cc[s];
        c = v.x;
        cd = v.y;
        l = left[s];
    }
    __device__ __forceinline__ void put(uint32_t s, int, double c, double cd, uint32_t l, DevCounters*)
    {
        cc[s] = make_double2(c, cd);
        left[s] = l;
    }
};

// Validation and adjacency as in the batched ingest (same checks, same
// status codes), into shared memory.
__device__ int ingest_one(int n, int m, const double* __restrict__ card, const mpdp_edge* __restrict__ edges,
                          SharedQuery& sq)
{
    if (n < 1 || n > kNoAllocRels) return MPDP_ERR_TOO_LARGE;
    if (m < 0 || m > n * (n - 1) / 2) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        const double c = card[i];
        if (!(c > 0.0) || !(c <= 1.7976931348623157e308)) return MPDP_ERR_INVALID_ARG;
    }
    uint32_t adj[kMaxRels];
    for (int i = 0; i < kMaxRels; i++) adj[i] = 0u;
    for (int e = 0; e < m; e++) {
        const int u = edges[e].u, v = edges[e].v;
        const double s = edges[e].sel;
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(s > 0.0) || !(s <= 1.0) || (adj[u] >> v & 1u))
            return MPDP_ERR_INVALID_ARG;
        adj[u] |= 1u << v;
        adj[v] |= 1u << u;
    }
    const uint32_t full = (1u << n) - 1u;
    if (grow(1u, full, adj) != full) return MPDP_ERR_DISCONNECTED;
    uint32_t base = 0;
    for (int r = 0; r < kMaxRels; r++) {
        sq.adj[r] = adj[r];
        sq.nbase[r] = base;
        sq.card[r] = r < n ? card[r] : 1.0;
        sq.desc[r] = 1u << r;
        base += __popc(adj[r]);
    }
    // neighbour selectivities of each relation in ascending neighbour order
    for (int e = 0; e < m; e++) {
        const int u = edges[e].u, v = edges[e].v;
        sq.nsel[sq.nbase[u] + __popc(adj[u] & ((1u << v) - 1u))] = edges[e].sel;
        sq.nsel[sq.nbase[v] + __popc(adj[v] & ((1u << u) - 1u))] = edges[e].sel;
    }
    return MPDP_OK;
}

__global__ void __launch_bounds__(kNoAllocThreads)
k_optimize_noalloc(int n, int m, const double* __restrict__ card, const mpdp_edge* __restrict__ edges,
                   unsigned char* scratch, mpdp_plan_node* __restrict__ nodes, double* __restrict__ cost,
                   int32_t* __restrict__ status)
{
    __shared__ SharedQuery sq;
    __shared__ int s_status;
    __shared__ uint32_t s_blk[kNoAllocWarps][kMaxRels];
    __shared__ uint32_t s_bpref[kNoAllocWarps][kMaxRels + 1];
    __shared__ int s_nb[kNoAllocWarps];
    __shared__ mpdp_plan_node s_nodes[2 * kNoAllocRels - 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_status = ingest_one(n, m, card, edges, sq);
    __syncthreads();
    if (s_status != MPDP_OK) {
        if (tid == 0) {
            *cost = 0.0;
            *status = s_status;
        }
        return;
    }
    ScratchMemo memo{reinterpret_cast<double2*>(scratch),
                     reinterpret_cast<uint32_t*>(scratch + kNoAllocCcBytes)};
    if (tid < n) memo.put(1u << tid, 1, 0.0, sq.card[tid], 0u, nullptr);
    __syncthreads();
    const uint32_t nsets = 1u << n;
    for (int k = 2; k <= n; k++) {
        for (uint32_t b0 = (uint32_t)warp * 32u; b0 < nsets; b0 += kNoAllocThreads) {
            const uint32_t cand = b0 + (uint32_t)lane;
            const bool keep = cand < nsets && __popc(cand) == k && connected(cand, sq.adj);
            unsigned todo = __ballot_sync(kFull, keep);
            while (todo) {
                const uint32_t s = b0 + (uint32_t)(__ffs(todo) - 1);
                todo &= todo - 1u;
                if (lane == 0) {
                    const int nb = find_blocks(s, sq.adj, s_blk[warp]);
                    uint32_t acc = 0u;
                    for (int j = 0; j < nb; j++) {
                        s_bpref[warp][j] = acc;
                        acc += block_pairs(s_blk[warp][j]);
                    }
                    s_bpref[warp][nb] = acc;
                    s_nb[warp] = nb;
                }
                __syncwarp();
                const int nb = s_nb[warp];
                const uint32_t* bpref = s_bpref[warp];
                const uint32_t* blk = s_blk[warp];
                const uint32_t total = bpref[nb];
                unsigned long long bx = kNoX;
                uint32_t bl = kFull;
                for (uint32_t p = (uint32_t)lane; p < total; p += 32u) {
                    int j = 0;
                    while (j + 1 < nb && bpref[j + 1] <= p) j++;
                    const uint32_t bb = blk[j];
                    const uint32_t mn = bb & (0u - bb);
                    const uint32_t lb = mn | deposit(p - bpref[j], bb ^ mn), rb = bb ^ lb;
                    if (connected(lb, sq.adj) && connected(rb, sq.adj)) {
                        const uint32_t sl = grow(lb, s & ~rb, sq.adj);
                        fold_pair(sl, s ^ sl, memo, nullptr, bx, bl);
                    }
                }
                warp_min_x(bx, bl);
                if (lane == 0) {
                    const double card_s = peel_card(s, block_peel_vertex(s, blk, nb), sq, memo, nullptr);
                    memo.put(s, k, set_cost(bx, card_s), card_s, bl, nullptr);
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
    // plan fetch: breadth-first expansion from the full set, one lane per
    // node of the current depth (the node order of the batched plan fetch)
    if (warp != 0) return;
    if (lane == 0) s_nodes[0].set = nsets - 1u;
    __syncwarp();
    int lo = 0, hi = 1;
    bool bad = false;
    while (lo < hi) {
        int next = hi;
        for (int base = lo; base < hi; base += 32) {
            const int i = base + lane;
            bool internal = false;
            uint32_t s = 0u, l = 0u;
            double c = 0.0, cd = 0.0;
            if (i < hi) {
                s = (uint32_t)s_nodes[i].set;
                internal = (s & (s - 1u)) != 0u;
                if (internal) {
                    memo.get(s, c, cd, l, nullptr);
                    if (l == 0u || (l & ~s) != 0u || l == s) {
                        bad = true;
                        internal = false;
                    }
                }
            }
            const unsigned bal = __ballot_sync(kFull, internal);
            const int pos = next + 2 * __popc(bal & ((1u << lane) - 1u));
            if (i < hi) {
                mpdp_plan_node& nd = s_nodes[i];
                nd.n_leaves = __popc(s);
                if (internal && pos + 1 < 2 * kNoAllocRels - 1) {
                    nd.left = pos;
                    nd.right = pos + 1;
                    nd.rel = -1;
                    nd.cost = c;
                    nd.card = cd;
                    s_nodes[pos].set = l;
                    s_nodes[pos + 1].set = s ^ l;
                } else {
                    nd.left = nd.right = -1;
                    nd.rel = lowest(s);
                    nd.card = sq.card[nd.rel];
                    nd.cost = 0.0;
                }
            }
            next += 2 * __popc(bal);
            __syncwarp();
        }
        lo = hi;
        hi = next;
        if (hi > 2 * n - 1) {
            bad = true;
            break;
        }
    }
    bad = __any_sync(kFull, bad);
    if (!bad)
        for (int i = lane; i < hi; i += 32) nodes[i] = s_nodes[i];
    if (lane == 0) {
        *cost = bad ? 0.0 : s_nodes[0].cost;
        *status = bad ? MPDP_ERR_INTERNAL : MPDP_OK;
    }
}

// Address of the scratch array in the current context.  The runtime maps
// the array into each context that loads this library's device code, so the
// address is looked up (cudaGetSymbolAddress) once per context, with that
// context's device current, and kept per device with the context's unique
// id (cuCtxGetId, found through the runtime's driver entry points, so the
// library does not link the driver library).  A call in a different or
// re-created context of that device (after cudaDeviceReset, say) looks the
// address up again, so a stale address is never used.
using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    unsigned long long ctx_id = 0;  // 0: not looked up yet (context ids start at 1)
    unsigned char* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

bool resolve_driver_calls()
{
    if (g_ctx_get_current && g_ctx_get_id) return true;
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b) {
        cudaGetLastError();
        return false;
    }
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(a);
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(b);
    return true;
}

// Unique id of the calling thread's current context (0: none current).
unsigned long long current_ctx_id()
{
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (g_ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int scratch_for_device(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!resolve_driver_calls()) return MPDP_ERR_CUDA;
    ScratchAddr& e = g_scratch[dev];
    const unsigned long long id = current_ctx_id();
    if (id == 0 || e.ctx_id != id || !e.ptr) {
        // first call in this context (it becomes current here if none was)
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MPDP_ERR_CUDA;
        }
        const unsigned long long now = current_ctx_id();
        if (now == 0) return MPDP_ERR_CUDA;
        e.ctx_id = now;
        e.ptr = static_cast<unsigned char*>(p);
    }
    *out = e.ptr;
    return MPDP_OK;
}

}  // namespace
}  // namespace mpdp

extern "C" int mpdp_optimize_device_noalloc(int32_t n_rels, int32_t n_edges, const double* d_card,
                                            const mpdp_edge* d_edges, int32_t cost_model,
                                            mpdp_plan_node* d_nodes, double* d_cost, int32_t* d_status,
                                            void* cuda_stream)
{
    using namespace mpdp;
    if (!d_card || !d_nodes || !d_cost || !d_status || (n_edges > 0 && !d_edges)) return MPDP_ERR_INVALID_ARG;
    if (cost_model != MPDP_COST_COUT || n_rels < 1 || n_edges < 0) return MPDP_ERR_INVALID_ARG;
    if (n_rels > MPDP_NOALLOC_MAX_RELS) return MPDP_ERR_TOO_LARGE;
    if (n_edges > n_rels * (n_rels - 1) / 2) return MPDP_ERR_INVALID_ARG;
    unsigned char* scratch = nullptr;
    const int rc = scratch_for_device(&scratch);
    if (rc != MPDP_OK) return rc;
    k_optimize_noalloc<<<1, kNoAllocThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        n_rels, n_edges, d_card, d_edges, scratch, d_nodes, d_cost, d_status);
    if (cudaGetLastError() != cudaSuccess) return MPDP_ERR_CUDA;
    return MPDP_OK;
}
