// Exact DP over sub-problems of the heuristic modes, in extended range (XD).
//
// A sub-problem joins up to 25 "relations" that are plans of many base
// relations (IDP2's re-planned subtrees, UnionDP's partitions), with
// cardinalities far beyond binary64.  The structure of the DP does not
// depend on the arithmetic, so a batch of sub-problems goes through the
// ordinary ingest and bitmap filter (with placeholder values, which only
// have to pass validation) to get every connected set of every level; then
// per level one launch evaluates every set with the block enumeration of
// Algorithm 4, one warp per set, costs and cards in XD.  The result is the
// (x, left) choice of every connected set, and the plan fetch reads it back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mpdp_launch.h"
#include "mpdp_xd.cuh"
#include "mpdp_xd_exec.h"

namespace mpdp {

namespace {

constexpr int kXdWarps = 8;  // sets per block iteration (one per warp)
constexpr int kXdMaxBatch = 256;

struct XdEntry {
    XD cost;
    XD card;
};

struct XdArgs {
    BatchArgs a;
    const XdExtra* extra;   // [nq]
    XdEntry* memo;          // dense per query, from desc[q].memo_base
    uint32_t* left;
    XdPlanOut* plans;       // [nq]
};

// tiles (8 sets) of level k of every query, as a block-local prefix
__device__ uint32_t xd_prefix(const XdArgs& x, int k, uint32_t* s_pref)
{
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int q = 0; q < x.a.nq; q++) {
            s_pref[q] = acc;
            const QDesc& d = x.a.desc[q];
            const DevCounters& c = x.a.out[q].counters;
            if (d.n >= k && c.status == 0) acc += (c.list_count[k] + kXdWarps - 1) / kXdWarps;
        }
        s_pref[x.a.nq] = acc;
    }
    __syncthreads();
    return s_pref[x.a.nq];
}

__device__ int xd_find_q(const uint32_t* s_pref, int nq, uint32_t t)
{
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pref[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_xd_base(XdArgs x)
{
    const int q = blockIdx.x;
    const QDesc& d = x.a.desc[q];
    if (x.a.out[q].counters.status != 0) return;
    XdEntry* memo = x.memo + d.memo_base;
    uint32_t* left = x.left + d.memo_base;
    for (int r = threadIdx.x; r < d.n; r += blockDim.x) {
        memo[1u << r] = XdEntry{xd_zero(), x.extra[q].card[r]};
        left[1u << r] = 0u;
    }
}

__global__ void __launch_bounds__(32 * kXdWarps) k_eval_xd(XdArgs x, int k)
{
    __shared__ uint32_t s_pref[kXdMaxBatch + 1];
    __shared__ uint32_t s_blk[kXdWarps][kMaxRels];
    __shared__ uint32_t s_bpref[kXdWarps][kMaxRels + 1];
    __shared__ int s_nb[kXdWarps];
    const uint32_t tiles = xd_prefix(x, k, s_pref);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int qi = xd_find_q(s_pref, x.a.nq, t);
        const QDesc& d = x.a.desc[qi];
        const DevQuery* __restrict__ q = x.a.query + qi;
        const uint32_t idx = (t - s_pref[qi]) * kXdWarps + warp;
        if (idx >= x.a.out[qi].counters.list_count[k]) continue;  // warp-uniform
        const uint32_t s = x.a.lists[d.list_base + d.list_off[k] + idx];
        XdEntry* memo = x.memo + d.memo_base;
        uint32_t* left = x.left + d.memo_base;
        const XdExtra& ex = x.extra[qi];
        if (lane == 0) {
            const int nb = find_blocks(s, q->adj, s_blk[warp]);
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
        XD bx = xd_zero();
        uint32_t bl = kFull;
        bool have = false;
        for (uint32_t p = (uint32_t)lane; p < total; p += 32u) {
            int j = 0;
            while (j + 1 < nb && bpref[j + 1] <= p) j++;
            const uint32_t b = blk[j];
            const uint32_t mn = b & (0u - b);
            const uint32_t lb = mn | deposit(p - bpref[j], b ^ mn), rb = b ^ lb;
            if (!connected(lb, q->adj) || !connected(rb, q->adj)) continue;
            const uint32_t sl = grow(lb, s & ~rb, q->adj), sr = s ^ sl;
            const XD xv = xd_add(memo[sl].cost, memo[sr].cost);
            const uint32_t l = sl < sr ? sl : sr;
            if (!have || xd_less(xv, bx) || (xd_equal(xv, bx) && l < bl)) {
                bx = xv;
                bl = l;
                have = true;
            }
        }
        // warp minimum of (x, left); lanes with no pair hold left = all ones
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            XD ox;
            ox.m = __shfl_xor_sync(kFull, bx.m, o);
            ox.e = __shfl_xor_sync(kFull, bx.e, o);
            ox.pad = 0;
            const uint32_t ol = __shfl_xor_sync(kFull, bl, o);
            const bool oh = __shfl_xor_sync(kFull, have ? 1 : 0, o) != 0;
            if (oh && (!have || xd_less(ox, bx) || (xd_equal(ox, bx) && ol < bl))) {
                bx = ox;
                bl = ol;
                have = true;
            }
        }
        if (lane == 0) {
            // card(S) by peeling v: card(S \ {v}) * card[v] * sel(j, v), j ascending
            const int v = block_peel_vertex(s, blk, nb);
            const uint32_t rest = s & ~(1u << v);
            XD c = (rest & (rest - 1u)) ? memo[rest].card : ex.card[lowest(rest)];
            c = xd_mul(c, ex.card[v]);
            const uint32_t nv = q->adj[v];
            uint32_t nbm = nv & s;
            while (nbm) {
                const int jj = lowest(nbm);
                nbm &= nbm - 1u;
                c = xd_mul(c, ex.nsel[q->nbase[v] + __popc(nv & ((1u << jj) - 1u))]);
            }
            memo[s] = XdEntry{xd_add(bx, c), c};
            left[s] = bl;
        }
        __syncwarp();
    }
}

// Plan fetch: breadth-first from the full set, one thread per query.
__global__ void k_extract_xd(XdArgs x)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= x.a.nq) return;
    const QDesc& d = x.a.desc[q];
    XdPlanOut& o = x.plans[q];
    o.status = x.a.out[q].counters.status;
    o.n_nodes = 0;
    if (o.status != 0) return;
    const uint32_t* left = x.left + d.memo_base;
    const XdEntry* memo = x.memo + d.memo_base;
    const uint32_t full = (d.n == 32) ? kFull : ((1u << d.n) - 1u);
    o.set[0] = full;
    o.cost = memo[full].cost;
    int hi = 1;
    for (int i = 0; i < hi; i++) {
        const uint32_t s = o.set[i];
        if ((s & (s - 1u)) == 0u) {
            o.left[i] = o.right[i] = -1;
            continue;
        }
        const uint32_t l = left[s];
        if (l == 0u || (l & ~s) != 0u || l == s || hi + 2 > kPlanNodes) {
            o.status = MPDP_ERR_INTERNAL;
            return;
        }
        o.left[i] = hi;
        o.right[i] = hi + 1;
        o.set[hi++] = l;
        o.set[hi++] = s ^ l;
    }
    o.n_nodes = hi;
}

}  // namespace

XdExecutor::~XdExecutor()
{
    if (fixed_) cudaFree(fixed_);
    if (var_) cudaFree(var_);
    if (host_) cudaFreeHost(host_);
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int XdExecutor::run(const std::vector<XdSubQuery>& qs, std::vector<XdSubPlan>& out, cudaStream_t st,
                    int num_sms)
{
    out.clear();
    size_t b0 = 0;
    while (b0 < qs.size()) {
        // as many sub-problems as fit the batch size and the memo bytes
        size_t b1 = b0, bytes = 0;
        while (b1 < qs.size() && b1 - b0 < (size_t)kXdMaxBatch) {
            const size_t q = ((size_t)1 << std::min(qs[b1].n, 30)) * sizeof(XdEntry);
            if (b1 > b0 && bytes + q > kXdBatchMemoBytes) break;
            bytes += q;
            b1++;
        }
        const int rc = run_batch(qs, b0, b1, out, st, num_sms);
        if (rc != MPDP_OK) return rc;
        b0 = b1;
    }
    return MPDP_OK;
}

int XdExecutor::run_batch(const std::vector<XdSubQuery>& qs, size_t b0, size_t b1, std::vector<XdSubPlan>& out,
                          cudaStream_t st, int num_sms)
{
    const int nq = (int)(b1 - b0);
    // fixed part: per query descriptors, staging, device records, extras, plans
    const size_t f_desc = up256(sizeof(QDesc) * kXdMaxBatch), f_pref = up256(sizeof(uint32_t) * (kXdMaxBatch + 1)),
                 f_stage = up256(sizeof(StagedQuery) * kXdMaxBatch), f_query = up256(sizeof(DevQuery) * kXdMaxBatch),
                 f_out = up256(sizeof(DevOut) * kXdMaxBatch), f_extra = up256(sizeof(XdExtra) * kXdMaxBatch),
                 f_plan = up256(sizeof(XdPlanOut) * kXdMaxBatch);
    const size_t fixed_bytes = f_desc + f_pref + f_stage + f_query + f_out + f_extra + f_plan;
    const size_t host_bytes = f_desc + f_pref + f_stage + f_extra + f_plan;
    if (!fixed_) {
        if (cudaMalloc(&fixed_, fixed_bytes) != cudaSuccess) {
            cudaGetLastError();
            fixed_ = nullptr;
            return MPDP_ERR_OOM;
        }
        if (cudaMallocHost(&host_, host_bytes) != cudaSuccess) {
            cudaGetLastError();
            host_ = nullptr;
            return MPDP_ERR_OOM;
        }
    }
    char* dbase = static_cast<char*>(fixed_);
    QDesc* d_desc = reinterpret_cast<QDesc*>(dbase);
    uint32_t* d_pref = reinterpret_cast<uint32_t*>(dbase + f_desc);
    StagedQuery* d_stage = reinterpret_cast<StagedQuery*>(dbase + f_desc + f_pref);
    DevQuery* d_query = reinterpret_cast<DevQuery*>(dbase + f_desc + f_pref + f_stage);
    DevOut* d_out = reinterpret_cast<DevOut*>(dbase + f_desc + f_pref + f_stage + f_query);
    XdExtra* d_extra = reinterpret_cast<XdExtra*>(dbase + f_desc + f_pref + f_stage + f_query + f_out);
    XdPlanOut* d_plan = reinterpret_cast<XdPlanOut*>(dbase + f_desc + f_pref + f_stage + f_query + f_out + f_extra);
    char* hbase = static_cast<char*>(host_);
    QDesc* h_desc = reinterpret_cast<QDesc*>(hbase);
    uint32_t* h_pref = reinterpret_cast<uint32_t*>(hbase + f_desc);
    StagedQuery* h_stage = reinterpret_cast<StagedQuery*>(hbase + f_desc + f_pref);
    XdExtra* h_extra = reinterpret_cast<XdExtra*>(hbase + f_desc + f_pref + f_stage);
    XdPlanOut* h_plan = reinterpret_cast<XdPlanOut*>(hbase + f_desc + f_pref + f_stage + f_extra);

    // per query layout: level lists and the dense XD memo
    size_t lists = 0, memo = 0;
    uint32_t fblocks = 0;
    BatchPlan bp;
    bp.num_sms = num_sms;
    int max_n = 0;
    for (int i = 0; i < nq; i++) {
        const XdSubQuery& q = qs[b0 + i];
        if (q.n < 2 || q.n > kXdMaxRels || (int)q.card.size() != q.n || q.eu.size() != q.sel.size() ||
            q.eu.size() != q.ev.size() || (int)q.eu.size() > kMaxEdges)
            return MPDP_ERR_INVALID_ARG;
        QDesc& d = h_desc[i];
        memset(&d, 0, sizeof(d));
        d.n = q.n;
        d.n_edges = (int)q.eu.size();
        d.enumeration = MPDP_ENUM_BLOCKS;
        d.cost_model = MPDP_COST_COUT;
        d.memo_base = memo;
        d.list_base = lists;
        uint32_t qb = 0;
        fill_levels(d, 32, MPDP_FILTER_BITMAPS, qb);
        d.filter_block_base = fblocks;
        h_pref[i] = fblocks;
        fblocks += qb;
        unsigned long long le = 0;
        for (int k = 2; k <= q.n; k++) le += binom_host(q.n, k);
        lists += le;
        memo += (size_t)1 << q.n;
        max_n = std::max(max_n, q.n);
        // staging with placeholder values: ingest and filter only need the graph
        StagedQuery& sq = h_stage[i];
        sq.n = q.n;
        sq.n_edges = d.n_edges;
        sq.cost_model = MPDP_COST_COUT;
        sq.pad = 0;
        for (int r = 0; r < kMaxRels; r++) sq.card[r] = 1.0;
        uint32_t adj[kMaxRels] = {};
        for (int e = 0; e < d.n_edges; e++) {
            sq.edges[e] = mpdp_edge{q.eu[e], q.ev[e], 0.5};
            adj[q.eu[e]] |= 1u << q.ev[e];
            adj[q.ev[e]] |= 1u << q.eu[e];
        }
        // XD values: cards, and the neighbour selectivities in the layout
        // ingest gives DevQuery::nsel (relation r's block at the popcount
        // prefix, neighbours ascending)
        XdExtra& ex = h_extra[i];
        for (int r = 0; r < kMaxRels; r++) ex.card[r] = r < q.n ? q.card[r] : xd_zero();
        uint32_t nbase[kMaxRels];
        uint32_t acc = 0;
        for (int r = 0; r < kMaxRels; r++) {
            nbase[r] = acc;
            acc += __builtin_popcount(adj[r]);
        }
        for (int e = 0; e < d.n_edges; e++) {
            const int u = q.eu[e], v = q.ev[e];
            ex.nsel[nbase[u] + __builtin_popcount(adj[u] & ((1u << v) - 1u))] = q.sel[e];
            ex.nsel[nbase[v] + __builtin_popcount(adj[v] & ((1u << u) - 1u))] = q.sel[e];
        }
    }
    h_pref[nq] = fblocks;
    bp.filter_blocks = fblocks;
    const size_t v_lists = up256(lists * 4), v_memo = up256(memo * sizeof(XdEntry)), v_left = up256(memo * 4);
    const size_t need = v_lists + v_memo + v_left;
    if (need > var_bytes_) {
        if (var_) cudaFree(var_);
        var_ = nullptr;
        var_bytes_ = 0;
        if (cudaMalloc(&var_, need) != cudaSuccess) {
            cudaGetLastError();
            var_ = nullptr;
            return MPDP_ERR_OOM;
        }
        var_bytes_ = need;
    }
    char* vbase = static_cast<char*>(var_);
    XdArgs x;
    memset(&x, 0, sizeof(x));
    x.a.nq = nq;
    x.a.max_n = max_n;
    x.a.desc = d_desc;
    x.a.filter_block_prefix = d_pref;
    x.a.staged = d_stage;
    x.a.query = d_query;
    x.a.out = d_out;
    x.a.lists = reinterpret_cast<uint32_t*>(vbase);
    x.a.run = 32;
    x.a.filter_mode = MPDP_FILTER_BITMAPS;
    x.extra = d_extra;
    x.memo = reinterpret_cast<XdEntry*>(vbase + v_lists);
    x.left = reinterpret_cast<uint32_t*>(vbase + v_lists + v_memo);
    x.plans = d_plan;

    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    if (!ck(cudaMemcpyAsync(d_desc, h_desc, sizeof(QDesc) * nq, cudaMemcpyHostToDevice, st)) ||
        !ck(cudaMemcpyAsync(d_pref, h_pref, sizeof(uint32_t) * (nq + 1), cudaMemcpyHostToDevice, st)) ||
        !ck(cudaMemcpyAsync(d_stage, h_stage, sizeof(StagedQuery) * nq, cudaMemcpyHostToDevice, st)) ||
        !ck(cudaMemcpyAsync(d_extra, h_extra, sizeof(XdExtra) * nq, cudaMemcpyHostToDevice, st)))
        return MPDP_ERR_CUDA;
    if (!ck(enqueue_structure(x.a, bp, st))) return MPDP_ERR_CUDA;
    k_xd_base<<<nq, 32, 0, st>>>(x);
    const int grid = num_sms * 8;
    for (int k = 2; k <= max_n; k++) k_eval_xd<<<grid, 32 * kXdWarps, 0, st>>>(x, k);
    k_extract_xd<<<(nq + 63) / 64, 64, 0, st>>>(x);
    if (!ck(cudaGetLastError())) return MPDP_ERR_CUDA;
    if (!ck(cudaMemcpyAsync(h_plan, d_plan, sizeof(XdPlanOut) * nq, cudaMemcpyDeviceToHost, st)) ||
        !ck(cudaStreamSynchronize(st)))
        return MPDP_ERR_CUDA;
    for (int i = 0; i < nq; i++) {
        const XdPlanOut& o = h_plan[i];
        if (o.status != MPDP_OK) return o.status;
        XdSubPlan p;
        p.cost = o.cost;
        p.set.assign(o.set, o.set + o.n_nodes);
        p.left.assign(o.left, o.left + o.n_nodes);
        p.right.assign(o.right, o.right + o.n_nodes);
        out.push_back(std::move(p));
    }
    return MPDP_OK;
}

}  // namespace mpdp
