// C ABI of the MPDP optimizer: contexts, batches, handles, workspace, graphs.
//
// Queries are optimized in device batches.  One batch is enqueued as:
//   host -> device copy of the batch descriptors (and, on the host path, of
//   the staged queries) or a gather kernel (device path); the DP pipeline,
//   replayed from a CUDA graph captured once per batch shape; a device ->
//   host copy of every query's plan + counters (host path) or a publish
//   kernel (device path).  Nothing in between waits for the host: the
//   paper's per-level host round trip (Sec. 7.2, small queries) is gone, and
//   all queries of a batch share every launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mpdp.h"
#include "mpdp_heuristic.h"
#include "mpdp_launch.h"
#include "mpdp_xd_exec.h"

using namespace mpdp;

namespace {

const mpdp_config kDefaultConfig = {MPDP_MEMO_DENSE, MPDP_ENUM_AUTO, 64, 1, 1, 32, MPDP_FILTER_CONNECTED, 8, 4, 1, 18};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int edges_max(int n) { return n * (n - 1) / 2; }

// One submitted device batch and its pinned results.
struct Record {
    bool in_use = false;
    int nq = 0;
    int cap = 0;
    int refs = 0;
    unsigned long long seq = 0;
    DevOut* host = nullptr;  // pinned, cap entries (same layout as DevOut)
    cudaEvent_t done = nullptr, t0 = nullptr, t1 = nullptr;
    int memo_kind = 0;
    std::vector<int> n, enumeration;
    std::vector<unsigned long long> h2d;
};

struct HandleRef {
    int rec;
    int idx;
};

// Pinned staging for one batch upload.
struct StageSlot {
    char* host = nullptr;
    size_t cap = 0;
    cudaEvent_t free_ev = nullptr;  // the copies out of this slot have run
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

// Profiling mode: a pair of events around every launch, summed per class.
// Every batch also records an origin event before its first launch, so that
// launches of one batch on different streams share a time line: the union of
// a class's launch intervals is the wall time during which it was active.
struct EventHook : LaunchHook {
    struct Rec {
        int cls;
        size_t begin;  // index of the begin event (the end event follows)
        int group;     // batch (index into origins), -1 before the first mark
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    std::vector<size_t> origins;  // event index of each batch's origin
    size_t next = 0;
    cudaError_t err = cudaSuccess;

    cudaEvent_t take()
    {
        if (next == pool.size()) {
            cudaEvent_t e = nullptr;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) err = r;
            pool.push_back(e);
        }
        return pool[next++];
    }
    void mark(cudaStream_t st)
    {
        origins.push_back(next);
        cudaError_t r = cudaEventRecord(take(), st);
        if (r != cudaSuccess) err = r;
    }
    void begin(int cls, cudaStream_t st) override
    {
        recs.push_back(Rec{cls, next, (int)origins.size() - 1});
        cudaError_t r = cudaEventRecord(take(), st);
        if (r != cudaSuccess) err = r;
    }
    void end(int, cudaStream_t st) override
    {
        cudaError_t r = cudaEventRecord(take(), st);
        if (r != cudaSuccess) err = r;
    }
    void reset()
    {
        recs.clear();
        origins.clear();
        next = 0;
    }
    ~EventHook()
    {
        for (auto e : pool)
            if (e) cudaEventDestroy(e);
    }
};

// Query as the host planner sees it.
struct PlanQuery {
    int n, m, enumeration;
    const double* card;        // host path
    const mpdp_edge* edges;    // host path
    unsigned long long card_off, edge_off;  // device path
};

}  // namespace

struct mpdp_ctx {
    mpdp::XdExecutor* xd = nullptr;                      // heuristic sub-problems (created on first use)
    std::map<int64_t, mpdp::HeuristicResult> heur;      // finished heuristic-mode plans by handle
    mpdp_mlp* model = nullptr;                          // learned proposal (borrowed)
    int device = 0;
    cudaStream_t stream = nullptr;          // work stream (borrowed; nullptr = default stream)
    cudaStream_t capture_stream = nullptr;  // private, only used to capture graphs
    // lanes: private streams of the concurrent sub-batches, forked from and
    // joined back into the work (or capture) stream by events
    cudaStream_t lane_stream[MPDP_MAX_LANES] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[MPDP_MAX_LANES] = {};
    size_t budget = 0;
    mpdp_config cfg = kDefaultConfig;
    int num_sms = 152;
    // fixed device part (kMaxBatch queries)
    void* fixed = nullptr;
    char* d_upload = nullptr;  // [prefixes | descriptors | packed cards and edges]
    QDesc* d_desc = nullptr;
    uint32_t* d_prefix = nullptr;
    StagedQuery* d_staged = nullptr;
    DevQuery* d_query = nullptr;
    DevOut* d_out = nullptr;
    HashLayout* d_layout = nullptr;
    uint32_t* d_level_pref = nullptr;  // per lane: [2][kLevels][kMaxBatch + 1] (tree, block mode)
    // variable device part
    void* var = nullptr;
    size_t var_bytes = 0;
    size_t list_words = 0, heavy_entries = 0, memo_entries = 0, arena_slots = 0;
    uint32_t* d_lists = nullptr;
    HeavyMain* d_hmain = nullptr;
    HeavyExtra* d_hextra = nullptr;
    double2* d_memo = nullptr;
    uint32_t* d_left = nullptr;
    HashSlot* d_arena = nullptr;
    PairRec* d_pairs = nullptr;  // unfused ablation only
    size_t pair_records = 0;
    // host side
    static constexpr int kRing = 4;
    StageSlot ring[kRing];
    int ring_next = 0;
    std::vector<Record> recs;
    std::map<int64_t, HandleRef> handles;
    int64_t next_handle = 1;
    unsigned long long seq = 0;
    unsigned long long last_seq = 0;  // seq of the batch whose memo is in the workspace
    std::map<std::vector<int>, GraphEntry> graphs;
    int last_launches = 0;
    int profiling = 0;  // MPDP_PROFILE_*
    EventHook hook;
    std::string last_error;
};

#define CK(ctx, call)                                                                \
    do {                                                                             \
        cudaError_t e__ = (call);                                                    \
        if (e__ != cudaSuccess) {                                                    \
            (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(e__); \
            return MPDP_ERR_CUDA;                                                    \
        }                                                                            \
    } while (0)

static bool finite_pos(double x) { return x > 0.0 && x <= 1.7976931348623157e308; }

// Host-side validation of a query (same rules as the device ingest kernel).
static int validate_query(const mpdp_query* q, int max_n)
{
    if (!q) return MPDP_ERR_INVALID_ARG;
    const int n = q->n_rels, m = q->n_edges;
    if (n < 1) return MPDP_ERR_INVALID_ARG;
    if (n > max_n) return MPDP_ERR_TOO_LARGE;
    if (q->cost_model != MPDP_COST_COUT || q->t != 0 || q->mode != MPDP_MODE_EXACT) return MPDP_ERR_INVALID_ARG;
    if (m < 0 || m > edges_max(n)) return MPDP_ERR_INVALID_ARG;
    if (!q->card || (m > 0 && !q->edges)) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++)
        if (!finite_pos(q->card[i])) return MPDP_ERR_INVALID_ARG;
    const int words = (n + 63) / 64;
    std::vector<uint64_t> adj((size_t)n * words, 0);
    std::vector<int> parent(n);
    for (int i = 0; i < n; i++) parent[i] = i;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    int comps = n;
    for (int e = 0; e < m; e++) {
        const int u = q->edges[e].u, v = q->edges[e].v;
        const double s = q->edges[e].sel;
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return MPDP_ERR_INVALID_ARG;
        if (!(s > 0.0) || !(s <= 1.0)) return MPDP_ERR_INVALID_ARG;
        uint64_t& w = adj[(size_t)u * words + v / 64];
        if (w >> (v % 64) & 1ull) return MPDP_ERR_INVALID_ARG;
        w |= 1ull << (v % 64);
        adj[(size_t)v * words + u / 64] |= 1ull << (u % 64);
        const int a = find(u), b = find(v);
        if (a != b) {
            parent[a] = b;
            comps--;
        }
    }
    if (comps != 1) return MPDP_ERR_DISCONNECTED;
    return MPDP_OK;
}

// Tree enumeration needs a tree join graph (a connected graph with n - 1
// edges); BLOCKS is correct for every graph.
static int resolve_enumeration(const mpdp_config& cfg, int n, int m)
{
    if (cfg.enumeration == MPDP_ENUM_BLOCKS || cfg.enumeration == MPDP_ENUM_DPSUB || m != n - 1)
        return MPDP_ENUM_BLOCKS;
    return MPDP_ENUM_TREE;
}

// Variable workspace of one query: list words, heavy-set entries (main and
// extra, reused by every level), dense entries, hash slots.
struct QuerySize {
    size_t lists = 0, heavy = 0, memo = 0, hash = 0;
};

static QuerySize query_size(int n, int enumeration, int memo_kind)
{
    QuerySize z;
    z.lists = list_entries(n);
    // block mode: the connectivity bitmap (2^n bits) follows the level lists,
    // then the block CCP lists, then the Find-Blocks cache
    if (enumeration == MPDP_ENUM_BLOCKS)
        z.lists += conn_words(n) + block_list_words(n, enumeration) + fb_cache_words(n, enumeration);
    z.heavy = enumeration == MPDP_ENUM_BLOCKS ? binom_host(n, n / 2) : 0;
    if (memo_kind == MPDP_MEMO_DENSE) z.memo = (size_t)1 << n;
    else z.hash = hash_arena_slots(n);
    return z;
}

static size_t var_bytes_of(size_t lists, size_t heavy, size_t memo, size_t hash)
{
    return align_up(lists * 4) + align_up(heavy * sizeof(HeavyMain)) + align_up(heavy * sizeof(HeavyExtra)) +
           align_up(memo * sizeof(double2)) +
           align_up(memo * sizeof(uint32_t)) + align_up(hash * sizeof(HashSlot));
}

// Upload region: one host-to-device copy per batch carries the filter-block
// prefixes, the query descriptors and (host path) the packed cardinalities
// and predicates, laid out as [prefixes | descriptors | cards | edges].  The
// prefixes and descriptors sit at fixed offsets (captured graphs read them);
// the packed arrays follow the batch's descriptors.
constexpr size_t kUploadPrefixBytes = ((sizeof(uint32_t) * (kMaxBatch + MPDP_MAX_LANES + 1)) + 255) & ~(size_t)255;

static size_t upload_bytes_max()
{
    return kUploadPrefixBytes + align_up(sizeof(QDesc) * kMaxBatch) + align_up(sizeof(double) * kMaxRels * kMaxBatch) +
           align_up(sizeof(mpdp_edge) * kMaxEdges * kMaxBatch);
}

static size_t fixed_bytes()
{
    return upload_bytes_max() + align_up(sizeof(StagedQuery) * kMaxBatch) + align_up(sizeof(DevQuery) * kMaxBatch) +
           align_up(sizeof(DevOut) * kMaxBatch) + align_up(sizeof(HashLayout) * kMaxBatch) +
           align_up(sizeof(uint32_t) * MPDP_MAX_LANES * 2 * kLevels * (kMaxBatch + 2));
}

static void destroy_graphs(mpdp_ctx* ctx)
{
    for (auto& kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
}

static int ensure_fixed(mpdp_ctx* ctx)
{
    if (ctx->fixed) return MPDP_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, fixed_bytes()) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_OOM;
    }
    ctx->fixed = p;
    char* c = static_cast<char*>(p);
    auto take = [&](size_t sz) {
        char* r = c;
        c += align_up(sz);
        return r;
    };
    ctx->d_upload = take(upload_bytes_max());
    ctx->d_prefix = reinterpret_cast<uint32_t*>(ctx->d_upload);
    ctx->d_desc = reinterpret_cast<QDesc*>(ctx->d_upload + kUploadPrefixBytes);
    ctx->d_staged = reinterpret_cast<StagedQuery*>(take(sizeof(StagedQuery) * kMaxBatch));
    ctx->d_query = reinterpret_cast<DevQuery*>(take(sizeof(DevQuery) * kMaxBatch));
    ctx->d_out = reinterpret_cast<DevOut*>(take(sizeof(DevOut) * kMaxBatch));
    ctx->d_layout = reinterpret_cast<HashLayout*>(take(sizeof(HashLayout) * kMaxBatch));
    ctx->d_level_pref =
        reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * MPDP_MAX_LANES * 2 * kLevels * (kMaxBatch + 2)));
    CK(ctx, cudaMemsetAsync(ctx->d_out, 0, sizeof(DevOut) * kMaxBatch, ctx->stream));
    return MPDP_OK;
}

// Grow the variable workspace to hold at least the given sizes.
static int ensure_var(mpdp_ctx* ctx, size_t lists, size_t heavy, size_t memo, size_t hash)
{
    if (ctx->var && lists <= ctx->list_words && heavy <= ctx->heavy_entries && memo <= ctx->memo_entries &&
        hash <= ctx->arena_slots)
        return MPDP_OK;
    // grow every part to at least what it had, so alternating shapes do not thrash
    size_t L = std::max(lists, ctx->list_words), V = std::max(heavy, ctx->heavy_entries),
           M = std::max(memo, ctx->memo_entries), H = std::max(hash, ctx->arena_slots);
    if (var_bytes_of(L, V, M, H) + fixed_bytes() > ctx->budget) {
        L = lists;  // only what this batch needs
        V = heavy;
        M = memo;
        H = hash;
        if (var_bytes_of(L, V, M, H) + fixed_bytes() > ctx->budget) return MPDP_ERR_ADMISSION;
    }
    const size_t bytes = var_bytes_of(L, V, M, H);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    destroy_graphs(ctx);
    if (ctx->var) cudaFree(ctx->var);
    ctx->var = nullptr;
    ctx->list_words = ctx->heavy_entries = ctx->memo_entries = ctx->arena_slots = 0;
    ctx->last_seq = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->last_error = "cudaMalloc of the batch workspace failed";
        return MPDP_ERR_OOM;
    }
    ctx->var = p;
    ctx->var_bytes = bytes;
    char* c = static_cast<char*>(p);
    auto take = [&](size_t sz) {
        char* r = c;
        c += align_up(sz);
        return r;
    };
    ctx->d_lists = reinterpret_cast<uint32_t*>(take(L * 4));
    ctx->d_hmain = reinterpret_cast<HeavyMain*>(take(V * sizeof(HeavyMain)));
    ctx->d_hextra = reinterpret_cast<HeavyExtra*>(take(V * sizeof(HeavyExtra)));
    ctx->d_memo = reinterpret_cast<double2*>(take(M * sizeof(double2)));
    ctx->d_left = reinterpret_cast<uint32_t*>(take(M * sizeof(uint32_t)));
    ctx->d_arena = reinterpret_cast<HashSlot*>(take(H * sizeof(HashSlot)));
    ctx->list_words = L;
    ctx->heavy_entries = V;
    ctx->memo_entries = M;
    ctx->arena_slots = H;
    return MPDP_OK;
}

static BatchArgs batch_args(const mpdp_ctx* ctx, int nq, int max_n)
{
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.nq = nq;
    a.max_n = max_n;
    a.desc = ctx->d_desc;
    a.filter_block_prefix = ctx->d_prefix;
    a.staged = ctx->d_staged;
    a.query = ctx->d_query;
    a.out = ctx->d_out;
    a.lists = ctx->d_lists;
    a.hmain = ctx->d_hmain;
    a.hextra = ctx->d_hextra;
    a.memo = ctx->d_memo;
    a.left = ctx->d_left;
    a.arena = ctx->d_arena;
    a.layout = ctx->d_layout;
    a.arena_slots = ctx->arena_slots;
    a.run = ctx->cfg.run_length;
    a.heavy_threshold = ctx->cfg.heavy_threshold;
    a.use_ccc = ctx->cfg.use_ccc;
    a.dpsub = ctx->cfg.enumeration == MPDP_ENUM_DPSUB ? 1 : 0;
    a.filter_mode = ctx->cfg.filter;
    return a;
}

// Split [0, count) into consecutive sub-batches that fit the budget.
static int split_batches(mpdp_ctx* ctx, const std::vector<PlanQuery>& qs, std::vector<std::pair<int, int>>& out)
{
    const int kind = ctx->cfg.memo_kind;
    size_t L = 0, V = 0, M = 0, A = 0;
    int start = 0;
    for (int i = 0; i < (int)qs.size(); i++) {
        const QuerySize z = query_size(qs[i].n, qs[i].enumeration, kind);
        if (var_bytes_of(z.lists, z.heavy, z.memo, z.hash) + fixed_bytes() > ctx->budget)
            return MPDP_ERR_ADMISSION;
        const bool full = (i - start) >= kMaxBatch;
        const size_t need = var_bytes_of(L + z.lists, V + z.heavy, M + z.memo, A + z.hash) + fixed_bytes();
        if (i > start && (full || need > ctx->budget)) {
            out.emplace_back(start, i);
            start = i;
            L = V = M = A = 0;
        }
        L += z.lists;
        V += z.heavy;
        M += z.memo;
        A += z.hash;
    }
    if (start < (int)qs.size()) out.emplace_back(start, (int)qs.size());
    return MPDP_OK;
}

static int acquire_record(mpdp_ctx* ctx, int nq)
{
    int best = -1;
    for (int i = 0; i < (int)ctx->recs.size(); i++)
        if (!ctx->recs[i].in_use && ctx->recs[i].cap >= nq) {
            best = i;
            break;
        }
    if (best < 0) {
        for (int i = 0; i < (int)ctx->recs.size(); i++)
            if (!ctx->recs[i].in_use) {
                best = i;
                break;
            }
        if (best < 0) {
            ctx->recs.emplace_back();
            best = (int)ctx->recs.size() - 1;
        }
    }
    Record& r = ctx->recs[best];
    if (r.cap < nq) {
        if (r.host) cudaFreeHost(r.host);
        r.host = nullptr;
        r.cap = 0;
        if (cudaMallocHost(reinterpret_cast<void**>(&r.host), sizeof(DevOut) * nq) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        r.cap = nq;
    }
    if (!r.done) {
        if (cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&r.t0) != cudaSuccess || cudaEventCreate(&r.t1) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
    }
    r.in_use = true;
    r.nq = nq;
    r.refs = 0;
    return best;
}

// Next staging slot with room for `bytes`, once its previous copies have run.
static int acquire_stage(mpdp_ctx* ctx, size_t bytes, char** host, int* slot)
{
    const int i = ctx->ring_next;
    ctx->ring_next = (i + 1) % mpdp_ctx::kRing;
    StageSlot& s = ctx->ring[i];
    CK(ctx, cudaEventSynchronize(s.free_ev));
    if (s.cap < bytes) {
        if (s.host) cudaFreeHost(s.host);
        s.host = nullptr;
        s.cap = 0;
        CK(ctx, cudaMallocHost(reinterpret_cast<void**>(&s.host), bytes));
        s.cap = bytes;
    }
    *host = s.host;
    *slot = i;
    return MPDP_OK;
}

// One sub-batch of a device batch: queries [q0, q1), their arguments (query
// arrays offset by q0, own filter-block prefix, own hash-arena range) and
// launch plan.
struct Lane {
    int q0 = 0, q1 = 0;
    BatchArgs a;
    BatchPlan bp;
};

static int ensure_lane_streams(mpdp_ctx* ctx, int lanes)
{
    if (!ctx->fork_ev) CK(ctx, cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
    for (int l = 0; l < lanes; l++) {
        if (!ctx->lane_stream[l]) CK(ctx, cudaStreamCreateWithFlags(&ctx->lane_stream[l], cudaStreamNonBlocking));
        if (!ctx->join_ev[l]) CK(ctx, cudaEventCreateWithFlags(&ctx->join_ev[l], cudaEventDisableTiming));
    }
    return MPDP_OK;
}

// Enqueue every lane's pipeline on `st`: one lane directly; several on the
// lane streams, forked from and joined back into `st` (inside a capture this
// makes parallel branches of one graph).  In serial profiling the lanes run
// one after the other on `st`, so that per-kernel-class times add up; in
// concurrent profiling they run as in normal operation.
static cudaError_t enqueue_lanes(mpdp_ctx* ctx, const std::vector<Lane>& lanes, cudaStream_t st, int* launches,
                                 LaunchHook* hook)
{
    int total = 0;
    cudaError_t e = cudaSuccess;
    if (lanes.size() == 1 || (hook && ctx->profiling != MPDP_PROFILE_CONCURRENT)) {
        for (const Lane& ln : lanes) {
            int c = 0;
            e = enqueue_pipeline(ln.a, ln.bp, ctx->cfg.memo_kind, st, &c, hook);
            if (e != cudaSuccess) return e;
            total += c;
        }
    } else {
        if ((e = cudaEventRecord(ctx->fork_ev, st)) != cudaSuccess) return e;
        for (size_t l = 0; l < lanes.size(); l++) {
            cudaStream_t ls = ctx->lane_stream[l];
            int c = 0;
            if ((e = cudaStreamWaitEvent(ls, ctx->fork_ev, 0)) != cudaSuccess) return e;
            if ((e = enqueue_pipeline(lanes[l].a, lanes[l].bp, ctx->cfg.memo_kind, ls, &c, hook)) != cudaSuccess)
                return e;
            total += c;
            if ((e = cudaEventRecord(ctx->join_ev[l], ls)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, ctx->join_ev[l], 0)) != cudaSuccess) return e;
        }
    }
    if (launches) *launches = total;
    return cudaSuccess;
}

// Enqueue the DP pipeline of a planned batch: graph replay or direct launches.
static int run_pipeline(mpdp_ctx* ctx, const std::vector<Lane>& lanes, const std::vector<int>& key, int* launches)
{
    if (lanes.size() > 1) {
        const int rc = ensure_lane_streams(ctx, (int)lanes.size());
        if (rc != MPDP_OK) return rc;
    }
    if (ctx->profiling || !ctx->cfg.use_graphs) {
        CK(ctx, enqueue_lanes(ctx, lanes, ctx->stream, launches, ctx->profiling ? &ctx->hook : nullptr));
        return MPDP_OK;
    }
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        if (ctx->graphs.size() >= 256) destroy_graphs(ctx);
        GraphEntry g;
        cudaGraph_t graph = nullptr;
        CK(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_lanes(ctx, lanes, ctx->capture_stream, &g.launches, nullptr);
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            ctx->last_error = std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
            return MPDP_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->last_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
            return MPDP_ERR_CUDA;
        }
        it = ctx->graphs.emplace(key, g).first;
    }
    CK(ctx, cudaGraphLaunch(it->second.exec, ctx->stream));
    if (launches) *launches = it->second.launches;
    return MPDP_OK;
}

// Unfused ablation: pair records for every lane (each lane its own range),
// grown on demand inside the memo budget; a move invalidates the graphs.
static int ensure_pairs(mpdp_ctx* ctx, std::vector<Lane>& lanes)
{
    size_t need = 0;
    for (const Lane& ln : lanes) need += unfused_pair_records(ln.bp);
    if (need > ctx->pair_records) {
        if (ctx->var_bytes + fixed_bytes() + need * sizeof(PairRec) > ctx->budget) return MPDP_ERR_ADMISSION;
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        destroy_graphs(ctx);
        if (ctx->d_pairs) cudaFree(ctx->d_pairs);
        ctx->d_pairs = nullptr;
        ctx->pair_records = 0;
        if (cudaMalloc(&ctx->d_pairs, need * sizeof(PairRec)) != cudaSuccess) {
            cudaGetLastError();
            ctx->d_pairs = nullptr;
            ctx->last_error = "cudaMalloc of the unfused pair buffer failed";
            return MPDP_ERR_OOM;
        }
        ctx->pair_records = need;
    }
    size_t off = 0;
    for (Lane& ln : lanes) {
        ln.bp.pairs = ctx->d_pairs + off;
        off += unfused_pair_records(ln.bp);
    }
    return MPDP_OK;
}

// Split queries [0, nq) into at most `lanes` runs of consecutive queries with
// about equal sums of 2^n (the filter's work; the evaluation's grows with it
// too).  Returns the run starts followed by nq.
static std::vector<int> lane_bounds(const std::vector<PlanQuery>& qs, int lanes)
{
    const int nq = (int)qs.size();
    lanes = std::max(1, std::min(lanes, nq));
    double total = 0.0;
    for (const auto& q : qs) total += std::ldexp(1.0, q.n);
    std::vector<int> b = {0};
    double acc = 0.0;
    for (int i = 0; i < nq && (int)b.size() < lanes; i++) {
        acc += std::ldexp(1.0, qs[i].n);
        // close this run once it holds its share, leaving a query for each later run
        if (acc >= total * (double)b.size() / lanes && i + 1 < nq && nq - (i + 1) >= lanes - (int)b.size())
            b.push_back(i + 1);
    }
    b.push_back(nq);
    return b;
}

// Plan, upload and enqueue one device batch.  host_path: queries come from
// host arrays (staged + copied); otherwise from caller device arrays.
static int submit_batch(mpdp_ctx* ctx, const std::vector<PlanQuery>& qs, bool host_path, const double* d_card,
                        const mpdp_edge* d_edges, int* record_out, mpdp_plan_node* d_nodes, double* d_cost,
                        int32_t* d_status)
{
    const int nq = (int)qs.size();
    const int kind = ctx->cfg.memo_kind;
    int rc = ensure_fixed(ctx);
    if (rc != MPDP_OK) return rc;
    size_t L = 0, V = 0, M = 0, A = 0;
    for (const auto& q : qs) {
        const QuerySize z = query_size(q.n, q.enumeration, kind);
        L += z.lists;
        V += z.heavy;
        M += z.memo;
        A += z.hash;
    }
    rc = ensure_var(ctx, L, V, M, A);
    if (rc != MPDP_OK) return rc;
    const std::vector<int> bounds = lane_bounds(qs, ctx->cfg.lanes);
    const int n_lanes = (int)bounds.size() - 1;
    std::vector<Lane> lanes(n_lanes);
    // one copy: [prefixes | descriptors | cards | edges], the same layout as
    // the device upload region (cards and edges on the host path only)
    const size_t desc_bytes = sizeof(QDesc) * nq;
    size_t sum_n = 0, sum_m = 0;
    if (host_path)
        for (const auto& q : qs) {
            sum_n += (size_t)q.n;
            sum_m += (size_t)q.m;
        }
    const size_t card_at = kUploadPrefixBytes + align_up(desc_bytes);
    const size_t edge_at = card_at + align_up(sizeof(double) * sum_n);
    const size_t stage_bytes = host_path ? edge_at + sizeof(mpdp_edge) * sum_m : kUploadPrefixBytes + desc_bytes;
    char* h = nullptr;
    int slot = 0;
    rc = acquire_stage(ctx, stage_bytes, &h, &slot);
    if (rc != MPDP_OK) return rc;
    uint32_t* hp = reinterpret_cast<uint32_t*>(h);
    QDesc* hd = reinterpret_cast<QDesc*>(h + kUploadPrefixBytes);
    double* hcard = reinterpret_cast<double*>(h + card_at);
    mpdp_edge* hedge = reinterpret_cast<mpdp_edge*>(h + edge_at);
    unsigned long long pack_card = 0, pack_edge = 0;
    std::vector<int> key = {nq,
                            kind,
                            ctx->cfg.heavy_threshold,
                            ctx->cfg.use_ccc,
                            ctx->cfg.run_length,
                            ctx->cfg.filter,
                            ctx->cfg.grid_blocks_per_sm,
                            ctx->cfg.enumeration,
                            ctx->cfg.fuse_prune,
                            ctx->cfg.group_threads_log2,
                            n_lanes};
    unsigned long long lbase = 0, mbase = 0, hbase = 0, abase = 0;
    uint32_t fblocks = 0;
    int max_n = 0, lane = 0, lane_max_n = 0;
    unsigned long long conn_blocks = 0;  // k_filter_connected blocks the lane's tree queries could use
    std::vector<unsigned long long> h2d(nq, 0);
    for (int i = 0; i < nq; i++) {
        const PlanQuery& q = qs[i];
        QDesc& d = hd[i];
        if (i == bounds[lane]) {  // first query of a lane
            Lane& ln = lanes[lane];
            ln.q0 = i;
            ln.q1 = bounds[lane + 1];
            ln.bp.num_sms = ctx->num_sms;
            ln.bp.blocks_per_sm = ctx->cfg.grid_blocks_per_sm;
            ln.bp.group_threads = ctx->cfg.group_threads_log2 ? 1u << ctx->cfg.group_threads_log2 : 0u;
            ln.bp.level_pref = ctx->d_level_pref + (size_t)lane * 2 * kLevels * (kMaxBatch + 2);
            ln.a.arena_begin = abase;
            fblocks = 0;
            lane_max_n = 0;
            conn_blocks = 0;
            lane++;
        }
        BatchPlan& bp = lanes[lane - 1].bp;
        memset(&d, 0, sizeof(d));
        d.n = q.n;
        d.n_edges = q.m;
        d.enumeration = q.enumeration;
        d.cost_model = MPDP_COST_COUT;
        d.memo_base = mbase;
        d.list_base = lbase;
        if (host_path) {  // packed behind the descriptors
            d.card_off = pack_card;
            d.edge_off = pack_edge;
            memcpy(hcard + pack_card, q.card, sizeof(double) * q.n);
            if (q.m > 0) memcpy(hedge + pack_edge, q.edges, sizeof(mpdp_edge) * q.m);
            pack_card += (unsigned long long)q.n;
            pack_edge += (unsigned long long)q.m;
        } else {
            d.card_off = q.card_off;
            d.edge_off = q.edge_off;
        }
        uint32_t qb = 0;
        fill_levels(d, ctx->cfg.run_length, ctx->cfg.filter, qb);
        d.filter_block_base = fblocks;
        hp[i + lane - 1] = fblocks;  // the lane's own prefix: lane l's starts at q0 + l
        fblocks += qb;
        if (ctx->cfg.filter == MPDP_FILTER_CONNECTED && q.m == q.n - 1 && q.n >= 2) {
            // at most 2^(n-1) + n - 1 connected sets (a star): warps of 32 ranks, 8 per block
            const unsigned long long warps = ((1ull << (q.n - 1)) + (unsigned long long)q.n + 31ull) / 32ull;
            conn_blocks += (warps + kFilterThreads / 32 - 1) / (kFilterThreads / 32);
        }
        const QuerySize z = query_size(q.n, q.enumeration, kind);
        d.heavy_base = hbase;
        d.heavy_cap = (uint32_t)z.heavy;
        // the bitmap sweep writes the connectivity bitmap of the block-mode
        // queries it serves (the unranking filter forms no bitmap)
        d.use_conn = (q.enumeration == MPDP_ENUM_BLOCKS && ctx->cfg.filter != MPDP_FILTER_UNRANK) ? 1u : 0u;
        d.conn_base = lbase + list_entries(q.n);
        // block CCP lists, except in the DPSUB ablation (which enumerates every
        // bipartition of the whole set)
        d.use_bl = (block_list_words(q.n, q.enumeration) > 0 && ctx->cfg.enumeration != MPDP_ENUM_DPSUB) ? 1u : 0u;
        d.bl_base = d.conn_base + conn_words(q.n);
        if (d.use_bl) bp.block_lists = true;
        lbase += z.lists;
        mbase += z.memo;
        hbase += z.heavy;
        abase += z.hash;
        if (q.n > max_n) max_n = q.n;
        if (q.n > lane_max_n) lane_max_n = q.n;
        if (i + 1 == bounds[lane]) {  // last query of the lane
            Lane& ln = lanes[lane - 1];
            hp[i + lane] = fblocks;
            // the bitmap sweep strides over the blocks the device assigns it
            // (trees may go to the connected-set unranking): one resident
            // wave of 6 blocks per SM; the unranking filter maps blocks to
            // queries by this prefix and takes all of them
            const uint32_t sweep_cap = (uint32_t)ctx->num_sms * 6u;
            bp.filter_blocks = (ctx->cfg.filter == MPDP_FILTER_UNRANK || fblocks < sweep_cap) ? fblocks : sweep_cap;
            const unsigned long long cap = (unsigned long long)ctx->num_sms * 8ull;  // grid-stride beyond
            bp.connected_blocks = (uint32_t)(conn_blocks < cap ? conn_blocks : cap);
            const BatchArgs whole = batch_args(ctx, nq, max_n);
            const unsigned long long begin = ln.a.arena_begin;
            ln.a = batch_args(ctx, ln.q1 - ln.q0, lane_max_n);
            ln.a.desc = whole.desc + ln.q0;
            ln.a.filter_block_prefix = ctx->d_prefix + ln.q0 + (lane - 1);
            ln.a.staged = whole.staged + ln.q0;
            ln.a.query = whole.query + ln.q0;
            ln.a.out = whole.out + ln.q0;
            ln.a.layout = whole.layout + ln.q0;
            // hash memo: every lane has its own arena range (the last one the rest)
            ln.a.arena_begin = n_lanes == 1 ? 0 : begin;
            ln.a.arena_slots = lane == n_lanes ? ctx->arena_slots : abase;
        }
        for (int k = 2; k <= q.n; k++) {
            const unsigned long long c = binom_host(q.n, k);
            if (q.enumeration == MPDP_ENUM_TREE) {
                bp.tree_tiles[k] += (c + kEvalThreads - 1) / kEvalThreads;
            } else {
                bp.block_tiles[k] += (c + kEvalThreads - 1) / kEvalThreads;
                bp.block_sets[k] += (c + z.heavy + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
            }
        }
        key.push_back(q.n);
        key.push_back(q.enumeration);
        key.push_back(q.m == q.n - 1 ? 1 : 0);  // trees take another filter kernel
    }
    if (!ctx->cfg.fuse_prune) {
        rc = ensure_pairs(ctx, lanes);
        if (rc != MPDP_OK) return rc;
    }
    CK(ctx, cudaMemcpyAsync(ctx->d_upload, h, stage_bytes, cudaMemcpyHostToDevice, ctx->stream));
    if (host_path) {
        // bytes copied per query: its descriptor, cards and edges; the first
        // query also carries the prefixes and the alignment padding
        unsigned long long rest = stage_bytes;
        for (int i = 0; i < nq; i++) {
            h2d[i] = sizeof(QDesc) + sizeof(double) * qs[i].n + sizeof(mpdp_edge) * qs[i].m;
            rest -= h2d[i];
        }
        h2d[0] += rest;
    }
    CK(ctx, cudaEventRecord(ctx->ring[slot].free_ev, ctx->stream));
    const BatchArgs a = batch_args(ctx, nq, max_n);
    LaunchHook* hook = ctx->profiling ? &ctx->hook : nullptr;
    if (ctx->profiling) ctx->hook.mark(ctx->stream);
    int launches = 0;
    if (host_path) {
        d_card = reinterpret_cast<const double*>(ctx->d_upload + card_at);
        d_edges = reinterpret_cast<const mpdp_edge*>(ctx->d_upload + edge_at);
    }
    CK(ctx, enqueue_stage_device(a, d_card, d_edges, ctx->stream, hook));
    launches++;
    int ri = -1;
    if (host_path) {
        ri = acquire_record(ctx, nq);
        if (ri < 0) return MPDP_ERR_CUDA;
        CK(ctx, cudaEventRecord(ctx->recs[ri].t0, ctx->stream));
    }
    int pl = 0;
    rc = run_pipeline(ctx, lanes, key, &pl);
    if (rc != MPDP_OK) {
        if (ri >= 0) ctx->recs[ri].in_use = false;
        return rc;
    }
    launches += pl;
    ctx->last_seq = ++ctx->seq;
    if (host_path) {
        Record& r = ctx->recs[ri];
        CK(ctx, cudaEventRecord(r.t1, ctx->stream));
        CK(ctx, cudaMemcpyAsync(r.host, ctx->d_out, sizeof(DevOut) * nq, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaEventRecord(r.done, ctx->stream));
        r.seq = ctx->seq;
        r.memo_kind = kind;
        r.n.resize(nq);
        r.enumeration.resize(nq);
        r.h2d = h2d;
        for (int i = 0; i < nq; i++) {
            r.n[i] = qs[i].n;
            r.enumeration[i] = qs[i].enumeration;
        }
    } else {
        CK(ctx, enqueue_publish(a, d_nodes, d_cost, d_status, ctx->stream, hook));
        launches++;
    }
    ctx->last_launches = launches;
    if (record_out) *record_out = ri;
    return MPDP_OK;
}

extern "C" {

int32_t mpdp_abi_version(void) { return MPDP_ABI_VERSION; }

const char* mpdp_strerror(int code)
{
    switch (code) {
    case MPDP_OK: return "ok";
    case MPDP_ERR_INVALID_ARG: return "invalid argument";
    case MPDP_ERR_DISCONNECTED: return "join graph is disconnected (no plan without cross products)";
    case MPDP_ERR_TOO_LARGE: return "query too large for this mode";
    case MPDP_ERR_OOM: return "out of device memory";
    case MPDP_ERR_ADMISSION: return "request exceeds the memo budget";
    case MPDP_ERR_BUFFER_TOO_SMALL: return "output buffer too small";
    case MPDP_ERR_TIMEOUT: return "bounded device wait timed out";
    case MPDP_ERR_PROBE_LIMIT: return "memo probe limit reached";
    case MPDP_ERR_CUDA: return "CUDA runtime error";
    case MPDP_ERR_BAD_HANDLE: return "unknown handle";
    case MPDP_ERR_NOT_IMPLEMENTED: return "not implemented";
    case MPDP_ERR_STALE: return "memo of this handle was overwritten";
    case MPDP_ERR_INTERNAL: return "internal consistency check failed";
    case MPDP_ERR_NOT_READY: return "result not ready yet";
    default: return "unknown error";
    }
}

const char* mpdp_last_error(const mpdp_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int32_t mpdp_last_launch_count(const mpdp_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

size_t mpdp_workspace_bytes(int32_t n_rels, const mpdp_config* cfg)
{
    if (n_rels < 1 || n_rels > MPDP_MAX_EXACT_RELS) return 0;
    const int kind = cfg ? cfg->memo_kind : MPDP_MEMO_DENSE;
    const int en = cfg && (cfg->enumeration == MPDP_ENUM_BLOCKS || cfg->enumeration == MPDP_ENUM_DPSUB)
                       ? MPDP_ENUM_BLOCKS
                       : MPDP_ENUM_TREE;
    const QuerySize z = query_size(n_rels, en, kind);
    return var_bytes_of(z.lists, z.heavy, z.memo, z.hash) + fixed_bytes();
}

int mpdp_create(mpdp_ctx** out, int device, size_t memo_budget_bytes, void* cuda_stream)
{
    if (!out) return MPDP_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    mpdp_ctx* ctx = new mpdp_ctx();
    ctx->device = device;
    ctx->budget = memo_budget_bytes ? memo_budget_bytes : ((size_t)64 << 30);
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    bool ok = cudaSetDevice(device) == cudaSuccess &&
              cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) == cudaSuccess &&
              configure_kernels() == cudaSuccess;
    for (int i = 0; ok && i < mpdp_ctx::kRing; i++)
        ok = cudaEventCreateWithFlags(&ctx->ring[i].free_ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mpdp_destroy(ctx);
        return MPDP_ERR_CUDA;
    }
    *out = ctx;
    return MPDP_OK;
}

void mpdp_destroy(mpdp_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete ctx->xd;
    ctx->xd = nullptr;
    destroy_graphs(ctx);
    for (auto& r : ctx->recs) {
        if (r.host) cudaFreeHost(r.host);
        if (r.done) cudaEventDestroy(r.done);
        if (r.t0) cudaEventDestroy(r.t0);
        if (r.t1) cudaEventDestroy(r.t1);
    }
    for (int i = 0; i < mpdp_ctx::kRing; i++) {
        if (ctx->ring[i].host) cudaFreeHost(ctx->ring[i].host);
        if (ctx->ring[i].free_ev) cudaEventDestroy(ctx->ring[i].free_ev);
    }
    if (ctx->var) cudaFree(ctx->var);
    if (ctx->fixed) cudaFree(ctx->fixed);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->d_pairs) cudaFree(ctx->d_pairs);
    for (int l = 0; l < MPDP_MAX_LANES; l++) {
        if (ctx->lane_stream[l]) cudaStreamDestroy(ctx->lane_stream[l]);
        if (ctx->join_ev[l]) cudaEventDestroy(ctx->join_ev[l]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    cudaGetLastError();
    delete ctx;
}

int mpdp_set_config(mpdp_ctx* ctx, const mpdp_config* cfg)
{
    if (!ctx || !cfg) return MPDP_ERR_INVALID_ARG;
    if (cfg->memo_kind != MPDP_MEMO_DENSE && cfg->memo_kind != MPDP_MEMO_HASH) return MPDP_ERR_INVALID_ARG;
    if (cfg->enumeration < MPDP_ENUM_AUTO || cfg->enumeration > MPDP_ENUM_DPSUB) return MPDP_ERR_INVALID_ARG;
    if (cfg->heavy_threshold < 0 || cfg->run_length < 1 || cfg->run_length > 32) return MPDP_ERR_INVALID_ARG;
    if (cfg->filter != MPDP_FILTER_BITMAPS && cfg->filter != MPDP_FILTER_UNRANK &&
        cfg->filter != MPDP_FILTER_CONNECTED)
        return MPDP_ERR_INVALID_ARG;
    if (cfg->grid_blocks_per_sm < 1 || cfg->grid_blocks_per_sm > 32) return MPDP_ERR_INVALID_ARG;
    if (cfg->lanes < 1 || cfg->lanes > MPDP_MAX_LANES) return MPDP_ERR_INVALID_ARG;
    if (cfg->fuse_prune != 0 && cfg->fuse_prune != 1) return MPDP_ERR_INVALID_ARG;
    if (cfg->group_threads_log2 != 0 && (cfg->group_threads_log2 < 8 || cfg->group_threads_log2 > 24))
        return MPDP_ERR_INVALID_ARG;
    ctx->cfg = *cfg;
    return MPDP_OK;
}

int mpdp_get_config(const mpdp_ctx* ctx, mpdp_config* cfg)
{
    if (!cfg) return MPDP_ERR_INVALID_ARG;
    *cfg = ctx ? ctx->cfg : kDefaultConfig;
    return MPDP_OK;
}

int mpdp_optimize_batch(mpdp_ctx* ctx, const mpdp_query* qs, int32_t nq, int64_t* handles)
{
    if (!ctx || nq < 0 || (nq > 0 && (!qs || !handles))) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < nq; i++) handles[i] = -1;
    std::vector<PlanQuery> pq(nq);
    for (int i = 0; i < nq; i++) {
        if (qs[i].mode != MPDP_MODE_EXACT) return MPDP_ERR_NOT_IMPLEMENTED;
        const int rc = validate_query(&qs[i], MPDP_MAX_EXACT_RELS);
        if (rc != MPDP_OK) return rc;
        pq[i] = PlanQuery{qs[i].n_rels, qs[i].n_edges, resolve_enumeration(ctx->cfg, qs[i].n_rels, qs[i].n_edges),
                          qs[i].card, qs[i].edges, 0, 0};
    }
    if (nq == 0) return MPDP_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    std::vector<std::pair<int, int>> parts;
    int rc = split_batches(ctx, pq, parts);
    if (rc != MPDP_OK) return rc;
    for (const auto& pr : parts) {
        std::vector<PlanQuery> sub(pq.begin() + pr.first, pq.begin() + pr.second);
        int ri = -1;
        rc = submit_batch(ctx, sub, true, nullptr, nullptr, &ri, nullptr, nullptr, nullptr);
        if (rc != MPDP_OK) return rc;
        for (int i = pr.first; i < pr.second; i++) {
            const int64_t h = ctx->next_handle++;
            ctx->handles[h] = HandleRef{ri, i - pr.first};
            ctx->recs[ri].refs++;
            handles[i] = h;
        }
    }
    return MPDP_OK;
}

// Host checks of a heuristic-mode query (any n up to the heuristic limit).
static int validate_heuristic(const mpdp_query* q)
{
    const int n = q->n_rels, m = q->n_edges;
    if (q->cost_model != MPDP_COST_COUT) return MPDP_ERR_INVALID_ARG;
    const bool idp = q->mode == MPDP_MODE_IDP2 || q->mode == MPDP_MODE_IDP2_LEARNED ||
                     q->mode == MPDP_MODE_IDP2_WEIGHT_START;
    if (!idp && q->mode != MPDP_MODE_UNIONDP && q->mode != MPDP_MODE_UNIONDP_LEARNED &&
        q->mode != MPDP_MODE_UNIONDP_SIZEFIRST)
        return MPDP_ERR_INVALID_ARG;
    if (n < 1 || m < 0 || (long long)m > (long long)n * (n - 1) / 2 || !q->card || (m > 0 && !q->edges))
        return MPDP_ERR_INVALID_ARG;
    if (n > MPDP_MAX_HEURISTIC_RELS) return MPDP_ERR_TOO_LARGE;
    if (q->k > 25) return MPDP_ERR_TOO_LARGE;
    if (idp && q->t != 0) return MPDP_ERR_INVALID_ARG;
    if (!idp && (q->k < 2 || (q->t != 0 && (q->t < 2 || q->t > q->k))))
        return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++)
        if (!finite_pos(q->card[i])) return MPDP_ERR_INVALID_ARG;
    std::vector<int> parent(n);
    for (int i = 0; i < n; i++) parent[i] = i;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    std::vector<std::pair<int, int>> seen;
    seen.reserve(m);
    int comps = n;
    for (int e = 0; e < m; e++) {
        const int u = q->edges[e].u, v = q->edges[e].v;
        const double s = q->edges[e].sel;
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(s > 0.0) || !(s <= 1.0)) return MPDP_ERR_INVALID_ARG;
        seen.push_back({std::min(u, v), std::max(u, v)});
        const int a = find(u), b = find(v);
        if (a != b) {
            parent[a] = b;
            comps--;
        }
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return MPDP_ERR_INVALID_ARG;
    if (comps != 1) return MPDP_ERR_DISCONNECTED;
    return MPDP_OK;
}

int mpdp_optimize(mpdp_ctx* ctx, const mpdp_query* q, int64_t* handle)
{
    if (!ctx || !q || !handle) return MPDP_ERR_INVALID_ARG;
    *handle = -1;
    if (q->mode == MPDP_MODE_EXACT) return mpdp_optimize_batch(ctx, q, 1, handle);
    const int vrc = validate_heuristic(q);
    if (vrc != MPDP_OK) return vrc;
    CK(ctx, cudaSetDevice(ctx->device));
    if (!ctx->xd) ctx->xd = new mpdp::XdExecutor();
    mpdp::HeuristicQuery hq;
    hq.n = q->n_rels;
    hq.mode = q->mode;
    hq.k = q->k;
    hq.t = q->t;
    hq.card = q->card;
    hq.model = ctx->model;
    for (int e = 0; e < q->n_edges; e++) {
        hq.eu.push_back(q->edges[e].u);
        hq.ev.push_back(q->edges[e].v);
        hq.sel.push_back(q->edges[e].sel);
    }
    mpdp::HeuristicResult res;
    const int rc = mpdp::run_heuristic(hq, *ctx->xd, ctx->stream, ctx->num_sms, res);
    if (rc != MPDP_OK) {
        ctx->last_error = "heuristic optimization failed";
        return rc;
    }
    const int64_t h = ctx->next_handle++;
    ctx->heur[h] = std::move(res);
    *handle = h;
    return MPDP_OK;
}

int mpdp_set_model(mpdp_ctx* ctx, mpdp_mlp* model)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    if (model && mpdp_mlp_param_count(model) != (int64_t)mpdp::kEdgeFeatures * 256 + 256 * 3 + 256 * 256 * 2 + 256 + 1)
        return MPDP_ERR_INVALID_ARG;
    ctx->model = model;
    return MPDP_OK;
}

int mpdp_edge_features(const mpdp_query* q, float* out, int32_t cap_rows)
{
    if (!q || !out) return MPDP_ERR_INVALID_ARG;
    const int n = q->n_rels, m = q->n_edges;
    if (n < 1 || m < 0 || !q->card || (m > 0 && !q->edges)) return MPDP_ERR_INVALID_ARG;
    if (cap_rows < m) return MPDP_ERR_BUFFER_TOO_SMALL;
    std::vector<double> lcard(n), lsel(m);
    std::vector<int> eu(m), ev(m);
    for (int i = 0; i < n; i++) {
        if (!finite_pos(q->card[i])) return MPDP_ERR_INVALID_ARG;
        lcard[i] = mpdp::xd_log2(mpdp::xd_make(q->card[i], 0));
    }
    for (int e = 0; e < m; e++) {
        const int u = q->edges[e].u, v = q->edges[e].v;
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(q->edges[e].sel > 0.0) || !(q->edges[e].sel <= 1.0))
            return MPDP_ERR_INVALID_ARG;
        eu[e] = std::min(u, v);
        ev[e] = std::max(u, v);
        lsel[e] = mpdp::xd_log2(mpdp::xd_make(q->edges[e].sel, 0));
    }
    std::vector<float> f;
    mpdp::edge_features(n, lcard, eu, ev, lsel, f);
    if (!f.empty()) memcpy(out, f.data(), f.size() * sizeof(float));
    return MPDP_OK;
}

int mpdp_get_cost_xd(mpdp_ctx* ctx, int64_t handle, double* mant, int32_t* exp2)
{
    if (!ctx || !mant || !exp2) return MPDP_ERR_INVALID_ARG;
    auto hit = ctx->heur.find(handle);
    if (hit != ctx->heur.end()) {
        *mant = hit->second.cost.m;
        *exp2 = hit->second.cost.e;
        return MPDP_OK;
    }
    double c = 0.0;
    const int rc = mpdp_get_plan(ctx, handle, nullptr, 0, nullptr, &c, nullptr);
    if (rc != MPDP_OK) return rc;
    const mpdp::XD x = mpdp::xd_make(c, 0);
    *mant = x.m;
    *exp2 = x.e;
    return MPDP_OK;
}

int mpdp_get_plan(mpdp_ctx* ctx, int64_t handle, mpdp_plan_node* nodes, int32_t cap, int32_t* n_nodes,
                  double* cost, mpdp_stats* st)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    auto hit = ctx->heur.find(handle);
    if (hit != ctx->heur.end()) {
        const mpdp::HeuristicResult& r = hit->second;
        const int nn = (int)r.nodes.size();
        if (nodes && cap < nn) return MPDP_ERR_BUFFER_TOO_SMALL;
        if (nodes) memcpy(nodes, r.nodes.data(), sizeof(mpdp_plan_node) * nn);
        if (n_nodes) *n_nodes = nn;
        if (cost) *cost = nn ? r.nodes[0].cost : 0.0;
        if (st) {
            memset(st, 0, sizeof(*st));
            st->enumeration = MPDP_ENUM_BLOCKS;
            st->heavy_sets = (uint64_t)r.subproblems;  // exact sub-problems solved
            st->filter_steps = r.learned_won ? 1 : 0;  // learned modes: the learned plan was kept
        }
        return MPDP_OK;
    }
    auto it = ctx->handles.find(handle);
    if (it == ctx->handles.end()) return MPDP_ERR_BAD_HANDLE;
    Record& rec = ctx->recs[it->second.rec];
    const int idx = it->second.idx;
    CK(ctx, cudaEventSynchronize(rec.done));
    const DevOut& r = rec.host[idx];
    const int status = r.counters.status;
    if (status != MPDP_OK) return status;
    if (r.result.status != MPDP_OK) return r.result.status;
    if (nodes && cap < r.result.n_nodes) return MPDP_ERR_BUFFER_TOO_SMALL;
    if (nodes)
        for (int i = 0; i < r.result.n_nodes; i++) nodes[i] = r.result.nodes[i];
    if (n_nodes) *n_nodes = r.result.n_nodes;
    if (cost) *cost = r.result.cost;
    if (st) {
        memset(st, 0, sizeof(*st));
        const DevCounters& c = r.counters;
        const int n = rec.n[idx];
        st->sets_unranked = c.unranked;
        for (int k = 2; k <= n && k < kLevels; k++) {
            st->connected_per_level[k] = c.list_count[k];
            st->evaluated_per_level[k] = c.evaluated[k];
            st->ccp_per_level[k] = c.ccp[k];
            st->sets_connected += c.list_count[k];
            st->pairs_evaluated += c.evaluated[k];
            st->ccp_pairs += c.ccp[k];
        }
        st->connected_per_level[1] = (uint64_t)n;
        st->heavy_sets = c.heavy;
        st->memo_bytes = rec.memo_kind == MPDP_MEMO_DENSE ? ((uint64_t)20 << n)
                                                          : (uint64_t)c.memo_slots * sizeof(HashSlot);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, rec.t0, rec.t1) == cudaSuccess) st->device_ms = ms;
        else cudaGetLastError();
        st->enumeration = rec.enumeration[idx];
        st->memo_kind = rec.memo_kind;
        st->h2d_bytes = rec.h2d[idx];
        st->d2h_bytes = sizeof(DevOut);
        st->filter_steps = c.filter_steps;
    }
    return MPDP_OK;
}

int mpdp_release(mpdp_ctx* ctx, int64_t handle)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    if (ctx->heur.erase(handle)) return MPDP_OK;
    auto it = ctx->handles.find(handle);
    if (it == ctx->handles.end()) return MPDP_ERR_BAD_HANDLE;
    Record& rec = ctx->recs[it->second.rec];
    CK(ctx, cudaEventSynchronize(rec.done));
    ctx->handles.erase(it);
    if (--rec.refs <= 0) rec.in_use = false;
    return MPDP_OK;
}

int mpdp_get_plans(mpdp_ctx* ctx, const int64_t* handles, int32_t count, mpdp_plan_node* nodes, int32_t stride,
                   int32_t* n_nodes, double* costs, int32_t* status, mpdp_stats* stats)
{
    if (!ctx || count < 0 || (count > 0 && (!handles || !n_nodes || !costs || !status)) || stride < 0 ||
        (nodes == nullptr && stride != 0))
        return MPDP_ERR_INVALID_ARG;
    int rc = MPDP_OK;
    for (int i = 0; i < count; i++) {
        n_nodes[i] = 0;
        costs[i] = 0.0;
        const int r = mpdp_get_plan(ctx, handles[i], nodes ? nodes + (size_t)i * stride : nullptr, stride,
                                    &n_nodes[i], &costs[i], stats ? &stats[i] : nullptr);
        status[i] = r;
        if (r == MPDP_ERR_BAD_HANDLE) {
            rc = MPDP_ERR_BAD_HANDLE;
            continue;
        }
        const int rr = mpdp_release(ctx, handles[i]);
        if (rr != MPDP_OK && status[i] == MPDP_OK) status[i] = rr;
    }
    return rc;
}

int mpdp_optimize_batch_device(mpdp_ctx* ctx, int32_t nq, const int32_t* n_rels, const int32_t* n_edges,
                               const double* d_card, const mpdp_edge* d_edges, int32_t cost_model,
                               mpdp_plan_node* d_nodes, double* d_cost, int32_t* d_status)
{
    if (!ctx || nq < 0 || (nq > 0 && (!n_rels || !n_edges || !d_card || !d_nodes || !d_cost || !d_status)))
        return MPDP_ERR_INVALID_ARG;
    if (cost_model != MPDP_COST_COUT) return MPDP_ERR_INVALID_ARG;
    if (nq > kMaxBatch) return MPDP_ERR_TOO_LARGE;
    std::vector<PlanQuery> pq(nq);
    unsigned long long co = 0, eo = 0;
    for (int i = 0; i < nq; i++) {
        const int n = n_rels[i], m = n_edges[i];
        if (n < 1 || m < 0 || m > edges_max(n)) return MPDP_ERR_INVALID_ARG;
        if (n > MPDP_MAX_EXACT_RELS) return MPDP_ERR_TOO_LARGE;
        pq[i] = PlanQuery{n, m, resolve_enumeration(ctx->cfg, n, m), nullptr, nullptr, co, eo};
        co += n;
        eo += m;
    }
    if (eo > 0 && !d_edges) return MPDP_ERR_INVALID_ARG;
    if (nq == 0) return MPDP_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    std::vector<std::pair<int, int>> parts;
    int rc = split_batches(ctx, pq, parts);
    if (rc != MPDP_OK) return rc;
    if (parts.size() != 1) return MPDP_ERR_ADMISSION;
    return submit_batch(ctx, pq, false, d_card, d_edges, nullptr, d_nodes, d_cost, d_status);
}

int mpdp_optimize_device(mpdp_ctx* ctx, int32_t n_rels, int32_t n_edges, const double* d_card,
                         const mpdp_edge* d_edges, int32_t cost_model, mpdp_plan_node* d_nodes, double* d_cost,
                         int32_t* d_status)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    return mpdp_optimize_batch_device(ctx, 1, &n_rels, &n_edges, d_card, d_edges, cost_model, d_nodes, d_cost,
                                      d_status);
}

int mpdp_profile(mpdp_ctx* ctx, int mode)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    if (mode != MPDP_PROFILE_OFF && mode != MPDP_PROFILE_SERIAL && mode != MPDP_PROFILE_CONCURRENT)
        return MPDP_ERR_INVALID_ARG;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->profiling = mode;
    ctx->hook.reset();
    return MPDP_OK;
}

int mpdp_profile_read(mpdp_ctx* ctx, double* ms, uint64_t* launches)
{
    std::vector<double> active(MPDP_KC_COUNT);
    return mpdp_profile_read_active(ctx, ms, active.data(), launches);
}

int mpdp_profile_read_active(mpdp_ctx* ctx, double* ms, double* active_ms, uint64_t* launches)
{
    if (!ctx || !ms || !active_ms || !launches) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < MPDP_KC_COUNT; i++) {
        ms[i] = 0.0;
        active_ms[i] = 0.0;
        launches[i] = 0;
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));  // the lanes join back into it
    EventHook& h = ctx->hook;
    if (h.err != cudaSuccess) {
        ctx->last_error = std::string("profiling events: ") + cudaGetErrorString(h.err);
        h.err = cudaSuccess;
        h.reset();
        return MPDP_ERR_CUDA;
    }
    // per (batch, class): launch intervals on the batch's time line
    std::map<std::pair<int, int>, std::vector<std::pair<float, float>>> spans;
    for (const auto& r : h.recs) {
        float t = 0.f;
        CK(ctx, cudaEventElapsedTime(&t, h.pool[r.begin], h.pool[r.begin + 1]));
        if (r.cls < 0 || r.cls >= MPDP_KC_COUNT) continue;
        ms[r.cls] += t;
        launches[r.cls] += 1;
        if (r.group < 0) {
            active_ms[r.cls] += t;
            continue;
        }
        float t0 = 0.f;
        CK(ctx, cudaEventElapsedTime(&t0, h.pool[h.origins[r.group]], h.pool[r.begin]));
        spans[{r.group, r.cls}].emplace_back(t0, t0 + t);
    }
    for (auto& kv : spans) {
        auto& v = kv.second;
        std::sort(v.begin(), v.end());
        double total = 0.0, lo = v[0].first, hi = v[0].second;
        for (size_t i = 1; i < v.size(); i++) {
            if (v[i].first > hi) {
                total += hi - lo;
                lo = v[i].first;
                hi = v[i].second;
            } else if (v[i].second > hi) {
                hi = v[i].second;
            }
        }
        active_ms[kv.first.second] += total + (hi - lo);
    }
    h.reset();
    return MPDP_OK;
}

int mpdp_sync(mpdp_ctx* ctx)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MPDP_OK;
}

int mpdp_memo_lookup(mpdp_ctx* ctx, int64_t handle, const uint64_t* sets, int32_t count, double* costs,
                     uint64_t* lefts)
{
    if (!ctx || count < 0 || (count > 0 && (!sets || !costs || !lefts))) return MPDP_ERR_INVALID_ARG;
    auto it = ctx->handles.find(handle);
    if (it == ctx->handles.end()) return MPDP_ERR_BAD_HANDLE;
    Record& rec = ctx->recs[it->second.rec];
    const int idx = it->second.idx;
    if (rec.seq != ctx->last_seq) return MPDP_ERR_STALE;
    if (count == 0) return MPDP_OK;
    const uint64_t full = ((uint64_t)1 << rec.n[idx]) - 1;
    std::vector<uint32_t> hs(count);
    for (int i = 0; i < count; i++) {
        if (sets[i] == 0 || (sets[i] & ~full)) return MPDP_ERR_INVALID_ARG;
        hs[i] = (uint32_t)sets[i];
    }
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaEventSynchronize(rec.done));
    if (rec.host[idx].counters.status != MPDP_OK) return rec.host[idx].counters.status;
    uint32_t* d_sets = nullptr;
    double* d_costs = nullptr;
    uint32_t* d_lefts = nullptr;
    int rc = MPDP_OK;
    if (cudaMalloc(&d_sets, count * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&d_costs, count * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_lefts, count * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        rc = MPDP_ERR_OOM;
    }
    std::vector<uint32_t> hl(count);
    if (rc == MPDP_OK) {
        const BatchArgs a = batch_args(ctx, rec.nq, 0);
        cudaError_t e =
            cudaMemcpyAsync(d_sets, hs.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = enqueue_memo_lookup(a, rec.memo_kind, idx, d_sets, count, d_costs, d_lefts, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(costs, d_costs, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hl.data(), d_lefts, count * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            ctx->last_error = std::string("memo lookup: ") + cudaGetErrorString(e);
            rc = MPDP_ERR_CUDA;
        }
    }
    cudaFree(d_sets);
    cudaFree(d_costs);
    cudaFree(d_lefts);
    if (rc != MPDP_OK) return rc;
    for (int i = 0; i < count; i++) lefts[i] = hl[i];
    return MPDP_OK;
}

}  // extern "C"

namespace mpdp {

int validate_host_query(const mpdp_query* q) { return validate_query(q, MPDP_MAX_EXACT_RELS); }

// Workspace of one device batch under the same rules as a context's batch
// split (for callers that form batches themselves).
size_t batch_workspace_bytes(const int* n, const int* m, int count, const mpdp_config& cfg)
{
    size_t L = 0, V = 0, M = 0, A = 0;
    for (int i = 0; i < count; i++) {
        const QuerySize z = query_size(n[i], resolve_enumeration(cfg, n[i], m[i]), cfg.memo_kind);
        L += z.lists;
        V += z.heavy;
        M += z.memo;
        A += z.hash;
    }
    return var_bytes_of(L, V, M, A) + fixed_bytes();
}

}  // namespace mpdp
