// C ABI of the MPDP optimizer: contexts, handles, workspace, CUDA graphs.
//
// One exact optimization (Algorithm "MPDP on GPU", Sec. 5) is enqueued as:
//   host -> device copy of the staged query (host path) or a gather kernel
//   (device path); the DP pipeline (replayed from a CUDA graph captured once
//   per shape); a device -> host copy of plan + counters (host path) or a
//   publish kernel (device path).  Nothing in between waits for the host:
//   the paper's per-level host round trip (Sec. 6.2, small queries) is gone.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mpdp.h"
#include "mpdp_launch.h"

using namespace mpdp;

namespace {

struct HandleSlot {
    bool used = false;
    int64_t handle = -1;
    HostResult* host = nullptr;  // pinned
    cudaEvent_t done = nullptr, t0 = nullptr, t1 = nullptr;
    int n = 0;
    int enumeration = 0;
    int memo_kind = 0;
    uint64_t h2d_bytes = 0;
};

// Profiling mode: a pair of events around every launch, summed per class.
struct EventHook : LaunchHook {
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, size_t>> recs;  // (class, index of the begin event)
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
    void begin(int cls, cudaStream_t st) override
    {
        recs.emplace_back(cls, next);
        cudaError_t r = cudaEventRecord(take(), st);
        if (r != cudaSuccess) err = r;
    }
    void end(int, cudaStream_t st) override
    {
        cudaError_t r = cudaEventRecord(take(), st);
        if (r != cudaSuccess) err = r;
    }
    ~EventHook()
    {
        for (auto e : pool)
            if (e) cudaEventDestroy(e);
    }
};

struct DevOut {  // device twin of HostResult: one copy reads both back
    DevResult result;
    DevCounters counters;
};

using GraphKey = std::tuple<int, int, int, int, int, int>;

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

const mpdp_config kDefaultConfig = {MPDP_MEMO_DENSE, MPDP_ENUM_AUTO, 64, 1, 1, 32};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int edges_max(int n) { return n * (n - 1) / 2; }

}  // namespace

struct mpdp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;          // work stream (borrowed; nullptr = default stream)
    cudaStream_t capture_stream = nullptr;  // private, only used to capture graphs
    size_t budget = 0;
    mpdp_config cfg = kDefaultConfig;
    int num_sms = 152;
    Workspace ws;
    DevOut* out = nullptr;
    void* ws_block = nullptr;  // one allocation for all workspace buffers
    size_t ws_bytes = 0;
    bool ws_dense = false, ws_hash = false;
    // ring of pinned staging buffers: the host can stage queries ahead of
    // the device; each buffer's event marks its host->device copy as done
    static constexpr int kStageRing = 32;
    StagedQuery* h_staged = nullptr;  // pinned, kStageRing entries
    cudaEvent_t staged_free[kStageRing] = {};
    int stage_next = 0;
    std::map<GraphKey, GraphEntry> graphs;
    std::vector<HandleSlot> slots;
    int64_t next_handle = 1;
    int64_t last_exact_handle = -1;
    int last_memo_kind = MPDP_MEMO_DENSE;
    int last_launches = 0;
    bool profiling = false;
    EventHook hook;
    std::string last_error;
};

#define CK(ctx, call)                                                       \
    do {                                                                    \
        cudaError_t e__ = (call);                                           \
        if (e__ != cudaSuccess) {                                           \
            (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(e__); \
            return MPDP_ERR_CUDA;                                           \
        }                                                                   \
    } while (0)

static bool finite_pos(double x) { return x > 0.0 && x <= 1.7976931348623157e308; }

// Host-side validation of a query (same rules as the device ingest kernel).
static int validate_query(const mpdp_query* q, int max_n)
{
    if (!q) return MPDP_ERR_INVALID_ARG;
    const int n = q->n_rels, m = q->n_edges;
    if (n < 1) return MPDP_ERR_INVALID_ARG;
    if (n > max_n) return MPDP_ERR_TOO_LARGE;
    if (q->cost_model != MPDP_COST_COUT || q->reserved != 0) return MPDP_ERR_INVALID_ARG;
    if (m < 0 || m > edges_max(n)) return MPDP_ERR_INVALID_ARG;
    if (!q->card || (m > 0 && !q->edges)) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++)
        if (!finite_pos(q->card[i])) return MPDP_ERR_INVALID_ARG;
    std::vector<uint64_t> adj((size_t)n * ((n + 63) / 64), 0);
    const int words = (n + 63) / 64;
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

static size_t workspace_bytes(int n, bool dense, bool hash)
{
    size_t b = align_up(sizeof(StagedQuery)) + align_up(sizeof(DevQuery)) + align_up(sizeof(DevOut));
    const size_t le = list_entries(n);
    b += 2 * align_up(le * sizeof(uint32_t));
    if (dense) {
        const size_t full = (size_t)1 << n;
        b += align_up(full * sizeof(double)) + align_up(full * sizeof(uint32_t));
    }
    if (hash) b += align_up(hash_arena_slots(n) * sizeof(HashSlot)) + align_up(sizeof(HashLayout));
    return b;
}

static void destroy_graphs(mpdp_ctx* ctx)
{
    for (auto& kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
}

// Make sure the workspace holds n relations with the memo kind requested.
static int ensure_workspace(mpdp_ctx* ctx, int n, int memo_kind)
{
    const bool need_dense = memo_kind == MPDP_MEMO_DENSE;
    const bool need_hash = memo_kind == MPDP_MEMO_HASH;
    if (ctx->ws_block && ctx->ws.n_cap >= n && (!need_dense || ctx->ws_dense) &&
        (!need_hash || ctx->ws_hash))
        return MPDP_OK;
    // keep the capacity reached so far, but only the memo kind asked for now
    const int new_n = n > ctx->ws.n_cap ? n : ctx->ws.n_cap;
    const bool dense = need_dense;
    const bool hash = need_hash;
    const size_t bytes = workspace_bytes(new_n, dense, hash);
    if (bytes > ctx->budget) return MPDP_ERR_ADMISSION;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    destroy_graphs(ctx);
    if (ctx->ws_block) cudaFree(ctx->ws_block);
    ctx->ws_block = nullptr;
    ctx->ws = Workspace();
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->last_error = std::string("cudaMalloc workspace: ") + cudaGetErrorString(e);
        ctx->ws_dense = ctx->ws_hash = false;
        return MPDP_ERR_OOM;
    }
    ctx->ws_block = p;
    ctx->ws_bytes = bytes;
    char* c = static_cast<char*>(p);
    auto take = [&](size_t sz) {
        char* r = c;
        c += align_up(sz);
        return r;
    };
    Workspace& ws = ctx->ws;
    ws.n_cap = new_n;
    ws.staged = reinterpret_cast<StagedQuery*>(take(sizeof(StagedQuery)));
    ws.query = reinterpret_cast<DevQuery*>(take(sizeof(DevQuery)));
    ctx->out = reinterpret_cast<DevOut*>(take(sizeof(DevOut)));
    ws.result = &ctx->out->result;
    ws.counters = &ctx->out->counters;
    const size_t le = list_entries(new_n);
    ws.lists = reinterpret_cast<uint32_t*>(take(le * sizeof(uint32_t)));
    ws.heavy = reinterpret_cast<uint32_t*>(take(le * sizeof(uint32_t)));
    if (dense) {
        const size_t full = (size_t)1 << new_n;
        ws.dcost = reinterpret_cast<double*>(take(full * sizeof(double)));
        ws.dleft = reinterpret_cast<uint32_t*>(take(full * sizeof(uint32_t)));
    }
    if (hash) {
        ws.arena_slots = hash_arena_slots(new_n);
        ws.arena = reinterpret_cast<HashSlot*>(take(ws.arena_slots * sizeof(HashSlot)));
        ws.layout = reinterpret_cast<HashLayout*>(take(sizeof(HashLayout)));
    }
    ctx->ws_dense = dense;
    ctx->ws_hash = hash;
    ctx->last_exact_handle = -1;
    // start from zeroed counters and result
    CK(ctx, cudaMemsetAsync(ctx->out, 0, sizeof(DevOut), ctx->stream));
    return MPDP_OK;
}

static PipelineCfg pipeline_cfg(const mpdp_ctx* ctx, int n, int enumeration)
{
    PipelineCfg pc;
    pc.n = n;
    pc.enumeration = enumeration;
    pc.memo_kind = ctx->cfg.memo_kind;
    pc.heavy_threshold = ctx->cfg.heavy_threshold;
    pc.use_ccc = ctx->cfg.use_ccc;
    pc.run_length = ctx->cfg.run_length;
    pc.num_sms = ctx->num_sms;
    pc.blocks_per_sm = 4;
    return pc;
}

// Enqueue the DP pipeline on the work stream: graph replay or direct launches.
static int run_pipeline(mpdp_ctx* ctx, int n, int enumeration, int* launches)
{
    const PipelineCfg pc = pipeline_cfg(ctx, n, enumeration);
    if (ctx->profiling || !ctx->cfg.use_graphs) {
        CK(ctx, enqueue_pipeline(ctx->ws, pc, ctx->stream, launches,
                                 ctx->profiling ? &ctx->hook : nullptr));
        return MPDP_OK;
    }
    const GraphKey key(n, enumeration, pc.memo_kind, pc.heavy_threshold, pc.use_ccc, pc.run_length);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        GraphEntry g;
        cudaGraph_t graph = nullptr;
        CK(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_pipeline(ctx->ws, pc, ctx->capture_stream, &g.launches);
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            ctx->last_error = std::string("graph capture: ") +
                              cudaGetErrorString(e != cudaSuccess ? e : e2);
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

static int resolve_enumeration(const mpdp_ctx* ctx, int n, int m)
{
    if (ctx->cfg.enumeration == MPDP_ENUM_TREE || ctx->cfg.enumeration == MPDP_ENUM_BLOCKS)
        return ctx->cfg.enumeration;
    return (m == n - 1) ? MPDP_ENUM_TREE : MPDP_ENUM_BLOCKS;
}

static int acquire_slot(mpdp_ctx* ctx, HandleSlot** out)
{
    for (auto& s : ctx->slots)
        if (!s.used) {
            *out = &s;
            return MPDP_OK;
        }
    HandleSlot s;
    CK(ctx, cudaMallocHost(reinterpret_cast<void**>(&s.host), sizeof(HostResult)));
    CK(ctx, cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    CK(ctx, cudaEventCreate(&s.t0));
    CK(ctx, cudaEventCreate(&s.t1));
    ctx->slots.push_back(s);
    *out = &ctx->slots.back();
    return MPDP_OK;
}

static HandleSlot* find_slot(mpdp_ctx* ctx, int64_t handle)
{
    for (auto& s : ctx->slots)
        if (s.used && s.handle == handle) return &s;
    return nullptr;
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
    default: return "unknown error";
    }
}

const char* mpdp_last_error(const mpdp_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int32_t mpdp_last_launch_count(const mpdp_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

size_t mpdp_workspace_bytes(int32_t n_rels, const mpdp_config* cfg)
{
    if (n_rels < 1 || n_rels > MPDP_MAX_EXACT_RELS) return 0;
    const int kind = cfg ? cfg->memo_kind : MPDP_MEMO_DENSE;
    return workspace_bytes(n_rels, kind == MPDP_MEMO_DENSE, kind == MPDP_MEMO_HASH);
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
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&ctx->h_staged),
                       sizeof(StagedQuery) * mpdp_ctx::kStageRing) != cudaSuccess) {
        cudaGetLastError();
        mpdp_destroy(ctx);
        return MPDP_ERR_CUDA;
    }
    for (int i = 0; i < mpdp_ctx::kStageRing; i++) {
        if (cudaEventCreateWithFlags(&ctx->staged_free[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            mpdp_destroy(ctx);
            return MPDP_ERR_CUDA;
        }
    }
    *out = ctx;
    return MPDP_OK;
}

void mpdp_destroy(mpdp_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    destroy_graphs(ctx);
    for (auto& s : ctx->slots) {
        if (s.host) cudaFreeHost(s.host);
        if (s.done) cudaEventDestroy(s.done);
        if (s.t0) cudaEventDestroy(s.t0);
        if (s.t1) cudaEventDestroy(s.t1);
    }
    if (ctx->ws_block) cudaFree(ctx->ws_block);
    if (ctx->h_staged) cudaFreeHost(ctx->h_staged);
    for (int i = 0; i < mpdp_ctx::kStageRing; i++)
        if (ctx->staged_free[i]) cudaEventDestroy(ctx->staged_free[i]);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    cudaGetLastError();
    delete ctx;
}

int mpdp_set_config(mpdp_ctx* ctx, const mpdp_config* cfg)
{
    if (!ctx || !cfg) return MPDP_ERR_INVALID_ARG;
    if (cfg->memo_kind != MPDP_MEMO_DENSE && cfg->memo_kind != MPDP_MEMO_HASH) return MPDP_ERR_INVALID_ARG;
    if (cfg->enumeration < MPDP_ENUM_AUTO || cfg->enumeration > MPDP_ENUM_BLOCKS) return MPDP_ERR_INVALID_ARG;
    if (cfg->heavy_threshold < 0 || cfg->run_length < 1 || cfg->run_length > 32) return MPDP_ERR_INVALID_ARG;
    ctx->cfg = *cfg;
    return MPDP_OK;
}

int mpdp_get_config(const mpdp_ctx* ctx, mpdp_config* cfg)
{
    if (!cfg) return MPDP_ERR_INVALID_ARG;
    *cfg = ctx ? ctx->cfg : kDefaultConfig;
    return MPDP_OK;
}

int mpdp_optimize(mpdp_ctx* ctx, const mpdp_query* q, int64_t* handle)
{
    if (!ctx || !q || !handle) return MPDP_ERR_INVALID_ARG;
    *handle = -1;
    if (q->mode != MPDP_MODE_EXACT) return MPDP_ERR_NOT_IMPLEMENTED;
    int rc = validate_query(q, MPDP_MAX_EXACT_RELS);
    if (rc != MPDP_OK) return rc;
    CK(ctx, cudaSetDevice(ctx->device));
    const int n = q->n_rels, m = q->n_edges;
    rc = ensure_workspace(ctx, n, ctx->cfg.memo_kind);
    if (rc != MPDP_OK) return rc;
    const int enumeration = resolve_enumeration(ctx, n, m);
    HandleSlot* slot = nullptr;
    rc = acquire_slot(ctx, &slot);
    if (rc != MPDP_OK) return rc;

    // stage the query in the next ring buffer, once its previous copy has run
    const int ring = ctx->stage_next;
    ctx->stage_next = (ring + 1) % mpdp_ctx::kStageRing;
    CK(ctx, cudaEventSynchronize(ctx->staged_free[ring]));
    StagedQuery* h = ctx->h_staged + ring;
    h->n = n;
    h->n_edges = m;
    h->cost_model = q->cost_model;
    h->pad = 0;
    for (int i = 0; i < kMaxRels; i++) h->card[i] = i < n ? q->card[i] : 1.0;
    for (int e = 0; e < m; e++) h->edges[e] = q->edges[e];
    const size_t bytes = offsetof(StagedQuery, edges) + (size_t)m * sizeof(mpdp_edge);
    CK(ctx, cudaMemcpyAsync(ctx->ws.staged, h, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->staged_free[ring], ctx->stream));

    CK(ctx, cudaEventRecord(slot->t0, ctx->stream));
    int launches = 0;
    rc = run_pipeline(ctx, n, enumeration, &launches);
    if (rc != MPDP_OK) return rc;
    CK(ctx, cudaEventRecord(slot->t1, ctx->stream));
    CK(ctx, cudaMemcpyAsync(slot->host, ctx->out, sizeof(HostResult), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaEventRecord(slot->done, ctx->stream));
    slot->used = true;
    slot->handle = ctx->next_handle++;
    slot->n = n;
    slot->enumeration = enumeration;
    slot->memo_kind = ctx->cfg.memo_kind;
    slot->h2d_bytes = bytes;
    ctx->last_exact_handle = slot->handle;
    ctx->last_memo_kind = ctx->cfg.memo_kind;
    ctx->last_launches = launches;
    *handle = slot->handle;
    return MPDP_OK;
}

int mpdp_optimize_batch(mpdp_ctx* ctx, const mpdp_query* qs, int32_t nq, int64_t* handles)
{
    if (!ctx || (nq > 0 && (!qs || !handles)) || nq < 0) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < nq; i++) handles[i] = -1;
    for (int i = 0; i < nq; i++) {
        int rc = mpdp_optimize(ctx, &qs[i], &handles[i]);
        if (rc != MPDP_OK) return rc;
    }
    return MPDP_OK;
}

int mpdp_get_plan(mpdp_ctx* ctx, int64_t handle, mpdp_plan_node* nodes, int32_t cap, int32_t* n_nodes,
                  double* cost, mpdp_stats* st)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    HandleSlot* slot = find_slot(ctx, handle);
    if (!slot) return MPDP_ERR_BAD_HANDLE;
    CK(ctx, cudaEventSynchronize(slot->done));
    const HostResult& r = *slot->host;
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
        st->sets_unranked = c.unranked;
        for (int k = 2; k <= slot->n && k < kLevels; k++) {
            st->connected_per_level[k] = c.list_count[k];
            st->evaluated_per_level[k] = c.evaluated[k];
            st->ccp_per_level[k] = c.ccp[k];
            st->sets_connected += c.list_count[k];
            st->pairs_evaluated += c.evaluated[k];
            st->ccp_pairs += c.ccp[k];
        }
        st->connected_per_level[1] = (uint64_t)slot->n;
        st->heavy_sets = c.heavy;
        st->memo_bytes = slot->memo_kind == MPDP_MEMO_DENSE
                             ? ((uint64_t)12 << slot->n)
                             : (uint64_t)c.memo_slots * sizeof(HashSlot);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, slot->t0, slot->t1) == cudaSuccess) st->device_ms = ms;
        else cudaGetLastError();
        st->enumeration = slot->enumeration;
        st->memo_kind = slot->memo_kind;
        st->h2d_bytes = slot->h2d_bytes;
        st->d2h_bytes = sizeof(HostResult);
        st->filter_steps = c.filter_steps;
    }
    return MPDP_OK;
}

int mpdp_release(mpdp_ctx* ctx, int64_t handle)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    HandleSlot* slot = find_slot(ctx, handle);
    if (!slot) return MPDP_ERR_BAD_HANDLE;
    CK(ctx, cudaEventSynchronize(slot->done));
    slot->used = false;
    slot->handle = -1;
    return MPDP_OK;
}

int mpdp_optimize_device(mpdp_ctx* ctx, int32_t n_rels, int32_t n_edges, const double* d_card,
                         const mpdp_edge* d_edges, int32_t cost_model, mpdp_plan_node* d_nodes,
                         double* d_cost, int32_t* d_status)
{
    if (!ctx || !d_card || (n_edges > 0 && !d_edges) || !d_nodes || !d_cost || !d_status)
        return MPDP_ERR_INVALID_ARG;
    if (n_rels < 1 || n_edges < 0 || n_edges > edges_max(n_rels)) return MPDP_ERR_INVALID_ARG;
    if (n_rels > MPDP_MAX_EXACT_RELS) return MPDP_ERR_TOO_LARGE;
    if (cost_model != MPDP_COST_COUT) return MPDP_ERR_INVALID_ARG;
    CK(ctx, cudaSetDevice(ctx->device));
    int rc = ensure_workspace(ctx, n_rels, ctx->cfg.memo_kind);
    if (rc != MPDP_OK) return rc;
    const int enumeration = resolve_enumeration(ctx, n_rels, n_edges);
    LaunchHook* hook = ctx->profiling ? &ctx->hook : nullptr;
    CK(ctx, enqueue_stage_device(d_card, d_edges, n_rels, n_edges, cost_model, ctx->ws.staged,
                                 ctx->stream, hook));
    int launches = 0;
    rc = run_pipeline(ctx, n_rels, enumeration, &launches);
    if (rc != MPDP_OK) return rc;
    CK(ctx, enqueue_publish(ctx->ws, d_nodes, d_cost, d_status, ctx->stream, hook));
    ctx->last_launches = launches + 2;
    ctx->last_exact_handle = -1;
    return MPDP_OK;
}

int mpdp_profile(mpdp_ctx* ctx, int enable)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->profiling = enable != 0;
    ctx->hook.recs.clear();
    ctx->hook.next = 0;
    return MPDP_OK;
}

int mpdp_profile_read(mpdp_ctx* ctx, double* ms, uint64_t* launches)
{
    if (!ctx || !ms || !launches) return MPDP_ERR_INVALID_ARG;
    for (int i = 0; i < MPDP_KC_COUNT; i++) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    EventHook& h = ctx->hook;
    if (h.err != cudaSuccess) {
        ctx->last_error = std::string("profiling events: ") + cudaGetErrorString(h.err);
        h.err = cudaSuccess;
        h.recs.clear();
        h.next = 0;
        return MPDP_ERR_CUDA;
    }
    for (auto& r : h.recs) {
        float t = 0.f;
        CK(ctx, cudaEventElapsedTime(&t, h.pool[r.second], h.pool[r.second + 1]));
        if (r.first >= 0 && r.first < MPDP_KC_COUNT) {
            ms[r.first] += t;
            launches[r.first] += 1;
        }
    }
    h.recs.clear();
    h.next = 0;
    return MPDP_OK;
}

int mpdp_sync(mpdp_ctx* ctx)
{
    if (!ctx) return MPDP_ERR_INVALID_ARG;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!ctx->out) return MPDP_OK;
    int status = 0;
    CK(ctx, cudaMemcpy(&status, &ctx->out->counters.status, sizeof(int), cudaMemcpyDeviceToHost));
    return status;
}

int mpdp_memo_lookup(mpdp_ctx* ctx, int64_t handle, const uint64_t* sets, int32_t count, double* costs,
                     uint64_t* lefts)
{
    if (!ctx || count < 0 || (count > 0 && (!sets || !costs || !lefts))) return MPDP_ERR_INVALID_ARG;
    HandleSlot* slot = find_slot(ctx, handle);
    if (!slot) return MPDP_ERR_BAD_HANDLE;
    if (handle != ctx->last_exact_handle) return MPDP_ERR_STALE;
    if (count == 0) return MPDP_OK;
    const uint64_t full = ((uint64_t)1 << slot->n) - 1;
    std::vector<uint32_t> hs(count);
    for (int i = 0; i < count; i++) {
        if (sets[i] == 0 || (sets[i] & ~full)) return MPDP_ERR_INVALID_ARG;
        hs[i] = (uint32_t)sets[i];
    }
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaEventSynchronize(slot->done));
    if (slot->host->counters.status != MPDP_OK) return slot->host->counters.status;
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
        cudaError_t e = cudaMemcpyAsync(d_sets, hs.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                        ctx->stream);
        if (e == cudaSuccess)
            e = enqueue_memo_lookup(ctx->ws, slot->memo_kind, d_sets, count, d_costs, d_lefts, ctx->stream);
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
