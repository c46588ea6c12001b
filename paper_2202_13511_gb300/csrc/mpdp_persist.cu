// Persistent serving kernel: one resident grid optimizes many exact-mode
// queries of uneven size and shape at once, and takes new ones while it runs.
//
// Every query occupies a query slot with its own workspace (staged query,
// device record, counters, level lists, connectivity bitmap, heavy-set
// entries, dense memo), sized for queries of up to max_rels relations: a
// request is admitted when a slot is free, and the slot count is what the
// memo memory allows.  A slot walks through the steps of the DP as phases,
// each a number of tiles:
//   ingest (1) -> filter (the bitmap sweep's or the connected-set
//   unranking's items) -> level k = 2..n (tiles of the level's connected
//   sets; block mode: then the heavy-set chunks of level k) -> plan fetch (1).
// A tile of a phase runs the same device code as the batched kernels
// (mpdp_kernels.cu), for a one-query batch view of the slot, so results are
// bit-identical to the batched path.  The level barrier of the DP (Sec.
// 2.1.1; Sec. 5) becomes a per-slot counter: the block that finishes a
// phase's last tile computes the next phase (its tile count from the
// counters the finished phase left) and publishes it.  Slots advance
// independently, so the levels of different queries overlap on the GPU.
//
// Claiming work: each slot has one 64-bit word, epoch (high half, bumped at
// every phase change) and next tile (low half).  A block adds 1 to it; the
// old value names the epoch and the tile it got.  The phase of an epoch is
// kept in one of two records chosen by the epoch's parity, written before
// the epoch is published, so a block reads the record of the epoch it
// claimed from; it re-reads the word afterwards and keeps the tile only if
// the epoch is unchanged and the tile is below the phase's tile count.  The
// block that publishes a phase (the one that ended the previous phase, or
// admitted the query) publishes it with its first tile already claimed and
// runs that tile next, so a run of one-tile phases (small levels, heavy-set
// phases of one chunk group, the plan fetch) costs no other block's poll,
// scan and claim between phases.
//
// Requests: the host writes each request (its slot, ticket, query and the
// query's layout) into a ring of pinned, device-mapped memory and publishes
// it by writing its sequence number last.  An idle block takes the next
// request (compare-and-swap on the count of requests taken), copies it into
// the slot and publishes the slot's ingest phase.  A finished query's plan,
// cost and status go to a device-mapped result record of its slot; its
// ticket, written last, tells the host the record is complete.
//
// No block ever waits for another: work is only ever published once it can
// run.  The only loop without work to do is the idle poll, which ends the
// block after `idle_polls` empty polls in a row (the host starts the kernel
// again when it has work) or when the host sets the stop flag.
//
// Memory written and read within this one launch (the memo, lists, counters
// and records of a slot, reused by later requests) must never be read
// through a stale L1 line.  MPDP_COHERENT_LOADS keeps every load a plain
// global load (no non-coherent read-only path, no restrict pointers), and
// every read of another block's writes follows an acquire: a block runs a
// tile only after its claim (an atomic on the slot word that the phase's
// publisher wrote after a fence) and a GPU-scope fence, so the PTX memory
// model makes the phase's inputs, and a reused slot's new contents, visible
// to it, L1 included.
#define MPDP_COHERENT_LOADS
#define MPDP_PHASES_ONLY
#include "mpdp_kernels.cu"

#include <vector>

#include "mpdp_persist.h"

namespace mpdp {
namespace {

enum : int32_t { PH_FREE = 0, PH_INGEST = 1, PH_FILTER = 2, PH_LEVEL = 3, PH_HEAVY = 4, PH_EXTRACT = 5 };

constexpr int kPersistThreads = 256;
constexpr int kPrefRows = 2 * kLevels * kPrefStride;  // level prefix rows of one slot

struct PhaseInfo {
    int32_t phase;
    int32_t level;
    uint32_t total;  // tiles
    uint32_t pad;
};

struct alignas(64) PSlot {
    unsigned long long word;  // epoch << 32 | next tile
    unsigned int done[2];     // tiles finished, by epoch parity
    PhaseInfo info[2];        // phase of the epoch, by epoch parity
    long long ticket;         // request the slot serves
};

struct PRequest {
    unsigned int seq;  // r + 1 for the ring's r-th request; written last
    int32_t slot;
    long long ticket;
    QDesc desc;  // the query's layout within its slot
    int32_t n, m;
    double card[kMaxRels];
    mpdp_edge edges[kMaxEdges];
};

struct PResult {
    long long ticket;
    int32_t status, n_nodes;
    double cost;
    mpdp_plan_node nodes[kPlanNodes];
    unsigned long long done_ticket;  // ticket + 1 once everything above is written
};

struct PArgs {
    int nslots;
    int ring_size;
    int idle_polls;
    uint32_t group_threads;
    PSlot* slots;
    const BatchArgs* slot_args;  // one-query batch view of each slot's workspace
    uint32_t* pref;              // kPrefRows per slot
    PRequest* ring;              // device-mapped host memory
    PResult* results;            // device-mapped host memory
    unsigned long long* taken;   // requests taken from the ring
    const int* stop;             // device-mapped host memory
};

__device__ __forceinline__ PhaseInfo read_info(const PSlot* s, unsigned int parity)
{
    const volatile PhaseInfo* v = &s->info[parity & 1u];
    PhaseInfo r;
    r.phase = v->phase;
    r.level = v->level;
    r.total = v->total;
    r.pad = 0u;
    return r;
}

// Publish epoch `epoch` of slot s with phase `inf` (one thread), its tiles
// below `taken` already claimed by the publishing block.
__device__ void publish_phase(PSlot* s, unsigned int epoch, PhaseInfo inf, unsigned int taken = 0u)
{
    volatile PhaseInfo* v = &s->info[epoch & 1u];
    v->phase = inf.phase;
    v->level = inf.level;
    v->total = inf.total;
    reinterpret_cast<volatile unsigned int*>(s->done)[epoch & 1u] = 0u;
    __threadfence();
    atomicExch(&s->word, ((unsigned long long)epoch << 32) | taken);
}

// Claim the next tiles of slot s (one thread): [tile, tile + count).  A
// phase with many tiles left hands them out kClaim at a time, so that the
// blocks do not all queue on the slot's word for every tile.
constexpr unsigned int kClaim = 4u;

// w, i0: the slot's word and the record of its epoch as the caller's scan
// read them (a hint that sizes the claim; the claim itself is validated).
__device__ bool claim_tile(const PArgs& p, int s, unsigned long long w, PhaseInfo i0, unsigned int& epoch,
                           unsigned int& tile, unsigned int& count, PhaseInfo& inf)
{
    PSlot* sl = p.slots + s;
    const unsigned int want = i0.total - (unsigned int)w >= kClaim * 2u * gridDim.x ? kClaim : 1u;
    const unsigned long long old = atomicAdd(&sl->word, (unsigned long long)want);
    const unsigned int e = (unsigned int)(old >> 32), t = (unsigned int)old;
    __threadfence();
    const PhaseInfo i1 = read_info(sl, e);
    __threadfence();
    const unsigned long long w2 = *reinterpret_cast<volatile unsigned long long*>(&sl->word);
    // a tile below the count holds the epoch, so it cannot have moved on
    if ((unsigned int)(w2 >> 32) != e || i1.phase == PH_FREE || t >= i1.total) return false;
    epoch = e;
    tile = t;
    count = i1.total - t < want ? i1.total - t : want;
    inf = i1;
    return true;
}

// Phase of level k of slot s, or the plan fetch past the last level; writes
// the level's prefix row for the evaluate bodies (one thread).
__device__ PhaseInfo level_phase(const PArgs& p, int s, int k)
{
    const BatchArgs& a = p.slot_args[s];
    const QDesc& d = a.desc[0];
    const volatile DevCounters* cnt = &a.out[0].counters;
    uint32_t* pref = p.pref + (size_t)s * kPrefRows;
    for (; k <= d.n; k++) {
        const uint32_t sets = cnt->list_count[k];
        const uint32_t tiles = (sets + kEvalThreads - 1u) / kEvalThreads;
        uint32_t total = tiles;
        if (d.enumeration == MPDP_ENUM_TREE) {
            uint32_t* row = pref + k * kPrefStride;
            const uint32_t g = group_size(sets, k, p.group_threads);
            const uint32_t G = g > 1u ? g : 0u;
            row[0] = 0u;
            row[1] = G ? sets : tiles;
            row[kMaxBatch + 1] = G;
            if (G) total = (uint32_t)(((unsigned long long)sets * G + kEvalThreads - 1u) / kEvalThreads);
        } else {
            uint32_t* row = pref + (kLevels + k) * kPrefStride;
            row[0] = 0u;
            row[1] = tiles;
            row[kMaxBatch + 1] = 0u;
        }
        if (total) return PhaseInfo{PH_LEVEL, k, total, 0u};
    }
    return PhaseInfo{PH_EXTRACT, 0, 1u, 0u};
}

// What follows phase `cur` of slot s (one thread, after its last tile).
__device__ PhaseInfo next_phase(const PArgs& p, int s, PhaseInfo cur)
{
    const BatchArgs& a = p.slot_args[s];
    const QDesc& d = a.desc[0];
    const volatile DevCounters* cnt = &a.out[0].counters;
    const PhaseInfo fetch{PH_EXTRACT, 0, 1u, 0u};
    if (cnt->status != 0) return fetch;
    switch (cur.phase) {
    case PH_INGEST: {
        const uint32_t items = a.query[0].use_connected ? connected_items(a, 0) : bitmap_items(a, 0);
        return items ? PhaseInfo{PH_FILTER, 0, items, 0u} : fetch;
    }
    case PH_FILTER:
        return level_phase(p, s, 2);
    case PH_LEVEL:
        if (d.enumeration == MPDP_ENUM_BLOCKS) {
            const int k = cur.level;
            const uint32_t extra = cnt->extra_count[k] < d.heavy_cap ? cnt->extra_count[k] : d.heavy_cap;
            const uint32_t items = cnt->heavy_count[k] + extra;
            constexpr uint32_t kWarps = kEvalThreads / 32;
            if (items) return PhaseInfo{PH_HEAVY, k, (items + kWarps - 1u) / kWarps, 0u};
        }
        return level_phase(p, s, cur.level + 1);
    case PH_HEAVY:
        return level_phase(p, s, cur.level + 1);
    default:
        return PhaseInfo{PH_FREE, 0, 0u, 0u};
    }
}

// Plan fetch of slot s, then its result record for the host and the slot
// freed (whole block; the fetch is the phase's only tile).
__device__ void fetch_and_publish(const PArgs& p, int s, unsigned int epoch)
{
    const BatchArgs& a = p.slot_args[s];
    if (threadIdx.x < 32) extract_body(a, DenseMemo{a.memo, a.left, nullptr, nullptr}, 0u, 1u);
    __syncthreads();
    const DevResult& res = a.out[0].result;
    PResult* r = p.results + s;
    const int n_nodes = res.n_nodes;
    for (int i = threadIdx.x; i < n_nodes && i < kPlanNodes; i += blockDim.x) r->nodes[i] = res.nodes[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        PSlot* sl = p.slots + s;
        const long long ticket = *reinterpret_cast<volatile long long*>(&sl->ticket);
        r->ticket = ticket;
        r->status = res.status;
        r->n_nodes = n_nodes;
        r->cost = res.cost;
        // free the slot before the host can see the result and reuse it
        publish_phase(sl, epoch + 1u, PhaseInfo{PH_FREE, 0, 0u, 0u});
        __threadfence_system();
        *reinterpret_cast<volatile unsigned long long*>(&r->done_ticket) = (unsigned long long)ticket + 1ull;
    }
}

// One tile of phase `inf` of slot s (whole block).  Returns false when the
// tile already advanced the slot (the plan fetch).
__device__ bool run_tile(const PArgs& p, int s, unsigned int epoch, unsigned int tile, PhaseInfo inf)
{
    const BatchArgs& a = p.slot_args[s];
    const uint32_t* pref = p.pref + (size_t)s * kPrefRows;
    switch (inf.phase) {
    case PH_INGEST:
        ingest_body(a, 1, 0u, 1u);
        break;
    case PH_FILTER:
        if (a.query[0].use_connected) filter_connected_body<1>(a, tile, inf.total);
        else filter_bitmaps_body<1>(a, tile, inf.total);
        break;
    case PH_LEVEL:
        if (a.desc[0].enumeration == MPDP_ENUM_TREE)
            eval_tree_body<DenseMemo, 1>(a, inf.level, DenseMemo{a.memo, a.left, nullptr, nullptr}, pref, tile, inf.total);
        else
            eval_blocks_body<DensePlainMemo, 1, false>(a, inf.level, DensePlainMemo{a.memo, a.left, nullptr, nullptr}, pref, tile,
                                                inf.total);
        break;
    case PH_HEAVY:
        eval_heavy_body<DensePlainMemo, 1, false>(a, inf.level, DensePlainMemo{a.memo, a.left, nullptr, nullptr}, tile, inf.total);
        break;
    case PH_EXTRACT:
        fetch_and_publish(p, s, epoch);
        return false;
    default:
        break;
    }
    return true;
}

// Take the next published request, if any (one thread).
__device__ bool take_request(const PArgs& p, unsigned long long& req)
{
    const unsigned long long t = *reinterpret_cast<volatile unsigned long long*>(p.taken);
    const PRequest* e = p.ring + (t % (unsigned long long)p.ring_size);
    const unsigned int seq = *reinterpret_cast<const volatile unsigned int*>(&e->seq);
    if (seq != (unsigned int)(t + 1ull)) return false;
    if (atomicCAS(p.taken, t, t + 1ull) != t) return false;
    __threadfence_system();
    req = t;
    return true;
}

// Copy request `req` into its slot and start the slot's ingest (whole block),
// whose one tile the block claims for itself: thread 0 gets the slot and the
// ingest's epoch.
__device__ void admit(const PArgs& p, unsigned long long req, int& slot, unsigned int& epoch)
{
    const PRequest* e = p.ring + (req % (unsigned long long)p.ring_size);
    const int s = *reinterpret_cast<const volatile int32_t*>(&e->slot);
    const BatchArgs& a = p.slot_args[s];
    const int n = *reinterpret_cast<const volatile int32_t*>(&e->n);
    const int m = *reinterpret_cast<const volatile int32_t*>(&e->m);
    StagedQuery* st = a.staged;
    const volatile double* card = e->card;
    for (int i = threadIdx.x; i < kMaxRels; i += blockDim.x) st->card[i] = i < n ? card[i] : 1.0;
    const volatile int32_t* ew = reinterpret_cast<const volatile int32_t*>(e->edges);
    int32_t* sw = reinterpret_cast<int32_t*>(st->edges);
    const int edge_words = m * (int)(sizeof(mpdp_edge) / sizeof(int32_t));
    for (int i = threadIdx.x; i < edge_words && m <= kMaxEdges; i += blockDim.x) sw[i] = ew[i];
    const volatile int32_t* dw = reinterpret_cast<const volatile int32_t*>(&e->desc);
    int32_t* qd = reinterpret_cast<int32_t*>(const_cast<QDesc*>(a.desc));
    for (int i = threadIdx.x; i < (int)(sizeof(QDesc) / sizeof(int32_t)); i += blockDim.x) qd[i] = dw[i];
    if (threadIdx.x == 0) {
        st->n = n;
        st->n_edges = m;
        st->cost_model = MPDP_COST_COUT;
        st->pad = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        PSlot* sl = p.slots + s;
        *reinterpret_cast<volatile long long*>(&sl->ticket) = *reinterpret_cast<const volatile long long*>(&e->ticket);
        const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(&sl->word);
        __threadfence();
        slot = s;
        epoch = (unsigned int)(w >> 32) + 1u;
        publish_phase(sl, epoch, PhaseInfo{PH_INGEST, 0, 1u, 0u}, 1u);
    }
}

// 4 blocks per SM (64 registers, some spilled; 35 KB of shared memory each):
// against 3 (80 registers) the mixed stream's saturated rate rose from 12,785
// to 14,571 queries/s and its latency at equal offered rates fell (p50 / p99
// at 12,700 queries/s 3.24 / 13.7 -> 1.81 / 10.5 ms), while a lone query's
// phases run slower (snowflake-25 0.40 -> 0.52 ms).
__global__ void __launch_bounds__(kPersistThreads, 4) k_persist(PArgs p)
{
    __shared__ int s_cmd, s_slot;
    __shared__ unsigned int s_epoch, s_tile, s_count;
    __shared__ PhaseInfo s_inf;
    __shared__ unsigned long long s_req;
    // s_chain: the block published a phase (or admitted a query) and holds
    // its first tile in s_slot / s_epoch / s_tile / s_count / s_inf
    __shared__ int s_chain;
    enum { kIdle = 0, kTile = 1, kAdmit = 2, kExit = 3 };
    int idle = 0;
    int start = (int)(blockIdx.x % (unsigned int)p.nslots);
    if (threadIdx.x == 0) s_chain = 0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x < 32) {
            // warp 0 picks the block's next work: the tile the block claimed
            // when it published a phase, else the 32 lanes look at 32 slots
            // at once (from the one this block last worked on), the first
            // slot with tiles left is claimed; else a new request is taken
            const int lane = threadIdx.x;
            int cmd = kIdle;
            int stop = 0, chain = 0;
            if (lane == 0) {
                chain = s_chain;
                s_chain = 0;
                if (!chain) stop = *reinterpret_cast<const volatile int*>(p.stop);
            }
            if (__shfl_sync(kFull, chain, 0)) {
                cmd = kTile;
            } else if (__shfl_sync(kFull, stop, 0)) {
                cmd = kExit;
            } else {
                for (int base = 0; base < p.nslots && cmd == kIdle; base += 32) {
                    const int i = base + lane;
                    const int s = (start + i) % p.nslots;
                    bool has = false;
                    unsigned long long w = 0ull;
                    PhaseInfo seen{PH_FREE, 0, 0u, 0u};
                    if (i < p.nslots) {
                        w = *reinterpret_cast<volatile unsigned long long*>(&p.slots[s].word);
                        seen = read_info(p.slots + s, (unsigned int)(w >> 32));
                        has = seen.phase != PH_FREE && (unsigned int)w < seen.total;
                    }
                    unsigned int cand = __ballot_sync(kFull, has);
                    while (cand && cmd == kIdle) {
                        const int l = __ffs(cand) - 1;
                        cand &= cand - 1u;
                        int got = 0;
                        if (lane == l) {
                            unsigned int e = 0u, t = 0u, c = 0u;
                            PhaseInfo inf;
                            if (claim_tile(p, s, w, seen, e, t, c, inf)) {
                                got = 1;
                                s_slot = s;
                                s_epoch = e;
                                s_tile = t;
                                s_count = c;
                                s_inf = inf;
                            }
                        }
                        if (__shfl_sync(kFull, got, l)) cmd = kTile;
                    }
                }
                if (cmd == kIdle) {
                    int adm = 0;
                    if (lane == 0) {
                        unsigned long long req = 0ull;
                        if (take_request(p, req)) {
                            adm = 1;
                            s_req = req;
                        }
                    }
                    if (__shfl_sync(kFull, adm, 0)) cmd = kAdmit;
                }
            }
            if (lane == 0) s_cmd = cmd;
        }
        __syncthreads();
        const int cmd = s_cmd;
        if (cmd == kExit) break;
        if (cmd == kTile) {
            const int s = s_slot;
            const unsigned int epoch = s_epoch, tile = s_tile, ntiles = s_count;
            const PhaseInfo inf = s_inf;
            start = s;  // stay with this slot while it has tiles
            idle = 0;
            bool count = true;
            for (unsigned int j = 0; j < ntiles && count; j++) {
                count = run_tile(p, s, epoch, tile + j, inf);
                __syncthreads();
            }
            if (count && threadIdx.x == 0) {
                __threadfence();
                PSlot* sl = p.slots + s;
                if (atomicAdd(&sl->done[epoch & 1u], ntiles) + ntiles == inf.total) {
                    __threadfence();
                    // the block that ends a phase claims the next phase's
                    // first tile as it publishes it: a chain of one-tile
                    // phases (small levels, the plan fetch) then runs
                    // back to back in this block, with no other block's
                    // poll, scan and claim between two phases
                    const PhaseInfo nx = next_phase(p, s, inf);
                    const bool own = nx.phase != PH_FREE && nx.total > 0u;
                    publish_phase(sl, epoch + 1u, nx, own ? 1u : 0u);
                    if (own) {
                        s_slot = s;
                        s_epoch = epoch + 1u;
                        s_tile = 0u;
                        s_count = 1u;
                        s_inf = nx;
                        s_chain = 1;
                    }
                }
            }
        } else if (cmd == kAdmit) {
            idle = 0;
            int slot = 0;
            unsigned int ep = 0u;
            admit(p, s_req, slot, ep);
            if (threadIdx.x == 0) {
                s_slot = slot;
                s_epoch = ep;
                s_tile = 0u;
                s_count = 1u;
                s_inf = PhaseInfo{PH_INGEST, 0, 1u, 0u};
                s_chain = 1;
            }
        } else {
            if (++idle > p.idle_polls) break;  // block-uniform
            // an idle block polls less often the longer it stays idle (200 ns
            // doubling to 1.6 us), so that hundreds of idle blocks do not keep
            // the slot words busy for the few that work: a lone snowflake-25
            // 0.52 -> 0.49 ms, loaded rates unchanged
            if (threadIdx.x == 0) __nanosleep(min(200u << min(idle, 3), 1600u));
        }
        __syncthreads();
    }
}

int resolve_enum(const mpdp_config& cfg, int n, int m)
{
    return (cfg.enumeration == MPDP_ENUM_BLOCKS || m != n - 1) ? MPDP_ENUM_BLOCKS : MPDP_ENUM_TREE;
}

size_t slot_bytes(int n)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t heavy = binom_host(n, n / 2);
    return up(sizeof(QDesc)) + up(sizeof(StagedQuery)) + up(sizeof(DevQuery)) + up(sizeof(DevOut)) +
           up((list_entries(n) + conn_words(n)) * 4) + up(heavy * sizeof(HeavyMain)) + up(heavy * sizeof(HeavyExtra)) +
           up(((size_t)1 << n) * sizeof(double2)) + up(((size_t)1 << n) * sizeof(uint32_t));
}

}  // namespace

struct PersistEngine {
    int device = 0, slots = 0, max_rels = 0, grid = 0;
    mpdp_config cfg{};
    cudaStream_t stream = nullptr;
    void* dev = nullptr;
    PSlot* d_slots = nullptr;
    BatchArgs* d_args = nullptr;
    uint32_t* d_pref = nullptr;
    unsigned long long* d_taken = nullptr;
    PRequest* h_ring = nullptr;
    PResult* h_res = nullptr;
    int* h_stop = nullptr;
    PArgs args{};
    unsigned long long submitted = 0;
    std::vector<int64_t> ticket;  // per slot; -1: free
    bool launched = false;
};

int persist_max_rels(uint64_t slot_budget_bytes)
{
    if (slot_budget_bytes == 0) return 25;
    int best = 0;
    for (int n = 2; n <= 25; n++)
        if (slot_bytes(n) <= slot_budget_bytes) best = n;
    return best;
}

int persist_slots(const PersistEngine* e) { return e ? e->slots : 0; }
int persist_max_rels(const PersistEngine* e) { return e ? e->max_rels : 0; }

void persist_destroy(PersistEngine* e)
{
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->h_stop) __atomic_store_n(e->h_stop, 1, __ATOMIC_RELEASE);
    if (e->stream) cudaStreamSynchronize(e->stream);
    cudaFree(e->dev);
    cudaFreeHost(e->h_ring);
    cudaFreeHost(e->h_res);
    cudaFreeHost(e->h_stop);
    if (e->stream) cudaStreamDestroy(e->stream);
    cudaGetLastError();
    delete e;
}

int persist_create(PersistEngine** out, int device, int slots, int max_rels, const mpdp_config& kernel)
{
    if (!out || slots < 1 || slots > 1024 || max_rels < 2 || max_rels > 25) return MPDP_ERR_INVALID_ARG;
    if (kernel.memo_kind != MPDP_MEMO_DENSE || kernel.filter == MPDP_FILTER_UNRANK ||
        kernel.enumeration == MPDP_ENUM_DPSUB)
        return MPDP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    PersistEngine* e = new PersistEngine();
    e->device = device;
    e->slots = slots;
    e->max_rels = max_rels;
    e->cfg = kernel;
    e->ticket.assign(slots, -1);
    auto fail = [&](int rc) {
        cudaGetLastError();
        persist_destroy(e);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(MPDP_ERR_CUDA);
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int n = max_rels;
    const size_t heavy = binom_host(n, n / 2), lists = list_entries(n) + conn_words(n), memo = (size_t)1 << n;
    const size_t common = up(sizeof(PSlot) * slots) + up(sizeof(BatchArgs) * slots) + up(sizeof(unsigned long long)) +
                          up(sizeof(uint32_t) * kPrefRows * (size_t)slots);
    const size_t total = common + slot_bytes(n) * (size_t)slots;
    if (cudaMalloc(&e->dev, total) != cudaSuccess) return fail(MPDP_ERR_OOM);
    char* c = static_cast<char*>(e->dev);
    auto take = [&](size_t b) {
        char* r = c;
        c += up(b);
        return r;
    };
    e->d_slots = reinterpret_cast<PSlot*>(take(sizeof(PSlot) * slots));
    e->d_args = reinterpret_cast<BatchArgs*>(take(sizeof(BatchArgs) * slots));
    e->d_taken = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long)));
    e->d_pref = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * kPrefRows * (size_t)slots));
    std::vector<BatchArgs> h_args(slots);
    for (int s = 0; s < slots; s++) {
        BatchArgs& a = h_args[s];
        memset(&a, 0, sizeof(a));
        a.nq = 1;
        a.max_n = n;
        a.desc = reinterpret_cast<QDesc*>(take(sizeof(QDesc)));
        a.staged = reinterpret_cast<StagedQuery*>(take(sizeof(StagedQuery)));
        a.query = reinterpret_cast<DevQuery*>(take(sizeof(DevQuery)));
        a.out = reinterpret_cast<DevOut*>(take(sizeof(DevOut)));
        a.lists = reinterpret_cast<uint32_t*>(take(lists * 4));
        a.hmain = reinterpret_cast<HeavyMain*>(take(heavy * sizeof(HeavyMain)));
        a.hextra = reinterpret_cast<HeavyExtra*>(take(heavy * sizeof(HeavyExtra)));
        a.memo = reinterpret_cast<double2*>(take(memo * sizeof(double2)));
        a.left = reinterpret_cast<uint32_t*>(take(memo * sizeof(uint32_t)));
        a.run = kernel.run_length;
        a.heavy_threshold = kernel.heavy_threshold;
        a.use_ccc = kernel.use_ccc;
        a.dpsub = 0;
        a.filter_mode = kernel.filter;
    }
    if (cudaMemset(e->dev, 0, common) != cudaSuccess) return fail(MPDP_ERR_CUDA);
    if (cudaMemcpy(e->d_args, h_args.data(), sizeof(BatchArgs) * slots, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(MPDP_ERR_CUDA);
    if (cudaHostAlloc(reinterpret_cast<void**>(&e->h_ring), sizeof(PRequest) * slots, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&e->h_res), sizeof(PResult) * slots, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&e->h_stop), sizeof(int), cudaHostAllocMapped) != cudaSuccess)
        return fail(MPDP_ERR_OOM);
    memset(e->h_ring, 0, sizeof(PRequest) * slots);
    memset(e->h_res, 0, sizeof(PResult) * slots);
    *e->h_stop = 0;
    PArgs& p = e->args;
    p.nslots = slots;
    p.ring_size = slots;
    p.idle_polls = 12000;  // about 20 ms of idle polls (1.6 us apart) before a block leaves
    p.group_threads = kernel.group_threads_log2 ? 1u << kernel.group_threads_log2 : 0u;
    p.slots = e->d_slots;
    p.slot_args = e->d_args;
    p.pref = e->d_pref;
    p.taken = e->d_taken;
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, e->h_ring, 0) != cudaSuccess) return fail(MPDP_ERR_CUDA);
    p.ring = static_cast<PRequest*>(dp);
    if (cudaHostGetDevicePointer(&dp, e->h_res, 0) != cudaSuccess) return fail(MPDP_ERR_CUDA);
    p.results = static_cast<PResult*>(dp);
    if (cudaHostGetDevicePointer(&dp, e->h_stop, 0) != cudaSuccess) return fail(MPDP_ERR_CUDA);
    p.stop = static_cast<const int*>(dp);
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPersistThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return fail(MPDP_ERR_CUDA);
    e->grid = sms * (per_sm < 4 ? per_sm : 4);
    *out = e;
    return MPDP_OK;
}

namespace {

int ensure_running(PersistEngine* e)
{
    if (e->launched) {
        const cudaError_t q = cudaStreamQuery(e->stream);
        if (q == cudaErrorNotReady) return MPDP_OK;
        if (q != cudaSuccess) {
            cudaGetLastError();
            return MPDP_ERR_CUDA;
        }
    }
    k_persist<<<e->grid, kPersistThreads, 0, e->stream>>>(e->args);
    if (cudaGetLastError() != cudaSuccess) return MPDP_ERR_CUDA;
    e->launched = true;
    return MPDP_OK;
}

}  // namespace

int persist_submit(PersistEngine* e, int slot, int64_t ticket, int n, int m, const double* card,
                   const mpdp_edge* edges)
{
    if (!e || slot < 0 || slot >= e->slots || e->ticket[slot] >= 0 || n < 1 || n > e->max_rels || m < 0 ||
        m > kMaxEdges)
        return MPDP_ERR_INVALID_ARG;
    PRequest& r = e->h_ring[e->submitted % (unsigned long long)e->slots];
    QDesc d;
    memset(&d, 0, sizeof(d));
    d.n = n;
    d.n_edges = m;
    d.enumeration = resolve_enum(e->cfg, n, m);
    d.cost_model = MPDP_COST_COUT;
    uint32_t qb = 0;
    fill_levels(d, e->cfg.run_length, e->cfg.filter, qb);
    d.heavy_cap = d.enumeration == MPDP_ENUM_BLOCKS ? (uint32_t)binom_host(n, n / 2) : 0u;
    d.use_conn = d.enumeration == MPDP_ENUM_BLOCKS ? 1u : 0u;
    d.conn_base = list_entries(n);
    r.slot = slot;
    r.ticket = ticket;
    r.desc = d;
    r.n = n;
    r.m = m;
    for (int i = 0; i < kMaxRels; i++) r.card[i] = i < n ? card[i] : 1.0;
    if (m > 0) memcpy(r.edges, edges, sizeof(mpdp_edge) * m);
    __atomic_store_n(&e->h_res[slot].done_ticket, 0ull, __ATOMIC_RELAXED);
    // the sequence number last, with release order: the kernel that sees it
    // sees the whole request
    __atomic_store_n(&r.seq, (unsigned int)(e->submitted + 1ull), __ATOMIC_RELEASE);
    e->submitted++;
    e->ticket[slot] = ticket;
    if (cudaSetDevice(e->device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    return ensure_running(e);
}

int persist_poll(PersistEngine* e, std::vector<PersistResult>& done)
{
    if (!e) return MPDP_ERR_INVALID_ARG;
    int busy = 0;
    for (int s = 0; s < e->slots; s++) {
        const int64_t t = e->ticket[s];
        if (t < 0) continue;
        // acquire: the record's fields, written before its ticket, are visible
        const unsigned long long dt = __atomic_load_n(&e->h_res[s].done_ticket, __ATOMIC_ACQUIRE);
        if (dt != (unsigned long long)t + 1ull) {
            busy++;
            continue;
        }
        const PResult& r = e->h_res[s];
        PersistResult out;
        out.slot = s;
        out.ticket = t;
        out.status = r.status;
        out.cost = r.cost;
        if (r.status == MPDP_OK && r.n_nodes > 0 && r.n_nodes <= kPlanNodes) out.nodes.assign(r.nodes, r.nodes + r.n_nodes);
        done.push_back(std::move(out));
        e->ticket[s] = -1;
    }
    if (busy) {
        if (cudaSetDevice(e->device) != cudaSuccess) {
            cudaGetLastError();
            return MPDP_ERR_CUDA;
        }
        return ensure_running(e);
    }
    return MPDP_OK;
}

int persist_busy(const PersistEngine* e)
{
    int b = 0;
    if (e)
        for (int64_t t : e->ticket) b += t >= 0 ? 1 : 0;
    return b;
}

}  // namespace mpdp
