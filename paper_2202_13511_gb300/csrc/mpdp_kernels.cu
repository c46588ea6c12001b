// MPDP kernels for sm_103a.  Every launch covers a batch of queries.
//
// A batch runs as: ingest (block per query) -> unrank+filter (all levels of
// all queries, one launch) -> [hash layout + clear] -> evaluate level
// 2 .. max n (one launch per level for the whole batch, plus the
// block-per-set launch in block mode) -> plan fetch (block per query).
// Level k's launch only reads memo entries of levels < k, so launches are the
// level barrier of the DP (Sec. 2.1.1; Sec. 5, Algorithm "MPDP on GPU").
//
// Every kernel's work is a device function over an explicit block index and
// block count (`bid`, `nblk`); the __global__ wrappers pass blockIdx and
// gridDim.  A file that defines MPDP_PHASES_ONLY before including this one
// gets those device functions alone (the persistent serving kernel runs them
// tile by tile).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "mpdp_device.cuh"
#include "mpdp_launch.h"

namespace mpdp {

// ---------------------------------------------------------------------------
// Block-wide helpers.

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Exclusive prefix over the batch's queries of f(q) into s_pref[0..nq];
// returns the total.  Every thread of the block must call it.
template <class F>
__device__ uint32_t block_prefix(int nq, uint32_t* s_pref, F f)
{
    __shared__ uint32_t s_warp[32];
    const int per = (nq + blockDim.x - 1) / blockDim.x;
    const int lo = min(nq, (int)threadIdx.x * per), hi = min(nq, lo + per);
    uint32_t sum = 0;
    for (int q = lo; q < hi; q++) sum += f(q);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; w++) wbase += s_warp[w];
    uint32_t run = wbase + incl - sum;
    for (int q = lo; q < hi; q++) {
        s_pref[q] = run;
        run += f(q);
    }
    if (threadIdx.x == blockDim.x - 1) s_pref[nq] = run;
    __syncthreads();
    const uint32_t total = s_pref[nq];
    __syncthreads();
    return total;
}

// Query owning item t: the largest q with s_pref[q] <= t (items of queries
// with no work are skipped since their range is empty).
__device__ __forceinline__ int find_q(const uint32_t* s_pref, int nq, uint32_t t)
{
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pref[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_query(SharedQuery& sq, const DevQuery* MPDP_RESTRICT q)
{
    const int nsel = 2 * q->n_edges;
    for (int i = threadIdx.x; i < nsel; i += blockDim.x) sq.nsel[i] = q->nsel[i];
    if (threadIdx.x < kMaxRels) {
        sq.adj[threadIdx.x] = q->adj[threadIdx.x];
        sq.nbase[threadIdx.x] = q->nbase[threadIdx.x];
        sq.card[threadIdx.x] = q->card[threadIdx.x];
        sq.desc[threadIdx.x] = q->desc[threadIdx.x];
    }
}

// ---------------------------------------------------------------------------
// Device-path staging: gather each query from the caller's device buffers.
#ifndef MPDP_PHASES_ONLY
__global__ void k_stage(BatchArgs a, const double* MPDP_RESTRICT card, const mpdp_edge* MPDP_RESTRICT edges)
{
    const int q = blockIdx.x;
    const QDesc& d = a.desc[q];
    StagedQuery* st = a.staged + q;
    const int n = d.n, m = d.n_edges;
    if (threadIdx.x == 0) {
        st->n = n;
        st->n_edges = m;
        st->cost_model = d.cost_model;
    }
    for (int i = threadIdx.x; i < n && i < kMaxRels; i += blockDim.x) st->card[i] = card[d.card_off + i];
    for (int e = threadIdx.x; e < m && e < kMaxEdges; e += blockDim.x) st->edges[e] = edges[d.edge_off + e];
}
#endif

// Device-path outputs: plan, cost and status of each query to caller buffers.
#ifndef MPDP_PHASES_ONLY
__global__ void k_publish(BatchArgs a, mpdp_plan_node* MPDP_RESTRICT nodes, double* MPDP_RESTRICT cost,
                          int32_t* MPDP_RESTRICT status)
{
    const int q = blockIdx.x;
    const DevResult& r = a.out[q].result;
    const int n_nodes = r.n_nodes;
    for (int i = threadIdx.x; i < n_nodes; i += blockDim.x) nodes[(size_t)q * kPlanNodes + i] = r.nodes[i];
    if (threadIdx.x == 0) {
        cost[q] = r.cost;
        status[q] = a.out[q].counters.status;
    }
}
#endif

// ---------------------------------------------------------------------------
// a0: ingest (block per query).  Validates the staged query, builds the
// adjacency bitmaps, per-relation ascending neighbour selectivity lists and
// the byte neighbourhood tables, checks that the join graph is connected and
// zeroes the counters.  The dense memo's base entries cost({R_i}) = 0 are
// written here (Algorithm "MPDP on GPU", memo fill).
static __device__ void ingest_body(const BatchArgs& a, int dense, uint32_t bid, uint32_t nblk)
{
    const int qi = bid, tid = threadIdx.x;
    const StagedQuery* MPDP_RESTRICT st = a.staged + qi;
    DevQuery* MPDP_RESTRICT q = a.query + qi;
    DevCounters* MPDP_RESTRICT cnt = &a.out[qi].counters;
    int* cw = reinterpret_cast<int*>(cnt);
    for (int i = tid; i < (int)(sizeof(DevCounters) / sizeof(int)); i += blockDim.x) cw[i] = 0;
    __shared__ int s_status;
    __shared__ uint32_t s_adj[kMaxRels], s_children[kMaxRels], s_desc[kMaxRels], s_nsub[kMaxRels], s_nbase[kMaxRels];
    __shared__ uint32_t s_top_pref[kMaxRels + 1], s_lowrun[16], s_leaves, s_flags;
    // the query's edges and cards, staged by all threads at once
    __shared__ mpdp_edge s_edges[kMaxEdges];
    __shared__ double s_card[kMaxRels];
    const int n = st->n, m = st->n_edges;
    const bool shape_ok = n >= 1 && n <= MPDP_MAX_EXACT_RELS && m >= 0 && m <= kMaxEdges;
    if (shape_ok)
        for (int e = tid; e < m; e += blockDim.x) s_edges[e] = st->edges[e];
    if (tid < kMaxRels) {
        s_card[tid] = st->card[tid];
        s_adj[tid] = 0u;
    }
    if (tid == 0) {
        int status = 0;
        if (n < 1 || n > MPDP_MAX_EXACT_RELS) status = MPDP_ERR_TOO_LARGE;
        else if (m < 0 || m > kMaxEdges || st->cost_model != MPDP_COST_COUT) status = MPDP_ERR_INVALID_ARG;
        s_status = status;
    }
    __syncthreads();
    // values and edges, in parallel: a duplicate pair shows as a bit that
    // another edge's atomic OR already set in one of the pair's two words
    if (s_status == 0) {
        if (tid < n) {
            const double c = s_card[tid];
            if (!(c > 0.0) || !(c <= 1.7976931348623157e308)) atomicCAS(&s_status, 0, MPDP_ERR_INVALID_ARG);
        }
        for (int e = tid; e < m; e += blockDim.x) {
            const int u = s_edges[e].u, v = s_edges[e].v;
            const double sel = s_edges[e].sel;
            if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(sel > 0.0) || !(sel <= 1.0)) {
                atomicCAS(&s_status, 0, MPDP_ERR_INVALID_ARG);
                continue;
            }
            const uint32_t o1 = atomicOr(&s_adj[u], 1u << v), o2 = atomicOr(&s_adj[v], 1u << u);
            if ((o1 >> v & 1u) || (o2 >> u & 1u)) atomicCAS(&s_status, 0, MPDP_ERR_INVALID_ARG);
        }
    }
    __syncthreads();
    // the short serial walks: connectivity, spanning tree T rooted at
    // relation 0 (children, discovery order, descendants), the bitmap
    // filter's run tables and the unranking's subtree counts
    uint8_t order[kMaxRels];
    int cnt_order = 0;
    if (tid == 0) {
        int status = s_status;
        uint32_t adj[kMaxRels];
        for (int r = 0; r < kMaxRels; r++) adj[r] = status == 0 ? s_adj[r] : 0u;
        if (status == 0) {
            const uint32_t full = (n == 32) ? kFull : ((1u << n) - 1u);
            if (grow(1u, full, adj) != full) status = MPDP_ERR_DISCONNECTED;
        }
        uint32_t desc[kMaxRels], children[kMaxRels];
        for (int r = 0; r < kMaxRels; r++) {
            children[r] = 0u;
            desc[r] = 1u << r;
        }
        if (status == 0) {
            uint32_t seen = 1u, frontier = 1u;
            order[cnt_order++] = 0;
            while (frontier) {
                const int x = lowest(frontier);
                frontier &= frontier - 1u;
                const uint32_t ch = adj[x] & ~seen;
                children[x] = ch;
                seen |= ch;
                frontier |= ch;
                for (uint32_t c = ch; c; c &= c - 1u) order[cnt_order++] = (uint8_t)lowest(c);
            }
            // every vertex is discovered after its parent
            for (int i = cnt_order - 1; i >= 0; i--) {
                const int v = order[i];
                uint32_t dsc = 1u << v;
                for (uint32_t c = children[v]; c; c &= c - 1u) dsc |= desc[lowest(c)];
                desc[v] = dsc;
            }
        }
        // run tables of the bitmap filter (low relations r < 5 of T)
        uint32_t lowkids = 0u;
        for (int r = 0; r < 5; r++) {
            const bool in = status == 0 && r < n;
            int par = -1;
            for (int p = 0; p < n && in; p++)
                if (children[p] >> r & 1u) par = p;
            s_lowrun[r] = in ? children[r] : 0u;
            s_lowrun[5 + r] = in ? ((par >= 0 && par < 5) ? low_bit(r) & ~low_bit(par) : low_bit(r)) : 0u;
            s_lowrun[10 + r] = (in && par >= 5) ? (uint32_t)par : 0xffffffffu;
            if (in) lowkids |= children[r];
        }
        s_lowrun[15] = lowkids;
        // connected-set unranking tables (tree join graphs): nsub bottom-up
        // over the discovery order; a subtree of t relations has at most
        // 2^(t-1) connected sets with its root on top, so 32 bits suffice
        const bool tree = status == 0 && m == n - 1;
        uint32_t leaves = 0u, nsub[kMaxRels];
        for (int r = 0; r < kMaxRels; r++) {
            nsub[r] = 0u;
            if (tree && r < n && children[r] == 0u) leaves |= 1u << r;
        }
        if (tree)
            for (int i = cnt_order - 1; i >= 0; i--) {
                const int v = order[i];
                uint32_t prod = 1u;
                for (uint32_t c = children[v]; c; c &= c - 1u) prod *= 1u + nsub[lowest(c)];
                nsub[v] = prod;
            }
        uint32_t acc = 0u;
        for (int r = 0; r <= kMaxRels; r++) {
            s_top_pref[r] = acc;
            if (r < kMaxRels) {
                s_nsub[r] = nsub[r];
                s_desc[r] = desc[r];
                s_children[r] = children[r];
            }
            if (tree && r < n) acc += nsub[r];
        }
        s_leaves = leaves;
        // filter CONNECTED: unrank a tree's connected sets when they are at
        // most a quarter of the 2^n bitmaps (forming a set costs a few times
        // testing a bitmap); denser trees such as stars take the sweep
        const bool use_connected =
            a.filter_mode == MPDP_FILTER_CONNECTED && tree && 4ull * (unsigned long long)acc <= (1ull << n);
        s_flags = (tree ? 1u : 0u) | (use_connected ? 2u : 0u);
        s_status = status;
    }
    __syncthreads();
    const int status = s_status;
    const bool tree = (s_flags & 1u) != 0u;
    // the device record, in parallel
    if (tid < kMaxRels) {
        const uint32_t adj = status == 0 ? s_adj[tid] : 0u;
        // neighbour-list bases: exclusive prefix of the degrees over the warp
        const uint32_t deg = __popc(adj);
        uint32_t incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (tid >= o) incl += t;
        }
        s_nbase[tid] = incl - deg;
        q->nbase[tid] = incl - deg;
        q->adj[tid] = adj;
        q->card[tid] = (status == 0 && tid < n) ? s_card[tid] : 1.0;
        q->desc[tid] = s_desc[tid];
        q->chmask[tid] = tree ? s_children[tid] : 0u;
        q->nsub[tid] = s_nsub[tid];
        q->top_pref[tid] = s_top_pref[tid];
        if (tid < 16) q->lowrun[tid] = s_lowrun[tid];
        if (tid == 0) {
            q->top_pref[kMaxRels] = s_top_pref[kMaxRels];
            q->leaves = s_leaves;
            q->use_connected = (s_flags & 2u) ? 1u : 0u;
            q->n = n;
            q->n_edges = status == 0 ? m : 0;
            q->is_tree = tree ? 1 : 0;
            cnt->status = status;
        }
        // the divisors 1 + nsub[r] of the unranking's mixed-radix digits
        const unsigned long long d = 1ull + s_nsub[tid];
        int l = 0;
        while ((1ull << l) < d) l++;
        q->dmag[tid] = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1ull);
        q->dsh[tid] = (uint8_t)((l > 0 ? 1 : 0) | ((l > 0 ? l - 1 : 0) << 1));
    }
    __syncthreads();
    if (status == 0)
        for (int e = tid; e < m; e += blockDim.x) {  // neighbour selectivities, ascending by neighbour
            const int u = s_edges[e].u, v = s_edges[e].v;
            const double sel = s_edges[e].sel;
            q->nsel[s_nbase[u] + __popc(s_adj[u] & ((1u << v) - 1u))] = sel;
            q->nsel[s_nbase[v] + __popc(s_adj[v] & ((1u << u) - 1u))] = sel;
        }
    if (status == 0 && dense) {
        DenseMemo memo{a.memo, a.left, nullptr, nullptr};
        memo.bind(a, qi);
        if (tid < n) memo.put(1u << tid, 1, 0.0, s_card[tid], 0u, cnt);
    }
    {
        // block CCP lists of this batch: counters and table empty
        const QDesc& d = a.desc[qi];
        if (d.use_bl)
            for (uint32_t i = tid; i < kBlHead; i += blockDim.x) a.lists[d.bl_base + i] = 0u;
    }
    for (int e = tid; e < 4 * 256; e += blockDim.x) {
        const int b = e >> 8, x = e & 255;
        uint32_t u = 0u, c = 0u;
        for (int i = 0; i < 8; i++)
            if (x >> i & 1) {
                u |= status == 0 ? s_adj[8 * b + i] : 0u;
                c |= s_children[8 * b + i];
            }
        q->nbt[b][x] = u;
        q->ctt[b][x] = c;
    }
}

#ifndef MPDP_PHASES_ONLY
__global__ void __launch_bounds__(256) k_ingest(BatchArgs a, int dense)
{
    ingest_body(a, dense, blockIdx.x, gridDim.x);
}
#endif

// ---------------------------------------------------------------------------
// Binomial coefficients C(i, j), i, j <= 32, built at compile time by
// Pascal's rule (C(32, 16) < 2^32, so every entry fits 32 bits).
struct BinomTable {
    uint32_t v[33 * 33];
};

constexpr BinomTable make_binom_table()
{
    BinomTable t{};
    for (int i = 0; i <= 32; i++)
        for (int j = 0; j <= 32; j++)
            t.v[i * 33 + j] = (j == 0) ? 1u : (i == 0 ? 0u : t.v[(i - 1) * 33 + j - 1] + t.v[(i - 1) * 33 + j]);
    return t;
}

static __device__ const BinomTable kBinom = make_binom_table();

// Combinatorial number system (colex order): the k-subset of {0..n-1} with
// rank r is {c_k > ... > c_1} where r = sum_i C(c_i, i); each c_i is the
// largest value with C(c_i, i) <= what remains of r.
__device__ __forceinline__ uint32_t unrank_colex(uint32_t r, int k, int n,
                                                 const uint32_t* MPDP_RESTRICT binom)
{
    uint32_t s = 0u;
    int c = n - 1;
    for (int i = k; i >= 1; i--) {
        while (binom[c * 33 + i] > r) c--;
        s |= 1u << c;
        r -= binom[c * 33 + i];
        c--;
    }
    return s;
}

// Next k-subset in colex order = next larger integer with the same number of
// set bits (the bit-permutation step the paper's unrank enhancement uses).
__device__ __forceinline__ uint32_t next_colex(uint32_t s)
{
    const uint32_t t = s | (s - 1u);
    return (t + 1u) | (((~t & (0u - ~t)) - 1u) >> __ffs(s));
}

// ---------------------------------------------------------------------------
// a2 + a3: unrank every k-subset of every level of every query and keep the
// connected ones.  Each block belongs to one query; each warp to one level;
// lane l of a warp takes the run of `run` consecutive ranks starting at
// warp_base + l * run, unranks its first set and steps with next_colex.
// Pass 1 tests connectivity (isolated-vertex rejection, then BFS rounds by
// byte tables) and keeps one flag bit per rank; a warp scan places every
// lane's connected sets, one atomic per warp reserves room in the level's
// list, and pass 2 replays the run writing the kept sets: each warp's output
// is a colex-ordered slice.
#ifndef MPDP_PHASES_ONLY
__global__ void __launch_bounds__(kFilterThreads) k_filter(BatchArgs a)
{
    __shared__ uint32_t s_binom[33 * 33];
    __shared__ uint32_t s_nbt[4][256];
    __shared__ uint32_t s_ctt[4][256];
    // query of this block: the largest q with prefix[q] <= blockIdx.x
    int lo = 0, hi = a.nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.filter_block_prefix[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const int qi = lo;
    const QDesc& d = a.desc[qi];
    const DevQuery* MPDP_RESTRICT q = a.query + qi;
    DevCounters* MPDP_RESTRICT cnt = &a.out[qi].counters;
    for (int t = threadIdx.x; t < 33 * 33; t += blockDim.x) s_binom[t] = kBinom.v[t];
    for (int t = threadIdx.x; t < 4 * 256; t += blockDim.x) {
        s_nbt[t >> 8][t & 255] = q->nbt[t >> 8][t & 255];
        s_ctt[t >> 8][t & 255] = q->ctt[t >> 8][t & 255];
    }
    __syncthreads();
    if (cnt->status != 0) return;
    const bool is_tree = q->is_tree != 0;
    const uint32_t warp = (blockIdx.x - a.filter_block_prefix[qi]) * (kFilterThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int n = d.n;
    int k = -1;
    for (int j = 2; j <= n; j++)
        if (warp >= d.warp_begin[j] && warp < d.warp_begin[j + 1]) k = j;
    if (k < 0) return;  // whole warp: padding past the query's last level
    const uint32_t nr = s_binom[n * 33 + k];
    const unsigned long long r0 = (unsigned long long)(warp - d.warp_begin[k]) * 32ull * (unsigned long long)a.run +
                                  (unsigned long long)lane * (unsigned long long)a.run;
    uint32_t len = 0;
    if (r0 < nr) len = (uint32_t)min((unsigned long long)a.run, (unsigned long long)nr - r0);
    const uint32_t s0 = len ? unrank_colex((uint32_t)r0, k, n, s_binom) : 0u;
    uint32_t s = s0, flags = 0u, rounds = 0u;
    // In colex order the high half of S rarely changes along a run: its part
    // of the table lookups is cached and redone only when bits 16..31 change.
    uint32_t s_hi = 0xffffffffu, ch_hi = 0u, nb_hi = 0u;
    if (is_tree) {
        // tree join graph: connected(S) iff exactly one member of S has its
        // parent outside S (one top per component), with no search at all
        for (uint32_t i = 0; i < len; i++) {
            if ((s >> 16) != s_hi) {
                s_hi = s >> 16;
                ch_hi = s_ctt[2][s_hi & 255u] | s_ctt[3][s_hi >> 8];
            }
            const uint32_t ch = ch_hi | s_ctt[0][s & 255u] | s_ctt[1][(s >> 8) & 255u];
            if (__popc(tops_of(s, ch)) == 1) flags |= 1u << i;
            s = next_colex(s);
        }
    } else {
        // general join graph: accept when the spanning tree alone connects
        // S; reject when some member has no neighbour in S; else BFS rounds
        for (uint32_t i = 0; i < len; i++) {
            if ((s >> 16) != s_hi) {
                s_hi = s >> 16;
                ch_hi = s_ctt[2][s_hi & 255u] | s_ctt[3][s_hi >> 8];
                nb_hi = s_nbt[2][s_hi & 255u] | s_nbt[3][s_hi >> 8];
            }
            const uint32_t ch = ch_hi | s_ctt[0][s & 255u] | s_ctt[1][(s >> 8) & 255u];
            bool ok = __popc(tops_of(s, ch)) == 1;
            if (!ok) {
                const uint32_t nb = nb_hi | s_nbt[0][s & 255u] | s_nbt[1][(s >> 8) & 255u];
                ok = (s & ~nb) == 0u && connected_rounds_from(s, s_nbt, rounds);
            }
            if (ok) flags |= 1u << i;
            s = next_colex(s);
        }
    }
    const uint32_t c = __popc(flags);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(&cnt->list_count[k], total);
    base = __shfl_sync(kFull, base, 0);
    uint32_t* out = a.lists + d.list_base + d.list_off[k] + base + (incl - c);
    s = s0;
    uint32_t w = 0;
    const uint32_t last = flags ? 32u - __clz(flags) : 0u;  // replay only up to the last kept rank
    for (uint32_t i = 0; i < last; i++) {
        if (flags >> i & 1u) out[w++] = s;
        s = next_colex(s);
    }
    uint32_t done = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        done += __shfl_xor_sync(kFull, done, o);
        rounds += __shfl_xor_sync(kFull, rounds, o);
    }
    if (lane == 0 && done) {
        atomicAdd(&cnt->unranked, (unsigned long long)done);
        atomicAdd(&cnt->filter_steps, (unsigned long long)rounds);
    }
}
#endif

// ---------------------------------------------------------------------------
// a2 + a3 for tree join graphs (filter mode CONNECTED): the connected sets
// themselves are unranked, so no disconnected set is ever formed.  A query's
// ranks r < top_pref[n] cover its connected sets: the top is the v with
// top_pref[v] <= r < top_pref[v + 1], and x = r - top_pref[v] < nsub[v]
// decodes over v's children: the leaf children first, one bit of x each (in
// or out, ascending), then every other child c in ascending order with digit
// d = x mod (1 + nsub[c]), x /= 1 + nsub[c]; d = 0 leaves c's subtree out,
// d > 0 takes c's connected set of rank d - 1, decoded the same way.
__device__ __forceinline__ uint32_t unrank_connected(const DevQuery* MPDP_RESTRICT q, int v, uint32_t x)
{
    uint8_t st_v[kMaxRels];
    uint32_t st_x[kMaxRels];
    int sp = 1;
    st_v[0] = (uint8_t)v;
    st_x[0] = x;
    const uint32_t leaves = MPDP_LDG(&q->leaves);
    uint32_t s = 0u;
    while (sp > 0) {
        --sp;
        const int u = st_v[sp];
        uint32_t r = st_x[sp];
        s |= 1u << u;
        const uint32_t ch = MPDP_LDG(&q->chmask[u]);
        for (uint32_t c = ch & leaves; c; c &= c - 1u) {
            if (r & 1u) s |= c & (0u - c);
            r >>= 1;
        }
        for (uint32_t c = ch & ~leaves; c; c &= c - 1u) {
            const int w = lowest(c);
            const uint32_t radix = MPDP_LDG(&q->nsub[w]) + 1u;
            const uint32_t t = __umulhi(r, MPDP_LDG(&q->dmag[w]));
            const uint32_t sh = MPDP_LDG(&q->dsh[w]);
            const uint32_t quo = (t + ((r - t) >> (sh & 1u))) >> (sh >> 1);
            const uint32_t dgt = r - quo * radix;
            r = quo;
            if (dgt) {
                st_v[sp] = (uint8_t)w;
                st_x[sp] = dgt - 1u;
                sp++;
            }
        }
    }
    return s;
}

// The connected set that follows s among the sets with top v, in the order
// unrank_connected decodes them (false when s is the last one).  An
// odometer over the same digits: v's leaf children (one bit each, lowest
// first), then its other children, whose digit is their own odometer (0:
// the child's subtree left out; a child that overflows drops its subtree and
// carries to the next digit).  Consecutive ranks differ in their low digits,
// so a step touches a few digits on average.
__device__ __forceinline__ bool next_connected(const DevQuery* MPDP_RESTRICT q, int v, uint32_t& s)
{
    uint8_t st_u[kMaxRels];
    uint32_t st_l[kMaxRels], st_n[kMaxRels];
    const uint32_t leaves = MPDP_LDG(&q->leaves);
    const uint32_t ch = MPDP_LDG(&q->chmask[v]);
    st_u[0] = (uint8_t)v;
    st_l[0] = ch & leaves;
    st_n[0] = ch & ~leaves;
    int sp = 1;
    uint32_t x = s;
    while (sp > 0) {
        const int f = sp - 1;
        if (st_l[f]) {  // a leaf child's bit
            const uint32_t c = st_l[f] & (0u - st_l[f]);
            st_l[f] ^= c;
            if (!(x & c)) {
                s = x | c;
                return true;
            }
            x &= ~c;
            continue;
        }
        if (st_n[f]) {  // another child: in with its first set, or its own odometer
            const uint32_t c = st_n[f] & (0u - st_n[f]);
            st_n[f] ^= c;
            if (!(x & c)) {
                s = x | c;
                return true;
            }
            const int w = lowest(c);
            const uint32_t cw = MPDP_LDG(&q->chmask[w]);
            st_u[sp] = (uint8_t)w;
            st_l[sp] = cw & leaves;
            st_n[sp] = cw & ~leaves;
            sp++;
            continue;
        }
        // every digit of this node wrapped
        if (--sp == 0) return false;
        x &= ~MPDP_LDG(&q->desc[st_u[f]]);
    }
    return false;
}

// Ranks per thread and per block item of the connected-set filter: a thread
// decodes the first rank of its run and steps to the others.
constexpr int kConnPerThread = 8;
constexpr uint32_t kConnPerItem = kFilterThreads * kConnPerThread;

// Items of kConnPerItem consecutive ranks of a tree query in mode CONNECTED
// (0 for the other queries and after an error).
__device__ __forceinline__ uint32_t connected_items(const BatchArgs& a, int q)
{
    const DevQuery& dq = a.query[q];
    if (a.out[q].counters.status != 0 || !dq.use_connected) return 0u;
    return (dq.top_pref[dq.n] + kConnPerItem - 1u) / kConnPerItem;
}

// A block takes an item of kConnPerItem consecutive ranks of one query
// (grid-stride over the batch's items); thread t takes the run of
// kConnPerThread ranks from item * kConnPerItem + t * kConnPerThread on:
// the first decoded, the next ones by next_connected (the top moves to the
// next relation when its sets run out).  Places within the block come from
// shared-memory counters per level, and one global atomic per level present
// reserves the block's room in that level's list.
template <int kQ = kMaxBatch>  // kQ: the most queries of a batch it serves
static __device__ void filter_connected_body(const BatchArgs& a, uint32_t bid, uint32_t nblk)
{
    __shared__ uint32_t s_pref[kQ + 1];
    __shared__ uint32_t s_cnt[kLevels];
    __shared__ uint32_t s_base[kLevels];
    const uint32_t items = block_prefix(a.nq, s_pref, [&](int q) { return connected_items(a, q); });
    const int tid = threadIdx.x;
    int cur = -1;
    unsigned long long formed = 0;  // threads tid < kLevels: sets of level tid formed for query cur
    for (uint32_t it = bid; it < items; it += nblk) {
        const int qi = find_q(s_pref, a.nq, it);  // block-uniform
        if (qi != cur) {
            if (cur >= 0 && tid < kLevels && formed) atomicAdd(&a.out[cur].counters.unranked, formed);
            formed = 0;
            cur = qi;
        }
        if (tid < kLevels) s_cnt[tid] = 0u;
        __syncthreads();
        const DevQuery* MPDP_RESTRICT q = a.query + qi;
        const int n = q->n;
        const uint32_t total = MPDP_LDG(&q->top_pref[n]);
        const uint32_t r0 = (it - s_pref[qi]) * kConnPerItem + (uint32_t)tid * kConnPerThread;
        uint32_t sv[kConnPerThread], off[kConnPerThread];
        int top = 0;
        uint32_t cur_s = 0u;
        if (r0 < total) {
            int lo = 0, hi = n - 1;  // largest v with top_pref[v] <= r0
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (MPDP_LDG(&q->top_pref[mid]) <= r0) lo = mid;
                else hi = mid - 1;
            }
            top = lo;
            cur_s = unrank_connected(q, lo, r0 - MPDP_LDG(&q->top_pref[lo]));
        }
#pragma unroll 1
        for (int j = 0; j < kConnPerThread; j++) {
            const uint32_t r = r0 + (uint32_t)j;
            uint32_t s = 0u;
            if (r < total) {
                if (j > 0 && !next_connected(q, top, cur_s)) {
                    top++;  // the next relation's first set: itself
                    cur_s = 1u << top;
                }
                s = cur_s;
            }
            sv[j] = s;
            const int lv = __popc(s);
            off[j] = lv >= 2 ? atomicAdd(&s_cnt[lv], 1u) : 0u;  // the empty set and single relations are not DP sets
        }
        __syncthreads();
        if (tid < kLevels) {
            const uint32_t c = s_cnt[tid];
            s_base[tid] = c ? atomicAdd(&a.out[qi].counters.list_count[tid], c) : 0u;
            formed += c;
        }
        __syncthreads();
        const QDesc& d = a.desc[qi];
#pragma unroll
        for (int j = 0; j < kConnPerThread; j++) {
            const int lv = __popc(sv[j]);
            if (lv >= 2) a.lists[d.list_base + d.list_off[lv] + s_base[lv] + off[j]] = sv[j];
        }
    }
    if (cur >= 0 && tid < kLevels && formed) atomicAdd(&a.out[cur].counters.unranked, formed);
}

#ifndef MPDP_PHASES_ONLY
__global__ void __launch_bounds__(kFilterThreads) k_filter_connected(BatchArgs a)
{
    filter_connected_body(a, blockIdx.x, gridDim.x);
}
#endif

// ---------------------------------------------------------------------------
// a2 + a3, bitmap form: every bitmap S < 2^n of every query is tested, in
// index order, all levels at once (no unranking).  A thread takes aligned
// runs of 32 bitmaps base | i, i < 32: bits 5..31 are fixed along a run, so
// their share of the work is done once per run.  Connected sets (|S| >= 2)
// go straight into the list of their level, in bitmap order within each
// warp's slice.  A block covers kFilterRounds consecutive slices of
// kFilterThreads runs, so its table loads are shared by 8 x 8192 bitmaps.
constexpr uint32_t kBitmapsPerThread = 32;
constexpr uint32_t kFilterRounds = 8;
constexpr uint32_t kBitmapsPerBlock = kFilterThreads * kBitmapsPerThread * kFilterRounds;

// kPopcMask.v[j]: the i in [0, 32) with popcount(i) == j, as a 32-bit mask.
struct PopcMasks {
    uint32_t v[6];
};

constexpr PopcMasks make_popc_masks()
{
    PopcMasks m{};
    for (int i = 0; i < 32; i++) {
        int c = 0;
        for (int b = 0; b < 5; b++) c += (i >> b) & 1;
        m.v[c] |= 1u << i;
    }
    return m;
}

static __device__ const PopcMasks kPopcMask = make_popc_masks();

// Items of kBitmapsPerBlock bitmaps of a query the bitmap sweep serves: all
// queries but the trees whose connected sets are unranked directly.
__device__ __forceinline__ uint32_t bitmap_items(const BatchArgs& a, int q)
{
    const DevQuery& dq = a.query[q];
    if (a.out[q].counters.status != 0 || dq.use_connected || dq.n < 2) return 0u;
    return (uint32_t)(((1ull << dq.n) + kBitmapsPerBlock - 1) / kBitmapsPerBlock);
}

__device__ __forceinline__ void flush_filter_counts(DevCounters* cnt, uint32_t& examined, uint32_t& rounds)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        examined += __shfl_xor_sync(kFull, examined, o);
        rounds += __shfl_xor_sync(kFull, rounds, o);
    }
    if ((threadIdx.x & 31) == 0 && examined) {
        atomicAdd(&cnt->unranked, (unsigned long long)examined);
        if (rounds) atomicAdd(&cnt->filter_steps, (unsigned long long)rounds);
    }
    examined = 0u;
    rounds = 0u;
}

template <int kQ = kMaxBatch>  // kQ: the most queries of a batch it serves
static __device__ void filter_bitmaps_body(const BatchArgs& a, uint32_t bid, uint32_t nblk)
{
    __shared__ uint32_t s_nbt[4][256];
    __shared__ uint32_t s_ctt[4][256];
    __shared__ uint32_t s_stage[kFilterThreads / 32][32];
    __shared__ uint32_t s_run[16];     // DevQuery::lowrun
    __shared__ uint32_t s_pref[kQ + 1];
    // items of kBitmapsPerBlock bitmaps of every query this filter serves,
    // grid-stride; a block reloads the tables when its query changes
    const uint32_t items = block_prefix(a.nq, s_pref, [&](int q) { return bitmap_items(a, q); });
    const int lane = threadIdx.x & 31;
    int cur = -1;
    const QDesc* d = nullptr;
    DevCounters* cnt = nullptr;
    bool is_tree = false;
    unsigned long long limit = 0;
    uint32_t rounds = 0u, examined = 0u;
    for (uint32_t it = bid; it < items; it += nblk) {
        const int qi = find_q(s_pref, a.nq, it);  // block-uniform
        if (qi != cur) {
            if (cur >= 0) flush_filter_counts(cnt, examined, rounds);
            __syncthreads();  // every warp is done with the previous tables
            const DevQuery* MPDP_RESTRICT q = a.query + qi;
            d = a.desc + qi;
            cnt = &a.out[qi].counters;
            is_tree = q->is_tree != 0;
            for (int t = threadIdx.x; t < 4 * 256; t += blockDim.x) {
                if (!is_tree) s_nbt[t >> 8][t & 255] = q->nbt[t >> 8][t & 255];
                s_ctt[t >> 8][t & 255] = q->ctt[t >> 8][t & 255];
            }
            if (threadIdx.x < 16) s_run[threadIdx.x] = q->lowrun[threadIdx.x];
            __syncthreads();
            limit = 1ull << d->n;
            cur = qi;
        }
        const uint32_t blk = it - s_pref[qi];
        for (uint32_t rd = 0; rd < kFilterRounds; rd++) {
            const unsigned long long base64 =
                (((unsigned long long)blk * kFilterRounds + rd) * kFilterThreads +
                 threadIdx.x) *
                kBitmapsPerThread;
            if (base64 - (unsigned long long)lane * kBitmapsPerThread >= limit) break;  // warp-uniform
            uint32_t flags = 0u;
            const uint32_t base = (uint32_t)base64;
            if (base64 < limit) {
                const uint32_t c_run = s_ctt[0][base & 0xe0u] | s_ctt[1][(base >> 8) & 255u] |
                                       s_ctt[2][(base >> 16) & 255u] | s_ctt[3][base >> 24];
                if (is_tree) {
                    // Tree join graph: S is connected iff exactly one member's
                    // parent lies outside S.  Evaluated for the whole run at
                    // once, bit-sliced over i: `one` / `two` collect the runs'
                    // bitmaps with at least one / at least two such members.
                    // High members (bits >= 5) with a high parent outside the
                    // run's high part are a top in every bitmap of the run.
                    const uint32_t fixed = base & ~c_run & ~s_run[15];
                    if ((fixed & (fixed - 1u)) == 0u) {
                        uint32_t one = fixed ? kFull : 0u, two = 0u;
                        const uint32_t g = base & s_run[15];  // high members with a low parent
#pragma unroll
                        for (int p = 0; p < 5; p++) {
                            const uint32_t gp = g & s_run[p];
                            if (gp) {
                                const uint32_t t = ~low_bit(p);  // a top unless p is in S
                                two |= (one & t) | ((gp & (gp - 1u)) ? t : 0u);
                                one |= t;
                            }
                        }
#pragma unroll
                        for (int r = 0; r < 5; r++) {
                            const uint32_t hp = s_run[10 + r];
                            const uint32_t t = (hp < 32u && (base >> hp & 1u)) ? 0u : s_run[5 + r];
                            two |= one & t;
                            one |= t;
                        }
                        flags = one & ~two;
                    }
                } else {
                    const uint32_t n_run = s_nbt[0][base & 0xe0u] | s_nbt[1][(base >> 8) & 255u] |
                                           s_nbt[2][(base >> 16) & 255u] | s_nbt[3][base >> 24];
                    for (uint32_t i = 0; i < kBitmapsPerThread; i++) {
                        const uint32_t s = base | i;
                        bool ok = __popc(s & ~(c_run | s_ctt[0][i])) == 1;
                        if (!ok) ok = (s & ~(n_run | s_nbt[0][i])) == 0u && connected_rounds_from(s, s_nbt, rounds);
                        if (ok) flags |= 1u << i;
                    }
                }
                if (d->use_conn) {
                    // the query's connectivity bitmap: this run's word, single
                    // relations included, the empty set excluded
                    uint32_t w = flags;
                    if (base == 0u) w &= ~1u;
                    if (limit - base64 < kBitmapsPerThread) w &= (1u << (uint32_t)(limit - base64)) - 1u;
                    a.lists[d->conn_base + (base >> 5)] = w;
                }
                uint32_t valid = 0xffffffffu;
                if (limit - base64 < kBitmapsPerThread) valid = (1u << (uint32_t)(limit - base64)) - 1u;
                if (__popc(base) <= 1)  // the empty set and single relations are not DP sets
                    for (uint32_t i = 0; i < kBitmapsPerThread; i++)
                        if (__popc(base | i) < 2) valid &= ~(1u << i);
                flags &= valid;
                examined += __popc(valid);
            }
            // Ordered output straight into the level lists.  The warp covers the
            // 1024 bitmaps w0 .. w0+1023 (w0 = its first bitmap), so bitmap
            // base | i of lane l has level popc(w0) + popc(l) + popc(i): 11 level
            // bins per warp.  Sets leave in bitmap order within each level.
            if (!__any_sync(kFull, flags != 0u)) continue;
            uint32_t fincl = (uint32_t)__popc(flags);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(kFull, fincl, o);
                if (lane >= o) fincl += u;
            }
            const uint32_t ftotal = __shfl_sync(kFull, fincl, 31);
            const int pw = __popc((uint32_t)(base64 - (unsigned long long)lane * kBitmapsPerThread));
            if (ftotal != 0u && ftotal <= 32u) {
                // Sparse warp: compact its sets into one set per lane (bitmap
                // order), then one ballot per level present places them.
                uint32_t o = fincl - (uint32_t)__popc(flags), f = flags;
                while (f) {
                    const int i = lowest(f);
                    f &= f - 1u;
                    s_stage[threadIdx.x >> 5][o++] = base | (uint32_t)i;
                }
                __syncwarp();
                const bool has = (uint32_t)lane < ftotal;
                const uint32_t sv = has ? s_stage[threadIdx.x >> 5][lane] : 0u;
                const int lv = __popc(sv);
                const int lb = has ? lv - pw : 0;  // level bin, 0..10
                uint32_t present = __reduce_or_sync(kFull, has ? 1u << lb : 0u);
                unsigned bin_mask = 0u;  // lane t <= 10: the lanes holding a set of bin t
                while (present) {
                    const int t = lowest(present);
                    present &= present - 1u;
                    const unsigned m = __ballot_sync(kFull, has && lb == t);
                    if (lane == t) bin_mask = m;
                }
                // every bin reserves its list room at once: one atomic latency
                uint32_t bpos = 0u;
                if (bin_mask) bpos = atomicAdd(&cnt->list_count[pw + lane], (uint32_t)__popc(bin_mask));
                const uint32_t b0 = __shfl_sync(kFull, bpos, lb);
                const unsigned mm = __shfl_sync(kFull, bin_mask, lb);
                if (has) a.lists[d->list_base + d->list_off[pw + lb] + b0 + __popc(mm & ((1u << lane) - 1u))] = sv;
                __syncwarp();
            } else if (ftotal != 0u) {
                // Dense warp: a shuffle scan per level bin places every lane's sets
                // and one atomic per non-empty bin reserves list room.
                const int pl = __popc((uint32_t)lane);
                uint32_t cj[6], ex[6];
#pragma unroll
                for (int j = 0; j < 6; j++) cj[j] = __popc(flags & kPopcMask.v[j]);
                uint32_t my_total = 0u;
#pragma unroll
                for (int t = 0; t <= 10; t++) {
                    uint32_t v = 0u;
#pragma unroll
                    for (int j = 0; j < 6; j++) v = (t - pl == j) ? cj[j] : v;
                    uint32_t incl = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t u = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o) incl += u;
                    }
                    const uint32_t tot = __shfl_sync(kFull, incl, 31);
                    if (lane == t) my_total = tot;
#pragma unroll
                    for (int j = 0; j < 6; j++)
                        if (t - pl == j) ex[j] = incl - v;
                }
                uint32_t bpos = 0u;
                if (lane <= 10 && my_total) bpos = atomicAdd(&cnt->list_count[pw + lane], my_total);
                uint32_t* lists = a.lists + d->list_base;
                uint32_t start[6];
#pragma unroll
                for (int j = 0; j < 6; j++) start[j] = __shfl_sync(kFull, bpos, pl + j) + ex[j];
                uint32_t f = flags;
                while (f) {
                    const int i = lowest(f);
                    f &= f - 1u;
                    const int j = __popc((uint32_t)i);
                    uint32_t pos = 0u;
#pragma unroll
                    for (int jj = 0; jj < 6; jj++)
                        if (j == jj) pos = start[jj]++;
                    lists[d->list_off[pw + pl + j] + pos] = base | (uint32_t)i;
                }
            }
        }
    }
    if (cur >= 0) flush_filter_counts(cnt, examined, rounds);
}

#ifndef MPDP_PHASES_ONLY
__global__ void __launch_bounds__(kFilterThreads, 6) k_filter_bitmaps(BatchArgs a)
{
    filter_bitmaps_body(a, blockIdx.x, gridDim.x);
}
#endif

// ---------------------------------------------------------------------------
// Hash memo layout: per query and level k, capacity = the power of two >= 2x
// the level's connected count (at least 16), carved from one arena.
#ifndef MPDP_PHASES_ONLY
__global__ void k_hash_layout(BatchArgs a)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long base = a.arena_begin;
    for (int qi = 0; qi < a.nq; qi++) {
        DevCounters* cnt = &a.out[qi].counters;
        HashLayout* lay = a.layout + qi;
        for (int k = 0; k < kLevels; k++) {
            lay->base[k] = 0;
            lay->mask[k] = 0;
        }
        const unsigned long long start = base;
        const int n = a.desc[qi].n;
        if (cnt->status == 0)
            for (int k = 2; k <= n; k++) {
                const unsigned long long want = 2ull * cnt->list_count[k];
                unsigned long long cap = 16;
                while (cap < want) cap <<= 1;
                lay->base[k] = base;
                lay->mask[k] = (unsigned int)(cap - 1);
                base += cap;
            }
        lay->total_slots = base;  // end of this query's tables
        cnt->memo_slots = base - start;
        if (base > a.arena_slots) raise_status(cnt, MPDP_ERR_OOM);
    }
}
#endif

#ifndef MPDP_PHASES_ONLY
__global__ void __launch_bounds__(256) k_hash_clear(BatchArgs a)
{
    const unsigned long long total = a.layout[a.nq - 1].total_slots;
    const unsigned long long lim = total < a.arena_slots ? total : a.arena_slots;
    const double4_32a z = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    for (unsigned long long i = a.arena_begin + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < lim;
         i += (unsigned long long)gridDim.x * blockDim.x)
        reinterpret_cast<double4_32a*>(a.arena)[i] = z;
}
#endif

// ---------------------------------------------------------------------------
// Tiles of kEvalThreads sets of one query at level k for queries in mode `mode`.
__device__ __forceinline__ uint32_t level_tiles(const BatchArgs& a, int q, int k, int mode)
{
    const QDesc& d = a.desc[q];
    if (d.n < k || d.enumeration != mode) return 0u;
    const DevCounters& c = a.out[q].counters;
    if (c.status != 0) return 0u;
    return (c.list_count[k] + kEvalThreads - 1) / kEvalThreads;
}

// ---------------------------------------------------------------------------
// Tile prefix of every level over the lane's tree queries and, in a second
// table, over its block-mode queries, once after the filter (a block per
// level and mode): each evaluate launch then loads its row instead of
// recomputing it from the queries' counters.  A tree level evaluated by
// groups of lanes (see group_size) gets a set prefix instead.
// Top of a connected set in a tree query: the member whose descendants cover it.
__device__ __forceinline__ int set_top_of(const DevQuery* MPDP_RESTRICT q, uint32_t s)
{
    uint32_t t = s;
    int top = lowest(t);
    while ((MPDP_LDG(&q->desc[top]) & s) != s) {
        t &= t - 1u;
        top = lowest(t);
    }
    return top;
}

constexpr int kPrefStride = kMaxBatch + 2;  // prefix [0, nq], then the level's mapping flag
// A tree level may be evaluated by groups of G lanes per set, G the power
// of two at or above the set's k - 1 splits (2..32): each lane takes one
// split, so a set's cost pairs cost one round of memory latency instead of a
// thread's ceil((k - 1) / 2).  A level goes to groups when its sets x G stay
// within `limit` threads (the context's per-level split knob; 0: never),
// else it runs a thread per set.
__device__ __forceinline__ uint32_t group_size(uint32_t sets, int k, uint32_t limit)
{
    if (k < 4) return 1u;  // one or two splits: a thread takes them in one round
    uint32_t g = 2u;
    while (g < (uint32_t)(k - 1)) g <<= 1;
    return (unsigned long long)sets * g <= limit ? g : 1u;
}

#ifndef MPDP_PHASES_ONLY
__global__ void __launch_bounds__(256) k_level_prefix(BatchArgs a, uint32_t* MPDP_RESTRICT pref, uint32_t group_threads)
{
    __shared__ uint32_t s_pref[kMaxBatch + 1];
    const int k = blockIdx.x / 2 + 2, mode = (blockIdx.x & 1) ? MPDP_ENUM_BLOCKS : MPDP_ENUM_TREE;
    uint32_t* row = pref + ((mode == MPDP_ENUM_BLOCKS ? kLevels : 0) + k) * kPrefStride;
    uint32_t group = 0u;
    if (mode == MPDP_ENUM_TREE) {
        const uint32_t sets = block_prefix(a.nq, s_pref, [&](int q) {
            return level_tiles(a, q, k, mode) ? a.out[q].counters.list_count[k] : 0u;
        });
        const uint32_t g = group_size(sets, k, group_threads);  // block-uniform
        group = g > 1u ? g : 0u;
    }
    if (!group) block_prefix(a.nq, s_pref, [&](int q) { return level_tiles(a, q, k, mode); });
    for (int i = threadIdx.x; i <= a.nq; i += blockDim.x) row[i] = s_pref[i];
    if (threadIdx.x == 0) row[kMaxBatch + 1] = group;
}
#endif

// (x, left) minimum over the g lanes of a group (g a power of two <= 32,
// groups aligned within the warp; mask: the group's lanes).
__device__ __forceinline__ void group_min_x(unsigned long long& bx, uint32_t& bl, uint32_t g, unsigned mask)
{
    for (uint32_t o = g >> 1; o > 0u; o >>= 1) {
        const unsigned long long ox = __shfl_xor_sync(mask, bx, o);
        const uint32_t ol = __shfl_xor_sync(mask, bl, o);
        if (better_x(ox, ol, bx, bl)) {
            bx = ox;
            bl = ol;
        }
    }
}

// One tree level by groups of G lanes per set (set g of the level's set
// prefix s_pref, grid-stride): lane j of a group forms the split below the
// member of rank j of S minus its top; the group's (x, left) minimum goes to
// its first lane, which writes the memo and counts the set in s_sets.
template <class Memo>
__device__ __forceinline__ void eval_tree_groups(const BatchArgs& a, int k, uint32_t G, Memo& memo,
                                                 const uint32_t* s_pref, uint32_t* s_sets, uint32_t bid,
                                                 uint32_t nblk)
{
    const uint32_t nsets = s_pref[a.nq];
    const uint32_t gl = threadIdx.x & (G - 1u);
    const unsigned gmask = G == 32u ? kFull : ((1u << G) - 1u) << ((threadIdx.x & 31u) & ~(G - 1u));
    for (uint32_t g = (bid * kEvalThreads + threadIdx.x) / G; g < nsets; g += nblk * (kEvalThreads / G)) {
        const int qi = find_q(s_pref, a.nq, g);
        const DevQuery* MPDP_RESTRICT q = a.query + qi;
        DevCounters* cnt = &a.out[qi].counters;
        memo.bind(a, qi);
        const QDesc& d = a.desc[qi];
        const uint32_t s = a.lists[d.list_base + d.list_off[k] + (g - s_pref[qi])];
        const int top = set_top_of(q, s);
        const int pv = tree_peel_vertex(s, q->adj);
        const double pbase = gl == 0u ? peel_base(s, pv, *q, memo, cnt) : 0.0;
        unsigned long long bx = kNoX;
        uint32_t bl = kFull;
        const uint32_t rest = s & ~(1u << top);
        // this lane's split: the member of rest of rank gl (G >= k - 1)
        if ((int)gl < k - 1) {
            const uint32_t sl = MPDP_LDG(&q->desc[__fns(rest, 0u, gl + 1)]) & s;
            fold_pair(sl, s ^ sl, memo, cnt, bx, bl);
        }
        group_min_x(bx, bl, G, gmask);
        if (gl == 0u) {
            const double card_s = peel_finish(pbase, s, pv, *q);
            memo.put(s, k, set_cost(bx, card_s), card_s, bl, cnt);
            atomicAdd(&s_sets[qi], 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// a4-a8, tree join graphs (Algorithm 2, MPDP:Tree).  One thread per connected
// set S of level k (tiles of 256 sets of one query per block iteration), or
// a group of lanes per set on levels with few sets.  Every connected S
// induces a subtree of the query tree T (rooted at relation 0), hanging from
// its top member (the one whose descendants cover S); its CCP pairs are the
// k-1 splits made by removing one edge of G[S].  Removing the edge above any
// other member v leaves S_l = desc[v] & S (the part of S under v) and
// S_r = S \ S_l: one AND per split, no search.  The best (cost, left) over
// the k-1 splits is written to the memo: evaluate, prune and scatter fused
// in one pass, one memo write per set.
template <class Memo, int kQ = kMaxBatch>  // kQ: the most queries of a batch it serves
__device__ void eval_tree_body(const BatchArgs& a, int k, Memo memo, const uint32_t* MPDP_RESTRICT level_pref, uint32_t bid, uint32_t nblk)
{
    __shared__ uint32_t s_pref[kQ + 1];
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    const uint32_t G = level_pref[k * kPrefStride + kMaxBatch + 1];
    {
        // a block with no tile (or no group) of this level leaves at once
        const uint32_t total = level_pref[k * kPrefStride + a.nq];  // tiles, or sets in group mode
        if (G ? bid * (kEvalThreads / G) >= total : bid >= total) return;  // block-uniform
    }
    memo.setup(s_memo);
    for (int i = threadIdx.x; i <= a.nq; i += blockDim.x) s_pref[i] = level_pref[k * kPrefStride + i];
    __syncthreads();
    if (G) {  // groups of G lanes per set (s_pref: set prefix); block-uniform
        __shared__ uint32_t s_sets[kQ];  // sets evaluated per query
        for (int i = threadIdx.x; i < a.nq; i += blockDim.x) s_sets[i] = 0u;
        __syncthreads();
        eval_tree_groups(a, k, G, memo, s_pref, s_sets, bid, nblk);
        __syncthreads();
        for (int i = threadIdx.x; i < a.nq; i += blockDim.x)
            if (s_sets[i]) {
                atomicAdd(&a.out[i].counters.evaluated[k], (unsigned long long)s_sets[i] * (unsigned long long)(k - 1));
                atomicAdd(&a.out[i].counters.ccp[k], (unsigned long long)s_sets[i] * (unsigned long long)(k - 1));
            }
        return;
    }
    const uint32_t tiles = s_pref[a.nq];
    // Tiles go round-robin over the blocks, so the sets in flight at any
    // time are neighbours in the level lists (their memo reads are close).
    // The query is read through the cache, not staged in shared memory:
    // consecutive tiles of a block belong to different queries and a
    // switch then costs no block barrier.
    int cur = -1;
    const DevQuery* MPDP_RESTRICT q = nullptr;
    unsigned long long sets = 0;
    for (uint32_t t = bid; t < tiles; t += nblk) {
        const int qi = find_q(s_pref, a.nq, t);
        if (qi != cur) {  // block-uniform
            if (cur >= 0) {
                sets = warp_sum(sets);
                if ((threadIdx.x & 31) == 0 && sets) {
                    atomicAdd(&a.out[cur].counters.evaluated[k], sets * (unsigned long long)(k - 1));
                    atomicAdd(&a.out[cur].counters.ccp[k], sets * (unsigned long long)(k - 1));
                }
                sets = 0;
            }
            q = a.query + qi;
            memo.bind(a, qi);
            cur = qi;
        }
        DevCounters* cnt = &a.out[qi].counters;
        const uint32_t idx = (t - s_pref[qi]) * kEvalThreads + threadIdx.x;
        if (idx < cnt->list_count[k]) {
            const QDesc& d = a.desc[qi];
            const uint32_t s = a.lists[d.list_base + d.list_off[k] + idx];
            // G[S] is the query tree restricted to S, hanging from its top
            // vertex (the member whose descendants cover S).  Removing the
            // edge above any other member v leaves the subtree under v,
            // desc[v] & S, and the rest: the k-1 CCP pairs of S, one AND each.
            uint32_t t2 = s;
            int top = lowest(t2);
            while ((MPDP_LDG(&q->desc[top]) & s) != s) {
                t2 &= t2 - 1u;
                top = lowest(t2);
            }
            // card(S \ {v}) is loaded before the pairs and used after them,
            // so its latency overlaps theirs
            const int pv = tree_peel_vertex(s, q->adj);
            const double pbase = peel_base(s, pv, *q, memo, cnt);
            unsigned long long bx = kNoX;
            uint32_t bl = kFull;
            uint32_t rest = s & ~(1u << top);
            // two splits at a time: both left sides, then their four cost
            // loads together, then the fold (one more load in flight per
            // thread without raising the register count)
            for (int i = 1; i < k; i += 2) {
                const int v0 = lowest(rest);
                rest &= rest - 1u;
                const uint32_t sl0 = MPDP_LDG(&q->desc[v0]) & s;
                uint32_t sl1 = 0u;
                if (i + 1 < k) {
                    const int v1 = lowest(rest);
                    rest &= rest - 1u;
                    sl1 = MPDP_LDG(&q->desc[v1]) & s;
                }
                const uint32_t sr0 = s ^ sl0, sr1 = s ^ sl1;
                const double cl0 = (sl0 & (sl0 - 1u)) ? memo.get_cost(sl0, cnt) : 0.0;
                const double cr0 = (sr0 & (sr0 - 1u)) ? memo.get_cost(sr0, cnt) : 0.0;
                const double cl1 = (sl1 & (sl1 - 1u)) ? memo.get_cost(sl1, cnt) : 0.0;
                const double cr1 = (sl1 != 0u && (sr1 & (sr1 - 1u))) ? memo.get_cost(sr1, cnt) : 0.0;
                fold_costs(sl0, sr0, cl0, cr0, bx, bl);
                if (sl1 != 0u) fold_costs(sl1, sr1, cl1, cr1, bx, bl);
            }
            const double card_s = peel_finish(pbase, s, pv, *q);
            memo.put(s, k, set_cost(bx, card_s), card_s, bl, cnt);
            sets++;
        }
    }
    if (cur >= 0) {
        sets = warp_sum(sets);
        if ((threadIdx.x & 31) == 0 && sets) {
            atomicAdd(&a.out[cur].counters.evaluated[k], sets * (unsigned long long)(k - 1));
            atomicAdd(&a.out[cur].counters.ccp[k], sets * (unsigned long long)(k - 1));
        }
    }
}

#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_tree(BatchArgs a, int k, Memo memo, const uint32_t* MPDP_RESTRICT level_pref)
{
    eval_tree_body(a, k, memo, level_pref, blockIdx.x, gridDim.x);
}
#endif

// ---------------------------------------------------------------------------
// Ablation of the fusion (Sec. 5: evaluate and prune in one kernel): the same
// tree-mode work as k_eval_tree in two kernels.  The first writes every CCP
// pair's (x, left) to global memory, slot (tile * 256 + thread) * (k - 1) + i;
// the second reads a set's k - 1 records back, keeps the (x, left) minimum,
// computes card(S) and writes the memo.  Same tiles, same results.
#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_tree_pairs(BatchArgs a, int k, Memo memo,
                                                                  PairRec* MPDP_RESTRICT pairs)
{
    __shared__ uint32_t s_pref[kMaxBatch + 1];
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    memo.setup(s_memo);
    const uint32_t tiles = block_prefix(a.nq, s_pref, [&](int q) { return level_tiles(a, q, k, MPDP_ENUM_TREE); });
    int cur = -1;
    unsigned long long sets = 0;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int qi = find_q(s_pref, a.nq, t);
        if (qi != cur) {
            if (cur >= 0) {
                sets = warp_sum(sets);
                if ((threadIdx.x & 31) == 0 && sets) {
                    atomicAdd(&a.out[cur].counters.evaluated[k], sets * (unsigned long long)(k - 1));
                    atomicAdd(&a.out[cur].counters.ccp[k], sets * (unsigned long long)(k - 1));
                }
                sets = 0;
            }
            memo.bind(a, qi);
            cur = qi;
        }
        const DevQuery* MPDP_RESTRICT q = a.query + qi;
        DevCounters* cnt = &a.out[qi].counters;
        const uint32_t idx = (t - s_pref[qi]) * kEvalThreads + threadIdx.x;
        if (idx < cnt->list_count[k]) {
            const QDesc& d = a.desc[qi];
            const uint32_t s = a.lists[d.list_base + d.list_off[k] + idx];
            uint32_t t2 = s;
            int top = lowest(t2);
            while ((MPDP_LDG(&q->desc[top]) & s) != s) {
                t2 &= t2 - 1u;
                top = lowest(t2);
            }
            PairRec* out = pairs + ((unsigned long long)t * kEvalThreads + threadIdx.x) * (unsigned long long)(k - 1);
            uint32_t rest = s & ~(1u << top);
            for (int i = 1; i < k; i++) {
                const int v = lowest(rest);
                rest &= rest - 1u;
                const uint32_t sl = MPDP_LDG(&q->desc[v]) & s;
                unsigned long long bx = kNoX;
                uint32_t bl = kFull;
                fold_pair(sl, s ^ sl, memo, cnt, bx, bl);  // one pair: its own (x, left)
                out[i - 1].x = bx;
                out[i - 1].left = bl;
            }
            sets++;
        }
    }
    if (cur >= 0) {
        sets = warp_sum(sets);
        if ((threadIdx.x & 31) == 0 && sets) {
            atomicAdd(&a.out[cur].counters.evaluated[k], sets * (unsigned long long)(k - 1));
            atomicAdd(&a.out[cur].counters.ccp[k], sets * (unsigned long long)(k - 1));
        }
    }
}
#endif

#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_prune_tree(BatchArgs a, int k, Memo memo,
                                                             const PairRec* MPDP_RESTRICT pairs)
{
    __shared__ uint32_t s_pref[kMaxBatch + 1];
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    memo.setup(s_memo);
    const uint32_t tiles = block_prefix(a.nq, s_pref, [&](int q) { return level_tiles(a, q, k, MPDP_ENUM_TREE); });
    int cur = -1;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int qi = find_q(s_pref, a.nq, t);
        if (qi != cur) {
            memo.bind(a, qi);
            cur = qi;
        }
        const DevQuery* MPDP_RESTRICT q = a.query + qi;
        DevCounters* cnt = &a.out[qi].counters;
        const uint32_t idx = (t - s_pref[qi]) * kEvalThreads + threadIdx.x;
        if (idx < cnt->list_count[k]) {
            const QDesc& d = a.desc[qi];
            const uint32_t s = a.lists[d.list_base + d.list_off[k] + idx];
            const int pv = tree_peel_vertex(s, q->adj);
            const double pbase = peel_base(s, pv, *q, memo, cnt);
            const PairRec* in = pairs + ((unsigned long long)t * kEvalThreads + threadIdx.x) * (unsigned long long)(k - 1);
            unsigned long long bx = kNoX;
            uint32_t bl = kFull;
            for (int i = 0; i < k - 1; i++) {
                const PairRec r = in[i];
                if (better_x(r.x, r.left, bx, bl)) {
                    bx = r.x;
                    bl = r.left;
                }
            }
            const double card_s = peel_finish(pbase, s, pv, *q);
            memo.put(s, k, set_cost(bx, card_s), card_s, bl, cnt);
        }
    }
}
#endif

// ---------------------------------------------------------------------------
// Block CCP lists (the cache described at kBlTab).  Lookup of block b in a
// query's area: the first left side and the count, false when b is not
// listed.
__device__ __forceinline__ bool bl_find(const uint32_t* MPDP_RESTRICT area, uint32_t b, uint32_t& off, uint32_t& cnt)
{
    uint32_t h = fmix32(b) & (kBlTab - 1u);
    for (uint32_t i = 0; i < kBlTab; i++) {
        const uint32_t* e = area + 4u + 4u * h;
        const uint32_t key = MPDP_LDG(e);
        if (key == b) {
            off = MPDP_LDG(e + 1);
            cnt = MPDP_LDG(e + 2);
            return true;
        }
        if (key == 0u) return false;
        h = (h + 1u) & (kBlTab - 1u);
    }
    return false;
}

#ifndef MPDP_PHASES_ONLY
// The query's connected sets of 3 to kBlMaxBlock relations (all levels, a
// thread per set) that are 2-connected and not cliques, appended to the
// area's set array: S is 2-connected when S \ {x} stays connected for every
// member x, one bit of the connectivity bitmap each.
__global__ void __launch_bounds__(256) k_block_detect(BatchArgs a)
{
    __shared__ uint32_t s_pref[kMaxBatch + 1];
    const uint32_t tiles = block_prefix(a.nq, s_pref, [&](int q) -> uint32_t {
        const QDesc& d = a.desc[q];
        const DevCounters& c = a.out[q].counters;
        if (!d.use_bl || c.status != 0) return 0u;
        uint32_t t = 0u;
        for (int k = 3; k <= d.n && k <= kBlMaxBlock; k++) t += (c.list_count[k] + 255u) / 256u;
        return t;
    });
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int qi = find_q(s_pref, a.nq, t);  // block-uniform
        const QDesc& d = a.desc[qi];
        const DevCounters& c = a.out[qi].counters;
        uint32_t r = t - s_pref[qi];
        int k = 3;
        for (; k <= d.n && k <= kBlMaxBlock; k++) {
            const uint32_t lt = (c.list_count[k] + 255u) / 256u;
            if (r < lt) break;
            r -= lt;
        }
        const uint32_t idx = r * 256u + threadIdx.x;
        if (k > d.n || k > kBlMaxBlock || idx >= c.list_count[k]) continue;
        const DevQuery* MPDP_RESTRICT q = a.query + qi;
        const uint32_t s = a.lists[d.list_base + d.list_off[k] + idx];
        if (is_clique(s, q->adj)) continue;
        const uint32_t* MPDP_RESTRICT cw = conn_bitmap(a, qi);
        bool two = true;
        for (uint32_t x = s; x != 0u && two; x &= x - 1u) two = conn_of(s & ~(x & (0u - x)), cw, q->adj);
        if (!two) continue;
        uint32_t* area = a.lists + d.bl_base;
        const uint32_t i = atomicAdd(&area[0], 1u);
        if (i < kBlSets) area[kBlHead + i] = s;
    }
}

// One block per set B found by k_block_detect: its bipartitions (lb holding
// min(B), lb != B) are split over the threads in contiguous runs (the first
// lb of a run by deposit, the next by stepping to the next submask); a
// first pass counts the CCPs (lb and rb both connected), the block reserves
// room in the store, a second pass writes the left sides, and B goes into
// the table.  No room left: B stays unlisted.
__global__ void __launch_bounds__(256) k_block_list(BatchArgs a)
{
    __shared__ uint32_t s_pref[kMaxBatch + 1];
    __shared__ uint32_t s_found[256], s_off[257];
    __shared__ uint32_t s_base, s_total;
    const uint32_t items = block_prefix(a.nq, s_pref, [&](int q) -> uint32_t {
        const QDesc& d = a.desc[q];
        if (!d.use_bl || a.out[q].counters.status != 0) return 0u;
        const uint32_t f = a.lists[d.bl_base];
        return f < kBlSets ? f : kBlSets;
    });
    for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int qi = find_q(s_pref, a.nq, it);  // block-uniform
        const QDesc& d = a.desc[qi];
        const DevQuery* MPDP_RESTRICT q = a.query + qi;
        const uint32_t* MPDP_RESTRICT cw = conn_bitmap(a, qi);
        uint32_t* area = a.lists + d.bl_base;
        const uint32_t b = area[kBlHead + (it - s_pref[qi])];
        const uint32_t mn = b & (0u - b), rest = b ^ mn;
        const uint32_t total = block_pairs(b);
        const uint32_t per = (total + blockDim.x - 1u) / blockDim.x;
        const uint32_t i0 = threadIdx.x * per < total ? threadIdx.x * per : total;
        const uint32_t i1 = i0 + per < total ? i0 + per : total;
        uint32_t found = 0u;
        {
            uint32_t sub = i0 < i1 ? deposit(i0, rest) : 0u;
            for (uint32_t i = i0; i < i1; i++, sub = (sub - rest) & rest) {
                const uint32_t lb = mn | sub, rb = b ^ lb;
                if (conn_of(lb, cw, q->adj) && conn_of(rb, cw, q->adj)) found++;
            }
        }
        s_found[threadIdx.x] = found;
        __syncthreads();
        const uint32_t all = block_prefix((int)blockDim.x, s_off, [&](int i) { return s_found[i]; });
        if (threadIdx.x == 0) {
            // once the store is full no block adds to its count (no wrap)
            const uint32_t used = *reinterpret_cast<volatile uint32_t*>(&area[1]);
            s_base = (all <= kBlLbs && used < kBlLbs) ? atomicAdd(&area[1], all) : kBlLbs + 1u;
            s_total = all;
        }
        __syncthreads();
        const uint32_t base = s_base;
        if (base <= kBlLbs && s_total <= kBlLbs - base) {  // block-uniform
            uint32_t* lbs = area + kBlHead + kBlTab + base + s_off[threadIdx.x];
            uint32_t w = 0u;
            uint32_t sub = i0 < i1 ? deposit(i0, rest) : 0u;
            for (uint32_t i = i0; i < i1 && w < found; i++, sub = (sub - rest) & rest) {
                const uint32_t lb = mn | sub, rb = b ^ lb;
                if (conn_of(lb, cw, q->adj) && conn_of(rb, cw, q->adj)) lbs[w++] = lb;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t h = fmix32(b) & (kBlTab - 1u);
                for (uint32_t i = 0; i < kBlTab; i++) {
                    uint32_t* e = area + 4u + 4u * h;
                    if (atomicCAS(e, 0u, b) == 0u) {
                        e[1] = base;
                        e[2] = s_total;
                        break;
                    }
                    h = (h + 1u) & (kBlTab - 1u);
                }
            }
        }
        __syncthreads();
    }
}
#endif

// ---------------------------------------------------------------------------
// a4-a8, general join graphs (Algorithm 4), thread per set for light sets.
// For each block B of G[S] and each lb (min(B) in lb, lb != B): rb = B \ lb;
// the CCP block keeps the pair when lb and rb both induce connected subgraphs
// (they are adjacent since B is connected); then S_l = grow(lb, S \ rb),
// S_r = S \ S_l.  Sets whose work exceeds the heavy threshold go to the warp
// path instead.  On a level with at least kFullLevelSets sets (enough to
// fill the GPU a thread per set) a thread's work counts the pairs of a
// clique block at 1/kCliqueWeight: each is a CCP with no connectivity test,
// and sets of up to about a thousand of them then run faster here than on
// the warp path (measured on clique-14; with fewer sets per level, as on
// clique-12, the warp path's spread wins).  On a level with fewer sets the
// threshold is halved: a set's thread then works alone at the end of the
// level, and the warp path's split of its CCPs over 32 lanes is shorter.
// The work of the other blocks (candidate bipartitions, listed CCPs) meets a
// limit that follows the level's size: heavy_threshold * slots / kNcRefSlots
// for a level of `slots` thread slots, clamped to [kFullLevelSets,
// kNcMaxSlots] (a quarter to twice heavy_threshold).  On a level that leaves
// most of the GPU's threads idle the warp path's spread shortens the level's
// longest chains, and a set whose candidates each cost two dependent bitmap
// reads is worth spreading at a smaller size than a clique block, whose pairs
// are all CCPs (measured against one limit for both kinds, 64-query batches:
// cyclic-16 and cyclic-18 13-14 % faster, cyclic-20 and cyclic-22 6 %,
// cyclic-25 and the cliques unchanged).  A set mixing both kinds weighs each
// against its own limit.
constexpr uint32_t kCliqueWeight = 16u;
constexpr uint32_t kFullLevelSets = 16384u;
constexpr uint32_t kNcRefSlots = 65536u;
constexpr uint32_t kNcMaxSlots = 131072u;
// Find-Blocks cache (batched kernels): the thread-per-set kernel, which
// finds a set's blocks to weigh its work, leaves them for the warp path when
// it appends the set as heavy (main entry i < kFbCap of the level): one line
// per set, word 0 the block count, words 1.. the blocks (64 B for queries of
// up to 16 relations, whose sets have at most 15 blocks; else 128 B).  Every
// chunk of the set then reads the line (a word per lane) instead of running
// Find-Blocks again on one lane while the others wait.  The cache sits after
// the block CCP lists in the query's list words.
constexpr uint32_t kFbCap = 4096u;
__host__ __device__ __forceinline__ uint32_t fb_stride(int n) { return n <= 16 ? 16u : 32u; }
__device__ __forceinline__ uint32_t* fb_cache(const BatchArgs& a, const QDesc& d)
{
    return a.lists + d.bl_base + (d.n >= kBlMinRels ? kBlWords : 0u);
}
// The block-mode bodies' staged query.  At file scope, a kernel that runs
// both bodies (the persistent kernel) holds one copy rather than two; each
// batched kernel holds its own as before.
__shared__ SharedQuery g_block_sq;

// kQ: the most queries of a batch it serves.  kBatched: the batched
// kernels' form, where the non-clique limit follows the level's size and
// heavy sets leave their blocks in the Find-Blocks cache.  The persistent
// kernel's one-query phases take neither: such a phase shares the GPU with
// the other slots' phases, so its own level size says little about idle
// threads, and its slots have no cache.
template <class Memo, int kQ = kMaxBatch, bool kBatched = true>
__device__ void eval_blocks_body(const BatchArgs& a, int k, Memo memo, const uint32_t* MPDP_RESTRICT level_pref, uint32_t bid, uint32_t nblk)
{
    SharedQuery& sq = g_block_sq;
    __shared__ uint32_t s_pref[kQ + 1];
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    memo.setup(s_memo);
    for (int i = threadIdx.x; i <= a.nq; i += blockDim.x) s_pref[i] = level_pref[(kLevels + k) * kPrefStride + i];
    __syncthreads();
    const uint32_t tiles = s_pref[a.nq];
    const unsigned long long slots = (unsigned long long)tiles * kEvalThreads;
    const bool full = slots >= kFullLevelSets;
    // The heavy test in 1/16 units: 16 * work_cl + nc_w16 * work_nc > lim16.
    const uint32_t nc_slots = !full ? kFullLevelSets : (slots > kNcMaxSlots ? kNcMaxSlots : (uint32_t)slots);
    const uint32_t nc_w16 = kBatched ? (full ? 16u : 8u) * kNcRefSlots / nc_slots : 16u;
    const unsigned long long lim16 = 16ull * (full ? (uint32_t)a.heavy_threshold : (uint32_t)a.heavy_threshold / 2u);
    int cur = -1;
    unsigned long long evaluated = 0, ccp = 0;
    const int lane = threadIdx.x & 31;
    for (uint32_t t = bid; t < tiles; t += nblk) {
        const int qi = find_q(s_pref, a.nq, t);
        if (qi != cur) {
            if (cur >= 0) {
                evaluated = warp_sum(evaluated);
                ccp = warp_sum(ccp);
                if (lane == 0) {
                    if (evaluated) atomicAdd(&a.out[cur].counters.evaluated[k], evaluated);
                    if (ccp) atomicAdd(&a.out[cur].counters.ccp[k], ccp);
                }
                evaluated = ccp = 0;
            }
            __syncthreads();
            load_query(sq, a.query + qi);
            memo.bind(a, qi);
            __syncthreads();
            cur = qi;
        }
        DevCounters* cnt = &a.out[qi].counters;
        const QDesc& d = a.desc[qi];
        const uint32_t* MPDP_RESTRICT cw = conn_bitmap(a, qi);
        const uint32_t* MPDP_RESTRICT blist = d.use_bl ? a.lists + d.bl_base : nullptr;
        const uint32_t idx = (t - s_pref[qi]) * kEvalThreads + threadIdx.x;
        bool to_heavy = false;
        uint32_t s = 0u, want = 0u;  // want: extra chunks asked for
        uint32_t blk[kMaxRels];
        int nb = 0;
        if (idx < cnt->list_count[k]) {
            s = a.lists[d.list_base + d.list_off[k] + idx];
            uint32_t side[kMaxRels];
            nb = find_blocks(s, sq.adj, blk, a.dpsub ? nullptr : side);
            // pairs: the set's bipartitions; work: what a thread pays for
            // them, a clique block's pairs at 1/kCliqueWeight (no
            // connectivity test, every pair a CCP)
            // listed: bit j, block j's CCPs come from the block CCP lists
            // (its work then their count)
            // index: the warp path's pair index space (a listed block's CCPs,
            // any other block's bipartitions)
            // work_cl, work_nc: the work of the clique blocks and of the others
            uint32_t pairs = 0u, work_cl = 0u, work_nc = 0u, index = 0u, cliq = 0u, listed = 0u;  // cliq: bit j, block j is a clique
            for (int j = 0; j < nb; j++) {
                const uint32_t p = block_pairs(blk[j]);
                pairs += p;
                uint32_t off = 0u, nl = 0u;
                if (!a.dpsub && !side[j] && is_clique(blk[j], sq.adj)) {
                    cliq |= 1u << j;
                    work_cl += full ? (p + kCliqueWeight - 1u) / kCliqueWeight : p;
                    index += p;
                } else if (blist && !side[j] && bl_find(blist, blk[j], off, nl)) {
                    listed |= 1u << j;
                    work_nc += nl;
                    index += nl;
                } else {
                    work_nc += p;
                    index += p;
                }
            }
            if (a.dpsub) {  // the whole set as one block
                pairs = work_nc = index = block_pairs(s);
                work_cl = 0u;
            }
            if (16ull * work_cl + (unsigned long long)nc_w16 * work_nc > lim16) {
                to_heavy = true;
                const uint32_t nch = (index - 1u) / kChunkPairs + 1u;
                want = (nch < kMaxChunks ? nch : kMaxChunks) - 1u;
            } else {
                const double card_s = peel_card(s, block_peel_vertex(s, blk, nb), sq, memo, cnt);
                unsigned long long bx = kNoX;
                uint32_t bl = kFull;
                evaluated += pairs;
                const int enb = a.dpsub ? 1 : nb;
                for (int j = 0; j < enb; j++) {
                    const uint32_t b = a.dpsub ? s : blk[j];
                    if (!a.dpsub && side[j]) {
                        // a bridge: its one pair is a CCP, the lower vertex's side known
                        ccp++;
                        fold_pair(side[j], s ^ side[j], memo, cnt, bx, bl);
                        continue;
                    }
                    if (listed >> j & 1u) {  // its CCPs, listed once for the query
                        uint32_t off = 0u, nl = 0u;
                        bl_find(blist, b, off, nl);
                        const uint32_t* MPDP_RESTRICT lbs = blist + kBlHead + kBlTab + off;
                        for (uint32_t i = 0; i < nl; i++) {
                            const uint32_t lb = MPDP_LDG(&lbs[i]);
                            ccp++;
                            const uint32_t sl = left_side(s, lb, b ^ lb, sq.adj);
                            fold_pair(sl, s ^ sl, memo, cnt, bx, bl);
                        }
                        continue;
                    }
                    const uint32_t mn = b & (0u - b), rest = b ^ mn;
                    const bool all_ccp = !a.dpsub && (cliq >> j & 1u);
                    for (uint32_t sub = 0u; sub != rest; sub = (sub - rest) & rest) {
                        const uint32_t lb = mn | sub, rb = b ^ lb;
                        if (!all_ccp && (!conn_of(lb, cw, sq.adj) || !conn_of(rb, cw, sq.adj))) continue;
                        ccp++;
                        const uint32_t sl = left_side(s, lb, rb, sq.adj);
                        fold_pair(sl, s ^ sl, memo, cnt, bx, bl);
                    }
                }
                memo.put(s, k, set_cost(bx, card_s), card_s, bl, cnt);
            }
        }
        // Warp-aggregated append of heavy sets.  The main entries never
        // overflow (at most C(n, k) sets per level).  Extra chunks are
        // reserved with one atomicAdd per warp; a reservation that runs past
        // the capacity keeps only its part below it, so the written extra
        // entries are exactly [0, min(extra_count, heavy_cap)) and a set
        // that gets fewer chunks just has longer ones.
        const unsigned bal = __ballot_sync(kFull, to_heavy);
        if (bal) {
            uint32_t pre = want;  // inclusive warp scan of the extra chunks asked for
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(kFull, pre, o);
                if (lane >= o) pre += v;
            }
            const uint32_t total = __shfl_sync(kFull, pre, 31);
            pre -= want;
            uint32_t base = 0, ebase = 0;
            if (lane == 0) {
                base = atomicAdd(&cnt->heavy_count[k], (uint32_t)__popc(bal));
                // once full, stop adding: keeps the counter far from wrapping
                const uint32_t seen = *reinterpret_cast<volatile uint32_t*>(&cnt->extra_count[k]);
                ebase = d.heavy_cap;
                if (total && seen < d.heavy_cap) ebase = atomicAdd(&cnt->extra_count[k], total);
            }
            base = __shfl_sync(kFull, base, 0);
            ebase = __shfl_sync(kFull, ebase, 0);
            if (to_heavy) {
                const uint32_t cap = d.heavy_cap;
                const uint32_t room = ebase < cap ? cap - ebase : 0u;
                const uint32_t got = pre >= room ? 0u : (want < room - pre ? want : room - pre);
                const uint32_t i = base + __popc(bal & ((1u << lane) - 1u));
                HeavyMain* hm = a.hmain + d.heavy_base;
                hm[i] = HeavyMain{s, 1u + got, ebase + pre, 0u, kNoX, kFull, 0u};
                HeavyExtra* he = a.hextra + d.heavy_base + ebase + pre;
                for (uint32_t c = 0; c < got; c++) he[c] = HeavyExtra{i, kFull, kNoX};
                if (kBatched && i < min(d.heavy_cap, kFbCap)) {
                    uint32_t* e = fb_cache(a, d) + (size_t)i * fb_stride(d.n);
                    e[0] = (uint32_t)nb;
                    for (int j = 0; j < nb; j++) e[1 + j] = blk[j];
                }
            }
        }
    }
    if (cur >= 0) {
        evaluated = warp_sum(evaluated);
        ccp = warp_sum(ccp);
        if (lane == 0) {
            if (evaluated) atomicAdd(&a.out[cur].counters.evaluated[k], evaluated);
            if (ccp) atomicAdd(&a.out[cur].counters.ccp[k], ccp);
        }
    }
}

#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_blocks(BatchArgs a, int k, Memo memo, const uint32_t* MPDP_RESTRICT level_pref)
{
    eval_blocks_body(a, k, memo, level_pref, blockIdx.x, gridDim.x);
}
#endif

// Heavy-set evaluation (general mode).  The work items of level k are the
// pair chunks reserved by k_eval_blocks: a block takes a tile of 8 items of
// one query, one per warp (the paper evaluates a set with one warp, Sec. 5
// "Evaluate"; a set with many pairs is spread over several warps here so that
// no level waits on one warp working through its largest set).  Lane 0 finds
// the blocks of the item's set; the lanes split the chunk's pair indices.
// With Collaborative Context Collection (Sec. 5, "Avoiding 'If' branch
// divergence") each warp stashes the pairs that pass the CCP test in shared
// memory and grows/costs them only when 32 are ready, so no lane idles on an
// invalid pair during the expensive part.  The prune is a warp shuffle
// reduction of (x, left); a set cut into several chunks is folded by the
// warp that finishes it last (fence, then an arrival count), with no waiting.
template <class Memo, int kQ = kMaxBatch, bool kBatched = true>  // as eval_blocks_body
__device__ void eval_heavy_body(const BatchArgs& a, int k, Memo memo, uint32_t bid, uint32_t nblk)
{
    constexpr int kWarps = kEvalThreads / 32;
    SharedQuery& sq = g_block_sq;
    __shared__ uint32_t s_pref[kQ + 1];
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    __shared__ uint32_t s_blk[kWarps][kMaxRels];
    __shared__ uint32_t s_bpref[kWarps][kMaxRels + 1];
    __shared__ int s_nb[kWarps];
    __shared__ int s_pv[kWarps];
    __shared__ uint32_t s_cliq[kWarps];  // bit j: block j is a clique
    __shared__ uint32_t s_list[kWarps];  // bit j: block j's CCPs are listed (block CCP lists)
    __shared__ uint32_t s_loff[kWarps][kMaxRels];  // first listed left side of block j
    __shared__ uint32_t s_stash_l[kWarps][64];
    __shared__ uint32_t s_stash_r[kWarps][64];
    memo.setup(s_memo);
    const uint32_t tiles = block_prefix(a.nq, s_pref, [&](int q) -> uint32_t {
        const QDesc& d = a.desc[q];
        const DevCounters& c = a.out[q].counters;
        if (d.n < k || d.enumeration != MPDP_ENUM_BLOCKS || c.status != 0) return 0u;
        const uint32_t extra = c.extra_count[k] < d.heavy_cap ? c.extra_count[k] : d.heavy_cap;
        return (c.heavy_count[k] + extra + kWarps - 1) / kWarps;
    });
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cur = -1;
    unsigned long long ccp = 0, evaluated = 0, heavy = 0;
    for (uint32_t t = bid; t < tiles; t += nblk) {
        const int qi = find_q(s_pref, a.nq, t);
        if (qi != cur) {
            if (cur >= 0 && lane == 0) {
                if (ccp) atomicAdd(&a.out[cur].counters.ccp[k], ccp);
                if (evaluated) atomicAdd(&a.out[cur].counters.evaluated[k], evaluated);
                if (heavy) atomicAdd(&a.out[cur].counters.heavy, heavy);
            }
            ccp = evaluated = heavy = 0;
            __syncthreads();
            load_query(sq, a.query + qi);
            memo.bind(a, qi);
            __syncthreads();
            cur = qi;
        }
        DevCounters* cnt = &a.out[qi].counters;
        const QDesc& d = a.desc[qi];
        const uint32_t nmain = cnt->heavy_count[k];
        const uint32_t nextra = cnt->extra_count[k] < d.heavy_cap ? cnt->extra_count[k] : d.heavy_cap;
        const uint32_t item = (t - s_pref[qi]) * kWarps + warp;
        if (item >= nmain + nextra) continue;  // warp-uniform
        HeavyMain* hm = a.hmain + d.heavy_base;
        HeavyExtra* he = a.hextra + d.heavy_base;
        const uint32_t mi = item < nmain ? item : he[item - nmain].main;
        const uint32_t s = hm[mi].set, nch = hm[mi].nch, ebase = hm[mi].ebase;
        const uint32_t chunk = item < nmain ? 0u : item - nmain - ebase + 1u;
        // the set's blocks: from the Find-Blocks cache when the thread-per-set
        // kernel left them there (one line, a word per lane), else found here
        const bool cached = kBatched && mi < min(d.heavy_cap, kFbCap);  // warp-uniform
        int nb_cached = 0;
        if (cached) {
            const uint32_t st = fb_stride(d.n);
            const uint32_t v = (uint32_t)lane < st ? MPDP_LDG(fb_cache(a, d) + (size_t)mi * st + lane) : 0u;
            nb_cached = (int)__shfl_sync(kFull, v, 0);
            if (lane >= 1 && lane <= nb_cached) s_blk[warp][lane - 1] = v;
            __syncwarp();
        }
        if (lane == 0) {
            int nb = cached ? nb_cached : find_blocks(s, sq.adj, s_blk[warp]);
            s_pv[warp] = block_peel_vertex(s, s_blk[warp], nb);
            if (a.dpsub) {  // the whole set as one block
                s_blk[warp][0] = s;
                nb = 1;
            }
            // pair index space: a listed block contributes its CCPs, any
            // other block all its bipartitions (the evaluated counter counts
            // the bipartitions either way)
            const uint32_t* MPDP_RESTRICT blist = d.use_bl ? a.lists + d.bl_base : nullptr;
            uint32_t acc = 0u, cliq = 0u, listed = 0u, paper = 0u;
            for (int j = 0; j < nb; j++) {
                const uint32_t b = s_blk[warp][j], p = block_pairs(b);
                uint32_t off = 0u, nl = 0u;
                s_bpref[warp][j] = acc;
                paper += p;
                if (is_clique(b, sq.adj)) {
                    cliq |= 1u << j;
                    acc += p;
                } else if (blist && __popc(b) > 2 && bl_find(blist, b, off, nl)) {
                    listed |= 1u << j;
                    s_loff[warp][j] = off;
                    acc += nl;
                } else {
                    acc += p;
                }
            }
            s_cliq[warp] = cliq;
            s_list[warp] = listed;
            s_bpref[warp][nb] = acc;
            s_nb[warp] = nb;
            if (chunk == 0u) {
                evaluated += paper;
                heavy++;
            }
        }
        __syncwarp();
        const int nb = s_nb[warp];
        const uint32_t* bpref = s_bpref[warp];
        const uint32_t* blk = s_blk[warp];
        const uint32_t total = bpref[nb];
        const uint32_t lo = (uint32_t)((unsigned long long)total * chunk / nch);
        const uint32_t hi = (uint32_t)((unsigned long long)total * (chunk + 1u) / nch);
        const uint32_t* MPDP_RESTRICT cw = conn_bitmap(a, qi);
        const uint32_t cliq = s_cliq[warp], listed = s_list[warp];
        const uint32_t* MPDP_RESTRICT lbs = d.use_bl ? a.lists + d.bl_base + kBlHead + kBlTab : nullptr;
        unsigned long long bx = kNoX;
        uint32_t bl = kFull;
        uint32_t stash = 0u;  // warp-uniform stash fill
        // Each lane takes a contiguous run of the chunk's pair indices: the
        // first one's lb by deposit, the next ones by stepping to the next
        // submask of the block, (sub - rest) & rest, in index order.
        const uint32_t per = (hi - lo + 31u) >> 5;
        uint32_t p = lo + (uint32_t)lane * per;
        const uint32_t pend = p + per < hi ? p + per : hi;
        int j = 0;
        while (j + 1 < nb && bpref[j + 1] <= p) j++;
        uint32_t b = blk[j], mn = b & (0u - b), rest = b ^ mn;
        bool lst = (listed >> j) & 1u;
        uint32_t sub = (p < pend && !lst) ? deposit(p - bpref[j], rest) : 0u;
        for (uint32_t round = 0; round < per; round++) {  // warp-uniform trip count
            bool valid = false;
            uint32_t lb = 0u, rb = 0u;
            if (p < pend) {
                if (lst) {  // a listed CCP
                    lb = MPDP_LDG(&lbs[s_loff[warp][j] + (p - bpref[j])]);
                    valid = true;
                } else {
                    lb = mn | sub;
                    valid = ((cliq >> j) & 1u) || (conn_of(lb, cw, sq.adj) && conn_of(b ^ lb, cw, sq.adj));
                    sub = (sub - rest) & rest;
                }
                rb = b ^ lb;
                p++;
                if (p < pend && p == bpref[j + 1]) {  // the next block's pairs
                    j++;
                    b = blk[j];
                    mn = b & (0u - b);
                    rest = b ^ mn;
                    sub = 0u;
                    lst = (listed >> j) & 1u;
                }
            }
            const unsigned bal = __ballot_sync(kFull, valid);
            ccp += (lane == 0) ? (unsigned long long)__popc(bal) : 0ull;
            if (!a.use_ccc) {
                if (valid) {
                    const uint32_t sl = left_side(s, lb, rb, sq.adj);
                    fold_pair(sl, s ^ sl, memo, cnt, bx, bl);
                }
                continue;
            }
            if (valid) {
                const uint32_t pos = stash + __popc(bal & ((1u << lane) - 1u));
                s_stash_l[warp][pos] = lb;
                s_stash_r[warp][pos] = rb;
            }
            stash += __popc(bal);
            __syncwarp();
            if (stash >= 32u) {
                const uint32_t i = stash - 32u + lane;
                const uint32_t l2 = s_stash_l[warp][i], r2 = s_stash_r[warp][i];
                const uint32_t sl = left_side(s, l2, r2, sq.adj);
                fold_pair(sl, s ^ sl, memo, cnt, bx, bl);
                stash -= 32u;
            }
            __syncwarp();
        }
        if (a.use_ccc && lane < (int)stash) {
            const uint32_t l2 = s_stash_l[warp][lane], r2 = s_stash_r[warp][lane];
            const uint32_t sl = left_side(s, l2, r2, sq.adj);
            fold_pair(sl, s ^ sl, memo, cnt, bx, bl);
        }
        warp_min_x(bx, bl);
        if (nch > 1u) {
            // leave this chunk's best, then count the arrival; the warp whose
            // arrival is the last folds every chunk's best
            uint32_t last = 0u;
            if (lane == 0) {
                if (chunk == 0u) {
                    hm[mi].x = bx;
                    hm[mi].left = bl;
                } else {
                    he[item - nmain].x = bx;
                    he[item - nmain].left = bl;
                }
                __threadfence();
                last = atomicAdd(&hm[mi].arrived, 1u) == nch - 1u;
                if (last) __threadfence();
            }
            if (!__shfl_sync(kFull, last, 0)) continue;
            bx = kNoX;
            bl = kFull;
            for (uint32_t c = (uint32_t)lane; c < nch; c += 32u) {
                unsigned long long cx;
                uint32_t cl;
                if (c == 0u) {
                    cx = __ldcg(&hm[mi].x);
                    cl = __ldcg(&hm[mi].left);
                } else {
                    cx = __ldcg(&he[ebase + c - 1u].x);
                    cl = __ldcg(&he[ebase + c - 1u].left);
                }
                if (better_x(cx, cl, bx, bl)) {
                    bx = cx;
                    bl = cl;
                }
            }
            warp_min_x(bx, bl);
        }
        if (lane == 0) {
            const double card_s = peel_card(s, s_pv[warp], sq, memo, cnt);
            memo.put(s, k, set_cost(bx, card_s), card_s, bl, cnt);
        }
        __syncwarp();
    }
    if (cur >= 0 && lane == 0) {
        if (ccp) atomicAdd(&a.out[cur].counters.ccp[k], ccp);
        if (evaluated) atomicAdd(&a.out[cur].counters.evaluated[k], evaluated);
        if (heavy) atomicAdd(&a.out[cur].counters.heavy, heavy);
    }
}

#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_heavy(BatchArgs a, int k, Memo memo)
{
    eval_heavy_body(a, k, memo, blockIdx.x, gridDim.x);
}
#endif

// ---------------------------------------------------------------------------
// a9: plan fetch (one warp per query).  From the full set, read (cost, card,
// left) from the memo and expand left and S \ left, one tree depth at a time
// with one lane per node of that depth; nodes end up in breadth-first order.
template <class Memo>
__device__ void extract_body(const BatchArgs& a, Memo memo, uint32_t bid, uint32_t nblk)
{
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    const int qi = bid, lane = threadIdx.x;
    memo.setup(s_memo);
    memo.bind(a, qi);
    __syncwarp();
    DevOut& o = a.out[qi];
    DevResult& res = o.result;
    DevCounters* cnt = &o.counters;
    const DevQuery* q = a.query + qi;
    const int n = a.desc[qi].n;
    if (cnt->status != 0 || n < 1) {
        if (lane == 0) {
            res.n_nodes = 0;
            res.cost = 0.0;
            res.status = cnt->status;
        }
        return;
    }
    const uint32_t full = (n == 32) ? kFull : ((1u << n) - 1u);
    if (lane == 0) res.nodes[0].set = full;
    __syncwarp();
    int lo = 0, hi = 1;  // current depth: nodes [lo, hi)
    bool bad = false;
    while (lo < hi) {
        int next = hi;
        for (int base = lo; base < hi; base += 32) {
            const int i = base + lane;
            bool internal = false;
            uint32_t s = 0u, l = 0u;
            double c = 0.0, card = 0.0;
            if (i < hi) {
                s = (uint32_t)res.nodes[i].set;
                internal = (s & (s - 1u)) != 0u;
                if (internal) {
                    memo.get(s, c, card, l, cnt);
                    if (l == 0u || (l & ~s) != 0u || l == s) {
                        bad = true;
                        internal = false;
                    }
                }
            }
            const unsigned bal = __ballot_sync(kFull, internal);
            const int pos = next + 2 * __popc(bal & ((1u << lane) - 1u));
            if (i < hi) {
                mpdp_plan_node& nd = res.nodes[i];
                nd.n_leaves = __popc(s);
                if (internal && pos + 1 < kPlanNodes) {
                    nd.left = pos;
                    nd.right = pos + 1;
                    nd.rel = -1;
                    nd.cost = c;
                    nd.card = card;
                    res.nodes[pos].set = l;
                    res.nodes[pos + 1].set = s ^ l;
                } else {
                    nd.left = nd.right = -1;
                    nd.rel = lowest(s);
                    nd.card = q->card[nd.rel];
                    nd.cost = 0.0;
                }
            }
            next += 2 * __popc(bal);
            __syncwarp();
        }
        lo = hi;
        hi = next;
        if (hi > kPlanNodes) {
            bad = true;
            break;
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) raise_status(cnt, MPDP_ERR_INTERNAL);
    __syncwarp();
    if (lane == 0) {
        res.n_nodes = hi;
        res.cost = res.nodes[0].cost;
        res.status = cnt->status;
    }
}

#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void __launch_bounds__(32) k_extract(BatchArgs a, Memo memo)
{
    extract_body(a, memo, blockIdx.x, gridDim.x);
}
#endif

// Memo read-back of arbitrary connected sets of one query (parity checks).
#ifndef MPDP_PHASES_ONLY
template <class Memo>
__global__ void k_memo_lookup(BatchArgs a, int qi, const uint32_t* MPDP_RESTRICT sets, int count,
                              double* MPDP_RESTRICT costs, uint32_t* MPDP_RESTRICT lefts, Memo memo)
{
    __shared__ __align__(16) char s_memo[Memo::kSharedBytes];
    memo.setup(s_memo);
    memo.bind(a, qi);
    __syncthreads();
    DevCounters* cnt = &a.out[qi].counters;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t s = sets[i];
        if ((s & (s - 1u)) == 0u) {
            costs[i] = 0.0;
            lefts[i] = 0u;
            continue;
        }
        double c, card;
        uint32_t l;
        memo.get(s, c, card, l, cnt);
        costs[i] = c;
        lefts[i] = l;
    }
}
#endif

// ---------------------------------------------------------------------------
// Host-side launch sequencing.

#ifndef MPDP_PHASES_ONLY
unsigned long long binom_host(int n, int k)
{
    if (k < 0 || k > n) return 0;
    unsigned long long r = 1;
    for (int x = 1; x <= k; x++) r = r * (unsigned long long)(n - k + x) / (unsigned long long)x;
    return r;
}

size_t list_entries(int n)
{
    unsigned long long off = 0;
    for (int k = 2; k <= n; k++) off += binom_host(n, k);
    return (size_t)off;
}

size_t conn_words(int n) { return n >= 5 ? (size_t)1 << (n - 5) : 1; }
size_t block_list_words(int n, int enumeration)
{
    return (enumeration == MPDP_ENUM_BLOCKS && n >= kBlMinRels) ? kBlWords : 0;
}
size_t fb_cache_words(int n, int enumeration)
{
    if (enumeration != MPDP_ENUM_BLOCKS) return 0;
    const unsigned long long c = binom_host(n, n / 2);
    return (size_t)(c < kFbCap ? c : kFbCap) * fb_stride(n);
}

size_t hash_arena_slots(int n)
{
    unsigned long long total = 0;
    for (int k = 2; k <= n; k++) {
        unsigned long long want = 2ull * binom_host(n, k), cap = 16;
        while (cap < want) cap <<= 1;
        total += cap;
    }
    return (size_t)total;
}

unsigned long long unfused_pair_records(const BatchPlan& bp)
{
    unsigned long long most = 0;
    for (int k = 2; k < kLevels; k++) {
        const unsigned long long r = bp.tree_tiles[k] * (unsigned long long)kEvalThreads * (unsigned long long)(k - 1);
        if (r > most) most = r;
    }
    return most;
}

void fill_levels(QDesc& d, int run, int filter_mode, uint32_t& filter_blocks)
{
    const int n = d.n;
    unsigned long long off = 0, wb = 0;
    for (int k = 0; k < kLevels; k++) d.list_off[k] = 0;
    for (int k = 0; k <= kLevels; k++) d.warp_begin[k] = 0;
    for (int k = 2; k <= n; k++) {
        const unsigned long long c = binom_host(n, k);
        d.list_off[k] = (uint32_t)off;
        off += c;
        d.warp_begin[k] = (uint32_t)wb;
        wb += (c + 32ull * run - 1) / (32ull * run);
    }
    for (int k = (n >= 2 ? n + 1 : 0); k <= kLevels; k++) d.warp_begin[k] = (uint32_t)wb;
    const unsigned warps_per_block = kFilterThreads / 32;
    if (filter_mode != MPDP_FILTER_UNRANK)
        filter_blocks = n >= 2 ? (uint32_t)(((1ull << n) + kBitmapsPerBlock - 1) / kBitmapsPerBlock) : 0u;
    else
        filter_blocks = (uint32_t)((wb + warps_per_block - 1) / warps_per_block);
}

struct HookScope {
    LaunchHook* h;
    int cls;
    cudaStream_t st;
    HookScope(LaunchHook* h_, int c, cudaStream_t s) : h(h_), cls(c), st(s)
    {
        if (h) h->begin(cls, st);
    }
    ~HookScope()
    {
        if (h) h->end(cls, st);
    }
};

template <class Memo>
struct BlockMemoOf {
    using type = Memo;
};
template <>
struct BlockMemoOf<DenseMemo> {
    using type = DensePlainMemo;
};
static inline HashMemo block_memo(const HashMemo& m) { return m; }
static inline DensePlainMemo block_memo(const DenseMemo& m) { return DensePlainMemo{m.cc0, m.left0, nullptr, nullptr}; }

template <class Memo>
static void launch_levels(const BatchArgs& a, const BatchPlan& bp, Memo memo, cudaStream_t st, int& launches,
                          LaunchHook* hook)
{
    // block-mode kernels: plain-bitmap entries (see DensePlainMemo)
    using BlockMemo = typename BlockMemoOf<Memo>::type;

    const int cap_blocks = bp.num_sms * bp.blocks_per_sm;
    bool any = false;  // levels to evaluate (k >= 2)
    for (int k = 2; k <= a.max_n; k++) any = any || bp.tree_tiles[k] != 0 || bp.block_tiles[k] != 0;
    if (any) {
        HookScope hs(hook, MPDP_KC_MEMO_INIT, st);
        k_level_prefix<<<2 * (a.max_n - 1), 256, 0, st>>>(a, bp.level_pref, bp.group_threads);
        launches++;
    }
    if (bp.block_lists) {  // block CCP lists, before the levels that read them
        HookScope hs(hook, MPDP_KC_EVAL, st);
        k_block_detect<<<cap_blocks, 256, 0, st>>>(a);
        k_block_list<<<cap_blocks, 256, 0, st>>>(a);
        launches += 2;
    }
    for (int k = 2; k <= a.max_n; k++) {
        const unsigned long long tree_tiles = bp.tree_tiles[k], block_tiles = bp.block_tiles[k];
        if (tree_tiles) {
            // enough blocks for a level evaluated by groups of lanes: up to
            // group_threads threads, at most 32 per set
            unsigned long long want = tree_tiles;
            if (!bp.pairs && bp.group_threads) {
                const unsigned long long groups = bp.group_threads / kEvalThreads;
                const unsigned long long most = tree_tiles * 32ull < groups ? tree_tiles * 32ull : groups;
                if (most > want) want = most;
            }
            const int grid = (int)(want < (unsigned long long)cap_blocks ? want : cap_blocks);
            if (bp.pairs) {
                {
                    HookScope hs(hook, MPDP_KC_EVAL, st);
                    k_eval_tree_pairs<Memo><<<grid, kEvalThreads, 0, st>>>(a, k, memo, bp.pairs);
                }
                HookScope hs(hook, MPDP_KC_EVAL, st);
                k_prune_tree<Memo><<<grid, kEvalThreads, 0, st>>>(a, k, memo, bp.pairs);
                launches += 2;
            } else {
                HookScope hs(hook, MPDP_KC_EVAL, st);
                k_eval_tree<Memo><<<grid, kEvalThreads, 0, st>>>(a, k, memo, bp.level_pref);
                launches++;
            }
        }
        if (block_tiles) {
            {
                HookScope hs(hook, MPDP_KC_EVAL, st);
                const int grid = (int)(block_tiles < (unsigned long long)cap_blocks ? block_tiles : cap_blocks);
                k_eval_blocks<BlockMemo><<<grid, kEvalThreads, 0, st>>>(a, k, block_memo(memo), bp.level_pref);
            }
            {
                HookScope hs(hook, MPDP_KC_HEAVY, st);
                const unsigned long long hs_max = bp.block_sets[k];
                const int grid = (int)(hs_max < (unsigned long long)cap_blocks ? hs_max : cap_blocks);
                k_eval_heavy<BlockMemo><<<grid > 0 ? grid : 1, kEvalThreads, 0, st>>>(a, k, block_memo(memo));
            }
            launches += 2;
        }
    }
    HookScope hs(hook, MPDP_KC_EXTRACT, st);
    k_extract<Memo><<<a.nq, 32, 0, st>>>(a, memo);
    launches++;
}

cudaError_t enqueue_pipeline(const BatchArgs& a, const BatchPlan& bp, int memo_kind, cudaStream_t st,
                             int* launches_out, LaunchHook* hook)
{
    int launches = 0;
    const bool dense = memo_kind == MPDP_MEMO_DENSE;
    {
        HookScope hs(hook, MPDP_KC_INGEST, st);
        k_ingest<<<a.nq, 256, 0, st>>>(a, dense ? 1 : 0);
    }
    launches++;
    if (bp.connected_blocks > 0) {
        HookScope hs(hook, MPDP_KC_FILTER, st);
        k_filter_connected<<<bp.connected_blocks, kFilterThreads, 0, st>>>(a);
        launches++;
    }
    if (bp.filter_blocks > 0) {
        HookScope hs(hook, MPDP_KC_FILTER, st);
        if (a.filter_mode == MPDP_FILTER_UNRANK) {
            k_filter<<<bp.filter_blocks, kFilterThreads, 0, st>>>(a);
            launches++;
        } else {
            k_filter_bitmaps<<<bp.filter_blocks, kFilterThreads, 0, st>>>(a);
            launches++;
        }
    }
    if (dense) {
        DenseMemo memo{a.memo, a.left, nullptr, nullptr};
        launch_levels(a, bp, memo, st, launches, hook);
    } else {
        {
            HookScope hs(hook, MPDP_KC_MEMO_INIT, st);
            k_hash_layout<<<1, 1, 0, st>>>(a);
            k_hash_clear<<<bp.num_sms * 4, 256, 0, st>>>(a);
        }
        launches += 2;
        HashMemo memo{a.arena, nullptr};
        launch_levels(a, bp, memo, st, launches, hook);
    }
    if (launches_out) *launches_out = launches;
    return cudaGetLastError();
}

cudaError_t enqueue_structure(const BatchArgs& a, const BatchPlan& bp, cudaStream_t st)
{
    k_ingest<<<a.nq, 256, 0, st>>>(a, 0);
    if (bp.filter_blocks > 0) k_filter_bitmaps<<<bp.filter_blocks, kFilterThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t enqueue_stage_device(const BatchArgs& a, const double* card, const mpdp_edge* edges, cudaStream_t st,
                                 LaunchHook* hook)
{
    HookScope hs(hook, MPDP_KC_STAGE, st);
    k_stage<<<a.nq, 256, 0, st>>>(a, card, edges);
    return cudaGetLastError();
}

cudaError_t enqueue_publish(const BatchArgs& a, mpdp_plan_node* nodes, double* cost, int32_t* status,
                            cudaStream_t st, LaunchHook* hook)
{
    HookScope hs(hook, MPDP_KC_PUBLISH, st);
    k_publish<<<a.nq, 64, 0, st>>>(a, nodes, cost, status);
    return cudaGetLastError();
}

cudaError_t enqueue_memo_lookup(const BatchArgs& a, int memo_kind, int qi, const uint32_t* d_sets, int count,
                                double* d_costs, uint32_t* d_lefts, cudaStream_t st)
{
    const int grid = (count + 255) / 256 > 0 ? (count + 255) / 256 : 1;
    if (memo_kind == MPDP_MEMO_DENSE) {
        DenseMemo memo{a.memo, a.left, nullptr, nullptr};
        k_memo_lookup<DenseMemo><<<grid, 256, 0, st>>>(a, qi, d_sets, count, d_costs, d_lefts, memo);
    } else {
        HashMemo memo{a.arena, nullptr};
        k_memo_lookup<HashMemo><<<grid, 256, 0, st>>>(a, qi, d_sets, count, d_costs, d_lefts, memo);
    }
    return cudaGetLastError();
}

// The tree evaluate's memo reads are mostly L1 and L2 hits; a carveout of
// about a third of the SM's unified L1/shared memory for shared memory still
// fits 8 blocks' 8 KB each and leaves the rest to the L1 (measured on the
// 64-query snowflake-25 batch: 0.767 against 0.79 ms per batch with the
// default; 0 % or 100 % cost occupancy or L1 and run 2-3x slower).
cudaError_t configure_kernels()
{
    constexpr int kTreeCarveout = 32;  // percent of the maximum shared memory
    cudaError_t e = cudaFuncSetAttribute(k_eval_tree<DenseMemo>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         kTreeCarveout);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_eval_tree<HashMemo>, cudaFuncAttributePreferredSharedMemoryCarveout, kTreeCarveout);
    return e;
}

#endif  // MPDP_PHASES_ONLY

}  // namespace mpdp
