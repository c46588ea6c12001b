// MPDP kernels for sm_103a.
//
// One query runs as: ingest -> unrank+filter (all levels, one launch) ->
// [hash layout + clear] -> evaluate level 2 .. n (one launch per level, plus
// the block-per-set launch in block mode) -> plan fetch.  Level k's launch
// only reads memo entries of levels < k, so launches are the level barrier
// of the DP (Sec. 2.1.1; Sec. 5, Algorithm "MPDP on GPU").
#include <cuda_runtime.h>

#include <cstdio>

#include "mpdp_device.cuh"
#include "mpdp_launch.h"

namespace mpdp {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// a0: ingest.  Builds adjacency bitmaps and the selectivity matrix from the
// staged edge list, validates every value, checks that the whole join graph
// is connected, zeroes the counters and writes the implicit base entries
// cost({R_i}) = 0 of the dense memo (Algorithm "MPDP on GPU", memo fill).
__global__ void __launch_bounds__(256) k_ingest(const StagedQuery* __restrict__ st,
                                                DevQuery* __restrict__ q,
                                                DevCounters* __restrict__ cnt,
                                                double* __restrict__ dcost,
                                                uint32_t* __restrict__ dleft, int dense)
{
    const int tid = threadIdx.x;
    int* cw = reinterpret_cast<int*>(cnt);
    for (int i = tid; i < (int)(sizeof(DevCounters) / sizeof(int)); i += blockDim.x) cw[i] = 0;
    const int n = st->n;
    const int m = st->n_edges;
    for (int i = tid; i < kMaxRels * kMaxRels; i += blockDim.x) q->sel[i] = 1.0;
    if (tid < kMaxRels) {
        q->adj[tid] = 0u;
        q->card[tid] = (tid < n) ? st->card[tid] : 1.0;
    }
    __syncthreads();
    if (tid != 0) return;
    int status = 0;
    if (n < 1 || n > MPDP_MAX_EXACT_RELS) status = MPDP_ERR_TOO_LARGE;
    else if (m < 0 || m > kMaxEdges || st->cost_model != MPDP_COST_COUT) status = MPDP_ERR_INVALID_ARG;
    if (status == 0) {
        for (int i = 0; i < n; i++) {
            double c = st->card[i];
            if (!(c > 0.0) || !(c <= 1.7976931348623157e308)) status = MPDP_ERR_INVALID_ARG;
        }
    }
    uint32_t adj[kMaxRels];
    for (int i = 0; i < kMaxRels; i++) adj[i] = 0u;
    for (int e = 0; e < m && status == 0; e++) {
        int u = st->edges[e].u, v = st->edges[e].v;
        double s = st->edges[e].sel;
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(s > 0.0) || !(s <= 1.0) ||
            (adj[u] >> v & 1u)) {
            status = MPDP_ERR_INVALID_ARG;
            break;
        }
        adj[u] |= 1u << v;
        adj[v] |= 1u << u;
        q->sel[u * kMaxRels + v] = s;
        q->sel[v * kMaxRels + u] = s;
    }
    if (status == 0) {
        uint32_t full = (n == 32) ? kFull : ((1u << n) - 1u);
        if (grow(1u, full, adj) != full) status = MPDP_ERR_DISCONNECTED;
    }
    for (int i = 0; i < kMaxRels; i++) q->adj[i] = adj[i];
    q->n = n;
    q->n_edges = m;
    cnt->status = status;
    if (dense && status == 0) {
        for (int i = 0; i < n; i++) {
            dcost[1u << i] = 0.0;
            dleft[1u << i] = 0u;
        }
    }
}

// Device-path staging: gather caller device buffers into the staged query.
__global__ void k_stage(const double* __restrict__ card, const mpdp_edge* __restrict__ edges,
                        int n, int m, int cost_model, StagedQuery* __restrict__ st)
{
    int tid = threadIdx.x;
    if (tid == 0) {
        st->n = n;
        st->n_edges = m;
        st->cost_model = cost_model;
    }
    for (int i = tid; i < n && i < kMaxRels; i += blockDim.x) st->card[i] = card[i];
    for (int e = tid; e < m && e < kMaxEdges; e += blockDim.x) st->edges[e] = edges[e];
}

// Device-path outputs: copy plan, cost and status to caller device buffers.
__global__ void k_publish(const DevResult* __restrict__ res, const DevCounters* __restrict__ cnt,
                          mpdp_plan_node* __restrict__ nodes, double* __restrict__ cost,
                          int32_t* __restrict__ status)
{
    int n_nodes = res->n_nodes;
    for (int i = threadIdx.x; i < n_nodes; i += blockDim.x) nodes[i] = res->nodes[i];
    if (threadIdx.x == 0) {
        *cost = res->cost;
        *status = cnt->status;
    }
}

// ---------------------------------------------------------------------------
// Binomial coefficient C(i, j) for i, j <= 32 (exact in 64-bit arithmetic).
__device__ __forceinline__ uint32_t binom_dev(int i, int j)
{
    if (j < 0 || j > i) return 0u;
    unsigned long long r = 1;
    for (int x = 1; x <= j; x++) r = r * (unsigned long long)(i - j + x) / (unsigned long long)x;
    return (uint32_t)r;
}

// Combinatorial number system (colex order): the k-subset of {0..n-1} with
// rank r is {c_k > ... > c_1} where r = sum_i C(c_i, i); each c_i is the
// largest value with C(c_i, i) <= what remains of r.
__device__ __forceinline__ uint32_t unrank_colex(uint32_t r, int k, int n,
                                                 const uint32_t* __restrict__ binom)
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
    uint32_t t = s | (s - 1u);
    return (t + 1u) | (((~t & (0u - ~t)) - 1u) >> __ffs(s));
}

// ---------------------------------------------------------------------------
// a2 + a3: unrank every k-subset of every level and keep the connected ones.
// Warps are assigned to one level each; lane l of a warp takes the run of
// `run` consecutive ranks starting at warp_base + l * run, unranks its first
// set and steps with next_colex.  Pass 1 tests connectivity and keeps one
// flag bit per rank; a warp scan places every lane's connected sets, one
// atomic per warp reserves room in the level's list, and pass 2 replays the
// run writing the kept sets: each warp's output is a colex-ordered slice.
__global__ void __launch_bounds__(256) k_filter(FilterParams p, const DevQuery* __restrict__ q,
                                                DevCounters* __restrict__ cnt,
                                                uint32_t* __restrict__ lists)
{
    __shared__ uint32_t s_binom[33 * 33];
    __shared__ uint32_t s_adj[kMaxRels];
    for (int t = threadIdx.x; t < 33 * 33; t += blockDim.x) s_binom[t] = binom_dev(t / 33, t % 33);
    if (threadIdx.x < kMaxRels) s_adj[threadIdx.x] = q->adj[threadIdx.x];
    __syncthreads();
    if (cnt->status != 0) return;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    int k = -1;
    for (int j = 2; j <= p.n; j++)
        if (warp >= p.warp_begin[j] && warp < p.warp_begin[j + 1]) k = j;
    if (k < 0) return;  // whole warp: past the last level
    const uint32_t nr = p.nranks[k];
    const unsigned long long r0 =
        (unsigned long long)(warp - p.warp_begin[k]) * 32ull * (unsigned long long)p.run +
        (unsigned long long)lane * (unsigned long long)p.run;
    uint32_t len = 0;
    if (r0 < nr) len = (uint32_t)min((unsigned long long)p.run, (unsigned long long)nr - r0);
    const uint32_t s0 = len ? unrank_colex((uint32_t)r0, k, p.n, s_binom) : 0u;
    uint32_t s = s0, flags = 0u, steps = 0u;
    for (uint32_t i = 0; i < len; i++) {
        // connected(S), counting the vertices expanded
        uint32_t seen = s & (0u - s), frontier = seen;
        while (frontier) {
            const int x = lowest(frontier);
            frontier &= frontier - 1u;
            steps++;
            const uint32_t nb = s_adj[x] & s & ~seen;
            seen |= nb;
            frontier |= nb;
            if (seen == s) break;
        }
        if (seen == s) flags |= 1u << i;
        s = next_colex(s);
    }
    const uint32_t c = __popc(flags);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(&cnt->list_count[k], total);
    base = __shfl_sync(kFull, base, 0);
    uint32_t* out = lists + p.list_off[k] + base + (incl - c);
    s = s0;
    uint32_t w = 0;
    for (uint32_t i = 0; i < len; i++) {
        if (flags >> i & 1u) out[w++] = s;
        s = next_colex(s);
    }
    uint32_t done = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        done += __shfl_xor_sync(kFull, done, o);
        steps += __shfl_xor_sync(kFull, steps, o);
    }
    if (lane == 0 && done) {
        atomicAdd(&cnt->unranked, (unsigned long long)done);
        atomicAdd(&cnt->filter_steps, (unsigned long long)steps);
    }
}

// ---------------------------------------------------------------------------
// Hash memo layout: per level k, capacity = the power of two >= 2x the level's
// connected count (at least 16), carved from one arena.
__global__ void k_hash_layout(int n, DevCounters* __restrict__ cnt, HashLayout* __restrict__ lay,
                              unsigned long long arena_slots)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long base = 0;
    for (int k = 0; k < kLevels; k++) {
        lay->base[k] = 0;
        lay->mask[k] = 0;
    }
    for (int k = 2; k <= n; k++) {
        unsigned long long want = 2ull * cnt->list_count[k];
        unsigned long long cap = 16;
        while (cap < want) cap <<= 1;
        lay->base[k] = base;
        lay->mask[k] = (unsigned int)(cap - 1);
        base += cap;
    }
    lay->total_slots = base;
    cnt->memo_slots = base;
    if (base > arena_slots) raise_status(cnt, MPDP_ERR_OOM);
}

__global__ void __launch_bounds__(256) k_hash_clear(const HashLayout* __restrict__ lay,
                                                    const DevCounters* __restrict__ cnt,
                                                    HashSlot* __restrict__ arena)
{
    if (cnt->status != 0) return;
    const unsigned long long total = lay->total_slots;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x)
        reinterpret_cast<uint4*>(arena)[i] = z;
}

// ---------------------------------------------------------------------------
// Shared-memory copy of the query for the evaluate kernels.
struct SharedQuery {
    uint32_t adj[kMaxRels];
    double card[kMaxRels];
    double sel[kMaxRels * kMaxRels];
};

__device__ __forceinline__ void load_query(SharedQuery& sq, const DevQuery* __restrict__ q)
{
    for (int i = threadIdx.x; i < kMaxRels * kMaxRels; i += blockDim.x) sq.sel[i] = q->sel[i];
    if (threadIdx.x < kMaxRels) {
        sq.adj[threadIdx.x] = q->adj[threadIdx.x];
        sq.card[threadIdx.x] = q->card[threadIdx.x];
    }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Cost one CCP pair (S_l, S_r) of S and fold it into the running best.
// Singleton sides cost 0 (C_out base case) and need no memo read.
template <class Memo>
__device__ __forceinline__ void cost_pair(uint32_t sl, uint32_t sr, double card_s, const Memo& memo,
                                          DevCounters* cnt, double& bc, uint32_t& bl)
{
    double cl = (sl & (sl - 1u)) ? memo.get_cost(sl, cnt) : 0.0;
    double cr = (sr & (sr - 1u)) ? memo.get_cost(sr, cnt) : 0.0;
    double c = __dadd_rn(__dadd_rn(cl, cr), card_s);
    uint32_t l = sl < sr ? sl : sr;
    if (better(c, l, bc, bl)) {
        bc = c;
        bl = l;
    }
}

// ---------------------------------------------------------------------------
// a4-a8, tree join graphs (Algorithm 2, MPDP:Tree).  One thread per connected
// set S of level k.  Every connected S induces a tree; its CCP pairs are the
// k-1 splits made by removing one edge of G[S].  A search from min(S) finds
// each tree edge (x, v) once, with v on the far side from the root; the split
// is S_l = grow({v}, S \ {x}) (the subtree under v), S_r = S \ S_l.  The best
// (cost, left) over the k-1 splits is written to the memo: evaluate, prune and
// scatter fused in one pass, one memo write per set.
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_tree(int k, uint32_t list_off,
                                                            const DevQuery* __restrict__ q,
                                                            DevCounters* __restrict__ cnt,
                                                            const uint32_t* __restrict__ lists,
                                                            Memo memo)
{
    __shared__ SharedQuery sq;
    __shared__ __align__(16) char s_memo[HashMemo::kSharedBytes];
    load_query(sq, q);
    memo.setup(s_memo);
    __syncthreads();
    if (cnt->status != 0) return;
    const uint32_t count = cnt->list_count[k];
    const uint32_t* list = lists + list_off;
    unsigned long long sets = 0;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count;
         idx += gridDim.x * blockDim.x) {
        const uint32_t s = list[idx];
        const double card_s = card_of(s, sq.adj, sq.card, sq.sel);
        double bc = __longlong_as_double(0x7ff0000000000000ll);  // +inf
        uint32_t bl = kFull;
        uint32_t vis = s & (0u - s), queue = vis;
        while (queue) {
            const int x = lowest(queue);
            queue &= queue - 1u;
            uint32_t ch = sq.adj[x] & s & ~vis;
            vis |= ch;
            queue |= ch;
            const uint32_t rest = s & ~(1u << x);
            while (ch) {
                const int v = lowest(ch);
                ch &= ch - 1u;
                const uint32_t sl = grow(1u << v, rest, sq.adj);
                cost_pair(sl, s ^ sl, card_s, memo, cnt, bc, bl);
            }
        }
        memo.put(s, k, bc, bl, cnt);
        sets++;
    }
    sets = warp_sum(sets);
    if ((threadIdx.x & 31) == 0 && sets) {
        atomicAdd(&cnt->evaluated[k], sets * (unsigned long long)(k - 1));
        atomicAdd(&cnt->ccp[k], sets * (unsigned long long)(k - 1));
    }
}

// ---------------------------------------------------------------------------
// Find-Blocks (Sec. 3.2.2; Algorithm 4): the blocks of G[S] as bitmaps.
// A search from min(S) gives a spanning tree (parent of each vertex; anc[v] =
// the tree edges on the path root..v, each edge named by its child vertex).
// Every non-tree edge (x, y) closes the fundamental cycle whose tree edges are
// anc[x] xor anc[y].  Two tree edges lie in one block exactly when a chain of
// fundamental cycles sharing tree edges joins them, so merging overlapping
// cycle edge-sets gives one class per block with a cycle; its vertices are
// the class's child vertices plus their parents.  A tree edge on no cycle is
// a bridge, a block of its own two vertices.  Returns the number of blocks.
__device__ __forceinline__ int find_blocks(uint32_t s, const uint32_t* __restrict__ adj,
                                           uint32_t* __restrict__ blk)
{
    uint8_t par[kMaxRels];
    uint32_t anc[kMaxRels];
    const int root = lowest(s);
    par[root] = 0xff;
    anc[root] = 0u;
    uint32_t vis = 1u << root, queue = vis;
    while (queue) {
        const int x = lowest(queue);
        queue &= queue - 1u;
        uint32_t ch = adj[x] & s & ~vis;
        vis |= ch;
        queue |= ch;
        while (ch) {
            const int v = lowest(ch);
            ch &= ch - 1u;
            par[v] = (uint8_t)x;
            anc[v] = anc[x] | (1u << v);
        }
    }
    uint32_t cls[kMaxRels];
    int nc = 0;
    uint32_t t = s;
    while (t) {
        const int x = lowest(t);
        t &= t - 1u;
        uint32_t ys = adj[x] & s & ~((2u << x) - 1u);  // neighbours y > x
        while (ys) {
            const int y = lowest(ys);
            ys &= ys - 1u;
            if (par[y] == x || par[x] == y) continue;  // tree edge
            uint32_t c = anc[x] ^ anc[y];
            int j = 0;
            while (j < nc) {
                if (cls[j] & c) {
                    c |= cls[j];
                    cls[j] = cls[--nc];
                } else {
                    j++;
                }
            }
            cls[nc++] = c;
        }
    }
    int nb = 0;
    uint32_t in_cycle = 0u;
    for (int j = 0; j < nc; j++) {
        uint32_t c = cls[j], b = c;
        in_cycle |= c;
        while (c) {
            const int v = lowest(c);
            c &= c - 1u;
            b |= 1u << par[v];
        }
        blk[nb++] = b;
    }
    uint32_t br = s & ~in_cycle & ~(1u << root);
    while (br) {
        const int v = lowest(br);
        br &= br - 1u;
        blk[nb++] = (1u << v) | (1u << par[v]);
    }
    return nb;
}

// Unordered bipartitions of a block B visited by the enumeration: every lb
// holding min(B), except lb = B: 2^(|B|-1) - 1.
__device__ __forceinline__ uint32_t block_pairs(uint32_t b) { return (1u << (__popc(b) - 1)) - 1u; }

// Deposit the low bits of t into the set bits of mask, lowest first.
__device__ __forceinline__ uint32_t deposit(uint32_t t, uint32_t mask)
{
    uint32_t r = 0u;
    while (t && mask) {
        const uint32_t low = mask & (0u - mask);
        if (t & 1u) r |= low;
        t >>= 1;
        mask ^= low;
    }
    return r;
}

// ---------------------------------------------------------------------------
// a4-a8, general join graphs (Algorithm 4), thread per set for light sets.
// For each block B of G[S] and each lb (min(B) in lb, lb != B): rb = B \ lb;
// the CCP block keeps the pair when lb and rb both induce connected subgraphs
// (they are adjacent since B is connected); then S_l = grow(lb, S \ rb),
// S_r = S \ S_l.  Sets whose pair count exceeds heavy_threshold go to the
// block-per-set kernel instead.
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_blocks(int k, uint32_t list_off,
                                                              uint32_t heavy_threshold,
                                                              const DevQuery* __restrict__ q,
                                                              DevCounters* __restrict__ cnt,
                                                              const uint32_t* __restrict__ lists,
                                                              uint32_t* __restrict__ heavy, Memo memo)
{
    __shared__ SharedQuery sq;
    __shared__ __align__(16) char s_memo[HashMemo::kSharedBytes];
    load_query(sq, q);
    memo.setup(s_memo);
    __syncthreads();
    if (cnt->status != 0) return;
    const uint32_t count = cnt->list_count[k];
    const uint32_t* list = lists + list_off;
    unsigned long long evaluated = 0, ccp = 0;
    const uint32_t iters = (count + gridDim.x * blockDim.x - 1) / (gridDim.x * blockDim.x);
    for (uint32_t it = 0; it < iters; it++) {
        const uint32_t idx = it * gridDim.x * blockDim.x + blockIdx.x * blockDim.x + threadIdx.x;
        bool to_heavy = false;
        uint32_t s = 0u;
        if (idx < count) {
            s = list[idx];
            uint32_t blk[kMaxRels];
            const int nb = find_blocks(s, sq.adj, blk);
            uint32_t pairs = 0u;
            for (int j = 0; j < nb; j++) pairs += block_pairs(blk[j]);
            if (pairs > heavy_threshold) {
                to_heavy = true;
            } else {
                const double card_s = card_of(s, sq.adj, sq.card, sq.sel);
                double bc = __longlong_as_double(0x7ff0000000000000ll);
                uint32_t bl = kFull;
                evaluated += pairs;
                for (int j = 0; j < nb; j++) {
                    const uint32_t b = blk[j];
                    const uint32_t mn = b & (0u - b), rest = b ^ mn;
                    for (uint32_t sub = 0u; sub != rest; sub = (sub - rest) & rest) {
                        const uint32_t lb = mn | sub, rb = b ^ lb;
                        if (!connected(lb, sq.adj) || !connected(rb, sq.adj)) continue;
                        ccp++;
                        const uint32_t sl = grow(lb, s & ~rb, sq.adj);
                        cost_pair(sl, s ^ sl, card_s, memo, cnt, bc, bl);
                    }
                }
                memo.put(s, k, bc, bl, cnt);
            }
        }
        // warp-aggregated append of heavy sets
        const unsigned bal = __ballot_sync(kFull, to_heavy);
        if (bal) {
            const int lane = threadIdx.x & 31;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&cnt->heavy_count[k], (uint32_t)__popc(bal));
            base = __shfl_sync(kFull, base, 0);
            if (to_heavy) heavy[list_off + base + __popc(bal & ((1u << lane) - 1u))] = s;
        }
    }
    evaluated = warp_sum(evaluated);
    ccp = warp_sum(ccp);
    if ((threadIdx.x & 31) == 0) {
        if (evaluated) atomicAdd(&cnt->evaluated[k], evaluated);
        if (ccp) atomicAdd(&cnt->ccp[k], ccp);
    }
}

// Block-per-set evaluation of heavy sets (general mode).  Thread 0 finds the
// blocks; the block's threads split the set's pair index space.  With
// Collaborative Context Collection (Sec. 5, "Avoiding 'If' branch
// divergence") each warp stashes the pairs that pass the CCP block in shared
// memory and grows/costs them only when 32 are ready, so no lane idles on an
// invalid pair during the expensive part.
template <class Memo>
__global__ void __launch_bounds__(kEvalThreads) k_eval_heavy(int k, uint32_t list_off, int use_ccc,
                                                             const DevQuery* __restrict__ q,
                                                             DevCounters* __restrict__ cnt,
                                                             const uint32_t* __restrict__ heavy,
                                                             Memo memo)
{
    constexpr int kWarps = kEvalThreads / 32;
    __shared__ SharedQuery sq;
    __shared__ __align__(16) char s_memo[HashMemo::kSharedBytes];
    __shared__ uint32_t s_blk[kMaxRels];
    __shared__ uint32_t s_pref[kMaxRels + 1];
    __shared__ int s_nb;
    __shared__ double s_card;
    __shared__ uint32_t s_stash_l[kWarps][64];
    __shared__ uint32_t s_stash_r[kWarps][64];
    __shared__ double s_bc[kWarps];
    __shared__ uint32_t s_bl[kWarps];
    load_query(sq, q);
    memo.setup(s_memo);
    __syncthreads();
    if (cnt->status != 0) return;
    const uint32_t count = cnt->heavy_count[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long ccp = 0, evaluated = 0;
    for (uint32_t h = blockIdx.x; h < count; h += gridDim.x) {
        const uint32_t s = heavy[list_off + h];
        if (threadIdx.x == 0) {
            uint32_t blk[kMaxRels];
            const int nb = find_blocks(s, sq.adj, blk);
            uint32_t acc = 0u;
            for (int j = 0; j < nb; j++) {
                s_blk[j] = blk[j];
                s_pref[j] = acc;
                acc += block_pairs(blk[j]);
            }
            s_pref[nb] = acc;
            s_nb = nb;
            s_card = card_of(s, sq.adj, sq.card, sq.sel);
            evaluated += acc;
        }
        __syncthreads();
        const int nb = s_nb;
        const uint32_t total = s_pref[nb];
        const double card_s = s_card;
        double bc = __longlong_as_double(0x7ff0000000000000ll);
        uint32_t bl = kFull;
        uint32_t stash = 0u;  // warp-uniform stash fill
        const uint32_t rounds = (total + blockDim.x - 1) / blockDim.x;
        for (uint32_t rd = 0; rd < rounds; rd++) {
            const uint32_t p = rd * blockDim.x + threadIdx.x;
            bool valid = false;
            uint32_t lb = 0u, rb = 0u;
            if (p < total) {
                int j = 0;
                while (j + 1 < nb && s_pref[j + 1] <= p) j++;
                const uint32_t b = s_blk[j];
                const uint32_t mn = b & (0u - b);
                lb = mn | deposit(p - s_pref[j], b ^ mn);
                rb = b ^ lb;
                valid = connected(lb, sq.adj) && connected(rb, sq.adj);
            }
            const unsigned bal = __ballot_sync(kFull, valid);
            ccp += (lane == 0) ? (unsigned long long)__popc(bal) : 0ull;
            if (!use_ccc) {
                if (valid) {
                    const uint32_t sl = grow(lb, s & ~rb, sq.adj);
                    cost_pair(sl, s ^ sl, card_s, memo, cnt, bc, bl);
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
                const uint32_t sl = grow(l2, s & ~r2, sq.adj);
                cost_pair(sl, s ^ sl, card_s, memo, cnt, bc, bl);
                stash -= 32u;
            }
            __syncwarp();
        }
        if (use_ccc && lane < (int)stash) {
            const uint32_t l2 = s_stash_l[warp][lane], r2 = s_stash_r[warp][lane];
            const uint32_t sl = grow(l2, s & ~r2, sq.adj);
            cost_pair(sl, s ^ sl, card_s, memo, cnt, bc, bl);
        }
        // prune: warp then block lexicographic min of (cost, left)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double oc = __shfl_xor_sync(kFull, bc, o);
            const uint32_t ol = __shfl_xor_sync(kFull, bl, o);
            if (better(oc, ol, bc, bl)) {
                bc = oc;
                bl = ol;
            }
        }
        if (lane == 0) {
            s_bc[warp] = bc;
            s_bl[warp] = bl;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kWarps; w++)
                if (better(s_bc[w], s_bl[w], bc, bl)) {
                    bc = s_bc[w];
                    bl = s_bl[w];
                }
            memo.put(s, k, bc, bl, cnt);
        }
        __syncthreads();
    }
    if (lane == 0 && ccp) atomicAdd(&cnt->ccp[k], ccp);
    if (threadIdx.x == 0) {
        if (evaluated) atomicAdd(&cnt->evaluated[k], evaluated);
        if (count && blockIdx.x == 0) atomicAdd(&cnt->heavy, (unsigned long long)count);
    }
}

// ---------------------------------------------------------------------------
// a9: plan fetch.  From the full set, read (cost, left) from the memo and
// expand left and S \ left, breadth first; leaves are single relations.
template <class Memo>
__global__ void k_extract(const DevQuery* __restrict__ q, DevCounters* __restrict__ cnt,
                          DevResult* __restrict__ res, Memo memo)
{
    __shared__ __align__(16) char s_memo[HashMemo::kSharedBytes];
    memo.setup(s_memo);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int n = q->n;
    res->n_nodes = 0;
    res->cost = 0.0;
    if (cnt->status != 0 || n < 1) {
        res->status = cnt->status;
        return;
    }
    const uint32_t full = (n == 32) ? kFull : ((1u << n) - 1u);
    int m = 1;
    res->nodes[0].set = full;
    for (int i = 0; i < m; i++) {
        mpdp_plan_node& nd = res->nodes[i];
        const uint32_t s = (uint32_t)nd.set;
        nd.n_leaves = __popc(s);
        if ((s & (s - 1u)) == 0u) {
            nd.left = nd.right = -1;
            nd.rel = lowest(s);
            nd.card = q->card[nd.rel];
            nd.cost = 0.0;
            continue;
        }
        double c;
        uint32_t l;
        memo.get(s, c, l, cnt);
        if (l == 0u || (l & ~s) != 0u || l == s || m + 2 > 2 * kMaxRels - 1) {
            raise_status(cnt, MPDP_ERR_INTERNAL);
            break;
        }
        nd.rel = -1;
        nd.cost = c;
        nd.card = card_of(s, q->adj, q->card, q->sel);
        nd.left = m;
        res->nodes[m].set = l;
        nd.right = m + 1;
        res->nodes[m + 1].set = s ^ l;
        m += 2;
    }
    res->n_nodes = m;
    res->cost = res->nodes[0].cost;
    res->status = cnt->status;
}

// Memo read-back of arbitrary connected sets (parity checks).
template <class Memo>
__global__ void k_memo_lookup(const uint32_t* __restrict__ sets, int count, double* __restrict__ costs,
                              uint32_t* __restrict__ lefts, DevCounters* __restrict__ cnt, Memo memo)
{
    __shared__ __align__(16) char s_memo[HashMemo::kSharedBytes];
    memo.setup(s_memo);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t s = sets[i];
        if ((s & (s - 1u)) == 0u) {
            costs[i] = 0.0;
            lefts[i] = 0u;
            continue;
        }
        double c;
        uint32_t l;
        memo.get(s, c, l, cnt);
        costs[i] = c;
        lefts[i] = l;
    }
}

// ---------------------------------------------------------------------------
// Host-side launch sequencing.

static unsigned long long binom_host(int n, int k)
{
    if (k < 0 || k > n) return 0;
    unsigned long long r = 1;
    for (int x = 1; x <= k; x++) r = r * (unsigned long long)(n - k + x) / (unsigned long long)x;
    return r;
}

void level_layout(int n, uint32_t* list_off /* [kLevels] */)
{
    unsigned long long off = 0;
    for (int k = 0; k < kLevels; k++) list_off[k] = 0;
    for (int k = 2; k <= n; k++) {
        list_off[k] = (uint32_t)off;
        off += binom_host(n, k);
    }
}

size_t list_entries(int n)
{
    unsigned long long off = 0;
    for (int k = 2; k <= n; k++) off += binom_host(n, k);
    return (size_t)(off ? off : 1);
}

size_t hash_arena_slots(int n)
{
    unsigned long long total = 0;
    for (int k = 2; k <= n; k++) {
        unsigned long long want = 2ull * binom_host(n, k), cap = 16;
        while (cap < want) cap <<= 1;
        total += cap;
    }
    return (size_t)(total ? total : 16);
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
static void launch_levels(const Workspace& ws, const PipelineCfg& pc, const uint32_t* list_off,
                          Memo memo, cudaStream_t st, int& launches, LaunchHook* hook)
{
    const int n = pc.n;
    const int cap_blocks = pc.num_sms * pc.blocks_per_sm;
    for (int k = 2; k <= n; k++) {
        const unsigned long long c = binom_host(n, k);
        int grid = (int)((c + kEvalThreads - 1) / kEvalThreads);
        if (grid > cap_blocks) grid = cap_blocks;
        if (grid < 1) grid = 1;
        if (pc.enumeration == MPDP_ENUM_TREE) {
            HookScope hs(hook, MPDP_KC_EVAL, st);
            k_eval_tree<Memo><<<grid, kEvalThreads, 0, st>>>(k, list_off[k], ws.query, ws.counters,
                                                             ws.lists, memo);
            launches++;
        } else {
            {
                HookScope hs(hook, MPDP_KC_EVAL, st);
                k_eval_blocks<Memo><<<grid, kEvalThreads, 0, st>>>(
                    k, list_off[k], (uint32_t)pc.heavy_threshold, ws.query, ws.counters, ws.lists,
                    ws.heavy, memo);
            }
            int hgrid = (int)(c < (unsigned long long)cap_blocks ? c : (unsigned long long)cap_blocks);
            if (hgrid < 1) hgrid = 1;
            {
                HookScope hs(hook, MPDP_KC_HEAVY, st);
                k_eval_heavy<Memo><<<hgrid, kEvalThreads, 0, st>>>(k, list_off[k], pc.use_ccc, ws.query,
                                                                   ws.counters, ws.heavy, memo);
            }
            launches += 2;
        }
    }
    {
        HookScope hs(hook, MPDP_KC_EXTRACT, st);
        k_extract<Memo><<<1, 32, 0, st>>>(ws.query, ws.counters, ws.result, memo);
    }
    launches++;
}

cudaError_t enqueue_pipeline(const Workspace& ws, const PipelineCfg& pc, cudaStream_t st,
                             int* launches_out, LaunchHook* hook)
{
    int launches = 0;
    const int n = pc.n;
    const bool dense = pc.memo_kind == MPDP_MEMO_DENSE;
    {
        HookScope hs(hook, MPDP_KC_INGEST, st);
        k_ingest<<<1, 256, 0, st>>>(ws.staged, ws.query, ws.counters, ws.dcost, ws.dleft, dense ? 1 : 0);
    }
    launches++;

    FilterParams fp;
    memset(&fp, 0, sizeof(fp));
    fp.n = n;
    fp.run = pc.run_length;
    level_layout(n, fp.list_off);
    unsigned long long wb = 0;
    for (int k = 0; k <= kLevels; k++) fp.warp_begin[k] = 0;
    for (int k = 2; k <= n; k++) {
        const unsigned long long c = binom_host(n, k);
        fp.nranks[k] = (uint32_t)c;
        fp.warp_begin[k] = (uint32_t)wb;
        wb += (c + 32ull * pc.run_length - 1) / (32ull * pc.run_length);
    }
    for (int k = n + 1; k <= kLevels; k++) fp.warp_begin[k] = (uint32_t)wb;
    if (n >= 2) fp.warp_begin[n + 1] = (uint32_t)wb;
    if (wb > 0) {
        const unsigned long long threads = wb * 32ull;
        const int blocks = (int)((threads + 255) / 256);
        HookScope hs(hook, MPDP_KC_FILTER, st);
        k_filter<<<blocks, 256, 0, st>>>(fp, ws.query, ws.counters, ws.lists);
        launches++;
    }
    if (dense) {
        DenseMemo memo{ws.dcost, ws.dleft};
        launch_levels(ws, pc, fp.list_off, memo, st, launches, hook);
    } else {
        {
            HookScope hs(hook, MPDP_KC_MEMO_INIT, st);
            k_hash_layout<<<1, 1, 0, st>>>(n, ws.counters, ws.layout, ws.arena_slots);
            k_hash_clear<<<pc.num_sms * 4, 256, 0, st>>>(ws.layout, ws.counters, ws.arena);
        }
        launches += 2;
        HashMemo memo{ws.arena, ws.layout, nullptr, nullptr};
        launch_levels(ws, pc, fp.list_off, memo, st, launches, hook);
    }
    if (launches_out) *launches_out = launches;
    return cudaGetLastError();
}

cudaError_t enqueue_stage_device(const double* card, const mpdp_edge* edges, int n, int m,
                                 int cost_model, StagedQuery* staged, cudaStream_t st, LaunchHook* hook)
{
    HookScope hs(hook, MPDP_KC_STAGE, st);
    k_stage<<<1, 256, 0, st>>>(card, edges, n, m, cost_model, staged);
    return cudaGetLastError();
}

cudaError_t enqueue_publish(const Workspace& ws, mpdp_plan_node* nodes, double* cost, int32_t* status,
                            cudaStream_t st, LaunchHook* hook)
{
    HookScope hs(hook, MPDP_KC_PUBLISH, st);
    k_publish<<<1, 64, 0, st>>>(ws.result, ws.counters, nodes, cost, status);
    return cudaGetLastError();
}

cudaError_t enqueue_memo_lookup(const Workspace& ws, int memo_kind, const uint32_t* d_sets, int count,
                                double* d_costs, uint32_t* d_lefts, cudaStream_t st)
{
    const int grid = (count + 255) / 256 > 0 ? (count + 255) / 256 : 1;
    if (memo_kind == MPDP_MEMO_DENSE) {
        DenseMemo memo{ws.dcost, ws.dleft};
        k_memo_lookup<DenseMemo><<<grid, 256, 0, st>>>(d_sets, count, d_costs, d_lefts, ws.counters, memo);
    } else {
        HashMemo memo{ws.arena, ws.layout, nullptr, nullptr};
        k_memo_lookup<HashMemo><<<grid, 256, 0, st>>>(d_sets, count, d_costs, d_lefts, ws.counters, memo);
    }
    return cudaGetLastError();
}

}  // namespace mpdp
