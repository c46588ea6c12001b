/* Multi-threaded CPU MPDP (Sec. 3.3): the paper's host implementation of
 * the method, kept as the "MPDP (24CPU)" comparison of Sec. 7.2.
 *
 * The structure follows the paper's description of its CPU version:
 *   - levels k = 2..n in order, a barrier between them (every set of size
 *     k reads only memo entries of smaller sets);
 *   - inside a level, a shared atomic counter holds the rank of the next
 *     k-subset to unrank; a worker takes a chunk of consecutive ranks,
 *     unranks the first with the combinatorial number system and steps to
 *     the next ones (colex order, the next bit permutation);
 *   - each connected set gets its best join pair by MPDP's block
 *     enumeration (Algorithm 4): the blocks of G[S], for each block B every
 *     unordered bipartition {lb, rb} with min(B) in lb, kept when both
 *     sides are connected (a CCP of the block), expanded to the split
 *     S_l = grow(lb, S \ rb), S_r = S \ S_l;
 *   - the results go to a thread-local list that the worker stores into
 *     the memo when the level's ranks run out.
 * The memo here is a dense array indexed by the relation bitmap, so the
 * stores of different sets never collide and need no lock (the paper's
 * workers store their lists under a mutex into a shared table).
 *
 * Blocks come from a depth-first search with low points (Hopcroft and
 * Tarjan's biconnected components), popping a vertex stack at each
 * articulation point.  card(S) is a product over S's relations and inner
 * edges in one order that depends on S alone: card(S \ {v}) * card[v] *
 * sel(j, v) for the neighbours j of v in S ascending, v the highest
 * non-cut vertex of G[S].  Among splits of equal cost sum x the one whose
 * smaller side has the smaller bitmap wins; cost(S) = x + card(S).  Every
 * floating-point operation is a single IEEE binary64 operation (built with
 * -ffp-contract=off). */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#include <unistd.h>

#include "../../include/mpdp_cpu.h"

#define MAXN MPDP_CPU_MAX_RELS
#define CHUNK 2048

typedef struct {
    uint32_t set, left;
    double cost, card;
} Result;

typedef struct {
    Result *v;
    size_t n, cap;
} ResultList;

typedef struct {
    int n;
    uint32_t adj[MAXN];
    double card[MAXN];
    double sel[MAXN][MAXN];
    uint64_t binom[MAXN + 1][MAXN + 1];
    double *cost, *cardm;
    uint32_t *left;
    int threads;
    pthread_barrier_t barrier;
    _Atomic uint64_t next[MAXN + 1]; /* next rank of each level */
    _Atomic uint64_t unranked, connected, evaluated, ccp;
    _Atomic int oom;
    /* start gate: workers wait until every one of them has been created */
    pthread_mutex_t gate_lock;
    pthread_cond_t gate;
    int go;       /* 1: run, -1: a thread could not be created, leave */
} Shared;

static inline int low_bit(uint32_t s) { return __builtin_ctz(s); }
static inline int popc(uint32_t s) { return __builtin_popcount(s); }

/* Every relation of `restriction` reachable from `source` inside it. */
static uint32_t grow(uint32_t source, uint32_t restriction, const uint32_t *adj)
{
    uint32_t seen = source, front = source;
    while (front) {
        const int x = low_bit(front);
        front &= front - 1u;
        const uint32_t nb = adj[x] & restriction & ~seen;
        seen |= nb;
        front |= nb;
    }
    return seen;
}

static inline int is_connected(uint32_t s, const uint32_t *adj)
{
    return s != 0u && grow(s & (0u - s), s, adj) == s;
}

/* Blocks of the connected G[S] (|S| >= 2), by depth-first search with low
 * points; returns how many. */
static int find_blocks(uint32_t s, const uint32_t *adj, uint32_t *blk)
{
    int disc[MAXN], low[MAXN], parent[MAXN];
    uint32_t rest[MAXN];
    int dfs[MAXN], vst[MAXN];
    int nd = 0, nv = 0, nb = 0, timer = 0;
    for (int i = 0; i < MAXN; i++) disc[i] = -1;
    const int root = low_bit(s);
    disc[root] = low[root] = timer++;
    parent[root] = -1;
    rest[root] = adj[root] & s;
    dfs[nd++] = root;
    vst[nv++] = root;
    while (nd) {
        const int v = dfs[nd - 1];
        if (rest[v]) {
            const int w = low_bit(rest[v]);
            rest[v] &= rest[v] - 1u;
            if (w == parent[v]) continue;
            if (disc[w] < 0) {
                disc[w] = low[w] = timer++;
                parent[w] = v;
                rest[w] = adj[w] & s;
                dfs[nd++] = w;
                vst[nv++] = w;
            } else if (disc[w] < low[v]) {
                low[v] = disc[w];
            }
            continue;
        }
        nd--;
        if (!nd) break;
        const int u = dfs[nd - 1];
        if (low[v] < low[u]) low[u] = low[v];
        if (low[v] >= disc[u]) {
            /* u separates v's subtree: one block, popped off the vertex stack */
            uint32_t b = 1u << u;
            int x;
            do {
                x = vst[--nv];
                b |= 1u << x;
            } while (x != v);
            blk[nb++] = b;
        }
    }
    return nb;
}

static int push(ResultList *l, Result r)
{
    if (l->n == l->cap) {
        const size_t cap = l->cap ? 2 * l->cap : 4096;
        Result *v = realloc(l->v, cap * sizeof(Result));
        if (!v) return 0;
        l->v = v;
        l->cap = cap;
    }
    l->v[l->n++] = r;
    return 1;
}

/* Best split, cost and card of one connected set S (|S| >= 2). */
static Result evaluate(const Shared *g, uint32_t s, uint64_t *evaluated, uint64_t *ccp)
{
    uint32_t blk[MAXN];
    const int nb = find_blocks(s, g->adj, blk);
    uint64_t best_x = UINT64_MAX;
    uint32_t best_l = UINT32_MAX;
    uint32_t once = 0u, twice = 0u;
    for (int j = 0; j < nb; j++) {
        const uint32_t b = blk[j];
        twice |= once & b;
        once |= b;
        *evaluated += (1ull << (popc(b) - 1)) - 1ull;
        const uint32_t mn = b & (0u - b), rest = b ^ mn;
        for (uint32_t sub = 0u; sub != rest; sub = (sub - rest) & rest) {
            const uint32_t lb = mn | sub, rb = b ^ lb;
            if (!is_connected(lb, g->adj) || !is_connected(rb, g->adj)) continue;
            (*ccp)++;
            const uint32_t sl = grow(lb, s & ~rb, g->adj), sr = s ^ sl;
            const double x = g->cost[sl] + g->cost[sr];
            uint64_t xb;
            memcpy(&xb, &x, sizeof xb);
            const uint32_t l = sl < sr ? sl : sr;
            if (xb < best_x || (xb == best_x && l < best_l)) {
                best_x = xb;
                best_l = l;
            }
        }
    }
    /* peel the highest non-cut vertex (a vertex of exactly one block) */
    const uint32_t noncut = s & ~twice;
    const int v = 31 - __builtin_clz(noncut);
    double p = g->cardm[s & ~(1u << v)];
    p = p * g->card[v];
    uint32_t nbr = g->adj[v] & s;
    while (nbr) {
        const int j = low_bit(nbr);
        nbr &= nbr - 1u;
        p = p * g->sel[j][v];
    }
    double x;
    memcpy(&x, &best_x, sizeof x);
    Result r = {s, best_l, x + p, p};
    return r;
}

/* colex unranking of a k-subset of {0..n-1} */
static uint32_t unrank(const Shared *g, int k, uint64_t r)
{
    uint32_t s = 0u;
    int c = g->n - 1;
    for (int i = k; i >= 1; i--) {
        while (g->binom[c][i] > r) c--;
        s |= 1u << c;
        r -= g->binom[c][i];
        c--;
    }
    return s;
}

static inline uint32_t next_perm(uint32_t s)
{
    const uint64_t v = s;
    const uint64_t t = v | (v - 1u);
    return (uint32_t)((t + 1u) | (((~t & (t + 1u)) - 1u) >> (__builtin_ctzll(v) + 1)));
}

typedef struct {
    Shared *g;
} WorkerArg;

static void *worker(void *arg)
{
    Shared *g = ((WorkerArg *)arg)->g;
    pthread_mutex_lock(&g->gate_lock);
    while (g->go == 0) pthread_cond_wait(&g->gate, &g->gate_lock);
    const int go = g->go;
    pthread_mutex_unlock(&g->gate_lock);
    if (go < 0) return NULL;
    ResultList list = {NULL, 0, 0};
    for (int k = 2; k <= g->n; k++) {
        const uint64_t total = g->binom[g->n][k];
        uint64_t unranked = 0, connected = 0, evaluated = 0, ccp = 0;
        for (;;) {
            const uint64_t r0 = atomic_fetch_add(&g->next[k], CHUNK);
            if (r0 >= total) break;
            const uint64_t r1 = r0 + CHUNK < total ? r0 + CHUNK : total;
            uint32_t s = unrank(g, k, r0);
            for (uint64_t r = r0; r < r1; r++, s = next_perm(s)) {
                unranked++;
                if (!is_connected(s, g->adj)) continue;
                connected++;
                if (!push(&list, evaluate(g, s, &evaluated, &ccp))) atomic_store(&g->oom, 1);
            }
        }
        for (size_t i = 0; i < list.n; i++) {
            const Result *x = &list.v[i];
            g->cost[x->set] = x->cost;
            g->cardm[x->set] = x->card;
            g->left[x->set] = x->left;
        }
        list.n = 0;
        atomic_fetch_add(&g->unranked, unranked);
        atomic_fetch_add(&g->connected, connected);
        atomic_fetch_add(&g->evaluated, evaluated);
        atomic_fetch_add(&g->ccp, ccp);
        pthread_barrier_wait(&g->barrier);
    }
    free(list.v);
    return NULL;
}

/* One memo for the process, grown on demand and reused by later calls (the
 * GPU library keeps its memo in its context the same way); calls take turns
 * on it. */
static pthread_mutex_t ws_lock = PTHREAD_MUTEX_INITIALIZER;
static void *ws_mem = NULL;
static size_t ws_bytes = 0;

static int finite_pos(double x) { return isfinite(x) && x > 0.0; }

int mpdp_cpu_optimize(int32_t n_rels, const double *card, int32_t n_edges, const mpdp_edge *edges,
                      int32_t threads, mpdp_plan_node *nodes, int32_t cap, int32_t *n_nodes, double *cost,
                      mpdp_cpu_stats *st)
{
    const int n = n_rels;
    if (n < 1 || n_edges < 0 || !card || (n_edges > 0 && !edges) || threads < 0) return MPDP_ERR_INVALID_ARG;
    if (n > MAXN) return MPDP_ERR_TOO_LARGE;
    if ((long long)n_edges > (long long)n * (n - 1) / 2) return MPDP_ERR_INVALID_ARG;
    if (cap > 0 && !nodes) return MPDP_ERR_INVALID_ARG;
    if (cap > 0 && cap < 2 * n - 1) return MPDP_ERR_BUFFER_TOO_SMALL;
    Shared *g = calloc(1, sizeof(Shared));
    if (!g) return MPDP_ERR_OOM;
    g->n = n;
    for (int i = 0; i < n; i++) {
        if (!finite_pos(card[i])) {
            free(g);
            return MPDP_ERR_INVALID_ARG;
        }
        g->card[i] = card[i];
        for (int j = 0; j < n; j++) g->sel[i][j] = 1.0;
    }
    for (int e = 0; e < n_edges; e++) {
        const int u = edges[e].u, v = edges[e].v;
        const double sv = edges[e].sel;
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(sv > 0.0) || !(sv <= 1.0) ||
            (g->adj[u] >> v & 1u)) {
            free(g);
            return MPDP_ERR_INVALID_ARG;
        }
        g->adj[u] |= 1u << v;
        g->adj[v] |= 1u << u;
        g->sel[u][v] = g->sel[v][u] = sv;
    }
    const uint32_t full = n == 32 ? 0xffffffffu : (1u << n) - 1u;
    if (grow(1u, full, g->adj) != full) {
        free(g);
        return MPDP_ERR_DISCONNECTED;
    }
    for (int a = 0; a <= n; a++) {
        g->binom[a][0] = 1;
        for (int b = 1; b <= a; b++) g->binom[a][b] = g->binom[a - 1][b - 1] + (b <= a - 1 ? g->binom[a - 1][b] : 0);
    }
    if (threads == 0) {
        const long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int)c : 1;
    }
    if (threads > 1024) threads = 1024;
    g->threads = threads;

    pthread_mutex_lock(&ws_lock);
    const size_t entries = (size_t)1 << n;
    const size_t need = entries * (2 * sizeof(double) + sizeof(uint32_t));
    if (ws_bytes < need) {
        free(ws_mem);
        ws_mem = malloc(need);
        ws_bytes = ws_mem ? need : 0;
    }
    if (!ws_mem) {
        pthread_mutex_unlock(&ws_lock);
        free(g);
        return MPDP_ERR_OOM;
    }
    g->cost = (double *)ws_mem;
    g->cardm = g->cost + entries;
    g->left = (uint32_t *)(g->cardm + entries);
    for (int i = 0; i < n; i++) {
        g->cost[1u << i] = 0.0;
        g->cardm[1u << i] = card[i];
        g->left[1u << i] = 0u;
    }
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    int rc = MPDP_OK;
    if (n >= 2) {
        pthread_mutex_init(&g->gate_lock, NULL);
        pthread_cond_init(&g->gate, NULL);
        pthread_t *tid = malloc(sizeof(pthread_t) * (size_t)threads);
        WorkerArg wa = {g};
        int started = 0;
        if (tid)
            for (int i = 0; i < threads; i++) {
                if (pthread_create(&tid[i], NULL, worker, &wa) != 0) break;
                started++;
            }
        /* the level barrier counts every worker, so either all of them run
         * or none does */
        if (started == threads) pthread_barrier_init(&g->barrier, NULL, (unsigned)threads);
        pthread_mutex_lock(&g->gate_lock);
        g->go = started == threads ? 1 : -1;
        pthread_cond_broadcast(&g->gate);
        pthread_mutex_unlock(&g->gate_lock);
        for (int i = 0; i < started; i++) pthread_join(tid[i], NULL);
        if (started == threads) pthread_barrier_destroy(&g->barrier);
        else rc = MPDP_ERR_OOM;
        free(tid);
        pthread_cond_destroy(&g->gate);
        pthread_mutex_destroy(&g->gate_lock);
        if (atomic_load(&g->oom)) rc = MPDP_ERR_OOM;
    }
    if (rc != MPDP_OK) {
        pthread_mutex_unlock(&ws_lock);
        free(g);
        return rc;
    }
    clock_gettime(CLOCK_MONOTONIC, &t1);
    if (cost) *cost = g->cost[full];
    int count = 0;
    if (cap > 0) {
        /* breadth-first from the full set */
        uint32_t sets[2 * MAXN];
        sets[0] = full;
        int m = 1;
        for (int i = 0; i < m; i++) {
            const uint32_t s = sets[i];
            mpdp_plan_node *nd = &nodes[i];
            nd->set = s;
            nd->n_leaves = popc(s);
            nd->card = g->cardm[s];
            if ((s & (s - 1u)) == 0u) {
                nd->left = nd->right = -1;
                nd->rel = low_bit(s);
                nd->cost = 0.0;
            } else {
                nd->rel = -1;
                nd->cost = g->cost[s];
                nd->left = m;
                nd->right = m + 1;
                sets[m++] = g->left[s];
                sets[m++] = s ^ g->left[s];
            }
        }
        count = m;
    }
    pthread_mutex_unlock(&ws_lock);
    if (n_nodes) *n_nodes = count;
    if (st) {
        st->sets_unranked = g->unranked;
        st->sets_connected = g->connected;
        st->pairs_evaluated = g->evaluated;
        st->ccp_pairs = g->ccp;
        st->threads = threads;
        st->reserved = 0;
        st->wall_ms = (double)(t1.tv_sec - t0.tv_sec) * 1e3 + (double)(t1.tv_nsec - t0.tv_nsec) * 1e-6;
    }
    free(g);
    return MPDP_OK;
}
