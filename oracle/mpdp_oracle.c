/*
 * CPU oracle for the MPDP join-order dynamic program.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it is plain, slow on purpose,
 * and written so that each function can be checked against the paper by eye.
 * Build with -O2 -ffp-contract=off (no FMA contraction, no fast-math) so that
 * every floating-point operation below is one IEEE-754 double operation with
 * round-to-nearest, in the order written.
 *
 * What is computed (paper: "Efficient Massively Parallel Join Optimization for
 * Large Queries", arXiv 2202.13511):
 *   - the join graph G(R,E) of Sec. 2.1; relation sets are bitmaps (Sec. 2.2,
 *     "Implementation Details");
 *   - grow(source, restriction) and connected(S) (Sec. 3.2.1, "Grow Function");
 *   - a join pair (S_left, S_right) is a CCP pair iff both parts are non-empty,
 *     induce connected subgraphs, are disjoint and are joined by an edge
 *     (Sec. 2.1, conditions 1-4);
 *   - BestPlan(S) for every connected S by generic DPSUB (Algorithm 1), and by
 *     DPCCP (Moerkotte & Neumann, cited in Sec. 1 and Sec. 5), which enumerates
 *     only CCP pairs and so reaches 25 relations;
 *   - blocks (maximal nonseparable induced subgraphs) and cut vertices
 *     (Sec. 2.4), by their plain definitions, to count what the block-based
 *     enumeration of Algorithm 4 evaluates.
 *
 * Readings where the paper is silent (the cost model is unspecified, Sec. 7.1):
 *   - cost model C_out: cost({R_i}) = 0,
 *       cost(L join R) = (cost(L) + cost(R)) + card(L u R);
 *   - card(S) is the product of card[r] over the relations of S and sel over
 *     the edges inside S, taken in one fixed order that depends on S alone
 *     ("peeling"): card({r}) = card[r]; otherwise let v be the highest-index
 *     relation of S whose removal does not increase the number of connected
 *     components of G[S] (for a connected S: its highest non-cut vertex), and
 *     card(S) = ((card(S \ {v}) * card[v]) * sel(j1, v)) * sel(j2, v) ...
 *     over the neighbours j1 < j2 < ... of v in S.  Every way of building S
 *     gets the same bits;
 *   - BestPlan(S) is the split with the lexicographic minimum of
 *     (x, left), x = cost(S_left) + cost(S_right) and left = the numerically
 *     smaller of the two masks; cost(S) = x + card(S).  Since card(S) is common
 *     to every split of S and IEEE addition is monotone, the minimum x gives
 *     the minimum cost; the rule replaces Algorithm 1's "first strict
 *     improvement wins", whose result would depend on enumeration order;
 *   - counters: ccp counts each unordered CCP pair once (this is the reading
 *     under which the 2805x ratio printed in Sec. 2.3 and Sec. 7.2.1 holds).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID (-1)
#define OR_DISCONNECTED (-2)
#define OR_TOO_LARGE (-3)
#define OR_NOMEM (-4)
#define OR_ORDER (-5) /* DPCCP used a plan before it was final: internal error */

#define OR_MAXN 64

typedef struct {
    int n;
    uint64_t adj[OR_MAXN];      /* adjacency bitmap of each relation */
    double card[OR_MAXN];       /* base cardinalities */
    double sel[OR_MAXN][OR_MAXN]; /* selectivity of edge (i,j); 1.0 if no edge */
} og_graph;

static uint64_t bit(int i) { return (uint64_t)1 << i; }

static int lowest_index(uint64_t s) { return __builtin_ctzll(s); }

static int popcount(uint64_t s) { return __builtin_popcountll(s); }

/* Build the join graph; rejects bad indices, self loops, duplicate edges,
 * non-finite or non-positive cardinalities and selectivities outside (0,1]. */
static int og_build(og_graph *g, int n, const double *card, int m, const int32_t *eu,
                    const int32_t *ev, const double *esel)
{
    if (n < 1 || n > OR_MAXN) return OR_TOO_LARGE;
    memset(g, 0, sizeof(*g));
    g->n = n;
    for (int i = 0; i < n; i++) {
        if (!(card[i] > 0.0) || !isfinite(card[i])) return OR_INVALID;
        g->card[i] = card[i];
        for (int j = 0; j < n; j++) g->sel[i][j] = 1.0;
    }
    for (int e = 0; e < m; e++) {
        int u = eu[e], v = ev[e];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return OR_INVALID;
        if (!(esel[e] > 0.0) || !(esel[e] <= 1.0)) return OR_INVALID;
        if (g->adj[u] & bit(v)) return OR_INVALID;
        g->adj[u] |= bit(v);
        g->adj[v] |= bit(u);
        g->sel[u][v] = esel[e];
        g->sel[v][u] = esel[e];
    }
    return OR_OK;
}

/* Neighbours of a set: union of the adjacency lists of its members. */
static uint64_t neighbours(const og_graph *g, uint64_t s)
{
    uint64_t r = 0;
    for (uint64_t t = s; t; t &= t - 1) r |= g->adj[lowest_index(t)];
    return r;
}

/* grow(source, restriction), Sec. 3.2.1: the vertices reachable from the
 * source set while staying inside the restriction set.  V starts empty, N
 * starts as the source; repeatedly take the first element x of N, put it in V
 * and add x's neighbours that lie in the restriction, minus V, to N. */
static uint64_t og_grow(const og_graph *g, uint64_t source, uint64_t restriction)
{
    uint64_t V = 0, N = source;
    while (N) {
        int x = lowest_index(N);
        V |= bit(x);
        N = (N | (g->adj[x] & restriction)) & ~V;
    }
    return V;
}

/* connected(S): S is non-empty and grow(min(S), S) = S. */
static int og_connected(const og_graph *g, uint64_t s)
{
    if (s == 0) return 0;
    return og_grow(g, s & (~s + 1), s) == s;
}

static int count_components(const og_graph *g, uint64_t s)
{
    int c = 0;
    while (s) {
        uint64_t comp = og_grow(g, s & (~s + 1), s);
        s &= ~comp;
        c++;
    }
    return c;
}

/* The peel vertex of S (|S| >= 2): the highest-index member whose removal
 * does not increase the number of connected components of G[S]. */
static int peel_vertex(const og_graph *g, uint64_t s)
{
    int base = count_components(g, s);
    for (int v = g->n - 1; v >= 0; v--) {
        if (!(s & bit(v))) continue;
        if (count_components(g, s & ~bit(v)) <= base) return v;
    }
    return -1; /* not reached: every non-empty graph has such a vertex */
}

/* The factors of the peel vertex v on top of card(S \ {v}). */
static double peel_factors(const og_graph *g, uint64_t s, int v, double p)
{
    p = p * g->card[v];
    for (int j = 0; j < g->n; j++)
        if ((s & bit(j)) && (g->adj[v] & bit(j))) p = p * g->sel[j][v];
    return p;
}

/* card(S) by peeling, as stated in the header (plain recursion). */
static double og_card(const og_graph *g, uint64_t s)
{
    if (popcount(s) == 1) return g->card[lowest_index(s)];
    int v = peel_vertex(g, s);
    return peel_factors(g, s, v, og_card(g, s & ~bit(v)));
}

/* The same definition with a per-set cache (NaN = not yet known). */
static double card_memo(const og_graph *g, double *cache, uint64_t s)
{
    double c = cache[s];
    if (c == c) return c;
    if (popcount(s) == 1) {
        c = g->card[lowest_index(s)];
    } else {
        int v = peel_vertex(g, s);
        c = peel_factors(g, s, v, card_memo(g, cache, s & ~bit(v)));
    }
    cache[s] = c;
    return c;
}

/* (c, l) is better than (bc, bl) under the lexicographic rule. */
static int better(double c, uint64_t l, double bc, uint64_t bl)
{
    return c < bc || (c == bc && l < bl);
}

/* ---------------------------------------------------------------------- */
/* Exported scalar helpers (used by the tests to pin the definitions).      */

int oracle_card(int n, const double *card, int m, const int32_t *eu, const int32_t *ev,
                const double *esel, uint64_t s, double *out)
{
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc == OR_OK) *out = og_card(g, s);
    free(g);
    return rc;
}

int oracle_grow(int n, const double *card, int m, const int32_t *eu, const int32_t *ev,
                const double *esel, uint64_t source, uint64_t restriction, uint64_t *out)
{
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc == OR_OK) *out = og_grow(g, source, restriction);
    free(g);
    return rc;
}

int oracle_connected(int n, const double *card, int m, const int32_t *eu, const int32_t *ev,
                     const double *esel, uint64_t s, int32_t *out)
{
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc == OR_OK) *out = og_connected(g, s);
    free(g);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Blocks and cut vertices of G[S] by their plain definitions (Sec. 2.4).   */

/* G[B] is nonseparable: connected, and (for |B| >= 3) still connected after
 * removing any single vertex. */
static int og_nonseparable(const og_graph *g, uint64_t b)
{
    if (!og_connected(g, b)) return 0;
    if (popcount(b) <= 2) return 1;
    for (uint64_t t = b; t; t &= t - 1) {
        uint64_t v = t & (~t + 1);
        if (!og_connected(g, b & ~v)) return 0;
    }
    return 1;
}

/* Blocks of G[S]: the maximal vertex sets B (|B| >= 2) inducing a nonseparable
 * subgraph.  Brute force over all subsets of S; for |S| <= 16.  Writes the
 * blocks in ascending mask order.  Returns the number of blocks, or < 0. */
int oracle_blocks(int n, const double *card, int m, const int32_t *eu, const int32_t *ev,
                  const double *esel, uint64_t s, uint64_t *blocks, int32_t cap,
                  uint64_t *cut_vertices)
{
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc != OR_OK) { free(g); return rc; }
    if (popcount(s) > 16) { free(g); return OR_TOO_LARGE; }
    int k = popcount(s);
    int idx[64], t = 0;
    for (int i = 0; i < g->n; i++)
        if (s & bit(i)) idx[t++] = i;
    uint64_t *ns = malloc(sizeof(uint64_t) << k);
    int nns = 0;
    for (uint64_t code = 1; code < ((uint64_t)1 << k); code++) {
        uint64_t b = 0;
        for (int i = 0; i < k; i++)
            if (code & bit(i)) b |= bit(idx[i]);
        if (popcount(b) >= 2 && og_nonseparable(g, b)) ns[nns++] = b;
    }
    int nb = 0;
    for (int i = 0; i < nns; i++) {
        int maximal = 1;
        for (int j = 0; j < nns; j++)
            if (j != i && (ns[i] & ns[j]) == ns[i] && ns[j] != ns[i]) { maximal = 0; break; }
        if (maximal) {
            if (nb < cap) blocks[nb] = ns[i];
            nb++;
        }
    }
    /* cut vertex: removal increases the number of connected components */
    uint64_t cuts = 0;
    int base = count_components(g, s);
    for (uint64_t r = s; r; r &= r - 1) {
        uint64_t v = r & (~r + 1);
        if (count_components(g, s & ~v) > base) cuts |= v;
    }
    if (cut_vertices) *cut_vertices = cuts;
    free(ns);
    free(g);
    /* ascending order */
    int w = nb < cap ? nb : cap;
    for (int i = 1; i < w; i++)
        for (int j = i; j > 0 && blocks[j - 1] > blocks[j]; j--) {
            uint64_t x = blocks[j]; blocks[j] = blocks[j - 1]; blocks[j - 1] = x;
        }
    return nb;
}

/* Per-level counts of what the block-based enumeration of Algorithm 4 visits,
 * from the plain block definition: for each connected S (|S| >= 2) and each of
 * its blocks B, the unordered bipartitions {lb, rb} of B number 2^(|B|-1) - 1
 * (Algorithm 4's loop over all non-empty proper lb visits each twice). Also
 * counts, per level, how many of those block bipartitions pass the CCP block
 * (both halves connected; they are always adjacent since B is connected).
 * Brute force; for n <= 12. */
int oracle_block_enum_counts(int n, const double *card, int m, const int32_t *eu,
                             const int32_t *ev, const double *esel,
                             uint64_t *evaluated_per_level, uint64_t *valid_per_level)
{
    if (n > 12) return OR_TOO_LARGE;
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc != OR_OK) { free(g); return rc; }
    for (int i = 0; i <= n; i++) evaluated_per_level[i] = valid_per_level[i] = 0;
    uint64_t blocks[64];
    for (uint64_t s = 1; s < ((uint64_t)1 << n); s++) {
        int k = popcount(s);
        if (k < 2 || !og_connected(g, s)) continue;
        int nb = oracle_blocks(n, card, m, eu, ev, esel, s, blocks, 64, NULL);
        if (nb < 0) { free(g); return nb; }
        for (int i = 0; i < nb; i++) {
            uint64_t b = blocks[i];
            int bs = popcount(b);
            evaluated_per_level[k] += ((uint64_t)1 << (bs - 1)) - 1;
            uint64_t mn = b & (~b + 1);
            uint64_t rest = b & ~mn;
            /* every submask of rest, the full one excluded (it leaves rb empty) */
            for (uint64_t sub = 0;; sub = (sub - rest) & rest) {
                uint64_t lb = mn | sub, rb = b & ~lb;
                if (rb && og_connected(g, lb) && og_connected(g, rb) &&
                    (neighbours(g, lb) & rb))
                    valid_per_level[k]++;
                if (sub == rest) break;
            }
        }
    }
    free(g);
    return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* Generic DPSUB, Algorithm 1.                                              */
/*
 * Outputs, indexed by relation bitmap (size 2^n):
 *   best_cost[S], best_left[S] for every connected S (singletons: 0, 0);
 *   other entries are left untouched.
 * counters[k] (k = 0..n) per level:  [0*(n+1)+k] connected sets of size k,
 * [1*(n+1)+k] join pairs evaluated (every S_left subset of S, empty and full
 * ones included, as Algorithm 1's inner loop does), [2*(n+1)+k] CCP pairs
 * counted once per unordered pair.
 */
int oracle_dpsub(int n, const double *card, int m, const int32_t *eu, const int32_t *ev,
                 const double *esel, double *best_cost, uint32_t *best_left, uint64_t *counters)
{
    if (n > 20) return OR_TOO_LARGE;
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc != OR_OK) { free(g); return rc; }
    uint64_t full = (n == 64) ? ~(uint64_t)0 : (bit(n) - 1);
    if (!og_connected(g, full)) { free(g); return OR_DISCONNECTED; }
    int L = n + 1;
    double *cardc = malloc(sizeof(double) << n);
    if (!cardc) { free(g); return OR_NOMEM; }
    for (uint64_t s = 0; s <= full; s++) cardc[s] = NAN;
    memset(counters, 0, sizeof(uint64_t) * 3 * L);
    for (int i = 0; i < n; i++) {       /* BestPlan({R_i}) = R_i */
        best_cost[bit(i)] = 0.0;
        best_left[bit(i)] = 0;
        counters[0 * L + 1]++;
    }
    for (int i = 2; i <= n; i++) {
        for (uint64_t s = 1; s <= full; s++) {  /* every S of size i */
            if (popcount(s) != i || !og_connected(g, s)) continue;
            counters[0 * L + i]++;
            double card_s = card_memo(g, cardc, s);
            double bx = INFINITY;
            uint64_t bl = UINT64_MAX;
            uint64_t ordered_ccp = 0;
            for (uint64_t sl = s;; sl = (sl - 1) & s) {  /* every S_left subset of S */
                counters[1 * L + i]++;
                uint64_t sr = s & ~sl;
                int ok = 1;
                if (sl == 0 || sr == 0) ok = 0;
                else if (!og_connected(g, sl)) ok = 0;
                else if (!og_connected(g, sr)) ok = 0;
                else if (sl & sr) ok = 0;
                else if (!(neighbours(g, sl) & sr)) ok = 0;
                if (ok) {
                    ordered_ccp++;
                    double x = best_cost[sl] + best_cost[sr];
                    uint64_t l = sl < sr ? sl : sr;
                    if (better(x, l, bx, bl)) { bx = x; bl = l; }
                }
                if (sl == 0) break;
            }
            counters[2 * L + i] += ordered_ccp / 2;
            best_cost[s] = bx + card_s;
            best_left[s] = (uint32_t)bl;
        }
    }
    free(cardc);
    free(g);
    return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* DPCCP: enumerate every connected subgraph (csg) S1 and, for each, every
 * connected complement S2 (cmp) that is disjoint from S1, adjacent to it and
 * has min(S2) > min(S1), so that each unordered CCP pair appears once.  The
 * enumeration follows Moerkotte & Neumann (VLDB 2006): csgs are grown from each
 * start vertex v_i (descending i) into neighbourhoods that exclude every vertex
 * with index <= i, and within one start vertex subsets are emitted before
 * supersets (submasks in ascending order), so that when a pair (S1, S2) is
 * costed both BestPlan(S1) and BestPlan(S2) are final.  That ordering property
 * is checked at run time: a set whose plan has already been read as an
 * operand may not be improved afterwards (OR_ORDER otherwise).
 */
typedef struct {
    const og_graph *g;
    double *cost;    /* final cost, NaN until the set is first read as an operand */
    double *xbest;   /* best x = cost(S_left) + cost(S_right) so far */
    uint32_t *left;
    double *cardc;   /* card(S) cache, NaN = not yet computed */
    uint8_t *used;   /* bit per set: plan already read as an operand */
    uint64_t *counters;
    int L;
    int status;
} dpccp_state;

static void mark_used(dpccp_state *st, uint64_t s) { st->used[s >> 3] |= (uint8_t)(1u << (s & 7)); }
static int is_used(dpccp_state *st, uint64_t s) { return (st->used[s >> 3] >> (s & 7)) & 1; }

/* cost(S) of a set whose pairs have all been seen: 0 for a relation,
 * x + card(S) otherwise (fixed at the first read). */
static double final_cost(dpccp_state *st, uint64_t s)
{
    if ((s & (s - 1)) == 0) return 0.0;
    double c = st->cost[s];
    if (c != c) {
        c = st->xbest[s] + card_memo(st->g, st->cardc, s);
        st->cost[s] = c;
    }
    return c;
}

static void emit_pair(dpccp_state *st, uint64_t s1, uint64_t s2)
{
    uint64_t s = s1 | s2;
    int k = popcount(s);
    st->counters[2 * st->L + k]++;
    mark_used(st, s1);
    mark_used(st, s2);
    double x = final_cost(st, s1) + final_cost(st, s2);
    uint64_t l = s1 < s2 ? s1 : s2;
    if (st->left[s] == UINT32_MAX) {
        st->counters[0 * st->L + k]++;   /* first time this set is formed */
    }
    if (better(x, l, st->xbest[s], st->left[s] == UINT32_MAX ? UINT64_MAX : st->left[s])) {
        if (is_used(st, s)) st->status = OR_ORDER;
        st->xbest[s] = x;
        st->left[s] = (uint32_t)l;
    }
}

/* Connected supersets S u S' of a csg S grown into N(S) \ X; for each one
 * found, call on_set.  Subsets are emitted before supersets. */
typedef void (*set_cb)(dpccp_state *, uint64_t ctx, uint64_t s);

static void grow_rec(dpccp_state *st, uint64_t s, uint64_t x, set_cb cb, uint64_t ctx)
{
    uint64_t nb = neighbours(st->g, s) & ~s & ~x;
    if (!nb) return;
    for (uint64_t sub = (0 - nb) & nb; sub; sub = (sub - nb) & nb) cb(st, ctx, s | sub);
    for (uint64_t sub = (0 - nb) & nb; sub; sub = (sub - nb) & nb)
        grow_rec(st, s | sub, x | nb, cb, ctx);
}

static void cmp_found(dpccp_state *st, uint64_t s1, uint64_t s2) { emit_pair(st, s1, s2); }

static void enumerate_cmp(dpccp_state *st, uint64_t s1)
{
    int mn = lowest_index(s1);
    uint64_t bmin = (bit(mn) << 1) - 1;           /* B_min(S1): indices <= min(S1) */
    uint64_t x = bmin | s1;
    uint64_t nb = neighbours(st->g, s1) & ~x;
    for (int v = st->g->n - 1; v >= 0; v--) {     /* v in N by descending index */
        if (!(nb & bit(v))) continue;
        uint64_t bv = (bit(v) << 1) - 1;
        emit_pair(st, s1, bit(v));
        grow_rec(st, bit(v), x | (bv & nb), (set_cb)cmp_found, s1);
    }
}

static void csg_found(dpccp_state *st, uint64_t unused, uint64_t s1)
{
    (void)unused;
    enumerate_cmp(st, s1);
}

int oracle_dpccp(int n, const double *card, int m, const int32_t *eu, const int32_t *ev,
                 const double *esel, double *best_cost, uint32_t *best_left, uint64_t *counters)
{
    if (n > 28) return OR_TOO_LARGE;
    og_graph *g = malloc(sizeof(og_graph));
    if (!g) return OR_NOMEM;
    int rc = og_build(g, n, card, m, eu, ev, esel);
    if (rc != OR_OK) { free(g); return rc; }
    uint64_t full = bit(n) - 1;
    if (!og_connected(g, full)) { free(g); return OR_DISCONNECTED; }
    size_t sz = (size_t)1 << n;
    dpccp_state st;
    st.g = g;
    st.cost = best_cost;
    st.left = best_left;
    st.xbest = malloc(sizeof(double) * sz);
    st.cardc = malloc(sizeof(double) * sz);
    st.used = calloc(sz / 8 + 1, 1);
    st.counters = counters;
    st.L = n + 1;
    st.status = OR_OK;
    if (!st.cardc || !st.used || !st.xbest) {
        free(st.cardc); free(st.used); free(st.xbest); free(g); return OR_NOMEM;
    }
    for (size_t i = 0; i < sz; i++) {
        best_cost[i] = NAN;
        st.xbest[i] = INFINITY;
        best_left[i] = UINT32_MAX;
        st.cardc[i] = NAN;
    }
    memset(counters, 0, sizeof(uint64_t) * 3 * st.L);
    for (int i = 0; i < n; i++) {
        best_cost[bit(i)] = 0.0;
        best_left[bit(i)] = 0;
        counters[0 * st.L + 1]++;
    }
    for (int i = n - 1; i >= 0; i--) {
        uint64_t s = bit(i);
        enumerate_cmp(&st, s);
        grow_rec(&st, s, (bit(i) << 1) - 1, csg_found, 0);
    }
    /* pairs evaluated = CCP pairs: DPCCP only ever enumerates CCP pairs */
    for (int k = 0; k <= n; k++) counters[1 * st.L + k] = counters[2 * st.L + k];
    /* fix the cost of every formed set not read as an operand (the full set
     * among them); sets never formed (disconnected) keep cost +inf */
    for (size_t i = 1; i < sz; i++) {
        if ((i & (i - 1)) == 0) continue;
        if (best_left[i] == UINT32_MAX) best_cost[i] = INFINITY;
        else final_cost(&st, i);
    }
    free(st.xbest);
    free(st.cardc);
    free(st.used);
    free(g);
    return st.status;
}
