/*
 * CPU oracle, extended range: the exact DP of mpdp_oracle.c in "XD"
 * arithmetic, for the heuristic modes (IDP2 and UnionDP; paper Sec. 4),
 * whose sub-problems join composite relations with cardinalities far
 * beyond binary64's range.
 *
 * TEST INFRASTRUCTURE ONLY, like mpdp_oracle.c: only the test suite, the
 * smoke check and the benchmark's CPU legs may load it; it shares no code
 * with the CUDA path.  Build with -O2 -ffp-contract=off.
 *
 * XD (a reading; the paper works with bounded PK-FK cardinalities and is
 * silent on range): a value is m * 2^e with m = 0, or 1 <= m < 2, and e a
 * 32-bit integer.
 *   mul: p = m_a * m_b (one binary64 multiply, round to nearest), e = e_a +
 *        e_b; if p >= 2 then p = p / 2, e = e + 1.
 *   add: with e_a >= e_b and d = e_a - e_b: s = m_a + m_b * 2^-d (one
 *        binary64 add; for d > 60 the second term is dropped, which is the
 *        same rounding), e = e_a; if s >= 2 then s = s / 2, e = e + 1.
 *   compare: 0 is smallest; otherwise by e, then by m.
 * Scaling by powers of two is exact, so each operation rounds exactly as
 * binary64 does on the same real values whenever binary64 would neither
 * overflow nor leave the normal range: XD results are then the binary64
 * results, bit for bit.
 *
 * Everything else (graph, CCP enumeration, peeling card, the (x, left)
 * rule) is the definition of mpdp_oracle.c with XD in place of double:
 *   card({r}) = card[r]; card(S) = ((card(S \ {v}) * card[v]) * sel(j1, v))
 *   * ... over v's neighbours j1 < j2 < ... in S, v = the highest-index
 *   member whose removal does not increase the number of components;
 *   cost({r}) = 0; x = cost(S_left) + cost(S_right); the split with the
 *   least (x, left) wins; cost(S) = x + card(S).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define XO_OK 0
#define XO_INVALID (-1)
#define XO_DISCONNECTED (-2)
#define XO_TOO_LARGE (-3)
#define XO_NOMEM (-4)
#define XO_MAXN 25

typedef struct {
    double m;
    int32_t e;
} xd;

static xd xd_zero(void)
{
    xd r = {0.0, 0};
    return r;
}

/* c * 2^e2 for a finite c >= 0 (any binary64, subnormals included) */
static xd xd_make(double c, int32_t e2)
{
    if (c == 0.0) return xd_zero();
    int ex;
    double f = frexp(c, &ex); /* c = f * 2^ex, 0.5 <= f < 1 */
    xd r = {f * 2.0, e2 + ex - 1};
    return r;
}

static xd xd_mul(xd a, xd b)
{
    if (a.m == 0.0 || b.m == 0.0) return xd_zero();
    xd r;
    r.m = a.m * b.m;
    r.e = a.e + b.e;
    if (r.m >= 2.0) {
        r.m = r.m * 0.5;
        r.e = r.e + 1;
    }
    return r;
}

static xd xd_add(xd a, xd b)
{
    if (a.m == 0.0) return b;
    if (b.m == 0.0) return a;
    if (a.e < b.e) {
        xd t = a;
        a = b;
        b = t;
    }
    int64_t d = (int64_t)a.e - (int64_t)b.e;
    xd r;
    r.e = a.e;
    r.m = a.m;
    if (d <= 60) r.m = a.m + ldexp(b.m, (int)-d);
    if (r.m >= 2.0) {
        r.m = r.m * 0.5;
        r.e = r.e + 1;
    }
    return r;
}

/* -1, 0, 1 as a is below, equal to, above b */
static int xd_cmp(xd a, xd b)
{
    if (a.m == 0.0 || b.m == 0.0) {
        if (a.m == b.m) return 0;
        return a.m == 0.0 ? -1 : 1;
    }
    if (a.e != b.e) return a.e < b.e ? -1 : 1;
    if (a.m != b.m) return a.m < b.m ? -1 : 1;
    return 0;
}

/* ---------------------------------------------------------------------- */

typedef struct {
    int n;
    uint32_t adj[XO_MAXN];
    xd card[XO_MAXN];
    xd sel[XO_MAXN][XO_MAXN];
} xgraph;

static uint32_t xbit(int i) { return (uint32_t)1 << i; }

static int xbuild(xgraph *g, int n, const double *cm, const int32_t *ce, int m, const int32_t *eu,
                  const int32_t *ev, const double *sm, const int32_t *se)
{
    if (n < 1 || n > XO_MAXN) return XO_TOO_LARGE;
    memset(g, 0, sizeof(*g));
    g->n = n;
    for (int i = 0; i < n; i++) {
        if (!(cm[i] > 0.0) || !(cm[i] <= 1.7976931348623157e308)) return XO_INVALID;
        g->card[i] = xd_make(cm[i], ce[i]);
    }
    for (int k = 0; k < m; k++) {
        int u = eu[k], v = ev[k];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return XO_INVALID;
        if (!(sm[k] > 0.0) || !(sm[k] <= 1.7976931348623157e308)) return XO_INVALID;
        if (g->adj[u] & xbit(v)) return XO_INVALID;
        g->adj[u] |= xbit(v);
        g->adj[v] |= xbit(u);
        g->sel[u][v] = g->sel[v][u] = xd_make(sm[k], se[k]);
    }
    return XO_OK;
}

static uint32_t xgrow(const xgraph *g, uint32_t src, uint32_t restr)
{
    uint32_t seen = src & restr, frontier = seen;
    while (frontier) {
        int v = __builtin_ctz(frontier);
        frontier &= frontier - 1;
        uint32_t nb = g->adj[v] & restr & ~seen;
        seen |= nb;
        frontier |= nb;
    }
    return seen;
}

static int xcomponents(const xgraph *g, uint32_t s)
{
    int c = 0;
    while (s) {
        s &= ~xgrow(g, s & (0u - s), s);
        c++;
    }
    return c;
}

static int xpeel_vertex(const xgraph *g, uint32_t s)
{
    int base = xcomponents(g, s);
    for (int v = g->n - 1; v >= 0; v--)
        if ((s & xbit(v)) && xcomponents(g, s & ~xbit(v)) <= base) return v;
    return -1;
}

static xd xcard(const xgraph *g, xd *cache, uint8_t *known, uint32_t s)
{
    if (known[s]) return cache[s];
    xd c;
    if ((s & (s - 1)) == 0) {
        c = g->card[__builtin_ctz(s)];
    } else {
        int v = xpeel_vertex(g, s);
        c = xd_mul(xcard(g, cache, known, s & ~xbit(v)), g->card[v]);
        for (int j = 0; j < g->n; j++)
            if ((s & xbit(j)) && (g->adj[v] & xbit(j))) c = xd_mul(c, g->sel[j][v]);
    }
    cache[s] = c;
    known[s] = 1;
    return c;
}

/* The exact DP as the plain definition: for every connected S in order of
 * size, every unordered CCP pair (S1, S2) of S (S1 holding min(S)).
 * O(3^n): for small n, to pin the DPCCP form below. */
int oracle_xd_dpsub(int n, const double *cm, const int32_t *ce, int m, const int32_t *eu, const int32_t *ev,
                 const double *sm, const int32_t *se, double *cost_m, int32_t *cost_e, uint32_t *left)
{
    xgraph *g = malloc(sizeof(xgraph));
    if (!g) return XO_NOMEM;
    int rc = xbuild(g, n, cm, ce, m, eu, ev, sm, se);
    if (rc != XO_OK) {
        free(g);
        return rc;
    }
    uint32_t full = (n == 32) ? 0xffffffffu : ((uint32_t)1 << n) - 1;
    if (xgrow(g, 1u, full) != full) {
        free(g);
        return XO_DISCONNECTED;
    }
    size_t sz = (size_t)1 << n;
    xd *cost = malloc(sizeof(xd) * sz);
    xd *cardc = malloc(sizeof(xd) * sz);
    uint8_t *known = calloc(sz, 1);
    uint8_t *conn = calloc(sz, 1);
    if (!cost || !cardc || !known || !conn) {
        free(cost); free(cardc); free(known); free(conn); free(g);
        return XO_NOMEM;
    }
    cost[0] = xd_zero();
    left[0] = UINT32_MAX;
    for (size_t s = 1; s < sz; s++) {
        conn[s] = xgrow(g, (uint32_t)(s & (0 - s)), (uint32_t)s) == (uint32_t)s;
        cost[s] = xd_zero();
        left[s] = UINT32_MAX;
    }
    for (int i = 0; i < n; i++) left[xbit(i)] = 0;
    for (int k = 2; k <= n; k++) {
        for (size_t si = 1; si < sz; si++) {
            uint32_t s = (uint32_t)si;
            if (__builtin_popcount(s) != k || !conn[s]) continue;
            uint32_t mn = s & (0u - s), rest = s ^ mn;
            int have = 0;
            xd bx = xd_zero();
            uint32_t bl = UINT32_MAX;
            for (uint32_t sub = 0;; sub = (sub - rest) & rest) {
                uint32_t s1 = mn | sub, s2 = s ^ s1;
                if (s2 && conn[s1] && conn[s2]) {
                    xd x = xd_add(cost[s1], cost[s2]);
                    uint32_t l = s1 < s2 ? s1 : s2;
                    int c = have ? xd_cmp(x, bx) : -1;
                    if (c < 0 || (c == 0 && l < bl)) {
                        bx = x;
                        bl = l;
                        have = 1;
                    }
                }
                if (sub == rest) break;
            }
            cost[s] = xd_add(bx, xcard(g, cardc, known, s));
            left[s] = bl;
        }
    }
    for (size_t s = 0; s < sz; s++) {
        cost_m[s] = cost[s].m;
        cost_e[s] = cost[s].e;
    }
    free(cost); free(cardc); free(known); free(conn); free(g);
    return XO_OK;
}

/* ---------------------------------------------------------------------- */
/* XD DPCCP: the csg-cmp enumeration of mpdp_oracle.c (Moerkotte & Neumann:
 * csgs grown from each start vertex in descending order, complements
 * restricted to indices above min(S1), subsets before supersets), so that
 * both operands of every pair are final when it is costed. */
typedef struct {
    const xgraph *g;
    xd *xbest;
    uint32_t *left;
    xd *cost;
    uint8_t *fixed;
    xd *cardc;
    uint8_t *known;
} xstate;

static xd xfinal(xstate *st, uint32_t s)
{
    if ((s & (s - 1)) == 0) return xd_zero();
    if (!st->fixed[s]) {
        st->cost[s] = xd_add(st->xbest[s], xcard(st->g, st->cardc, st->known, s));
        st->fixed[s] = 1;
    }
    return st->cost[s];
}

static void xemit(xstate *st, uint32_t s1, uint32_t s2)
{
    uint32_t s = s1 | s2;
    xd x = xd_add(xfinal(st, s1), xfinal(st, s2));
    uint32_t l = s1 < s2 ? s1 : s2;
    int c = st->left[s] == UINT32_MAX ? -1 : xd_cmp(x, st->xbest[s]);
    if (c < 0 || (c == 0 && l < st->left[s])) {
        st->xbest[s] = x;
        st->left[s] = l;
    }
}

static uint32_t xnbhd(const xgraph *g, uint32_t s)
{
    uint32_t r = 0;
    for (uint32_t t = s; t; t &= t - 1) r |= g->adj[__builtin_ctz(t)];
    return r & ~s;
}

typedef void (*xcb)(xstate *, uint32_t ctx, uint32_t s);

static void xgrow_rec(xstate *st, uint32_t s, uint32_t x, xcb cb, uint32_t ctx)
{
    uint32_t nb = xnbhd(st->g, s) & ~x;
    if (!nb) return;
    for (uint32_t sub = (0u - nb) & nb; sub; sub = (sub - nb) & nb) cb(st, ctx, s | sub);
    for (uint32_t sub = (0u - nb) & nb; sub; sub = (sub - nb) & nb) xgrow_rec(st, s | sub, x | nb, cb, ctx);
}

static void xcmp_found(xstate *st, uint32_t s1, uint32_t s2) { xemit(st, s1, s2); }

static void xenumerate_cmp(xstate *st, uint32_t s1)
{
    int mn = __builtin_ctz(s1);
    uint32_t bmin = (xbit(mn) << 1) - 1;
    uint32_t x = bmin | s1;
    uint32_t nb = xnbhd(st->g, s1) & ~x;
    for (int v = st->g->n - 1; v >= 0; v--) {
        if (!(nb & xbit(v))) continue;
        uint32_t bv = (xbit(v) << 1) - 1;
        xemit(st, s1, xbit(v));
        xgrow_rec(st, xbit(v), x | (bv & nb), (xcb)xcmp_found, s1);
    }
}

static void xcsg_found(xstate *st, uint32_t unused, uint32_t s1)
{
    (void)unused;
    xenumerate_cmp(st, s1);
}

int oracle_xd_dpccp(int n, const double *cm, const int32_t *ce, int m, const int32_t *eu, const int32_t *ev,
                    const double *sm, const int32_t *se, double *cost_m, int32_t *cost_e, uint32_t *left)
{
    xgraph *g = malloc(sizeof(xgraph));
    if (!g) return XO_NOMEM;
    int rc = xbuild(g, n, cm, ce, m, eu, ev, sm, se);
    if (rc != XO_OK) {
        free(g);
        return rc;
    }
    uint32_t full = ((uint32_t)1 << n) - 1;
    if (xgrow(g, 1u, full) != full) {
        free(g);
        return XO_DISCONNECTED;
    }
    size_t sz = (size_t)1 << n;
    xstate st;
    st.g = g;
    st.left = left;
    st.xbest = malloc(sizeof(xd) * sz);
    st.cost = malloc(sizeof(xd) * sz);
    st.fixed = calloc(sz, 1);
    st.cardc = malloc(sizeof(xd) * sz);
    st.known = calloc(sz, 1);
    if (!st.xbest || !st.cost || !st.fixed || !st.cardc || !st.known) {
        free(st.xbest); free(st.cost); free(st.fixed); free(st.cardc); free(st.known); free(g);
        return XO_NOMEM;
    }
    for (size_t i = 0; i < sz; i++) {
        left[i] = UINT32_MAX;
        st.cost[i] = xd_zero();
    }
    for (int i = 0; i < n; i++) left[xbit(i)] = 0;
    for (int i = n - 1; i >= 0; i--) {
        uint32_t s = xbit(i);
        xenumerate_cmp(&st, s);
        xgrow_rec(&st, s, (xbit(i) << 1) - 1, xcsg_found, 0);
    }
    for (size_t i = 1; i < sz; i++)
        if ((i & (i - 1)) != 0 && left[i] != UINT32_MAX) xfinal(&st, (uint32_t)i);
    for (size_t i = 0; i < sz; i++) {
        cost_m[i] = st.cost[i].m;
        cost_e[i] = st.cost[i].e;
    }
    free(st.xbest); free(st.cost); free(st.fixed); free(st.cardc); free(st.known); free(g);
    return XO_OK;
}

/* The two operations and the order, exported so that tests can pin them
 * against exact rational arithmetic. */
void oracle_xd_ops(double am, int32_t ae, double bm, int32_t be, double *sum_m, int32_t *sum_e, double *prod_m,
                   int32_t *prod_e, int32_t *cmp)
{
    xd a = xd_make(am, ae), b = xd_make(bm, be);
    xd s = xd_add(a, b), p = xd_mul(a, b);
    *sum_m = s.m;
    *sum_e = s.e;
    *prod_m = p.m;
    *prod_e = p.e;
    *cmp = xd_cmp(a, b);
}
