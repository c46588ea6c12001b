"""Pins of the extended-range oracle and the heuristic drivers (CPU only).

* XD add / multiply equal exact rational arithmetic rounded to 53
  significant bits (round half to even), in both the C and Python forms.
* The XD DP equals the binary64 DP bit for bit when nothing leaves the
  binary64 range, and its DPCCP and DPSUB forms agree far outside that range.
* An XD brute force over every bushy plan of tiny queries, with cards near
  2^1000.
* Heuristic invariants: IDP2 and UnionDP with k >= n return the exact plan;
  every plan is a cross-product-free bushy tree over all relations; UnionDP
  partitions respect the threshold t; GOO's first join is the cheapest edge.
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import heuristics as H
from paper_2202_13511_gb300 import workloads as W


def exact(v):
    return Fraction(v[0]) * (Fraction(2) ** v[1]) if v[0] != 0.0 else Fraction(0)


def round53(x: Fraction):
    """x > 0 rounded to 53 significant bits, half to even, as (m, e)."""
    if x == 0:
        return (0.0, 0)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    while Fraction(2) ** (e + 1) <= x:
        e += 1
    scaled = x / Fraction(2) ** (e - 52)          # in [2^52, 2^53)
    q, r = divmod(scaled.numerator, scaled.denominator)
    twice = 2 * r
    if twice > scaled.denominator or (twice == scaled.denominator and q % 2 == 1):
        q += 1
    if q == 1 << 53:
        q >>= 1
        e += 1
    return (q / float(1 << 52), e)


def rand_xd(rng):
    m = 1.0 + rng.random()
    if rng.random() < 0.3:
        m = float(np.float64(1.0) + np.float64(rng.randrange(1 << 52)) / (1 << 52))
    return (m, rng.randrange(-3000, 3000))


def test_xd_ops_against_exact_rationals():
    rng = random.Random(5)
    for i in range(3000):
        a = rand_xd(rng)
        b = rand_xd(rng)
        if i % 4 == 0:
            b = (b[0], a[1] + rng.randrange(-70, 70))   # close exponents: real additions
        want_sum = round53(exact(a) + exact(b))
        want_prod = round53(exact(a) * exact(b))
        s, p, c = oracle.xd_ops(a, b)
        assert s == want_sum and p == want_prod, (a, b)
        assert H.xd_add(a, b) == want_sum and H.xd_mul(a, b) == want_prod
        assert c == (exact(a) > exact(b)) - (exact(a) < exact(b))
        assert (H.xd_key(a) > H.xd_key(b)) - (H.xd_key(a) < H.xd_key(b)) == c


def test_xd_zero_and_normalisation():
    s, p, c = oracle.xd_ops((0.0, 0), (1.5, 7))
    assert s == (1.5, 7) and p == (0.0, 0) and c == -1
    assert H.xd(3.0, 10) == (1.5, 11) and H.xd(5e-324) == (1.0, -1074)


def as_xd(q, scale=0):
    return [H.xd(c, scale) for c in q.card], [(u, v, H.xd(s)) for (u, v, s) in q.edges]


@pytest.mark.parametrize("kind,n,seed", [("star", 10, 1), ("chain", 12, 2), ("cyclic", 13, 3),
                                         ("clique", 9, 4), ("snowflake", 14, 5), ("cycle", 11, 6)])
def test_xd_dp_equals_binary64_in_range(kind, n, seed):
    q = W.make(kind, n, seed)
    ref = oracle.dpccp(q)
    cards, edges = as_xd(q)
    x = oracle.xd_dp(n, cards, edges)
    for s in range(1, 1 << n):
        if ref.left[s] == 0xFFFFFFFF:
            continue
        if s & (s - 1):
            assert x.left[s] == ref.left[s]
            assert math.ldexp(*x.cost(s)) == ref.cost[s]


@pytest.mark.parametrize("kind,n,seed", [("cyclic", 11, 7), ("star", 9, 8), ("clique", 8, 9)])
def test_xd_dpccp_equals_dpsub_out_of_range(kind, n, seed):
    q = W.make(kind, n, seed)
    rng = random.Random(seed)
    cards = [H.xd(c, rng.randrange(900, 2000)) for c in q.card]
    edges = [(u, v, H.xd(s, -rng.randrange(0, 900))) for (u, v, s) in q.edges]
    a = oracle.xd_dp(n, cards, edges, "dpccp")
    b = oracle.xd_dp(n, cards, edges, "dpsub")
    full = (1 << n) - 1
    assert a.cost(full)[1] > 1024  # far beyond binary64
    for s in range(1, 1 << n):
        if a.left[s] != 0xFFFFFFFF and s & (s - 1):
            assert a.left[s] == b.left[s] and a.cost(s) == b.cost(s)


def _peel_card(n, adj, card, sel, s):
    """card(S) by peeling in Python XD (the definition, written again)."""
    def comps(t):
        c = 0
        while t:
            seen = t & -t
            frontier = seen
            while frontier:
                low = frontier & -frontier
                v = low.bit_length() - 1
                frontier ^= low
                nb = adj[v] & t & ~seen
                seen |= nb
                frontier |= nb
            t &= ~seen
            c += 1
        return c
    if s & (s - 1) == 0:
        return card[s.bit_length() - 1]
    base = comps(s)
    v = next(v for v in range(n - 1, -1, -1) if (s >> v) & 1 and comps(s & ~(1 << v)) <= base)
    c = H.xd_mul(_peel_card(n, adj, card, sel, s & ~(1 << v)), card[v])
    for j in range(n):
        if (s >> j) & 1 and (adj[v] >> j) & 1:
            c = H.xd_mul(c, sel[(min(j, v), max(j, v))])
    return c


def test_xd_brute_force_tiny():
    """Every bushy cross-product-free plan of 5-relation queries with cards
    near 2^1000, minimised under the recursive (x, left) rule."""
    for seed in range(6):
        q = W.make(["cyclic", "star", "chain"][seed % 3], 5, seed)
        rng = random.Random(seed)
        n = q.n
        card = [H.xd(c, rng.randrange(900, 1100)) for c in q.card]
        sel = {(min(u, v), max(u, v)): H.xd(s) for (u, v, s) in q.edges}
        adj = [0] * n
        for u, v, _ in q.edges:
            adj[u] |= 1 << v
            adj[v] |= 1 << u

        def _comps(t):
            c = 0
            while t:
                seen = t & -t
                frontier = seen
                while frontier:
                    low = frontier & -frontier
                    v = low.bit_length() - 1
                    frontier ^= low
                    nb = adj[v] & t & ~seen
                    seen |= nb
                    frontier |= nb
                t &= ~seen
                c += 1
            return c

        best = {}

        def solve(s):
            if s in best:
                return best[s]
            if s & (s - 1) == 0:
                best[s] = ((0.0, 0), 0)
                return best[s]
            cand = None
            mn = s & -s
            rest = s ^ mn
            sub = 0
            while True:
                s1 = mn | sub
                s2 = s ^ s1
                if s2 and _comps(s1) == 1 and _comps(s2) == 1:
                    x = H.xd_add(solve(s1)[0], solve(s2)[0])
                    key = (H.xd_key(x), min(s1, s2))
                    if cand is None or key < cand[0]:
                        cand = (key, x, min(s1, s2))
                if sub == rest:
                    break
                sub = (sub - rest) & rest
            cost = H.xd_add(cand[1], _peel_card(n, adj, card, sel, s))
            best[s] = (cost, cand[2])
            return best[s]

        full = (1 << n) - 1
        want = solve(full)
        got = oracle.xd_dp(n, card, [(u, v, sel[(min(u, v), max(u, v))]) for (u, v, _) in q.edges])
        assert got.cost(full) == want[0] and int(got.left[full]) == want[1]


def cross_product_free(g, p):
    if p.is_leaf:
        return True
    return (g.cut_sel(p.left.rels, p.right.rels) is not None and cross_product_free(g, p.left)
            and cross_product_free(g, p.right))


@pytest.mark.parametrize("kind,n,seed", [("snowflake", 14, 1), ("cyclic", 12, 2), ("star", 11, 3)])
def test_heuristics_with_k_at_least_n_are_exact(kind, n, seed):
    q = W.make(kind, n, seed)
    g = H.Graph(q)
    ex = H.exact_over(g, [g.leaf(r) for r in range(n)])
    ref = oracle.dpccp(q)
    assert H.canonical(ex) == _canon_from_oracle(q, ref)
    for p in (H.idp2(g, n), H.uniondp(g, n, n)):
        assert H.canonical(p) == H.canonical(ex)
        assert p.cost == ex.cost


def _canon_from_oracle(q, ref):
    def build(s):
        if s & (s - 1) == 0:
            return s.bit_length() - 1
        l = int(ref.left[s])
        a, b = build(l), build(s ^ l)
        lo_a = (l & -l).bit_length() - 1
        r = s ^ l
        lo_b = (r & -r).bit_length() - 1
        return (a, b) if lo_a < lo_b else (b, a)
    return build((1 << q.n) - 1)


@pytest.mark.parametrize("n,seed", [(40, 1), (60, 2)])
def test_heuristic_plans_valid(n, seed):
    q = W.make("snowflake_plus", n, seed)
    g = H.Graph(q)
    for p in (H.goo(g), H.idp2(g, 8), H.uniondp(g, 10, 6)):
        assert p.rels == (1 << n) - 1 and p.leaves == n
        assert cross_product_free(g, p)
        assert H.plan_cost(g, p).cost == p.cost


def test_goo_first_join_is_cheapest_edge():
    q = W.make("cyclic", 12, 3)
    g = H.Graph(q)
    p = H.goo(g)
    joins = []

    def walk(t):
        if not t.is_leaf:
            walk(t.left)
            walk(t.right)
            if t.left.is_leaf and t.right.is_leaf:
                joins.append(t)

    walk(p)
    cheapest = min((H.xd_key(g.join(g.leaf(u), g.leaf(v)).card), u, v) for (u, v, _) in g.edges)
    assert any((H.xd_key(j.card), j.left.rel, j.right.rel) == cheapest for j in joins)


def test_uniondp_partitions_respect_threshold(monkeypatch):
    q = W.make("snowflake_plus", 50, 4)
    g = H.Graph(q)
    seen = []
    real = H.exact_over

    def spy(g_, parts, dp=None):
        seen.append(len(parts))
        return real(g_, parts, dp)

    monkeypatch.setattr(H, "exact_over", spy)
    p = H.uniondp(g, 12, 5)
    assert p.leaves == 50
    assert seen[-1] <= 12 and all(s <= 5 for s in seen[:-1])


def test_uniondp_partition_hand_worked():
    """The partition phase of Algorithm 5 on a 7-relation graph, worked by
    hand from the algorithm's text.  Every card is 10, so an edge weighs
    100 * sel: (0,1) 1, (1,2) 2, (2,3) 3, (4,5) 4, (4,6) 5, (3,4) 50,
    (5,6) 90.  t = 3.

    Edges ordered once, before the loop (all sets single nodes, so by
    weight): (0,1) unites {0,1}; (1,2) makes {0,1,2}; (2,3) would make 4 > 3;
    (4,5) unites {4,5}; (4,6) makes {4,5,6}; (3,4) would make 4; (5,6) is
    inside {4,5,6}.  Partition {0,1,2}, {3}, {4,5,6}.

    Size-first re-picking: (0,1) [sum 2, w 1]; then (2,3) [2, w 3] beats
    (1,2) [3]; then (4,5) [2, w 4]; then (4,6) [3, w 5] (every pair of
    singletons is gone: (3,4) is now 2 + 2); then (1,2) [4] and (3,4) [5]
    are dropped.  Partition {0,1}, {2,3}, {4,5,6}."""
    q = W.Query(n=7, card=[10.0] * 7,
                edges=[(0, 1, 0.01), (1, 2, 0.02), (2, 3, 0.03), (3, 4, 0.5), (4, 5, 0.04), (4, 6, 0.05),
                       (5, 6, 0.9)])
    g = H.Graph(q)
    nodes = [g.leaf(r) for r in range(7)]
    assert H.uniondp_partition(g, nodes, 3) == [[0, 1, 2], [3], [4, 5, 6]]
    assert H.uniondp_partition(g, nodes, 3, order="size_first") == [[0, 1], [2, 3], [4, 5, 6]]
    # t = 2: only pairs; the fixed order takes (0,1), (2,3), (4,5) and
    # leaves 6 alone; size-first does the same here (all sums are 2 first)
    assert H.uniondp_partition(g, nodes, 2) == [[0, 1], [2, 3], [4, 5], [6]]
    assert H.uniondp_partition(g, nodes, 2, order="size_first") == [[0, 1], [2, 3], [4, 5], [6]]
    # the whole UnionDP(k = 4, t = 3): one partition round, then the final
    # exact DP over the three partition plans, so each partition is a
    # subtree of the result
    p = H.uniondp(g, 4, 3)
    assert p.leaves == 7 and cross_product_free(g, p)
    subtrees = set()

    def walk(t):
        subtrees.add(t.rels)
        if not t.is_leaf:
            walk(t.left)
            walk(t.right)

    walk(p)
    assert {0b0000111, 0b0001000, 0b1110000} <= subtrees
    assert H.plan_cost(g, p).cost == p.cost


def _scores_rebuilding(g, p):
    """Scores for g's edges under which the learned start rebuilds the tree-
    query plan p: each join's one cut edge scores its post-order rank (a join
    comes after the joins below it), the other edges score higher."""
    rank = {}

    def walk(t):
        if t.is_leaf:
            return
        walk(t.left)
        walk(t.right)
        cut = g._cut(t.left.rels, t.right.rels, t.left.leaves, t.right.leaves)
        assert len(cut) == 1
        rank[cut[0][:2]] = len(rank)

    walk(p)
    return [float(rank.get((u, v), len(g.edges) + i)) for i, (u, v, _) in enumerate(g.edges)]


@pytest.mark.parametrize("kind,n,seed", [("snowflake", 30, 1), ("chain", 20, 2), ("star", 16, 3)])
def test_learned_start_rebuilds_a_plan_from_its_join_order(kind, n, seed):
    """On a tree query, joins taken in any children-first order of a plan's
    joins rebuild that plan: GOO's, and the exact optimum."""
    q = W.make(kind, n, seed)
    g = H.Graph(q)
    for p in (H.goo(g), H.exact_over(g, [g.leaf(r) for r in range(n)]) if n <= 16 else H.idp2(g, 8)):
        got = H.learned_start(g, _scores_rebuilding(g, p))
        assert H.canonical(got) == H.canonical(p)
        assert got.cost == p.cost


def test_learned_start_orders_by_score_then_edge():
    """Chain 0-1-2-3: equal scores keep the edge order, so (0,1) joins
    before (1,2) and the plan is left-deep; the reverse score order builds
    the mirror image, and scores making (0,1), (2,3) first give the bushy
    plan."""
    q = W.Query(n=4, card=[10.0, 20.0, 30.0, 40.0], edges=[(0, 1, 0.1), (1, 2, 0.1), (2, 3, 0.1)])
    g = H.Graph(q)
    assert H.canonical(H.learned_start(g, [0.0, 0.0, 0.0])) == (((0, 1), 2), 3)
    assert H.canonical(H.learned_start(g, [2.0, 1.0, 0.0])) == (0, (1, (2, 3)))
    bushy = H.learned_start(g, [0.0, 1.0, 0.0])
    assert H.canonical(bushy) == ((0, 1), (2, 3))
    assert bushy.cost == H.plan_cost(g, bushy).cost


def test_learned_start_plans_valid():
    q = W.make("snowflake_plus", 60, 5)
    g = H.Graph(q)
    rng = random.Random(5)
    p = H.learned_start(g, [rng.random() for _ in g.edges])
    assert p.rels == (1 << 60) - 1 and p.leaves == 60
    assert cross_product_free(g, p)
    assert H.plan_cost(g, p).cost == p.cost
