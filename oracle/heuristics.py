"""Oracle for the heuristic modes (paper Sec. 4): GOO, IDP2 and UnionDP over
the exact DP in extended range (``xd_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain Python, slow on
purpose, written to be read against Sec. 4.1 (IDP2), Algorithm 5 (UnionDP)
and the GOO description of Sec. 7.3.

Values are extended-range ("XD") pairs (m, e) meaning m * 2^e, with m = 0 or
1 <= m < 2.  The operations are the ones xd_oracle.c documents, written again
here in Python, which has binary64 floats with round to nearest.

Readings where the paper is silent (the product path follows the same ones):
  * card of a join of two plans L and R: ((card(L) * card(R)) * sel(e1)) *
    sel(e2) ... over the query edges between L's and R's relations, in
    ascending (min(u, v), max(u, v)).  cost(leaf) = 0 and cost(L join R) =
    (cost(L) + cost(R)) + card(L join R) (C_out).  A plan's reported cost is
    this value over its whole tree.
  * a sub-problem over plans P_1..P_m (IDP2's subtree leaves, a UnionDP
    partition or the final graph) numbers the plans by their smallest base
    relation.  Relation i has card(P_i).  There is one edge (i, j) whenever
    query edges join P_i and P_j, with sel the product of those edges' sels
    in the order above.  The exact DP (peeling card, (x, left) rule) picks
    the plan over P_1..P_m.
  * GOO (Fegaras, as the paper uses it for IDP2's initial plan): while more
    than one tree remains, join the two trees, connected by a query edge,
    whose join has the least card.  Ties go to the pair with the least
    (smallest relation of the pair, smallest relation of the other tree).
    The tree holding the smaller relation goes on the left.
  * IDP2(k): T = GOO.  While T has more than one leaf, pick the subtree T'
    with 2..k leaves (plans count as one leaf) whose joins cost most: C(T')
    is the C_out of T' with its leaves at cost 0, because re-planning T'
    cannot change its leaves.  Ties go to the first in pre-order (left
    first).  Re-plan T' with the exact DP over its leaves and replace it by
    the resulting plan, a single leaf.
  * UnionDP(k, t) (Algorithm 5): if the graph has at most k nodes, the
    exact DP over all of them.  Otherwise each edge weighs the card of
    joining its two nodes, and union-find runs over the nodes (size =
    number of nodes).  The edges are ordered once, before the union loop,
    by (size of the sets across the edge, weight, smaller node, larger
    node).  Every set is a single node when the order is fixed, so the
    order is increasing weight (Kruskal's order).  One pass over that
    order unites the two sets across an edge when they differ and their
    size sum is at most t.  Each set of two or more nodes is re-planned
    with the exact DP.  The sets become the nodes of the next graph
    (numbered by smallest base relation) and the procedure recurses.
    Algorithm 5 has a single bound k.  The paper runs UnionDP with k = 25
    and a partition threshold t = 15 (Sec. 7.3), which is read here as
    partitions <= t and the final DP at <= k nodes.
  * UnionDP, size-first variant (order="size_first"): the same, except
    that the next edge is re-picked after every union as the one with the
    least (current size sum, weight, smaller node, larger node), and an
    edge whose sum exceeds t is dropped.  This evaluates the ordering key
    on the current sets instead of fixing it before the loop.  It is kept
    as a comparison; Table 1's ranking (UnionDP best on snowflakes,
    because it removes single expensive edges, Sec. 7.3) supports the
    fixed order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import xd_dp

XD = Tuple[float, int]
ZERO: XD = (0.0, 0)


def xd(c: float, e: int = 0) -> XD:
    """c * 2^e for a finite c >= 0, normalised."""
    if c == 0.0:
        return ZERO
    f, ex = math.frexp(c)  # c = f * 2^ex, 0.5 <= f < 1
    return (f * 2.0, e + ex - 1)


def xd_mul(a: XD, b: XD) -> XD:
    if a[0] == 0.0 or b[0] == 0.0:
        return ZERO
    m, e = a[0] * b[0], a[1] + b[1]
    if m >= 2.0:
        m, e = m * 0.5, e + 1
    return (m, e)


def xd_add(a: XD, b: XD) -> XD:
    if a[0] == 0.0:
        return b
    if b[0] == 0.0:
        return a
    if a[1] < b[1]:
        a, b = b, a
    d = a[1] - b[1]
    m = a[0] + math.ldexp(b[0], -d) if d <= 60 else a[0]
    e = a[1]
    if m >= 2.0:
        m, e = m * 0.5, e + 1
    return (m, e)


def xd_key(a: XD):
    """Sort key realising the XD order (0 smallest, then exponent, mantissa)."""
    return (0,) if a[0] == 0.0 else (1, a[1], a[0])


def xd_float(a: XD) -> float:
    """The value as a binary64 (inf when out of range)."""
    try:
        return math.ldexp(a[0], a[1])
    except OverflowError:
        return math.inf


# ---------------------------------------------------------------------------
# Plans

@dataclass
class Plan:
    left: Optional["Plan"] = None
    right: Optional["Plan"] = None
    rel: int = -1
    rels: int = 0            # bitmap of base relations (Python int)
    minrel: int = 0
    leaves: int = 1          # base relations below
    card: XD = ZERO
    cost: XD = ZERO          # C_out of the whole subtree

    @property
    def is_leaf(self) -> bool:
        return self.left is None


class Graph:
    """The query: base cards (XD) and edges, with per-pair edge lists."""

    def __init__(self, q):
        self.n = int(q.n)
        self.card = [xd(float(c)) for c in q.card]
        self.edges = sorted((min(u, v), max(u, v), float(s)) for (u, v, s) in q.edges)
        self.adj: List[List[Tuple[int, float]]] = [[] for _ in range(self.n)]
        for u, v, s in self.edges:
            self.adj[u].append((v, s))
            self.adj[v].append((u, s))

    def leaf(self, r: int) -> Plan:
        return Plan(rel=r, rels=1 << r, minrel=r, leaves=1, card=self.card[r], cost=ZERO)

    def _cut(self, a: int, b: int, na: int, nb: int):
        """Query edges between relation sets a and b, as (min, max, sel) in
        ascending order (scanning the smaller side)."""
        if nb < na:
            a, b = b, a
        out = []
        x = a
        while x:
            low = x & -x
            u = low.bit_length() - 1
            x ^= low
            for v, s in self.adj[u]:
                if (b >> v) & 1:
                    out.append((min(u, v), max(u, v), s))
        out.sort()
        return out

    def cut_sel(self, a: int, b: int, na: int = 0, nb: int = 0) -> Optional[XD]:
        """Product of the sels of the edges between relation sets a and b (in
        ascending (u, v)), or None when no edge joins them."""
        p = None
        for _, _, s in self._cut(a, b, na, nb):
            p = xd(s) if p is None else xd_mul(p, xd(s))
        return p

    def join(self, l: Plan, r: Plan) -> Plan:
        """The join node of two plans (left = the one with the smaller relation)."""
        if r.minrel < l.minrel:
            l, r = r, l
        c = xd_mul(l.card, r.card)
        for _, _, s in self._cut(l.rels, r.rels, l.leaves, r.leaves):
            c = xd_mul(c, xd(s))
        return Plan(left=l, right=r, rels=l.rels | r.rels, minrel=l.minrel, leaves=l.leaves + r.leaves,
                    card=c, cost=xd_add(xd_add(l.cost, r.cost), c))


def canonical(p: Plan):
    """Shape of a plan as nested pairs of relation ids, children ordered by
    their smallest relation."""
    if p.is_leaf:
        return p.rel
    a, b = canonical(p.left), canonical(p.right)
    return (a, b) if p.left.minrel < p.right.minrel else (b, a)


def plan_cost(g: Graph, p: Plan) -> Plan:
    """Recompute cards and costs bottom-up (the reported cost)."""
    if p.is_leaf:
        return g.leaf(p.rel)
    return g.join(plan_cost(g, p.left), plan_cost(g, p.right))


# ---------------------------------------------------------------------------
# Sub-problems over plans, solved by the exact DP in extended range

def exact_over(g: Graph, parts: Sequence[Plan], dp=None) -> Plan:
    """The optimal plan over the given plans (each one a relation of the
    sub-problem), as the exact DP picks it; then expanded."""
    parts = sorted(parts, key=lambda p: p.minrel)
    m = len(parts)
    if m == 1:
        return parts[0]
    cards = [p.card for p in parts]
    edges = []
    for i in range(m):
        for j in range(i + 1, m):
            s = g.cut_sel(parts[i].rels, parts[j].rels, parts[i].leaves, parts[j].leaves)
            if s is not None:
                edges.append((i, j, s))
    left = (dp or _oracle_dp)(m, cards, edges)

    def build(s: int) -> Plan:
        if s & (s - 1) == 0:
            return parts[s.bit_length() - 1]
        l = int(left[s])
        return g.join(build(l), build(s ^ l))

    return build((1 << m) - 1)


def _oracle_dp(m, cards, edges):
    return xd_dp(m, cards, edges, "dpccp").left


# ---------------------------------------------------------------------------
# GOO

def goo(g: Graph) -> Plan:
    trees: Dict[int, Plan] = {r: g.leaf(r) for r in range(g.n)}  # keyed by minrel
    owner = list(range(g.n))
    while len(trees) > 1:
        best = None
        seen = set()
        for u, v, _ in g.edges:
            a, b = owner[u], owner[v]
            if a == b:
                continue
            pair = (min(a, b), max(a, b))
            if pair in seen:
                continue
            seen.add(pair)
            j = g.join(trees[pair[0]], trees[pair[1]])
            key = (xd_key(j.card), pair[0], pair[1])
            if best is None or key < best[0]:
                best = (key, pair, j)
        _, (a, b), j = best
        del trees[a], trees[b]
        trees[j.minrel] = j
        for r in range(g.n):
            if (j.rels >> r) & 1:
                owner[r] = j.minrel
    return next(iter(trees.values()))


# ---------------------------------------------------------------------------
# Learned start for IDP2 (a project addition): edges in ascending score

def learned_start(g: Graph, scores: Sequence[float]) -> Plan:
    """The plan that takes the query's edges (g.edges order) in ascending
    score, equal scores in edge order, and joins the plans of each edge's two
    ends while they are still apart.  The scores are the model's outputs,
    given as inputs here."""
    assert len(scores) == len(g.edges)
    order = sorted(range(len(g.edges)), key=lambda e: (scores[e], e))
    comp = list(range(g.n))          # relation -> component id
    plans = {r: g.leaf(r) for r in range(g.n)}
    for e in order:
        u, v, _ = g.edges[e]
        a, b = comp[u], comp[v]
        if a == b:
            continue
        j = g.join(plans.pop(a), plans.pop(b))
        plans[a] = j
        for r in range(g.n):
            if comp[r] == b:
                comp[r] = a
    assert len(plans) == 1
    return next(iter(plans.values()))


# ---------------------------------------------------------------------------
# IDP2

def _joins_cost(t: Plan) -> XD:
    """C_out of a subtree with its leaves at cost 0."""
    if t.is_leaf:
        return ZERO
    return xd_add(xd_add(_joins_cost(t.left), _joins_cost(t.right)), t.card)


def idp2(g: Graph, k: int, dp=None, start: Optional[Plan] = None) -> Plan:
    """IDP2 with GOO's plan as the start (or `start`).  The working tree's
    leaves are base relations or re-planned subtrees (opaque plans)."""
    # working tree nodes: ["leaf", plan] or ["join", left, right]; annotated
    # per pass with (plan, leaf count, joins-only cost)
    def wrap(p: Plan):
        return ["leaf", p] if p.is_leaf else ["join", wrap(p.left), wrap(p.right)]

    def annotate(w):
        if w[0] == "leaf":
            return w[1], 1, ZERO, [w[1]]
        pl, nl, cl, ll = annotate(w[1])
        pr, nr, cr, lr = annotate(w[2])
        p = g.join(pl, pr)
        return p, nl + nr, xd_add(xd_add(cl, cr), p.card), ll + lr

    w = wrap(start if start is not None else goo(g))
    while w[0] != "leaf":
        best = None  # (key, node)

        def visit(node):
            nonlocal best
            if node[0] == "leaf":
                return None
            info = annotate(node)
            if info[1] <= k and (best is None or xd_key(info[2]) > best[0]):
                best = (xd_key(info[2]), node, info[3])
            visit(node[1])
            visit(node[2])

        visit(w)
        _, node, parts = best
        re = exact_over(g, parts, dp)
        node[:] = ["leaf", re]
    return w[1]


# ---------------------------------------------------------------------------
# UnionDP

def uniondp_partition(g: Graph, nodes: Sequence[Plan], t: int, order: str = "paper") -> List[List[int]]:
    """The partition phase of Algorithm 5 over the current nodes: groups of
    node indices (each ascending), ordered by their first index."""
    m = len(nodes)
    edges = []
    for i in range(m):
        for j in range(i + 1, m):
            s = g.cut_sel(nodes[i].rels, nodes[j].rels, nodes[i].leaves, nodes[j].leaves)
            if s is not None:
                w = xd_mul(xd_mul(nodes[i].card, nodes[j].card), s)
                edges.append((i, j, w))
    parent = list(range(m))
    size = [1] * m

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    if order == "paper":
        # the order is fixed before the loop, when every set is one node
        ranked = sorted(edges, key=lambda e: (size[e[0]] + size[e[1]], xd_key(e[2]), e[0], e[1]))
        for i, j, _ in ranked:
            a, b = find(i), find(j)
            if a != b and size[a] + size[b] <= t:
                parent[b] = a
                size[a] += size[b]
    elif order == "size_first":
        dropped = set()
        while True:
            best = None
            for idx, (i, j, w) in enumerate(edges):
                if idx in dropped:
                    continue
                a, b = find(i), find(j)
                if a == b:
                    continue
                key = (size[a] + size[b], xd_key(w), i, j)
                if best is None or key < best[0]:
                    best = (key, idx, a, b)
            if best is None:
                break
            (ssum, _, _, _), idx, a, b = best
            if ssum <= t:
                parent[b] = a
                size[a] += size[b]
            else:
                dropped.add(idx)
    else:
        raise ValueError(order)
    groups: Dict[int, List[int]] = {}
    for i in range(m):
        groups.setdefault(find(i), []).append(i)
    return sorted(groups.values(), key=lambda grp: grp[0])


def uniondp(g: Graph, k: int, t: Optional[int] = None, dp=None, order: str = "paper") -> Plan:
    t = k if t is None else t
    nodes = [g.leaf(r) for r in range(g.n)]
    while len(nodes) > k:
        groups = uniondp_partition(g, nodes, t, order)
        nodes = sorted((exact_over(g, [nodes[i] for i in grp], dp) for grp in groups), key=lambda p: p.minrel)
    return exact_over(g, nodes, dp)
