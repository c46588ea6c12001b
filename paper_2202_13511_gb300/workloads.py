"""Seeded synthetic join-graph workloads.

This module is shared by the CUDA path, the CPU oracle tests and the benchmark.
It only draws random numbers and lays out graphs; it holds none of the join
ordering arithmetic (no cardinality products, no costs, no connectivity).

Workload shapes follow the paper's synthetic experiments (Sec. 7.2.1, "Synthetic
Workload"): star graphs (one fact relation joined by every dimension), snowflake
graphs (trees of maximum depth 4), cliques, plus chains and cyclic graphs built
from a random spanning tree with extra edges as stand-ins for the real
MusicBrainz random-walk queries (Sec. 7.2.2), whose data is not available.

Values:
  * base cardinality  card[i] = 10 ** U(2, 8)   (log-uniform in [1e2, 1e8])
  * edge selectivity  sel     = 10 ** U(-6, -1) (log-uniform in [1e-6, 1e-1])
Uniform draws come from SplitMix64 (Steele, Lea, Flood 2014): the top 53 bits of
each 64-bit output divided by 2**53.  ``10 ** x`` is evaluated once here, on the
host, and the resulting doubles are what both implementations consume.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator, written from its published definition."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive), by scaling a uniform double."""
        span = hi - lo + 1
        v = lo + int(self.uniform() * span)
        return min(v, hi)


@dataclass
class Query:
    """A join query graph: relation cardinalities and selectivity-labelled edges."""

    n: int
    card: List[float]
    edges: List[Tuple[int, int, float]]
    kind: str = "custom"
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return len(self.edges)

    def edge_arrays(self):
        """Edges as three parallel lists (u, v, sel)."""
        return ([e[0] for e in self.edges], [e[1] for e in self.edges],
                [e[2] for e in self.edges])


def _draw_cards(rng: SplitMix64, n: int) -> List[float]:
    return [10.0 ** (2.0 + 6.0 * rng.uniform()) for _ in range(n)]


def _draw_sel(rng: SplitMix64) -> float:
    return 10.0 ** (-6.0 + 5.0 * rng.uniform())


def _finish(rng: SplitMix64, n: int, card, pairs, kind, seed, **meta) -> Query:
    edges = [(u, v, _draw_sel(rng)) for (u, v) in pairs]
    return Query(n=n, card=card, edges=edges, kind=kind, seed=seed, meta=meta)


def star(n: int, seed: int = 0) -> Query:
    """Relation 0 is the fact table; relations 1..n-1 each join it."""
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    return _finish(rng, n, card, [(0, i) for i in range(1, n)], "star", seed)


def chain(n: int, seed: int = 0) -> Query:
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    return _finish(rng, n, card, [(i, i + 1) for i in range(n - 1)], "chain", seed)


def cycle(n: int, seed: int = 0) -> Query:
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    pairs = [(i, i + 1) for i in range(n - 1)]
    if n >= 3:
        pairs.append((0, n - 1))
    return _finish(rng, n, card, pairs, "cycle", seed)


def clique(n: int, seed: int = 0) -> Query:
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return _finish(rng, n, card, pairs, "clique", seed)


def _random_tree_pairs(rng: SplitMix64, n: int, max_depth, max_fanout: int = 5):
    """Random rooted tree: node 0 is the root; every node draws a fanout in
    U{1..max_fanout}; each new node attaches to a uniformly chosen node that has
    depth < max_depth and spare fanout.  If none has spare fanout the drawn
    fanouts are lifted to max_fanout; if the depth cap cannot hold n nodes it is
    lifted too (``max_depth=None`` means no cap)."""
    depth = [0]
    fan = [rng.randint(1, max_fanout)]
    kids = [0]
    pairs = []
    for i in range(1, n):
        def ok_depth(j):
            return max_depth is None or depth[j] < max_depth
        cand = [j for j in range(i) if ok_depth(j) and kids[j] < fan[j]]
        if not cand:
            cand = [j for j in range(i) if ok_depth(j) and kids[j] < max_fanout]
        if not cand:
            cand = [j for j in range(i) if kids[j] < max_fanout]
        p = cand[min(int(rng.uniform() * len(cand)), len(cand) - 1)]
        pairs.append((p, i))
        kids[p] += 1
        depth.append(depth[p] + 1)
        fan.append(rng.randint(1, max_fanout))
        kids.append(0)
    return pairs, depth


def snowflake(n: int, seed: int = 0, max_depth=4, max_fanout: int = 5) -> Query:
    """Snowflake / random tree query: tree of depth <= 4, fanout 1..5."""
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    pairs, depth = _random_tree_pairs(rng, n, max_depth, max_fanout)
    return _finish(rng, n, card, pairs, "snowflake", seed, depth=max(depth))


def _pruefer_tree_pairs(rng: SplitMix64, n: int):
    """Uniform random labelled tree from a random Pruefer sequence."""
    if n == 1:
        return []
    if n == 2:
        return [(0, 1)]
    seq = [rng.randint(0, n - 1) for _ in range(n - 2)]
    degree = [1] * n
    for x in seq:
        degree[x] += 1
    pairs = []
    for x in seq:
        leaf = min(j for j in range(n) if degree[j] == 1)
        pairs.append((min(leaf, x), max(leaf, x)))
        degree[leaf] -= 1
        degree[x] -= 1
    rest = [j for j in range(n) if degree[j] == 1]
    pairs.append((rest[0], rest[1]))
    return pairs


def cyclic(n: int, seed: int = 0, p=None) -> Query:
    """Random spanning tree (Pruefer) plus round(p*(n-1)) extra distinct edges,
    p ~ U[0.1, 0.3] unless given."""
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    pairs = _pruefer_tree_pairs(rng, n)
    if p is None:
        p = 0.1 + 0.2 * rng.uniform()
    extra = int(round(p * (n - 1)))
    have = set(pairs)
    max_edges = n * (n - 1) // 2
    extra = min(extra, max_edges - len(have))
    while extra > 0:
        a = rng.randint(0, n - 1)
        b = rng.randint(0, n - 1)
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        if e in have:
            continue
        have.add(e)
        pairs.append(e)
        extra -= 1
    return _finish(rng, n, card, pairs, "cyclic", seed, p=p)


def snowflake_plus(n: int, seed: int = 0, extra_frac: float = 0.05) -> Query:
    """Large-query shape: snowflake (fanout 1..5, depth cap lifted) plus
    extra_frac * n extra random edges."""
    rng = SplitMix64(seed)
    card = _draw_cards(rng, n)
    pairs, _ = _random_tree_pairs(rng, n, None, 5)
    have = set((min(a, b), max(a, b)) for a, b in pairs)
    extra = int(round(extra_frac * n))
    while extra > 0:
        a = rng.randint(0, n - 1)
        b = rng.randint(0, n - 1)
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        if e in have:
            continue
        have.add(e)
        pairs.append(e)
        extra -= 1
    return _finish(rng, n, card, pairs, "snowflake_plus", seed)


def snowflake_plus_pkfk(n: int, seed: int = 0, extra_frac: float = 0.05) -> Query:
    """The snowflake_plus graph with primary-key / foreign-key joins, the
    setting of the paper's heuristic experiments (Sec. 7.3): every edge
    joins a foreign key to the other relation's primary key, so its
    selectivity is 1 / card(key side).  A tree edge's key side is the child;
    an extra edge's is the relation with the larger index."""
    q = snowflake_plus(n, seed, extra_frac)
    edges = [(u, v, 1.0 / q.card[v]) for (u, v, _s) in q.edges]
    return Query(n=n, card=q.card, edges=edges, kind="snowflake_plus_pkfk", seed=seed, meta=q.meta)


def snowflake_schema_pkfk(n: int, seed: int = 0, extra_frac: float = 0.0) -> Query:
    """A snowflake schema with primary-key / foreign-key joins: the same tree
    shapes as snowflake_plus (fanout 1-5, depth uncapped), the fact table
    (relation 0) the largest, card 10^U(6,8), and every dimension smaller
    than the table that references it, card(child) = card(parent) *
    10^-U(0,2) (at least 10).  An edge's selectivity is 1 / card(key side),
    the child for a tree edge, the larger index for an extra edge."""
    rng = SplitMix64(seed)
    pairs, _depth = _random_tree_pairs(rng, n, None, 5)
    parent = {c: p for p, c in pairs}
    card = [0.0] * n
    card[0] = 10.0 ** (6.0 + 2.0 * rng.uniform())
    for i in range(1, n):
        card[i] = max(10.0, card[parent[i]] * 10.0 ** -(2.0 * rng.uniform()))
    have = set((min(a, b), max(a, b)) for a, b in pairs)
    extra = int(round(extra_frac * n))
    while extra > 0:
        a = rng.randint(0, n - 1)
        b = rng.randint(0, n - 1)
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        if e in have:
            continue
        have.add(e)
        pairs.append(e)
        extra -= 1
    edges = [(u, v, 1.0 / card[v]) for (u, v) in pairs]
    return Query(n=n, card=card, edges=edges, kind="snowflake_schema_pkfk", seed=seed)


def uniform_values(n: int, edges_uv, card: float = 1000.0, sel: float = 0.01,
                   kind: str = "uniform") -> Query:
    """All cardinalities and selectivities equal: a case with many exact cost ties."""
    return Query(n=n, card=[card] * n, edges=[(u, v, sel) for (u, v) in edges_uv],
                 kind=kind)


GENERATORS = {
    "star": star,
    "chain": chain,
    "cycle": cycle,
    "clique": clique,
    "snowflake": snowflake,
    "cyclic": cyclic,
    "snowflake_plus": snowflake_plus,
    "snowflake_plus_pkfk": snowflake_plus_pkfk,
    "snowflake_schema_pkfk": snowflake_schema_pkfk,
}


def make(kind: str, n: int, seed: int = 0, **kw) -> Query:
    return GENERATORS[kind](n, seed, **kw)


def mixed_stream(count: int, seed: int = 0, n_lo: int = 8, n_hi: int = 25):
    """Mixed query stream for the batched form: classes star / snowflake / cyclic
    uniformly; sizes in [n_lo, n_hi] with weight 3 for 12..18 and 1 otherwise."""
    rng = SplitMix64(seed ^ 0x5DEECE66D)
    sizes = list(range(n_lo, n_hi + 1))
    weights = [3 if 12 <= s <= 18 else 1 for s in sizes]
    total = sum(weights)
    out = []
    for i in range(count):
        cls = ("star", "snowflake", "cyclic")[min(int(rng.uniform() * 3), 2)]
        u = rng.uniform() * total
        acc = 0
        n = sizes[-1]
        for s, w in zip(sizes, weights):
            acc += w
            if u < acc:
                n = s
                break
        out.append(make(cls, n, seed * 100003 + i))
    return out
