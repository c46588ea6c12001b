"""Writes card_peel.json: card(S) of every connected set of a small cyclic
join graph, by the peeling reading of card(S) (the paper leaves card(S)
unspecified; Sec. 2.1 defines C_out over the cardinalities of the joins):

    card({r}) = card[r];  for |S| >= 2, v = the highest-index relation of S
    whose removal leaves G[S \\ {v}] connected, and
    card(S) = (((card(S \\ {v}) * card[v]) * sel(j1, v)) * sel(j2, v)) ...
    over the neighbours j1 < j2 < ... of v in S,

every product one IEEE binary64 multiplication rounded to nearest (even).
Each product is formed exactly as a fraction and rounded once
(float(Fraction) rounds correctly), so nothing here depends on a
floating-point unit or on the oracle's C code.

The script also checks that the graph and values make the pin sharp: peeling
the lowest non-cut vertex instead, taking v's selectivities in descending
order, or multiplying all cards then all selectivities in ascending order
each change the bits of some card(S).  Run from the repository root:
    python tests/golden/make_card_peel.py
"""
import json
import os
import random
from fractions import Fraction

N = 7
EDGES = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 5), (3, 5), (5, 6), (1, 4)]


def mul(a: float, b: float) -> float:
    return float(Fraction(a) * Fraction(b))


def values(seed=2202):
    rng = random.Random(seed)
    card = [float(10 ** rng.uniform(2, 8)) for _ in range(N)]
    sel = {e: float(10 ** rng.uniform(-6, -1)) for e in EDGES}
    return card, sel


def adj_of():
    adj = [0] * N
    for u, v in EDGES:
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    return adj


def connected(s, adj):
    if s == 0:
        return False
    seen = front = s & -s
    while front:
        x = (front & -front).bit_length() - 1
        front &= front - 1
        nb = adj[x] & s & ~seen
        seen |= nb
        front |= nb
    return seen == s


def card_of(s, card, sel, adj, memo, peel="highest", sel_order="ascending"):
    if s in memo:
        return memo[s]
    members = [i for i in range(N) if s >> i & 1]
    if len(members) == 1:
        memo[s] = card[members[0]]
        return memo[s]
    noncut = [v for v in members if connected(s & ~(1 << v), adj)]
    v = max(noncut) if peel == "highest" else min(noncut)
    p = card_of(s & ~(1 << v), card, sel, adj, memo, peel, sel_order)
    p = mul(p, card[v])
    nbrs = sorted(j for j in members if adj[v] >> j & 1)
    if sel_order == "descending":
        nbrs.reverse()
    for j in nbrs:
        p = mul(p, sel[(min(j, v), max(j, v))])
    memo[s] = p
    return p


def ascending_product(s, card, sel):
    p = 1.0
    for r in range(N):
        if s >> r & 1:
            p = mul(p, card[r])
    for (u, v) in sorted(EDGES):
        if s >> u & 1 and s >> v & 1:
            p = mul(p, sel[(u, v)])
    return p


def main():
    card, sel = values()
    adj = adj_of()
    sets = [s for s in range(1, 1 << N) if connected(s, adj)]
    ref = {}
    for s in sets:
        card_of(s, card, sel, adj, ref)
    for kw in (dict(peel="lowest"), dict(sel_order="descending")):
        alt = {}
        differ = sum(card_of(s, card, sel, adj, alt, **kw) != ref[s] for s in sets)
        assert differ > 0, kw
    assert any(ascending_product(s, card, sel) != ref[s] for s in sets)
    out = {
        "source": "card(S) by peeling, the reading of the unspecified card(S) (Sec. 2.1 C_out); "
                  "exact products rounded once each to binary64 (nearest even)",
        "n": N,
        "card": [c.hex() for c in card],
        "edges": [[u, v, sel[(u, v)].hex()] for (u, v) in EDGES],
        "card_of_set": {str(s): ref[s].hex() for s in sets},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "card_peel.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"{len(sets)} connected sets written to {path}")


if __name__ == "__main__":
    main()
