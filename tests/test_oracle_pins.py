"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute force
over every join tree, closed-form counts, numbers printed in the paper, exact
products of powers of two, and two independent DP formulations.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2202_13511_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

KINDS = ["star", "chain", "cycle", "clique", "snowflake", "cyclic"]


def mask(rels, base=0):
    m = 0
    for r in rels:
        m |= 1 << (r - base)
    return m


# -- brute force over every cross-product-free bushy tree ------------------

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_dp_matches_brute_force(kind, n):
    """Principle of optimality under IEEE round-to-nearest: addition is
    monotone, so the DP optimum equals the minimum over every join tree
    exactly, and the recursive (cost, left) rule picks the same tree."""
    for seed in range(3 if n <= 6 else 1):
        q = W.make(kind, n, seed=seed)
        bc, bsig, ntrees = oracle.brute_force(q)
        for res in (oracle.dpsub(q), oracle.dpccp(q)):
            assert res.opt_cost == bc
            assert oracle.plan_signature(oracle.plan_from_memo(q, res)) == bsig


def test_brute_force_tree_counts():
    """Number of cross-product-free bushy trees (unordered children) that the
    brute force enumerates: a clique allows every bushy tree, (2n-3)!!; a
    chain allows one tree per full bracketing, Catalan(n-1); a star allows
    (n-1)! (every join adds one dimension to the side holding the hub)."""
    for n in range(2, 8):
        _, _, t = oracle.brute_force(W.clique(n, 0))
        assert t == math.prod(range(1, 2 * n - 2, 2))
        _, _, t = oracle.brute_force(W.star(n, 0))
        assert t == math.factorial(n - 1)
        _, _, t = oracle.brute_force(W.chain(n, 0))
        # unordered trees over a path: the Catalan number C_{n-1}
        assert t == math.comb(2 * (n - 1), n - 1) // n


@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_ties_all_equal_values(n):
    """All cardinalities and selectivities equal: many exact cost ties; the
    DP's tie rule must still pick exactly the brute-force tree."""
    for kind in ("star", "clique", "cycle", "chain"):
        base = W.make(kind, n, 0)
        q = W.uniform_values(n, [(u, v) for (u, v, _s) in base.edges], card=1000.0, sel=0.01)
        bc, bsig, _ = oracle.brute_force(q)
        for res in (oracle.dpsub(q), oracle.dpccp(q)):
            assert res.opt_cost == bc
            assert oracle.plan_signature(oracle.plan_from_memo(q, res)) == bsig


# -- closed-form counts ----------------------------------------------------

@pytest.mark.parametrize("n", range(2, 15))
def test_closed_form_counts(n):
    """Unordered CCP pairs: chain (n^3-n)/6, star (n-1)2^(n-2),
    clique (3^n - 2^(n+1) + 1)/2.  Connected sets (all sizes): chain
    n(n+1)/2, star 2^(n-1)+n-1, clique 2^n - 1."""
    cases = {
        "chain": ((n ** 3 - n) // 6, n * (n + 1) // 2),
        "star": ((n - 1) * 2 ** (n - 2), 2 ** (n - 1) + n - 1),
        "clique": ((3 ** n - 2 ** (n + 1) + 1) // 2, 2 ** n - 1),
    }
    for kind, (ccp, conn) in cases.items():
        q = W.make(kind, n, 0)
        res = oracle.dpccp(q)
        assert int(res.ccp.sum()) == ccp
        assert int(res.connected.sum()) == conn
        if n <= 12:
            r2 = oracle.dpsub(q)
            assert int(r2.ccp.sum()) == ccp
            assert int(r2.connected.sum()) == conn


@pytest.mark.parametrize("n", range(2, 13))
def test_per_level_counts(n):
    """Level k: a chain has n-k+1 connected k-sets, a star C(n-1,k-1) (k>=2),
    a clique C(n,k)."""
    for kind, f in (("chain", lambda k: n - k + 1),
                    ("star", lambda k: math.comb(n - 1, k - 1)),
                    ("clique", lambda k: math.comb(n, k))):
        res = oracle.dpsub(W.make(kind, n, 0))
        for k in range(2, n + 1):
            assert int(res.connected[k]) == f(k)


@pytest.mark.parametrize("n", range(2, 13))
def test_dpsub_evaluated_on_stars(n):
    """Algorithm 1 visits every subset of every connected S; on a star that is
    sum_{i>=2} C(n-1,i-1) 2^i = 2(3^(n-1) - 1)."""
    res = oracle.dpsub(W.star(n, 0))
    assert int(res.evaluated.sum()) == 2 * (3 ** (n - 1) - 1)


def test_printed_2805_ratio():
    """Sec. 2.3 / Sec. 7.2.1 print ~2805x more join pairs evaluated by DPSUB
    than CCP pairs at 25 relations (star).  With the two closed forms pinned
    above, the ratio is 2(3^24-1) / (24 * 2^23)."""
    g = json.load(open(os.path.join(GOLDEN, "printed_ratios.json")))
    n = g["star_25_dpsub_evaluated_over_ccp"]["relations"]
    ratio = 2 * (3 ** (n - 1) - 1) / ((n - 1) * 2 ** (n - 2))
    assert int(ratio) == g["star_25_dpsub_evaluated_over_ccp"]["printed"]


# -- the two DP formulations agree ----------------------------------------

@pytest.mark.parametrize("kind", KINDS)
def test_dpsub_equals_dpccp(kind):
    """Every connected set's (cost, left) is identical under DPSUB
    (Algorithm 1) and DPCCP: the memo is the plain definition."""
    for n in (8, 11, 14):
        for seed in range(2):
            q = W.make(kind, n, seed=seed)
            a, b = oracle.dpsub(q), oracle.dpccp(q)
            fa, fb = np.isfinite(a.cost), np.isfinite(b.cost)
            assert np.array_equal(fa, fb)
            assert np.array_equal(a.cost[fa], b.cost[fa])
            assert np.array_equal(a.left[fa], b.left[fa])
            assert np.array_equal(a.ccp, b.ccp)
            assert np.array_equal(a.connected, b.connected)


# -- card(S) ----------------------------------------------------------------

def test_card_exact_powers_of_two():
    """With powers-of-two inputs every product is exact, so card(S) must equal
    2^(sum of the exponents of S's cardinalities and of the selectivities of
    the edges inside S): a dropped or extra factor changes the value."""
    rng = W.SplitMix64(7)
    for trial in range(30):
        base = W.cyclic(9, seed=trial)
        ce = [rng.randint(1, 20) for _ in range(base.n)]
        se = [-rng.randint(1, 10) for _ in base.edges]
        q = W.Query(n=base.n, card=[2.0 ** e for e in ce],
                    edges=[(u, v, 2.0 ** s) for (u, v, _), s in zip(base.edges, se)])
        for s in range(1, 1 << q.n, 37):
            exp = sum(ce[i] for i in range(q.n) if s >> i & 1)
            exp += sum(x for (u, v, _), x in zip(q.edges, se) if (s >> u & 1) and (s >> v & 1))
            assert oracle.card(q, s) == 2.0 ** exp


def test_card_error_bound():
    """card(S) is within the sequential-product rounding bound of the exact
    rational product: |p - P| <= ((1+u)^(f-1) - 1) |P|, u = 2^-53."""
    u = Fraction(1, 2 ** 53)
    for seed in range(5):
        q = W.clique(10, seed=seed)
        for s in range(3, 1 << q.n, 97):
            exact = Fraction(1)
            f = 0
            for i in range(q.n):
                if s >> i & 1:
                    exact *= Fraction(q.card[i])
                    f += 1
            for (a, b, sel) in q.edges:
                if (s >> a & 1) and (s >> b & 1):
                    exact *= Fraction(sel)
                    f += 1
            got = Fraction(oracle.card(q, s))
            assert abs(got - exact) <= ((1 + u) ** (f - 1) - 1) * exact


# -- graph notions on the paper's Fig. 5 example -------------------------

def _fig5():
    g = json.load(open(os.path.join(GOLDEN, "fig5_graph.json")))
    edges = [(a - 1, b - 1, 0.5) for (a, b) in g["edges_paper_labels"]]
    q = W.Query(n=9, card=[10.0] * 9, edges=edges, kind="fig5")
    return g, q


def test_fig5_blocks_and_cut_vertices():
    g, q = _fig5()
    full = (1 << 9) - 1
    blocks, cuts = oracle.blocks(q, full)
    assert cuts == mask(g["printed"]["cut_vertices"], 1)
    assert sorted(blocks) == sorted(mask(b, 1) for b in g["printed"]["blocks"])
    e = mask(g["printed"]["edge_in_cycle"], 1)
    assert any((b & e) == e and bin(b).count("1") >= 3 for b in blocks)


def test_fig5_grow_example():
    g, q = _fig5()
    p = g["printed"]
    assert oracle.grow(q, mask(p["grow_source"], 1), mask(p["grow_restriction"], 1)) == \
        mask(p["grow_result"], 1)


def test_fig5_512_to_32():
    """DPSUB visits 2^9 = 512 subsets of the full set (Algorithm 1); the block
    loop of Algorithm 4 visits every non-empty proper lb of each block, i.e.
    twice each unordered bipartition: 2 * sum_B (2^(|B|-1) - 1) = 32."""
    g, q = _fig5()
    res = oracle.dpsub(q)
    assert int(res.evaluated[9]) == g["printed"]["dpsub_subsets_full_set"]
    ev, va = oracle.block_enum_counts(q)
    assert 2 * int(ev[9]) == g["printed"]["mpdp_subsets_full_set"]


# -- lemma invariants of the block-based enumeration ----------------------

@pytest.mark.parametrize("kind", KINDS)
def test_block_enumeration_lemmas(kind):
    """Sec. 3.2.2-3.2.3: every CCP pair arises from exactly one block
    bipartition that passes the CCP block (so the valid count equals the CCP
    count found by DPSUB's subset loop); evaluated >= valid; evaluated equals
    the CCP count when every block is a clique (trees, cliques)."""
    for n in (5, 8, 10):
        for seed in range(2):
            q = W.make(kind, n, seed=seed)
            ev, va = oracle.block_enum_counts(q)
            res = oracle.dpsub(q)
            assert np.array_equal(va, res.ccp)
            assert (ev >= va).all()
            if kind in ("star", "chain", "snowflake", "clique"):
                assert np.array_equal(ev, va)
            # DPSUB evaluates at least twice as many (Lemma "complexity")
            assert (res.evaluated[2:] >= 2 * ev[2:]).all()


# -- input validation ------------------------------------------------------

def test_invalid_inputs_rejected():
    q = W.chain(4, 0)
    bad = [
        W.Query(n=4, card=q.card, edges=q.edges + [(0, 1, 0.5)]),          # duplicate
        W.Query(n=4, card=q.card, edges=q.edges + [(2, 2, 0.5)]),          # self loop
        W.Query(n=4, card=q.card, edges=q.edges[:-1] + [(2, 3, 1.5)]),     # sel > 1
        W.Query(n=4, card=[1.0, -1.0, 1.0, 1.0], edges=q.edges),           # card <= 0
        W.Query(n=4, card=q.card, edges=q.edges[:-1] + [(2, 7, 0.5)]),     # bad index
    ]
    for b in bad:
        with pytest.raises(oracle.OracleError) as ei:
            oracle.dpccp(b)
        assert ei.value.code == oracle.OR_INVALID
    with pytest.raises(oracle.OracleError) as ei:
        oracle.dpccp(W.Query(n=4, card=q.card, edges=q.edges[:2]))
    assert ei.value.code == oracle.OR_DISCONNECTED


# -- card(S): the peeling order, bit for bit --------------------------------

def card_peel_golden():
    g = json.load(open(os.path.join(GOLDEN, "card_peel.json")))
    q = W.Query(n=g["n"], card=[float.fromhex(c) for c in g["card"]],
                edges=[(u, v, float.fromhex(sel)) for u, v, sel in g["edges"]])
    return q, {int(k): float.fromhex(v) for k, v in g["card_of_set"].items()}


def test_card_peel_order_golden():
    """card(S) of every connected set of a 7-relation cyclic graph equals,
    bit for bit, the values tests/golden/make_card_peel.py computed with
    exact fractions and one rounding per product.  That script checks that
    peeling the lowest non-cut vertex, descending selectivities or the
    plain ascending product each change some of these bits."""
    q, want = card_peel_golden()
    assert len(want) == 61
    for s, c in want.items():
        assert oracle.card(q, s).hex() == c.hex(), (bin(s), oracle.card(q, s).hex(), c.hex())
