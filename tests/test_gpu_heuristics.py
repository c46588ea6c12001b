"""Heuristic modes on the GPU (IDP2, UnionDP, GOO through IDP2 with k = 1)
against the oracle's drivers: the same plan (canonical shape) and the same
extended-range cost, bit for bit."""
import numpy as np
import pytest

from oracle import heuristics as H
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opt():
    o = mpdp.Optimizer(0)
    yield o
    o.close()


def shape_from_nodes(nodes):
    """The plan as the set of its join nodes' relation sets (Python ints;
    they identify a binary plan tree), from a breadth-first node array
    whose children follow their parent; no recursion, so plans of any
    depth work."""
    sets = [0] * len(nodes)
    for i in range(len(nodes) - 1, -1, -1):
        nd = nodes[i]
        if nd["left"] < 0:
            sets[i] = 1 << int(nd["rel"])
        else:
            sets[i] = sets[int(nd["left"])] | sets[int(nd["right"])]
    return frozenset(sets[i] for i in range(len(nodes)) if nodes[i]["left"] >= 0)


def shape_of_plan(p):
    """The same form for an oracle plan."""
    out, stack = set(), [p]
    while stack:
        t = stack.pop()
        if not t.is_leaf:
            out.add(t.rels)
            stack.extend((t.left, t.right))
    return frozenset(out)


def run(opt, q, mode, k, t=0):
    p = opt.optimize(q, mode=mode, k=k, t=t)
    assert len(p.nodes) == 2 * q.n - 1
    return shape_from_nodes(p.nodes), p.cost_xd


def ref(q, mode, k, t=0):
    g = H.Graph(q)
    if mode == mpdp.MODE_IDP2:
        p = H.goo(g) if k <= 1 else H.idp2(g, k)
    elif mode == mpdp.MODE_UNIONDP_SIZEFIRST:
        p = H.uniondp(g, k, t or k, order="size_first")
    else:
        p = H.uniondp(g, k, t or k)
    return shape_of_plan(p), p.cost


def same(got, want):
    assert got[0] == want[0]
    assert got[1] == want[1], (got[1], want[1])


@pytest.mark.parametrize("kind,n,seed", [("snowflake", 18, 1), ("cyclic", 16, 2), ("star", 14, 3)])
def test_k_at_least_n_gives_exact_plan(opt, kind, n, seed):
    q = W.make(kind, n, seed)
    exact = opt.optimize(q)
    for mode in (mpdp.MODE_IDP2, mpdp.MODE_UNIONDP):
        shape, cost = run(opt, q, mode, n)
        assert shape == shape_from_nodes(exact.nodes)
        same((shape, cost), ref(q, mode, n))


CASES = [
    ("snowflake_plus", 40, 1, mpdp.MODE_IDP2, 1, 0),    # GOO
    ("snowflake_plus", 40, 1, mpdp.MODE_IDP2, 8, 0),
    ("snowflake_plus", 60, 2, mpdp.MODE_IDP2, 10, 0),
    ("snowflake_plus", 60, 2, mpdp.MODE_UNIONDP, 10, 6),
    ("snowflake_plus", 100, 3, mpdp.MODE_UNIONDP, 12, 8),
    ("snowflake_plus", 100, 4, mpdp.MODE_IDP2, 12, 0),
    ("star", 30, 5, mpdp.MODE_IDP2, 10, 0),
    ("star", 30, 5, mpdp.MODE_UNIONDP, 10, 5),
    ("cyclic", 24, 6, mpdp.MODE_UNIONDP, 8, 4),
    ("snowflake_plus", 60, 2, mpdp.MODE_UNIONDP_SIZEFIRST, 10, 6),
    ("snowflake_plus_pkfk", 80, 8, mpdp.MODE_UNIONDP, 12, 6),
    ("snowflake_plus_pkfk", 80, 8, mpdp.MODE_UNIONDP_SIZEFIRST, 12, 6),
    ("star", 30, 5, mpdp.MODE_UNIONDP_SIZEFIRST, 10, 5),
    ("cyclic", 24, 6, mpdp.MODE_UNIONDP_SIZEFIRST, 8, 4),
]


@pytest.mark.parametrize("kind,n,seed,mode,k,t", CASES)
def test_heuristic_matches_oracle(opt, kind, n, seed, mode, k, t):
    q = W.make(kind, n, seed)
    same(run(opt, q, mode, k, t), ref(q, mode, k, t))


@pytest.mark.parametrize("mode,k,t", [(mpdp.MODE_IDP2, 25, 0), (mpdp.MODE_UNIONDP, 25, 15),
                                     (mpdp.MODE_UNIONDP_SIZEFIRST, 25, 15)])
def test_paper_parameters_at_100_relations(opt, mode, k, t):
    q = W.make("snowflake_plus", 100, 11)
    same(run(opt, q, mode, k, t), ref(q, mode, k, t))


@pytest.mark.parametrize("kind,n,seed,mode,k,t", [
    ("snowflake_plus", 300, 12, mpdp.MODE_IDP2, 25, 0),
    ("snowflake_plus", 300, 12, mpdp.MODE_UNIONDP, 25, 15),
    ("snowflake_plus_pkfk", 300, 14, mpdp.MODE_IDP2, 25, 0),
    ("snowflake_plus", 1000, 11, mpdp.MODE_IDP2, 25, 0),
    ("snowflake_plus_pkfk", 1000, 13, mpdp.MODE_UNIONDP, 25, 15),
    ("snowflake_plus_pkfk", 1000, 13, mpdp.MODE_UNIONDP_SIZEFIRST, 25, 15),
])
def test_paper_parameters_at_300_and_1000_relations(opt, kind, n, seed, mode, k, t):
    """The large-query sizes of the heuristic tables (Sec. 7.3): hundreds of
    IDP2 rounds and several levels of UnionDP recursion, every plan and
    extended-range cost equal to the oracle's."""
    q = W.make(kind, n, seed)
    same(run(opt, q, mode, k, t), ref(q, mode, k, t))


def test_out_of_binary64_range(opt):
    """Cards near 1e100: every sub-problem is far beyond binary64, the plan
    cost is reported in extended range."""
    base = W.make("snowflake_plus", 45, 7)
    q = W.Query(n=base.n, card=[c * 1e100 for c in base.card], edges=base.edges)
    for mode, k, t in ((mpdp.MODE_IDP2, 9, 0), (mpdp.MODE_UNIONDP, 9, 5), (mpdp.MODE_IDP2, 1, 0)):
        got = run(opt, q, mode, k, t)
        want = ref(q, mode, k, t)
        same(got, want)
        assert got[1][1] > 4000  # cost ~ 2^exp, exp far above 1024
    plan = opt.optimize(q, mode=mpdp.MODE_IDP2, k=9)
    assert np.isinf(plan.cost)


def test_heuristic_errors(opt):
    q = W.make("snowflake_plus", 40, 1)
    for kw, code in ((dict(mode=mpdp.MODE_IDP2, k=26), "TOO_LARGE"),
                     (dict(mode=mpdp.MODE_UNIONDP, k=1), "INVALID_ARG"),
                     (dict(mode=mpdp.MODE_UNIONDP, k=10, t=11), "INVALID_ARG"),
                     (dict(mode=mpdp.MODE_IDP2_LEARNED, k=10, t=3), "INVALID_ARG"),
                     (dict(mode=mpdp.MODE_IDP2_LEARNED, k=26), "TOO_LARGE")):
        with pytest.raises(mpdp.MPDPError) as ei:
            opt.optimize(q, **kw)
        assert ei.value.code == mpdp.ERR[code]
    bad = W.Query(n=40, card=q.card, edges=q.edges + [q.edges[0]])
    with pytest.raises(mpdp.MPDPError) as ei:
        opt.optimize(bad, mode=mpdp.MODE_IDP2, k=10)
    assert ei.value.code == mpdp.ERR["INVALID_ARG"]
