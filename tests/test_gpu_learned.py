"""Learned proposal on the GPU: without a model the learned modes are plain
UnionDP and plain IDP2 bit for bit; with a model, learned IDP2 matches the
oracle's IDP2 from the learned start (the model's scores passed in); trained
by the library's kernels on exact plans of <= 25-relation queries, the
proposal beats plain UnionDP on held-out larger queries."""
import math

import numpy as np
import pytest

from oracle import heuristics as H
from paper_2202_13511_gb300 import learned as L
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opt():
    o = mpdp.Optimizer(0)
    yield o
    o.close()


_DATA = {}


def trained_data():
    return _DATA["xt"]


@pytest.fixture(scope="module")
def trained(opt):
    """6,000 exact plans, 10 epochs (deterministic)."""
    x, t = L.build_dataset(opt, L.training_queries(6000, seed=21))
    _DATA["xt"] = (x, t)
    log = []
    mlp = L.train(x, t, epochs=10, seed=22, log=log)
    yield mlp, log
    opt.set_model(None)
    mlp.close()


def sorted_query(q):
    """q with its edges as (min, max, sel) in ascending order: the edge order
    of the learned start, so that the scores line up with the oracle's."""
    return W.Query(n=q.n, card=q.card, edges=sorted((min(u, v), max(u, v), s) for u, v, s in q.edges))


def model_scores(mlp, q):
    import torch
    x = torch.from_numpy(mpdp.edge_features(q)).cuda()
    y = torch.empty(len(q.edges), dtype=torch.float32, device="cuda")
    mlp.forward(x, len(q.edges), y)
    torch.cuda.synchronize()
    return [float(v) for v in y.cpu().numpy()]


def canonical_from_nodes(nodes):
    def walk(i):
        nd = nodes[i]
        if nd["left"] < 0:
            return int(nd["rel"]), int(nd["rel"])
        a, ma = walk(int(nd["left"]))
        b, mb = walk(int(nd["right"]))
        return ((a, b) if ma < mb else (b, a)), min(ma, mb)
    return walk(0)[0]


def test_learned_idp2_without_model_is_plain_idp2(opt):
    opt.set_model(None)
    for seed in range(3):
        q = W.snowflake_plus_pkfk(50, seed=200 + seed)
        a = opt.optimize(q, mode=mpdp.MODE_IDP2, k=10)
        b = opt.optimize(q, mode=mpdp.MODE_IDP2_LEARNED, k=10)
        assert a.cost_xd == b.cost_xd
        assert np.array_equal(a.nodes, b.nodes)


def _learned_idp2_parity(opt, mlp, cases):
    """GPU learned IDP2 against the oracle: IDP2 from GOO's plan and from the
    learned start built on the model's own scores; the cheaper wins, GOO's
    on ties.  Returns how often the learned plan won."""
    opt.set_model(mlp)
    wins = 0
    for n, seed, k in cases:
        q = sorted_query(W.snowflake_plus_pkfk(n, seed=seed))
        g = H.Graph(q)
        start = H.learned_start(g, model_scores(mlp, q))
        plain = H.goo(g) if k <= 1 else H.idp2(g, k)
        learned = start if k <= 1 else H.idp2(g, k, start=start)
        won = H.xd_key(learned.cost) < H.xd_key(plain.cost)
        want = learned if won else plain
        got = opt.optimize(q, mode=mpdp.MODE_IDP2_LEARNED, k=k)
        assert canonical_from_nodes(got.nodes) == H.canonical(want), (n, seed, k)
        assert got.cost_xd == want.cost, (n, seed, k)
        assert int(got.stats["filter_steps"]) == int(won)
        wins += won
    opt.set_model(None)
    return wins


def test_learned_idp2_matches_oracle_untrained(opt):
    """A freshly initialised model: arbitrary scores, the learned start
    still has to be the one the oracle builds from them."""
    import torch
    mlp = mpdp.Mlp(mpdp.EDGE_FEATURES, 0, stream=torch.cuda.current_stream())
    mlp.init_params(5)
    try:
        _learned_idp2_parity(opt, mlp, [(30, 301, 1), (30, 302, 6), (40, 303, 8), (24, 305, 5)])
    finally:
        mlp.close()


def weight_scores(q):
    """The non-learned control's scores: float32 of log2 of each edge's join
    card, (log2 card(u) + log2 card(v)) + log2 sel, each log2 taken on the
    value's extended-range form m * 2^e as e + log2(m)."""
    def lg(v):
        m, e = H.xd(v)
        return e + math.log2(m)
    return [float(np.float32((lg(q.card[u]) + lg(q.card[v])) + lg(s))) for u, v, s in q.edges]


@pytest.mark.parametrize("n,seed,k", [(30, 401, 6), (50, 402, 8), (60, 403, 10), (100, 404, 12)])
def test_weight_start_idp2_matches_oracle(opt, n, seed, k):
    """MODE_IDP2_WEIGHT_START: IDP2 from GOO's plan and from the start that
    joins edges in ascending join card, the cheaper wins (GOO's on ties),
    equal to the oracle's plan and extended-range cost."""
    opt.set_model(None)
    q = sorted_query(W.snowflake_plus_pkfk(n, seed=seed))
    g = H.Graph(q)
    plain = H.idp2(g, k)
    alt = H.idp2(g, k, start=H.learned_start(g, weight_scores(q)))
    won = H.xd_key(alt.cost) < H.xd_key(plain.cost)
    want = alt if won else plain
    got = opt.optimize(q, mode=mpdp.MODE_IDP2_WEIGHT_START, k=k)
    assert canonical_from_nodes(got.nodes) == H.canonical(want)
    assert got.cost_xd == want.cost
    assert int(got.stats["filter_steps"]) == int(won)


def one_feature_params(feat, n_in=mpdp.EDGE_FEATURES, hidden=mpdp.HIDDEN):
    """Weights under which the network's score is input feature `feat`
    itself: one unit carries bf16(x_feat) + 4 through the three ReLU layers
    and the head subtracts the 4 again (every step exact in bf16 / f32)."""
    W1 = np.zeros((n_in, hidden)); b1 = np.zeros(hidden)
    W2 = np.zeros((hidden, hidden)); W3 = np.zeros((hidden, hidden)); w4 = np.zeros(hidden)
    W1[feat, 0] = 1.0; b1[0] = 4.0; W2[0, 0] = 1.0; W3[0, 0] = 1.0; w4[0] = 1.0
    parts = [W1, b1, W2, np.zeros(hidden), W3, np.zeros(hidden), w4, np.array([-4.0])]
    return np.concatenate([x.ravel() for x in parts]).astype(np.float32)


def test_learned_idp2_matches_oracle_when_learned_wins(opt):
    """Score = the smaller end's log card: on this 30-relation PK-FK query
    IDP2(6) from the learned start costs 0.84x IDP2 from GOO's plan, so the
    learned branch is the one returned."""
    import torch
    mlp = mpdp.Mlp(mpdp.EDGE_FEATURES, 0, stream=torch.cuda.current_stream())
    mlp.set_params(one_feature_params(0))
    try:
        assert _learned_idp2_parity(opt, mlp, [(30, 3, 6)]) == 1
    finally:
        mlp.close()


def test_learned_idp2_matches_oracle_trained(opt, trained):
    mlp, _ = trained
    sizes = [(30, 1), (40, 1), (60, 1), (30, 8), (40, 10)] + [(n, 12) for n in (60, 80, 100) for _ in range(5)]
    cases = [(n, 7100 + i, k) for i, (n, k) in enumerate(sizes)]
    wins = _learned_idp2_parity(opt, mlp, cases)
    print("learned IDP2 wins", wins, "of", len(cases))


def test_learned_mode_without_model_is_plain_uniondp(opt):
    opt.set_model(None)
    for seed in range(3):
        q = W.snowflake_plus_pkfk(50, seed=100 + seed)
        a = opt.optimize(q, mode=mpdp.MODE_UNIONDP, k=12, t=6)
        b = opt.optimize(q, mode=mpdp.MODE_UNIONDP_LEARNED, k=12, t=6)
        assert a.cost_xd == b.cost_xd
        assert np.array_equal(a.nodes, b.nodes)


def test_training_learns(trained):
    """Training lowers the loss well below the initial network's and below
    the best constant prediction (half the labels' variance: the loss is
    sum (y - t)^2 / (2 rows)), over the logged rows."""
    mlp, log = trained
    x, t = trained_data()
    n_eval = min(len(t), 16384)
    constant = float(np.var(t[:n_eval].astype(np.float64))) / 2.0
    assert log[0][0] == -1
    first, last = log[0][1], log[-1][1]
    print("loss before training", first, "after", last, "constant predictor", constant)
    assert last < 0.9 * first
    assert last < 0.8 * constant


def test_labels_from_exact_plans(opt):
    q = W.snowflake_plus_pkfk(12, seed=3)
    p = opt.optimize(q)
    lab = L.edge_labels(q, p.nodes)
    assert lab.shape == (len(q.edges),) and np.all(lab > 0) and np.all(lab <= 1)
    assert np.isclose(lab.max(), 1.0) or lab.max() < 1.0
    assert np.min(lab) == 2 / q.n  # some edge is a first join of two relations


def test_trained_proposal_beats_plain_uniondp(opt, trained):
    """40 held-out queries of 40-100 relations: the geometric mean of
    cost(learned) / cost(plain) is well below 1 (0.47 measured on GB300 with
    these seeds; the run is deterministic)."""
    mlp, log = trained
    test = [W.snowflake_plus_pkfk(n, seed=7000 + i) for i, n in enumerate([40, 60, 80, 100] * 10)]
    rows = L.evaluate(opt, mlp, test, k=12, t=8)
    logs = [math.log2(L.cost_ratio(l, p)) for p, l, _ in rows]
    gain = 2.0 ** np.mean(logs)
    assert gain < 0.8, gain
    opt.set_model(None)


def test_trained_proposal_learned_idp2_never_worse(opt, trained):
    """Learned IDP2 keeps the cheaper of its two plans, so its cost never
    exceeds plain IDP2's; the geometric mean over held-out queries is
    printed."""
    mlp, _ = trained
    logs = []
    for i, n in enumerate([40, 60, 80, 100] * 5):
        q = W.snowflake_plus_pkfk(n, seed=7500 + i)
        opt.set_model(None)
        plain = opt.optimize(q, mode=mpdp.MODE_IDP2, k=12).cost_xd
        opt.set_model(mlp)
        learned = opt.optimize(q, mode=mpdp.MODE_IDP2_LEARNED, k=12).cost_xd
        r = L.cost_ratio(learned, plain)
        assert r <= 1.0
        logs.append(math.log2(r))
    opt.set_model(None)
    print("learned IDP2 gain", 2.0 ** np.mean(logs))
