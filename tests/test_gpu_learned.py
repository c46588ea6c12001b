"""Learned proposal on the GPU: without a model the learned mode is plain
UnionDP bit for bit; trained by the library's kernels on exact plans of
<= 25-relation queries, it beats plain UnionDP on held-out larger queries."""
import math

import numpy as np
import pytest

from paper_2202_13511_gb300 import learned as L
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opt():
    o = mpdp.Optimizer(0)
    yield o
    o.close()


def test_learned_mode_without_model_is_plain_uniondp(opt):
    opt.set_model(None)
    for seed in range(3):
        q = W.snowflake_plus_pkfk(50, seed=100 + seed)
        a = opt.optimize(q, mode=mpdp.MODE_UNIONDP, k=12, t=6)
        b = opt.optimize(q, mode=mpdp.MODE_UNIONDP_LEARNED, k=12, t=6)
        assert a.cost_xd == b.cost_xd
        assert np.array_equal(a.nodes, b.nodes)


def test_labels_from_exact_plans(opt):
    q = W.snowflake_plus_pkfk(12, seed=3)
    p = opt.optimize(q)
    lab = L.edge_labels(q, p.nodes)
    assert lab.shape == (len(q.edges),) and np.all(lab > 0) and np.all(lab <= 1)
    assert np.isclose(lab.max(), 1.0) or lab.max() < 1.0
    assert np.min(lab) == 2 / q.n  # some edge is a first join of two relations


def test_trained_proposal_beats_plain_uniondp(opt):
    """6,000 exact plans, 10 epochs; 40 held-out queries of 40-100
    relations: the geometric mean of cost(learned) / cost(plain) is well
    below 1 (0.47 measured on GB300 with these seeds; the run is
    deterministic)."""
    x, t = L.build_dataset(opt, L.training_queries(6000, seed=21))
    log = []
    mlp = L.train(x, t, epochs=10, seed=22, log=log)
    assert log[-1][1] < log[0][1] * 1.01
    test = [W.snowflake_plus_pkfk(n, seed=7000 + i) for i, n in enumerate([40, 60, 80, 100] * 10)]
    rows = L.evaluate(opt, mlp, test, k=12, t=8)
    logs = [math.log2(L.cost_ratio(l, p)) for p, l, _ in rows]
    gain = 2.0 ** np.mean(logs)
    assert gain < 0.8, gain
    opt.set_model(None)
    mlp.close()
