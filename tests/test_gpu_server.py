"""The serving loop (mpdp_server_*) on the GPU: every result of a mixed
stream is bit-identical to the same query optimized alone and to the CPU
oracle's DPCCP (optimal cost and plan), under a burst and under Poisson
arrivals; admission by memo memory; bad requests are refused at submit
without touching their neighbours."""
import numpy as np
import pytest

import oracle
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def mix(count, seed, n_lo=8, n_hi=20):
    rng = np.random.default_rng(seed)
    kinds = ["star", "snowflake", "cyclic"]
    return [W.make(kinds[i % 3], int(rng.integers(n_lo, n_hi + 1)), seed=int(rng.integers(0, 1 << 30)))
            for i in range(count)]


@pytest.fixture(scope="module")
def alone():
    o = mpdp.Optimizer(0)
    yield lambda q: (q, o.optimize(q))
    o.close()


def same(p, alone_result):
    """p equals the query optimized alone, and both equal the oracle."""
    q, ref = alone_result
    assert np.float64(p.cost).tobytes() == np.float64(ref.cost).tobytes()
    assert p.signature() == ref.signature()
    want = oracle.dpccp(q)
    assert np.float64(p.cost).tobytes() == np.float64(want.opt_cost).tobytes()
    assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, want))


def test_burst_results_equal_alone(alone):
    qs = mix(120, seed=1)
    with mpdp.Server(0, slots=3, max_batch=16) as srv:
        tickets = [srv.submit(q) for q in qs]
        srv.drain()
        done = set()
        while True:
            got = srv.poll()
            if not got:
                break
            done.update(got)
        assert done == set(tickets)
        for q, t in zip(qs, tickets):
            p, lat_us = srv.result(t)
            assert lat_us > 0
            same(p, alone(q))
        assert srv.pending() == (0, 0)


def test_poisson_replay_results_equal_alone(alone):
    qs = mix(60, seed=2, n_lo=10, n_hi=18)
    rng = np.random.default_rng(7)
    arrivals = np.cumsum(rng.exponential(1.0 / 2000.0, size=len(qs)))
    with mpdp.Server(0, slots=4, max_batch=8) as srv:
        plans, lats, makespan = srv.replay(qs, arrivals, limit_s=120.0)
    assert makespan >= arrivals[-1]
    assert np.all(lats > 0)
    for q, p in zip(qs, plans):
        same(p, alone(q))


def test_admission_by_memo_memory(alone):
    # a slot budget that holds one 16-relation query but not a 20-relation one
    budget = mpdp.workspace_bytes(16) + 4096
    with mpdp.Server(0, slots=2, max_batch=64, slot_budget_bytes=budget) as srv:
        with pytest.raises(mpdp.MPDPError) as ei:
            srv.submit(W.snowflake(20, seed=0))
        assert ei.value.code == mpdp.ERR["ADMISSION"]
        qs = [W.snowflake(16, seed=s) for s in range(5)] + [W.star(12, seed=3)]
        tickets = [srv.submit(q) for q in qs]
        srv.drain()
        for q, t in zip(qs, tickets):
            same(srv.result(t)[0], alone(q))


def test_bad_request_refused_at_submit_neighbours_fine(alone):
    good = [W.cyclic(12, seed=s) for s in range(4)]
    q = W.chain(6, 0)
    dup = W.Query(n=6, card=q.card, edges=q.edges + [(0, 1, 0.5)])
    disc = W.Query(n=6, card=q.card, edges=q.edges[:2] + q.edges[3:])
    with mpdp.Server(0, slots=1, max_batch=64) as srv:
        t0 = srv.submit(good[0])
        with pytest.raises(mpdp.MPDPError) as ei:
            srv.submit(dup)
        assert ei.value.code == mpdp.ERR["INVALID_ARG"]
        with pytest.raises(mpdp.MPDPError) as ei:
            srv.submit(disc)
        assert ei.value.code == mpdp.ERR["DISCONNECTED"]
        ts = [t0] + [srv.submit(g) for g in good[1:]]
        srv.drain()
        for g, t in zip(good, ts):
            same(srv.result(t)[0], alone(g))


# ---------------------------------------------------------------------------
# Persistent mode: one resident kernel over query slots.

SLOT_20 = 40 << 20  # a slot budget that holds queries of up to 20 relations


def persistent(slots=8, budget=SLOT_20):
    return mpdp.Server(0, slots=slots, slot_budget_bytes=budget, persistent=True)


def test_persistent_burst_results_equal_alone_and_oracle(alone):
    """120 mixed queries at once through 8 query slots: every plan equals the
    same query optimized alone and the oracle's."""
    qs = mix(120, seed=11)
    with persistent() as srv:
        tickets = [srv.submit(q) for q in qs]
        srv.drain()
        done = set()
        while True:
            got = srv.poll()
            if not got:
                break
            done.update(got)
        assert done == set(tickets)
        for q, t in zip(qs, tickets):
            p, lat_us = srv.result(t)
            assert lat_us > 0
            same(p, alone(q))
        assert srv.pending() == (0, 0)


def test_persistent_poisson_replay(alone):
    qs = mix(80, seed=12, n_lo=8, n_hi=20)
    rng = np.random.default_rng(13)
    arrivals = np.cumsum(rng.exponential(1.0 / 3000.0, size=len(qs)))
    with persistent(slots=16) as srv:
        plans, lats, makespan = srv.replay(qs, arrivals, limit_s=120.0)
    assert makespan >= arrivals[-1]
    assert np.all(lats > 0)
    for q, p in zip(qs, plans):
        same(p, alone(q))


def test_persistent_one_slot_and_restart_after_idle(alone):
    """One slot serves the requests one after another; after the kernel has
    ended itself for lack of work (about 20 ms idle) the next request starts
    it again."""
    import time
    qs = [W.cyclic(14, seed=3), W.star(12, seed=4), W.snowflake(18, seed=5)]
    with persistent(slots=1) as srv:
        for q in qs:
            t = srv.submit(q)
            srv.drain()
            same(srv.result(t)[0], alone(q))
            time.sleep(0.1)


def test_persistent_admission_and_bad_requests(alone):
    with persistent(slots=2, budget=SLOT_20) as srv:
        with pytest.raises(mpdp.MPDPError) as ei:
            srv.submit(W.snowflake(21, seed=0))
        assert ei.value.code == mpdp.ERR["ADMISSION"]
        q = W.chain(6, 0)
        with pytest.raises(mpdp.MPDPError) as ei:
            srv.submit(W.Query(n=6, card=q.card, edges=q.edges + [(0, 1, 0.5)]))
        assert ei.value.code == mpdp.ERR["INVALID_ARG"]
        good = [W.snowflake(20, seed=s) for s in range(3)] + [W.cyclic(16, seed=7), W.clique(12, seed=8)]
        ts = [srv.submit(g) for g in good]
        srv.drain()
        for g, t in zip(good, ts):
            same(srv.result(t)[0], alone(g))
