"""The multi-threaded CPU MPDP (the paper's "MPDP (24CPU)" comparison,
Sec. 3.3) against the oracle, on the host: optimal cost and plan bit for
bit, the same CCP and connected-set counts, and the same result for every
thread count."""
import numpy as np
import pytest

import oracle
from paper_2202_13511_gb300 import cpu_mpdp
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W


def check(q, threads):
    plan, st = cpu_mpdp.optimize(q, threads=threads)
    ref = oracle.dpccp(q)
    assert np.float64(plan.cost).tobytes() == np.float64(ref.opt_cost).tobytes()
    assert plan.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
    assert st["ccp_pairs"] == int(ref.ccp.sum())
    assert st["sets_connected"] == int(ref.connected[2:].sum())
    assert st["threads"] == threads
    assert st["sets_unranked"] == 2 ** q.n - q.n - 1
    return plan, st


@pytest.mark.parametrize("kind,n", [("star", 12), ("chain", 14), ("cycle", 12), ("clique", 10),
                                    ("snowflake", 16), ("cyclic", 15)])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_matches_oracle(kind, n, threads):
    for seed in range(2):
        check(W.make(kind, n, seed=seed), threads)


def test_block_enumeration_counts():
    """pairs_evaluated is Algorithm 4's unordered block bipartitions,
    sum over sets of sum over blocks of 2^(|B|-1) - 1, as the oracle counts
    them from its own blocks."""
    for kind, n in (("cyclic", 12), ("clique", 9), ("snowflake", 12)):
        q = W.make(kind, n, seed=3)
        _, st = cpu_mpdp.optimize(q, threads=4)
        ev, valid = oracle.block_enum_counts(q)
        assert st["pairs_evaluated"] == int(ev.sum())
        assert st["ccp_pairs"] == int(valid.sum())


def test_ties_and_small():
    for q in (W.uniform_values(8, [(0, i) for i in range(1, 8)], kind="star"),
              W.uniform_values(7, [(i, j) for i in range(7) for j in range(i + 1, 7)], kind="clique"),
              W.chain(2, 0), W.chain(3, 1)):
        for threads in (1, 5):
            check(q, threads)
    plan, st = cpu_mpdp.optimize(W.Query(n=1, card=[7.0], edges=[]), threads=2)
    assert plan.cost == 0.0 and len(plan.nodes) == 1 and st["ccp_pairs"] == 0


def test_every_thread_count_same_memo_result():
    q = W.make("cyclic", 17, seed=5)
    base, _ = cpu_mpdp.optimize(q, threads=1)
    for threads in (2, 7, 16, 0):
        plan, st = cpu_mpdp.optimize(q, threads=threads)
        assert plan.cost == base.cost and plan.signature() == base.signature()
        assert st["threads"] >= 1


def test_errors():
    q = W.chain(5, 0)
    cases = [(W.Query(n=5, card=q.card, edges=q.edges + [(0, 1, 0.5)]), "INVALID_ARG"),
             (W.Query(n=5, card=q.card, edges=q.edges[:3]), "DISCONNECTED"),
             (W.Query(n=5, card=[1.0, 2.0, 0.0, 1.0, 1.0], edges=q.edges), "INVALID_ARG"),
             (W.Query(n=5, card=q.card, edges=[(0, 1, 1.5)] + q.edges[1:]), "INVALID_ARG"),
             (W.Query(n=31, card=[1.0] * 31, edges=[(i, i + 1, 0.5) for i in range(30)]), "TOO_LARGE")]
    for bad, code in cases:
        with pytest.raises(mpdp.MPDPError) as ei:
            cpu_mpdp.optimize(bad, threads=2)
        assert ei.value.code == mpdp.ERR[code]
