"""The allocation-free entry point (mpdp_optimize_device_noalloc) against the
context-based device entry point (mpdp_optimize_device), both through the C
ABI on the same device tensors.

Each query runs twice in a row through the allocation-free call; both results
must equal the context path's bit for bit (cost, status and the raw bytes of
every plan node).  The second call finds the fixed memo holding the first
call's entries, and the queries run largest-first, so a result that leaned
on leftover or zeroed memory would show.  The file is collected last and
keeps no state between tests, so it passes alone and after the others.
"""
import numpy as np
import pytest

import oracle
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def device_query(q):
    d_card = torch.tensor(q.card, dtype=torch.float64, device="cuda")
    d_edges = torch.from_numpy(mpdp.pack_edges(q.edges).view(np.uint8).copy()).cuda()
    return d_card, d_edges


def run_context(opt, q, d_card, d_edges):
    d_nodes = torch.zeros(mpdp.PLAN_STRIDE * 40, dtype=torch.uint8, device="cuda")
    d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    d_status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    opt.optimize_device(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status)
    assert opt.sync() == 0
    return (int(d_status.item()), d_cost.cpu().numpy().tobytes(),
            d_nodes[: (2 * q.n - 1) * 40].cpu().numpy())


def run_noalloc(q, d_card, d_edges):
    d_nodes = torch.zeros((2 * q.n - 1) * 40, dtype=torch.uint8, device="cuda")
    d_cost = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    d_status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    mpdp.optimize_device_noalloc(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status)
    torch.cuda.synchronize()
    return int(d_status.item()), d_cost.cpu().numpy().tobytes(), d_nodes.cpu().numpy()


@pytest.fixture(scope="module")
def opt():
    o = mpdp.Optimizer(0)
    yield o
    o.close()


QUERIES = [
    ("clique", 16, 0), ("cyclic", 16, 3), ("star", 16, 1), ("snowflake", 16, 2),
    ("cycle", 15, 0), ("chain", 14, 5), ("cyclic", 12, 7), ("clique", 9, 4),
    ("snowflake", 10, 9), ("star", 5, 2), ("chain", 2, 0), ("chain", 1, 0),
]


@pytest.mark.parametrize("kind,n,seed", QUERIES)
def test_noalloc_matches_context_path_twice(opt, kind, n, seed):
    q = W.make(kind, n, seed=seed)
    d_card, d_edges = device_query(q)
    ref_status, ref_cost, ref_nodes = run_context(opt, q, d_card, d_edges)
    assert ref_status == 0
    for _ in range(2):
        status, cost, nodes = run_noalloc(q, d_card, d_edges)
        assert status == 0
        assert cost == ref_cost
        assert np.array_equal(nodes, ref_nodes)
    if n <= 12:
        assert np.frombuffer(ref_cost, dtype=np.float64)[0] == oracle.dpccp(q).opt_cost


def test_noalloc_back_to_back_mixed_sizes(opt):
    """Large then small then large again, without a sync between the calls:
    ordered on one stream, each call sees only its own entries."""
    qs = [W.clique(16, seed=1), W.chain(4, seed=0), W.cyclic(16, seed=5), W.star(3, seed=0)]
    refs, outs = [], []
    for q in qs:
        d_card, d_edges = device_query(q)
        refs.append(run_context(opt, q, d_card, d_edges))
        d_nodes = torch.zeros((2 * q.n - 1) * 40, dtype=torch.uint8, device="cuda")
        d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
        d_status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        outs.append((d_card, d_edges, d_nodes, d_cost, d_status))
    for q, (d_card, d_edges, d_nodes, d_cost, d_status) in zip(qs, outs):
        mpdp.optimize_device_noalloc(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status)
    torch.cuda.synchronize()
    for (rs, rc, rn), (_, _, d_nodes, d_cost, d_status) in zip(refs, outs):
        assert int(d_status.item()) == rs == 0
        assert d_cost.cpu().numpy().tobytes() == rc
        assert np.array_equal(d_nodes.cpu().numpy(), rn)


def test_noalloc_on_a_non_default_stream(opt):
    """Two calls back to back on one torch.cuda.Stream, given once as the
    torch object and once as its raw cudaStream_t: ordered on that stream,
    neither sees the other's entries, and both equal the context path."""
    qs = [W.cyclic(16, seed=21), W.clique(13, seed=22)]
    refs, outs = [], []
    for q in qs:
        d_card, d_edges = device_query(q)
        refs.append(run_context(opt, q, d_card, d_edges))
        outs.append((d_card, d_edges, torch.zeros((2 * q.n - 1) * 40, dtype=torch.uint8, device="cuda"),
                     torch.zeros(1, dtype=torch.float64, device="cuda"),
                     torch.full((1,), 99, dtype=torch.int32, device="cuda")))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # inputs written on the current stream
    for (q, o), stream in zip(zip(qs, outs), (side, side.cuda_stream)):
        d_card, d_edges, d_nodes, d_cost, d_status = o
        mpdp.optimize_device_noalloc(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status,
                                     stream=stream)
    side.synchronize()
    for (rs, rc, rn), (_, _, d_nodes, d_cost, d_status) in zip(refs, outs):
        assert int(d_status.item()) == rs == 0
        assert d_cost.cpu().numpy().tobytes() == rc
        assert np.array_equal(d_nodes.cpu().numpy(), rn)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    q = W.chain(mpdp.NOALLOC_MAX_RELS + 1, seed=0)
    d_card, d_edges = device_query(q)
    d_nodes = torch.zeros((2 * q.n - 1) * 40, dtype=torch.uint8, device="cuda")
    d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    d_status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    with pytest.raises(mpdp.MPDPError) as ei:
        mpdp.optimize_device_noalloc(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status)
    assert ei.value.code == mpdp.ERR["TOO_LARGE"]
    torch.cuda.synchronize()
    assert int(d_status.item()) == 99  # nothing was launched
    with pytest.raises(mpdp.MPDPError) as ei:
        mpdp.optimize_device_noalloc(0, 0, d_card, None, d_nodes, d_cost, d_status)
    assert ei.value.code == mpdp.ERR["INVALID_ARG"]


def test_noalloc_invalid_and_disconnected_inputs_report_status(opt):
    """Device-side validation gives the context path's status codes."""
    q = W.chain(6, 0)
    cases = [
        (q.card, q.edges + [(0, 1, 0.5)], "INVALID_ARG"),            # duplicate pair
        (q.card, q.edges[:2] + q.edges[3:], "DISCONNECTED"),         # no cross-product-free plan
        ([0.0] + list(q.card[1:]), q.edges, "INVALID_ARG"),          # card <= 0
        (q.card, q.edges[:-1] + [(4, 5, 1.5)], "INVALID_ARG"),       # sel > 1
    ]
    for card, edges, name in cases:
        bad = W.Query(n=6, card=list(card), edges=edges)
        d_card, d_edges = device_query(bad)
        ref_status, ref_cost, _ = run_context(opt, bad, d_card, d_edges)
        status, cost, _ = run_noalloc(bad, d_card, d_edges)
        assert status == ref_status == mpdp.ERR[name]
        assert cost == ref_cost


def test_noalloc_allocates_no_device_memory():
    """After the first call (the set-up), calls leave the device's free
    memory unchanged."""
    q = W.cyclic(16, seed=11)
    d_card, d_edges = device_query(q)
    d_nodes = torch.zeros((2 * q.n - 1) * 40, dtype=torch.uint8, device="cuda")
    d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    d_status = torch.full((1,), 99, dtype=torch.int32, device="cuda")

    def call():
        mpdp.optimize_device_noalloc(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status)

    call()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(d_status.item()) == 0
