"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The bar is bit-exact: optimal cost bits, chosen plan, every compared memo
entry (cost and left mask) and the integer counters (connected sets, CCP
pairs and evaluated pairs per level).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2202_13511_gb300 import mpdp
from paper_2202_13511_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KINDS = ["star", "chain", "cycle", "clique", "snowflake", "cyclic"]
CONFIGS = {
    "dense_auto": dict(memo_kind=mpdp.MEMO_DENSE, enumeration=mpdp.ENUM_AUTO),
    "hash_auto": dict(memo_kind=mpdp.MEMO_HASH, enumeration=mpdp.ENUM_AUTO),
    "dense_blocks": dict(memo_kind=mpdp.MEMO_DENSE, enumeration=mpdp.ENUM_BLOCKS),
    "hash_blocks": dict(memo_kind=mpdp.MEMO_HASH, enumeration=mpdp.ENUM_BLOCKS),
    "unrank_auto": dict(filter=mpdp.FILTER_UNRANK),
    "unrank_hash_blocks": dict(filter=mpdp.FILTER_UNRANK, memo_kind=mpdp.MEMO_HASH,
                               enumeration=mpdp.ENUM_BLOCKS),
    "bitmaps_auto": dict(filter=mpdp.FILTER_BITMAPS),
    "dense_unfused": dict(fuse_prune=0),
    "hash_unfused": dict(memo_kind=mpdp.MEMO_HASH, fuse_prune=0),
}


@pytest.fixture(scope="module")
def opt():
    o = mpdp.Optimizer(0)
    yield o
    o.close()


def set_cfg(opt, **kw):
    base = dict(memo_kind=mpdp.MEMO_DENSE, enumeration=mpdp.ENUM_AUTO, heavy_threshold=64,
                use_ccc=1, use_graphs=1, run_length=32, filter=mpdp.FILTER_CONNECTED,
                grid_blocks_per_sm=8, lanes=4, fuse_prune=1, group_threads_log2=18)
    base.update(kw)
    opt.set_config(**base)


def is_tree(q):
    return len(q.edges) == q.n - 1


def check(opt, q, ref=None, memo="all", sample=20000, block_counts=None):
    """Optimize q on the GPU and compare with the oracle result ref."""
    if ref is None:
        ref = oracle.dpccp(q)
    plan = opt.optimize(q, keep=True)
    try:
        assert np.float64(plan.cost).tobytes() == np.float64(ref.opt_cost).tobytes()
        assert plan.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
        st = plan.stats
        n = q.n
        assert np.array_equal(st["connected_per_level"][2:], ref.connected[2:n + 1])
        assert np.array_equal(st["ccp_per_level"][2:], ref.ccp[2:n + 1])
        total = int(np.sum(ref.connected[1:n + 1]))
        if opt.get_config()["filter"] == mpdp.FILTER_CONNECTED and is_tree(q) and 4 * total <= 2 ** n:
            # a tree with few connected sets: only those are ever formed
            assert st["sets_unranked"] == total - n
        else:
            assert st["sets_unranked"] == 2 ** n - n - 1
        tree_mode = st["enumeration"] == mpdp.ENUM_TREE
        if tree_mode:
            assert np.array_equal(st["evaluated_per_level"], st["ccp_per_level"])
        elif block_counts is not None:
            assert np.array_equal(st["evaluated_per_level"][2:], block_counts[2:n + 1])
        if memo and n >= 2:
            sets = ref.connected_sets()
            if memo == "sample" and len(sets) > sample:
                rng = np.random.default_rng(q.seed + 17 * n)
                sets = np.sort(rng.choice(sets, size=sample, replace=False))
            costs, lefts = opt.memo_lookup(plan.handle, sets)
            assert np.array_equal(costs.view(np.uint64), ref.cost[sets].view(np.uint64))
            assert np.array_equal(lefts, ref.left[sets].astype(np.uint64))
        return plan
    finally:
        opt.release(plan.handle)


@pytest.mark.parametrize("cfg", list(CONFIGS))
@pytest.mark.parametrize("kind", KINDS)
def test_small_exhaustive(opt, cfg, kind):
    """Every n from 1 to 12, two seeds: whole memo, plan, counters."""
    set_cfg(opt, **CONFIGS[cfg])
    for n in range(1, 13):
        for seed in range(2):
            q = W.make(kind, n, seed=seed)
            ref = oracle.dpccp(q)
            bc = None
            if n <= 12 and ("blocks" in cfg or not is_tree(q)):
                bc, _ = oracle.block_enum_counts(q)
            check(opt, q, ref, block_counts=bc)


@pytest.mark.parametrize("kind", ["star", "snowflake", "cyclic", "cycle", "chain"])
@pytest.mark.parametrize("n", [14, 16, 18])
def test_medium_whole_memo(opt, kind, n):
    for cfg in ("dense_auto", "hash_auto", "unrank_auto"):
        set_cfg(opt, **CONFIGS[cfg])
        q = W.make(kind, n, seed=n)
        check(opt, q)


@pytest.mark.parametrize("cfg", ["dense_auto", "hash_auto"])
def test_clique_14(opt, cfg):
    """Config: 14-relation cliques (one block per set; the heavy path)."""
    set_cfg(opt, **CONFIGS[cfg])
    for seed in range(2):
        q = W.clique(14, seed=seed)
        plan = check(opt, q, memo="all")
        assert plan.stats["ccp_pairs"] == (3 ** 14 - 2 ** 15 + 1) // 2
        assert plan.stats["pairs_evaluated"] == plan.stats["ccp_pairs"]


@pytest.mark.parametrize("n", [20, 25])
def test_snowflake_full_size(opt, n):
    """Config: acyclic snowflake queries of 20 and 25 relations (tree mode),
    with all three connected-set filters."""
    for seed in range(3):
        q = W.snowflake(n, seed=seed)
        ref = oracle.dpccp(q)
        for flt in (mpdp.FILTER_CONNECTED, mpdp.FILTER_BITMAPS, mpdp.FILTER_UNRANK):
            set_cfg(opt, filter=flt)
            check(opt, q, ref, memo="sample")


def test_bench_batch_full_size(opt):
    """The benchmark's own step: 64 snowflake-25 queries (seeds 0..63) in one
    device batch in the library's default launch configuration (4 lanes of
    16; the middle levels then run a thread per set, the small ones groups of
    lanes).  Every query's cost and plan equal the oracle's, and so do sampled
    memo entries of one query per lane."""
    set_cfg(opt)
    qs = [W.snowflake(25, seed=i) for i in range(64)]
    refs = [oracle.dpccp(q) for q in qs]
    hs = opt.submit_batch(qs)
    try:
        for i in (0, 21, 42, 63):
            sets = refs[i].connected_sets()
            rng = np.random.default_rng(1000 + i)
            sets = np.sort(rng.choice(sets, size=min(len(sets), 20000), replace=False))
            costs, lefts = opt.memo_lookup(hs[i], sets)
            assert np.array_equal(costs.view(np.uint64), refs[i].cost[sets].view(np.uint64))
            assert np.array_equal(lefts, refs[i].left[sets].astype(np.uint64))
    finally:
        plans = opt.collect(hs)
    for q, p, ref in zip(qs, plans, refs):
        assert np.float64(p.cost).tobytes() == np.float64(ref.opt_cost).tobytes()
        assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
        assert np.array_equal(p.stats["ccp_per_level"][2:], ref.ccp[2:26])


def test_snowflake_25_blocks_and_hash(opt):
    """Block-based enumeration and the hash memo agree on trees too."""
    q = W.snowflake(25, seed=5)
    ref = oracle.dpccp(q)
    for cfg in ("hash_auto", "dense_blocks", "hash_blocks"):
        set_cfg(opt, **CONFIGS[cfg])
        check(opt, q, ref, memo="sample")


def test_star_25(opt):
    """The headline shape: 25-relation star, 16.8M connected sets, 201M CCPs."""
    set_cfg(opt)
    q = W.star(25, seed=0)
    ref = oracle.dpccp(q)
    plan = check(opt, q, ref, memo="sample")
    assert plan.stats["ccp_pairs"] == 24 * 2 ** 23
    assert plan.stats["sets_connected"] == 2 ** 24 - 1  # sets of >= 2 relations


@pytest.mark.parametrize("n", [15, 17, 20])
def test_cyclic(opt, n):
    """Config: random spanning tree + 10-30% extra edges (block enumeration)."""
    for cfg in ("dense_auto", "hash_auto"):
        set_cfg(opt, **CONFIGS[cfg])
        for seed in range(2):
            q = W.cyclic(n, seed=seed)
            check(opt, q, memo="sample")


@pytest.mark.parametrize("threshold", [0, 3, 1 << 30])
@pytest.mark.parametrize("ccc", [0, 1])
def test_heavy_path_and_ccc(opt, threshold, ccc):
    """All sets through the block-per-set kernel, some, or none; with and
    without collaborative context collection: same results."""
    set_cfg(opt, heavy_threshold=threshold, use_ccc=ccc)
    for q in (W.cyclic(12, seed=3), W.clique(9, seed=1), W.cycle(11, seed=2)):
        bc, _ = oracle.block_enum_counts(q)
        check(opt, q, block_counts=bc)


def _dense_graph(n, p, seed):
    """Random graph: a path through all relations plus every other pair with
    probability p (seeded SplitMix64), cards and sels as the generators draw
    them."""
    rng = W.SplitMix64(seed)
    card = [10.0 ** (2.0 + 6.0 * rng.uniform()) for _ in range(n)]
    pairs = [(i, i + 1) for i in range(n - 1)]
    pairs += [(i, j) for i in range(n) for j in range(i + 2, n) if rng.uniform() < p]
    edges = [(u, v, 10.0 ** (-6.0 + 5.0 * rng.uniform())) for (u, v) in pairs]
    return W.Query(n=n, card=card, edges=edges, kind="dense", seed=seed)


def _two_connected_non_cliques(q, sizes):
    """Vertex sets of the given sizes whose induced subgraph is 2-connected
    and not complete (brute force over the subsets)."""
    adj = [0] * q.n
    for u, v, _ in q.edges:
        adj[u] |= 1 << v
        adj[v] |= 1 << u

    def connected(s):
        seen = s & -s
        frontier = seen
        while frontier:
            nb = 0
            x = frontier
            while x:
                low = x & -x
                nb |= adj[low.bit_length() - 1]
                x ^= low
            frontier = nb & s & ~seen
            seen |= frontier
        return seen == s

    count = 0
    for k in sizes:
        for members in itertools.combinations(range(q.n), k):
            s = sum(1 << v for v in members)
            if all((adj[v] & s) == s & ~(1 << v) for v in members):
                continue  # a clique
            if connected(s) and all(connected(s & ~(1 << v)) for v in members):
                count += 1
    return count


def test_block_lists_overflow_falls_back(opt):
    """A dense 18-relation graph has more 2-connected non-clique sets of at
    most 14 relations than the block CCP lists take (512 of them, half the
    table's 1,024 slots; 1,163 of 4-6 relations alone), so some blocks stay
    unlisted and are enumerated: the oracle's costs, plans, CCP counts and
    memo entries all the same.  A 19-relation graph of lower density lists
    its blocks."""
    q = _dense_graph(18, 0.35, seed=11)
    assert _two_connected_non_cliques(q, (4, 5, 6)) > 1024
    check(opt, q, memo="sample")
    q = _dense_graph(19, 0.25, seed=12)
    check(opt, q, memo="sample")


@pytest.mark.parametrize("threshold", [0, 64])
def test_heavy_find_blocks_cache_overflow(opt, threshold):
    """With every set heavy (threshold 0), the middle levels of a 15-clique
    (C(15, 7) = 6,435 sets) and of a dense 16-relation graph append more
    heavy sets than the Find-Blocks cache keeps (4,096 per level): the sets
    past it find their blocks again in the warp path, the ones below read
    them.  Every result is the oracle's."""
    set_cfg(opt, heavy_threshold=threshold)
    for q in (W.clique(15, seed=2), _dense_graph(16, 0.5, seed=5)):
        check(opt, q, memo="sample")


@pytest.mark.parametrize("run", [1, 5, 32])
def test_run_lengths(opt, run):
    """Ragged unrank runs (run lengths that do not divide C(n,k))."""
    set_cfg(opt, run_length=run, filter=mpdp.FILTER_UNRANK)
    for q in (W.snowflake(13, seed=1), W.cyclic(11, seed=4), W.star(9, seed=2)):
        check(opt, q)


@pytest.mark.parametrize("graphs", [0, 1])
def test_graphs_on_off(opt, graphs):
    set_cfg(opt, use_graphs=graphs)
    for q in (W.snowflake(16, seed=2), W.cyclic(13, seed=1)):
        p1 = check(opt, q)
        assert opt.launch_count() > 0
        del p1


@pytest.mark.parametrize("kind,n,seed", [("snowflake", 14, 1), ("cyclic", 13, 2), ("clique", 10, 3),
                                         ("star", 12, 4), ("chain", 15, 5)])
@pytest.mark.parametrize("memo", [mpdp.MEMO_DENSE, mpdp.MEMO_HASH])
def test_dpsub_enumeration(opt, kind, n, seed, memo):
    """The DPSUB ablation on the block kernels: same plans, costs and CCP
    pairs; evaluated = 2^(|S|-1) - 1 per connected set S."""
    set_cfg(opt, enumeration=mpdp.ENUM_DPSUB, memo_kind=memo)
    q = W.make(kind, n, seed)
    ref = oracle.dpccp(q)
    plan = opt.optimize(q)
    assert np.float64(plan.cost).tobytes() == np.float64(ref.opt_cost).tobytes()
    assert plan.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
    st = plan.stats
    assert np.array_equal(st["ccp_per_level"][2:], ref.ccp[2:n + 1])
    want = np.zeros(n + 1, dtype=np.uint64)
    for s in ref.connected_sets():
        k = bin(s).count("1")
        if k >= 2:
            want[k] += (1 << (k - 1)) - 1
    assert np.array_equal(st["evaluated_per_level"][2:], want[2:])
    set_cfg(opt)


@pytest.mark.parametrize("grid", [1, 3, 32])
def test_grid_sizes(opt, grid):
    """Results do not depend on how many blocks the evaluate grids get."""
    set_cfg(opt, grid_blocks_per_sm=grid)
    for q in (W.snowflake(18, seed=6), W.cyclic(15, seed=4), W.clique(12, seed=2)):
        check(opt, q)
    set_cfg(opt)


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("memo", ["dense", "hash"])
@pytest.mark.parametrize("lanes", [1, 2, 3, 8])
def test_lanes(opt, lanes, memo, graphs):
    """A batch run as concurrent sub-batches of consecutive queries (lanes):
    every query's cost, plan and whole memo (read back for the queries of
    every lane) equal the oracle's, whatever the lane count."""
    set_cfg(opt, lanes=lanes, use_graphs=graphs,
            memo_kind=mpdp.MEMO_DENSE if memo == "dense" else mpdp.MEMO_HASH)
    qs = W.mixed_stream(11, seed=31, n_lo=3, n_hi=15)
    refs = [oracle.dpccp(q) for q in qs]
    hs = opt.submit_batch(qs)
    try:
        for q, h, ref in zip(qs, hs, refs):
            sets = ref.connected_sets()
            costs, lefts = opt.memo_lookup(h, sets)
            assert np.array_equal(costs.view(np.uint64), ref.cost[sets].view(np.uint64))
            assert np.array_equal(lefts, ref.left[sets].astype(np.uint64))
    finally:
        plans = opt.collect(hs)
    for q, p, ref in zip(qs, plans, refs):
        assert p.cost == ref.opt_cost
        assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
    set_cfg(opt)


def test_host_upload(opt):
    """The host path packs a batch's cardinalities and predicates behind the
    descriptors and sends them in one copy: a mixed batch (single relations
    without edges, trees, cycles, a clique) gets the oracle's costs and plans
    back, and the bytes charged to each query cover at least its own values."""
    set_cfg(opt)
    qs = [W.Query(n=1, card=[42.0], edges=[]), W.chain(2, seed=3), W.snowflake(17, seed=8),
          W.Query(n=1, card=[7.0], edges=[]), W.cyclic(13, seed=5), W.clique(9, seed=1),
          W.star(12, seed=4)]
    plans = opt.optimize_batch(qs)
    for q, p in zip(qs, plans):
        ref = oracle.dpccp(q)
        assert p.cost == ref.opt_cost
        assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
    own = [8 * q.n + 16 * len(q.edges) for q in qs]
    got = [int(p.stats["h2d_bytes"]) for p in plans]
    assert all(g >= o for g, o in zip(got, own))
    # the rest is one descriptor per query, the prefix slot and alignment
    assert sum(got) - sum(own) < 1024 * len(qs) + 8192
    # the same batch in columnar form, submitted twice while in flight
    packed = mpdp.pack_batch(qs)
    h1 = opt.submit_batch(packed)
    h2 = opt.submit_batch(packed)
    for again in (opt.collect(h1), opt.collect(h2)):
        for p, a in zip(plans, again):
            assert a.cost == p.cost and a.signature() == p.signature()


@pytest.mark.parametrize("lanes", [1, 4])
def test_unfused_ablation(opt, lanes):
    """The unfused tree path (pairs to a buffer, then prune + scatter) gives
    the fused path's costs, plans and memo at full tree sizes."""
    set_cfg(opt, fuse_prune=0, lanes=lanes)
    for q in (W.snowflake(20, seed=5), W.star(16, seed=2), W.chain(22, seed=1)):
        check(opt, q, memo="sample")
    qs = [W.snowflake(18, seed=s) for s in range(6)]
    for q, p in zip(qs, opt.optimize_batch(qs)):
        ref = oracle.dpccp(q)
        assert p.cost == ref.opt_cost
        assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
    set_cfg(opt)


@pytest.mark.parametrize("log2", [0, 8, 16, 20, 24])
def test_group_split_knob(opt, log2):
    """The tree levels' work split (a thread per set, or groups of lanes
    while sets x G stay within 2^log2 threads) changes no result: costs,
    plans, CCP counts and sampled memo entries equal the oracle's at both
    ends of the knob and with it off."""
    set_cfg(opt, group_threads_log2=log2)
    qs = ([W.snowflake(20, seed=s) for s in range(6)] + [W.star(16, seed=1), W.chain(22, seed=2)]
          + [W.snowflake(25, seed=7)])
    refs = [oracle.dpccp(q) for q in qs]
    hs = opt.submit_batch(qs)
    try:
        for h, ref in zip(hs, refs):
            sets = ref.connected_sets()
            rng = np.random.default_rng(77)
            sets = np.sort(rng.choice(sets, size=min(len(sets), 5000), replace=False))
            costs, lefts = opt.memo_lookup(h, sets)
            assert np.array_equal(costs.view(np.uint64), ref.cost[sets].view(np.uint64))
            assert np.array_equal(lefts, ref.left[sets].astype(np.uint64))
    finally:
        plans = opt.collect(hs)
    for q, p, ref in zip(qs, plans, refs):
        assert np.float64(p.cost).tobytes() == np.float64(ref.opt_cost).tobytes()
        assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
        assert np.array_equal(p.stats["evaluated_per_level"], p.stats["ccp_per_level"])
        assert np.array_equal(p.stats["ccp_per_level"][2:], ref.ccp[2:q.n + 1])
    set_cfg(opt)


def test_lanes_bad_config(opt):
    for kw in (dict(lanes=0), dict(lanes=9), dict(fuse_prune=2), dict(group_threads_log2=7),
               dict(group_threads_log2=25), dict(group_threads_log2=-1)):
        with pytest.raises(mpdp.MPDPError) as ei:
            opt.set_config(**kw)
        assert ei.value.code == mpdp.ERR["INVALID_ARG"]
    set_cfg(opt)


@pytest.mark.parametrize("kind", ["star", "clique", "cycle", "chain"])
@pytest.mark.parametrize("n", [6, 9, 12])
def test_ties(opt, kind, n):
    """All-equal cardinalities and selectivities: many exact ties."""
    set_cfg(opt)
    base = W.make(kind, n, 0)
    q = W.uniform_values(n, [(u, v) for (u, v, _s) in base.edges])
    check(opt, q)
    set_cfg(opt, memo_kind=mpdp.MEMO_HASH, enumeration=mpdp.ENUM_BLOCKS)
    check(opt, q)


def test_max_size_chain(opt):
    """Largest exact size the oracle reaches (28) on a chain: 268M subsets
    unranked, 406 connected sets."""
    set_cfg(opt)
    q = W.chain(28, seed=0)
    plan = check(opt, q, memo="all")
    assert plan.stats["ccp_pairs"] == (28 ** 3 - 28) // 6


@pytest.mark.parametrize("filt", ["connected", "bitmaps"])
def test_max_size_30_counts(opt, filt):
    """n = 30, the exact-mode maximum: closed-form counts on a chain.  The
    bitmap sweep forms every one of the 2^30 - 31 sets of two or more
    relations; the connected-set unranking forms only the connected ones."""
    set_cfg(opt, filter=mpdp.FILTER_CONNECTED if filt == "connected" else mpdp.FILTER_BITMAPS)
    q = W.chain(30, seed=0)
    plan = opt.optimize(q)
    assert plan.stats["sets_connected"] == 30 * 31 // 2 - 30
    assert plan.stats["ccp_pairs"] == (30 ** 3 - 30) // 6
    assert plan.stats["sets_unranked"] == (2 ** 30 - 31 if filt == "bitmaps" else 30 * 31 // 2 - 30)
    assert len(plan.nodes) == 59
    set_cfg(opt)


def test_card_peel_order_golden(opt):
    """The golden card(S) values of the peeling order: the GPU's cost of
    every 2-relation set is its card (cost = 0 + 0 + card), bit for bit,
    and every larger set's cost equals the oracle's."""
    from tests.test_oracle_pins import card_peel_golden
    q, want = card_peel_golden()
    plan = opt.optimize(q, keep=True)
    sets = sorted(want)
    costs, _ = opt.memo_lookup(plan.handle, sets)
    ref = oracle.dpccp(q)
    for s, c in zip(sets, costs):
        if bin(s).count("1") == 2:
            assert float(c).hex() == want[s].hex(), bin(s)
        if bin(s).count("1") >= 2:
            assert float(c).hex() == float(ref.cost[s]).hex(), bin(s)
    opt.release(plan.handle)


def test_single_relation(opt):
    set_cfg(opt)
    q = W.Query(n=1, card=[123.0], edges=[])
    plan = opt.optimize(q)
    assert plan.cost == 0.0 and len(plan.nodes) == 1 and plan.nodes[0]["rel"] == 0


def test_errors(opt):
    set_cfg(opt)
    q = W.chain(5, 0)
    bad = [W.Query(n=5, card=q.card, edges=q.edges + [(0, 1, 0.5)]),
           W.Query(n=5, card=q.card, edges=q.edges[:-1] + [(3, 4, 0.0)]),
           W.Query(n=5, card=[1.0, float("nan"), 1.0, 1.0, 1.0], edges=q.edges)]
    for b in bad:
        with pytest.raises(mpdp.MPDPError) as ei:
            opt.optimize(b)
        assert ei.value.code == mpdp.ERR["INVALID_ARG"]
    with pytest.raises(mpdp.MPDPError) as ei:
        opt.optimize(W.Query(n=5, card=q.card, edges=q.edges[:2]))
    assert ei.value.code == mpdp.ERR["DISCONNECTED"]
    with pytest.raises(mpdp.MPDPError) as ei:
        opt.optimize(W.chain(31, 0))
    assert ei.value.code == mpdp.ERR["TOO_LARGE"]
    # the context stays usable
    check(opt, W.cyclic(10, seed=9))


def test_determinism(opt):
    set_cfg(opt)
    q = W.cyclic(16, seed=7)
    ref = oracle.dpccp(q)
    a = check(opt, q, ref)
    b = check(opt, q, ref)
    assert a.signature() == b.signature() and a.cost == b.cost


def test_batch_matches_single(opt):
    set_cfg(opt)
    qs = W.mixed_stream(12, seed=3, n_lo=6, n_hi=14)
    plans = opt.optimize_batch(qs)
    for q, p in zip(qs, plans):
        ref = oracle.dpccp(q)
        assert p.cost == ref.opt_cost
        assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))


def test_device_path(opt):
    """Inputs and outputs resident in device memory (torch tensors)."""
    torch = pytest.importorskip("torch")
    set_cfg(opt)
    for q in (W.snowflake(18, seed=4), W.cyclic(14, seed=2), W.star(12, seed=1)):
        ref = oracle.dpccp(q)
        d_card = torch.tensor(q.card, dtype=torch.float64, device="cuda")
        e = mpdp.pack_edges(q.edges)
        d_edges = torch.from_numpy(e.view(np.uint8).copy()).cuda()
        d_nodes = torch.zeros((2 * q.n - 1) * 40, dtype=torch.uint8, device="cuda")
        d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
        d_status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        opt.optimize_device(q.n, len(q.edges), d_card, d_edges, d_nodes, d_cost, d_status)
        assert opt.sync() == 0
        assert int(d_status.item()) == 0
        assert float(d_cost.item()) == ref.opt_cost
        nodes = mpdp.nodes_from_bytes(d_nodes.cpu().numpy())
        plan = mpdp.Plan(cost=float(d_cost.item()), nodes=nodes)
        assert plan.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))


def test_device_path_invalid_input_reports_status(opt):
    """The device path validates on the device and reports, without faulting."""
    torch = pytest.importorskip("torch")
    set_cfg(opt)
    q = W.chain(6, 0)
    edges = q.edges + [(0, 1, 0.5)]  # duplicate pair
    d_card = torch.tensor(q.card, dtype=torch.float64, device="cuda")
    d_edges = torch.from_numpy(mpdp.pack_edges(edges).view(np.uint8).copy()).cuda()
    d_nodes = torch.zeros(11 * 40, dtype=torch.uint8, device="cuda")
    d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    d_status = torch.zeros(1, dtype=torch.int32, device="cuda")
    opt.optimize_device(6, len(edges), d_card, d_edges, d_nodes, d_cost, d_status)
    opt.sync()
    assert int(d_status.item()) == mpdp.ERR["INVALID_ARG"]
    check(opt, W.cyclic(9, seed=1))


def test_device_batch_path(opt):
    """A device-resident batch of mixed queries (tree and block mode, sizes
    1..20) gives the same plans as the oracle, query by query."""
    torch = pytest.importorskip("torch")
    set_cfg(opt)
    qs = W.mixed_stream(40, seed=11, n_lo=1, n_hi=20)
    d_card = torch.tensor([c for q in qs for c in q.card], dtype=torch.float64, device="cuda")
    d_edges = torch.from_numpy(
        mpdp.pack_edges([e for q in qs for e in q.edges]).view(np.uint8).copy()).cuda()
    nq = len(qs)
    d_nodes = torch.zeros((nq, mpdp.PLAN_STRIDE * 40), dtype=torch.uint8, device="cuda")
    d_cost = torch.zeros(nq, dtype=torch.float64, device="cuda")
    d_status = torch.full((nq,), 99, dtype=torch.int32, device="cuda")
    opt.optimize_batch_device([q.n for q in qs], [len(q.edges) for q in qs], d_card, d_edges,
                              d_nodes, d_cost, d_status)
    opt.sync()
    status = d_status.cpu().numpy()
    costs = d_cost.cpu().numpy()
    nodes = d_nodes.cpu().numpy()
    for i, q in enumerate(qs):
        ref = oracle.dpccp(q)
        assert status[i] == 0
        assert costs[i] == ref.opt_cost
        plan = mpdp.Plan(cost=costs[i], nodes=mpdp.nodes_from_bytes(nodes[i]))
        assert plan.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))


def test_batch_split_by_budget():
    """A small memo budget splits one call into several device batches; every
    result stays exact, and a query larger than the budget is refused."""
    # room for one 16-relation query (plus the fixed per-context part), so
    # every query below runs in a device batch of its own
    small = mpdp.workspace_bytes(16) + 4096
    assert mpdp.workspace_bytes(20) > small
    with mpdp.Optimizer(0, memo_budget_bytes=small) as o:
        qs = [W.snowflake(16, seed=s) for s in range(3)] + [W.cyclic(15, seed=2), W.star(14, seed=1)]
        plans = o.optimize_batch(qs)
        for q, p in zip(qs, plans):
            ref = oracle.dpccp(q)
            assert p.cost == ref.opt_cost
            assert p.signature() == oracle.plan_signature(oracle.plan_from_memo(q, ref))
        with pytest.raises(mpdp.MPDPError) as ei:
            o.optimize(W.snowflake(20, seed=0))
        assert ei.value.code == mpdp.ERR["ADMISSION"]


def test_batch_with_invalid_member_is_rejected_whole(opt):
    """Host-path batches are validated before anything is enqueued."""
    set_cfg(opt)
    q = W.chain(5, 0)
    bad = W.Query(n=5, card=q.card, edges=q.edges + [(0, 1, 0.5)])
    with pytest.raises(mpdp.MPDPError) as ei:
        opt.optimize_batch([W.star(6, 0), bad])
    assert ei.value.code == mpdp.ERR["INVALID_ARG"]
    check(opt, W.cyclic(9, seed=3))
