"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/mpdp.h, and its host-only helpers behave."""
import ctypes
import os
import re

import pytest

from paper_2202_13511_gb300 import mpdp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "mpdp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mpdp_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_binding_exports():
    assert declared_functions() == sorted(mpdp.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = mpdp.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_struct_sizes_match_header():
    assert ctypes.sizeof(mpdp.Edge) == 16
    assert ctypes.sizeof(mpdp.PlanNode) == 40
    assert ctypes.sizeof(mpdp.QueryC) == 40
    assert ctypes.sizeof(mpdp.ConfigC) == 44
    assert ctypes.sizeof(mpdp.StatsC) == 6 * 8 + 8 + 8 + 3 * 8 + 3 * 33 * 8


def test_binding_follows_the_header_abi():
    """The binding's struct layouts are written for one ABI version: the
    header's MPDP_ABI_VERSION, which the library also reports."""
    m = re.search(r"#define MPDP_ABI_VERSION (\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == mpdp.ABI_VERSION
    assert mpdp.load().mpdp_abi_version() == mpdp.ABI_VERSION
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for name, cls in (("mpdp_config", mpdp.ConfigC), ("mpdp_query", mpdp.QueryC),
                      ("mpdp_stats", mpdp.StatsC), ("mpdp_plan_node", mpdp.PlanNode),
                      ("mpdp_edge", mpdp.Edge), ("mpdp_server_config", mpdp.ServerConfigC)):
        body = re.search(r"typedef struct \{([^}]*)\} " + name + ";", src).group(1)
        declared = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:
                # "type a, b" or "type *p" or "type arr[N]": the field names in order
                rest = re.sub(r"^(const\s+)?\w+\s*", "", decl)
                declared += [re.sub(r"[*\s]|\[.*\]", "", v) for v in rest.split(",")]
        assert declared == [f for f, _ in cls._fields_], name


def test_abi_version_and_strerror():
    lib = mpdp.load()
    assert lib.mpdp_abi_version() == 6
    assert mpdp.strerror(0) == "ok"
    for code in mpdp.ERRORS:
        assert mpdp.strerror(code) != "unknown error"
    assert mpdp.strerror(-999) == "unknown error"


def test_workspace_bytes_host_only():
    # dense memo: 12 bytes per bitmap plus the per-level lists
    b20 = mpdp.workspace_bytes(20, mpdp.MEMO_DENSE)
    assert b20 >= 12 * 2 ** 20 + 8 * (2 ** 20 - 21)
    assert mpdp.workspace_bytes(21) > b20
    assert mpdp.workspace_bytes(0) == 0
    assert mpdp.workspace_bytes(31) == 0
    h = mpdp.workspace_bytes(20, mpdp.MEMO_HASH)
    assert h > 0


def test_block_workspace_holds_the_find_blocks_cache():
    """A general join graph's workspace adds to a tree query's the
    connectivity bitmap, the block CCP lists (18 relations up), the heavy
    entries (48 B each, C(n, n/2) of them) and the Find-Blocks cache
    (min(C(n, n/2), 4096) lines of 64 B up to 16 relations, 128 B above).
    A 15-relation one still fits the budget of a 16-relation tree query,
    which the GPU budget tests rely on."""
    from math import comb
    for n in range(4, 26):
        tree, blocks = mpdp.workspace_bytes(n), mpdp.workspace_bytes(n, enumeration=mpdp.ENUM_BLOCKS)
        c = comb(n, n // 2)
        cache = min(c, 4096) * (64 if n <= 16 else 128)
        assert blocks - tree >= 48 * c + cache + 2 ** n // 8, n
    assert mpdp.workspace_bytes(15, enumeration=mpdp.ENUM_BLOCKS) < mpdp.workspace_bytes(16)


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mpdp.MPDPError) as ei:
        mpdp.Optimizer(0)
    assert ei.value.code == mpdp.ERR["CUDA"]


def test_packed_batch_layout():
    """The columnar batch: cards and predicates back to back, one record per
    query pointing at its own slice (no edge pointer for an edgeless query)."""
    import numpy as np
    from paper_2202_13511_gb300 import workloads as W
    qs = [W.chain(3, seed=1), W.Query(n=1, card=[5.0], edges=[]), W.star(4, seed=2)]
    pb = mpdp.pack_batch(qs)
    assert len(pb) == 3 and pb.n == [3, 1, 4]
    assert pb.card.tolist() == qs[0].card + qs[1].card + qs[2].card
    flat = [e for q in qs for e in q.edges]
    assert [(int(e["u"]), int(e["v"]), float(e["sel"])) for e in pb.edges] == \
        [(u, v, s) for u, v, s in flat]
    assert pb.recs["n_rels"].tolist() == [3, 1, 4]
    assert pb.recs["n_edges"].tolist() == [2, 0, 3]
    assert pb.recs["card"].tolist() == [pb.card.ctypes.data + 8 * o for o in (0, 3, 4)]
    assert pb.recs["edges"].tolist() == [pb.edges.ctypes.data, 0, pb.edges.ctypes.data + 16 * 2]


CPU_HEADER = os.path.join(os.path.dirname(HEADER), "mpdp_cpu.h")


def test_cpu_baseline_library_exports_its_header():
    """libmpdp_cpu.so (the multi-threaded CPU MPDP) exports exactly what
    include/mpdp_cpu.h declares, and its stats struct has the header's size."""
    from paper_2202_13511_gb300 import cpu_mpdp
    src = re.sub(r"/\*.*?\*/", "", open(CPU_HEADER).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(mpdp_cpu_[a-z_]+)\s*\(", src)))
    assert names == ["mpdp_cpu_optimize"]
    lib = cpu_mpdp.load()
    for name in names:
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value
    assert ctypes.sizeof(cpu_mpdp.CpuStats) == 4 * 8 + 2 * 4 + 8
    m = re.search(r"#define MPDP_CPU_MAX_RELS (\d+)", open(CPU_HEADER).read())
    assert m and int(m.group(1)) == cpu_mpdp.MAX_RELS
