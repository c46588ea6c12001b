"""Python binding of the C ABI in ``include/mpdp.h`` (argument marshalling only).

Every step of the join-order DP runs in the CUDA library ``libmpdp.so``; this
module only converts queries into the ABI's structs, calls the entry points
with the same names, and converts plans back.  There is no CPU fallback: if
the library cannot be loaded, every call raises.

PyTorch is used only for device memory and streams (``optimize_device`` takes
tensors resident on the GPU; ``Optimizer(stream=...)`` borrows a CUDA stream).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import sys
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import _build

MPDP_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "DISCONNECTED", -3: "TOO_LARGE", -4: "OOM", -5: "ADMISSION",
    -6: "BUFFER_TOO_SMALL", -7: "TIMEOUT", -8: "PROBE_LIMIT", -9: "CUDA", -10: "BAD_HANDLE",
    -11: "NOT_IMPLEMENTED", -12: "STALE", -13: "INTERNAL", -14: "NOT_READY",
}
ERR = {v: k for k, v in ERRORS.items()}

(MODE_EXACT, MODE_IDP2, MODE_UNIONDP, MODE_IDP2_LEARNED, MODE_UNIONDP_LEARNED, MODE_UNIONDP_SIZEFIRST,
 MODE_IDP2_WEIGHT_START) = range(7)
PROFILE_OFF, PROFILE_SERIAL, PROFILE_CONCURRENT = range(3)
ENUM_AUTO, ENUM_TREE, ENUM_BLOCKS, ENUM_DPSUB = range(4)
MEMO_DENSE, MEMO_HASH = range(2)
FILTER_BITMAPS, FILTER_UNRANK, FILTER_CONNECTED = range(3)
MAX_LEVELS = 33


class MPDPError(RuntimeError):
    def __init__(self, code: int, what: str = "", detail: str = ""):
        name = ERRORS.get(code, str(code))
        msg = f"{what}: MPDP_ERR_{name} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code
        self.name = name


class Edge(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("v", ctypes.c_int32), ("sel", ctypes.c_double)]


class QueryC(ctypes.Structure):
    _fields_ = [("n_rels", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("card", ctypes.POINTER(ctypes.c_double)), ("edges", ctypes.POINTER(Edge)),
                ("cost_model", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("k", ctypes.c_int32), ("t", ctypes.c_int32)]


class PlanNode(ctypes.Structure):
    _fields_ = [("left", ctypes.c_int32), ("right", ctypes.c_int32), ("rel", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("set", ctypes.c_uint64),
                ("card", ctypes.c_double), ("cost", ctypes.c_double)]


class StatsC(ctypes.Structure):
    _fields_ = [("sets_unranked", ctypes.c_uint64), ("sets_connected", ctypes.c_uint64),
                ("pairs_evaluated", ctypes.c_uint64), ("ccp_pairs", ctypes.c_uint64),
                ("memo_bytes", ctypes.c_uint64), ("heavy_sets", ctypes.c_uint64),
                ("device_ms", ctypes.c_double), ("enumeration", ctypes.c_int32),
                ("memo_kind", ctypes.c_int32), ("h2d_bytes", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64), ("filter_steps", ctypes.c_uint64),
                ("connected_per_level", ctypes.c_uint64 * MAX_LEVELS),
                ("evaluated_per_level", ctypes.c_uint64 * MAX_LEVELS),
                ("ccp_per_level", ctypes.c_uint64 * MAX_LEVELS)]


class ConfigC(ctypes.Structure):
    _fields_ = [("memo_kind", ctypes.c_int32), ("enumeration", ctypes.c_int32),
                ("heavy_threshold", ctypes.c_int32), ("use_ccc", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("run_length", ctypes.c_int32),
                ("filter", ctypes.c_int32), ("grid_blocks_per_sm", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("fuse_prune", ctypes.c_int32),
                ("group_threads_log2", ctypes.c_int32)]


class ServerConfigC(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("slot_budget_bytes", ctypes.c_uint64), ("kernel", ConfigC),
                ("persistent", ctypes.c_int32), ("pad", ctypes.c_int32)]


EDGE_DTYPE = np.dtype([("u", "<i4"), ("v", "<i4"), ("sel", "<f8")])
NODE_DTYPE = np.dtype([("left", "<i4"), ("right", "<i4"), ("rel", "<i4"), ("n_leaves", "<i4"),
                       ("set", "<u8"), ("card", "<f8"), ("cost", "<f8")])
assert EDGE_DTYPE.itemsize == ctypes.sizeof(Edge) == 16
assert NODE_DTYPE.itemsize == ctypes.sizeof(PlanNode) == 40

# Every exported entry point declared in include/mpdp.h.
EXPORTS = [
    "mpdp_create", "mpdp_destroy", "mpdp_set_config", "mpdp_get_config",
    "mpdp_workspace_bytes", "mpdp_optimize", "mpdp_optimize_batch", "mpdp_get_plan",
    "mpdp_release", "mpdp_optimize_device", "mpdp_sync", "mpdp_memo_lookup",
    "mpdp_last_launch_count", "mpdp_strerror", "mpdp_last_error", "mpdp_abi_version",
    "mpdp_profile", "mpdp_profile_read", "mpdp_profile_read_active", "mpdp_optimize_batch_device",
    "mpdp_optimize_device_noalloc", "mpdp_get_plans", "mpdp_get_cost_xd",
    "mpdp_mlp_create", "mpdp_mlp_destroy", "mpdp_mlp_param_count", "mpdp_mlp_set_params",
    "mpdp_mlp_get_params", "mpdp_mlp_forward", "mpdp_mlp_gradients", "mpdp_mlp_train_step",
    "mpdp_set_model", "mpdp_edge_features",
    "mpdp_server_default_config", "mpdp_server_create", "mpdp_server_destroy", "mpdp_server_submit",
    "mpdp_server_poll", "mpdp_server_drain", "mpdp_server_pending", "mpdp_server_result",
    "mpdp_probe_read_gbs",
]
PLAN_STRIDE = 63
NOALLOC_MAX_RELS = 16
NOALLOC_SCRATCH_BYTES = 1310720

KERNEL_CLASSES = ["stage", "ingest", "filter", "memo_init", "eval", "heavy", "extract", "publish"]

_LIB = None


def lib_path() -> str:
    return _build.LIB_PATH


ABI_VERSION = 6  # MPDP_ABI_VERSION of include/mpdp.h this binding's structs follow


def load(build_if_missing: bool = True):
    """Load libmpdp.so (building it first when it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB_PATH
    if build_if_missing and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    L.mpdp_abi_version.restype = ctypes.c_int32
    if L.mpdp_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{path} has ABI {L.mpdp_abi_version()}, this binding needs {ABI_VERSION}; "
                           "rebuild with __graft_entry__.build()")
    P = ctypes.POINTER
    c_ctx = ctypes.c_void_p
    L.mpdp_create.argtypes = [P(c_ctx), ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]
    L.mpdp_destroy.argtypes = [c_ctx]
    L.mpdp_destroy.restype = None
    L.mpdp_set_config.argtypes = [c_ctx, P(ConfigC)]
    L.mpdp_get_config.argtypes = [c_ctx, P(ConfigC)]
    L.mpdp_workspace_bytes.argtypes = [ctypes.c_int32, P(ConfigC)]
    L.mpdp_workspace_bytes.restype = ctypes.c_size_t
    L.mpdp_optimize.argtypes = [c_ctx, P(QueryC), P(ctypes.c_int64)]
    L.mpdp_optimize_batch.argtypes = [c_ctx, P(QueryC), ctypes.c_int32, P(ctypes.c_int64)]
    L.mpdp_get_plan.argtypes = [c_ctx, ctypes.c_int64, P(PlanNode), ctypes.c_int32,
                                P(ctypes.c_int32), P(ctypes.c_double), P(StatsC)]
    L.mpdp_release.argtypes = [c_ctx, ctypes.c_int64]
    L.mpdp_get_cost_xd.argtypes = [c_ctx, ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32)]
    L.mpdp_get_cost_xd.restype = ctypes.c_int
    L.mpdp_get_plans.argtypes = [c_ctx, P(ctypes.c_int64), ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_double),
                                 P(ctypes.c_int32), ctypes.c_void_p]
    L.mpdp_get_plans.restype = ctypes.c_int
    L.mpdp_optimize_device.argtypes = [c_ctx, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.mpdp_optimize_batch_device.argtypes = [c_ctx, ctypes.c_int32, P(ctypes.c_int32),
                                             P(ctypes.c_int32), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
    L.mpdp_optimize_device_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.mpdp_optimize_device_noalloc.restype = ctypes.c_int
    L.mpdp_sync.argtypes = [c_ctx]
    c_mlp = ctypes.c_void_p
    L.mpdp_mlp_create.argtypes = [P(c_mlp), ctypes.c_int, ctypes.c_int32, ctypes.c_void_p]
    L.mpdp_mlp_destroy.argtypes = [c_mlp]
    L.mpdp_mlp_destroy.restype = None
    L.mpdp_mlp_param_count.argtypes = [c_mlp]
    L.mpdp_mlp_param_count.restype = ctypes.c_int64
    L.mpdp_mlp_set_params.argtypes = [c_mlp, P(ctypes.c_float), ctypes.c_int64]
    L.mpdp_mlp_get_params.argtypes = [c_mlp, P(ctypes.c_float), ctypes.c_int64]
    L.mpdp_mlp_forward.argtypes = [c_mlp, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    L.mpdp_mlp_gradients.argtypes = [c_mlp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     P(ctypes.c_float), P(ctypes.c_double)]
    L.mpdp_mlp_train_step.argtypes = [c_mlp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_float]
    for f in ("mpdp_mlp_create", "mpdp_mlp_set_params", "mpdp_mlp_get_params", "mpdp_mlp_forward",
              "mpdp_mlp_gradients", "mpdp_mlp_train_step"):
        getattr(L, f).restype = ctypes.c_int
    L.mpdp_set_model.argtypes = [c_ctx, c_mlp]
    L.mpdp_set_model.restype = ctypes.c_int
    L.mpdp_edge_features.argtypes = [P(QueryC), P(ctypes.c_float), ctypes.c_int32]
    L.mpdp_edge_features.restype = ctypes.c_int
    c_srv = ctypes.c_void_p
    L.mpdp_server_default_config.argtypes = [P(ServerConfigC)]
    L.mpdp_server_create.argtypes = [P(c_srv), ctypes.c_int, P(ServerConfigC)]
    L.mpdp_server_destroy.argtypes = [c_srv]
    L.mpdp_server_destroy.restype = None
    L.mpdp_server_submit.argtypes = [c_srv, P(QueryC), P(ctypes.c_int64)]
    L.mpdp_server_poll.argtypes = [c_srv, P(ctypes.c_int64), ctypes.c_int32, P(ctypes.c_int32)]
    L.mpdp_server_drain.argtypes = [c_srv]
    L.mpdp_server_pending.argtypes = [c_srv, P(ctypes.c_int32), P(ctypes.c_int32)]
    L.mpdp_server_result.argtypes = [c_srv, ctypes.c_int64, P(PlanNode), ctypes.c_int32,
                                     P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_double)]
    for f in ("mpdp_server_default_config", "mpdp_server_create", "mpdp_server_submit",
              "mpdp_server_poll", "mpdp_server_drain", "mpdp_server_pending", "mpdp_server_result"):
        getattr(L, f).restype = ctypes.c_int
    L.mpdp_probe_read_gbs.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, P(ctypes.c_double)]
    L.mpdp_probe_read_gbs.restype = ctypes.c_int
    L.mpdp_memo_lookup.argtypes = [c_ctx, ctypes.c_int64, P(ctypes.c_uint64), ctypes.c_int32,
                                   P(ctypes.c_double), P(ctypes.c_uint64)]
    L.mpdp_last_launch_count.argtypes = [c_ctx]
    L.mpdp_last_launch_count.restype = ctypes.c_int32
    L.mpdp_strerror.argtypes = [ctypes.c_int]
    L.mpdp_strerror.restype = ctypes.c_char_p
    L.mpdp_last_error.argtypes = [c_ctx]
    L.mpdp_last_error.restype = ctypes.c_char_p
    L.mpdp_abi_version.restype = ctypes.c_int32
    L.mpdp_profile.argtypes = [c_ctx, ctypes.c_int]
    L.mpdp_profile_read.argtypes = [c_ctx, P(ctypes.c_double), P(ctypes.c_uint64)]
    L.mpdp_profile_read_active.argtypes = [c_ctx, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_uint64)]
    for f in ("mpdp_optimize_batch_device", "mpdp_profile", "mpdp_profile_read", "mpdp_profile_read_active",
              "mpdp_create", "mpdp_set_config", "mpdp_get_config", "mpdp_optimize",
              "mpdp_optimize_batch", "mpdp_get_plan", "mpdp_release", "mpdp_optimize_device",
              "mpdp_sync", "mpdp_memo_lookup"):
        getattr(L, f).restype = ctypes.c_int
    _LIB = L
    return L


@dataclass
class Plan:
    cost: float
    nodes: np.ndarray                 # NODE_DTYPE records, node 0 = root
    raw_stats: Optional["StatsC"] = None
    n: int = 0
    handle: int = -1
    _stats: Optional[Dict] = None
    cost_xd: Optional[tuple] = None   # heuristic modes: (mantissa, exponent) of the cost

    @property
    def stats(self) -> Dict:
        """Counters of the run (built from the ABI record on first use)."""
        if self._stats is None:
            self._stats = _stats_dict(self.raw_stats, self.n) if self.raw_stats is not None else {}
        return self._stats

    def signature(self, i: int = 0):
        """Nested (set, left-subtree, right-subtree) form; leaves are their set."""
        nd = self.nodes[i]
        if nd["left"] < 0:
            return int(nd["set"])
        return (int(nd["set"]), self.signature(int(nd["left"])), self.signature(int(nd["right"])))


def pack_edges(edges) -> np.ndarray:
    """(u, v, sel) triples as mpdp_edge records (relation indices are small
    integers, exact in a double on the way through)."""
    flat = np.fromiter(itertools.chain.from_iterable(edges), dtype=np.float64, count=3 * len(edges))
    flat = flat.reshape(len(edges), 3)
    arr = np.empty(len(edges), dtype=EDGE_DTYPE)
    arr["u"] = flat[:, 0]
    arr["v"] = flat[:, 1]
    arr["sel"] = flat[:, 2]
    return arr


class _Packed:
    """ABI view of one query (keeps its arrays alive)."""

    def __init__(self, q, mode: int = MODE_EXACT, k: int = 0, t: int = 0):
        self.card = np.ascontiguousarray(np.asarray(q.card, dtype=np.float64))
        self.edges = pack_edges(q.edges)
        self.c = QueryC()
        self.c.n_rels = int(q.n)
        self.c.n_edges = len(q.edges)
        self.c.card = self.card.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.c.edges = self.edges.ctypes.data_as(ctypes.POINTER(Edge)) if len(q.edges) else \
            ctypes.cast(None, ctypes.POINTER(Edge))
        self.c.cost_model = 0
        self.c.mode = mode
        self.c.k = k
        self.c.t = t


QUERY_DTYPE = np.dtype({"names": ["n_rels", "n_edges", "card", "edges", "cost_model", "mode", "k",
                                   "t"],
                         "formats": ["<i4", "<i4", "<u8", "<u8", "<i4", "<i4", "<i4", "<i4"],
                         "offsets": [QueryC.n_rels.offset, QueryC.n_edges.offset, QueryC.card.offset,
                                     QueryC.edges.offset, QueryC.cost_model.offset, QueryC.mode.offset,
                                     QueryC.k.offset, QueryC.t.offset],
                         "itemsize": ctypes.sizeof(QueryC)})


def _pack_batch(queries, mode: int = MODE_EXACT, k: int = 0):
    """mpdp_query records of a batch over two shared arrays (cards, edges)."""
    ns = np.fromiter((q.n for q in queries), dtype=np.int64, count=len(queries))
    ms = np.fromiter((len(q.edges) for q in queries), dtype=np.int64, count=len(queries))
    card = np.fromiter(itertools.chain.from_iterable(q.card for q in queries), dtype=np.float64,
                       count=int(ns.sum()))
    edges = pack_edges([e for q in queries for e in q.edges])
    recs = np.zeros(len(queries), dtype=QUERY_DTYPE)
    recs["n_rels"] = ns
    recs["n_edges"] = ms
    co = np.concatenate([[0], np.cumsum(ns)[:-1]]) if len(queries) else ns
    eo = np.concatenate([[0], np.cumsum(ms)[:-1]]) if len(queries) else ms
    recs["card"] = card.ctypes.data + 8 * co
    recs["edges"] = np.where(ms > 0, edges.ctypes.data + EDGE_DTYPE.itemsize * eo, 0)
    recs["mode"] = mode
    recs["k"] = k
    return card, edges, recs


class PackedBatch:
    """A batch already in the ABI's columnar form: every query's cards back to
    back in one float64 array, its predicates in one mpdp_edge array, and one
    mpdp_query record per query pointing into them.  Callers that hold their
    queries as arrays submit this directly and skip the per-tuple conversion
    of Query objects; the library copies the values on every submit."""

    def __init__(self, queries: Sequence, mode: int = MODE_EXACT, k: int = 0):
        self.card, self.edges, self.recs = _pack_batch(queries, mode, k)
        self.n = [int(q.n) for q in queries]

    def __len__(self) -> int:
        return len(self.n)


def pack_batch(queries: Sequence, mode: int = MODE_EXACT, k: int = 0) -> PackedBatch:
    return PackedBatch(queries, mode, k)


def _stats_dict(st: StatsC, n: int) -> Dict:
    L = n + 1
    return dict(
        sets_unranked=st.sets_unranked, sets_connected=st.sets_connected,
        pairs_evaluated=st.pairs_evaluated, ccp_pairs=st.ccp_pairs, memo_bytes=st.memo_bytes,
        heavy_sets=st.heavy_sets, device_ms=st.device_ms, enumeration=st.enumeration,
        memo_kind=st.memo_kind, h2d_bytes=st.h2d_bytes, d2h_bytes=st.d2h_bytes,
        filter_steps=st.filter_steps,
        connected_per_level=np.array(st.connected_per_level[:L], dtype=np.uint64),
        evaluated_per_level=np.array(st.evaluated_per_level[:L], dtype=np.uint64),
        ccp_per_level=np.array(st.ccp_per_level[:L], dtype=np.uint64),
    )


class Optimizer:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, memo_budget_bytes: int = 0, stream: Optional[int] = None,
                 **config):
        self._lib = load()
        self._ctx = ctypes.c_void_p()
        rc = self._lib.mpdp_create(ctypes.byref(self._ctx), int(device), int(memo_budget_bytes),
                                   ctypes.c_void_p(stream or 0))
        self._check(rc, "mpdp_create")
        self._n = {}
        if config:
            self.set_config(**config)

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != MPDP_OK:
            detail = ""
            if getattr(self, "_ctx", None) and self._ctx.value:
                detail = (self._lib.mpdp_last_error(self._ctx) or b"").decode()
            raise MPDPError(rc, what, detail)

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.mpdp_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration ----------------------------------------------------
    def get_config(self) -> Dict:
        c = ConfigC()
        self._check(self._lib.mpdp_get_config(self._ctx, ctypes.byref(c)), "mpdp_get_config")
        return {f: getattr(c, f) for f, _ in ConfigC._fields_}

    def set_config(self, **kw):
        cur = self.get_config()
        for k, v in kw.items():
            if k not in cur:
                raise KeyError(k)
            cur[k] = int(v)
        c = ConfigC(**cur)
        self._check(self._lib.mpdp_set_config(self._ctx, ctypes.byref(c)), "mpdp_set_config")

    def set_model(self, mlp: Optional["Mlp"]):
        """Attach the learned proposal for MODE_UNIONDP_LEARNED (None: detach)."""
        self._model = mlp
        self._check(self._lib.mpdp_set_model(self._ctx, mlp.handle if mlp is not None else None),
                    "mpdp_set_model")

    def launch_count(self) -> int:
        return int(self._lib.mpdp_last_launch_count(self._ctx))

    # -- host path --------------------------------------------------------
    def submit(self, q, mode: int = MODE_EXACT, k: int = 0, t: int = 0) -> int:
        p = _Packed(q, mode, k, t)
        h = ctypes.c_int64(-1)
        self._check(self._lib.mpdp_optimize(self._ctx, ctypes.byref(p.c), ctypes.byref(h)),
                    "mpdp_optimize")
        self._n[h.value] = int(q.n)
        return h.value

    def get_plan(self, handle: int, release: bool = True) -> Plan:
        n = self._n.get(handle, 32)
        cap = max(2 * n - 1, 1)
        nodes = np.zeros(cap, dtype=NODE_DTYPE)
        nn = ctypes.c_int32(0)
        cost = ctypes.c_double(0.0)
        st = StatsC()
        rc = self._lib.mpdp_get_plan(self._ctx, handle,
                                     nodes.ctypes.data_as(ctypes.POINTER(PlanNode)), cap,
                                     ctypes.byref(nn), ctypes.byref(cost), ctypes.byref(st))
        if rc != MPDP_OK:
            if release:
                self.release(handle)
            self._check(rc, "mpdp_get_plan")
        plan = Plan(cost=cost.value, nodes=nodes[:nn.value].copy(), raw_stats=st, n=n, handle=handle)
        if release:
            self.release(handle)
        return plan

    def release(self, handle: int):
        self._check(self._lib.mpdp_release(self._ctx, handle), "mpdp_release")
        self._n.pop(handle, None)

    def optimize(self, q, mode: int = MODE_EXACT, k: int = 0, keep: bool = False, t: int = 0) -> Plan:
        """Optimize one query through mpdp_optimize + mpdp_get_plan.  In the
        heuristic modes (MODE_IDP2, MODE_UNIONDP) the plan also carries
        cost_xd = (mantissa, exponent): its cost is mantissa * 2^exponent."""
        h = self.submit(q, mode, k, t)
        xd = None
        if mode != MODE_EXACT:
            m, e = ctypes.c_double(0.0), ctypes.c_int32(0)
            self._check(self._lib.mpdp_get_cost_xd(self._ctx, h, ctypes.byref(m), ctypes.byref(e)),
                        "mpdp_get_cost_xd")
            xd = (m.value, e.value)
        plan = self.get_plan(h, release=not keep)
        plan.cost_xd = xd
        return plan

    def submit_batch(self, queries, mode: int = MODE_EXACT, k: int = 0) -> List[int]:
        """Enqueue the queries (mpdp_optimize_batch) and return their handles
        at once; the inputs are copied before this returns.  `queries` is a
        sequence of Query objects or a PackedBatch (whose own mode and k
        apply)."""
        pb = queries if isinstance(queries, PackedBatch) else PackedBatch(queries, mode, k)
        count = len(pb)
        hs = (ctypes.c_int64 * count)()
        rc = self._lib.mpdp_optimize_batch(self._ctx, pb.recs.ctypes.data_as(ctypes.POINTER(QueryC)),
                                           count, hs)
        for n, h in zip(pb.n, hs):
            if h >= 0:
                self._n[h] = n
        if rc != MPDP_OK:
            for h in hs:
                if h >= 0:
                    self.release(h)
            self._check(rc, "mpdp_optimize_batch")
        return list(hs)

    def collect(self, handles: Sequence[int]) -> List[Plan]:
        """Plans of submitted handles in one call (mpdp_get_plans: waits for
        each, releases all); raises the first failing handle's error."""
        count = len(handles)
        if count == 0:
            return []
        ns = [self._n.get(int(h), 32) for h in handles]
        stride = max(2 * max(ns) - 1, 1)
        hs = np.ascontiguousarray(np.asarray(handles, dtype=np.int64))
        nodes = np.zeros((count, stride), dtype=NODE_DTYPE)
        nn = np.zeros(count, dtype=np.int32)
        costs = np.zeros(count, dtype=np.float64)
        status = np.zeros(count, dtype=np.int32)
        stats = (StatsC * count)()
        rc = self._lib.mpdp_get_plans(self._ctx, hs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), count,
                                      nodes.ctypes.data, stride,
                                      nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      costs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), stats)
        for h in handles:
            self._n.pop(int(h), None)
        bad = np.flatnonzero(status != 0)
        if len(bad):
            self._check(int(status[bad[0]]), "mpdp_get_plans")
        self._check(rc, "mpdp_get_plans")
        return [Plan(cost=float(costs[i]), nodes=nodes[i, :nn[i]], raw_stats=stats[i], n=ns[i],
                     handle=int(handles[i])) for i in range(count)]

    def optimize_batch(self, queries, mode: int = MODE_EXACT, k: int = 0) -> List[Plan]:
        return self.collect(self.submit_batch(queries, mode, k))

    def memo_lookup(self, handle: int, sets) -> (np.ndarray, np.ndarray):
        s = np.ascontiguousarray(np.asarray(sets, dtype=np.uint64))
        costs = np.zeros(len(s), dtype=np.float64)
        lefts = np.zeros(len(s), dtype=np.uint64)
        rc = self._lib.mpdp_memo_lookup(self._ctx, handle,
                                        s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(s),
                                        costs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        lefts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        self._check(rc, "mpdp_memo_lookup")
        return costs, lefts

    # -- device path --------------------------------------------------------
    def optimize_device(self, n: int, n_edges: int, d_card, d_edges, d_nodes, d_cost, d_status):
        """Enqueue one optimization whose inputs and outputs are device
        tensors (or raw device pointers); returns without waiting."""
        def ptr(x):
            return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)
        rc = self._lib.mpdp_optimize_device(self._ctx, int(n), int(n_edges), ptr(d_card),
                                            ptr(d_edges), 0, ptr(d_nodes), ptr(d_cost),
                                            ptr(d_status))
        self._check(rc, "mpdp_optimize_device")

    def optimize_batch_device(self, n_rels: Sequence[int], n_edges: Sequence[int], d_card, d_edges,
                              d_nodes, d_cost, d_status):
        """Enqueue one device batch: d_card / d_edges hold the queries' values
        back to back in device memory; d_nodes receives PLAN_STRIDE nodes per
        query, d_cost and d_status one entry per query.  Returns at once."""
        def ptr(x):
            return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)
        nq = len(n_rels)
        nr = (ctypes.c_int32 * nq)(*[int(x) for x in n_rels])
        ne = (ctypes.c_int32 * nq)(*[int(x) for x in n_edges])
        rc = self._lib.mpdp_optimize_batch_device(self._ctx, nq, nr, ne, ptr(d_card), ptr(d_edges), 0,
                                                  ptr(d_nodes), ptr(d_cost), ptr(d_status))
        self._check(rc, "mpdp_optimize_batch_device")

    def sync(self) -> int:
        return int(self._lib.mpdp_sync(self._ctx))

    # -- profiling ----------------------------------------------------------
    def profile(self, mode):
        """PROFILE_OFF / PROFILE_SERIAL / PROFILE_CONCURRENT (True: serial)."""
        self._check(self._lib.mpdp_profile(self._ctx, int(mode)), "mpdp_profile")

    def profile_read(self) -> Dict[str, Dict]:
        """Per kernel class since the last read: summed device ms of its
        launches, their count, and active_ms, the wall time during which at
        least one of them was in flight."""
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        act = (ctypes.c_double * len(KERNEL_CLASSES))()
        ln = (ctypes.c_uint64 * len(KERNEL_CLASSES))()
        self._check(self._lib.mpdp_profile_read_active(self._ctx, ms, act, ln), "mpdp_profile_read_active")
        return {k: dict(ms=ms[i], active_ms=act[i], launches=int(ln[i])) for i, k in enumerate(KERNEL_CLASSES)}


HIDDEN = 256
EDGE_FEATURES = 12


def edge_features(q) -> np.ndarray:
    """mpdp_edge_features: the learned proposal's input rows for q's edges."""
    p = _Packed(q)
    out = np.zeros((max(len(q.edges), 1), EDGE_FEATURES), dtype=np.float32)
    rc = load().mpdp_edge_features(ctypes.byref(p.c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                   len(q.edges))
    if rc != MPDP_OK:
        raise MPDPError(rc, "mpdp_edge_features", strerror(rc))
    return out[:len(q.edges)]


def _dptr(x):
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


class Mlp:
    """The learned proposal's network (mpdp_mlp_*): forward, gradients and
    Adam steps run in the library's BF16 kernels; x / targets are device
    tensors (float32, rows x n_in / rows)."""

    def __init__(self, n_in: int, device: int = 0, stream=None):
        self._lib = load()
        self.n_in = int(n_in)
        self._m = ctypes.c_void_p()
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        rc = self._lib.mpdp_mlp_create(ctypes.byref(self._m), int(device), self.n_in, ctypes.c_void_p(int(st)))
        if rc != MPDP_OK:
            raise MPDPError(rc, "mpdp_mlp_create", strerror(rc))
        self.param_count = int(self._lib.mpdp_mlp_param_count(self._m))

    @property
    def handle(self):
        return self._m

    def close(self):
        if getattr(self, "_m", None) and self._m.value:
            self._lib.mpdp_mlp_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != MPDP_OK:
            raise MPDPError(rc, what, strerror(rc))

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.mpdp_mlp_set_params(self._m, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  p.size), "mpdp_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.param_count, dtype=np.float32)
        self._check(self._lib.mpdp_mlp_get_params(self._m, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  p.size), "mpdp_mlp_get_params")
        return p

    def init_params(self, seed: int = 0) -> np.ndarray:
        """He-normal weights, zero biases (host draw, then copied in)."""
        rng = np.random.default_rng(seed)
        parts = [rng.normal(0, np.sqrt(2.0 / self.n_in), (self.n_in, HIDDEN)), np.zeros(HIDDEN),
                 rng.normal(0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN)), np.zeros(HIDDEN),
                 rng.normal(0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN)), np.zeros(HIDDEN),
                 rng.normal(0, np.sqrt(1.0 / HIDDEN), HIDDEN), np.zeros(1)]
        p = np.concatenate([np.ravel(x) for x in parts]).astype(np.float32)
        self.set_params(p)
        return p

    def forward(self, d_x, rows: int, d_y):
        self._check(self._lib.mpdp_mlp_forward(self._m, _dptr(d_x), int(rows), _dptr(d_y)), "mpdp_mlp_forward")

    def gradients(self, d_x, d_t, rows: int):
        g = np.zeros(self.param_count, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        self._check(self._lib.mpdp_mlp_gradients(self._m, _dptr(d_x), _dptr(d_t), int(rows),
                                                 g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 ctypes.byref(loss)), "mpdp_mlp_gradients")
        return g, loss.value

    def train_step(self, d_x, d_t, rows: int, lr: float):
        self._check(self._lib.mpdp_mlp_train_step(self._m, _dptr(d_x), _dptr(d_t), int(rows), float(lr)),
                    "mpdp_mlp_train_step")


class Server:
    """Serving loop over the library's native scheduler (mpdp_server_*):
    continuous batching over `slots` concurrent device batches, admission
    by memo memory, or (persistent=True) one resident kernel over `slots`
    query slots that takes requests while it runs.  Results are
    bit-identical to optimizing alone."""

    def __init__(self, device: int = 0, slots: Optional[int] = None, max_batch: Optional[int] = None,
                 slot_budget_bytes: Optional[int] = None, persistent: bool = False, **kernel_config):
        self._lib = load()
        cfg = ServerConfigC()
        self._check(self._lib.mpdp_server_default_config(ctypes.byref(cfg)), "mpdp_server_default_config")
        cfg.persistent = 1 if persistent else 0
        if slots is not None:
            cfg.slots = int(slots)
        if max_batch is not None:
            cfg.max_batch = int(max_batch)
        if slot_budget_bytes is not None:
            cfg.slot_budget_bytes = int(slot_budget_bytes)
        for k, v in kernel_config.items():
            if k not in dict(ConfigC._fields_):
                raise KeyError(k)
            setattr(cfg.kernel, k, int(v))
        self._srv = ctypes.c_void_p()
        self._check(self._lib.mpdp_server_create(ctypes.byref(self._srv), int(device), ctypes.byref(cfg)),
                    "mpdp_server_create")
        self._n: Dict[int, int] = {}

    def _check(self, rc, what):
        if rc != MPDP_OK:
            raise MPDPError(rc, what, strerror(rc))

    def close(self):
        if getattr(self, "_srv", None) and self._srv.value:
            self._lib.mpdp_server_destroy(self._srv)
            self._srv = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, q) -> int:
        p = _Packed(q)
        t = ctypes.c_int64(-1)
        self._check(self._lib.mpdp_server_submit(self._srv, ctypes.byref(p.c), ctypes.byref(t)),
                    "mpdp_server_submit")
        self._n[t.value] = int(q.n)
        return t.value

    def poll(self, cap: int = 4096) -> List[int]:
        buf = (ctypes.c_int64 * cap)()
        cnt = ctypes.c_int32(0)
        self._check(self._lib.mpdp_server_poll(self._srv, buf, cap, ctypes.byref(cnt)), "mpdp_server_poll")
        return list(buf[:cnt.value])

    def drain(self):
        self._check(self._lib.mpdp_server_drain(self._srv), "mpdp_server_drain")

    def pending(self):
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._lib.mpdp_server_pending(self._srv, ctypes.byref(a), ctypes.byref(b)),
                    "mpdp_server_pending")
        return a.value, b.value

    def result(self, ticket: int):
        """(Plan, latency in microseconds) of a finished request."""
        n = self._n.get(ticket, 32)
        cap = max(2 * n - 1, 1)
        nodes = np.zeros(cap, dtype=NODE_DTYPE)
        nn = ctypes.c_int32(0)
        cost = ctypes.c_double(0.0)
        lat = ctypes.c_double(0.0)
        rc = self._lib.mpdp_server_result(self._srv, ticket, nodes.ctypes.data_as(ctypes.POINTER(PlanNode)),
                                          cap, ctypes.byref(nn), ctypes.byref(cost), ctypes.byref(lat))
        if rc != ERR["NOT_READY"]:
            self._n.pop(ticket, None)
        self._check(rc, "mpdp_server_result")
        return Plan(cost=cost.value, nodes=nodes[:nn.value].copy(), n=n, handle=ticket), lat.value

    def replay(self, queries: Sequence, arrivals_s: Sequence[float], limit_s: float = 600.0):
        """Submit queries[i] at arrivals_s[i] seconds after the start (busy
        waiting on the host clock, polling in between) and collect every
        result.  Returns (plans, latencies in seconds from each request's
        arrival time, makespan in seconds).  Raises TimeoutError after
        limit_s seconds."""
        import time
        order = np.argsort(np.asarray(arrivals_s), kind="stable")
        tickets = [None] * len(queries)
        lag = [0.0] * len(queries)
        done_lat: Dict[int, float] = {}
        t0 = time.perf_counter()
        nxt = 0
        outstanding = 0
        while nxt < len(order) or outstanding:
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals_s[order[nxt]] <= now:
                i = int(order[nxt])
                tickets[i] = self.submit(queries[i])
                lag[i] = (time.perf_counter() - t0) - arrivals_s[i]
                nxt += 1
                outstanding += 1
            for t in self.poll():
                done_lat[t] = 0.0
                outstanding -= 1
            if now > limit_s:
                raise TimeoutError(f"replay did not finish within {limit_s} s")
        makespan = time.perf_counter() - t0
        plans, lats = [], []
        for i, t in enumerate(tickets):
            p, lat_us = self.result(t)
            plans.append(p)
            lats.append(lag[i] + lat_us * 1e-6)
        return plans, np.asarray(lats), makespan


def optimize_device_noalloc(n: int, n_edges: int, d_card, d_edges, d_nodes, d_cost, d_status,
                            stream=None) -> None:
    """Enqueue the allocation-free optimization of one query of at most
    NOALLOC_MAX_RELS relations (no context; device tensors or raw device
    pointers in and out, as in Optimizer.optimize_device; d_nodes needs
    2n - 1 nodes).  stream: a torch.cuda.Stream, a raw cudaStream_t, or None
    for the current torch stream when torch is loaded, else the legacy
    default stream.  Calls on streams that can overlap share the library's
    fixed memo and race."""
    def ptr(x):
        if x is None:
            return 0
        return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)
    if stream is None:
        torch = sys.modules.get("torch")
        stream = torch.cuda.current_stream().cuda_stream if torch is not None else 0
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    rc = load().mpdp_optimize_device_noalloc(int(n), int(n_edges), ptr(d_card), ptr(d_edges), 0,
                                             ptr(d_nodes), ptr(d_cost), ptr(d_status), int(stream))
    if rc != 0:
        raise MPDPError(rc, "mpdp_optimize_device_noalloc", strerror(rc))


def workspace_bytes(n: int, memo_kind: int = MEMO_DENSE, enumeration: int = ENUM_AUTO) -> int:
    """Device workspace of one exact query of n relations (ENUM_AUTO: a tree
    query; ENUM_BLOCKS: a general join graph)."""
    L = load()
    c = ConfigC(memo_kind, enumeration, 64, 1, 1, 32, FILTER_CONNECTED, 8, 4, 1)
    return int(L.mpdp_workspace_bytes(n, ctypes.byref(c)))


def probe_read_gbs(nbytes: int, passes: int, device: int = 0) -> float:
    """Read bandwidth (GB/s) of one launch reading an nbytes buffer `passes`
    times: below the L2 size it measures the L2, far above it HBM."""
    out = ctypes.c_double()
    rc = load().mpdp_probe_read_gbs(int(device), int(nbytes), int(passes), ctypes.byref(out))
    if rc != MPDP_OK:
        raise MPDPError(rc, "mpdp_probe_read_gbs", strerror(rc))
    return out.value


def strerror(code: int) -> str:
    return load().mpdp_strerror(code).decode()


def nodes_from_bytes(buf: np.ndarray) -> np.ndarray:
    """View a raw byte buffer (e.g. copied from a device tensor) as plan nodes."""
    return np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=NODE_DTYPE)
