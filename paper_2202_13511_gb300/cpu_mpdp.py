"""Binding of the multi-threaded CPU MPDP (include/mpdp_cpu.h): the paper's
host implementation of the method (Sec. 3.3), kept as the "MPDP (24CPU)"
comparison of Sec. 7.2.  A baseline that runs on the host cores; the GPU
library never calls it."""
from __future__ import annotations

import ctypes
import os
from typing import Tuple

import numpy as np

from . import _build
from . import mpdp

MAX_RELS = 30


class CpuStats(ctypes.Structure):
    _fields_ = [("sets_unranked", ctypes.c_uint64), ("sets_connected", ctypes.c_uint64),
                ("pairs_evaluated", ctypes.c_uint64), ("ccp_pairs", ctypes.c_uint64),
                ("threads", ctypes.c_int32), ("reserved", ctypes.c_int32), ("wall_ms", ctypes.c_double)]


_LIB = None


def load():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build_cpu())
        lib.mpdp_cpu_optimize.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(CpuStats)]
        lib.mpdp_cpu_optimize.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def cores() -> int:
    return os.cpu_count() or 1


def optimize(q, threads: int = 0) -> Tuple["mpdp.Plan", dict]:
    """Exact MPDP of q on `threads` host threads (0: every online core)."""
    lib = load()
    card = np.ascontiguousarray(q.card, dtype=np.float64)
    edges = mpdp.pack_edges(q.edges)
    nodes = np.zeros(max(2 * q.n - 1, 1), dtype=mpdp.NODE_DTYPE)
    n_nodes = ctypes.c_int32()
    cost = ctypes.c_double()
    st = CpuStats()
    rc = lib.mpdp_cpu_optimize(int(q.n), card.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(q.edges),
                               edges.ctypes.data if len(q.edges) else None, int(threads),
                               nodes.ctypes.data, len(nodes), ctypes.byref(n_nodes), ctypes.byref(cost),
                               ctypes.byref(st))
    if rc != mpdp.MPDP_OK:
        raise mpdp.MPDPError(rc, "mpdp_cpu_optimize", mpdp.strerror(rc))
    stats = {f[0]: getattr(st, f[0]) for f in CpuStats._fields_ if f[0] != "reserved"}
    return mpdp.Plan(cost=cost.value, nodes=nodes[:n_nodes.value]), stats
