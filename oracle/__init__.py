"""CPU oracle for the MPDP join-order dynamic program.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The product path (``paper_2202_13511_gb300``) never imports this package, and
this package never imports the product path; the two share only the seeded
input generators of ``paper_2202_13511_gb300.workloads`` (which hold no join
ordering arithmetic).

Contents (each restates a definition of arXiv 2202.13511):
  * ``mpdp_oracle.c`` (plain C, fp64, -ffp-contract=off): card(S), grow and
    connected (Sec. 3.2.1), blocks and cut vertices (Sec. 2.4), generic DPSUB
    (Algorithm 1) and DPCCP (the CCP-only enumeration the paper compares
    against, Sec. 1 and Sec. 7.2), and the count of block bipartitions that
    Algorithm 4 visits.
  * ``brute_force`` (pure Python, n <= 7): every bushy join tree without cross
    products (Sec. 2.1.1 "Objective"), costed with C_out, minimised under the
    recursive (x, left) order (x = cost of the two subtrees); it pins the DP
    search of both DPSUB and DPCCP.
  * ``plan_from_memo``: the recursive plan fetch of Sec. 5 ("the final relation
    is recursively fetched using its left and right join relations").

Parity status: every exported function is pinned by ``tests/test_oracle_pins.py``
(brute force, closed-form counts, the paper's printed 2805x / 12024x ratios,
Fig. 5's printed blocks, cut vertices and grow example, exact power-of-two
products, DPSUB == DPCCP).  The one printed number with no unique reading, the
"512 -> 32" count of Sec. 3.2, is pinned under the reading that Algorithm 4's
loop visits both orientations of every block bipartition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "mpdp_oracle.c"), os.path.join(_HERE, "xd_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

OR_OK = 0
OR_INVALID = -1
OR_DISCONNECTED = -2
OR_TOO_LARGE = -3
OR_NOMEM = -4
OR_ORDER = -5


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, no FMA contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_LIB = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_GRAPH_ARGS = [ctypes.c_int, _D, ctypes.c_int, _I32, _I32, _D]


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        lib.oracle_card.argtypes = _GRAPH_ARGS + [ctypes.c_uint64, _D]
        lib.oracle_grow.argtypes = _GRAPH_ARGS + [ctypes.c_uint64, ctypes.c_uint64, _U64]
        lib.oracle_connected.argtypes = _GRAPH_ARGS + [ctypes.c_uint64, _I32]
        lib.oracle_blocks.argtypes = _GRAPH_ARGS + [ctypes.c_uint64, _U64, ctypes.c_int32, _U64]
        lib.oracle_block_enum_counts.argtypes = _GRAPH_ARGS + [_U64, _U64]
        lib.oracle_dpsub.argtypes = _GRAPH_ARGS + [_D, _U32, _U64]
        lib.oracle_dpccp.argtypes = _GRAPH_ARGS + [_D, _U32, _U64]
        xargs = [ctypes.c_int, _D, _I32, ctypes.c_int, _I32, _I32, _D, _I32, _D, _I32, _U32]
        lib.oracle_xd_dpsub.argtypes = xargs
        lib.oracle_xd_dpccp.argtypes = xargs
        lib.oracle_xd_ops.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                      _D, _I32, _D, _I32, _I32]
        lib.oracle_xd_ops.restype = None
        for f in ("oracle_card", "oracle_grow", "oracle_connected", "oracle_blocks",
                  "oracle_block_enum_counts", "oracle_dpsub", "oracle_dpccp", "oracle_xd_dpsub",
                  "oracle_xd_dpccp"):
            getattr(lib, f).restype = ctypes.c_int
        _LIB = lib
    return _LIB


class _Graph:
    """ctypes views of a query's arrays (kept alive for the call)."""

    def __init__(self, q):
        self.n = int(q.n)
        self.m = len(q.edges)
        self.card = np.ascontiguousarray(np.asarray(q.card, dtype=np.float64))
        self.eu = np.ascontiguousarray(np.asarray([e[0] for e in q.edges], dtype=np.int32))
        self.ev = np.ascontiguousarray(np.asarray([e[1] for e in q.edges], dtype=np.int32))
        self.es = np.ascontiguousarray(np.asarray([e[2] for e in q.edges], dtype=np.float64))

    def args(self):
        return (self.n, self.card.ctypes.data_as(_D), self.m, self.eu.ctypes.data_as(_I32),
                self.ev.ctypes.data_as(_I32), self.es.ctypes.data_as(_D))


def _check(rc, what):
    if rc != OR_OK:
        raise OracleError(rc, what)


def card(q, s: int) -> float:
    """card(S): fixed-order product of base cardinalities and selectivities."""
    g = _Graph(q)
    out = ctypes.c_double()
    _check(_lib().oracle_card(*g.args(), ctypes.c_uint64(s), ctypes.byref(out)), "card")
    return out.value


def grow(q, source: int, restriction: int) -> int:
    g = _Graph(q)
    out = ctypes.c_uint64()
    _check(_lib().oracle_grow(*g.args(), ctypes.c_uint64(source), ctypes.c_uint64(restriction),
                              ctypes.byref(out)), "grow")
    return out.value


def connected(q, s: int) -> bool:
    g = _Graph(q)
    out = ctypes.c_int32()
    _check(_lib().oracle_connected(*g.args(), ctypes.c_uint64(s), ctypes.byref(out)),
           "connected")
    return bool(out.value)


def blocks(q, s: int):
    """Blocks of G[S] (ascending masks) and the cut-vertex mask of G[S]."""
    g = _Graph(q)
    buf = (ctypes.c_uint64 * 64)()
    cuts = ctypes.c_uint64()
    nb = _lib().oracle_blocks(*g.args(), ctypes.c_uint64(s), buf, 64, ctypes.byref(cuts))
    if nb < 0:
        raise OracleError(nb, "blocks")
    return [buf[i] for i in range(nb)], cuts.value


def block_enum_counts(q):
    """Per level k: unordered block bipartitions Algorithm 4 visits, and how
    many of them pass the CCP block."""
    g = _Graph(q)
    ev = np.zeros(q.n + 1, dtype=np.uint64)
    va = np.zeros(q.n + 1, dtype=np.uint64)
    _check(_lib().oracle_block_enum_counts(*g.args(), ev.ctypes.data_as(_U64),
                                           va.ctypes.data_as(_U64)), "block_enum_counts")
    return ev, va


@dataclass
class DPResult:
    n: int
    cost: np.ndarray        # float64[2^n], BestPlan cost per connected set
    left: np.ndarray        # uint32[2^n], left mask per connected set
    connected: np.ndarray   # uint64[n+1], connected sets per level
    evaluated: np.ndarray   # uint64[n+1], join pairs evaluated per level
    ccp: np.ndarray         # uint64[n+1], unordered CCP pairs per level

    @property
    def full(self) -> int:
        return (1 << self.n) - 1

    @property
    def opt_cost(self) -> float:
        return float(self.cost[self.full])

    def connected_sets(self) -> np.ndarray:
        """Masks of every connected set with >= 2 relations."""
        idx = np.nonzero(np.isfinite(self.cost))[0]
        return idx[np.array([bin(int(i)).count("1") >= 2 for i in idx], dtype=bool)] \
            if idx.size < 200000 else idx[_popcount_ge2(idx)]


def _popcount_ge2(idx: np.ndarray) -> np.ndarray:
    x = idx.astype(np.uint64)
    return (x & (x - np.uint64(1))) != 0


def _run_dp(q, fn_name: str, init_nan: bool) -> DPResult:
    n = int(q.n)
    g = _Graph(q)
    size = 1 << n
    cost = np.full(size, np.inf, dtype=np.float64)
    left = np.full(size, 0xFFFFFFFF, dtype=np.uint32)
    counters = np.zeros(3 * (n + 1), dtype=np.uint64)
    rc = getattr(_lib(), fn_name)(*g.args(), cost.ctypes.data_as(_D), left.ctypes.data_as(_U32),
                                  counters.ctypes.data_as(_U64))
    _check(rc, fn_name)
    L = n + 1
    return DPResult(n=n, cost=cost, left=left, connected=counters[0:L].copy(),
                    evaluated=counters[L:2 * L].copy(), ccp=counters[2 * L:3 * L].copy())


def dpsub(q) -> DPResult:
    """Generic DPSUB, Algorithm 1 (n <= 20)."""
    return _run_dp(q, "oracle_dpsub", True)


def dpccp(q) -> DPResult:
    """DPCCP: enumerates only CCP pairs (n <= 28)."""
    return _run_dp(q, "oracle_dpccp", True)


def optimize(q) -> DPResult:
    """The oracle's exact optimum: DPCCP."""
    return dpccp(q)


def plan_from_memo(q, res: DPResult) -> List[Dict]:
    """Recursive plan fetch from the root (Sec. 5): nodes in pre-order; each
    node has its relation set, child indices (-1 for a leaf), the leaf's
    relation, card(S) and the memo cost.  The left child is the memo's left
    mask, the right child its complement within the node."""
    nodes: List[Dict] = []

    def visit(s: int) -> int:
        i = len(nodes)
        nodes.append({})
        if s & (s - 1) == 0:
            nodes[i] = dict(set=s, left=-1, right=-1, rel=s.bit_length() - 1,
                            card=float(q.card[s.bit_length() - 1]), cost=0.0)
            return i
        lm = int(res.left[s])
        rm = s & ~lm
        li = visit(lm)
        ri = visit(rm)
        nodes[i] = dict(set=s, left=li, right=ri, rel=-1, card=card(q, s),
                        cost=float(res.cost[s]))
        return i

    visit(res.full)
    return nodes


def plan_signature(nodes: List[Dict], i: int = 0):
    """Canonical nested form (set, left-subtree, right-subtree) of a plan."""
    nd = nodes[i]
    if nd["left"] < 0:
        return nd["set"]
    return (nd["set"], plan_signature(nodes, nd["left"]), plan_signature(nodes, nd["right"]))


# ---------------------------------------------------------------------------
# Brute force over every cross-product-free bushy join tree (pure Python).

def _adjacency(q):
    adj = [0] * q.n
    for (u, v, _s) in q.edges:
        adj[u] |= 1 << v
        adj[v] |= 1 << u
    return adj


def brute_force(q, max_n: int = 7):
    """Enumerate every bushy join tree over all relations whose every join has
    at least one predicate between its two inputs (no cross products, Sec. 2.1),
    cost each with C_out, and return the minimum under the recursive key
    (x, left mask, key of the subtree on the left mask, key of the other),
    where x = cost(left subtree) + cost(right subtree) and the tree's cost is
    x + card(S).  Returns (cost, signature, number of trees), the signature as
    in ``plan_signature``."""
    if q.n > max_n:
        raise ValueError("brute force is for tiny queries")
    adj = _adjacency(q)
    card_cache: Dict[int, float] = {}

    def card_of(s):
        if s not in card_cache:
            card_cache[s] = card(q, s)
        return card_cache[s]

    def joined(a, b):
        x = 0
        t = a
        while t:
            low = t & -t
            x |= adj[low.bit_length() - 1]
            t ^= low
        return (x & b) != 0

    memo: Dict[int, list] = {}

    def trees(s):
        """All cross-product-free trees over s as (key, signature, cost)."""
        if s in memo:
            return memo[s]
        if s & (s - 1) == 0:
            memo[s] = [((0.0,), s, 0.0)]
            return memo[s]
        out = []
        low = s & -s
        rest = s & ~low
        sub = rest
        while True:
            a = low | sub
            b = s & ~a
            if b and joined(a, b):
                for (ka, sa, ca) in trees(a):
                    for (kb, sb, cb) in trees(b):
                        x = ca + cb
                        c = x + card_of(s)
                        if a < b:
                            key = (x, a, ka, kb)
                            sig = (s, sa, sb)
                        else:
                            key = (x, b, kb, ka)
                            sig = (s, sb, sa)
                        out.append((key, sig, c))
            if sub == 0:
                break
            sub = (sub - 1) & rest
        memo[s] = out
        return out

    full = (1 << q.n) - 1
    all_trees = trees(full)
    if not all_trees:
        raise OracleError(OR_DISCONNECTED, "brute_force")
    best = min(all_trees, key=lambda t: t[0])
    # the minimum x gives the minimum cost (addition is monotone): check it
    assert best[2] == min(t[2] for t in all_trees)
    return best[2], best[1], len(all_trees)


# ---------------------------------------------------------------------------
# Extended range (xd_oracle.c): values m * 2^e, m = 0 or 1 <= m < 2.

def xd_ops(a, b):
    """(a + b, a * b, compare(a, b)) of two (mantissa, exponent) values,
    as xd_oracle.c computes them."""
    sm, se, pm, pe, c = (ctypes.c_double(), ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32(),
                         ctypes.c_int32())
    _lib().oracle_xd_ops(float(a[0]), int(a[1]), float(b[0]), int(b[1]), ctypes.byref(sm), ctypes.byref(se),
                         ctypes.byref(pm), ctypes.byref(pe), ctypes.byref(c))
    return (sm.value, se.value), (pm.value, pe.value), c.value


@dataclass
class XDResult:
    cost_m: np.ndarray   # [2^n] mantissa of cost(S) (0 for singletons and unformed sets)
    cost_e: np.ndarray   # [2^n] exponent
    left: np.ndarray     # [2^n] left(S); UINT32_MAX for sets never formed

    def cost(self, s: int):
        return (float(self.cost_m[s]), int(self.cost_e[s]))


def xd_dp(n, card, edges, method: str = "dpccp") -> XDResult:
    """The exact DP in extended range.  card: n (mantissa, exponent) pairs;
    edges: (u, v, (mantissa, exponent)) with the selectivity in XD."""
    cm = np.ascontiguousarray([float(c[0]) for c in card], dtype=np.float64)
    ce = np.ascontiguousarray([int(c[1]) for c in card], dtype=np.int32)
    eu = np.ascontiguousarray([int(e[0]) for e in edges], dtype=np.int32)
    ev = np.ascontiguousarray([int(e[1]) for e in edges], dtype=np.int32)
    sm = np.ascontiguousarray([float(e[2][0]) for e in edges], dtype=np.float64)
    se = np.ascontiguousarray([int(e[2][1]) for e in edges], dtype=np.int32)
    size = 1 << n
    out_m = np.zeros(size, dtype=np.float64)
    out_e = np.zeros(size, dtype=np.int32)
    left = np.zeros(size, dtype=np.uint32)
    fn = _lib().oracle_xd_dpccp if method == "dpccp" else _lib().oracle_xd_dpsub
    _check(fn(n, cm.ctypes.data_as(_D), ce.ctypes.data_as(_I32), len(edges), eu.ctypes.data_as(_I32),
              ev.ctypes.data_as(_I32), sm.ctypes.data_as(_D), se.ctypes.data_as(_I32),
              out_m.ctypes.data_as(_D), out_e.ctypes.data_as(_I32), left.ctypes.data_as(_U32)),
           "xd_" + method)
    return XDResult(out_m, out_e, left)
