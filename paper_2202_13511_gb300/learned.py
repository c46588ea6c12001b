"""Learned proposal for UnionDP and IDP2 (a project addition; the paper cites
learned optimizers only as related work).

A 3 x 256 MLP (mpdp_mlp_*: the library's own BF16 forward/backward kernels)
scores every edge of a query graph with a prediction of how much of the query
lies under that edge's join in an optimal plan.  UnionDP in
MODE_UNIONDP_LEARNED then unites edges in ascending score, so the joins an
optimal plan makes early stay inside partitions and the late ones become cut
edges.  IDP2 in MODE_IDP2_LEARNED starts from the plan that joins the edges
in ascending score instead of GOO's.  The plain heuristic is each proposal's
fallback: the optimizer costs both plans exactly and keeps the cheaper one.

Training data are exact MPDP plans of <= 25-relation queries: for an edge
(u, v), the label is n_leaves(LCA(u, v)) / n, where LCA(u, v) is the plan
node at which u and v first meet.  Features come from mpdp_edge_features,
the same C++ code the optimizer runs at every UnionDP round.
"""
from __future__ import annotations

import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import mpdp
from . import workloads as W


def training_queries(count: int, seed: int = 0, n_lo: int = 10, n_hi: int = 25) -> List:
    """Primary-key/foreign-key snowflakes with extra edges (the shape of the
    large queries the heuristics serve), sizes uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        frac = float(rng.choice([0.0, 0.05, 0.1, 0.15]))
        out.append(W.snowflake_plus_pkfk(n, seed=int(seed * 1_000_003 + i), extra_frac=frac))
    return out


def edge_labels(q, nodes: np.ndarray) -> np.ndarray:
    """n_leaves of the smallest plan node holding both ends of each edge,
    over n (plans of n <= 64 carry relation bitmaps)."""
    sets = nodes["set"].astype(np.uint64)
    leaves = nodes["n_leaves"].astype(np.int64)
    both = np.array([(1 << u) | (1 << v) for u, v, _s in q.edges], dtype=np.uint64)
    hit = (sets[None, :] & both[:, None]) == both[:, None]
    # the root holds every relation, so each edge has a hit
    return (np.where(hit, leaves[None, :], np.iinfo(np.int64).max).min(axis=1) / q.n).astype(np.float32)


def build_dataset(opt: "mpdp.Optimizer", queries: Sequence, batch: int = 256) -> Tuple[np.ndarray, np.ndarray]:
    """(features, labels) of every edge of every query, labels from the exact
    plans the optimizer itself returns."""
    xs, ts = [], []
    for b in range(0, len(queries), batch):
        part = queries[b:b + batch]
        for q, p in zip(part, opt.optimize_batch(part)):
            xs.append(mpdp.edge_features(q))
            ts.append(edge_labels(q, p.nodes))
    return np.concatenate(xs), np.concatenate(ts)


def train(x: np.ndarray, t: np.ndarray, epochs: int = 8, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          device: int = 0, log: Optional[list] = None) -> "mpdp.Mlp":
    """Train the proposal network on the GPU (minibatch Adam steps in the
    library's kernels).  log, when given, receives (epoch, loss, seconds):
    first (-1, loss of the initial network, 0), then one entry per epoch,
    each loss over the same first 16,384 rows."""
    import torch
    torch.cuda.set_device(device)
    mlp = mpdp.Mlp(x.shape[1], device, stream=torch.cuda.current_stream())
    mlp.init_params(seed)
    dx = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda()
    rows = dx.shape[0]
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    n_eval = min(rows, 16384)

    def eval_loss():
        _, loss = mlp.gradients(dx[:n_eval].contiguous(), dt[:n_eval].contiguous(), n_eval)
        torch.cuda.synchronize()
        return loss

    if log is not None:
        log.append((-1, eval_loss(), 0.0))
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(rows, generator=gen).cuda()
        for b in range(0, rows, batch):
            idx = perm[b:b + batch]
            bx = dx.index_select(0, idx).contiguous()
            bt = dt.index_select(0, idx).contiguous()
            mlp.train_step(bx, bt, bx.shape[0], lr)
        if log is not None:
            log.append((ep, eval_loss(), time.perf_counter() - t0))
    torch.cuda.synchronize()
    return mlp


def cost_ratio(a, b) -> float:
    """cost_xd a / cost_xd b."""
    return a[0] / b[0] * 2.0 ** (a[1] - b[1])


def evaluate(opt: "mpdp.Optimizer", mlp: "mpdp.Mlp", queries: Sequence, k: int = 25, t: int = 15):
    """Per query: costs of plain UnionDP, learned UnionDP (the learned
    proposal with plain UnionDP as its fallback) and IDP2(k)."""
    rows = []
    for q in queries:
        opt.set_model(None)
        plain = opt.optimize(q, mode=mpdp.MODE_UNIONDP, k=k, t=t).cost_xd
        opt.set_model(mlp)
        learned = opt.optimize(q, mode=mpdp.MODE_UNIONDP_LEARNED, k=k, t=t).cost_xd
        opt.set_model(None)
        idp2 = opt.optimize(q, mode=mpdp.MODE_IDP2, k=k).cost_xd
        rows.append((plain, learned, idp2))
    return rows


def evaluate_idp2(opt: "mpdp.Optimizer", mlp: "mpdp.Mlp", queries: Sequence, k: int = 25):
    """Per query: costs of plain IDP2(k) (GOO start) and learned IDP2(k)
    (learned start, plain IDP2 as its fallback)."""
    rows = []
    for q in queries:
        opt.set_model(None)
        plain = opt.optimize(q, mode=mpdp.MODE_IDP2, k=k).cost_xd
        opt.set_model(mlp)
        learned = opt.optimize(q, mode=mpdp.MODE_IDP2_LEARNED, k=k).cost_xd
        opt.set_model(None)
        rows.append((plain, learned))
    return rows
