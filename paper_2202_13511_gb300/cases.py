"""Run one workload shape through the device path (for profiler captures).

    python -m paper_2202_13511_gb300.cases --kind star --n 25 --reps 3
    python -m paper_2202_13511_gb300.cases --kind snowflake --n 25 --queries 4 --lanes 1

All queries of a rep go to the GPU as one device batch.  Nothing is checked
beyond the device status words; this only exists so that a profiler can
capture the kernels of one shape in isolation.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def main(argv=None) -> int:
    p = argparse.ArgumentParser()
    p.add_argument("--kind", default="snowflake")
    p.add_argument("--n", type=int, default=25)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--queries", type=int, default=1)
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--memo", choices=["dense", "hash"], default="dense")
    p.add_argument("--enumeration", choices=["auto", "tree", "blocks"], default="auto")
    p.add_argument("--lanes", type=int, default=0, help="concurrent sub-batches (0: library default)")
    a = p.parse_args(argv)
    import torch
    from . import mpdp
    from . import workloads as W
    torch.cuda.set_device(0)
    opt = mpdp.Optimizer(0, stream=torch.cuda.current_stream().cuda_stream,
                         memo_kind={"dense": mpdp.MEMO_DENSE, "hash": mpdp.MEMO_HASH}[a.memo],
                         enumeration={"auto": mpdp.ENUM_AUTO, "tree": mpdp.ENUM_TREE,
                                      "blocks": mpdp.ENUM_BLOCKS}[a.enumeration])
    if a.lanes:
        opt.set_config(lanes=a.lanes)
    qs = [W.make(a.kind, a.n, seed=a.seed + i) for i in range(a.queries)]
    d_card = torch.tensor([c for q in qs for c in q.card], dtype=torch.float64, device="cuda")
    d_edges = torch.from_numpy(
        mpdp.pack_edges([e for q in qs for e in q.edges]).view(np.uint8).copy()).cuda()
    nq = len(qs)
    d_nodes = torch.zeros((nq, mpdp.PLAN_STRIDE * 40), dtype=torch.uint8, device="cuda")
    d_cost = torch.zeros(nq, dtype=torch.float64, device="cuda")
    d_status = torch.full((nq,), -100, dtype=torch.int32, device="cuda")
    for _ in range(a.reps):
        opt.optimize_batch_device([q.n for q in qs], [len(q.edges) for q in qs], d_card, d_edges,
                                  d_nodes, d_cost, d_status)
    torch.cuda.synchronize()
    bad = [int(x) for x in d_status.cpu().numpy() if x != 0]
    opt.close()
    print(f"{a.kind}-{a.n} x{a.queries} reps={a.reps} status={'ok' if not bad else bad}")
    return 0 if not bad else 1


if __name__ == "__main__":
    sys.exit(main())
