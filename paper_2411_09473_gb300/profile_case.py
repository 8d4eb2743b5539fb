"""Run one sampling call (and optionally one selection) of a named workload
through the C ABI, for profiling the kernels under ncu on a case smaller than
a whole IMM run.

  python -m paper_2411_09473_gb300.profile_case --workload ic_u01_1m --theta 2000 [--select 50]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ic_u01_1m")
    ap.add_argument("--theta", type=int, default=2000)
    ap.add_argument("--select", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args()

    import torch

    import graphgen
    from paper_2411_09473_gb300 import imm

    w = graphgen.plain_workload(args.workload)
    g = w.graph
    ctx = imm.imm_create(device=0)
    imm.imm_load_graph(ctx, g.n, g.m, g.row, g.src, g.weight, g.model)
    out = []
    for _ in range(args.repeat):
        imm.imm_reset_sets(ctx)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        imm.imm_sample(ctx, g.model, args.theta, w.seed)
        rec = {"theta": args.theta}
        if args.select:
            seeds, cov = imm.imm_select(ctx, args.select)
            rec["covered"] = cov
            rec["seeds_head"] = [int(x) for x in seeds[:5]]
        torch.cuda.synchronize()
        rec["s"] = time.perf_counter() - t0
        rec["sets"], rec["members"] = imm.imm_stream_size(ctx)
        # in-edges examined = sum over members of their in-degree; IC coin
        # evaluations = (set, in-edge quad) pairs = sum over members of quads
        import numpy as np
        cnt = imm.imm_get_counts(ctx, g.n).astype(np.uint64)
        row = g.row.astype(np.int64)
        indeg = np.diff(row).astype(np.uint64)
        rec["edges"] = int((cnt * indeg).sum())
        quads = np.where(indeg > 0, ((row[1:] - 1) >> 2) - (row[:-1] >> 2) + 1, 0).astype(np.uint64)
        rec["quad_evals"] = int((cnt * quads).sum())
        out.append(rec)
    print(json.dumps(out))
    imm.imm_destroy(ctx)


if __name__ == "__main__":
    main()
