"""The batched workload on the GPU: 64 instances of uneven sizes and parameters.

    python -m paper_2507_02809_gb300.batch_study [--precision mixed|fp64] [--sequential] [--grouped]
                                                 [--count-1d 32] [--count-2d 32]

32 instances with d = 1 (n from 127..2047, S from 64..512) and 32 with d = 2 (n x n, n from 63..255,
S from 64..256), beta, omega, alpha, gamma1, gamma2 drawn per instance (workloads.config_batch).
All instances are solved by one tsfde_gmres_solve_batch call: their GMRES run in lockstep and every
round of preconditioner applications is one launch of the mixed-length persistent kernel (one
sub-grid per instance).  --grouped instead solves one batch per (d, transform length), each with
the kernel of that length.  Default: FP32 preconditioner inside flexible FP64 GMRES(30), true
residual 1e-10.  --sequential also solves every instance alone and reports the batched speedup.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import sys
import time


def _grid_len(n: int) -> int:
    p = 1
    while p < n + 1:
        p <<= 1
    return 2 * p


def run(precision: str = "mixed", sequential: bool = False, count_1d: int = 32, count_2d: int = 32,
        grouped: bool = False) -> dict:
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch

    from workloads import config_batch

    from . import tsfde as t
    if precision == "mixed":
        opts = t.tsfde_default_opts(precision=t.PREC_MIXED, side=t.SIDE_FLEXIBLE, tol=1e-10)
    else:
        opts = t.tsfde_default_opts(precision=t.PREC_FP64, side=t.SIDE_LEFT, tol=1e-10)
    ws = config_batch(count_1d, count_2d)
    groups = collections.OrderedDict()
    if grouped:
        for w in ws:
            groups.setdefault((w.d, _grid_len(w.ns[0])), []).append(w)
    else:
        groups[("all", "mixed")] = ws
    out = {"instances": len(ws), "unknowns": int(sum(w.U for w in ws)), "precision": precision,
           "launch": "one batch per (d, L)" if grouped else "one batch, mixed-length launches", "groups": []}
    tb_total = ts_total = 0.0
    for (d, L), gw in groups.items():
        solvers = [t.Solver(w, opts=opts) for w in gw]
        ys = [torch.zeros(s.U, dtype=torch.float64, device="cuda") for s in solvers]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = t.tsfde_gmres_solve_batch([s.handle for s in solvers], ys)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        g = {"d": d, "L": L, "count": len(gw), "unknowns": int(sum(w.U for w in gw)), "batched_s": tb,
             "iters": [i["iters"] for i in infos], "converged": all(i["converged"] for i in infos),
             "max_relres_true": max(i["relres_true"] for i in infos)}
        if sequential:
            ts = 0.0
            diffs = []
            for s, y in zip(solvers, ys):
                y2 = torch.zeros_like(y)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.solve(y2)
                torch.cuda.synchronize()
                ts += time.perf_counter() - t0
                diffs.append(float(torch.linalg.norm(y2 - y) / torch.linalg.norm(y2)))
            g["sequential_s"] = ts
            g["speedup"] = ts / tb
            g["max_rel_diff_batched_vs_single"] = max(diffs)
            ts_total += ts
        tb_total += tb
        for s in solvers:
            s.close()
        del ys
        torch.cuda.empty_cache()
        out["groups"].append(g)
    out["batched_s"] = tb_total
    if sequential:
        out["sequential_s"] = ts_total
        out["speedup"] = ts_total / tb_total
    out["all_converged"] = all(g["converged"] for g in out["groups"])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--sequential", action="store_true")
    ap.add_argument("--grouped", action="store_true")
    ap.add_argument("--count-1d", type=int, default=32)
    ap.add_argument("--count-2d", type=int, default=32)
    args = ap.parse_args(argv)
    res = run(args.precision, args.sequential, args.count_1d, args.count_2d, args.grouped)
    for g in res["groups"]:
        print("d=%s L=%4s: %2d instances, %9d unknowns, batched %.2f s%s, iters %s" % (
            g["d"], g["L"], g["count"], g["unknowns"], g["batched_s"],
            (", sequential %.2f s (x%.2f)" % (g["sequential_s"], g["speedup"])) if "speedup" in g else "",
            g["iters"]))
    print(json.dumps({k: v for k, v in res.items() if k != "groups"}))


if __name__ == "__main__":
    main()
