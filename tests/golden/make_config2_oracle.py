"""Write tests/golden/config2_oracle.json: the FP64 oracle's left-preconditioned GMRES(30)
solve (tol 1e-10, x0 = 0) of the 255 x 255, S = 256 workload for (beta, omega) =
(0.3, 1.2) and (0.7, 1.8), with the diagonal-block solves of the forward substitution
converged to 1e-13 (tau-preconditioned CG).  Records the Arnoldi step counts, the residual
estimates, the time of one Arnoldi step and summaries of the solution.

Calls only oracle/ and workloads/.  Takes about half an hour per instance on 8 cores.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import system as sy  # noqa: E402
from oracle.gmres import gmres  # noqa: E402
from workloads import config_2d  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_oracle.json")


def main():
    res = {"workload": "2-D 255x255, S=256, alpha=1e-4, 1% Gaussian noise (seed 250702809+2)",
           "solver": "oracle GMRES(30), left preconditioning, tol 1e-10, x0 = 0; block solves tau-PCG tol 1e-13",
           "instances": []}
    for (beta, omega) in [(0.3, 1.2), (0.7, 1.8)]:
        w = config_2d(beta, omega)
        p = sy.problem_from(w)
        z = sy.rhs(p)
        calls = {"n": 0, "t": 0.0}

        def A(v):
            return sy.matvec(p, v)

        def M(v):
            t0 = time.time()
            out = sy.precond_solve_structured(p, v, tol=1e-13)
            calls["n"] += 1
            calls["t"] += time.time() - t0
            return out

        t0 = time.time()
        r = gmres(A, z, M, side="left", restart=30, tol=1e-10, maxit=3000)
        wall = time.time() - t0
        f = r.x.reshape(p.S + 1, p.N)[-1]
        rtrue = np.linalg.norm(z - A(r.x)) / np.linalg.norm(z)
        res["instances"].append({
            "beta": beta, "omega": omega, "iters": r.iters, "converged": bool(r.converged),
            "relres_est": r.relres_est, "relres_true": float(rtrue), "seconds": wall,
            "precond_calls": calls["n"], "precond_seconds_per_call": calls["t"] / max(1, calls["n"]),
            "seconds_per_arnoldi_step": wall / max(1, r.iters),
            "f_norm2": float(np.linalg.norm(f)), "f_sum": float(f.sum()), "f_center": float(f[p.N // 2]),
            "history": [float(h) for h in r.history],
        })
        print(json.dumps(res["instances"][-1])[:400], flush=True)
        with open(OUT, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
