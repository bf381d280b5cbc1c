"""Write the full-size pins of the 255 x 255, S = 256 workload from the FP64 oracle.

For (beta, omega) = (0.3, 1.2) and (0.7, 1.8): the oracle's left-preconditioned
GMRES(30) solve (tol 1e-10, x0 = 0), with the diagonal-block solves of the forward
substitution converged to 1e-13 (tau-preconditioned CG).

* ``config2_oracle.json``: Arnoldi step counts, residual history and estimates, the
  true residual, wall time and host cores of each solve, summaries of f.
* ``config2_oracle_fields.npz``: per instance k, the solution itself: ``f_k`` (the
  source block y^(S+1), N = 65 025 values) and the time levels ``v1_k``, ``vmid_k``,
  ``vS_k`` (v^(1), v^(S/2), v^(S)), lexicographic node order, last index fastest.

Calls only oracle/ and workloads/.  The two instances run in two spawned processes
(the oracle's FFTs are single-threaded); about 70 minutes on an 8-core x86 host.
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
OUT_JSON = os.path.join(HERE, "config2_oracle.json")
OUT_NPZ = os.path.join(HERE, "config2_oracle_fields.npz")
INSTANCES = [(0.3, 1.2), (0.7, 1.8)]


def solve_one(k):
    sys.path.insert(0, ROOT)
    from oracle import system as sy
    from oracle.gmres import gmres
    from workloads import config_2d

    beta, omega = INSTANCES[k]
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
    Y = r.x.reshape(p.S + 1, p.N)
    f = Y[-1]
    rtrue = np.linalg.norm(z - A(r.x)) / np.linalg.norm(z)
    summary = {
        "beta": beta, "omega": omega, "iters": r.iters, "converged": bool(r.converged),
        "relres_est": r.relres_est, "relres_true": float(rtrue), "seconds": wall,
        "precond_calls": calls["n"], "precond_seconds_per_call": calls["t"] / max(1, calls["n"]),
        "seconds_per_arnoldi_step": wall / max(1, r.iters),
        "f_norm2": float(np.linalg.norm(f)), "f_sum": float(f.sum()), "f_center": float(f[p.N // 2]),
        "v_levels": [1, p.S // 2, p.S],
        "history": [float(h) for h in r.history],
    }
    fields = {"f": f.copy(), "v1": Y[0].copy(), "vmid": Y[p.S // 2 - 1].copy(), "vS": Y[p.S - 1].copy()}
    print(json.dumps(summary)[:400], flush=True)
    return summary, fields


def main():
    threads = os.environ.get("OMP_NUM_THREADS", "default")
    res = {"workload": "2-D 255x255, S=256, alpha=1e-4, 1% Gaussian noise (seed 250702809+2)",
           "solver": "oracle GMRES(30), left preconditioning, tol 1e-10, x0 = 0; block solves tau-PCG tol 1e-13",
           "host": {"cpu_count": os.cpu_count(), "processes": len(INSTANCES), "blas_threads": threads},
           "fields": os.path.basename(OUT_NPZ),
           "instances": []}
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(INSTANCES)) as pool:
        out = pool.map(solve_one, range(len(INSTANCES)))
    arrays = {}
    for k, (summary, fields) in enumerate(out):
        res["instances"].append(summary)
        for name, v in fields.items():
            arrays["%s_%d" % (name, k)] = v
    np.savez(OUT_NPZ, **arrays)
    with open(OUT_JSON, "w") as fh:
        json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
