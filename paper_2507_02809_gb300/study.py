"""Reconstruction study of Sec. 6.1.3 (1-D) on the GPU.

    python -m paper_2507_02809_gb300.study [--n 256] [--S 64] [--seed 3]

For each (beta, omega) of Tables 3-5: the exact source f = x sin x on (0, pi) (Sec. 6.1); the data
mu = u(., T) from the direct problem (tsfde_direct_solve: the first S stages of the forward
substitution); mu_eps = mu + eps delta with delta ~ U(-1, 1) per node and eps = level ||mu||_2; for
each regularisation parameter lambda the system of Eq. 11 is solved by GMRES with P (tol 1e-12) and
f~ compared with f.  Prints the relative errors beside the paper's row for n = 2^8, S = 2^6.
"""
from __future__ import annotations

import argparse
import dataclasses
import os
import sys

import numpy as np

LEVELS = ((0.001, (1e-5, 1e-4, 1e-3)), (0.01, (1e-4, 1e-3, 1e-2)))
# Tables 3, 4, 5 (Sec. 6.1.3), row n = 2^8, S = 2^6: level 0.001 (lambda 1e-5, 1e-4, 1e-3) and
# level 0.01 (lambda 1e-4, 1e-3, 1e-2)
PAPER_N256_S64 = {(0.1, 1.9): (0.06, 0.02, 0.05, 0.14, 0.05, 0.25),
                  (0.5, 1.5): (0.10, 0.02, 0.04, 0.20, 0.07, 0.22),
                  (0.9, 1.1): (0.11, 0.03, 0.04, 0.28, 0.07, 0.23)}


def reconstruction_errors(n: int, S: int, beta: float, omega: float, seed: int = 3, opts=None) -> list:
    """The six relative errors of one row of Tables 3-5 (levels x lambdas), computed on the GPU."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from workloads import add_noise_uniform, paper_1d

    from . import tsfde as t
    if opts is None:
        opts = t.tsfde_default_opts(tol=1e-12, inner_tol=1e-12)
    w = paper_1d(n, S, beta, omega)
    s = t.Solver(w.with_mu(np.zeros(n)), opts=opts)
    v = np.zeros(S * n)
    s.direct_solve(v, f=np.ascontiguousarray(w.f_true))
    s.close()
    mu = v[(S - 1) * n:]
    errs = []
    for level, lams in LEVELS:
        mue = add_noise_uniform(mu, level, np.random.default_rng(seed))
        for lam in lams:
            si = t.Solver(dataclasses.replace(w, alpha=lam, mu=mue), opts=opts)
            y = np.zeros(si.U)
            si.solve(y)
            si.close()
            f = y[-n:]
            errs.append(float(np.linalg.norm(f - w.f_true) / np.linalg.norm(w.f_true)))
    return errs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--S", type=int, default=64)
    ap.add_argument("--seed", type=int, default=3)
    args = ap.parse_args(argv)
    print("relative error of the recovered source, n = %d, S = %d (paper row: n = 256, S = 64)" % (args.n, args.S))
    print("beta omega | eps 0.001: lambda 1e-5 1e-4 1e-3 | eps 0.01: lambda 1e-4 1e-3 1e-2")
    for (b, o), paper in PAPER_N256_S64.items():
        got = reconstruction_errors(args.n, args.S, b, o, args.seed)
        print("%.1f  %.1f  GPU   | %s | %s" % (b, o, " ".join("%.3f" % e for e in got[:3]),
                                               " ".join("%.3f" % e for e in got[3:])))
        print("          paper | %s | %s" % (" ".join("%.2f " % e for e in paper[:3]),
                                             " ".join("%.2f " % e for e in paper[3:])))


if __name__ == "__main__":
    main()
