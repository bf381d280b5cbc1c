"""Spectral diagnostics of A_{n,S} and P_{n,S}^-1 A_{n,S} on the GPU (Sec. 6.1.1, 6.2.1).

    python -m paper_2507_02809_gb300.spectral [--n 256] [--S 64] [--k 80]

Condition numbers by Golub-Kahan bidiagonalisation (tsfde_spectral_bidiag: the singular values of
the small bidiagonal matrix estimate those of the operator; sigma_max converges first, sigma_min
after more steps, enough for P^-1 A); the far smaller sigma_min of A itself by inverse iteration on
A^T A through the GPU solves; eigenvalues by Arnoldi (tsfde_spectral_arnoldi: Ritz values).  The CLI prints
cond_2(A) and cond_2(P^-1 A) for the 1-D workload of Table 1 (lambda = 5e-3) beside the paper's row
for n = 2^8, S = 2^6.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

# Table 1 (Sec. 6.1.1), row n = 2^8, S = 2^6: (cond A, cond P^-1 A) for (beta, omega)
PAPER_TABLE1_N256_S64 = {(0.1, 1.9): (1751554, 74), (0.5, 1.5): (74164, 123), (0.9, 1.1): (19073, 213)}


def _bidiag_matrix(alpha, beta):
    k = len(alpha)
    B = np.zeros((k + 1, k))
    B[np.arange(k), np.arange(k)] = alpha
    B[np.arange(1, k + 1), np.arange(k)] = beta
    return B


def singular_values(solver, which: int, k: int, seed: int = 0) -> np.ndarray:
    """Singular values of the k-step bidiagonal matrix of M = A (which 0) or P^-1 A (1), largest
    first."""
    from . import tsfde as t
    u0 = np.random.default_rng(seed).standard_normal(solver.U)
    alpha, beta = t.tsfde_spectral_bidiag(solver.handle, which, k, u0)
    keep = int(np.count_nonzero(alpha))
    return np.linalg.svd(_bidiag_matrix(alpha[:keep], beta[:keep]), compute_uv=False)


def condition_estimate(solver, which: int, k: int, seed: int = 0):
    """(sigma_max, sigma_min, sigma_max / sigma_min) from k bidiagonalisation steps."""
    sv = singular_values(solver, which, k, seed)
    return sv[0], sv[-1], sv[0] / sv[-1]


def sigma_min_inverse_iteration(solver, iters: int = 30, seed: int = 0, rtol: float = 1e-6) -> float:
    """sigma_min(A) by inverse iteration on A^T A: each step one adjoint solve (A^T y = x) and one
    solve (A x' = y) by the handle's preconditioned GMRES; sigma_min^-2 is the growth ||x'|| / ||x||
    of a normalised x once it has converged (relative change below rtol)."""
    from . import tsfde as t
    x = np.random.default_rng(seed).standard_normal(solver.U)
    x /= np.linalg.norm(x)
    prev = None
    for _ in range(iters):
        y = np.zeros(solver.U)
        t.tsfde_adjoint(solver.handle, None, x, y)
        x2 = np.zeros(solver.U)
        t.tsfde_solve(solver.handle, y, x2)
        g = np.linalg.norm(x2)
        x = x2 / g
        if prev is not None and abs(g - prev) <= rtol * g:
            break
        prev = g
    return 1.0 / np.sqrt(g)


def ritz_values(solver, which: int, k: int, seed: int = 0):
    """Ritz values of M from up to k Arnoldi steps, and the number of steps done."""
    from . import tsfde as t
    v0 = np.random.default_rng(seed).standard_normal(solver.U)
    H, steps = t.tsfde_spectral_arnoldi(solver.handle, which, k, v0)
    return np.linalg.eigvals(H[:steps, :steps]), steps


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--S", type=int, default=64)
    ap.add_argument("--k", type=int, default=80)
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from workloads import paper_1d

    from . import tsfde as t
    print("cond_2 estimates, n = %d, S = %d (paper row: n = 256, S = 64): A by 40 bidiagonalisation steps for "
          "sigma_max and inverse iteration for sigma_min, P^-1 A by %d bidiagonalisation steps"
          % (args.n, args.S, args.k))
    for (b, o), (pa, pp) in PAPER_TABLE1_N256_S64.items():
        w = paper_1d(args.n, args.S, b, o)
        s = t.Solver(w.with_mu(np.zeros(args.n)), opts=t.tsfde_default_opts(inner_tol=1e-12))
        smax = singular_values(s, 0, 40)[0]
        smin = sigma_min_inverse_iteration(s)
        cp = condition_estimate(s, 1, args.k)
        s.close()
        print("beta %.1f omega %.1f: cond(A) %.6g (paper %d), cond(P^-1 A) %.4g (paper %d)"
              % (b, o, smax / smin, pa, cp[2], pp))


if __name__ == "__main__":
    main()
