"""Adjoint of the all-at-once system (oracle; test infrastructure only).

For a misfit J(y) of the solution y = A^{-1} z of Eq. 11 the gradient with respect to a
parameter theta of A or z is

    dJ/dtheta = lam^T (dz/dtheta - (dA/dtheta) y),   A^T lam = ybar := dJ/dy.

Where the parameters enter Eq. 11 (the block matrix A_{n,S} and the vector z printed with it):
  * alpha (lambda in Eq. 4) only in the last block row, (alpha / h^omega) D_2^(S) B_n f;
  * mu (the data mu_eps) only in z, as its last block;
  * gamma2 in the diagonal blocks (eta / h^omega) D_2^(s) B_n v^(s) of rows s = 1..S and in the
    last row's (alpha / h^omega) D_2^(S) B_n f (D_2^(S) appears in both, so both contribute).
Hence, with lam = [lam^(1); ...; lam^(S); lam_f] and c_s = eta / h^omega, c_f = alpha / h^omega:

    dJ/dalpha            = -lam_f^T (h^-omega D_2^(S) B_n f)
    dJ/dmu               =  lam_f
    dJ/dgamma2_j^(s)     = -lam_j^(s) c_s (B_n v^(s))_j - [s = S] lam_{f,j} c_f (B_n f)_j

The transposed preconditioner: P^T is block upper triangular (P is A without its last block
column, Sec. 5.1), so P^T lam = r is solved by backward substitution, the f block first:
(c_f B_n D_2^(S)) lam_f = r_f, then for s = S..1
(e_0 D_1^(s) + c_s B_n D_2^(s)) lam^(s) = r^(s) - sum_{m > s} e_{m-s} D_1^(m) lam^(m) - [s = S] lam_f.

Parity: the gradients are pinned by central finite differences of J through forward solves
(tests/test_oracle_adjoint.py); the backward substitution by a dense solve with P^T.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import system as sy


def adjoint_solve_dense(p: sy.Problem, ybar: np.ndarray) -> np.ndarray:
    """lam = A^{-T} ybar by LU of the assembled A (dense mode)."""
    return sla.solve(sy.dense_A(p).T, ybar)


def precond_transpose_solve_dense(p: sy.Problem, r: np.ndarray) -> np.ndarray:
    """lam = P^{-T} r by backward substitution with LU block solves."""
    S, N = p.S, p.N
    R = r.reshape(S + 1, N)
    Lm = np.zeros((S + 1, N))
    B = sy.dense_B(p.a, p.ns)
    Lm[S] = sla.solve(p.c_f * B * p.gamma2[S - 1][None, :], R[S])
    e = p.e
    for s in range(S, 0, -1):
        rhs_s = R[s - 1].copy()
        for m in range(s + 1, S + 1):
            rhs_s -= e[m - s] * p.gamma1[m - 1] * Lm[m - 1]
        if s == S:
            rhs_s -= Lm[S]
        Lm[s - 1] = sla.solve(sy.diag_block_dense(p, s).T, rhs_s)
    return Lm.reshape(-1)


def gradients(p: sy.Problem, y: np.ndarray, lam: np.ndarray):
    """(dJ/dalpha, dJ/dmu [N], dJ/dgamma2 [S, N]) from the forward solution y and the adjoint
    solution lam, by the formulas in the module docstring."""
    S, N = p.S, p.N
    Y = y.reshape(S + 1, N)
    Lm = lam.reshape(S + 1, N)
    BY = sy.apply_B(p.a, p.ns, Y)
    dalpha = -float(np.dot(Lm[S], p.gamma2[S - 1] * BY[S])) / p.h ** p.omega
    dmu = Lm[S].copy()
    dg2 = -p.c_s * Lm[:S] * BY[:S]
    dg2[S - 1] -= p.c_f * Lm[S] * BY[S]
    return dalpha, dmu, dg2


def misfit(p: sy.Problem, f_true: np.ndarray) -> float:
    """J = 1/2 ||f - f_true||^2 for the exact solution of Eq. 11 (dense LU)."""
    y = sla.solve(sy.dense_A(p), sy.rhs(p))
    f = y[-p.N:]
    return 0.5 * float(np.dot(f - f_true, f - f_true))


def misfit_gradients(p: sy.Problem, f_true: np.ndarray):
    """Gradients of J = 1/2 ||f - f_true||^2: forward solve, ybar = [0; f - f_true], adjoint
    solve, formulas.  Returns (J, dalpha, dmu, dgamma2, y, lam)."""
    y = sla.solve(sy.dense_A(p), sy.rhs(p))
    ybar = np.zeros(p.U)
    ybar[-p.N:] = y[-p.N:] - f_true
    lam = adjoint_solve_dense(p, ybar)
    da, dm, dg = gradients(p, y, lam)
    J = 0.5 * float(np.dot(ybar[-p.N:], ybar[-p.N:]))
    return J, da, dm, dg, y, lam


def with_params(p: sy.Problem, **changes) -> sy.Problem:
    """A copy of p with some parameters replaced (alpha, mu, gamma2, ...) and a fresh cache."""
    return dataclasses.replace(p, _cache={}, **changes)
