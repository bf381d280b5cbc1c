"""GMRES for the all-at-once system (oracle; test infrastructure only).

The paper calls MATLAB's built-in ``gmres`` with a custom matvec and the
preconditioner P (Sec. 5 "Implementation", Sec. 6.1.2): zero initial guess,
``tol`` on the relative residual, maxit = min(size, 1000).  With a
preconditioner that routine works on the left-preconditioned system
P^-1 A y = P^-1 z and stops when ||P^-1 (z - A y)|| <= tol ||P^-1 z||.  This
oracle implements GMRES with Householder-reflector Arnoldi (Walker's
formulation, which is what that routine uses) and Givens rotations for the
small least-squares problem; it also provides right preconditioning.
Iteration counts are the number of Arnoldi steps summed over restart cycles.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int            # Arnoldi steps in total
    converged: bool
    relres_est: float     # last residual estimate / reference norm
    history: list


def _givens(a: float, b: float):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(apply_A, b, apply_Minv=None, side: str = "left", restart: int | None = None,
          tol: float = 1e-8, maxit: int | None = None, x0=None) -> GmresResult:
    """Solve A x = b.  ``side`` is 'left' (P^-1 A x = P^-1 b, preconditioned
    residual test) or 'right' (A P^-1 u = b, x = P^-1 u, true residual test).
    ``restart`` None means unrestarted; ``maxit`` counts Arnoldi steps."""
    n = b.shape[0]
    if maxit is None:
        maxit = min(n, 1000)
    M = apply_Minv if apply_Minv is not None else (lambda v: v)
    if side == "left":
        op = lambda v: M(apply_A(v))
        resid = lambda x: M(b - apply_A(x))
        bnorm = np.linalg.norm(M(b))
    elif side == "right":
        op = lambda v: apply_A(M(v))
        resid = lambda x: b - apply_A(x)
        bnorm = np.linalg.norm(b)
    else:
        raise ValueError(side)
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    if bnorm == 0.0:
        return GmresResult(np.zeros(n), 0, True, 0.0, [])
    m = maxit if restart is None else restart
    total = 0
    history = []
    r = resid(x)
    while True:
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= tol * bnorm:
            return GmresResult(x, total, True, beta / bnorm, history)
        if total >= maxit:
            return GmresResult(x, total, False, beta / bnorm, history)
        steps = min(m, maxit - total, n)
        # Householder Arnoldi: reflectors U[:, j] act on components j..n-1
        U = np.zeros((n, steps + 1))
        R = np.zeros((steps + 1, steps))
        cs = np.zeros(steps)
        sn = np.zeros(steps)
        g = np.zeros(steps + 1)

        def make_reflector(w, j):
            """Reflector on w[j:] mapping it to (alpha, 0, ...)."""
            u = np.zeros(n)
            tail = w[j:]
            nrm = np.linalg.norm(tail)
            alpha = -nrm if tail[0] >= 0 else nrm
            u[j:] = tail
            u[j] -= alpha
            un = np.linalg.norm(u)
            if un > 0:
                u /= un
            return u, alpha

        def apply_refl(u, v):
            return v - 2.0 * u * (u @ v)

        U[:, 0], alpha = make_reflector(r, 0)
        g[0] = alpha
        k_done = 0
        converged = False
        for j in range(steps):
            # v_j = P_0 P_1 ... P_j e_j
            v = np.zeros(n)
            v[j] = 1.0
            for i in range(j, -1, -1):
                v = apply_refl(U[:, i], v)
            w = op(v)
            for i in range(0, j + 1):
                w = apply_refl(U[:, i], w)
            if j + 1 < n:
                U[:, j + 1], alpha = make_reflector(w, j + 1)
                w = apply_refl(U[:, j + 1], w)
                w[j + 1] = alpha
                w[j + 2:] = 0.0
            h = w[: j + 2].copy()
            for i in range(j):
                t = cs[i] * h[i] + sn[i] * h[i + 1]
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1]
                h[i] = t
            cs[j], sn[j] = _givens(h[j], h[j + 1])
            h[j] = cs[j] * h[j] + sn[j] * h[j + 1]
            h[j + 1] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            R[: j + 1, j] = h[: j + 1]
            k_done = j + 1
            total += 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm:
                converged = True
                break
        # x update: x += sum_i y_i v_i = P_0 (y_0 e_0 + P_1 (y_1 e_1 + ...))
        yk = np.linalg.solve(np.triu(R[:k_done, :k_done]), g[:k_done])
        z = np.zeros(n)
        for i in range(k_done - 1, -1, -1):
            z[i] += yk[i]
            z = apply_refl(U[:, i], z)
        x = x + (M(z) if side == "right" else z)
        r = resid(x)
        if converged:
            rel = np.linalg.norm(r) / bnorm
            if rel <= tol:
                return GmresResult(x, total, True, rel, history)
            # estimate and recomputed residual disagree: keep iterating
        if total >= maxit:
            return GmresResult(x, total, False, np.linalg.norm(r) / bnorm, history)
