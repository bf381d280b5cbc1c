"""The recovered source f(alpha, mu, gamma2) of Eq. 11 as a differentiable PyTorch function.

forward: a handle is set up with the given alpha, data mu and field gamma2 (gamma1, q, rho, the
grid, beta and omega are fixed), A y = z is solved by preconditioned GMRES on the GPU and f, the
last block of y, is returned.  backward: for the upstream gradient g = dJ/df, tsfde_adjoint
solves A^T lam = [0; g] (preconditioned with P^T) and forms dJ/dalpha, dJ/dmu and dJ/dgamma2
from lam and the forward solution.  Everything runs in libtsfde; torch supplies device memory
and the stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import tsfde as _t


@dataclass
class FixedInputs:
    """The inputs of one instance that are not differentiated."""

    d: int
    n: int
    S: int
    beta: float
    omega: float
    gamma1: torch.Tensor          # [S, N] float64 (host or CUDA)
    q: torch.Tensor               # [S]
    rho: torch.Tensor             # [N]
    length: float = 1.0
    T: float = 1.0
    opts: _t.TsfdeOpts | None = None

    @property
    def N(self) -> int:
        return self.n ** self.d


class _Handle:
    def __init__(self, h: int):
        self.h = h

    def close(self):
        if self.h:
            _t.tsfde_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _flat(x: torch.Tensor) -> torch.Tensor:
    return x.detach().to(torch.float64).contiguous().reshape(-1)


class InverseSourceSolve(torch.autograd.Function):
    """f = InverseSourceSolve.apply(alpha, mu, gamma2, fixed); alpha a 0-dim tensor, mu [N],
    gamma2 [S, N] (CUDA float64)."""

    @staticmethod
    def forward(ctx, alpha, mu, gamma2, fixed: FixedInputs):
        dev = mu.device
        S, N = fixed.S, fixed.N
        stream = int(torch.cuda.current_stream(dev).cuda_stream)
        h = _t.tsfde_setup(fixed.d, fixed.n, fixed.length, S, fixed.T, fixed.beta, fixed.omega, float(alpha),
                           _flat(fixed.gamma1), _flat(gamma2), _flat(fixed.q), _flat(fixed.rho), _flat(mu),
                           opts=fixed.opts, stream=stream)
        handle = _Handle(h)
        y = torch.zeros((S + 1) * N, dtype=torch.float64, device=dev)
        info = _t.tsfde_gmres_solve(h, y)
        ctx.handle = handle
        ctx.y = y
        ctx.shapes = (alpha.shape, mu.shape, gamma2.shape)
        ctx.info = info
        return y[S * N:].clone()

    @staticmethod
    def backward(ctx, grad_f):
        y = ctx.y
        N = grad_f.numel()
        S = y.numel() // N - 1
        ybar = torch.zeros_like(y)
        ybar[S * N:] = grad_f.to(torch.float64).reshape(-1)
        dmu = torch.empty(N, dtype=torch.float64, device=y.device)
        dg2 = torch.empty(S * N, dtype=torch.float64, device=y.device)
        out = _t.tsfde_adjoint(ctx.handle.h, y, ybar, None, dmu, dg2)
        ctx.handle.close()
        a_shape, m_shape, g_shape = ctx.shapes
        dalpha = torch.full(a_shape, out["dalpha"], dtype=torch.float64, device=y.device)
        return dalpha, dmu.reshape(m_shape), dg2.reshape(g_shape), None


def recover_source(alpha: torch.Tensor, mu: torch.Tensor, gamma2: torch.Tensor, fixed: FixedInputs) -> torch.Tensor:
    """f of Eq. 11 for the given alpha, data and gamma2 (differentiable in all three)."""
    return InverseSourceSolve.apply(alpha, mu, gamma2, fixed)
