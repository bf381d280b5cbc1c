"""T_{n,S} of Remark 1 on the GPU (block_solver = 1): every diagonal block solved by one
sine-transform solve with (dbar I + c tau(B_n)) (the level mean of e_0 gamma1/gamma2), the f
block with tau(B_n) exactly.

Against the oracle's structured tau forward substitution (1e-12 in FP64 mode: both sides are the
same direct computation), its transpose against the assembled T_{n,S} with constant coefficients,
and left-preconditioned GMRES(30) step counts against the oracle's GMRES with the same
preconditioner (+-1).
"""
import dataclasses

import numpy as np
import pytest

from oracle import system as sy
from oracle.gmres import gmres
from workloads import config_2d, config_3d, config_small_1d, random_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def t():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_02809_gb300 import build
    build.build()
    import paper_2507_02809_gb300 as pkg
    return pkg


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(x):
    import torch
    torch.cuda.synchronize()
    return x.cpu().numpy()


CASES = {
    "1d_n63_S64": lambda: config_small_1d(63, 64),
    "1d_n3_S5": lambda: config_small_1d(3, 5),
    "2d_n15_S8": lambda: config_2d(0.3, 1.2, n=15, S=8),
    "2d_n31_S12_b7": lambda: config_2d(0.7, 1.8, n=31, S=12),
    "3d_n7_S5": lambda: config_3d(n=7, S=5),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tau_precond_parity(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    r = random_vector(p.U, 401)
    ref = sy.precond_tau_solve(p, r)
    for prec, tol in ((t.PREC_FP64, 1e-12), (t.PREC_MIXED, 1e-5)):
        s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=1, precision=prec))
        yd = _dev(np.zeros(p.U))
        assert s.precond_apply(_dev(r), yd) == 0
        y = _host(yd)
        assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(ref), prec
        s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8"])
def test_tau_precond_transpose_constant_coefficients(t, case):
    w = CASES[case]()
    w = dataclasses.replace(w, gamma1=np.full_like(w.gamma1, 1.3), gamma2=np.full_like(w.gamma2, 0.8))
    p = sy.problem_from(w)
    r = random_vector(p.U, 402)
    T = sy.dense_P_tau(p)
    s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=1))
    ld = _dev(np.zeros(p.U))
    assert s.precond_apply_transpose(_dev(r), ld) == 0
    lam = _host(ld)
    assert np.linalg.norm(T.T @ lam - r) <= 1e-11 * np.linalg.norm(r)
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), yd) == 0
    assert np.linalg.norm(T @ _host(yd) - r) <= 1e-11 * np.linalg.norm(r)
    s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8", "2d_n31_S12_b7"])
def test_tau_gmres_iterations_match_oracle(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    z = sy.rhs(p)
    ref = gmres(lambda v: sy.matvec(p, v), z, lambda v: sy.precond_tau_solve(p, v), side="left",
                restart=30, tol=1e-10, maxit=3000)
    assert ref.converged
    s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=1))
    y = np.zeros(p.U)
    info = s.solve(y)
    s.close()
    assert info["converged"], info
    assert abs(info["iters"] - ref.iters) <= 1, (info["iters"], ref.iters)
    assert np.linalg.norm(y - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
