"""S_{n,S} of Remark 1 on the GPU (block_solver = 2): every diagonal block solved by one Fourier
solve with (dbar I + c s(B_n)), s(B_n) the Strang circulant and dbar the level mean of
e_0 gamma1/gamma2, the f block with s(B_n) exactly.  The length-n DFTs run as Bluestein chirp-z
transforms on the power-of-two FFTs, so odd, even and non-smooth n are all covered.

Against the oracle's FFT forward substitution (both sides are the same direct computation: the
bound is the transforms' rounding times the spread of the s(B_n) eigenvalues), its transpose and the forward solve against the assembled S_{n,S} with constant
coefficients, left-preconditioned GMRES(30) step counts against the oracle's GMRES with the same
preconditioner (+-1), the mixed-precision flexible solve, and a batched solve.
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
    "1d_n16_S6": lambda: config_small_1d(16, 6),       # even n, padded transform grid
    "1d_n3_S5": lambda: config_small_1d(3, 5),
    "2d_n15_S8": lambda: config_2d(0.3, 1.2, n=15, S=8),
    "2d_n20_S6": lambda: config_2d(0.5, 1.5, n=20, S=6),  # even n, padded
    "2d_n31_S12_b7": lambda: config_2d(0.7, 1.8, n=31, S=12),
    "3d_n7_S5": lambda: config_3d(n=7, S=5),
    "3d_n6_S4": lambda: config_3d(n=6, S=4),             # even n, padded
}


def _tolerance(p, eps):
    """Bound on the relative difference of two implementations of the same direct solve: each block
    (dbar I + c s(B_n))^-1 b is computed by transforms whose rounding, about 40 eps relative to ||b||
    (log2 L per FFT, four FFTs per chirp-z DFT pair and axis), is amplified by at most the spread
    kappa = lambda_max / lambda_min of the s(B_n) eigenvalues (the f block, dbar = 0, attains it).
    s(B_n) is far worse conditioned than tau(B_n) at large omega (3e3 against 2e2 at n = 31,
    omega = 1.8), so a fixed bound does not fit both."""
    lam = sy.strang_eigenvalues(p.a, p.ns)
    return max(1e-12 if eps < 1e-10 else 3e-5, 40.0 * eps * lam.max() / lam.min())


@pytest.mark.parametrize("case", list(CASES))
def test_strang_precond_parity(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    r = random_vector(p.U, 501)
    ref = sy.precond_strang_solve(p, r)
    for prec, tol in ((t.PREC_FP64, _tolerance(p, 1.1e-16)), (t.PREC_MIXED, _tolerance(p, 6e-8))):
        s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG, precision=prec))
        yd = _dev(np.zeros(p.U))
        assert s.precond_apply(_dev(r), yd) == 0
        y = _host(yd)
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        s.close()
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("case", ["1d_n16_S6", "2d_n15_S8", "2d_n20_S6"])
def test_strang_precond_and_transpose_constant_coefficients(t, case):
    w = CASES[case]()
    w = dataclasses.replace(w, gamma1=np.full_like(w.gamma1, 1.3), gamma2=np.full_like(w.gamma2, 0.8))
    p = sy.problem_from(w)
    r = random_vector(p.U, 502)
    Sm = sy.dense_P_strang(p)
    s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG))
    ld = _dev(np.zeros(p.U))
    assert s.precond_apply_transpose(_dev(r), ld) == 0
    lam = _host(ld)
    assert np.linalg.norm(Sm.T @ lam - r) <= 1e-11 * np.linalg.norm(r)
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), yd) == 0
    assert np.linalg.norm(Sm @ _host(yd) - r) <= 1e-11 * np.linalg.norm(r)
    s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8", "2d_n31_S12_b7"])
def test_strang_gmres_iterations_match_oracle(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    z = sy.rhs(p)
    ref = gmres(lambda v: sy.matvec(p, v), z, lambda v: sy.precond_strang_solve(p, v), side="left",
                restart=30, tol=1e-10, maxit=3000)
    assert ref.converged
    s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG))
    y = np.zeros(p.U)
    info = s.solve(y)
    s.close()
    assert info["converged"], info
    assert abs(info["iters"] - ref.iters) <= 1, (info["iters"], ref.iters)
    assert np.linalg.norm(y - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


def test_strang_mixed_flexible_solve_reaches_the_true_residual(t):
    w = CASES["2d_n20_S6"]()
    p = sy.problem_from(w)
    y_ref = np.linalg.solve(sy.dense_A(p), sy.rhs(p))
    s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG, precision=t.PREC_MIXED, side=t.SIDE_FLEXIBLE,
                                              tol=1e-11))
    y = np.zeros(p.U)
    info = s.solve(y)
    s.close()
    assert info["converged"] and info["relres_true"] <= 1e-10, info
    assert np.linalg.norm(y - y_ref) <= 1e-7 * np.linalg.norm(y_ref)


def test_strang_batched_solve_equals_single_solves(t):
    ws = [config_2d(0.3, 1.2, n=15, S=8), config_2d(0.7, 1.8, n=13, S=10)]  # same transform length 32
    singles = []
    for w in ws:
        s = t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG))
        y = np.zeros(s.U)
        info = s.solve(y)
        s.close()
        assert info["converged"], info
        singles.append((y, info["iters"]))
    solvers = [t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG)) for w in ws]
    ys = [np.zeros(s.U) for s in solvers]
    infos = t.tsfde_gmres_solve_batch([s.handle for s in solvers], ys)
    for s in solvers:
        s.close()
    for (y1, it1), y, info in zip(singles, ys, infos):
        assert info["converged"] and info["iters"] == it1, (info, it1)
        assert np.linalg.norm(y - y1) <= 1e-12 * np.linalg.norm(y1)


def test_switching_a_handle_to_strang_blocks_builds_the_tables(t):
    """A handle set up for P_{n,S} and switched to S_{n,S} by tsfde_set_opts (the Strang tables are
    built on first use) applies the same preconditioner as a handle set up for S_{n,S}, and switching
    back restores P_{n,S}."""
    w = CASES["2d_n20_S6"]()
    p = sy.problem_from(w)
    r = random_vector(p.U, 503)
    fresh = t.Solver(w, opts=t.tsfde_default_opts(block_solver=t.BLOCK_STRANG))
    y_fresh = _dev(np.zeros(p.U))
    assert fresh.precond_apply(_dev(r), y_fresh) == 0
    fresh.close()
    s = t.Solver(w)
    y0 = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), y0) == 0
    s.set_opts(t.tsfde_default_opts(block_solver=t.BLOCK_STRANG))
    y1 = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), y1) == 0
    s.set_opts(t.tsfde_default_opts())
    y2 = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), y2) == 0
    s.close()
    np.testing.assert_array_equal(_host(y1), _host(y_fresh))
    np.testing.assert_array_equal(_host(y2), _host(y0))
    ref = sy.precond_solve_dense(p, r)
    assert np.linalg.norm(_host(y0) - ref) <= 1e-8 * np.linalg.norm(ref)
