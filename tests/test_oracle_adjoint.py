"""Pins of the oracle's adjoint (oracle/adjoint.py).

The gradients of J = 1/2 ||f - f_true||^2 are compared with central finite differences of J
computed by forward dense solves only (no adjoint involved); the transposed preconditioner
with a dense solve against P^T; the adjoint solution with the defining identity A^T lam = ybar.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import system as sy
from workloads import config_2d, config_small_1d, random_vector


def _cases():
    return {
        "1d_n7_S6": lambda: sy.problem_from(config_small_1d(7, 6)),
        "2d_n3_S4": lambda: sy.problem_from(config_2d(0.5, 1.5, n=3, S=4, alpha=1e-3)),
        "2d_n7_S3_b3": lambda: sy.problem_from(config_2d(0.3, 1.2, n=7, S=3, alpha=1e-2)),
    }


def _f_true(p):
    rng = np.random.default_rng(11)
    return rng.standard_normal(p.N)


def _complex_step(p, ft, h, **changes):
    """Im J_c(theta + i h v) / h for the holomorphic misfit J_c = 1/2 sum (f - f_true)^2: the
    directional derivative without the cancellation of a finite difference."""
    q = adj.with_params(p, **changes)
    import scipy.linalg as sla
    y = sla.solve(sy.dense_A(q, np.complex128), sy.rhs(q, np.complex128))
    r = y[-p.N:] - ft
    return float((0.5 * np.sum(r * r)).imag / h)


@pytest.mark.parametrize("case", list(_cases()))
def test_precond_transpose_backward_substitution(case):
    p = _cases()[case]()
    r = random_vector(p.U, 31)
    lam = adj.precond_transpose_solve_dense(p, r)
    P = sy.dense_P(p)
    np.testing.assert_allclose(P.T @ lam, r, rtol=0, atol=1e-10 * np.abs(r).max())
    np.testing.assert_allclose(lam, np.linalg.solve(P.T, r), rtol=1e-9, atol=1e-12 * np.abs(lam).max())


@pytest.mark.parametrize("case", list(_cases()))
def test_adjoint_solve_identity(case):
    p = _cases()[case]()
    ybar = random_vector(p.U, 32)
    lam = adj.adjoint_solve_dense(p, ybar)
    np.testing.assert_allclose(sy.matvec_transpose(p, lam), ybar, rtol=0, atol=1e-9 * np.abs(ybar).max())


@pytest.mark.parametrize("case", list(_cases()))
def test_gradient_alpha_against_central_difference(case):
    p = _cases()[case]()
    ft = _f_true(p)
    J, da, _, _, _, _ = adj.misfit_gradients(p, ft)
    h = 1e-4 * p.alpha
    Jp = adj.misfit(adj.with_params(p, alpha=p.alpha + h), ft)
    Jm = adj.misfit(adj.with_params(p, alpha=p.alpha - h), ft)
    fd = (Jp - Jm) / (2 * h)
    assert da == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("case", list(_cases()))
def test_gradient_mu_against_central_difference_and_complex_step(case):
    p = _cases()[case]()
    ft = _f_true(p)
    J, _, dm, _, _, _ = adj.misfit_gradients(p, ft)
    rng = np.random.default_rng(5)
    scale = np.abs(p.mu).max() + 1.0
    # single components and one random direction
    dirs = [np.eye(p.N)[j] for j in (0, p.N // 2, p.N - 1)] + [rng.standard_normal(p.N)]
    for v in dirs:
        got = float(dm @ v)
        cs = _complex_step(p, ft, 1e-30, mu=p.mu + 1e-30j * v)
        assert got == pytest.approx(cs, rel=1e-9, abs=1e-13 * (abs(J) + 1))
        h = 1e-5 * scale
        Jp = adj.misfit(adj.with_params(p, mu=p.mu + h * v), ft)
        Jm = adj.misfit(adj.with_params(p, mu=p.mu - h * v), ft)
        fd = (Jp - Jm) / (2 * h)
        # central difference: O(h^2) truncation plus eps J / h cancellation
        assert got == pytest.approx(fd, rel=1e-6, abs=100 * 2.2e-16 * J / h)


@pytest.mark.parametrize("case", list(_cases()))
def test_gradient_gamma2_against_central_difference_and_complex_step(case):
    p = _cases()[case]()
    ft = _f_true(p)
    J, _, _, dg, _, _ = adj.misfit_gradients(p, ft)
    S, N = p.S, p.N
    rng = np.random.default_rng(6)
    dirs = []
    for (s, j) in [(0, 0), (S - 1, N - 1), (S - 1, N // 2), (S // 2, N // 3)]:
        v = np.zeros((S, N))
        v[s, j] = 1.0
        dirs.append(v)
    dirs.append(rng.standard_normal((S, N)))
    for v in dirs:
        got = float((dg * v).sum())
        cs = _complex_step(p, ft, 1e-30, gamma2=p.gamma2 + 1e-30j * v)
        assert got == pytest.approx(cs, rel=1e-9, abs=1e-13 * (abs(J) + 1))
        h = 1e-6
        Jp = adj.misfit(adj.with_params(p, gamma2=p.gamma2 + h * v), ft)
        Jm = adj.misfit(adj.with_params(p, gamma2=p.gamma2 - h * v), ft)
        fd = (Jp - Jm) / (2 * h)
        assert got == pytest.approx(fd, rel=1e-5, abs=100 * 2.2e-16 * J / h)


@pytest.mark.parametrize("case", list(_cases()))
def test_gradient_alpha_complex_step(case):
    p = _cases()[case]()
    ft = _f_true(p)
    J, da, _, _, _, _ = adj.misfit_gradients(p, ft)
    cs = _complex_step(p, ft, 1e-30 * p.alpha, alpha=p.alpha + 1e-30j * p.alpha)
    assert da == pytest.approx(cs, rel=1e-9)


def test_last_level_gets_both_gamma2_terms():
    """D_2^(S) multiplies B_n v^(S) in row S and B_n f in the last row: the gradient at level S
    is the sum of both terms (dropping either fails the finite-difference check above)."""
    p = _cases()["1d_n7_S6"]()
    ft = _f_true(p)
    _, _, _, dg, y, lam = adj.misfit_gradients(p, ft)
    S, N = p.S, p.N
    Y, Lm = y.reshape(S + 1, N), lam.reshape(S + 1, N)
    BY = sy.apply_B(p.a, p.ns, Y)
    only_row_s = -p.c_s * Lm[S - 1] * BY[S - 1]
    assert not np.allclose(dg[S - 1], only_row_s)
