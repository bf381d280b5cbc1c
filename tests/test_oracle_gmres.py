"""The oracle GMRES against direct solves on generic systems."""
import numpy as np
import pytest

from oracle.gmres import gmres


def _system(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    return A, b


@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("restart", [None, 7])
def test_gmres_solves_generic_system(side, restart):
    A, b = _system(60, 1)
    D = np.diag(A).copy()
    res = gmres(lambda v: A @ v, b, lambda v: v / D, side=side, restart=restart, tol=1e-12, maxit=500)
    assert res.converged
    np.testing.assert_allclose(res.x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)


def test_gmres_terminates_in_n_steps():
    A, b = _system(25, 2)
    res = gmres(lambda v: A @ v, b, tol=1e-13)
    assert res.converged and res.iters <= 25


def test_gmres_exact_inverse_preconditioner_one_step():
    A, b = _system(30, 3)
    Ainv = np.linalg.inv(A)
    res = gmres(lambda v: A @ v, b, lambda v: Ainv @ v, side="left", tol=1e-10)
    assert res.iters == 1


def test_gmres_residual_history_monotone():
    A, b = _system(40, 4)
    res = gmres(lambda v: A @ v, b, tol=1e-12)
    h = np.array(res.history[1:])
    assert np.all(np.diff(h) <= 1e-14)
