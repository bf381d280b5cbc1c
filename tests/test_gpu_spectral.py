"""Spectral diagnostics on the GPU against the oracle's assembled matrices.

With as many steps as the dimension, the bidiagonalisation's singular values are those of A and
P^-1 A (dense SVD, 1e-8 relative) and the Arnoldi Ritz values their eigenvalues; Arnoldi on
P^-1 A stops within N + 1 steps (P^-1 A - I has rank at most N, Sec. 5.1); a few steps already
give sigma_max at larger sizes.
"""
import numpy as np
import pytest

from oracle import system as sy
from workloads import config_2d, config_small_1d, paper_1d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def t():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_02809_gb300 import build
    build.build()
    import paper_2507_02809_gb300 as pkg
    return pkg


def _dense_M(p, which):
    A = sy.dense_A(p)
    return A if which == 0 else np.linalg.solve(sy.dense_P(p), A)


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("case", ["1d_n7_S8", "2d_n3_S6"])
def test_full_bidiagonalisation_gives_the_singular_values(t, case, which):
    from paper_2507_02809_gb300.spectral import singular_values
    w = config_small_1d(7, 8) if case == "1d_n7_S8" else config_2d(0.5, 1.5, n=3, S=6, alpha=1e-3)
    p = sy.problem_from(w)
    ref = np.linalg.svd(_dense_M(p, which), compute_uv=False)
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13))
    sv = singular_values(s, which, p.U)
    s.close()
    assert sv[0] == pytest.approx(ref[0], rel=1e-8)
    assert sv[-1] == pytest.approx(ref[-1], rel=1e-6)
    np.testing.assert_allclose(sv[: len(ref)], ref, rtol=1e-6, atol=1e-8 * ref[0])


def test_arnoldi_ritz_values_are_the_eigenvalues(t):
    from paper_2507_02809_gb300.spectral import ritz_values
    w = config_small_1d(7, 8)
    p = sy.problem_from(w)
    ev = np.linalg.eigvals(_dense_M(p, 0))
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13))
    rv, steps = ritz_values(s, 0, p.U)
    s.close()
    assert steps == p.U
    for lam in ev:
        assert np.min(np.abs(rv - lam)) <= 1e-6 * np.abs(ev).max()


def test_arnoldi_on_preconditioned_operator_closes_after_N_plus_1_steps(t):
    """P^-1 A - I has rank at most N (Sec. 5.1): the Krylov space of P^-1 A has dimension at most
    N + 1, so the subdiagonal entry h_{N+1, N} of the Hessenberg matrix vanishes (up to the
    accuracy of the block solves), and the Ritz values of the first N + 1 steps are eigenvalues."""
    import paper_2507_02809_gb300.tsfde as tt
    w = config_small_1d(7, 8)
    p = sy.problem_from(w)
    ev = np.linalg.eigvals(_dense_M(p, 1))
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13))
    v0 = np.random.default_rng(0).standard_normal(p.U)
    H, steps = tt.tsfde_spectral_arnoldi(s.handle, 1, p.N + 2, v0)
    s.close()
    assert steps >= p.N + 1
    Hn = np.abs(H[: steps + 1, :steps]).max()
    assert abs(H[p.N + 1, p.N]) <= 1e-8 * Hn
    for lam in np.linalg.eigvals(H[: p.N + 1, : p.N + 1]):
        assert np.min(np.abs(ev - lam)) <= 1e-6 * np.abs(ev).max()


def test_sigma_min_by_inverse_iteration(t):
    from paper_2507_02809_gb300.spectral import sigma_min_inverse_iteration
    w = paper_1d(31, 16, 0.1, 1.9).with_mu(np.zeros(31))
    p = sy.problem_from(w)
    ref = np.linalg.svd(sy.dense_A(p), compute_uv=False)[-1]
    s = t.Solver(w, opts=t.tsfde_default_opts(tol=1e-12, inner_tol=1e-13))
    got = sigma_min_inverse_iteration(s, iters=60, rtol=1e-9)
    s.close()
    assert got == pytest.approx(ref, rel=1e-4)


def test_sigma_max_from_few_steps(t):
    from paper_2507_02809_gb300.spectral import singular_values
    w = paper_1d(63, 16, 0.5, 1.5)
    w = w.with_mu(np.zeros(63))
    p = sy.problem_from(w)
    ref = np.linalg.svd(sy.dense_A(p), compute_uv=False)
    s = t.Solver(w)
    sv = singular_values(s, 0, 40)
    s.close()
    assert sv[0] == pytest.approx(ref[0], rel=1e-8)


def _table1_large():
    import os
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_condnum_large.txt")
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x) for x in line.split()]
            rows.append(v)
    return rows


@pytest.mark.parametrize("row", [r for r in _table1_large() if r[0] == 256 and r[1] in (16, 64)])
def test_preconditioned_condition_numbers_of_table_1(t, row):
    """cond_2(P^-1 A) at the paper's n = 256 (lambda = 5e-3) from 80 bidiagonalisation steps against
    Table 1: within 1 % (the paper prints integers)."""
    from paper_2507_02809_gb300.spectral import condition_estimate
    n, S = row[0], row[1]
    for j, (b, o) in enumerate(((0.1, 1.9), (0.5, 1.5), (0.9, 1.1))):
        w = paper_1d(n, S, b, o).with_mu(np.zeros(n))
        s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-12))
        _, _, c = condition_estimate(s, 1, 80)
        s.close()
        assert c == pytest.approx(row[3 + 2 * j], rel=0.01), (b, o, c, row[3 + 2 * j])
