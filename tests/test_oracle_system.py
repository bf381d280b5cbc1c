"""Pins of the oracle's operators: structured vs assembled forms, the rank
argument of Sec. 5.1, the time-convergence order, and the spectrum of B_n."""
import math

import numpy as np
import pytest

from oracle import system as sy
from workloads import config_small_1d, config_2d, paper_1d, random_vector


def _small_2d(beta=0.3, omega=1.2, n=7, S=6):
    return sy.problem_from(config_2d(beta, omega, n=n, S=S))


@pytest.mark.parametrize("ns", [(9,), (5, 6), (3, 4, 5)])
def test_B_structure_and_fft_apply(ns):
    from oracle import coefficients as co
    omega = 1.37
    if len(ns) == 1:
        a = co.frac_coeffs(omega, ns)
    else:
        a = co.frac_coeffs_dft(omega, ns, 64)
    B = sy.dense_B(a, ns)
    assert np.array_equal(B, B.T)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, B.shape[0]))
    np.testing.assert_allclose(sy.apply_B(a, ns, X), X @ B.T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d,omega", [(1, 1.2), (1, 1.9), (2, 1.5)])
def test_B_spectrum_inside_symbol_range(d, omega):
    """B_n is generated by g with 0 = min g < max g = (4 d)^(omega/2): its
    eigenvalues lie strictly inside (0, (4d)^(omega/2)) (SPD, Sec. 5)."""
    from oracle import coefficients as co
    ns = (12,) * d
    B = sy.dense_B(co.frac_coeffs(omega, ns), ns)
    ev = np.linalg.eigvalsh(B)
    assert ev[0] > 0
    assert ev[-1] < (4 * d) ** (omega / 2)


@pytest.mark.parametrize("prob", ["1d", "2d"])
def test_matvec_structured_equals_assembled(prob):
    p = sy.problem_from(config_small_1d(n=9, S=7)) if prob == "1d" else _small_2d()
    A = sy.dense_A(p)
    y = random_vector(p.U, 11)
    np.testing.assert_allclose(sy.matvec(p, y), A @ y, rtol=0, atol=1e-12 * np.abs(A).max() * 10)
    w = random_vector(p.U, 12)
    np.testing.assert_allclose(sy.matvec_transpose(p, w), A.T @ w, rtol=0, atol=1e-12 * np.abs(A).max() * 10)


def test_matvec_block_rows_written_out():
    """Spot-check single entries of z = A y against Eq. 11 written per node."""
    p = sy.problem_from(config_small_1d(n=6, S=5))
    y = random_vector(p.U, 5)
    Y = y.reshape(p.S + 1, p.N)
    z = sy.matvec(p, y).reshape(p.S + 1, p.N)
    a = p.a
    for (s, j) in [(1, 0), (3, 2), (5, 5)]:
        tsum = sum(p.e[s - m] * Y[m - 1, j] for m in range(1, s + 1))
        lap = sum(a[abs(j - k)] * Y[s - 1, k] for k in range(p.N))
        ref = p.gamma1[s - 1, j] * tsum + p.eta / p.h ** p.omega * p.gamma2[s - 1, j] * lap \
            - p.eta * p.q[s - 1] * Y[p.S, j]
        assert z[s - 1, j] == pytest.approx(ref, rel=1e-12)
    j = 3
    lapf = sum(a[abs(j - k)] * Y[p.S, k] for k in range(p.N))
    assert z[p.S, j] == pytest.approx(Y[p.S - 1, j] + p.alpha / p.h ** p.omega * p.gamma2[p.S - 1, j] * lapf,
                                      rel=1e-12)


def test_rhs_definition():
    w = config_small_1d(n=5, S=4)
    w.rho[:] = np.linspace(0.1, 0.5, 5)
    p = sy.problem_from(w)
    z = sy.rhs(p).reshape(p.S + 1, p.N)
    for s in range(1, p.S + 1):
        np.testing.assert_allclose(z[s - 1], p.b[s - 1] * p.gamma1[s - 1] * p.rho)
    np.testing.assert_array_equal(z[p.S], p.mu)


@pytest.mark.parametrize("prob", ["1d", "2d"])
def test_preconditioner_forward_substitution(prob):
    p = sy.problem_from(config_small_1d(n=9, S=7)) if prob == "1d" else _small_2d()
    P = sy.dense_P(p)
    r = random_vector(p.U, 21)
    y_dense = sy.precond_solve_dense(p, r)
    np.testing.assert_allclose(P @ y_dense, r, rtol=0, atol=1e-10 * np.abs(r).max())
    y_struct = sy.precond_solve_structured(p, r, tol=1e-14)
    np.testing.assert_allclose(y_struct, y_dense, rtol=0, atol=1e-10 * np.abs(y_dense).max())


@pytest.mark.parametrize("prob", ["1d", "2d"])
def test_low_rank_correction(prob):
    """A = P + R with rank(R) <= N, so P^-1 A - I has rank <= N (Sec. 5.1)."""
    p = sy.problem_from(config_small_1d(n=6, S=5)) if prob == "1d" else _small_2d(n=4, S=4)
    A = sy.dense_A(p)
    P = sy.dense_P(p)
    M = np.linalg.solve(P, A) - np.eye(p.U)
    sv = np.linalg.svd(M, compute_uv=False)
    rank = int((sv > 1e-10 * sv[0]).sum())
    assert rank <= p.N
    # the non-zero columns are exactly the f block
    assert np.abs(M[:, : p.S * p.N]).max() < 1e-12


def test_direct_problem_time_order():
    """Manufactured u = t^2 phi(x) with the discrete spatial operator in the
    source: the remaining error is the L1 truncation, of order 2 - beta
    (the estimate cited after Eq. 5)."""
    beta = 0.5
    n = 15
    errs = []
    for S in (16, 32, 64):
        w = config_small_1d(n=n, S=S)
        p = sy.problem_from(w)
        p.beta = beta
        x = np.arange(1, n + 1) / (n + 1)
        phi = x ** 2 * (1 - x) ** 2
        t = np.arange(1, S + 1) / S
        Bphi = sy.apply_B(p.a, p.ns, phi[None, :])[0] / p.h ** p.omega
        F = p.gamma1 * (2 * t[:, None] ** (2 - beta) / math.gamma(3 - beta)) * phi[None, :] \
            + p.gamma2 * (t[:, None] ** 2) * Bphi[None, :]
        v = sy.direct_solve(p, F=F).reshape(S, n)
        errs.append(np.max(np.abs(v[-1] - phi)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for r in rates:
        assert abs(r - (2 - beta)) < 0.06


def test_direct_problem_is_leading_block_of_P():
    w = paper_1d(8, 6, 0.5, 1.5)
    p = sy.problem_from(w.with_mu(np.zeros(8)))
    v = sy.direct_solve(p, w.f_true)
    P = sy.dense_P(p)
    Ahat = P[: p.S * p.N, : p.S * p.N]
    np.testing.assert_allclose(Ahat @ v, sy.direct_rhs(p, w.f_true), rtol=0, atol=1e-12)


@pytest.mark.parametrize("prob", ["1d", "2d"])
def test_entry_formulas_match_assembled(prob):
    p = sy.problem_from(config_small_1d(n=9, S=7)) if prob == "1d" else _small_2d()
    A = sy.dense_A(p)
    P = sy.dense_P(p)
    y = random_vector(p.U, 31)
    ents = [(0, 0), (2, 3), (p.S - 1, p.N - 1), (p.S, 1), (p.S, p.N - 2)]
    rows = [s * p.N + j for (s, j) in ents]
    np.testing.assert_allclose(sy.matvec_entries(p, y, ents), (A @ y)[rows], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sy.precond_entries(p, y, ents), (P @ y)[rows], rtol=1e-12, atol=1e-12)


def _constant_coefficient(p):
    """The same problem with gamma1, gamma2 frozen to constants (Remark 1's constant case)."""
    import dataclasses
    return dataclasses.replace(p, gamma1=np.full_like(p.gamma1, 1.3), gamma2=np.full_like(p.gamma2, 0.8), _cache={})


@pytest.mark.parametrize("prob", ["1d", "2d"])
def test_tau_preconditioner_is_T_of_remark_1_for_constant_coefficients(prob):
    """With constant gamma's the structured tau forward substitution solves T_{n,S} y = r, where
    T_{n,S} is P_{n,S} with every B_n replaced by tau(B_n) (Remark 1), assembled densely."""
    from workloads import config_2d, config_small_1d, random_vector
    w = config_small_1d(15, 6) if prob == "1d" else config_2d(0.5, 1.5, n=7, S=4)
    p = _constant_coefficient(sy.problem_from(w))
    r = random_vector(p.U, 41)
    y = sy.precond_tau_solve(p, r)
    T = sy.dense_P_tau(p)
    np.testing.assert_allclose(T @ y, r, rtol=0, atol=1e-11 * np.abs(r).max())


def test_tau_matrix_is_symmetric_and_close_to_B():
    """The DST route to tau(B_n) (tau_eigenvalues and the sine transform) against the closed form
    of the natural tau matrix: tau(B_n) = B_n - H_n with the Hankel matrix
    H_n[i, j] = a_{i+j+2} + a_{2n-i-j} (0-based, terms with index >= n dropped)."""
    from workloads import config_small_1d
    p = sy.problem_from(config_small_1d(31, 4))
    Tm = sy.dense_tau(p)
    B = sy.dense_B(p.a, p.ns)
    np.testing.assert_allclose(Tm, Tm.T, atol=1e-13)
    n = p.N
    a = p.a
    H = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            k = i + j + 2
            if k < n:
                H[i, j] = a[k]
            k2 = 2 * n - i - j
            if k2 < n:
                H[i, j] += a[k2]
    np.testing.assert_allclose(Tm, B - H, atol=1e-12)
