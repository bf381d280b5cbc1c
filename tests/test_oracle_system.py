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


# ---- the Strang circulant s(B_n) and S_{n,S} (Remark 1) -------------------------------------

@pytest.mark.parametrize("ns", [(15,), (16,), (5, 5), (6, 6), (4, 4, 4)])
def test_strang_matrix_is_the_circulant_keeping_the_central_diagonals(ns):
    """s(B_n) is fixed by two properties: it is a (multilevel) circulant, and it agrees with B_n on
    every entry whose level offsets all satisfy |i_k - j_k| <= floor(n_k / 2).  Checked entry by
    entry on the assembled matrix, for odd and even n."""
    from workloads import config_2d, config_3d, config_small_1d
    n = ns[0]
    w = {1: lambda: config_small_1d(n, 3), 2: lambda: config_2d(0.5, 1.5, n=n, S=3),
         3: lambda: config_3d(n=n, S=3)}[len(ns)]()
    p = sy.problem_from(w)
    C = sy.dense_strang(p)
    B = sy.dense_B(p.a, p.ns)
    d = len(ns)
    idx = np.indices(ns).reshape(d, -1)
    off = [idx[k][:, None] - idx[k][None, :] for k in range(d)]
    band = np.ones(C.shape, dtype=bool)
    for k in range(d):
        band &= np.abs(off[k]) <= ns[k] // 2
    np.testing.assert_array_equal(C[band], B[band])
    # circulant: the entry depends only on the offsets modulo n, level by level
    key = sum(((off[k] % ns[k]) * int(np.prod(ns[k + 1:]))) for k in range(d))
    for v in np.unique(key):
        vals = C[key == v]
        assert np.all(vals == vals[0])
    np.testing.assert_array_equal(C, C.T)


@pytest.mark.parametrize("ns", [(15,), (16,), (5, 5), (6, 6)])
def test_strang_eigenvalues_match_brute_force_and_are_positive(ns):
    """The DFT route to the eigenvalues of s(B_n) against eigvalsh of the assembled matrix; all are
    at least lambda_0 = sum of the first column > 0 (the off-diagonal a_l are negative)."""
    from workloads import config_2d, config_small_1d
    n = ns[0]
    w = config_small_1d(n, 3) if len(ns) == 1 else config_2d(0.7, 1.8, n=n, S=3)
    p = sy.problem_from(w)
    lam = sy.strang_eigenvalues(p.a, p.ns)
    ev = np.linalg.eigvalsh(sy.dense_strang(p))
    np.testing.assert_allclose(np.sort(lam), ev, rtol=0, atol=1e-13 * ev.max())
    lam0 = sy.strang_column(p.a, p.ns).sum()
    assert lam0 > 0
    assert lam.min() >= lam0 * (1 - 1e-12)
    np.testing.assert_allclose(lam[0], lam0, rtol=1e-13)


@pytest.mark.parametrize("n", [15, 16, 64])
def test_strang_eigenvalues_are_the_truncated_symbol(n):
    """d = 1: lambda_k is the Fourier series of g (Eq. 7) truncated to the central diagonals, so
    |lambda_k - g(2 pi k / n)| is at most the sum of the dropped |a_l|, which equals lambda_0
    because the a_l sum to g(0) = 0 and are negative off the diagonal."""
    from workloads import config_small_1d
    p = sy.problem_from(config_small_1d(n, 3))
    lam = sy.strang_eigenvalues(p.a, p.ns)
    th = 2 * np.pi * np.arange(n) / n
    g = np.abs(2 * np.sin(th / 2)) ** p.omega
    assert np.abs(lam - g).max() <= lam[0] * (1 + 1e-10)
    # and lambda_0 -> 0 like n^-omega (tail of a_l ~ l^(-1-omega))
    p2 = sy.problem_from(config_small_1d(2 * n, 3))
    ratio = sy.strang_eigenvalues(p2.a, p2.ns)[0] / lam[0]
    assert abs(np.log2(ratio) + p.omega) < 0.25, ratio


@pytest.mark.parametrize("prob", ["1d_even", "1d_odd", "2d"])
def test_strang_preconditioner_is_S_of_remark_1_for_constant_coefficients(prob):
    """With constant gamma's the FFT forward substitution solves S_{n,S} y = r, where S_{n,S} is
    P_{n,S} with every B_n replaced by s(B_n) (Remark 1), assembled densely."""
    from workloads import config_2d, config_small_1d, random_vector
    w = {"1d_even": lambda: config_small_1d(16, 6), "1d_odd": lambda: config_small_1d(15, 5),
         "2d": lambda: config_2d(0.5, 1.5, n=6, S=4)}[prob]()
    p = _constant_coefficient(sy.problem_from(w))
    r = random_vector(p.U, 43)
    y = sy.precond_strang_solve(p, r)
    P = sy.dense_P_strang(p)
    np.testing.assert_allclose(P @ y, r, rtol=0, atol=1e-11 * np.abs(r).max())


@pytest.mark.parametrize("case", ["1d_n63_S64", "1d_n31_S16", "2d_n15_S8", "2d_n31_S12"])
def test_remark_1_tau_needs_no_more_gmres_steps_than_strang(case):
    """Remark 1 expects T_{n,S} to outperform S_{n,S} because tau(B_n) follows the small
    eigenvalues of B_n more closely than the circulant does: left-preconditioned GMRES(30) to 1e-10
    takes no more steps with the tau blocks than with the Strang blocks on these problems."""
    from oracle.gmres import gmres
    from workloads import config_2d, config_small_1d
    w = {"1d_n63_S64": lambda: config_small_1d(63, 64), "1d_n31_S16": lambda: config_small_1d(31, 16),
         "2d_n15_S8": lambda: config_2d(0.3, 1.2, n=15, S=8),
         "2d_n31_S12": lambda: config_2d(0.7, 1.8, n=31, S=12)}[case]()
    p = sy.problem_from(w)
    z = sy.rhs(p)
    runs = {}
    for name, pc in (("tau", sy.precond_tau_solve), ("strang", sy.precond_strang_solve)):
        res = gmres(lambda v: sy.matvec(p, v), z, lambda v, pc=pc: pc(p, v), side="left", restart=30,
                    tol=1e-10, maxit=3000)
        assert res.converged, name
        runs[name] = res.iters
    assert runs["tau"] <= runs["strang"], runs
