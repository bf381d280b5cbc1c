"""Pins of the oracle's scalar tables against closed forms, the Lemma and
independent quadrature (no GPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import coefficients as co


@pytest.mark.parametrize("beta", [0.1, 0.5, 0.9])
def test_l1_weights_closed_values(beta):
    b = co.l1_b(beta, 6)
    # b_0 = 1, b_m = (m+1)^(1-beta) - m^(1-beta) written out for m = 3
    assert b[0] == 1.0
    assert b[3] == pytest.approx(4 ** (1 - beta) - 3 ** (1 - beta), rel=1e-15)
    e = co.l1_e(beta, 6)
    assert e[0] == 1.0
    # e_m = (m+1)^(1-b) - 2 m^(1-b) + (m-1)^(1-b) for m >= 1 (Sec. 4)
    for m in range(1, 6):
        assert e[m] == pytest.approx((m + 1) ** (1 - beta) - 2 * m ** (1 - beta) + (m - 1) ** (1 - beta),
                                     rel=1e-12, abs=1e-15)
        assert e[m] < 0.0
    # b_m is positive and strictly decreasing, the e_m telescope to b_{S-1}
    assert np.all(b > 0) and np.all(np.diff(b) < 0)
    assert e.sum() == pytest.approx(b[-1], rel=1e-13)


@pytest.mark.parametrize("beta", [0.2, 0.5, 0.8])
def test_l1_formula_exact_for_linear_functions(beta):
    """The L1 formula (Eq. 5) interpolates v linearly on each step, so it is exact
    for v(t) = t, whose Caputo derivative is t^(1-beta) / Gamma(2-beta)."""
    S, T = 12, 1.7
    dt = T / S
    b = co.l1_b(beta, S)
    e = co.l1_e(beta, S)
    v = dt * np.arange(S + 1)
    for s in range(1, S + 1):
        # bracket of Eq. 5 in the e-form of Eq. 10
        br = e[0] * v[s] + sum(e[s - m] * v[m] for m in range(1, s)) - b[s - 1] * v[0]
        approx = dt ** (-beta) / math.gamma(2 - beta) * br
        exact = (s * dt) ** (1 - beta) / math.gamma(2 - beta)
        assert approx == pytest.approx(exact, rel=1e-12)


def test_eta_definition():
    assert co.eta(0.5, 0.25) == pytest.approx(0.5 * math.gamma(1.5), rel=1e-15)


@pytest.mark.parametrize("omega", [1.1, 1.37, 1.5, 1.9])
def test_fractional_coeffs_recursion_matches_closed_form(omega):
    """Lemma 1(b) recursion against the Gamma-ratio closed form of Eq. 9."""
    n = 400
    a_rec = co.frac_coeffs_1d_recursion(omega, n)
    a_cf = co.frac_coeffs_1d_closed(omega, n)
    np.testing.assert_allclose(a_rec, a_cf, rtol=1e-11, atol=0)


@pytest.mark.parametrize("omega", [1.1, 1.5, 1.9])
def test_fractional_coeffs_lemma_properties(omega):
    a = co.frac_coeffs_1d_recursion(omega, 20001)
    # (a) a_0 formula, a_0 > 0 and a_l < 0 for l != 0
    assert a[0] == pytest.approx(math.gamma(omega + 1) / math.gamma(omega / 2 + 1) ** 2, rel=1e-15)
    assert a[0] > 0 and np.all(a[1:] < 0)
    # (c) the symmetric sum tends to zero: the tail -2 sum_{l>=L} a_l decays like L^-omega
    partial = a[0] + 2 * np.cumsum(a[1:])
    for L in (100, 1000, 10000):
        assert 0 < partial[L - 1] < 2.0 * L ** (-omega)
    assert partial[10000] < partial[1000] < partial[100]


def test_fractional_coeffs_laplacian_limit():
    """omega -> 2 gives the standard second difference [2, -1, 0, ...]."""
    a = co.frac_coeffs_1d_closed(2.0 - 1e-10, 5)
    np.testing.assert_allclose(a, [2.0, -1.0, 0.0, 0.0, 0.0], atol=1e-9)


@pytest.mark.parametrize("omega", [1.2, 1.5, 1.8])
def test_fractional_coeffs_dft_route_converges_to_closed_form_1d(omega):
    """The K-point trapezoid reading (used for d >= 2) reduces in d = 1 to
    aliasing of Eq. 9: error ~ sum_{m != 0} |a_{l + K m}| = O(K^-(1+omega))."""
    n = 16
    exact = co.frac_coeffs_1d_closed(omega, n)
    errs = []
    for K in (64, 256, 1024):
        errs.append(np.max(np.abs(co.frac_coeffs_dft(omega, (n,), K) - exact)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 5.0 * 1024.0 ** (-(1 + omega))


def _quad_coeff_2d(omega, l1, l2):
    """Eq. 8 for d = 2 by adaptive quadrature over [0, pi]^2 (even integrand)."""
    def f(t2, t1):
        g = (4 * np.sin(t1 / 2) ** 2 + 4 * np.sin(t2 / 2) ** 2) ** (omega / 2)
        return g * np.cos(l1 * t1) * np.cos(l2 * t2)
    val, _ = integrate.dblquad(f, 0.0, np.pi, 0.0, np.pi, epsabs=1e-12, epsrel=1e-12)
    return val / np.pi ** 2


@pytest.mark.parametrize("omega", [1.2, 1.8])
def test_fractional_coeffs_2d_against_quadrature(omega):
    """The d = 2 table (K-point trapezoid) against adaptive quadrature of Eq. 8."""
    a = co.frac_coeffs_dft(omega, (6, 6), 2048)
    for (l1, l2) in [(0, 0), (1, 0), (1, 1), (3, 2), (0, 5)]:
        assert a[l1, l2] == pytest.approx(_quad_coeff_2d(omega, l1, l2), abs=2e-8)


@pytest.mark.parametrize("omega", [1.2, 1.5, 1.9])
def test_fractional_coeffs_2d_invariants(omega):
    a = co.frac_coeffs(omega, (24, 24))
    assert a[0, 0] > 0
    off = a.copy()
    off[0, 0] = -1.0
    assert np.all(off < 0)                      # all off-centre coefficients negative
    np.testing.assert_allclose(a, a.T, rtol=0, atol=1e-15)   # symmetric under axis swap
    # the symbol of the truncated stencil at theta = 0 is the (small, positive) tail
    tot = a[0, 0] + 2 * a[1:, 0].sum() + 2 * a[0, 1:].sum() + 4 * a[1:, 1:].sum()
    assert 0 < tot < 0.1


@pytest.mark.parametrize("omega", [1.2, 1.5, 1.8])
def test_fractional_laplacian_getoor_1d(omega):
    """(-Delta)^(omega/2) (1 - x^2)_+^(omega/2) = Gamma(omega+1) on (-1, 1)
    (Getoor's closed form, with the hypersingular normalisation c_omega of Eq. 2):
    the discrete operator of Eq. 6 at x = 0 converges to it as h -> 0."""
    errs = []
    for m in (64, 256):
        h = 1.0 / m
        l = np.arange(-m, m + 1)
        u = np.clip(1 - (l * h) ** 2, 0, None) ** (omega / 2)
        a = co.frac_coeffs_1d_recursion(omega, m + 1)
        val = (a[np.abs(l)] * u).sum() / h ** omega
        errs.append(abs(val / math.gamma(omega + 1) - 1))
    assert errs[1] < errs[0] < 1e-3


@pytest.mark.parametrize("omega", [1.2, 1.5, 1.8])
def test_fractional_laplacian_getoor_2d(omega):
    """d = 2: (-Delta)^(omega/2) (1 - |x|^2)_+^(omega/2) = 2^omega Gamma(1+omega/2)^2;
    pins the normalisation of the d >= 2 coefficient reading."""
    exact = 2 ** omega * math.gamma(1 + omega / 2) ** 2
    m = 64
    h = 1.0 / m
    a = co.frac_coeffs(omega, (m + 1, m + 1))          # default K = 2048 here
    l = np.arange(-m, m + 1)
    L1, L2 = np.meshgrid(l, l, indexing="ij")
    u = np.clip(1 - (L1 * h) ** 2 - (L2 * h) ** 2, 0, None) ** (omega / 2)
    val = (a[np.abs(L1), np.abs(L2)] * u).sum() / h ** omega
    assert abs(val / exact - 1) < 1e-4


@pytest.mark.parametrize("omega", [1.2, 1.8])
def test_fractional_coeffs_3d_invariants(omega):
    """d = 3 (trapezoid size K = 2 * 2^ceil(log2 2n), smaller than for d <= 2): a_0 > 0, every
    off-centre coefficient negative, symmetric under every permutation of the axes."""
    a = co.frac_coeffs(omega, (12, 12, 12))
    assert a[0, 0, 0] > 0
    off = a.copy()
    off[0, 0, 0] = -1.0
    assert np.all(off < 0)
    for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)):
        np.testing.assert_allclose(a, a.transpose(perm), rtol=0, atol=1e-15)


@pytest.mark.parametrize("omega", [1.2, 1.8])
def test_fractional_laplacian_getoor_3d(omega):
    """d = 3: (-Delta)^(omega/2) (1 - |x|^2)_+^(omega/2) = 2^omega Gamma(1+omega/2) Gamma((3+omega)/2) /
    Gamma(3/2) on the unit ball (Getoor; the d-dependence enters through Gamma((d+omega)/2) / Gamma(d/2)).
    The discrete operator at the centre, h = 1/16, matches it to 1e-3 with the default K, and to 5e-5
    with 4 K: what remains at the default is the trapezoid rule's aliasing error."""
    exact = 2 ** omega * math.gamma(1 + omega / 2) * math.gamma((3 + omega) / 2) / math.gamma(1.5)
    m = 16
    h = 1.0 / m
    l = np.arange(-m, m + 1)
    L1, L2, L3 = np.meshgrid(l, l, l, indexing="ij")
    u = np.clip(1 - (L1 * h) ** 2 - (L2 * h) ** 2 - (L3 * h) ** 2, 0, None) ** (omega / 2)
    K = co.default_K(3, m + 1)
    errs = []
    for k in (K, 4 * K):
        a = co.frac_coeffs(omega, (m + 1,) * 3, K=k)
        val = (a[np.abs(L1), np.abs(L2), np.abs(L3)] * u).sum() / h ** omega
        errs.append(abs(val / exact - 1))
    assert errs[0] < 1e-3 and errs[1] < 5e-5 and errs[1] < errs[0], errs
