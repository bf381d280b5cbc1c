"""Scalar tables of the discretisation (oracle; test infrastructure only).

* b_m, e_m: weights of the L1 approximation of the Caputo derivative
  (Sec. 4, Eq. 5 and the definition of e_m just before Eq. 10).
* eta = dt^beta * Gamma(2 - beta) (Sec. 5, definition of eta).
* a_l: Fourier coefficients of the generating function g (Eq. 7, Eq. 8);
  in one dimension the closed Gamma-ratio form (Eq. 9) and the recursion of
  Lemma 1(b); in several dimensions a K-point trapezoid rule for Eq. 8
  (the paper only says "through the FFT"), which is the reading this project
  takes for d >= 2.

Every function is plain FP64 NumPy/SciPy.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def l1_b(beta: float, count: int) -> np.ndarray:
    """b_m = (m+1)^(1-beta) - m^(1-beta), m = 0..count-1 (Sec. 4, below Eq. 5)."""
    m = np.arange(count, dtype=np.float64)
    return (m + 1.0) ** (1.0 - beta) - m ** (1.0 - beta)


def l1_e(beta: float, count: int) -> np.ndarray:
    """e_0 = b_0 and e_m = b_m - b_{m-1} for m >= 1 (Sec. 4, before Eq. 10)."""
    b = l1_b(beta, count)
    e = np.empty_like(b)
    e[0] = b[0]
    e[1:] = b[1:] - b[:-1]
    return e


def eta(beta: float, dt: float) -> float:
    """eta = dt^beta * Gamma(2 - beta) (Sec. 5, first display)."""
    return dt ** beta * math.gamma(2.0 - beta)


def frac_a0(omega: float) -> float:
    """a_0 = Gamma(omega+1) / Gamma(omega/2+1)^2 (Lemma 1(a))."""
    return math.gamma(omega + 1.0) / math.gamma(omega / 2.0 + 1.0) ** 2


def frac_coeffs_1d_closed(omega: float, count: int) -> np.ndarray:
    """a_l, l = 0..count-1, from the Gamma-ratio form of Eq. 9.

    a_l = (-1)^l Gamma(omega+1) / (Gamma(omega/2 - l + 1) Gamma(omega/2 + l + 1)).
    The arguments omega/2 - l + 1 become negative (never integers, since
    omega is not an even integer), so the product is formed in log space with
    the sign of each Gamma value carried separately.
    """
    l = np.arange(count, dtype=np.float64)
    x1 = omega / 2.0 - l + 1.0
    x2 = omega / 2.0 + l + 1.0
    logmag = special.gammaln(omega + 1.0) - special.gammaln(x1) - special.gammaln(x2)
    sign = ((-1.0) ** l) * special.gammasgn(omega + 1.0) * special.gammasgn(x1) * special.gammasgn(x2)
    return sign * np.exp(logmag)


def frac_coeffs_1d_recursion(omega: float, count: int) -> np.ndarray:
    """a_l, l = 0..count-1, by the recursion of Lemma 1(b) started at Lemma 1(a)."""
    a = np.empty(count, dtype=np.float64)
    if count == 0:
        return a
    a[0] = frac_a0(omega)
    for l in range(count - 1):
        a[l + 1] = (1.0 - (omega + 1.0) / (omega / 2.0 + l + 1.0)) * a[l]
    return a


def generating_function(omega: float, thetas: list[np.ndarray]) -> np.ndarray:
    """g(theta) = [sum_i 4 sin^2(theta_i / 2)]^(omega/2) on a tensor grid (Eq. 7)."""
    grids = np.meshgrid(*thetas, indexing="ij")
    s = np.zeros(grids[0].shape, dtype=np.float64)
    for th in grids:
        s += 4.0 * np.sin(th / 2.0) ** 2
    return s ** (omega / 2.0)


def default_K(d: int, n: int) -> int:
    """Trapezoid-rule size K for the d >= 2 coefficient table.

    K = 8 * 2^ceil(log2(2n)) for d <= 2 and K = 2 * 2^ceil(log2(2n)) for d = 3
    (a reading of "through the FFT"; the aliasing error sum_{m != 0} a_{l+Km}
    decays like K^-(d+omega)).
    """
    base = 1 << int(math.ceil(math.log2(2 * n)))
    return (8 if d <= 2 else 2) * base


def frac_coeffs_dft(omega: float, ns: tuple[int, ...], K: int) -> np.ndarray:
    """a_l for 0 <= l_i < n_i by the K-point trapezoid rule applied to Eq. 8.

    a_l ~= K^-d sum_{k in [0,K)^d} g(2 pi k / K) exp(-i l . 2 pi k / K); the
    sum is taken with numpy's FFT (a library primitive) and its real part kept
    (g is real and even, so the exact sum is real).  By evenness of g in each
    theta_i the table is even in each l_i, so only l_i >= 0 is returned.
    Parity unpinned against paper values (no printed d >= 2 coefficients);
    pinned by invariants, by the d = 1 limit (-> Eq. 9) and by adaptive
    quadrature of Eq. 8 in tests.
    """
    d = len(ns)
    th = 2.0 * np.pi * np.arange(K, dtype=np.float64) / K
    g = generating_function(omega, [th] * d)
    full = np.fft.fftn(g).real / float(K) ** d
    return full[tuple(slice(0, n) for n in ns)].copy()


def frac_coeffs(omega: float, ns: tuple[int, ...], K: int | None = None) -> np.ndarray:
    """Coefficient table a_l, 0 <= l_i < n_i, for the d-level Toeplitz matrix B_n.

    d = 1: the Lemma 1(b) recursion (equal to Eq. 9); d >= 2: frac_coeffs_dft
    with K = default_K(d, max n_i) unless given.
    """
    if len(ns) == 1:
        return frac_coeffs_1d_recursion(omega, ns[0])
    if K is None:
        K = default_K(len(ns), max(ns))
    return frac_coeffs_dft(omega, ns, K)
