"""The all-at-once system A y = z and the block triangular preconditioner P
(oracle; test infrastructure only).

Notation follows Sec. 4-5: S time levels, N = n_1 ... n_d interior nodes in
lexicographic order with the last index fastest, y = [v^(1); ...; v^(S); f],
D_1^(s) = diag(gamma1 at t_s), D_2^(s) = diag(gamma2 at t_s), eta and the
fractional coefficients a_l from ``coefficients``.  The regularisation
parameter, written lambda in Eq. 4, is called ``alpha`` here.

Dense mode (assembled matrices, SciPy LU) is meant for U = (S+1) N up to a few
thousand; the structured functions apply the same operators without assembly.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla

from . import coefficients as coef


@dataclass
class Problem:
    """One instance of the discretised regularised problem (Eq. 10)."""

    ns: tuple[int, ...]          # interior points per dimension
    S: int                       # number of time steps
    T: float                     # final time
    beta: float
    omega: float
    alpha: float                 # regularisation parameter (lambda in Eq. 4)
    gamma1: np.ndarray           # [S, N]  gamma1(x_j, t_s), s = 1..S
    gamma2: np.ndarray           # [S, N]
    q: np.ndarray                # [S]     q(t_s)
    rho: np.ndarray              # [N]
    mu: np.ndarray               # [N]     noisy final data mu_eps
    length: float = 1.0          # side of the hypercube Omega = (lo, lo+length)^d
    K: int | None = None         # trapezoid size for d >= 2 coefficients
    _cache: dict = field(default_factory=dict, repr=False)

    # --- derived quantities ------------------------------------------------
    @property
    def d(self) -> int:
        return len(self.ns)

    @property
    def N(self) -> int:
        return int(np.prod(self.ns))

    @property
    def U(self) -> int:
        return (self.S + 1) * self.N

    @property
    def h(self) -> float:
        """Unique mesh size h = (b - a) / (n + 1): n interior points (Sec. 4)."""
        n0 = self.ns[0]
        assert all(n == n0 for n in self.ns), "a unique step size h needs equal n_i on a cube"
        return self.length / (n0 + 1)

    @property
    def dt(self) -> float:
        return self.T / self.S

    @property
    def eta(self) -> float:
        return coef.eta(self.beta, self.dt)

    @property
    def b(self) -> np.ndarray:
        return coef.l1_b(self.beta, self.S)

    @property
    def e(self) -> np.ndarray:
        return coef.l1_e(self.beta, self.S)

    @property
    def c_s(self) -> float:
        """eta / h^omega, the factor of D_2^(s) B_n in block row s (Sec. 5)."""
        return self.eta / self.h ** self.omega

    @property
    def c_f(self) -> float:
        """alpha / h^omega, the factor of D_2^(S) B_n in the last block row (Sec. 5)."""
        return self.alpha / self.h ** self.omega

    @property
    def a(self) -> np.ndarray:
        if "a" not in self._cache:
            self._cache["a"] = coef.frac_coeffs(self.omega, self.ns, self.K)
        return self._cache["a"]


# ---------------------------------------------------------------------------
# B_n: the d-level symmetric Toeplitz matrix generated by g (Sec. 5, after Eq. 10)
# ---------------------------------------------------------------------------

def dense_B(a: np.ndarray, ns: tuple[int, ...]) -> np.ndarray:
    """Assemble B_n with entries a_{|i - j|} (per level) for multi-indices i, j."""
    d = len(ns)
    idx = np.indices(ns).reshape(d, -1)
    diff = np.abs(idx[:, :, None] - idx[:, None, :])
    return a[tuple(diff[k] for k in range(d))]


def apply_B(a: np.ndarray, ns: tuple[int, ...], x: np.ndarray) -> np.ndarray:
    """B_n x for x of shape [..., N] by circulant embedding and the FFT (Sec. 5,
    matvec step 1(b)): each level n_i is embedded in a circulant of size 2 n_i
    whose first column is [a_0, ..., a_{n-1}, 0, a_{n-1}, ..., a_1]."""
    d = len(ns)
    lead = x.shape[:-1]
    L = tuple(2 * n for n in ns)
    col = np.zeros(L, dtype=np.float64)
    # place a_l at +l and -l (mod L) in every axis
    for signs in np.ndindex(*(2,) * d):
        sl_src = []
        sl_dst = []
        for k in range(d):
            n = ns[k]
            if signs[k] == 0:
                sl_src.append(slice(0, n))
                sl_dst.append(slice(0, n))
            else:
                sl_src.append(slice(1, n))
                sl_dst.append(slice(L[k] - 1, L[k] - n, -1))
        col[tuple(sl_dst)] = a[tuple(sl_src)]
    lam = np.fft.rfftn(col).real
    xs = x.reshape(lead + tuple(ns))
    axes = tuple(range(len(lead), len(lead) + d))
    X = np.fft.rfftn(xs, s=L, axes=axes)
    Y = np.fft.irfftn(X * lam, s=L, axes=axes)
    Y = Y[(Ellipsis,) + tuple(slice(0, n) for n in ns)]
    return Y.reshape(lead + (int(np.prod(ns)),))


# ---------------------------------------------------------------------------
# The coefficient matrix A_{n,S} (Eq. 11), the right-hand side z and P_{n,S}
# ---------------------------------------------------------------------------

def dense_A(p: Problem, dtype=np.float64) -> np.ndarray:
    """Assemble A_{n,S} of Eq. 11, size (S+1) N.  dtype=complex128 admits complex alpha and
    gamma's (complex-step derivatives in the tests)."""
    N, S = p.N, p.S
    B = dense_B(p.a, p.ns)
    e = p.e
    A = np.zeros((p.U, p.U), dtype=dtype)
    for s in range(1, S + 1):
        r = slice((s - 1) * N, s * N)
        D1 = p.gamma1[s - 1]
        D2 = p.gamma2[s - 1]
        for m in range(1, s):
            A[r, (m - 1) * N:m * N] = np.diag(e[s - m] * D1)
        A[r, (s - 1) * N:s * N] = np.diag(e[0] * D1) + p.c_s * D2[:, None] * B
        A[r, S * N:] = -p.eta * p.q[s - 1] * np.eye(N)
    r = slice(S * N, (S + 1) * N)
    A[r, (S - 1) * N:S * N] = np.eye(N)
    A[r, S * N:] = p.c_f * p.gamma2[S - 1][:, None] * B
    return A


def dense_P(p: Problem) -> np.ndarray:
    """Assemble P_{n,S} (Sec. 5.1): A_{n,S} with its upper-right column blocks
    -eta q^(s) I replaced by zero blocks."""
    P = dense_A(p)
    P[: p.S * p.N, p.S * p.N:] = 0.0
    return P


def rhs(p: Problem, dtype=np.float64) -> np.ndarray:
    """z = [b_0 D_1^(1) rho; ...; b_{S-1} D_1^(S) rho; mu_eps] (Eq. 11)."""
    b = p.b
    z = np.empty(p.U, dtype=dtype)
    for s in range(1, p.S + 1):
        z[(s - 1) * p.N:s * p.N] = b[s - 1] * p.gamma1[s - 1] * p.rho
    z[p.S * p.N:] = p.mu
    return z


def time_sum(e: np.ndarray, V: np.ndarray) -> np.ndarray:
    """W[s] = sum_{m=1}^{s} e_{s-m} V[m] for s = 1..S (rows of V are levels).

    This is the lower-triangular Toeplitz-in-time part of block rows 1..S of
    Eq. 11 (matvec step 1(a) of Sec. 5), written as the plain double loop."""
    S = V.shape[0]
    W = np.zeros_like(V)
    for s in range(S):
        for m in range(s + 1):
            W[s] += e[s - m] * V[m]
    return W


def matvec(p: Problem, y: np.ndarray) -> np.ndarray:
    """z = A_{n,S} y without assembly, following the steps of Sec. 5
    ("Implementation"): time sums, B_n by circulant embedding + FFT, the
    diagonal scalings and the -eta q^(s) f coupling, then the last block row
    y^(S) + (alpha/h^omega) D_2^(S) B_n f.  (Step 1(c) prints y^(s); the block
    matrix of Eq. 11 puts the f block y^(S+1) there, which is what is used.)"""
    S, N = p.S, p.N
    Y = y.reshape(S + 1, N)
    V, f = Y[:S], Y[S]
    W = time_sum(p.e, V)
    BY = apply_B(p.a, p.ns, Y)
    z = np.empty((S + 1, N))
    z[:S] = p.gamma1 * W + p.c_s * p.gamma2 * BY[:S] - p.eta * p.q[:, None] * f[None, :]
    z[S] = V[S - 1] + p.c_f * p.gamma2[S - 1] * BY[S]
    return z.reshape(-1)


def matvec_transpose(p: Problem, w: np.ndarray) -> np.ndarray:
    """A_{n,S}^T w without assembly (B_n is symmetric, D's are diagonal)."""
    S, N = p.S, p.N
    Wt = w.reshape(S + 1, N)
    out = np.zeros((S + 1, N))
    g1w = p.gamma1 * Wt[:S]
    # transpose of the lower-triangular time Toeplitz: sum over s >= m
    for m in range(S):
        for s in range(m, S):
            out[m] += p.e[s - m] * g1w[s]
    out[:S] += p.c_s * apply_B(p.a, p.ns, p.gamma2 * Wt[:S])
    out[S - 1] += Wt[S]
    out[S] = -p.eta * (p.q[:, None] * Wt[:S]).sum(axis=0)
    out[S] += p.c_f * apply_B(p.a, p.ns, (p.gamma2[S - 1] * Wt[S])[None, :])[0]
    return out.reshape(-1)


# ---------------------------------------------------------------------------
# Forward substitution for P_{n,S} y = r (Sec. 5.1, "Implementation")
# ---------------------------------------------------------------------------

def diag_block_dense(p: Problem, s: int) -> np.ndarray:
    """e_0 D_1^(s) + (eta/h^omega) D_2^(s) B_n, 1 <= s <= S (Sec. 5.1, step 1(a)/2(a))."""
    B = p._cache.get("B")
    if B is None:
        B = p._cache["B"] = dense_B(p.a, p.ns)
    return np.diag(p.e[0] * p.gamma1[s - 1]) + p.c_s * p.gamma2[s - 1][:, None] * B


def precond_solve_dense(p: Problem, r: np.ndarray, first_levels_only: bool = False) -> np.ndarray:
    """y = P^{-1} r by the forward substitution of Sec. 5.1 with LU block
    solves (the paper's backslash).  With ``first_levels_only`` only the S
    time levels are computed: that is the direct problem of Sec. 6.1
    (matrix \\hat A), whose right-hand side is r[:S]."""
    S, N = p.S, p.N
    R = r.reshape(-1, N)
    Y = np.zeros((S + 1, N))
    lus = p._cache.setdefault("lu", {})
    e = p.e
    for s in range(1, S + 1):
        rhs_s = R[s - 1].copy()
        hist = np.zeros(N)
        for m in range(1, s):
            hist += e[s - m] * Y[m - 1]
        rhs_s -= p.gamma1[s - 1] * hist
        if s not in lus:
            lus[s] = sla.lu_factor(diag_block_dense(p, s))
        Y[s - 1] = sla.lu_solve(lus[s], rhs_s)
    if first_levels_only:
        return Y[:S].reshape(-1)
    if "luf" not in lus:
        B = p._cache["B"]
        lus["luf"] = sla.lu_factor(p.c_f * p.gamma2[S - 1][:, None] * B)
    Y[S] = sla.lu_solve(lus["luf"], R[S] - Y[S - 1])
    return Y.reshape(-1)


def tau_eigenvalues(a: np.ndarray, ns: tuple[int, ...]) -> np.ndarray:
    """Eigenvalues of the natural tau approximation tau(B_n) (Bini-Di Benedetto,
    cited in Remark 1): the truncated symbol sum_{|l_i|<n_i} a_l prod cos(l_i th_k)
    at th_k = pi k/(n_i+1), k = 1..n_i; tau(B_n) = S diag(mu) S with S the
    orthonormal DST-I matrix."""
    d = len(ns)
    out = a.copy()
    for ax in range(d):
        n = ns[ax]
        k = np.arange(1, n + 1)
        l = np.arange(n)
        C = np.cos(np.outer(k, l) * np.pi / (n + 1))
        C[:, 1:] *= 2.0
        out = np.moveaxis(np.tensordot(C, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out.reshape(-1)


def _dst_apply(x: np.ndarray, ns: tuple[int, ...]) -> np.ndarray:
    """Orthonormal multi-d DST-I (an involution) of x [..., N]."""
    lead = x.shape[:-1]
    xs = x.reshape(lead + tuple(ns))
    axes = tuple(range(len(lead), len(lead) + len(ns)))
    return sfft.dstn(xs, type=1, axes=axes, norm="ortho").reshape(x.shape)


def pcg(apply_K, apply_M, rhs_v, x0, tol, maxit):
    """Preconditioned conjugate gradients (textbook form) for SPD K; stops when
    ||r|| <= tol ||rhs||.  Returns (x, iterations)."""
    x = x0.copy()
    r = rhs_v - apply_K(x)
    nb = np.linalg.norm(rhs_v)
    if nb == 0.0:
        return np.zeros_like(rhs_v), 0
    z = apply_M(r)
    pdir = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > tol * nb and it < maxit:
        Kp = apply_K(pdir)
        alpha = rz / (pdir @ Kp)
        x += alpha * pdir
        r -= alpha * Kp
        z = apply_M(r)
        rz_new = r @ z
        pdir = z + (rz_new / rz) * pdir
        rz = rz_new
        it += 1
    return x, it


def precond_solve_structured(p: Problem, r: np.ndarray, tol: float = 1e-14, maxit: int = 500,
                             first_levels_only: bool = False, stats: dict | None = None,
                             max_levels: int | None = None) -> np.ndarray:
    """y = P^{-1} r by the forward substitution of Sec. 5.1 without assembly.

    The diagonal-block systems (e_0 D_1^(s) + c_s D_2^(s) B_n) y = rhat are
    solved iteratively instead of by backslash: multiplied by D_2^(s)^-1 they
    become SPD (B_n is SPD since g >= 0), and are solved by CG preconditioned
    with mean(e_0 gamma1/gamma2) I + c_s tau(B_n) (tau from Remark 1), to a
    relative residual ``tol``.  The f block (alpha/h^omega) D_2^(S) B_n f = r_f - y^(S)
    is solved as B_n f = D_2^(S)^-1 (r_f - y^(S)) / c_f with tau(B_n) as preconditioner.
    ``max_levels`` stops the substitution after that many levels (the rest of y stays zero):
    a bounded piece of the same work, for timing samples.
    """
    S, N = p.S, p.N
    R = r.reshape(-1, N)
    Y = np.zeros((S + 1, N))
    e = p.e
    mu = tau_eigenvalues(p.a, p.ns)
    cs = p.c_s
    iters = []
    last = S if max_levels is None else min(S, max_levels)
    for s in range(1, last + 1):
        hist = np.zeros(N)
        for m in range(1, s):
            hist += e[s - m] * Y[m - 1]
        rhat = R[s - 1] - p.gamma1[s - 1] * hist
        dvec = e[0] * p.gamma1[s - 1] / p.gamma2[s - 1]
        dbar = dvec.mean()

        def apply_K(x, dvec=dvec):
            return dvec * x + cs * apply_B(p.a, p.ns, x[None, :])[0]

        def apply_M(x, dbar=dbar):
            return _dst_apply(_dst_apply(x, p.ns) / (dbar + cs * mu), p.ns)

        x0 = Y[s - 2] if s > 1 else np.zeros(N)
        Y[s - 1], it = pcg(apply_K, apply_M, rhat / p.gamma2[s - 1], x0, tol, maxit)
        iters.append(it)
    if max_levels is not None and last < S:
        return Y.reshape(-1)
    if not first_levels_only:
        g = (R[S] - Y[S - 1]) / (p.c_f * p.gamma2[S - 1])

        def apply_Bf(x):
            return apply_B(p.a, p.ns, x[None, :])[0]

        def apply_Mf(x):
            return _dst_apply(_dst_apply(x, p.ns) / mu, p.ns)

        Y[S], it = pcg(apply_Bf, apply_Mf, g, np.zeros(N), tol, maxit)
        iters.append(it)
    if stats is not None:
        stats["inner_iters"] = iters
    if first_levels_only:
        return Y[:S].reshape(-1)
    return Y.reshape(-1)


# ---------------------------------------------------------------------------
# Direct problem (Sec. 6.1): \hat A v = \hat z with the source f known
# ---------------------------------------------------------------------------

def dense_tau(p: Problem) -> np.ndarray:
    """tau(B_n) = S diag(mu) S assembled (S the orthonormal multi-d DST-I matrix)."""
    N = p.N
    Sm = _dst_apply(np.eye(N), p.ns)
    return Sm @ np.diag(tau_eigenvalues(p.a, p.ns)) @ Sm


def _dense_P_replacing(p: Problem, M: np.ndarray) -> np.ndarray:
    """P_{n,S} assembled with every B_n replaced by the N x N matrix M (Remark 1)."""
    N, S = p.N, p.S
    P = np.zeros((p.U, p.U))
    e = p.e
    for s in range(1, S + 1):
        r = slice((s - 1) * N, s * N)
        for m in range(1, s):
            P[r, (m - 1) * N:m * N] = np.diag(e[s - m] * p.gamma1[s - 1])
        P[r, (s - 1) * N:s * N] = np.diag(e[0] * p.gamma1[s - 1]) + p.c_s * p.gamma2[s - 1][:, None] * M
    r = slice(S * N, (S + 1) * N)
    P[r, (S - 1) * N:S * N] = np.eye(N)
    P[r, S * N:] = p.c_f * p.gamma2[S - 1][:, None] * M
    return P


def dense_P_tau(p: Problem) -> np.ndarray:
    """T_{n,S} of Remark 1: P_{n,S} with every B_n replaced by tau(B_n)."""
    return _dense_P_replacing(p, dense_tau(p))


def _substitution_mean_blocks(p: Problem, r: np.ndarray, block_inverse) -> np.ndarray:
    """Forward substitution of Sec. 5.1 in which every diagonal block e_0 D_1^(s) + c_s D_2^(s) B_n
    is replaced by D_2^(s) (dbar_s I + c_s M), dbar_s the level mean of e_0 gamma1/gamma2, and the
    f block c_f D_2^(S) B_n by c_f D_2^(S) M; block_inverse(b, dbar, c) = (dbar I + c M)^-1 b."""
    S, N = p.S, p.N
    R = r.reshape(-1, N)
    Y = np.zeros((S + 1, N))
    e = p.e
    for s in range(1, S + 1):
        hist = np.zeros(N)
        for m in range(1, s):
            hist += e[s - m] * Y[m - 1]
        b = (R[s - 1] - p.gamma1[s - 1] * hist) / p.gamma2[s - 1]
        dbar = float(np.mean(e[0] * p.gamma1[s - 1] / p.gamma2[s - 1]))
        Y[s - 1] = block_inverse(b, dbar, p.c_s)
    b = (R[S] - Y[S - 1]) / (p.c_f * p.gamma2[S - 1])
    Y[S] = block_inverse(b, 0.0, 1.0)
    return Y.reshape(-1)


def precond_tau_solve(p: Problem, r: np.ndarray) -> np.ndarray:
    """y = T~^{-1} r: the forward substitution of Sec. 5.1 in which every diagonal block
    e_0 D_1^(s) + c_s D_2^(s) B_n is replaced by D_2^(s) (dbar_s I + c_s tau(B_n)), dbar_s the
    level mean of e_0 gamma1/gamma2, so that each block is one DST-diagonal solve; the f block
    c_f D_2^(S) tau(B_n) is inverted exactly.  With constant coefficients this is T_{n,S} of
    Remark 1 (B_n -> tau(B_n) in P_{n,S}); with variable ones the paper notes that the tau
    structure is lost, and the level mean is this implementation's approximation."""
    mu = tau_eigenvalues(p.a, p.ns)
    return _substitution_mean_blocks(
        p, r, lambda b, dbar, c: _dst_apply(_dst_apply(b, p.ns) / (dbar + c * mu), p.ns))


# ---------------------------------------------------------------------------
# The Strang circulant s(B_n) and S_{n,S} (Remark 1)
# ---------------------------------------------------------------------------

def strang_column(a: np.ndarray, ns: tuple[int, ...]) -> np.ndarray:
    """First column of the d-level Strang circulant s(B_n), shape ns: in every level the central
    diagonals of B_n are kept and wrapped around, c_l = a_l for 0 <= l <= floor(n/2) and
    c_l = a_{n-l} for floor(n/2) < l < n (R. Chan's definition; for even n the middle entry is
    a_{n/2})."""
    src = []
    for n in ns:
        l = np.arange(n)
        src.append(np.where(l <= n // 2, l, n - l))
    return a[np.ix_(*src)]


def strang_eigenvalues(a: np.ndarray, ns: tuple[int, ...]) -> np.ndarray:
    """Eigenvalues of s(B_n) in DFT order (k_1, ..., k_d), flattened: the d-dimensional DFT of the
    first column, real because the column is even in every level."""
    return np.fft.fftn(strang_column(a, ns)).real.reshape(-1)


def dense_strang(p: Problem) -> np.ndarray:
    """s(B_n) assembled entry by entry: entry (i, j) is c_{(i - j) mod n} level by level."""
    d = p.d
    col = strang_column(p.a, p.ns)
    idx = np.indices(p.ns).reshape(d, -1)
    diff = [(idx[k][:, None] - idx[k][None, :]) % p.ns[k] for k in range(d)]
    return col[tuple(diff)]


def dense_P_strang(p: Problem) -> np.ndarray:
    """S_{n,S} of Remark 1: P_{n,S} with every B_n replaced by s(B_n)."""
    return _dense_P_replacing(p, dense_strang(p))


def precond_strang_solve(p: Problem, r: np.ndarray) -> np.ndarray:
    """y = S~^{-1} r: as precond_tau_solve with s(B_n) in place of tau(B_n), each block solved in
    the Fourier basis that diagonalises the circulant: (dbar I + c s(B_n))^-1 b =
    IDFT(DFT(b) / (dbar + c lambda_k)).  S_{n,S} of Remark 1 for constant coefficients."""
    lam = strang_eigenvalues(p.a, p.ns).reshape(p.ns)

    def inv(b, dbar, c):
        B = np.fft.fftn(b.reshape(p.ns))
        return np.fft.ifftn(B / (dbar + c * lam)).real.reshape(-1)

    return _substitution_mean_blocks(p, r, inv)


def direct_rhs(p: Problem, f: np.ndarray | None = None, F: np.ndarray | None = None) -> np.ndarray:
    """\\hat z^(s) = b_{s-1} D_1^(s) rho + eta q^(s) f, s = 1..S (Sec. 6.1).

    With ``F`` ([S, N]) the separable source f(x) q(t) is replaced by a general
    source F(x_j, t_s): \\hat z^(s) = b_{s-1} D_1^(s) rho + eta F^(s)."""
    b = p.b
    src = p.q[:, None] * f[None, :] if F is None else F
    return (b[:, None] * p.gamma1 * p.rho[None, :] + p.eta * src).reshape(-1)


def direct_solve(p: Problem, f: np.ndarray | None = None, dense: bool | None = None,
                 F: np.ndarray | None = None) -> np.ndarray:
    """v^(1..S) of the direct problem: \\hat A is the leading S x S block part
    of P_{n,S}, so the first S stages of the forward substitution solve it."""
    if dense is None:
        dense = p.N <= 1500
    zh = direct_rhs(p, f, F)
    if dense:
        return precond_solve_dense(p, zh, first_levels_only=True)
    return precond_solve_structured(p, zh, first_levels_only=True)


def problem_from(w, K: int | None = None) -> Problem:
    """Build a Problem from a workload object exposing ``problem_kwargs()``."""
    kw = w.problem_kwargs()
    return Problem(K=K, **kw)


# ---------------------------------------------------------------------------
# Single entries, for sampled checks at sizes too large for the full oracle
# ---------------------------------------------------------------------------

def _B_row_dot(p: Problem, j: int, x: np.ndarray) -> float:
    """(B_n x)_j = sum_k a_{|j - k|} x_k with per-level index differences."""
    idx_j = np.unravel_index(j, p.ns)
    grids = np.indices(p.ns).reshape(p.d, -1)
    diff = tuple(np.abs(grids[k] - idx_j[k]) for k in range(p.d))
    return float(p.a[diff] @ x)


def matvec_entries(p: Problem, y: np.ndarray, entries) -> np.ndarray:
    """(A y)[s, j] for (s, j) in ``entries`` (s = 0..S, 0-based block row; j node),
    written per node from block row s+1 of Eq. 11."""
    S, N = p.S, p.N
    Y = y.reshape(S + 1, N)
    out = []
    for (s, j) in entries:
        if s < S:
            tsum = sum(p.e[s - m] * Y[m, j] for m in range(s + 1))
            v = p.gamma1[s, j] * tsum + p.c_s * p.gamma2[s, j] * _B_row_dot(p, j, Y[s]) \
                - p.eta * p.q[s] * Y[S, j]
        else:
            v = Y[S - 1, j] + p.c_f * p.gamma2[S - 1, j] * _B_row_dot(p, j, Y[S])
        out.append(v)
    return np.array(out)


def precond_entries(p: Problem, y: np.ndarray, entries) -> np.ndarray:
    """(P y)[s, j] for (s, j) in ``entries``: A y without the -eta q^(s) f coupling."""
    S, N = p.S, p.N
    Y = y.reshape(S + 1, N)
    out = []
    for (s, j) in entries:
        if s < S:
            tsum = sum(p.e[s - m] * Y[m, j] for m in range(s + 1))
            v = p.gamma1[s, j] * tsum + p.c_s * p.gamma2[s, j] * _B_row_dot(p, j, Y[s])
        else:
            v = Y[S - 1, j] + p.c_f * p.gamma2[S - 1, j] * _B_row_dot(p, j, Y[S])
        out.append(v)
    return np.array(out)
