"""Workload definitions: grids, coefficient fields, data and seeded noise.

Grids follow Sec. 4: n interior points per direction on (lo, lo+length),
h = length / (n + 1), x_j = lo + j h for j = 1..n, multi-indices in
lexicographic order with the last index fastest; time levels t_s = s T / S,
s = 1..S.  Arrays are float64: gamma1, gamma2 have shape [S, N], q [S],
rho and mu [N].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

CONFIG_SEED_BASE = 250702809


@dataclass
class Workload:
    name: str
    ns: tuple
    S: int
    T: float
    beta: float
    omega: float
    alpha: float
    gamma1: np.ndarray
    gamma2: np.ndarray
    q: np.ndarray
    rho: np.ndarray
    mu: np.ndarray | None
    length: float = 1.0
    lo: float = 0.0
    f_true: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return len(self.ns)

    @property
    def N(self) -> int:
        return int(np.prod(self.ns))

    @property
    def U(self) -> int:
        return (self.S + 1) * self.N

    def with_mu(self, mu: np.ndarray) -> "Workload":
        return replace(self, mu=np.ascontiguousarray(mu, dtype=np.float64))

    def problem_kwargs(self) -> dict:
        """Keyword arguments for a solver object taking the paper's inputs."""
        return dict(ns=tuple(self.ns), S=self.S, T=self.T, beta=self.beta, omega=self.omega,
                    alpha=self.alpha, gamma1=self.gamma1, gamma2=self.gamma2, q=self.q,
                    rho=self.rho, mu=self.mu, length=self.length)


def _axes(ns, lo, length):
    h = length / (ns[0] + 1)
    return [lo + h * np.arange(1, n + 1, dtype=np.float64) for n in ns]


def _mesh(ns, lo, length):
    """Node coordinates, each of shape [N] (lexicographic, last index fastest)."""
    ax = _axes(ns, lo, length)
    grids = np.meshgrid(*ax, indexing="ij")
    return [g.reshape(-1) for g in grids]


def _times(S, T):
    return T * np.arange(1, S + 1, dtype=np.float64) / S


def add_noise_gaussian(mu: np.ndarray, level: float, rng: np.random.Generator) -> np.ndarray:
    """mu + xi with xi Gaussian, rescaled so ||xi||_2 = level ||mu||_2 exactly (Eq. 3)."""
    xi = rng.standard_normal(mu.shape)
    nrm = np.linalg.norm(xi)
    if nrm == 0 or level == 0:
        return mu.copy()
    return mu + xi * (level * np.linalg.norm(mu) / nrm)


def add_noise_uniform(mu: np.ndarray, rel: float, rng: np.random.Generator) -> np.ndarray:
    """mu + eps delta with delta ~ U(-1, 1) per node and eps = rel ||mu||_2 (Sec. 6.1)."""
    delta = rng.uniform(-1.0, 1.0, size=mu.shape)
    return mu + rel * np.linalg.norm(mu) * delta


def random_vector(U: int, seed: int) -> np.ndarray:
    """Seeded standard normal vector of length U."""
    return np.random.default_rng(seed).standard_normal(U)


def _manufactured_mu(ns, lo, length, T):
    """mu = u(x, T) for u = t^2 prod_i x_i^2 (1 - x_i)^2."""
    X = _mesh(ns, lo, length)
    phi = np.ones_like(X[0])
    for x in X:
        phi = phi * x ** 2 * (1.0 - x) ** 2
    return T ** 2 * phi


def config_small_1d(n: int = 63, S: int = 64) -> Workload:
    """d = 1 on (0,1), T = 1, beta = 0.5, omega = 1.5, alpha = 1e-3;
    gamma1 = 1 + 0.5 sin(pi x) e^-t, gamma2 = 1 + 0.3 x (1-x)(1+t), q = 1 + t,
    rho = 0, mu = u(., 1) for u = t^2 x^2 (1-x)^2, no noise."""
    ns = (n,)
    T = 1.0
    (x,) = _mesh(ns, 0.0, 1.0)
    t = _times(S, T)[:, None]
    g1 = 1.0 + 0.5 * np.sin(np.pi * x)[None, :] * np.exp(-t)
    g2 = 1.0 + 0.3 * (x * (1.0 - x))[None, :] * (1.0 + t)
    q = 1.0 + t[:, 0]
    rho = np.zeros(n)
    mu = _manufactured_mu(ns, 0.0, 1.0, T)
    return Workload("small_1d_n%d_S%d" % (n, S), ns, S, T, 0.5, 1.5, 1e-3, g1, g2, q, rho, mu)


def config_2d(beta: float = 0.3, omega: float = 1.2, n: int = 255, S: int = 256,
              alpha: float = 1e-4, noise: float = 0.01, seed: int | None = None) -> Workload:
    """d = 2 on (0,1)^2, T = 1; gamma1 = 1 + 0.5 sin(pi x) sin(pi y) e^-t,
    gamma2 = 1 + 0.2 (x + y) t, q = e^-t + 1, rho = 0, mu = u(., 1) for
    u = t^2 x^2(1-x)^2 y^2(1-y)^2 plus seeded Gaussian noise of relative level
    ``noise``."""
    ns = (n, n)
    T = 1.0
    x, y = _mesh(ns, 0.0, 1.0)
    t = _times(S, T)[:, None]
    g1 = 1.0 + 0.5 * (np.sin(np.pi * x) * np.sin(np.pi * y))[None, :] * np.exp(-t)
    g2 = 1.0 + 0.2 * (x + y)[None, :] * t
    q = np.exp(-t[:, 0]) + 1.0
    rho = np.zeros(n * n)
    mu = _manufactured_mu(ns, 0.0, 1.0, T)
    rng = np.random.default_rng(CONFIG_SEED_BASE + 2 if seed is None else seed)
    mu = add_noise_gaussian(mu, noise, rng)
    return Workload("2d_n%d_S%d_b%g_w%g" % (n, S, beta, omega), ns, S, T, beta, omega, alpha,
                    g1, g2, q, rho, mu)


def config_3d(n: int = 63, S: int = 256, beta: float = 0.6, omega: float = 1.6,
              alpha: float = 1e-4, noise: float = 0.005, seed: int | None = None) -> Workload:
    """d = 3 on (0,1)^3, T = 1; gamma1 = 1 + 0.4 sin(pi x) sin(pi y) sin(pi z) e^-t,
    gamma2 = 0.75 + 0.25 xyz (1 + t), q = 1 + t, rho = 0, mu from
    u = t^2 prod x_i^2 (1-x_i)^2 plus seeded Gaussian noise."""
    ns = (n, n, n)
    T = 1.0
    x, y, z = _mesh(ns, 0.0, 1.0)
    t = _times(S, T)[:, None]
    g1 = 1.0 + 0.4 * (np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z))[None, :] * np.exp(-t)
    g2 = 0.75 + 0.25 * (x * y * z)[None, :] * (1.0 + t)
    q = 1.0 + t[:, 0]
    rho = np.zeros(n ** 3)
    mu = _manufactured_mu(ns, 0.0, 1.0, T)
    rng = np.random.default_rng(CONFIG_SEED_BASE + 3 if seed is None else seed)
    mu = add_noise_gaussian(mu, noise, rng)
    return Workload("3d_n%d_S%d" % (n, S), ns, S, T, beta, omega, alpha, g1, g2, q, rho, mu)


def config_adjoint_2d(n: int = 127, S: int = 128, beta: float = 0.5, omega: float = 1.5,
                      alpha: float = 1e-4, noise: float = 0.01, seed: int | None = None) -> Workload:
    """Gradient workload: d = 2 on (0,1)^2, T = 1, gamma1 and gamma2 as in config_2d, q = 1 + t,
    rho = 0, mu = u(., 1) for u = t^2 x^2(1-x)^2 y^2(1-y)^2 plus seeded Gaussian noise, and the
    target source f_true = sin(pi x) sin(pi y) of the misfit J = 1/2 ||f - f_true||^2."""
    ns = (n, n)
    T = 1.0
    x, y = _mesh(ns, 0.0, 1.0)
    t = _times(S, T)[:, None]
    g1 = 1.0 + 0.5 * (np.sin(np.pi * x) * np.sin(np.pi * y))[None, :] * np.exp(-t)
    g2 = 1.0 + 0.2 * (x + y)[None, :] * t
    q = 1.0 + t[:, 0]
    rho = np.zeros(n * n)
    mu = _manufactured_mu(ns, 0.0, 1.0, T)
    rng = np.random.default_rng(CONFIG_SEED_BASE + 5 if seed is None else seed)
    mu = add_noise_gaussian(mu, noise, rng)
    f_true = np.sin(np.pi * x) * np.sin(np.pi * y)
    return Workload("adj2d_n%d_S%d" % (n, S), ns, S, T, beta, omega, alpha, g1, g2, q, rho, mu,
                    f_true=f_true)


def config_batch(count_1d: int = 32, count_2d: int = 32, seed: int | None = None) -> list:
    """Batched workload: count_1d instances with d = 1, n ~ U{127..2047}, S ~ U{64..512}, and count_2d
    with d = 2, n x n, n ~ U{63..255}, S ~ U{64..256}; beta ~ U(0.2, 0.9), omega ~ U(1.1, 1.9),
    alpha ~ log-U(1e-5, 1e-2); gamma1 = 1 + a prod sin(pi x_i) e^-t, gamma2 = 1 + b prod x_i(1 - x_i)
    (1 + t) with a ~ U(0, 0.5), b ~ U(0, 0.3); q = 1 + t, rho = 0; mu the manufactured final state
    t^2 prod x_i^2 (1 - x_i)^2 at T = 1 plus 1 % Gaussian noise.  Seeded."""
    rng = np.random.default_rng(CONFIG_SEED_BASE + 4 if seed is None else seed)
    out = []
    for i in range(count_1d + count_2d):
        d = 1 if i < count_1d else 2
        n = int(rng.integers(127, 2048)) if d == 1 else int(rng.integers(63, 256))
        S = int(rng.integers(64, 513)) if d == 1 else int(rng.integers(64, 257))
        beta = float(rng.uniform(0.2, 0.9))
        omega = float(rng.uniform(1.1, 1.9))
        alpha = float(10.0 ** rng.uniform(-5.0, -2.0))
        a = float(rng.uniform(0.0, 0.5))
        b = float(rng.uniform(0.0, 0.3))
        ns = (n,) * d
        xs = _mesh(ns, 0.0, 1.0)
        t = _times(S, 1.0)[:, None]
        sines = np.ones(n ** d)
        poly = np.ones(n ** d)
        for x in xs:
            sines = sines * np.sin(np.pi * x)
            poly = poly * x * (1 - x)
        g1 = 1.0 + a * sines[None, :] * np.exp(-t)
        g2 = 1.0 + b * poly[None, :] * (1.0 + t)
        q = 1.0 + t[:, 0]
        rho = np.zeros(n ** d)
        mu = add_noise_gaussian(_manufactured_mu(ns, 0.0, 1.0, 1.0), 0.01, rng)
        out.append(Workload("batch%d_d%d_n%d_S%d" % (i, d, n, S), ns, S, 1.0, beta, omega, alpha, g1, g2, q, rho, mu))
    return out


def paper_1d(n: int, S: int, beta: float, omega: float, alpha: float = 5e-3) -> Workload:
    """Sec. 6.1: Omega = (0, pi), T = 1, gamma1 = t e^x, gamma2 = t^2 x,
    q = t^2, rho = 0, exact source f = x sin x.  mu is left to the caller
    (it is the direct-problem solution at T, then noise is added)."""
    ns = (n,)
    T = 1.0
    (x,) = _mesh(ns, 0.0, math.pi)
    t = _times(S, T)[:, None]
    g1 = t * np.exp(x)[None, :]
    g2 = t ** 2 * x[None, :]
    q = t[:, 0] ** 2
    rho = np.zeros(n)
    f = x * np.sin(x)
    return Workload("paper1d_n%d_S%d" % (n, S), ns, S, T, beta, omega, alpha, g1, g2, q, rho,
                    None, length=math.pi, f_true=f)


def paper_2d(n: int, S: int, beta: float, omega: float, alpha: float = 5e-3) -> Workload:
    """Sec. 6.2: Omega = (0, pi)^2, T = 1, gamma1 = t e^(x1+x2),
    gamma2 = t^2 x1 x2, q = t^2, rho = 0, f = x1 x2 sin(x1 x2)."""
    ns = (n, n)
    T = 1.0
    x1, x2 = _mesh(ns, 0.0, math.pi)
    t = _times(S, T)[:, None]
    g1 = t * np.exp(x1 + x2)[None, :]
    g2 = t ** 2 * (x1 * x2)[None, :]
    q = t[:, 0] ** 2
    rho = np.zeros(n * n)
    f = x1 * x2 * np.sin(x1 * x2)
    return Workload("paper2d_n%d_S%d" % (n, S), ns, S, T, beta, omega, alpha, g1, g2, q, rho,
                    None, length=math.pi, f_true=f)
