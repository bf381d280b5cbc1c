"""The seeded synthetic inputs (workloads/): determinism, the grid of Sec. 4, the exact noise level
of Eq. 3, the coefficient ranges the solvers rely on, the batched workload's parameter ranges, and
the module's independence from the method's arithmetic."""
import ast
import math
import os

import numpy as np
import pytest

import workloads as wl
from workloads import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_same_seed_same_inputs_other_seed_other_noise():
    a, b = wl.config_2d(0.3, 1.2, n=15, S=8), wl.config_2d(0.3, 1.2, n=15, S=8)
    for name in ("gamma1", "gamma2", "q", "rho", "mu"):
        np.testing.assert_array_equal(getattr(a, name), getattr(b, name))
    c = wl.config_2d(0.3, 1.2, n=15, S=8, seed=7)
    assert not np.array_equal(a.mu, c.mu)
    np.testing.assert_array_equal(a.gamma1, c.gamma1)
    np.testing.assert_array_equal(wl.random_vector(100, 3), wl.random_vector(100, 3))


@pytest.mark.parametrize("make,level", [(lambda: wl.config_2d(0.3, 1.2, n=31, S=4), 0.01),
                                        (lambda: wl.config_3d(n=9, S=4), 0.005),
                                        (lambda: wl.config_adjoint_2d(n=15, S=4), 0.01)])
def test_gaussian_noise_has_exactly_the_requested_relative_level(make, level):
    """Eq. 3 reading: ||mu_eps - mu||_2 = level ||mu||_2 exactly, mu = u(., T) of
    u = t^2 prod x_i^2 (1 - x_i)^2."""
    w = make()
    clean = syn._manufactured_mu(w.ns, 0.0, 1.0, w.T)
    assert abs(np.linalg.norm(w.mu - clean) / np.linalg.norm(clean) - level) < 1e-12


def test_uniform_noise_is_bounded_by_eps():
    """Sec. 6.1 noise: mu + eps delta, delta ~ U(-1, 1) per node, eps = rel ||mu||_2."""
    mu = np.linspace(0.0, 1.0, 257)
    out = wl.add_noise_uniform(mu, 0.01, np.random.default_rng(1))
    eps = 0.01 * np.linalg.norm(mu)
    assert np.abs(out - mu).max() <= eps
    assert np.abs(out - mu).max() > 0.9 * eps          # the draws fill the interval


def test_grid_spacing_and_lexicographic_order():
    """x_j = j h, h = 1 / (n + 1), j = 1..n; node (i, j) of a 2-D grid at index i n + j (last index
    fastest); t_s = s T / S.  Read back from gamma2 = 1 + 0.2 (x + y) t of the 2-D workload."""
    n, S = 7, 4
    w = wl.config_2d(0.3, 1.2, n=n, S=S)
    h = 1.0 / (n + 1)
    for s in (0, S - 1):
        t = (s + 1) / S
        for i, j in ((0, 0), (0, n - 1), (n - 1, 0), (3, 5)):
            x, y = (i + 1) * h, (j + 1) * h
            assert w.gamma2[s, i * n + j] == pytest.approx(1.0 + 0.2 * (x + y) * t, rel=1e-15)
    # mu is u(., 1) before noise: symmetric under x <-> y
    clean = syn._manufactured_mu(w.ns, 0.0, 1.0, 1.0).reshape(n, n)
    np.testing.assert_allclose(clean, clean.T, rtol=0, atol=1e-18)


def test_coefficient_ranges():
    """gamma2 > 0 everywhere (the symmetrised block solves divide by it); the 3-D fields stay in the
    ranges the inputs are specified with: gamma1 in [1, 1.4], gamma2 in [0.75, 1.25]."""
    for w in (wl.config_small_1d(31, 8), wl.config_2d(0.7, 1.8, n=15, S=8), wl.config_3d(n=7, S=8),
              wl.config_adjoint_2d(n=15, S=8)):
        assert w.gamma2.min() > 0 and w.gamma1.min() >= 1.0 - 1e-15
        assert w.gamma1.shape == (w.S, w.N) and w.gamma2.shape == (w.S, w.N)
        assert w.q.shape == (w.S,) and w.rho.shape == (w.N,) and w.mu.shape == (w.N,)
    w3 = wl.config_3d(n=15, S=16)
    assert 1.0 <= w3.gamma1.min() and w3.gamma1.max() <= 1.4
    assert 0.75 <= w3.gamma2.min() and w3.gamma2.max() <= 1.25


def test_paper_replica_coefficients():
    """Sec. 6.1: Omega = (0, pi), gamma1 = t e^x, gamma2 = t^2 x, q = t^2, f = x sin x."""
    n, S = 9, 5
    w = wl.paper_1d(n, S, 0.5, 1.5)
    h = math.pi / (n + 1)
    x = h * np.arange(1, n + 1)
    t = np.arange(1, S + 1) / S
    np.testing.assert_allclose(w.gamma1, t[:, None] * np.exp(x)[None, :], rtol=1e-15)
    np.testing.assert_allclose(w.gamma2, (t ** 2)[:, None] * x[None, :], rtol=1e-15)
    np.testing.assert_allclose(w.q, t ** 2, rtol=1e-15)
    np.testing.assert_allclose(w.f_true, x * np.sin(x), rtol=1e-15)
    assert w.mu is None and w.length == math.pi


def test_batched_workload_parameter_ranges():
    """The first instances of the batched workload (the draws of instance i do not depend on how
    many follow): d = 1 with n in [127, 2047], S in [64, 512]; d = 2 with n in [63, 255],
    S in [64, 256]; beta in (0.2, 0.9), omega in (1.1, 1.9), alpha in [1e-5, 1e-2]; 1 % noise."""
    ws = wl.config_batch(count_1d=32, count_2d=2)
    assert len(ws) == 34
    ones, twos = ws[:32], ws[32:]
    assert all(w.d == 1 and 127 <= w.ns[0] <= 2047 and 64 <= w.S <= 512 for w in ones)
    assert all(w.d == 2 and 63 <= w.ns[0] <= 255 and 64 <= w.S <= 256 for w in twos)
    for w in ws:
        assert 0.2 <= w.beta <= 0.9 and 1.1 <= w.omega <= 1.9 and 1e-5 <= w.alpha <= 1e-2
        clean = syn._manufactured_mu(w.ns, 0.0, 1.0, 1.0)
        assert abs(np.linalg.norm(w.mu - clean) / np.linalg.norm(clean) - 0.01) < 1e-12
    # uneven sizes: several transform lengths among the 1-D instances
    lengths = {2 * (1 << math.ceil(math.log2(w.ns[0] + 1))) for w in ones}
    assert len(lengths) >= 3
    again = wl.config_batch(count_1d=32, count_2d=2)
    assert [(w.ns, w.S, w.beta) for w in again] == [(w.ns, w.S, w.beta) for w in ws]


def test_workloads_hold_none_of_the_method():
    """The input generators import only numpy and the standard library: no oracle, no solver."""
    for fname in ("__init__.py", "synthetic.py"):
        tree = ast.parse(open(os.path.join(ROOT, "workloads", fname)).read())
        mods = set()
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods.update(a.name.split(".")[0] for a in node.names)
            elif isinstance(node, ast.ImportFrom) and node.level == 0:
                mods.add(node.module.split(".")[0])
        assert mods <= {"numpy", "math", "dataclasses", "__future__"}, mods
