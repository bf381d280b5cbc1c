"""The largest supported grids and the 3-D workload at full size, on sampled entries computed one by
one by the oracle (matvec: 1e-11 relative; P^-1: the residual P y - r on the sampled rows, 1e-9 of
max |r|).

Largest transform per dimension: d = 1, n = 2047 (L = 4096); d = 2, n = 1023 (L = 2048, trapezoid
size K = 2048 on both sides, the same definition of a_l with a coefficient table the oracle can
build); the 3-D workload 63^3, S = 256 (64 M unknowns) in the launch configuration of its timed runs.
"""
import numpy as np
import pytest

from oracle import system as sy
from workloads import config_2d, config_3d, config_small_1d, random_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def t():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_02809_gb300 import build
    build.build()
    import paper_2507_02809_gb300 as pkg
    return pkg


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _samples(p, count=10, seed=7):
    rng = np.random.default_rng(seed)
    ents = [(0, 0), (p.S - 1, p.N - 1), (p.S, 0), (p.S, p.N // 2)]
    for _ in range(count):
        ents.append((int(rng.integers(0, p.S + 1)), int(rng.integers(0, p.N))))
    return ents


CASES = {
    "1d_n2047_S4": (lambda: config_small_1d(2047, 4), None),
    "2d_n1023_S2": (lambda: config_2d(0.5, 1.5, n=1023, S=2), 2048),
    "3d_n63_S256": (lambda: config_3d(), None),
}


@pytest.mark.parametrize("case", list(CASES))
def test_matvec_and_precond_sampled(t, case):
    make, K = CASES[case]
    w = make()
    p = sy.problem_from(w, K=K)
    opts = t.tsfde_default_opts(coeff_K=K or 0)
    s = t.Solver(w, opts=opts)
    y = random_vector(p.U, 501)
    zd = _dev(np.zeros(p.U))
    s.matvec(_dev(y), zd)
    z = zd.cpu().numpy().reshape(p.S + 1, p.N)
    ents = _samples(p)
    ref = sy.matvec_entries(p, y, ents)
    got = np.array([z[a, b] for (a, b) in ents])
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    r = random_vector(p.U, 502)
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), yd) == 0
    yy = yd.cpu().numpy()
    s.close()
    ents = _samples(p, seed=8)
    Py = sy.precond_entries(p, yy, ents)
    rr = np.array([r[a * p.N + b] for (a, b) in ents])
    assert np.abs(Py - rr).max() <= 1e-9 * np.abs(r).max()
