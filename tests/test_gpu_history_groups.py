"""The blocked history sums of the persistent forward substitution (far sums of each group of 16
positions formed at its first position, near terms per position) on medium instances: transform
lengths 256 and 512 (line groups of one and two warps), several groups of 16 positions and a last
group cut short by S (50 = 3 x 16 + 2, 40 = 2 x 16 + 8).

* P^-1 r in FP64 mode: (P y)[s, j] computed one by one by the oracle at levels in every group
  (most of them past position 32) against r, within 1e-9 max|r| (as the full-size sampled test);
  mixed mode within 1e-3 max|r| (block solves to 1e-5).
* P^-T r (the adjoint's backward substitution, whose history runs over later levels): duality
  with the forward application, <P^-1 a, b> = <a, P^-T b>, within 1e-8 (||P^-1 a|| ||b|| +
  ||a|| ||P^-T b||): both applications are within 1e-8 of exact (the FP64-mode bound of the
  parity tests), while a wrong history term moves the products by O(1).
"""
import numpy as np
import pytest

from oracle import system as sy
from workloads import config_2d, random_vector

pytestmark = pytest.mark.gpu

CASES = {
    "2d_n127_S50": lambda: config_2d(0.3, 1.2, n=127, S=50),     # L = 256: 8 groups of one warp
    "2d_n255_S40_b7": lambda: config_2d(0.7, 1.8, n=255, S=40),  # L = 512: 4 groups of two warps
}


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


def _host(x):
    import torch
    torch.cuda.synchronize()
    return x.cpu().numpy()


def _entries(p, seed):
    rng = np.random.default_rng(seed)
    levels = [0, 15, 16, 31, 32, 33, 47, 48, p.S - 1] + [int(v) for v in rng.integers(32, p.S, 12)]
    ents = [(min(s, p.S - 1), int(rng.integers(0, p.N))) for s in levels]
    ents.append((p.S, int(rng.integers(0, p.N))))
    return ents


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_forward_substitution_sampled(t, case, precision):
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(precision=precision))
    r = random_vector(p.U, 611)
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), yd) == 0
    y = _host(yd)
    ents = _entries(p, 612)
    Py = sy.precond_entries(p, y, ents)
    rr = np.array([r[s_ * p.N + j] for (s_, j) in ents])
    bound = (1e-9 if precision == 0 else 1e-3) * np.abs(r).max()
    assert np.abs(Py - rr).max() <= bound
    s.close()


@pytest.mark.parametrize("case", list(CASES))
def test_transposed_substitution_duality(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w)
    a = random_vector(p.U, 621)
    b = random_vector(p.U, 622)
    ya = _dev(np.zeros(p.U))
    lb = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(a), ya) == 0
    assert s.precond_apply_transpose(_dev(b), lb) == 0
    yah, lbh = _host(ya), _host(lb)
    lhs = float(np.dot(yah, b))
    rhs = float(np.dot(a, lbh))
    scale = np.linalg.norm(yah) * np.linalg.norm(b) + np.linalg.norm(a) * np.linalg.norm(lbh)
    assert abs(lhs - rhs) <= 1e-8 * scale
    s.close()
