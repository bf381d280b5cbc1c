"""FP64 row passes of the residual sweep on wide line groups (two line groups, L / 4 threads per row
pair, radix-4 transform with four values per thread), checked where their synchronisation differs:

* 2-D n = 511 (L = 1024) alone: k_fsub<1024> runs CTAs of 256 threads, so a wide group is the whole
  CTA (CTA barrier between the transform stages);
* a mixed-length batch of 2-D n = 127, 255, 511 (L = 256, 512, 1024) and a 1-D instance in one
  launch of the mixed-length kernel (CTAs of 512 threads: two to eight wide groups per CTA, named
  barriers).

Each P^-1 r (FP64 mode) against the oracle: (P y)[s, j] computed one by one at sampled levels and
nodes against r, within 1e-9 max|r| (as the full-size sampled test).
"""
import numpy as np
import pytest

from oracle import system as sy
from workloads import config_2d, config_small_1d, random_vector

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


def _check_sampled(p, r, y, seed):
    rng = np.random.default_rng(seed)
    ents = [(s, int(rng.integers(0, p.N))) for s in range(p.S + 1) for _ in range(3)]
    Py = sy.precond_entries(p, y, ents)
    rr = np.array([r[s * p.N + j] for (s, j) in ents])
    assert np.abs(Py - rr).max() <= 1e-9 * np.abs(r).max()


def test_single_instance_n511(t):
    import torch
    w = config_2d(0.3, 1.2, n=511, S=4)
    p = sy.problem_from(w)
    s = t.Solver(w)
    r = random_vector(p.U, 711)
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(r), yd) == 0
    torch.cuda.synchronize()
    _check_sampled(p, r, yd.cpu().numpy(), 712)
    s.close()


def test_mixed_length_batch(t):
    import torch
    ws = [config_2d(0.3, 1.2, n=127, S=5), config_2d(0.7, 1.8, n=255, S=4), config_2d(0.5, 1.5, n=511, S=3),
          config_small_1d(63, 6)]
    probs = [sy.problem_from(w) for w in ws]
    solvers = [t.Solver(w) for w in ws]
    rs = [random_vector(p.U, 720 + i) for i, p in enumerate(probs)]
    ys = [_dev(np.zeros(p.U)) for p in probs]
    assert t.tsfde_precond_apply_batch([s.handle for s in solvers], [_dev(r) for r in rs], ys) == 0
    torch.cuda.synchronize()
    for i, (p, r, yd) in enumerate(zip(probs, rs, ys)):
        _check_sampled(p, r, yd.cpu().numpy(), 730 + i)
    for s in solvers:
        s.close()
