"""Failure paths of the library, made to happen without faulting, trapping or hanging the GPU.

* A grid-barrier wait of the persistent forward substitution that runs out of polls: the launch
  returns TSFDE_ETIMEOUT (every CTA leaves at its next barrier), and the same handle then solves
  correctly with the default limit.  The short limit is an option (tsfde_opts.spin_limit), so the
  wait ends by itself after one poll; nothing is made to hang.
* Host-side injections: NaN in the data mu -> TSFDE_EBREAKDOWN; an iteration cap of one Arnoldi step
  -> TSFDE_NOT_CONVERGED with a finite best iterate; gamma2 <= 0 -> TSFDE_EINVAL at set-up.

The paper's only failure notion is the ">1000" non-convergence marker of Tables 2 and 7, which the
iteration cap reproduces.
"""
import numpy as np
import pytest
import torch

import paper_2507_02809_gb300 as t
from workloads import config_2d, config_small_1d, random_vector

pytestmark = pytest.mark.gpu


def _small2d():
    return config_2d(0.3, 1.2, n=31, S=16)


def test_barrier_timeout_then_same_handle_recovers():
    w = _small2d()
    s = t.Solver(w, opts=t.tsfde_default_opts(spin_limit=1))
    r = torch.as_tensor(random_vector(s.U, 7), device="cuda")
    y = torch.zeros_like(r)
    with pytest.raises(t.TsfdeError) as ei:
        s.precond_apply(r, y)
    assert ei.value.status == t.TSFDE_ETIMEOUT
    # the GMRES driver reports the same status
    x = torch.zeros_like(r)
    with pytest.raises(t.TsfdeError) as ei:
        s.solve(x)
    assert ei.value.status == t.TSFDE_ETIMEOUT
    # same handle, default limit: a correct application, equal to a fresh handle's
    s.set_opts(t.tsfde_default_opts())
    assert s.precond_apply(r, y) == t.TSFDE_OK
    s2 = t.Solver(w)
    y2 = torch.zeros_like(r)
    assert s2.precond_apply(r, y2) == t.TSFDE_OK
    assert torch.isfinite(y).all()
    assert float(torch.linalg.vector_norm(y - y2) / torch.linalg.vector_norm(y2)) <= 1e-12
    # and a full solve converges on it
    info = s.solve(x)
    assert info["status"] == t.TSFDE_OK and info["converged"]
    s.close()
    s2.close()


def test_spin_limit_must_be_positive():
    w = _small2d()
    with pytest.raises(t.TsfdeError) as ei:
        t.Solver(w, opts=t.tsfde_default_opts(spin_limit=0))
    assert ei.value.status == t.TSFDE_EINVAL


def test_nan_in_mu_is_a_breakdown():
    w = _small2d()
    w.mu = w.mu.copy()
    w.mu[len(w.mu) // 3] = np.nan
    s = t.Solver(w)
    y = torch.zeros(s.U, dtype=torch.float64, device="cuda")
    with pytest.raises(t.TsfdeError) as ei:
        s.solve(y)
    assert ei.value.status == t.TSFDE_EBREAKDOWN
    s.close()


@pytest.mark.parametrize("side", [t.SIDE_LEFT, t.SIDE_FLEXIBLE])
def test_iteration_cap_returns_best_iterate(side):
    w = config_small_1d()
    s = t.Solver(w, opts=t.tsfde_default_opts(max_iters=1, side=side))
    y = torch.zeros(s.U, dtype=torch.float64, device="cuda")
    info = s.solve(y)
    assert info["status"] == t.TSFDE_NOT_CONVERGED
    assert not info["converged"]
    assert info["iters"] == 1
    assert torch.isfinite(y).all() and float(torch.linalg.vector_norm(y)) > 0.0
    assert 0.0 < info["relres_est"] < 1.0
    s.close()


@pytest.mark.parametrize("bad", [0.0, -0.5, np.inf])
def test_nonpositive_gamma2_is_rejected(bad):
    w = config_small_1d()
    w.gamma2 = w.gamma2.copy()
    w.gamma2.reshape(-1)[5] = bad
    with pytest.raises(t.TsfdeError) as ei:
        t.Solver(w)
    assert ei.value.status == t.TSFDE_EINVAL
