"""Initial guesses of the block solves (tsfde_opts.warm_start and warm_start_mixed, 0..8: zero, the
previous level, and the polynomial through the last k levels evaluated one level further) in the
persistent forward substitution, against the oracle's dense block forward substitution (LU block
solves).

The guess changes how much work a block solve does, not the tolerance it meets: every order must
give the same P^-1 r to the FP64-mode accuracy (||P y - r|| <= 1e-10 ||r||, y within 1e-8), on a
random r and on the vector GMRES actually applies P^-1 to, A P^-1 z, whose levels vary smoothly in
time (where extrapolation acts); the mixed mode meets its own block tolerance 1e-5 at every order.
"""
import numpy as np
import pytest

from oracle import system as sy
from workloads import config_2d, config_3d, config_small_1d, random_vector

pytestmark = pytest.mark.gpu

CASES = {
    "1d_n63_S64": lambda: config_small_1d(63, 64),
    "2d_n15_S32": lambda: config_2d(0.3, 1.2, n=15, S=32),
    "2d_n15_S24_b7": lambda: config_2d(0.7, 1.8, n=15, S=24),
    "2d_n20_S16": lambda: config_2d(0.3, 1.2, n=20, S=16),
    "3d_n7_S24": lambda: config_3d(n=7, S=24),
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


def _inputs(p):
    x = sy.precond_solve_dense(p, sy.rhs(p))
    r_smooth = sy.matvec(p, x / np.linalg.norm(x))
    return {"krylov": r_smooth, "random": random_vector(p.U, 303)}


def _apply(t, w, p, rd, **opts):
    import torch
    s = t.Solver(w, opts=t.tsfde_default_opts(**opts))
    yd = _dev(np.zeros(p.U))
    st = s.precond_apply(rd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    stats = s.profile_read()
    s.close()
    return st, y, stats


@pytest.mark.parametrize("case", list(CASES))
def test_every_guess_gives_the_same_preconditioner(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    P = sy.dense_P(p)
    for name, r in _inputs(p).items():
        y_ref = sy.precond_solve_dense(p, r)
        rd = _dev(r)
        steps = {}
        for warm in (0, 1, 2, 3, 5, 6, 8):
            st, y, stats = _apply(t, w, p, rd, warm_start=warm)
            assert st == 0, (name, warm)
            assert np.linalg.norm(P @ y - r) <= 1e-10 * np.linalg.norm(r), (name, warm)
            assert np.linalg.norm(y - y_ref) <= 1e-8 * np.linalg.norm(y_ref), (name, warm)
            steps[warm] = stats["pcg_iterations"]
        if name == "krylov" and p.d >= 2:
            # on the smooth input, extrapolation lowers the CG work below the previous-level guess
            assert steps[6] < steps[1], steps


@pytest.mark.parametrize("case", ["2d_n15_S32", "1d_n63_S64"])
def test_mixed_mode_guesses(t, case):
    """Mixed mode: every block is an FP32 CG solve to 1e-5, so P^-1 is applied to about that
    accuracy whatever the guess."""
    w = CASES[case]()
    p = sy.problem_from(w)
    r = _inputs(p)["krylov"]
    y_ref = sy.precond_solve_dense(p, r)
    for warm in (0, 1, 3, 6):
        st, y, _ = _apply(t, w, p, _dev(r), precision=t.PREC_MIXED, warm_start_mixed=warm)
        assert st == 0, warm
        assert np.linalg.norm(y - y_ref) <= 1e-3 * np.linalg.norm(y_ref), warm


def test_guess_options_are_validated(t):
    w = config_small_1d(15, 4)
    for key in ("warm_start", "warm_start_mixed"):
        for bad in (-1, 9):
            with pytest.raises(t.TsfdeError) as ei:
                t.Solver(w, opts=t.tsfde_default_opts(**{key: bad}))
            assert ei.value.status == t.TSFDE_EINVAL
