"""The C ABI loads and exports every function include/tsfde.h declares; argument
validation that happens before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_02809_gb300 import build
    build.build()
    import paper_2507_02809_gb300 as t
    return t.load()


def _declared():
    with open(os.path.join(ROOT, "include", "tsfde.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsfde_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tsfde_setup", "tsfde_matvec", "tsfde_precond_apply", "tsfde_gmres_solve", "tsfde_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2507_02809_gb300 as t
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(t.EXPORTS) | set(_declared())


def test_default_opts(lib):
    import paper_2507_02809_gb300 as t
    o = t.tsfde_default_opts()
    assert o.restart == 30 and o.tol == 1e-10 and o.precision == t.PREC_FP64 and o.side == t.SIDE_LEFT


def test_status_strings(lib):
    for s in (0, 1, -1, -2, -3, -4, -5, -6):
        assert lib.tsfde_status_string(s)


def _setup_status(lib, d=1, n=63, S=8, beta=0.5, omega=1.5, alpha=1e-3, length=1.0):
    import paper_2507_02809_gb300.tsfde as tt
    N = n ** d
    g1 = np.ones(S * N)
    g2 = np.ones(S * N)
    q = np.ones(S)
    rho = np.zeros(N)
    mu = np.zeros(N)
    grid = tt.TsfdeGrid(d, n, length, S, 1.0)
    h = ctypes.c_void_p()
    st = lib.tsfde_setup(ctypes.byref(h), ctypes.byref(grid), beta, omega, alpha,
                         g1.ctypes.data, g2.ctypes.data, q.ctypes.data, rho.ctypes.data, mu.ctypes.data,
                         None, None)
    assert h.value is None
    return st


@pytest.mark.parametrize("kw,expected", [
    (dict(n=1), -5),             # too small
    (dict(d=2, n=2047), -5),     # 2-D transform longer than supported
    (dict(d=2, n=1100), -5),     # padded to 2048 points per axis: longer than supported
    (dict(d=3, n=300), -5),      # 3-D transform longer than supported
    (dict(d=4), -1),             # dimension
    (dict(beta=1.0), -1),        # Caputo order outside (0, 1)
    (dict(omega=2.0), -1),       # fractional order outside (1, 2)
    (dict(alpha=0.0), -1),       # regularisation parameter
    (dict(S=0), -1),
    (dict(length=-1.0), -1),
])
def test_setup_rejects_bad_arguments_before_touching_the_gpu(lib, kw, expected):
    assert _setup_status(lib, **kw) == expected


def test_null_handle_calls(lib):
    assert lib.tsfde_matvec(None, None, None) == -1
    assert lib.tsfde_precond_apply(None, None, None) == -1
    assert lib.tsfde_gmres_solve(None, None, None) == -1
    lib.tsfde_destroy(None)


def test_tau_blocks_need_a_power_of_two_grid(lib):
    """block_solver = 1 (T_{n,S}: tau(B_n) in the blocks) is refused before any GPU work when n + 1
    is not a power of two (the tau solves would run on a padded grid, another matrix)."""
    import paper_2507_02809_gb300.tsfde as tt
    n, S = 20, 4
    opts = tt.tsfde_default_opts(block_solver=1)
    g1 = np.ones(S * n)
    h = ctypes.c_void_p()
    grid = tt.TsfdeGrid(1, n, 1.0, S, 1.0)
    st = lib.tsfde_setup(ctypes.byref(h), ctypes.byref(grid), 0.5, 1.5, 1e-3, g1.ctypes.data, g1.ctypes.data,
                         np.ones(S).ctypes.data, np.zeros(n).ctypes.data, np.zeros(n).ctypes.data,
                         ctypes.byref(opts), None)
    assert st == -5 and h.value is None


@pytest.mark.parametrize("bs", [-1, 3])
def test_unknown_block_solver_is_refused_before_any_gpu_work(lib, bs):
    """block_solver takes 0 (P_{n,S}), 1 (T_{n,S}) or 2 (S_{n,S}); anything else is EINVAL."""
    import paper_2507_02809_gb300.tsfde as tt
    n, S = 15, 4
    opts = tt.tsfde_default_opts(block_solver=bs)
    g1 = np.ones(S * n)
    h = ctypes.c_void_p()
    grid = tt.TsfdeGrid(1, n, 1.0, S, 1.0)
    st = lib.tsfde_setup(ctypes.byref(h), ctypes.byref(grid), 0.5, 1.5, 1e-3, g1.ctypes.data, g1.ctypes.data,
                         np.ones(S).ctypes.data, np.zeros(n).ctypes.data, np.zeros(n).ctypes.data,
                         ctypes.byref(opts), None)
    assert st == -1 and h.value is None
