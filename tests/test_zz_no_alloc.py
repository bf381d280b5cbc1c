"""The allocation-free one-dimensional matvec (tsfde_matvec_1d_noalloc) against the
handle-based tsfde_matvec, through the C ABI.

Callers that cannot allocate device memory (memory owned by a pool or arena, no cudaMalloc
allowed while other work runs, plug-ins that may not allocate after start-up) use this entry
point; its tables and work buffer live in a fixed __device__ array.  Two calls in a row with
different sizes and orders check that nothing from one call leaks into the next.  Kept in its
own file, collected last, so that a stop at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from workloads import config_small_1d, random_vector

pytestmark = pytest.mark.gpu

TOL = 1e-12   # relative to max |z|, as for the matvec parity tests


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def _noalloc(lib, w, yd, zd):
    import torch
    g1, g2, q = _dev(w.gamma1), _dev(w.gamma2), _dev(w.q)
    st = lib.tsfde_matvec_1d_noalloc(w.ns[0], w.S, w.length, w.T, w.beta, w.omega, w.alpha,
                                     g1.data_ptr(), g2.data_ptr(), q.data_ptr(), yd.data_ptr(), zd.data_ptr(),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


def test_noalloc_matvec_matches_handle_matvec_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_2507_02809_gb300 import build
    build.build()
    import paper_2507_02809_gb300 as t
    lib = t.load()
    # two calls in a row with different sizes and orders, then the limits of the fixed array:
    # the largest transform (n + 1 = 2048, length 4096) and (S + 1) n just below 2^21 both ways
    cases = [config_small_1d(255, 40), config_small_1d(63, 64), config_small_1d(2047, 1023),
             config_small_1d(1023, 2047)]
    cases[1].beta, cases[1].omega = 0.35, 1.85
    for k, w in enumerate(cases):
        U = w.U
        yd = _dev(random_vector(U, 900 + k))
        ref = torch.zeros(U, dtype=torch.float64, device="cuda")
        s = t.Solver(w)
        s.matvec(yd, ref)
        torch.cuda.synchronize()
        s.close()
        z = torch.full((U,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, w, yd, z) == 0
        zr, zn = ref.cpu().numpy(), z.cpu().numpy()
        assert np.isfinite(zn).all()
        assert np.abs(zn - zr).max() <= TOL * np.abs(zr).max()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    import paper_2507_02809_gb300 as t
    lib = t.load()
    w = config_small_1d(63, 4)
    y = torch.zeros(w.U, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.U, dtype=torch.float64, device="cuda")
    for (n, S) in [(4095, 4), (2047, 4097), (2047, 2048), (16, 4)]:
        st = lib.tsfde_matvec_1d_noalloc(n, S, 1.0, 1.0, 0.5, 1.5, 1e-3, y.data_ptr(), y.data_ptr(), y.data_ptr(),
                                         y.data_ptr(), z.data_ptr(), None)
        assert st == -5, (n, S, st)
