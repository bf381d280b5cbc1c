"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small cases (several FFT tiles, odd row counts, S = 1, n = 3) are compared element by
element with the assembled or structured oracle; the 255 x 255, S = 256 workload is
checked on sampled entries computed one by one by the oracle.
Tolerances: matvec 1e-12 of max|z| (FP64 FFT against FP64 FFT); preconditioner in FP64
mode: residual ||P y - r|| <= 1e-10 ||r|| and y within 1e-8 (inner block solves stop
at a residual of 1e-13, amplified by at most the block condition number); GMRES solved
to 1e-12 against dense LU: 1e-10 in f and in u; iteration counts within +-1 of the
oracle's GMRES with the same side, restart and tolerance.
"""
import numpy as np
import pytest

from oracle import system as sy
from oracle.gmres import gmres
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


def _host(x):
    import torch
    torch.cuda.synchronize()
    return x.cpu().numpy()


CASES = {
    "1d_n63_S64": lambda: config_small_1d(63, 64),
    "1d_n7_S1": lambda: config_small_1d(7, 1),
    "1d_n3_S5": lambda: config_small_1d(3, 5),
    "1d_n255_S20": lambda: config_small_1d(255, 20),
    "2d_n15_S8": lambda: config_2d(0.3, 1.2, n=15, S=8),
    "2d_n31_S12_b7": lambda: config_2d(0.7, 1.8, n=31, S=12),
    "2d_n3_S2": lambda: config_2d(0.5, 1.5, n=3, S=2),
    "3d_n7_S5": lambda: config_3d(n=7, S=5),
    "3d_n15_S3": lambda: config_3d(n=15, S=3),
    # n + 1 not a power of two: transforms on the next power-of-two grid, tau solves zero-padded
    "1d_n20_S9": lambda: config_small_1d(20, 9),
    "1d_n100_S7": lambda: config_small_1d(100, 7),
    "2d_n20_S5": lambda: config_2d(0.3, 1.2, n=20, S=5),
    "2d_n10_S4_b7": lambda: config_2d(0.7, 1.8, n=10, S=4),
    "3d_n6_S3": lambda: config_3d(n=6, S=3),
    "3d_n10_S2": lambda: config_3d(n=10, S=2),
}


@pytest.mark.parametrize("case", list(CASES))
def test_matvec_and_rhs_parity(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w)
    y = random_vector(p.U, 101)
    z_ref = sy.matvec(p, y)
    yd = _dev(y)
    zd = _dev(np.zeros(p.U))
    s.matvec(yd, zd)
    z = _host(zd)
    scale = np.abs(z_ref).max()
    assert np.abs(z - z_ref).max() <= 1e-12 * scale
    s.rhs(zd)
    np.testing.assert_allclose(_host(zd), sy.rhs(p), rtol=1e-14, atol=1e-300)
    s.close()


# forms of the forward substitution: one persistent kernel with the four-pass inner CG, the
# same kernel with the six-pass inner CG, a CUDA graph of separate kernels
FORMS = {"fused": dict(persistent=1, fused_cg=1), "persistent": dict(persistent=1, fused_cg=0),
         "graph": dict(persistent=0)}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("case", ["1d_n63_S64", "1d_n7_S1", "1d_n3_S5", "2d_n15_S8", "2d_n3_S2", "3d_n7_S5",
                                  "3d_n15_S3", "1d_n255_S20", "1d_n20_S9", "1d_n100_S7", "2d_n20_S5",
                                  "2d_n10_S4_b7", "3d_n6_S3", "3d_n10_S2"])
def test_precond_parity_fp64(t, case, form):
    """Every form of the forward substitution against the dense block forward substitution."""
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13, **FORMS[form]))
    r = random_vector(p.U, 202)
    y_ref = sy.precond_solve_dense(p, r)
    rd = _dev(r)
    yd = _dev(np.zeros(p.U))
    st = s.precond_apply(rd, yd)
    assert st == 0
    y = _host(yd)
    P = sy.dense_P(p)
    assert np.linalg.norm(P @ y - r) <= 1e-10 * np.linalg.norm(r)
    assert np.linalg.norm(y - y_ref) <= 1e-8 * np.linalg.norm(y_ref)
    s.close()


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8", "3d_n7_S5"])
def test_precond_zero_leading_blocks(t, case, form):
    """P^-1 of a vector whose first levels vanish (as for z with rho = 0), applied after another
    application: those levels of y are exactly zero, every block solve converges (status 0),
    and y solves P y = r."""
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13, **FORMS[form]))
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(_dev(random_vector(p.U, 204)), yd) == 0
    r = random_vector(p.U, 205)
    k = max(1, p.S // 2)
    r[: k * p.N] = 0.0
    assert s.precond_apply(_dev(r), yd) == 0
    y = _host(yd)
    assert not np.any(y[: k * p.N])
    P = sy.dense_P(p)
    assert np.linalg.norm(P @ y - r) <= 1e-10 * np.linalg.norm(r)
    s.close()


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8", "3d_n7_S5", "3d_n15_S3", "2d_n20_S5", "3d_n10_S2"])
def test_precond_mixed_precision(t, case, form):
    """FP32 block solves to 1e-5: the result is an approximation of P^-1 r."""
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(precision=t.PREC_MIXED, **FORMS[form]))
    r = random_vector(p.U, 203)
    y_ref = sy.precond_solve_dense(p, r)
    rd = _dev(r)
    yd = _dev(np.zeros(p.U))
    s.precond_apply(rd, yd)
    y = _host(yd)
    assert np.linalg.norm(y - y_ref) <= 1e-3 * np.linalg.norm(y_ref)
    s.close()


def test_gmres_small_1d_against_dense_lu(t):
    """The 63-point, 64-level case: GMRES(30) to 1e-12 against a dense LU solve."""
    w = config_small_1d(63, 64)
    p = sy.problem_from(w)
    A = sy.dense_A(p)
    z = sy.rhs(p)
    y_lu = np.linalg.solve(A, z)
    s = t.Solver(w, opts=t.tsfde_default_opts(tol=1e-12, inner_tol=1e-13))
    y = np.zeros(p.U)
    info = s.solve(y)
    assert info["converged"], info
    Y, Yl = y.reshape(p.S + 1, p.N), y_lu.reshape(p.S + 1, p.N)
    assert np.linalg.norm(Y[-1] - Yl[-1]) <= 1e-10 * np.linalg.norm(Yl[-1])
    assert np.linalg.norm(Y[:-1] - Yl[:-1]) <= 1e-10 * np.linalg.norm(Yl[:-1])
    s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8", "2d_n31_S12_b7", "1d_n100_S7", "2d_n20_S5"])
def test_gmres_iterations_match_oracle(t, case):
    """Left-preconditioned GMRES(30), tol 1e-10: same iteration count as the oracle (+-1)."""
    w = CASES[case]()
    p = sy.problem_from(w)
    z = sy.rhs(p)
    ref = gmres(lambda v: sy.matvec(p, v), z, lambda v: sy.precond_solve_dense(p, v), side="left",
                restart=30, tol=1e-10, maxit=3000)
    assert ref.converged
    s = t.Solver(w)
    y = np.zeros(p.U)
    info = s.solve(y)
    assert info["converged"], info
    assert abs(info["iters"] - ref.iters) <= 1, (info["iters"], ref.iters)
    # same solution up to the attainable accuracy of two solves stopped at 1e-10
    assert np.linalg.norm(y - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8"])
def test_gmres_right_and_flexible(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    z = sy.rhs(p)
    y_lu = np.linalg.solve(sy.dense_A(p), z)
    for side, prec in ((t.SIDE_RIGHT, t.PREC_FP64), (t.SIDE_FLEXIBLE, t.PREC_MIXED)):
        s = t.Solver(w, opts=t.tsfde_default_opts(side=side, precision=prec, tol=1e-11))
        y = np.zeros(p.U)
        info = s.solve(y)
        assert info["converged"], (side, prec, info)
        assert info["relres_true"] <= 2e-11
        assert np.linalg.norm(y - y_lu) <= 1e-8 * np.linalg.norm(y_lu)
        s.close()


def test_mixed_f_within_1e8_of_fp64(t):
    w = config_2d(0.3, 1.2, n=31, S=16)
    s64 = t.Solver(w, opts=t.tsfde_default_opts(tol=1e-10))
    y64 = np.zeros(s64.U)
    i64 = s64.solve(y64)
    smx = t.Solver(w, opts=t.tsfde_default_opts(side=t.SIDE_FLEXIBLE, precision=t.PREC_MIXED, tol=1e-10))
    ymx = np.zeros(smx.U)
    imx = smx.solve(ymx)
    assert i64["converged"] and imx["converged"]
    assert imx["relres_true"] <= 1e-10
    N = s64.N
    f64, fmx = y64[-N:], ymx[-N:]
    assert np.linalg.norm(fmx - f64) <= 1e-8 * np.linalg.norm(f64)
    s64.close()
    smx.close()


@pytest.fixture(scope="module")
def big2d():
    w = config_2d(0.3, 1.2)   # 255 x 255, S = 256, the timed workload
    p = sy.problem_from(w)
    _ = p.a
    return w, p


def _samples(p, count=12, seed=7):
    rng = np.random.default_rng(seed)
    ents = [(0, 0), (p.S - 1, p.N - 1), (p.S, 0), (p.S, p.N // 2)]
    for _ in range(count):
        ents.append((int(rng.integers(0, p.S + 1)), int(rng.integers(0, p.N))))
    return ents


def test_full_size_2d_matvec_sampled(t, big2d):
    w, p = big2d
    s = t.Solver(w)
    y = random_vector(p.U, 301)
    yd = _dev(y)
    zd = _dev(np.zeros(p.U))
    s.matvec(yd, zd)
    z = _host(zd).reshape(p.S + 1, p.N)
    ents = _samples(p)
    ref = sy.matvec_entries(p, y, ents)
    got = np.array([z[s_, j] for (s_, j) in ents])
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    s.close()


@pytest.mark.parametrize("form", list(FORMS))
def test_full_size_2d_precond_sampled(t, big2d, form):
    w, p = big2d
    s = t.Solver(w, opts=t.tsfde_default_opts(**FORMS[form]))
    r = random_vector(p.U, 302)
    rd = _dev(r)
    yd = _dev(np.zeros(p.U))
    assert s.precond_apply(rd, yd) == 0
    y = _host(yd)
    ents = _samples(p, seed=8)
    Py = sy.precond_entries(p, y, ents)
    rr = np.array([r[s_ * p.N + j] for (s_, j) in ents])
    assert np.abs(Py - rr).max() <= 1e-9 * np.abs(r).max()
    s.close()


def load_golden():
    """The oracle's full-size solves (tests/golden/config2_oracle.json with the solution fields in
    config2_oracle_fields.npz, both written by tests/golden/make_config2_oracle.py), or None."""
    import json
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    path = os.path.join(here, "config2_oracle.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        golden = json.load(fh)
    fpath = os.path.join(here, golden.get("fields", "config2_oracle_fields.npz"))
    if not os.path.exists(fpath):
        return None
    golden["arrays"] = dict(np.load(fpath))
    return golden


def assert_matches_golden(golden, k, y, N, S):
    """f = y^(S+1) and the stored time levels v^(1), v^(S/2), v^(S) of the GPU solution against
    the oracle's, element by element: relative error in the 2-norm <= 1e-10 per field."""
    arr = golden["arrays"]
    Y = y.reshape(S + 1, N)
    for name, got in (("f", Y[S]), ("v1", Y[0]), ("vmid", Y[S // 2 - 1]), ("vS", Y[S - 1])):
        ref = arr["%s_%d" % (name, k)]
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (k, name, err)


def test_full_size_2d_iterations_match_oracle_golden(t):
    """The 255 x 255, S = 256 solves against the oracle's own GMRES on the same workload: the
    solution f and the time levels v^(1), v^(S/2), v^(S) element by element (relative error
    <= 1e-10), Arnoldi steps within +-1, and the true residual of the final iterate within 5e-3.
    GMRES with left preconditioning stops on the preconditioned residual, so the true residual at
    that point (4.7e-8 and 7.8e-6 here, far above 1e-10) carries the rounding of every P^-1
    application: GPU and oracle differ there by up to 8e-4 relative."""
    golden = load_golden()
    if golden is None:
        pytest.skip("golden oracle solve not generated")
    assert golden["instances"]
    for k, inst in enumerate(golden["instances"]):
        w = config_2d(inst["beta"], inst["omega"])
        s = t.Solver(w)
        y = np.zeros(s.U)
        info = s.solve(y)
        s.close()
        assert info["converged"]
        assert abs(info["iters"] - inst["iters"]) <= 1, (info["iters"], inst["iters"])
        assert info["relres_true"] == pytest.approx(inst["relres_true"], rel=5e-3)
        assert_matches_golden(golden, k, y, s.N, s.S)
