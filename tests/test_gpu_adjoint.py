"""The transposed operator, the backward substitution for P^T and the adjoint gradients on the
GPU (through the C ABI) against the oracle, and the gradients against central finite
differences of J = 1/2 ||f - f_true||^2 through GPU forward solves.

Tolerances: A^T lam 1e-12 of max|z| (FP64 FFT against FP64 FFT); P^-T in FP64 mode: residual
||P^T lam - r|| <= 1e-10 ||r||, lam within 1e-8 (block solves at 1e-13); gradients with the
forward and adjoint solves at tol 1e-13: 1e-8 relative to the oracle's dense solves; finite
differences (relative steps 1e-4, forward solves at 1e-12): 1e-5.
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import system as sy
from workloads import config_2d, config_3d, config_adjoint_2d, config_small_1d, random_vector

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
    "1d_n3_S5": lambda: config_small_1d(3, 5),
    "1d_n7_S1": lambda: config_small_1d(7, 1),
    "2d_n15_S8": lambda: config_2d(0.3, 1.2, n=15, S=8),
    "2d_n7_S8": lambda: config_2d(0.5, 1.5, n=7, S=8, alpha=1e-3),
    "2d_n31_S3_b7": lambda: config_2d(0.7, 1.8, n=31, S=3),
    "3d_n7_S5": lambda: config_3d(n=7, S=5),
    "1d_n20_S9": lambda: config_small_1d(20, 9),
    "2d_n20_S5": lambda: config_2d(0.3, 1.2, n=20, S=5),
    "3d_n6_S3": lambda: config_3d(n=6, S=3),
}

FORMS = {"fused": dict(persistent=1, fused_cg=1), "persistent": dict(persistent=1, fused_cg=0)}


@pytest.mark.parametrize("case", list(CASES))
def test_matvec_transpose_parity(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w)
    lam = random_vector(p.U, 111)
    ref = sy.matvec_transpose(p, lam)
    zd = _dev(np.zeros(p.U))
    s.matvec_transpose(_dev(lam), zd)
    z = _host(zd)
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("case", list(CASES))
def test_precond_transpose_parity(t, case, form):
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13, **FORMS[form]))
    r = random_vector(p.U, 112)
    ref = adj.precond_transpose_solve_dense(p, r)
    ld = _dev(np.zeros(p.U))
    assert s.precond_apply_transpose(_dev(r), ld) == 0
    lam = _host(ld)
    P = sy.dense_P(p)
    assert np.linalg.norm(P.T @ lam - r) <= 1e-10 * np.linalg.norm(r)
    assert np.linalg.norm(lam - ref) <= 1e-8 * np.linalg.norm(ref)
    s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8", "3d_n7_S5"])
def test_precond_transpose_zero_trailing_blocks(t, case):
    """The backward substitution starts from the f block and the last level: with those zero
    (after another application), they stay exactly zero and every block solve converges."""
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13))
    ld = _dev(np.zeros(p.U))
    assert s.precond_apply_transpose(_dev(random_vector(p.U, 113)), ld) == 0
    r = random_vector(p.U, 114)
    k = max(1, p.S // 2)
    r[(p.S - k) * p.N:] = 0.0
    assert s.precond_apply_transpose(_dev(r), ld) == 0
    lam = _host(ld)
    assert not np.any(lam[(p.S - k) * p.N:])
    assert np.linalg.norm(sy.dense_P(p).T @ lam - r) <= 1e-10 * np.linalg.norm(r)
    s.close()


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n15_S8"])
def test_precond_transpose_mixed(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    s = t.Solver(w, opts=t.tsfde_default_opts(precision=t.PREC_MIXED))
    r = random_vector(p.U, 115)
    ref = adj.precond_transpose_solve_dense(p, r)
    ld = _dev(np.zeros(p.U))
    s.precond_apply_transpose(_dev(r), ld)
    assert np.linalg.norm(_host(ld) - ref) <= 1e-3 * np.linalg.norm(ref)
    s.close()


def _f_true(p, seed=11):
    return np.random.default_rng(seed).standard_normal(p.N)


@pytest.mark.parametrize("case", ["1d_n63_S64", "2d_n7_S8", "2d_n15_S8", "3d_n7_S5", "2d_n20_S5"])
def test_adjoint_gradients_match_oracle(t, case):
    w = CASES[case]()
    p = sy.problem_from(w)
    ft = _f_true(p)
    J, da, dm, dg, y_ref, lam_ref = adj.misfit_gradients(p, ft)
    s = t.Solver(w, opts=t.tsfde_default_opts(tol=1e-13, inner_tol=1e-13))
    y = np.zeros(p.U)
    info = s.solve(y)
    assert info["converged"]
    ybar = np.zeros(p.U)
    ybar[-p.N:] = y[-p.N:] - ft
    lam = np.zeros(p.U)
    dmu = np.zeros(p.N)
    dg2 = np.zeros(p.S * p.N)
    out = s.adjoint(y, ybar, lam, dmu, dg2)
    s.close()
    assert out["converged"], out
    assert np.linalg.norm(lam - lam_ref) <= 1e-8 * np.linalg.norm(lam_ref)
    assert out["dalpha"] == pytest.approx(da, rel=1e-8)
    assert np.linalg.norm(dmu - dm) <= 1e-8 * np.linalg.norm(dm)
    assert np.linalg.norm(dg2 - dg.reshape(-1)) <= 1e-8 * np.linalg.norm(dg)


def test_adjoint_right_and_flexible_sides(t):
    w = CASES["2d_n15_S8"]()
    p = sy.problem_from(w)
    ybar = random_vector(p.U, 116)
    lam_ref = adj.adjoint_solve_dense(p, ybar)
    for side in (t.SIDE_RIGHT, t.SIDE_FLEXIBLE):
        s = t.Solver(w, opts=t.tsfde_default_opts(tol=1e-13, inner_tol=1e-13, side=side))
        lam = np.zeros(p.U)
        out = s.adjoint(None, ybar, lam)
        s.close()
        assert out["converged"]
        assert np.linalg.norm(lam - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)


def test_autograd_function_against_central_differences(t):
    """The 127 x 127, S = 128 gradient workload: dJ/dalpha, and dJ/dmu and dJ/dgamma2 along
    seeded random directions, from the autograd Function's backward (the adjoint solve)
    against central differences of J through forward GPU solves."""
    import torch
    from paper_2507_02809_gb300.autograd import FixedInputs, recover_source
    w = config_adjoint_2d()
    S, N = w.S, w.N
    opts = t.tsfde_default_opts(tol=1e-12, inner_tol=1e-13)
    fixed = FixedInputs(d=2, n=w.ns[0], S=S, beta=w.beta, omega=w.omega, gamma1=torch.as_tensor(w.gamma1),
                        q=torch.as_tensor(w.q), rho=torch.as_tensor(w.rho), opts=opts)
    ft = torch.as_tensor(w.f_true, device="cuda")
    alpha = torch.tensor(w.alpha, dtype=torch.float64, device="cuda", requires_grad=True)
    mu = torch.as_tensor(w.mu, device="cuda").clone().requires_grad_(True)
    g2 = torch.as_tensor(w.gamma2, device="cuda").clone().requires_grad_(True)

    def J(a, m, g):
        f = recover_source(a, m, g, fixed)
        return 0.5 * torch.sum((f - ft) ** 2)

    val = J(alpha, mu, g2)
    val.backward()
    rng = np.random.default_rng(7)
    vm = torch.as_tensor(rng.standard_normal(N), device="cuda")
    vg = torch.as_tensor(rng.standard_normal((S, N)), device="cuda")
    # central differences with relative steps h = 1e-6; the forward solves stop at 1e-12, so the
    # difference quotients carry an error of about 1e-12 / 1e-6 = 1e-6 relative
    h = 1e-6
    with torch.no_grad():
        ha = h * w.alpha
        fd_a = (J(alpha + ha, mu, g2) - J(alpha - ha, mu, g2)).item() / (2 * ha)
        hm = h * float(mu.abs().max()) / float(vm.abs().max())
        fd_m = (J(alpha, mu + hm * vm, g2) - J(alpha, mu - hm * vm, g2)).item() / (2 * hm)
        hg = h / float(vg.abs().max())
        fd_g = (J(alpha, mu, g2 + hg * vg) - J(alpha, mu, g2 - hg * vg)).item() / (2 * hg)
    assert alpha.grad.item() == pytest.approx(fd_a, rel=1e-5)
    assert float((mu.grad * vm).sum()) == pytest.approx(fd_m, rel=1e-5)
    assert float((g2.grad * vg).sum()) == pytest.approx(fd_g, rel=1e-5)
    # individual components at seeded nodes (mu) and seeded (level, node) pairs (gamma2); the
    # steps are relative to the largest entry, the tolerance to the largest gradient entry
    js = rng.choice(N, size=4, replace=False)
    for j in js:
        e = torch.zeros(N, dtype=torch.float64, device="cuda")
        e[int(j)] = 1.0
        hj = h * float(mu.detach().abs().max())
        with torch.no_grad():
            fd = (J(alpha, mu + hj * e, g2) - J(alpha, mu - hj * e, g2)).item() / (2 * hj)
        assert abs(float(mu.grad[int(j)]) - fd) <= 1e-5 * float(mu.grad.abs().max())
    # one gamma2 entry moves J by less than its rounding at h = 1e-6: these use h = 1e-4
    hg1 = 1e-4
    for _ in range(4):
        sl, j = int(rng.integers(S)), int(rng.integers(N))
        e = torch.zeros((S, N), dtype=torch.float64, device="cuda")
        e[sl, j] = 1.0
        with torch.no_grad():
            fd = (J(alpha, mu, g2 + hg1 * e) - J(alpha, mu, g2 - hg1 * e)).item() / (2 * hg1)
        assert abs(float(g2.grad[sl, j]) - fd) <= 1e-5 * float(g2.grad.abs().max())
