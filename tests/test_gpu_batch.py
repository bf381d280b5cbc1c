"""Batched forms on the GPU: several instances share each launch of the persistent substitution
kernel, one sub-grid each (instances of one transform length: the kernel of that length;
instances of different lengths and dimensions: the mixed-length kernel).

* tsfde_precond_apply_batch: each instance's P^-1 r against the dense block forward substitution
  (residual <= 1e-10, y within 1e-8 at block tolerance 1e-13), instances differing in S, beta,
  omega, alpha and precision;
* tsfde_gmres_solve_batch: the same Arnoldi step counts as the instances solved one by one and
  solutions within 1e-10; the two 255 x 255, S = 256 instances against the oracle's full-size run.
"""
import json
import os

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


BATCHES = {
    "1d": lambda: [config_small_1d(63, 64), config_small_1d(63, 20), config_small_1d(63, 1)],
    "2d": lambda: [config_2d(0.3, 1.2, n=15, S=8), config_2d(0.7, 1.8, n=15, S=12),
                   config_2d(0.5, 1.5, n=15, S=5, alpha=1e-3)],
    "3d": lambda: [config_3d(n=7, S=5), config_3d(n=7, S=3, beta=0.4, omega=1.3)],
    "2d_padded": lambda: [config_2d(0.3, 1.2, n=20, S=5), config_2d(0.7, 1.8, n=20, S=3)],
    # different n with one transform length (n + 1 rounded up to 32 / 64)
    "2d_uneven": lambda: [config_2d(0.3, 1.2, n=20, S=5), config_2d(0.7, 1.8, n=25, S=3),
                          config_2d(0.5, 1.5, n=31, S=4)],
    "1d_uneven": lambda: [config_small_1d(40, 9), config_small_1d(50, 5), config_small_1d(63, 7)],
}


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("name", list(BATCHES))
def test_precond_apply_batch_parity(t, name, fused):
    import torch
    ws = BATCHES[name]()
    solvers = [t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13, fused_cg=fused)) for w in ws]
    probs = [sy.problem_from(w) for w in ws]
    rs = [random_vector(p.U, 300 + i) for i, p in enumerate(probs)]
    ys = [_dev(np.zeros(p.U)) for p in probs]
    st = t.tsfde_precond_apply_batch([s.handle for s in solvers], [_dev(r) for r in rs], ys)
    assert st == 0
    torch.cuda.synchronize()
    for p, r, yd in zip(probs, rs, ys):
        y = yd.cpu().numpy()
        P = sy.dense_P(p)
        assert np.linalg.norm(P @ y - r) <= 1e-10 * np.linalg.norm(r)
        ref = sy.precond_solve_dense(p, r)
        assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(ref)
    for s in solvers:
        s.close()


def test_precond_apply_batch_mixed_precisions(t):
    """One FP64-mode and one mixed-mode instance in the same launch."""
    import torch
    ws = [config_2d(0.3, 1.2, n=15, S=8), config_2d(0.7, 1.8, n=15, S=6)]
    solvers = [t.Solver(ws[0], opts=t.tsfde_default_opts(inner_tol=1e-13)),
               t.Solver(ws[1], opts=t.tsfde_default_opts(precision=t.PREC_MIXED))]
    probs = [sy.problem_from(w) for w in ws]
    rs = [random_vector(p.U, 310 + i) for i, p in enumerate(probs)]
    ys = [_dev(np.zeros(p.U)) for p in probs]
    assert t.tsfde_precond_apply_batch([s.handle for s in solvers], [_dev(r) for r in rs], ys) == 0
    torch.cuda.synchronize()
    refs = [sy.precond_solve_dense(p, r) for p, r in zip(probs, rs)]
    y0, y1 = ys[0].cpu().numpy(), ys[1].cpu().numpy()
    assert np.linalg.norm(y0 - refs[0]) <= 1e-8 * np.linalg.norm(refs[0])
    assert np.linalg.norm(y1 - refs[1]) <= 1e-3 * np.linalg.norm(refs[1])
    for s in solvers:
        s.close()


@pytest.mark.parametrize("name", ["1d", "2d", "3d", "2d_padded", "2d_uneven", "1d_uneven"])
def test_gmres_solve_batch_equals_single_solves(t, name):
    ws = BATCHES[name]()
    opts = t.tsfde_default_opts(tol=1e-12, inner_tol=1e-13)
    single = []
    for w in ws:
        s = t.Solver(w, opts=opts)
        y = np.zeros(s.U)
        info = s.solve(y)
        single.append((info, y))
        s.close()
    solvers = [t.Solver(w, opts=opts) for w in ws]
    ys = [np.zeros(s.U) for s in solvers]
    infos = t.tsfde_gmres_solve_batch([s.handle for s in solvers], ys)
    for (info1, y1), info, y in zip(single, infos, ys):
        assert info["converged"]
        assert info["iters"] == info1["iters"]
        assert np.linalg.norm(y - y1) <= 1e-10 * np.linalg.norm(y1)
    for s in solvers:
        s.close()


# instances of DIFFERENT dimensions and transform lengths: one launch of the mixed-length kernel
MIXED = {
    "1d_2d": lambda: [config_small_1d(63, 20), config_2d(0.3, 1.2, n=15, S=8), config_small_1d(200, 9),
                      config_2d(0.7, 1.8, n=40, S=5)],
    "1d_2d_3d": lambda: [config_3d(n=7, S=5), config_2d(0.5, 1.5, n=31, S=6), config_small_1d(1500, 4),
                         config_small_1d(15, 3)],
}


@pytest.mark.parametrize("name", list(MIXED))
def test_precond_apply_batch_mixed_lengths(t, name):
    """Every instance's P^-1 r from one mixed-length launch against the dense block forward
    substitution (as for same-length batches)."""
    import torch
    ws = MIXED[name]()
    solvers = [t.Solver(w, opts=t.tsfde_default_opts(inner_tol=1e-13)) for w in ws]
    probs = [sy.problem_from(w) for w in ws]
    rs = [random_vector(p.U, 320 + i) for i, p in enumerate(probs)]
    ys = [_dev(np.zeros(p.U)) for p in probs]
    assert t.tsfde_precond_apply_batch([s.handle for s in solvers], [_dev(r) for r in rs], ys) == 0
    torch.cuda.synchronize()
    for p, r, yd in zip(probs, rs, ys):
        y = yd.cpu().numpy()
        if p.U <= 5000:
            P = sy.dense_P(p)
            assert np.linalg.norm(P @ y - r) <= 1e-10 * np.linalg.norm(r)
        ref = sy.precond_solve_dense(p, r)
        assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(ref)
    for s in solvers:
        s.close()


@pytest.mark.parametrize("name", list(MIXED))
def test_gmres_solve_batch_mixed_lengths(t, name):
    """Uneven instances solved in lockstep, each preconditioner round one mixed-length launch: the
    Arnoldi step counts of the instances solved alone (within +-1: a sub-grid of another size sums
    in another order) and solutions within 1e-10 of theirs."""
    ws = MIXED[name]()
    opts = t.tsfde_default_opts(tol=1e-12, inner_tol=1e-13)
    single = []
    for w in ws:
        s = t.Solver(w, opts=opts)
        y = np.zeros(s.U)
        single.append((s.solve(y), y))
        s.close()
    solvers = [t.Solver(w, opts=opts) for w in ws]
    ys = [np.zeros(s.U) for s in solvers]
    infos = t.tsfde_gmres_solve_batch([s.handle for s in solvers], ys)
    for (info1, y1), info, y in zip(single, infos, ys):
        assert info["converged"]
        assert abs(info["iters"] - info1["iters"]) <= 1
        assert np.linalg.norm(y - y1) <= 1e-10 * np.linalg.norm(y1)
    for s in solvers:
        s.close()


def test_mixed_batch_graph_replays_equal_direct_launches(t):
    """graphs = 1: each round of a mixed-length batch replays the captured launch sequence; the
    results are bitwise those of launching every round directly (graphs = 0), since the launch
    configuration is the same."""
    ws = MIXED["1d_2d"]()
    out = {}
    for graphs in (0, 1):
        opts = t.tsfde_default_opts(tol=1e-12, inner_tol=1e-13, graphs=graphs)
        solvers = [t.Solver(w, opts=opts) for w in ws]
        ys = [np.zeros(s.U) for s in solvers]
        infos = t.tsfde_gmres_solve_batch([s.handle for s in solvers], ys)
        sts = [s.profile_read() for s in solvers]   # the leading handle of a round holds its graph
        st = {k: sum(x[k] for x in sts) for k in ("batch_graph_builds", "batch_graph_replays")}
        st["error"] = " ".join(x["batch_graph_error"] for x in sts)
        for s in solvers:
            s.close()
        out[graphs] = (ys, infos, st)
    assert out[0][2]["batch_graph_replays"] == 0
    assert out[1][2]["batch_graph_builds"] >= 1, out[1][2]["error"]
    # every mixed-length round is a replay (a round left with instances of one length, or with a
    # single instance, uses that length's kernel directly)
    assert out[1][2]["batch_graph_replays"] >= out[1][2]["batch_graph_builds"]
    assert out[1][2]["batch_graph_replays"] >= min(i["iters"] for i in out[1][1])
    for y0, y1 in zip(out[0][0], out[1][0]):
        assert np.array_equal(y0, y1)


def test_batch_rejects_repeated_handles(t):
    a = t.Solver(config_2d(0.3, 1.2, n=15, S=4))
    with pytest.raises(t.TsfdeError):
        t.tsfde_gmres_solve_batch([a.handle, a.handle], [np.zeros(a.U), np.zeros(a.U)])
    a.close()


def test_full_size_2d_batched_solves_match_oracle_golden(t):
    """The two 255 x 255, S = 256 instances solved as one batch: Arnoldi steps within +-1 of the
    oracle's full-size run, f and the stored time levels element by element within 1e-10 (as for
    the single solves)."""
    from test_gpu_parity import assert_matches_golden, load_golden
    golden = load_golden()
    if golden is None:
        pytest.skip("golden oracle solve not generated")
    insts = golden["instances"]
    solvers = [t.Solver(config_2d(i["beta"], i["omega"])) for i in insts]
    ys = [np.zeros(s.U) for s in solvers]
    infos = t.tsfde_gmres_solve_batch([s.handle for s in solvers], ys)
    for k, (inst, info, y, s) in enumerate(zip(insts, infos, ys, solvers)):
        assert info["converged"]
        assert abs(info["iters"] - inst["iters"]) <= 1
        assert_matches_golden(golden, k, y, s.N, s.S)
    for s in solvers:
        s.close()
