"""The autotuner of the persistent forward substitution (launch shape, order of the initial guess, work
split): every accepted candidate gives P^-1 r as close to a tightly converged reference as the
defaults do, the chosen options are one of them, a full solve with them matches the oracle's GMRES
step count (+-1), and the cache returns them without tuning again."""
import numpy as np
import pytest

from oracle import system as sy
from oracle.gmres import gmres
from workloads import config_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def t():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_02809_gb300 import build
    build.build()
    import paper_2507_02809_gb300 as pkg
    return pkg


def test_autotune_small_2d(t):
    from paper_2507_02809_gb300.autotune import tune
    w = config_2d(0.5, 1.5, n=15, S=8)
    cands = {"pcg_iters": (4, 6, 8), "inner_tol_corr": (1e-5, 3e-6), "fused_cg": (0, 1), "warm_start": (2, 6),
             "grid_ctas": (0, 32)}
    res = tune(w, candidates=cands, exhaustive=True)
    assert len(res["table"]) == 48
    accepted = [row for row in res["table"] if row["ok"]]
    assert accepted
    best = res["opts"]
    assert any(all(row[k] == getattr(best, k) for k in cands) for row in accepted)
    assert res["ms"] == pytest.approx(min(row["ms"] for row in accepted))
    p = sy.problem_from(w)
    ref = gmres(lambda v: sy.matvec(p, v), sy.rhs(p), lambda v: sy.precond_solve_dense(p, v), side="left",
                restart=30, tol=1e-10, maxit=3000)
    s = t.Solver(w, opts=best)
    y = np.zeros(p.U)
    info = s.solve(y)
    s.close()
    assert info["converged"] and abs(info["iters"] - ref.iters) <= 1


def test_autotune_greedy_and_cache(t, tmp_path):
    from paper_2507_02809_gb300.autotune import tune, tuned_opts
    w = config_2d(0.3, 1.2, n=31, S=16)
    res = tune(w)
    assert any(row["ok"] for row in res["table"])
    path = str(tmp_path / "cache.json")
    o1 = tuned_opts(w, cache_path=path)
    o2 = tuned_opts(w, cache_path=path)          # from the cache
    for f, _ in t.TsfdeOpts._fields_:
        assert getattr(o1, f) == getattr(o2, f)
