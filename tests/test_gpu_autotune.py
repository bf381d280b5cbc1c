"""The autotuner of the forward substitution's work split: every accepted candidate gives P^-1 r as
close to a tightly converged reference as the defaults do, the chosen options are one of them, and
a full solve with them matches the oracle's GMRES step count (+-1)."""
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
    res = tune(w, candidates={"pcg_iters": (4, 6, 8), "inner_tol_corr": (1e-5, 3e-6), "fused_cg": (0, 1)})
    assert len(res["table"]) == 12
    accepted = [row for row in res["table"] if row["ok"]]
    assert accepted
    best = res["opts"]
    assert any(row["pcg_iters"] == best.pcg_iters and row["inner_tol_corr"] == best.inner_tol_corr and
               row["fused_cg"] == best.fused_cg for row in accepted)
    assert res["ms"] == pytest.approx(min(row["ms"] for row in accepted))
    p = sy.problem_from(w)
    ref = gmres(lambda v: sy.matvec(p, v), sy.rhs(p), lambda v: sy.precond_solve_dense(p, v), side="left",
                restart=30, tol=1e-10, maxit=3000)
    s = t.Solver(w, opts=best)
    y = np.zeros(p.U)
    info = s.solve(y)
    s.close()
    assert info["converged"] and abs(info["iters"] - ref.iters) <= 1
