"""Tuning of the forward substitution's work split for one instance.

    python -m paper_2507_02809_gb300.autotune [--n 255] [--S 256] [--beta 0.3] [--omega 1.2]

In FP64 mode a block solve is FP64 iterative refinement around FP32 tau-preconditioned CG
corrections.  How the work splits between the two is set by pcg_iters (CG steps per sweep),
inner_tol_corr (the relative residual each correction aims at) and the form of the CG step
(fused_cg); the result, a block residual below inner_tol, does not depend on them.  tune() times one
preconditioner application for each candidate (CUDA events, after a warm-up application), keeps
the candidates whose result lies as close to a tightly converged reference (block residual 1e-13) as
the default options' result does (within twice its distance, or tol_check), and returns the fastest.
"""
from __future__ import annotations

import argparse
import itertools
import os
import sys

import numpy as np

CANDIDATES = {"pcg_iters": (4, 6, 8, 12), "inner_tol_corr": (1e-4, 1e-5, 3e-6, 1e-6), "fused_cg": (1,)}


def _time_apply(solver, r, y, reps=2):
    import torch
    solver.precond_apply(r, y)        # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        st = solver.precond_apply(r, y)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, st


def tune(workload, base_opts=None, candidates=None, r=None, tol_check=1e-10, verbose=False) -> dict:
    """Time P^-1 r for each combination of the candidate options; returns
    {"opts": best TsfdeOpts, "ms": its time, "default_ms": the base options' time, "table": [...]}."""
    import torch

    from . import tsfde as t
    cands = candidates or CANDIDATES
    base = base_opts or t.tsfde_default_opts()
    s = t.Solver(workload, opts=base)
    if r is None:
        # a vector like those GMRES applies P^-1 to: the operator applied to a seeded random vector
        x = torch.as_tensor(np.random.default_rng(5).standard_normal(s.U), device="cuda")
        r = torch.zeros_like(x)
        s.matvec(x, r)
    y_def = torch.zeros_like(r)
    default_ms, _ = _time_apply(s, r, y_def)
    tight = t.tsfde_default_opts()
    for f, _ in t.TsfdeOpts._fields_:
        setattr(tight, f, getattr(base, f))
    tight.inner_tol = min(base.inner_tol, 1e-13)
    s.set_opts(tight)
    y_ref = torch.zeros_like(r)
    s.precond_apply(r, y_ref)
    ref_norm = float(torch.linalg.norm(y_ref))
    d0 = float(torch.linalg.norm(y_def - y_ref)) / ref_norm
    accept = max(2.0 * d0, tol_check)
    table = []
    best = None
    keys = list(cands)
    for combo in itertools.product(*(cands[k] for k in keys)):
        kw = dict(zip(keys, combo))
        o = t.tsfde_default_opts()
        for f, _ in t.TsfdeOpts._fields_:
            setattr(o, f, getattr(base, f))
        for k, v in kw.items():
            setattr(o, k, v)
        s.set_opts(o)
        y = torch.zeros_like(r)
        ms, st = _time_apply(s, r, y)
        diff = float(torch.linalg.norm(y - y_ref)) / ref_norm
        ok = st == 0 and diff <= accept
        table.append(dict(kw, ms=ms, status=st, rel_diff=diff, ok=ok))
        if verbose:
            print("  %-45s %8.2f ms  status %d  diff %.1e%s" % (kw, ms, st, diff, "" if ok else "  (rejected)"), flush=True)
        if ok and (best is None or ms < best[1]):
            best = (o, ms)
    s.close()
    return {"opts": best[0] if best else base, "ms": best[1] if best else default_ms, "default_ms": default_ms,
            "default_rel_diff": d0, "table": table}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=255)
    ap.add_argument("--S", type=int, default=256)
    ap.add_argument("--beta", type=float, default=0.3)
    ap.add_argument("--omega", type=float, default=1.2)
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from workloads import config_2d
    w = config_2d(args.beta, args.omega, n=args.n, S=args.S)
    res = tune(w, verbose=True)
    o = res["opts"]
    print("best: pcg_iters %d, inner_tol_corr %.0e, fused_cg %d: %.2f ms per application (defaults %.2f ms)"
          % (o.pcg_iters, o.inner_tol_corr, o.fused_cg, res["ms"], res["default_ms"]))


if __name__ == "__main__":
    main()
