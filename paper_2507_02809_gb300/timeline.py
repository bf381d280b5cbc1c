"""Timeline of one preconditioner application on the 2-D workload (255 x 255, S levels).

    python -m paper_2507_02809_gb300.timeline [--precision 0|1] [--S 256] [--n 255] [--warm 0..8]
                                              [--fused 0|1] [--d 2|3] [--input krylov|random]

Applies P^-1 once (after one warm-up application) to the vector GMRES applies it to in its first
Arnoldi step, A P^-1 z (--input krylov, z the right-hand side), or to a seeded random vector, with the
persistent forward substitution and prints, per kind of pass, how many passes ran and the
time between the grid barriers that close them (tsfde_profile(h, 2)).  With the four-pass
inner CG (--fused 1) its passes are counted as: columns of B p -> b32_cols, rows of B p with
q and its row sine transforms -> b32_rowinv, first strided pass of the tau solve -> tau_cols,
last row pass with z, x, r and the row spectra of z -> tau_rows_out.
"""
from __future__ import annotations

import argparse
import os
import sys

NAMES = ["rhs", "b64_rowfwd", "b64_cols", "b64_rowinv", "tau_rows_in", "tau_cols", "tau_rows_out",
         "b32_rowfwd", "b32_cols", "b32_rowinv", "cast"]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--S", type=int, default=256)
    ap.add_argument("--n", type=int, default=255)
    ap.add_argument("--warm", type=int, default=-1, help="extrapolation order of the block solves' initial "
                    "guess (warm_start, or warm_start_mixed with --precision 1); default: the library's")
    ap.add_argument("--input", choices=["krylov", "random"], default="krylov")
    ap.add_argument("--fused", type=int, default=1)
    ap.add_argument("--d", type=int, default=2)
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2507_02809_gb300 as t
    from workloads import config_2d, config_3d, random_vector

    w = config_2d(0.3, 1.2, n=args.n, S=args.S) if args.d == 2 else config_3d(n=args.n, S=args.S)
    over = {}
    if args.warm >= 0:
        over["warm_start" if args.precision == 0 else "warm_start_mixed"] = args.warm
    s = t.Solver(w, opts=t.tsfde_default_opts(precision=args.precision, **over,
                                               fused_cg=args.fused))
    if args.input == "random":
        y = torch.as_tensor(random_vector(s.U, 1), device="cuda")
    else:
        zr = torch.zeros(s.U, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(zr)
        y = torch.zeros_like(zr)
        s.rhs(zr)
        s.precond_apply(zr, x)
        s.matvec(x, y)
        y /= torch.linalg.vector_norm(y)
    z = torch.zeros_like(y)
    s.precond_apply(y, z)
    s.profile(2)
    s.precond_apply(y, z)
    st = s.profile_read()
    print("precision %d: application %.2f ms (events), timeline %.2f ms; FP64 block residuals %d, CG steps %d, "
          "guess fallbacks %d (the counters since set-up: two applications)"
          % (args.precision, st["precond_ms"], sum(st["phase_ms"]), st["fp64_block_residuals"],
             st["pcg_iterations"], st["guess_fallbacks"]))
    for i, nm in enumerate(NAMES):
        c = st["phase_count"][i]
        if c:
            print("   %-14s n=%7d  total %8.2f ms  avg %6.2f us" % (nm, c, st["phase_ms"][i],
                                                                   1000.0 * st["phase_ms"][i] / c))
    s.close()


if __name__ == "__main__":
    main()
