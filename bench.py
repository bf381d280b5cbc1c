#!/usr/bin/env python3
"""Benchmark: preconditioned GMRES solve of the all-at-once system on the 255 x 255 grid with
S = 256 time levels (2-D workload; (beta, omega) in {(0.3, 1.2), (0.7, 1.8)}; FP64 GMRES(30)
left-preconditioned by the block triangular preconditioner, tol 1e-10).

One step = one solve of each of the two instances, from x0 = 0, with the inputs resident in
HBM.  Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead
(a bounded sample of the same workload, scaled to the same unit).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun each rank solves its own copy of the two instances (replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES solve time to rel.res 1e-10, FP64 vs mixed/batched; matvec GB/s vs HBM peak"
UNIT = "s/solve"
PAIRS = [(0.3, 1.2), (0.7, 1.8)]
GOLDEN = os.path.join(ROOT, "tests", "golden", "config2_oracle.json")
# ALU peaks from unit counts and the SM clock the bench runs at (2070 MHz, recorded in "clocks"):
# 152 SMs x 2 FP64 FMA lanes (nominal 1.25 TFLOP/s) and x 128 FP32 lanes, 2 FLOPs per FMA; the
# measured-peaks file has no FP64 or non-tensor FP32 figure
SM_COUNT, SM_GHZ = 152, 2.07
FP64_PEAK_TFLOPS = SM_COUNT * 2 * 2 * SM_GHZ / 1e3     # 1.259
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_GHZ / 1e3   # 80.5
# DRAM bytes per launch of the persistent kernel at S = 256, from ncu's dram__bytes_read.sum +
# dram__bytes_write.sum of one launch at S = 16, 32, 64 on the 255 x 255 grid (48.9, 107.7,
# 252.3 MB; profiles/k_fsub_dram_fit_2d_n255.md) fitted as a + b S + c S^2 (the history sums read
# all earlier levels at every 16th level: the S^2 term) and evaluated at S = 256
# ncu DRAM bytes (read + write) of one k_fsub<512> launch at the full size (255 x 255, S = 256), the
# second application of the profiling timeline; one-pass metric set
FSUB_TRAFFIC_BYTES = 1577018368 + 625613312
FSUB_TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_fsub launch at 255 x 255, S = 256 "
                     "(1.58 GB read, 0.63 GB written); the level's working set is L2-resident, DRAM is far "
                     "from the bound")


def _config(n_gpus):
    return {"workload": "2-D fractional inverse source, 255x255 interior grid, S=256 time levels, "
                        "(beta,omega) in {(0.3,1.2),(0.7,1.8)}, alpha=1e-4, 1% noise; "
                        "FP64 GMRES(30), left block-triangular preconditioner, tol 1e-10",
            "grid": [255, 255], "S": 256, "unknowns_per_solve": 257 * 255 * 255,
            "instances_per_step": len(PAIRS),
            "l2": "inputs larger than L2: one vector is 134 MB, the Krylov basis 4.3 GB",
            "parallelism": "replicas" if n_gpus > 1 else "single GPU"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        smax.append(float(parts[2]))
                    except ValueError:
                        continue
                    for nm, v in zip(names, parts[5:9]):
                        if v.lower() == "active":
                            reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------------------
def _oracle_golden():
    """The oracle's own full-size solves of this workload (tests/golden/config2_oracle.json, written by
    tests/golden/make_config2_oracle.py on an x86 host), if present."""
    try:
        with open(GOLDEN) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


class OracleKrylovSample:
    """Bounded timing sample of the FP64 oracle on the (0.3, 1.2) instance of the workload, on the
    vectors its own GMRES works on: from x0 = 0, v_1 = P^-1 z / ||P^-1 z|| (the levels of z are zero
    here, rho = 0, so this first application is cheap and is not timed), then the second
    application's input A v_1.  Timed: one structured matvec (A v_1) and the forward substitution of
    A v_1 through its first `levels` levels (history sums + tau-PCG block solves to 1e-13, the
    oracle's block tolerance).  Scaled to s/solve as
        (t_matvec + (S + 1) t_level) x (preconditioner applications per solve),
    the applications per solve being those of the oracle's own full run (tests/golden), else the GPU
    solves' Arnoldi steps.  Levels late in the substitution carry longer history sums, so the
    per-level time of the first levels slightly underestimates the average."""

    def __init__(self):
        import numpy as np
        from oracle import system as sy
        from workloads import config_2d
        self.sy = sy
        self.p = sy.problem_from(config_2d(*PAIRS[0]))
        _ = self.p.a
        z = sy.rhs(self.p)
        v1 = sy.precond_solve_structured(self.p, z, tol=1e-13)
        self.v1 = v1 / np.linalg.norm(v1)
        self.t_matvec = None
        self.av1 = None

    def time_matvec(self):
        t0 = time.perf_counter()
        self.av1 = self.sy.matvec(self.p, self.v1)
        self.t_matvec = time.perf_counter() - t0
        return self.t_matvec

    def time_levels(self, levels):
        t0 = time.perf_counter()
        self.sy.precond_solve_structured(self.p, self.av1, tol=1e-13, max_levels=levels)
        return (time.perf_counter() - t0) / levels

    def estimate(self, t_level, levels, fallback_iters=None) -> dict:
        import numpy as np
        g = _oracle_golden()
        S = self.p.S
        if g:
            apps = float(np.mean([i["precond_calls"] for i in g["instances"]]))
            src = "preconditioner applications per solve of the oracle's own full run (tests/golden)"
        elif fallback_iters:
            apps = float(np.mean(fallback_iters)) + 1.0
            src = "Arnoldi steps of the GPU solves in this run + 1"
        else:
            apps, src = 1.0, "one application (no count available)"
        per_app = self.t_matvec + (S + 1) * t_level
        out = {"value": per_app * apps, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": ("FP64 oracle on the vectors of its own GMRES from x0 = 0 on the (0.3,1.2) instance: one "
                          "matvec A v_1 (%.2f s) and the forward substitution of A v_1 through its first %d of %d "
                          "levels (%.3f s per level, tau-PCG to 1e-13), scaled as (t_matvec + (S+1) t_level) x %.1f "
                          "%s" % (self.t_matvec, levels, S, t_level, apps, src))}
        if g:
            secs = [i["seconds"] for i in g["instances"]]
            out["oracle_full_solves"] = {
                "seconds": secs, "mean_s_per_solve": float(np.mean(secs)),
                "iters": [i["iters"] for i in g["instances"]],
                "host": g.get("host", {"cpu_count": 8}),
                "note": "the oracle's complete GMRES solves of both instances, timed once on the x86 host "
                        "that wrote tests/golden/config2_oracle.json (not this machine)"}
        return out


E2E_RUNS = 5                 # end-to-end runs (mean and spread reported)
CPU_SAMPLE_LEVELS = 24       # cpu_baseline leg: about 10-20 s of oracle work after its set-up
REF_STEP_LEVELS = 8          # reference arm: levels timed per step


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    smp = OracleKrylovSample()
    smp.time_matvec()
    for _ in range(args.warmup):
        smp.time_levels(REF_STEP_LEVELS)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(smp.estimate(smp.time_levels(REF_STEP_LEVELS), REF_STEP_LEVELS))
    total = time.perf_counter() - t0
    value = statistics.mean(v["value"] for v in vals)
    cpu = dict(vals[-1])
    cpu["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / max(1, args.steps),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args.gpus),
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if "oracle_full_solves" in cpu:
        line["cpu_baseline"]["oracle_full_solves"] = cpu["oracle_full_solves"]
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def max_over_ranks(x: float, dist) -> float:
    """The largest x over all ranks (the whole job takes as long as its slowest rank); x itself
    without a process group.  NCCL reduces on the GPU, gloo on the host."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(elapsed_max: float, steps: int, world: int, instances_per_step: int) -> float:
    """Seconds per solve of the whole job: every rank solves its own copy of the instances each step
    (replicas), and the job lasts as long as its slowest rank."""
    return elapsed_max / (steps * instances_per_step * world)


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1000.0


def _solve_all(solvers, xs):
    res = []
    for s, x in zip(solvers, xs):
        x.zero_()
        res.append(s.solve(x))
    return res


def fp64_right_form(t, loads, xs_fp64, fp64_value):
    """FP64 GMRES(30) right-preconditioned (A P^-1 u = z, y = P^-1 u): it stops on the TRUE relative
    residual 1e-10, like the mixed and batched-mixed forms, so it is the like-for-like FP64 time."""
    import torch
    opts = t.tsfde_default_opts(precision=t.PREC_FP64, side=t.SIDE_RIGHT, restart=30, tol=1e-10)
    solvers = [t.Solver(w, opts=opts) for w in loads]
    xs = [torch.zeros(s.U, dtype=torch.float64, device="cuda") for s in solvers]
    _solve_all(solvers, xs)             # warm-up
    infos, secs = _timed(lambda: _solve_all(solvers, xs))
    N = loads[0].N
    fdiff = [float(torch.linalg.norm(x[-N:] - x64[-N:]) / torch.linalg.norm(x64[-N:]))
             for x, x64 in zip(xs, xs_fp64)]
    for s in solvers:
        s.close()
    return {"value": secs / len(loads), "unit": UNIT, "speedup_vs_fp64": fp64_value / (secs / len(loads)),
            "f_rel_diff_vs_fp64": fdiff, "iters": [i["iters"] for i in infos],
            "relres_true": [i["relres_true"] for i in infos], "converged": [i["converged"] for i in infos],
            "note": "FP64 P^-1 (block solves to 1e-11), right preconditioning, stop on the true residual 1e-10"}


def other_forms(t, loads, xs_fp64, fp64_value):
    """The same instances in mixed precision (FP32 preconditioner inside flexible FP64 GMRES, true
    residual 1e-10) against the FP64 solutions, and the adjoint solve of the gradient workload."""
    import numpy as np
    import torch
    from workloads import config_adjoint_2d
    right = fp64_right_form(t, loads, xs_fp64, fp64_value)
    right_value = right["value"]
    opts = t.tsfde_default_opts(precision=t.PREC_MIXED, side=t.SIDE_FLEXIBLE, restart=30, tol=1e-10)
    solvers = [t.Solver(w, opts=opts) for w in loads]
    xs = [torch.zeros(s.U, dtype=torch.float64, device="cuda") for s in solvers]
    for s, x in zip(solvers, xs):       # warm-up
        x.zero_()
        s.solve(x)

    def run():
        res = []
        for s, x in zip(solvers, xs):
            x.zero_()
            res.append(s.solve(x))
        return res
    infos, secs = _timed(run)
    N = loads[0].N
    fdiff = [float(torch.linalg.norm(x[-N:] - x64[-N:]) / torch.linalg.norm(x64[-N:]))
             for x, x64 in zip(xs, xs_fp64)]
    for s in solvers:
        s.close()
    mixed = {"value": secs / len(loads), "unit": UNIT, "speedup_vs_fp64": fp64_value / (secs / len(loads)),
             "speedup_vs_fp64_right": right_value / (secs / len(loads)),
             "f_rel_diff_vs_fp64": fdiff, "iters": [i["iters"] for i in infos],
             "relres_true": [i["relres_true"] for i in infos],
             "precond_failures": [i["precond_failures"] for i in infos],
             "note": "FP32 tau-PCG block solves (tol 1e-5) inside flexible FP64 GMRES(30), stop on the "
                     "true residual 1e-10; FP64 Arnoldi, Givens and true-residual matvec"}

    w = config_adjoint_2d()
    s = t.Solver(w)
    y = torch.zeros(s.U, dtype=torch.float64, device="cuda")
    ft = torch.as_tensor(w.f_true, device="cuda")
    ybar = torch.zeros_like(y)
    dmu = torch.empty(s.N, dtype=torch.float64, device="cuda")
    dg2 = torch.empty(s.S * s.N, dtype=torch.float64, device="cuda")

    def fwd():
        y.zero_()
        return s.solve(y)

    def adj():
        ybar[-s.N:] = y[-s.N:] - ft
        return s.adjoint(y, ybar, None, dmu, dg2)
    fwd()
    adj()                               # warm-up
    finfo, fsec = _timed(fwd)
    ainfo, asec = _timed(adj)
    s.close()
    adjoint = {"workload": "127x127, S=128, beta=0.5, omega=1.5, alpha=1e-4, J = 1/2 ||f - sin(pi x) sin(pi y)||^2",
               "forward_s": fsec, "adjoint_s": asec, "forward_iters": finfo["iters"],
               "adjoint_iters": ainfo["iters"], "adjoint_relres_true": ainfo["relres_true"],
               "dJ_dalpha": ainfo["dalpha"],
               "note": "adjoint = A^T lam = [0; f - f_true] by GMRES(30) with P^T (backward substitution) "
                       "plus the gradients wrt alpha, mu and gamma2, all on the GPU"}
    # batched: both instances in lockstep, every preconditioner application of the solves still
    # running shares one launch (one sub-grid per instance)
    batched = {}
    for name, bopts in (("fp64", t.tsfde_default_opts(precision=t.PREC_FP64, side=t.SIDE_LEFT, restart=30, tol=1e-10)),
                        ("mixed", opts)):
        bs = [t.Solver(w, opts=bopts) for w in loads]
        bx = [torch.zeros(s.U, dtype=torch.float64, device="cuda") for s in bs]

        def brun():
            for x in bx:
                x.zero_()
            return t.tsfde_gmres_solve_batch([s.handle for s in bs], bx)
        brun()                          # warm-up
        binfos, bsecs = _timed(brun)
        bdiff = [float(torch.linalg.norm(x[-N:] - x64[-N:]) / torch.linalg.norm(x64[-N:]))
                 for x, x64 in zip(bx, xs_fp64)]
        for s in bs:
            s.close()
        batched[name] = {"value": bsecs / len(loads), "unit": UNIT,
                         "speedup_vs_fp64": fp64_value / (bsecs / len(loads)),
                         "speedup_vs_fp64_right": right_value / (bsecs / len(loads)),
                         "f_rel_diff_vs_fp64": bdiff, "iters": [i["iters"] for i in binfos],
                         "relres_true": [i["relres_true"] for i in binfos]}
    batched["note"] = ("tsfde_gmres_solve_batch: the instances' GMRES run in lockstep and each preconditioner "
                       "application of the solves still running shares one launch of the persistent kernel "
                       "(one sub-grid of CTAs per instance)")
    # T_{n,S} and S_{n,S} of Remark 1: tau(B_n) or the Strang circulant s(B_n) in every diagonal block,
    # one sine-transform (tau) or Fourier (Strang) solve per block
    block_forms = {}
    for key, bsolver in (("tau", t.BLOCK_TAU), ("strang", t.BLOCK_STRANG)):
        form = {}
        for name, topts in (("fp64", t.tsfde_default_opts(precision=t.PREC_FP64, side=t.SIDE_LEFT, restart=30,
                                                          tol=1e-10, block_solver=bsolver)),
                            ("mixed", t.tsfde_default_opts(precision=t.PREC_MIXED, side=t.SIDE_FLEXIBLE,
                                                           restart=30, tol=1e-10, block_solver=bsolver))):
            ts = [t.Solver(w, opts=topts) for w in loads]
            tx = [torch.zeros(s.U, dtype=torch.float64, device="cuda") for s in ts]

            def trun():
                res = []
                for s, x in zip(ts, tx):
                    x.zero_()
                    res.append(s.solve(x))
                return res
            trun()                          # warm-up
            tinfos, tsecs = _timed(trun)
            tdiff = [float(torch.linalg.norm(x[-N:] - x64[-N:]) / torch.linalg.norm(x64[-N:]))
                     for x, x64 in zip(tx, xs_fp64)]
            for s in ts:
                s.close()
            form[name] = {"value": tsecs / len(loads), "unit": UNIT,
                          "speedup_vs_fp64": fp64_value / (tsecs / len(loads)),
                          "f_rel_diff_vs_fp64": tdiff, "iters": [i["iters"] for i in tinfos],
                          "relres_true": [i["relres_true"] for i in tinfos],
                          "converged": [i["converged"] for i in tinfos]}
        block_forms[key] = form
    tau, strang = block_forms["tau"], block_forms["strang"]
    tau["note"] = ("block_solver = 1: T_{n,S} (B_n -> tau(B_n) in P, Remark 1), the variable diagonal by its "
                   "level mean; more GMRES steps, each preconditioner application one sine-transform solve per level")
    strang["note"] = ("block_solver = 2: S_{n,S} (B_n -> Strang circulant s(B_n) in P, Remark 1), the variable "
                      "diagonal by its level mean; each block one Fourier solve with length-n DFTs (Bluestein "
                      "chirp-z on the length-L FFTs); Remark 1 expects more GMRES steps than with T_{n,S}")
    return {"fp64_right": right, "mixed": mixed, "batched": batched, "tau": tau, "strang": strang,
            "adjoint": adjoint, "cfg3": cfg3_form(t), "batch64": batch64_form()}


def cfg3_form(t):
    """The 3-D workload (63^3 interior grid, S = 256, 64.3 M unknowns): FP64 right-preconditioned
    GMRES(30) and the mixed form (FP32 preconditioner in flexible FP64 GMRES(30)), both to the true
    relative residual 1e-10; one solve each after a warm-up preconditioner application."""
    import torch
    from workloads import config_3d
    w = config_3d()
    out = {"workload": "3-D 63x63x63, S=256, beta=0.6, omega=1.6, alpha=1e-4, 0.5% noise", "unknowns": w.U}
    x64 = None
    for name, o in (("fp64_right", t.tsfde_default_opts(precision=t.PREC_FP64, side=t.SIDE_RIGHT, tol=1e-10)),
                    ("mixed", t.tsfde_default_opts(precision=t.PREC_MIXED, side=t.SIDE_FLEXIBLE, tol=1e-10))):
        s = t.Solver(w, opts=o)
        x = torch.zeros(s.U, dtype=torch.float64, device="cuda")
        r = torch.zeros_like(x)
        s.rhs(r)
        s.precond_apply(r, x)           # warm-up
        x.zero_()
        info, secs = _timed(lambda: s.solve(x))
        out[name] = {"value": secs, "unit": "s/solve", "iters": info["iters"], "relres_true": info["relres_true"],
                     "converged": info["converged"]}
        N = s.N
        if x64 is None:
            x64 = x.clone()
        else:
            out[name]["f_rel_diff_vs_fp64"] = float(torch.linalg.norm(x[-N:] - x64[-N:]) / torch.linalg.norm(x64[-N:]))
            out[name]["speedup_vs_fp64"] = out["fp64_right"]["value"] / secs
        s.close()
        del x, r
    del x64
    torch.cuda.empty_cache()
    return out


def batch64_form():
    """The batched workload: 64 seeded instances of uneven sizes and parameters (32 one-dimensional,
    n 127..2047, S 64..512; 32 two-dimensional, n^2 with n 63..255, S 64..256), mixed precision, all
    solved by one tsfde_gmres_solve_batch call (every preconditioner round one launch of the
    mixed-length kernel, replayed from a captured CUDA graph), then every instance alone."""
    from paper_2507_02809_gb300 import batch_study
    res = batch_study.run("mixed", sequential=True)
    keep = ("instances", "unknowns", "launch", "batched_s", "sequential_s", "speedup", "all_converged")
    out = {k: res[k] for k in keep if k in res}
    out["groups"] = [{k: g[k] for k in ("d", "L", "count", "batched_s", "sequential_s", "max_relres_true",
                                        "max_rel_diff_batched_vs_single") if k in g} for g in res["groups"]]
    out["unit"] = "s (whole workload)"
    return out


def run_gb300(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2507_02809_gb300 import build as _build
    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    import paper_2507_02809_gb300 as t
    from workloads import config_2d

    opts = t.tsfde_default_opts(precision=t.PREC_FP64, side=t.SIDE_LEFT, restart=30, tol=1e-10)
    loads = [config_2d(b, o) for (b, o) in PAIRS]
    solvers = [t.Solver(w, opts=opts) for w in loads]
    xs = [torch.zeros(s.U, dtype=torch.float64, device="cuda") for s in solvers]
    infos = []

    def step(record):
        for s, x in zip(solvers, xs):
            x.zero_()
            info = s.solve(x)
            if record:
                infos.append(info)

    for _ in range(args.warmup):
        step(False)
    for s in solvers:
        s.profile(True)
    launches0 = sum(s.profile_read()["launches"] for s in solvers)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step(True)
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1000.0
    if dist is not None:
        elapsed = max_over_ranks(elapsed, dist)
    stats = [s.profile_read() for s in solvers]
    launches = sum(st["launches"] for st in stats) - launches0
    value = whole_job_value(elapsed, args.steps, world, len(PAIRS))

    # roofline of the dominant kernel: the persistent forward substitution (one cooperative launch
    # per preconditioner application), timed by CUDA events on the stream it runs on
    pc_ms = sum(st["precond_ms"] for st in stats)
    pc_n = sum(st["precond_count"] for st in stats)
    mv_ms = sum(st["matvec_ms"] for st in stats)
    mv_n = sum(st["matvec_count"] for st in stats)
    st0 = stats[0]
    S, N = 256, 255 * 255
    res64 = sum(st["fp64_block_residuals"] for st in stats)
    pcg32 = sum(st["pcg_iterations"] for st in stats)
    # work executed per launch: FP64 block residuals (one B_n apply each) and the history sums
    # in FP64, FP32 CG steps (one B_n apply and one tau solve each), averaged over the launches
    # since set-up (warm-up solves included: the counters are cumulative)
    apps_total = max(1, sum(st["precond_apps_total"] for st in stats))
    f64_per_app = (res64 / apps_total) * st0["flops_bapply"] + N * S * (S - 1)
    f32_per_app = (pcg32 / apps_total) * (st0["flops_bapply"] + st0["flops_tau"])
    app_ms = pc_ms / max(1, pc_n)
    # FP64-equivalent FLOPs: an FP32 FLOP costs peak64 / peak32 of an FP64 FLOP
    feq = f64_per_app + f32_per_app * (FP64_PEAK_TFLOPS / FP32_PEAK_TFLOPS)
    achieved = feq / (app_ms / 1000.0) / 1e12
    roof = {"kernel": "k_fsub<512>: persistent forward substitution (one launch per preconditioner application)",
            "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": FSUB_TRAFFIC_BYTES, "traffic_note": FSUB_TRAFFIC_NOTE,
            "ms_per_launch": app_ms, "launches": pc_n, "time_share": pc_ms / 1000.0 / elapsed,
            "fp64_gflop_per_launch": f64_per_app / 1e9, "fp32_gflop_per_launch": f32_per_app / 1e9,
            "peak_note": "FP64 peak from unit counts: 152 SMs x 2 FMA lanes x 2 FLOPs x 2.07 GHz = 1.26 TFLOP/s "
                         "(1.19 measured by an FMA probe); FP32 work weighted by the lane ratio 1/64; the kernel is "
                         "bound by the latency of its grid-synchronised passes"}
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    mv_avg = mv_ms / max(1, mv_n)
    matvec = {"ms_per_launch": mv_avg, "launches": mv_n, "time_share": mv_ms / 1000.0 / elapsed,
              "gbs": st0["bytes_matvec"] / (mv_avg / 1000.0) / 1e9, "hbm_peak_gbs": hbm,
              "frac_hbm": st0["bytes_matvec"] / (mv_avg / 1000.0) / 1e9 / hbm,
              "tflops_fp64": ((S + 1) * st0["flops_bapply"] + st0["flops_timesum"]) / (mv_avg / 1000.0) / 1e12}
    # the HBM-bound kernels: CGS2 orthogonalisation of each Arnoldi step (two k_multidot and two
    # k_multiaxpy launches), algorithmic bytes 16 U (2k + 3) for k basis vectors over their event time
    or_ms = sum(st["orth_ms"] for st in stats)
    or_n = sum(st["orth_count"] for st in stats)
    or_b = sum(st["orth_bytes"] for st in stats)
    or_gbs = or_b / max(1e-9, or_ms / 1000.0) / 1e9
    arnoldi = {"ms_per_step": or_ms / max(1, or_n), "steps": or_n, "time_share": or_ms / 1000.0 / elapsed,
               "gbs": or_gbs, "hbm_peak_gbs": hbm, "frac_hbm": or_gbs / hbm,
               "note": "CGS2 of the Arnoldi steps (multidot + multiaxpy, twice), 16 U (2k + 3) bytes for k "
                       "basis vectors, CUDA events on the handle's stream"}

    if args.no_forms:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
                              "higher_is_better": False, "note": "profiling variant (--no-forms)",
                              "roofline": roof, "matvec": matvec, "arnoldi": arnoldi, "clocks": clk,
                              "gpu_launches": launches,
                              "solves": [{"iters": i["iters"], "relres_true": i["relres_true"],
                                          "precond_failures": i["precond_failures"]} for i in infos[: len(PAIRS)]],
                              "guess_fallbacks": [st["guess_fallbacks"] for st in stats]}), flush=True)
        for s in solvers:
            s.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # end to end through the C ABI with pinned host buffers: setup (H2D of the inputs), solve,
    # D2H of the solution, destroy
    e2e_vals = []
    h2d = d2h = 0
    host = []
    for w in loads:
        arrs = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).pin_memory()
                for a in (w.gamma1, w.gamma2, w.q, w.rho, w.mu)]
        yh = torch.zeros(w.U, dtype=torch.float64).pin_memory()
        host.append((w, arrs, yh))
    for _ in range(E2E_RUNS):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (w, arrs, yh) in host:
            yh.zero_()
            h = t.tsfde_setup(2, 255, 1.0, 256, 1.0, w.beta, w.omega, w.alpha, *arrs, opts=opts)
            t.tsfde_gmres_solve(h, yh)
            t.tsfde_destroy(h)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist is not None:
            dt = max_over_ranks(dt, dist)
        e2e_vals.append(dt / (len(host) * world))
    for (w, arrs, yh) in host:
        h2d += sum(a.numel() * 8 for a in arrs)
        d2h += yh.numel() * 8

    forms = other_forms(t, loads, xs, value)

    if rank != 0:
        return 0
    smp = OracleKrylovSample()
    smp.time_matvec()
    cpu = smp.estimate(smp.time_levels(CPU_SAMPLE_LEVELS), CPU_SAMPLE_LEVELS, [i["iters"] for i in infos[: len(PAIRS)]])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(world), "clocks": clk,
            "e2e": {"value": statistics.mean(e2e_vals), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "runs": len(e2e_vals), "min": min(e2e_vals), "max": max(e2e_vals),
                    "stdev": statistics.stdev(e2e_vals) if len(e2e_vals) > 1 else 0.0},
            "gpu_launches": launches, "roofline": roof, "matvec": matvec, "arnoldi": arnoldi, "forms": forms,
            "solves": [{"beta": b, "omega": o, "iters": i["iters"], "relres_est": i["relres_est"],
                        "relres_true": i["relres_true"], "precond_failures": i["precond_failures"]}
                       for (b, o), i in zip(PAIRS, infos[: len(PAIRS)])],
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "oracle_full_solves")
                             if k in cpu}}
    print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-forms", action="store_true",
                    help="profiling variant: the timed steps only (no other forms, end-to-end runs or CPU baseline)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
