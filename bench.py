#!/usr/bin/env python
"""Factor + refined-solve benchmark of the GB300 H^2-ULV solver.

Metric: seconds for h2_factor + h2_solve to reach a relative residual
||b - A_H2 x|| / ||b|| <= 1e-10 at N = 2^18 (points uniform in the unit cube,
Yukawa kernel exp(-r)/(r+1e-3) with diagonal + 1, leaf 256, eta 1), mixed
precision (FP16 contractions + FP64 refinement) against the plain FP64
factorization on the same instance, one GB300.

One step = one full factorization (all levels) + one refined solve, with the
H^2 instance (h2_build, not timed) resident in HBM.  Inputs (13 GB of FP64
leaf blocks, ~30 GB of factors) are far larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own replica of the problem
("replicas only": the method has no data-path exchange on one system).
--impl reference times the FP64 CPU oracle per step on a smaller instance of
the same workload (--ref-n points, reported unscaled with that N), on the
host cores; --impl reference --ref-n 262144 --steps 1 --warmup 0 times it at
the full size.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "factor+solve s at N=2^18 to 1e-10 residual: mixed-prec vs FP64 H²-ULV, 1 GB300"
UNIT = "s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube262144_yukawa")
    ap.add_argument("--prec", default="fp16", choices=["fp16", "bf16", "fp64"])
    ap.add_argument("--target", type=float, default=1e-10)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-n", type=int, default=32768,
                    help="points of the oracle run timed for cpu_baseline (scaled to the workload's N)")
    ap.add_argument("--ref-n", type=int, default=8192,
                    help="points of the oracle run timed per step by --impl reference (not scaled)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rr-lu", default="fp32", choices=["fp64", "fp32"],
                    help="arithmetic of the LU / inverse of Ahat_ii^RR in FP16/BF16 factorizations")
    ap.add_argument("--residual", default="pair", choices=["pair", "fp64"],
                    help="arithmetic of the mixed refinement's residual: FP32 pairs or FP64 instructions")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of the single-system step: a batch of this many Gaussian-covariance systems of "
                         "uneven size (workloads.batch_systems), factored and solved concurrently")
    ap.add_argument("--batch-max-iters", type=int, default=600)
    ap.add_argument("--batch-mode", choices=["forest", "pool"], default="forest")
    ap.add_argument("--batch-leaf", type=int, default=0,
                    help="leaf size of every batch system (0: 128 below N = 16384, else 256)")
    ap.add_argument("--batch-near-samples", type=int, default=0)
    ap.add_argument("--batch-shift", type=float, default=None,
                    help="diagonal shift of the batch systems (default: the workload's)")
    ap.add_argument("--rank-study", action="store_true",
                    help="instead of the step: the learned rank predictor against the plain build at N = 2^20")
    ap.add_argument("--dense-rows", type=int, default=4096,
                    help="rows sampled for the check against the dense matrix after the timed region (0: none)")
    ap.add_argument("--build", default="plain", choices=["plain", "gpu"],
                    help="construction of the instance (untimed): the host rank-revealing pass, or the GPU "
                         "sketches at the level caps (h2_build_gpu)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="before the timed steps, h2_autotune picks the GEMM form and the substitution's launch "
                         "shapes on this instance (overrides --tc-kernel, --graphs, --box-stream)")
    ap.add_argument("--box-stream", type=int, default=0, choices=[0, 1],
                    help="substitution per-box steps on large levels: 1 streamed persistent kernels, 0 row-split")
    ap.add_argument("--tc-kernel", type=int, default=2, choices=[0, 1, 2],
                    help="tensor-core GEMM form: 0 one CTA per entry, 1 persistent grid, 2 warp-specialized")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay the FP32 substitution as a CUDA graph (1) or launch it kernel by kernel (0)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- oracle arm ---
def oracle_instance(wl, n_sample: int):
    """The FP64 oracle's H^2 instance of the workload at n_sample points (the
    same geometry, kernel, leaf, eta and tolerance), with its right-hand side.
    Construction is not timed (h2_build is not timed on the GPU side either)."""
    import dataclasses

    from oracle.construct import construct
    from oracle.kernels import Kernel
    ws = dataclasses.replace(wl, n=n_sample)
    P = ws.points()
    b = ws.rhs()
    H = construct(P, Kernel(wl.kernel, eps=wl.eps, ell=wl.ell, diag_shift=wl.diag_shift), wl.leaf, wl.eta, wl.tol,
                  wl.max_rank, wl.far_samples, wl.near_samples)
    return H, b


def oracle_step(H, b, target: float):
    """One timed oracle step: factorization plus FGMRES refinement to target.
    Returns (seconds, residual history)."""
    from oracle import ulv
    t0 = time.perf_counter()
    F = ulv.factor(H)
    x, hist, _ = ulv.refine_gmres(F, H, b, target, 200, 30)
    return time.perf_counter() - t0, hist


def threads_used() -> int:
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count() or 1


def run_reference(args, wl):
    """--impl reference: the FP64 CPU oracle on the host cores, each step one
    factorization plus refinement of the same workload at --ref-n points (the
    instance is built once, untimed).  The value is the measured seconds per
    step at that N, unscaled; config.N says which N ran."""
    n = min(args.ref_n, wl.n)
    H, b = oracle_instance(wl, n)
    steps, hist = [], None
    for k in range(args.warmup + args.steps):
        dt, hist = oracle_step(H, b, args.target)
        if k >= args.warmup:
            steps.append(dt)
    value = float(np.mean(steps))
    sample = (f"oracle factor + FGMRES refinement to {args.target:g} at N={n} (same kernel, leaf, eta, tol, "
              f"geometry as {wl.name}), measured per step, not scaled")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "N": n, "N_workload": wl.n, "kernel": wl.kernel, "leaf": wl.leaf,
                       "eta": wl.eta, "tol": wl.tol, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "refinement_history": hist}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm ---
PHASES = ("a1_qr", "a2_proj", "a3_lu", "a45_schur", "a2c_coupling", "a6_merge", "a7_root")
SOLVE_PHASES = ("solve_subst", "solve_matvec", "solve_matvec32")


def fp64_peak_tflops() -> float:
    """FP64 dense GEMM rate measured now (torch.matmul 4096^3, best of 3)."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn_like(a)
    a @ b
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


# DRAM traffic of one launch of the FP32 matvec's leaf kernel (the step's
# largest kernel: the symmetric-storage pair kernel), valid while the
# kernel's source is the one captured (digest of its text below).  Captured
# on the small case cube32768_yukawa (1323 stored pairs: 347.00 MB read +
# 4.45 MB written in one launch) and scaled to the 12875 stored pairs of
# cube262144_yukawa: the kernel reads each stored 256 x 256 block once, so
# its traffic grows with the stored pairs.
LEAF_TRAFFIC = {"digest": "1381b342a0b471df", "bytes_per_launch": (347.004160e6 + 4.454144e6) * 12875 / 1323,
                "profile": "profiles/mv_sym_pair_kernel_cube262144_yukawa.md"}


def leaf_kernel_digest() -> str:
    src = open(os.path.join(ROOT, "paper_2502_02395_gb300", "csrc", "kernels_solve.cu")).read()
    a = src.index("// -------------------------------------------- symmetric leaf near blocks ---")
    b = src.index("// y_i = X_i yh_i + sum of box i's partial products")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def kernel_roofline(stats, t_leaf, n_leaf, peaks):
    """Roofline of the FP32 leaf matvec kernel: algorithmic bytes per launch
    / its average CUDA-event duration inside the timed steps."""
    if n_leaf <= 0 or t_leaf <= 0:
        return None
    per = t_leaf / n_leaf
    by = stats["bytes_matvec32_leaf"]
    ach = by / per / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    if LEAF_TRAFFIC and LEAF_TRAFFIC.get("digest") == leaf_kernel_digest():
        traffic = LEAF_TRAFFIC["bytes_per_launch"]
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
            "kernel": stats.get("leaf_kernel", "mv_leaf_kernel<float>"), "launches_per_step": n_leaf,
            "bytes_per_launch": by,
            "ms_per_launch": per * 1e3,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}


def roofline_for(phase, stats, t_phase, calls, peaks, prec, tc, fp64_tf):
    """Roofline of one phase: algorithmic flops or bytes / CUDA-event time."""
    if t_phase <= 0:
        return None
    if phase == "solve_subst":
        achieved = stats["bytes_subst"] * calls["subst"] / t_phase / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "phase": phase, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    if phase == "solve_matvec32":
        gbs = stats["bytes_matvec32"] * calls["matvec32"] / t_phase / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "traffic": None, "phase": phase, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    if phase == "solve_matvec" and prec != "fp64":
        # the mixed refinement's residual: FP32-pair arithmetic on the FP32
        # split of the FP64 matrix, 8 bytes per entry read
        gbs = stats["bytes_matvec"] * calls["matvec"] / t_phase / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "traffic": None, "phase": phase, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    if phase == "solve_matvec":
        # FP64 multiply-adds on the leaf near blocks: the FP64 ALU rate binds
        # before HBM on this part (2 flops per 8-byte entry)
        flops = stats["flops_matvec"] * calls["matvec"] / t_phase / 1e12
        gbs = stats["bytes_matvec"] * calls["matvec"] / t_phase / 1e9
        return {"bound": "alu", "achieved": flops, "peak": fp64_tf, "unit": "TFLOP/s", "frac": flops / fp64_tf,
                "traffic": None, "phase": phase, "hbm_gbs": gbs, "hbm_frac": gbs / peaks.get("hbm_gbs", 6800.0),
                "peak_source": "FP64 peak measured live (torch.matmul float64 4096^3)"}
    fl = stats["flops"]
    if phase not in fl:
        return None
    achieved = fl[phase] / t_phase / 1e12
    if phase == "a2_proj" and tc:
        bound, peak, src = "tensor", peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops"), \
            "measured bf16 sustained (FP16 runs at the same dense rate)"
        # at K = 256 the projection GEMMs are memory-bound: also against HBM,
        # from the phase's algorithmic bytes (16-bit inputs and bases read
        # once, outputs written once)
        if stats.get("bytes_proj"):
            gbs = stats["bytes_proj"] / t_phase / 1e9
            return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None, "phase": phase, "peak_source": src, "hbm_gbs": gbs,
                    "hbm_frac": gbs / peaks.get("hbm_gbs", 6800.0)}
    elif prec == "fp64":
        bound, peak, src = "alu", fp64_tf, "FP64 peak measured live"
    else:
        bound = "alu"
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        src = "derived: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "phase": phase, "peak_source": src}


def run_batch(args):
    """--batch S: S independent Gaussian-covariance systems (N log-uniform
    in [4096, 65536], l in [0.05, 0.5], + I on the diagonal, tol 1e-8),
    factorizations in --prec refined to --target, one JSON line.
    Leaf size --batch-leaf (default 128 below N = 16384, else 256).
    --batch-mode forest (default): the systems grouped by (leaf, tree
    depth), each group one instance whose levels are single launches over
    its systems (points divided by l, l = 1; the FP64 leaf blocks released
    after each group is built, so that the padded forests fit); pool: one
    instance per system.  Close-field
    samples --batch-near-samples (0: every point of each close box; with 64
    the pre-factorization basis misses the Gaussian's fill-ins and the
    refinement stalls).  The library's worker pool runs the groups or
    systems with the worker count its tuner picks."""
    import torch
    import workloads as W
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import H2Solver
    from paper_2502_02395_gb300.binding import H2Batch
    specs = W.batch_systems(count=args.batch)
    if args.batch_shift is not None:
        for sp in specs:
            sp["shift"] = args.batch_shift
    t0 = time.perf_counter()
    solvers, rhs = [], []
    forest = args.batch_mode == "forest"
    if forest:
        shift = specs[0]["shift"]
        leaves = [args.batch_leaf or sp["leaf"] for sp in specs]
        batch = H2Batch.forest([W.cube_points(sp["n"], sp["point_seed"]) / sp["ell"] for sp in specs], leaves,
                               kernel="gaussian", ell=1.0, diag_shift=shift, leaf=256, eta=1.0,
                               tol=1e-8, far_samples=1024, near_samples=args.batch_near_samples)
        rhs = [W.uniform_rhs(sp["n"], sp["rhs_seed"]) for sp in specs]
    else:
        for sp in specs:
            P = W.cube_points(sp["n"], sp["point_seed"])
            solvers.append(H2Solver.build(P, kernel="gaussian", ell=sp["ell"], diag_shift=sp["shift"], leaf=args.batch_leaf or sp["leaf"],
                                          eta=1.0, tol=1e-8, far_samples=1024, near_samples=args.batch_near_samples))
            rhs.append(torch.from_numpy(W.uniform_rhs(sp["n"], sp["rhs_seed"])).cuda())
        batch = H2Batch(solvers)
    build_s = time.perf_counter() - t0
    workers = batch.tune(args.prec, rhs, target=args.target, max_iters=args.batch_max_iters, check=False)
    tune = batch.stats()["tune_seconds"]
    times, its_all, rel_all = [], None, None
    for k in range(args.warmup + args.steps):
        _, rel, its, sec = batch.run(args.prec, rhs, target=args.target, max_iters=args.batch_max_iters, check=False)
        if k >= args.warmup:
            times.append(sec)
            its_all, rel_all = its, rel
    value = float(np.mean(times))
    line = {"metric": f"factor+solve s for {args.batch} independent Gaussian-covariance systems to {args.target:g}",
            "value": value, "unit": "s", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
            "workers": workers, "tune_seconds_by_workers": tune, "sequential_s": tune.get("1"),
            "speedup_vs_one_worker": (tune.get("1") / value) if tune.get("1") else None,
            "mode": args.batch_mode, "groups": batch.stats().get("group_systems"),
            "leaf": args.batch_leaf or "128 below N = 16384, else 256", "near_samples": args.batch_near_samples,
            "diag_shift": specs[0]["shift"],
            "total_N": int(sum(s["n"] for s in specs)), "N": [s["n"] for s in specs],
            "iters": its_all, "converged": int(sum(r <= args.target for r in rel_all)),
            "relres_max": float(max(rel_all)), "build_s": build_s, "dtype": {"fp16": "f16/f32/f64", "bf16": "bf16/f32/f64"}.get(
                args.prec, "f64"), "data": "synthetic"}
    print(json.dumps(line), flush=True)
    batch.close()
    for S in solvers:
        S.close()


def kernel_rows_torch(wl, P, rows, cols):
    """Exact entries G(P[rows], P[cols]) of the workload's kernel (FP64, on
    the GPU), the diagonal where a row meets its own point."""
    import torch
    X = torch.from_numpy(P[rows]).cuda()
    Y = torch.from_numpy(P[cols]).cuda()
    r = torch.cdist(X, Y).double()
    same = torch.from_numpy(rows).cuda()[:, None] == torch.from_numpy(cols).cuda()[None, :]
    if wl.kernel == "laplace_eps":
        G, d = 1.0 / (r + wl.eps), 1.0 / wl.eps + wl.diag_shift
    elif wl.kernel == "yukawa_eps":
        G, d = torch.exp(-r) / (r + wl.eps), 1.0 / wl.eps + wl.diag_shift
    else:
        return None
    return torch.where(same, torch.full_like(G, d), G)


def dense_rows_check(wl, P, b, x, S, rows=4096, chunk=16384):
    """Accuracy against the dense matrix on sampled rows: the residual
    ||(A x - b)[rows]|| / ||b[rows]|| of the refined solution and the H^2
    approximation error ||(A_H2 x - A x)[rows]|| / ||(A x)[rows]||, with the
    kernel entries of those rows evaluated exactly (all rows when N <= rows)."""
    import torch
    if rows <= 0:
        return None
    n = len(P)
    rng = np.random.default_rng(11)
    sel = np.arange(n) if n <= rows else np.sort(rng.choice(n, rows, replace=False))
    Ax = torch.zeros(len(sel), dtype=torch.float64, device="cuda")
    xd = torch.from_numpy(x).cuda()
    for c0 in range(0, n, chunk):
        cols = np.arange(c0, min(n, c0 + chunk))
        G = kernel_rows_torch(wl, P, sel, cols)
        if G is None:
            return None
        Ax += G @ xd[c0:c0 + len(cols)]
    Ax = Ax.cpu().numpy()
    h2x = S.matvec(x)[sel]
    return {"rows": int(len(sel)), "relres_dense": float(np.linalg.norm(Ax - b[sel]) / np.linalg.norm(b[sel])),
            "h2_vs_dense": float(np.linalg.norm(h2x - Ax) / np.linalg.norm(Ax))}


def run_rank_study(args):
    """--rank-study: the learned rank predictor at N = 2^20
    (cube1048576_laplace: 1/(r+1e-3), leaf 256, eta 1, tol 1e-8).  The model
    is trained on the GPU on the plain compression's ranks of the solver
    workloads (workloads.rank_training_sets); then the same problem is built
    twice, by the plain rank-revealing host construction and by the
    predicted layout with GPU sketches (h2_build_gpu with the model), and
    each instance is factored (--prec) and solved to 1e-10.  Reported per
    build: construction seconds, per-level ranks, fallbacks, the refined
    solve's time and steps, and the H^2 approximation error on 1024 exactly
    evaluated rows.  One JSON line."""
    import torch
    import workloads as W
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding as B
    wl = W.workload("cube1048576_laplace")
    P, b = wl.points(), wl.rhs()
    kw = dict(kernel=wl.kernel, leaf=wl.leaf, eta=wl.eta, tol=wl.tol, far_samples=wl.far_samples,
              near_samples=wl.near_samples)
    t0 = time.perf_counter()
    F, Y = [], []
    for pts, k2 in W.rank_training_sets():
        f, y, _ = B.h2_rank_data(B.make_params(**k2), pts)
        F.append(f)
        Y.append(y)
    F, Y = np.concatenate(F), np.concatenate(Y)
    data_s = time.perf_counter() - t0
    m = B.h2_rank_model_create(7)
    loss0 = float(np.mean((B.h2_rank_model_predict(m, F) - Y) ** 2))
    t0 = time.perf_counter()
    loss = B.h2_rank_model_train(m, F, Y, steps=1500, lr=3e-3)
    train_s = time.perf_counter() - t0

    def measure(S, build_s):
        st = S.stats()
        c = st.get("construction", {})
        S.factor(args.prec)
        torch.cuda.synchronize()
        t = time.perf_counter()
        x, rel, its = S.solve(b, target=1e-10, max_iters=200)
        torch.cuda.synchronize()
        step = time.perf_counter() - t
        chk = dense_rows_check(wl, P, b, x, S, rows=1024)
        return {"build_s": build_s, "compress_s": c.get("compress_s"), "K": [lv["K"] for lv in st["levels"]],
                "fallback_boxes": c.get("fallback_boxes"), "fallback_levels": c.get("fallback_levels"),
                "gpu_levels": c.get("gpu_levels"), "solve_s": step, "relres": rel, "iters": its,
                "h2_vs_dense_rows": chk["h2_vs_dense"] if chk else None}

    t0 = time.perf_counter()
    S = B.H2Solver.build(P, **kw)
    plain = measure(S, time.perf_counter() - t0)
    S.close()
    t0 = time.perf_counter()
    S = B.H2Solver.build_gpu(P, m, 0, **kw)
    pred = measure(S, time.perf_counter() - t0)
    S.close()
    B.h2_rank_model_destroy(m)
    line = {"metric": "H2 construction at N=2^20: learned-rank GPU build vs plain rank-revealing build",
            "workload": wl.name, "N": wl.n, "prec": args.prec, "data": "synthetic",
            "training": {"samples": int(len(Y)), "data_s": data_s, "train_s": train_s, "loss0": loss0, "loss": loss,
                         "steps": 1500},
            "plain": plain, "predicted_gpu": pred,
            "build_speedup": plain["build_s"] / pred["build_s"] if pred["build_s"] else None}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.batch > 0:
        run_batch(args)
        return
    if args.rank_study:
        run_rank_study(args)
        return
    import workloads as W
    wl = W.workload(args.workload)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        from paper_2502_02395_gb300 import build as bld
        bld.build()
    if world > 1:
        dist.barrier()
    from paper_2502_02395_gb300 import H2Solver, h2_solve

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}

    P = wl.points()
    b = wl.rhs()
    t0 = time.perf_counter()
    kw = dict(kernel=wl.kernel, leaf=wl.leaf, eta=wl.eta, tol=wl.tol, max_rank=wl.max_rank,
              far_samples=wl.far_samples, near_samples=wl.near_samples, eps=wl.eps, ell=wl.ell,
              diag_shift=wl.diag_shift)
    S = H2Solver.build(P, **kw) if args.build == "plain" else H2Solver.build_gpu(P, None, 0, **kw)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    S.set_stream(stream)
    S.set_option("rr_lu_fp64", 1 if args.rr_lu == "fp64" else 0)
    S.set_option("residual_fp64", 1 if args.residual == "fp64" else 0)
    S.set_option("graphs", args.graphs)
    S.set_option("tc_kernel", args.tc_kernel)
    S.set_option("box_stream", args.box_stream)
    tuned = None
    if args.autotune and args.prec != "fp64":
        # kernel forms and launch shapes measured on this instance (untimed)
        tuned = S.autotune(args.prec)
        args.tc_kernel, args.graphs, args.box_stream = tuned["tc_kernel"], tuned["graphs"], tuned["box_stream"]
    b_dev = torch.from_numpy(b).cuda()
    x_dev = torch.zeros_like(b_dev)
    torch.cuda.synchronize()

    def step(prec):
        S.factor(prec)
        st, rel, its = h2_solve(S.ctx, b_dev, x_dev, args.target, 200, check=False)
        return st, rel, its

    for _ in range(args.warmup):
        step(args.prec)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = S.stats()["kernel_launches"]
    sampler = ClockSampler(local)
    sampler.start()
    ph = {p: 0.0 for p in PHASES + SOLVE_PHASES}
    ph["factor"] = 0.0
    ph["factor_wait_basis"] = 0.0
    ph["solve"] = 0.0
    t_leaf = 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rels, its_all = [], []
    for _ in range(args.steps):
        # the NVTX range lets a profiler select the timed steps alone
        # (ncu --nvtx --nvtx-include "timed_step/")
        torch.cuda.nvtx.range_push("timed_step")
        st, rel, its = step(args.prec)
        torch.cuda.nvtx.range_pop()
        s = S.stats()
        for p in PHASES + SOLVE_PHASES:
            ph[p] += s["times"][p]
        ph["factor"] += s["times"]["factor"]
        ph["factor_wait_basis"] += s["times"].get("wait_basis", 0.0)
        t_leaf += s["times"]["matvec32_leaf"]
        ph["solve"] += s["times"]["solve"]
        rels.append(rel)
        its_all.append(its)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_ms = e0.elapsed_time(e1) / args.steps
    launches = S.stats()["kernel_launches"] - launches0
    if world > 1:
        t = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    stats = S.stats()
    for k in ph:
        ph[k] /= args.steps
    x_host = x_dev.cpu().numpy()
    # the last step's solution checked with the FP64 H^2 matvec (h2_matvec),
    # outside the timed region
    r_check = float(np.linalg.norm(b - S.matvec(x_host)) / np.linalg.norm(b))
    dense = dense_rows_check(wl, P, b, x_host, S, rows=args.dense_rows)

    # end to end through the C ABI with host buffers (H2D of b, D2H of x inside)
    xh = np.zeros_like(b)
    from paper_2502_02395_gb300 import h2_factor
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h2_factor(S.ctx, args.prec)
        h2_solve(S.ctx, b, xh, args.target, 200, check=False)
    e2e_s = (time.perf_counter() - t0) / args.steps

    # the plain FP64 H^2-ULV on the same instance (the metric's comparison)
    fp64 = None
    if args.fp64_steps > 0 and args.prec != "fp64":
        step("fp64")
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64 = []
        for _ in range(args.fp64_steps):
            r64.append(step("fp64"))
        f1.record(stream)
        torch.cuda.synchronize()
        s64 = S.stats()
        fp64 = {"s_per_step": f0.elapsed_time(f1) / args.fp64_steps / 1e3, "relres": r64[-1][1],
                "iters": r64[-1][2], "factor_s": s64["times"]["factor"], "solve_s": s64["times"]["solve"],
                "phases": {p: s64["times"][p] for p in PHASES}, "stats": s64,
                "factor_gflops": sum(s64["flops"].values()) / s64["times"]["factor"] / 1e9}

    # dominant phase of the step and its roofline
    tc = stats.get("tensor_cores", False)
    fp64_tf = fp64_peak_tflops()
    calls = stats["calls"]
    # the largest single kernel of the step: the FP32 leaf matvec (mixed
    # precision); per-phase rooflines follow for the rest of the step
    roof = kernel_roofline(stats, t_leaf / args.steps, calls.get("matvec32_leaf", 0), peaks)
    if roof is None:
        top = max(PHASES + SOLVE_PHASES, key=lambda p: ph[p])
        roof = roofline_for(top, stats, ph[top], calls, peaks, args.prec, tc, fp64_tf)
    roofs = {p: roofline_for(p, stats, ph[p], calls, peaks, args.prec, tc, fp64_tf)
             for p in ("a1_qr", "a2_proj", "a3_lu", "solve_subst", "solve_matvec", "solve_matvec32")}
    if fp64:
        # the FP64 comparator's phases against the FP64 peak measured now
        s64 = fp64.pop("stats")
        fp64["rooflines"] = {p: roofline_for(p, s64, s64["times"][p], s64["calls"], peaks, "fp64", False, fp64_tf)
                             for p in ("a1_qr", "a2_proj", "a3_lu", "a45_schur", "solve_subst", "solve_matvec")
                             if s64["times"].get(p, 0) > 0}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = min(args.cpu_sample_n, wl.n)
        H, bs = oracle_instance(wl, n)
        dt, hist = oracle_step(H, bs, args.target)
        cpu = {"value": dt * wl.n / n, "unit": UNIT, "cores": threads_used(), "kind": "oracle",
               "sample": f"oracle factor + FGMRES refinement to {args.target:g} measured at N={n} of the same workload: "
                         f"{dt:.2f} s, scaled by N/{n} = {wl.n / n:g} (the method is O(N); a full N={wl.n} oracle "
                         f"run on these cores is recorded beside the baseline numbers)",
               "measured_n": n, "measured_s": dt}

    value = t_ms / 1e3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp16": "f16/f32/f64", "bf16": "bf16/f32/f64", "fp64": "f64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": wl.name, "N": wl.n, "geometry": wl.geometry, "kernel": wl.kernel, "leaf": wl.leaf,
                   "eta": wl.eta, "tol": wl.tol, "prec": args.prec, "target_relres": args.target,
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "no flush: inputs (13 GB leaf blocks, factors) exceed L2"},
        "relres": float(np.max(rels)), "relres_fp64_matvec": r_check, "dense_rows_check": dense,
        "iters": int(np.max(its_all)),
        "rr_lu": args.rr_lu, "residual": args.residual, "graphs": args.graphs, "tc_kernel": args.tc_kernel, "box_stream": args.box_stream,
        "autotune": tuned and {k: v for k, v in tuned.items() if k != "tried"},
        "phases_s": ph, "build_s": build_s, "build": args.build, "fp64": fp64,
        "speedup_vs_fp64": (fp64["s_per_step"] / value) if fp64 else None,
        "roofline": roof, "rooflines": roofs, "fp64_peak_tflops": fp64_tf, "calls": calls,
        # algorithmic flops of the factorization (QR, projection of the
        # projected pairs, inverses, Schur updates, couplings) over its time
        "factor_gflops": (sum(stats["flops"].values()) / ph["factor"] / 1e9) if ph.get("factor") else None,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(b.nbytes), "d2h_bytes_per_step": int(b.nbytes)},
        "gpu_launches": int(launches), "clocks": clocks,
        "levels": stats["levels"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
