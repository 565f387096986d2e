"""HSS (eta = 0) against H^2 (eta = 1) at fixed ranks: solution accuracy,
time and memory of the GPU H^2-ULV (the study of Section 6.3, Fig. 18-19).

Run on a GPU machine:
    python tests/study_hss_vs_h2.py [--n 8192] [--leaf 512] [--out FILE]

Setup as in Section 6.3: N points, leaf size 512, fixed-rank truncation
(tol 1e-14 and max_rank = r, so every level keeps rank r) over all
far-field points (no far-field or close-field sampling).  Points uniform
on the unit sphere, kernel 1/(r + 1e-3), right-hand side uniform in [-1, 1].
For each admissibility and rank: construction (h2_build), FP64
factorization and one ULV application (the direct solve) on the GPU, the
relative error of that solution against the dense LU solution (the oracle's
dense path, FP64 LAPACK on the host), the number of FP64 FGMRES
refinement steps to 1e-10, and the device bytes of the instance plus one
FP64 factorization.  Prints one JSON line per configuration and writes a
markdown table to --out.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402


def run(n=8192, leaf=512, configs=None, seed=3):
    import torch
    from oracle import dense
    from oracle.kernels import Kernel
    from paper_2502_02395_gb300 import binding as B
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    assert torch.cuda.is_available()
    P = W.sphere_points(n, seed)
    b = W.uniform_rhs(n, seed + 1)
    t0 = time.perf_counter()
    x_dense = dense.lu_solve(dense.dense_matrix(P, Kernel("laplace_eps")), b)
    t_dense = time.perf_counter() - t0
    rows = []
    for eta, r in configs:
        kw = dict(kernel="laplace_eps", leaf=leaf, eta=eta, tol=1e-14, max_rank=r, far_samples=0, near_samples=0)
        plan = B.h2_plan(B.make_params(**kw), P)
        t0 = time.perf_counter()
        S = B.H2Solver.build(P, **kw)
        t_build = time.perf_counter() - t0
        S.factor("fp64")
        st = S.stats()
        t_factor = st["times"]["factor"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = S.ulv_apply(b)
        t_solve = time.perf_counter() - t0
        err = float(np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense))
        S.set_refinement("gmres", 30)
        _, rel, its = S.solve(b, target=1e-10, max_iters=200)
        S.close()
        row = {"eta": eta, "rank": r, "K": [lv["K"] for lv in plan["levels"]],
               "near_pairs_leaf": plan["levels"][-1]["NP"], "build_s": t_build, "factor_s": t_factor,
               "ulv_apply_s": t_solve, "direct_solve_relerr": err, "refine_steps_to_1e-10": its,
               "device_bytes": plan["device_bytes_build"] + plan["device_bytes_factor_fp64"]}
        print(json.dumps(row), flush=True)
        rows.append(row)
    return rows, t_dense


def table(rows, n, leaf, t_dense):
    out = [f"N = {n}, leaf {leaf}, sphere, 1/(r + 1e-3), fixed-rank truncation over all far-field points; "
           f"dense LU reference on the host ({t_dense:.1f} s).", "",
           "| admissibility | rank | leaf near pairs | factor (ms) | ULV apply (ms) | direct-solve rel. error "
           "| FGMRES steps to 1e-10 | device MB |",
           "|---|---:|---:|---:|---:|---:|---:|---:|"]
    for r in rows:
        name = "HSS (eta 0)" if r["eta"] == 0 else f"H^2 (eta {r['eta']:g})"
        out.append(f"| {name} | {r['rank']} | {r['near_pairs_leaf']} | {r['factor_s'] * 1e3:.1f} | "
                   f"{r['ulv_apply_s'] * 1e3:.1f} | {r['direct_solve_relerr']:.2e} | {r['refine_steps_to_1e-10']} | "
                   f"{r['device_bytes'] / 1e6:.0f} |")
    return "\n".join(out) + "\n"


DEFAULT = [(1.0, r) for r in (10, 25, 50, 100, 200)] + [(0.0, r) for r in (50, 100, 200, 300, 400, 500)]

if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--leaf", type=int, default=512)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    rows, t_dense = run(a.n, a.leaf, DEFAULT)
    md = table(rows, a.n, a.leaf, t_dense)
    print(md)
    if a.out:
        with open(a.out, "w") as f:
            f.write(md)
