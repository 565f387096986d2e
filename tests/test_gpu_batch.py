"""Batches of independent systems (h2_batch_*): Gaussian-covariance systems
exp(-r^2 / l^2) + I of uneven size and length scale, factored and
solved concurrently by the library's worker pool.  Every system's result
must equal the one its context gives alone (the kernels and their order per
context do not depend on what runs beside them), and the tuner must pick a
worker count from measured times."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def systems():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding as B
    specs = W.batch_systems(count=8, n_min=2048, n_max=12288)
    solvers, rhs = [], []
    for sp in specs:
        P = W.cube_points(sp["n"], sp["point_seed"])
        solvers.append(B.H2Solver.build(P, kernel="gaussian", ell=sp["ell"], diag_shift=sp["shift"], leaf=sp["leaf"],
                                        eta=1.0, tol=1e-8, far_samples=512, near_samples=64))
        rhs.append(W.uniform_rhs(sp["n"], sp["rhs_seed"]))
    yield B, specs, solvers, rhs
    for S in solvers:
        S.close()


def test_batch_equals_systems_alone(systems):
    B, specs, solvers, rhs = systems
    batch = B.H2Batch(solvers)
    try:
        X, rel, its, sec = batch.run("fp16", rhs, target=1e-10, max_iters=200)
        print(f"batch of {len(specs)} systems (N {[s['n'] for s in specs]}): {sec:.3f} s, iterations {its}")
        assert all(r <= 1e-10 for r in rel)
        for S, b, x, r, k in zip(solvers, rhs, X, rel, its):
            S.set_stream(None)
            S.factor("fp16")
            x1, r1, k1 = S.solve(b, target=1e-10, max_iters=200)
            assert np.array_equal(x, x1) and k == k1, (S.n, k, k1)
    finally:
        batch.close()


def test_batch_tuner_picks_a_measured_worker_count(systems):
    B, specs, solvers, rhs = systems
    batch = B.H2Batch(solvers)
    try:
        w = batch.tune("fp16", rhs, target=1e-10, max_iters=200)
        st = batch.stats()
        print("tuning (workers: seconds):", st["tune_seconds"], "-> workers", w)
        times = {int(k): v for k, v in st["tune_seconds"].items()}
        assert w in times and times[w] == min(times.values())
        assert set(times) >= {1, 2, 4, 8}
    finally:
        batch.close()
