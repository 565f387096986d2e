"""Batched systems as forests (h2_build_forest, h2_batch_create_forest):
several independent systems of one tree depth as one instance whose level
arrays hold every system, so each level's kernels run once for all of them.

What is checked, and why it pins the combination:
  * A_H2 of the forest is block diagonal with the systems' own H^2 matrices:
    with one rank for every system (a rank cap all of them reach), its FP64
    matvec equals each system's own h2_matvec to 1e-13 (leaves padded with
    padding points add exact zeros only), so a wrong box offset, row layout
    or skeleton offset fails;
  * the factorization of the forest (one root per system) is a
    preconditioner for that block-diagonal matrix: the refined solution of
    every system matches its own instance's refined solution to 1e-8
    relative (both solve to 1e-12), FP64 and FP16;
  * systems whose tolerance ranks differ are compressed again at each
    level's largest rank; the forest then converges within a few steps of
    its slowest system alone (zero-padded ranks stalled here: the padding
    directions' near-field couplings are missing from the parent's
    pre-factorization basis);
  * the forest batch groups systems by depth, scales each right-hand side
    to unit norm and stops the group at target / sqrt(m): every system's
    residual, recomputed from an FP32-pair matvec, is at most the target;
  * releasing the FP64 leaf blocks (which forest batches do) leaves the
    FP16 path's results unchanged and turns every FP64 use into an error.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

# tol 1e-10 with a rank cap of 64 that every system reaches: equal ranks
KW = dict(kernel="laplace_eps", leaf=256, eta=1.0, tol=1e-10, max_rank=64, far_samples=1024, near_samples=64)


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding
    return binding


def systems(ns, seed):
    return [W.cube_points(n, seed + k) for k, n in enumerate(ns)]


def test_forest_matvec_is_block_diagonal(B):
    ns = [2600, 3500, 4096]  # depth 4 with leaf 256; ranks and leaves differ
    P = systems(ns, 31)
    assert len({B.h2_tree_depth(n, 256) for n in ns}) == 1
    F = B.H2Solver.build_forest(P, **KW)
    st = F.stats()
    assert st["systems"] == len(ns) and st["levels"][0]["nb"] == len(ns)
    singles = [B.H2Solver.build(p, **KW) for p in P]
    x = [W.uniform_rhs(n, 40 + k) for k, n in enumerate(ns)]
    y = F.matvec(np.concatenate(x))
    off = 0
    for k, S in enumerate(singles):
        ys = S.matvec(x[k])
        e = np.linalg.norm(y[off:off + ns[k]] - ys) / np.linalg.norm(ys)
        assert [lv["K"] for lv in S.stats()["levels"]] == [lv["K"] for lv in st["levels"]]
        print(f"system {k} (N {ns[k]}): forest vs own matvec {e:.2e}")
        assert e <= 1e-13
        off += ns[k]
    for S in singles:
        S.close()
    F.close()


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_forest_solve_matches_single_systems(B, prec):
    ns = [2300, 3000, 3900, 4096]
    P = systems(ns, 51)
    F = B.H2Solver.build_forest(P, **KW)
    b = [W.uniform_rhs(n, 60 + k) for k, n in enumerate(ns)]
    F.factor(prec)
    x, rel, its = F.solve(np.concatenate(b), target=1e-12, max_iters=200)
    assert rel <= 1e-12
    off = 0
    for k, p in enumerate(P):
        S = B.H2Solver.build(p, **KW)
        S.factor(prec)
        xs, rs, _ = S.solve(b[k], target=1e-12, max_iters=200)
        e = np.linalg.norm(x[off:off + ns[k]] - xs) / np.linalg.norm(xs)
        print(f"{prec} system {k}: forest vs single solution {e:.2e} ({its} forest steps)")
        assert rs <= 1e-12 and e <= 1e-8
        off += ns[k]
        S.close()
    F.close()


def test_forest_mixed_ranks_converge(B):
    """Gaussian systems of one depth whose tolerance ranks differ (length
    scales 0.15 .. 0.45, points divided by l, every close-field point
    sampled): the forest takes each level's largest rank, and its FP16
    refinement needs at most 3 steps more than the slowest system alone."""
    ns = [1300, 1600, 1800, 2048]
    ells = [0.15, 0.25, 0.35, 0.45]
    kw = dict(kernel="gaussian", ell=1.0, diag_shift=1.0, leaf=128, eta=1.0, tol=1e-8, far_samples=1024,
              near_samples=0)
    P = [p / l for p, l in zip(systems(ns, 91), ells)]
    b = [W.uniform_rhs(n, 95 + k) for k, n in enumerate(ns)]
    ks, its_single = [], []
    for k, p in enumerate(P):
        S = B.H2Solver.build(p, **kw)
        ks.append([lv["K"] for lv in S.stats()["levels"]])
        S.factor("fp16")
        _, rs, it = S.solve(b[k], target=1e-10, max_iters=200)
        assert rs <= 1e-10
        its_single.append(it)
        S.close()
    F = B.H2Solver.build_forest(P, **kw)
    kf = [lv["K"] for lv in F.stats()["levels"]]
    assert kf == [max(c) for c in zip(*ks)]
    assert len({tuple(k) for k in ks}) > 1
    F.factor("fp16")
    bn = np.concatenate([v / np.linalg.norm(v) for v in b])
    _, rel, its = F.solve(bn, target=1e-10 / 2, max_iters=200)
    print(f"ranks {ks} -> forest {kf}; steps alone {its_single}, forest {its}")
    assert rel <= 0.5e-10 and its <= max(its_single) + 3
    F.close()


def test_forest_batch_groups_and_targets(B):
    """Two depths (3 and 4 with leaf 256) give two groups; Gaussian systems
    with their own length scales pass points divided by l and l = 1."""
    ns = [1500, 1900, 2048, 2500, 3300, 4000]
    ells = [0.3, 0.45, 0.35, 0.5, 0.4, 0.3]
    P = systems(ns, 71)
    kw = dict(kernel="gaussian", ell=1.0, diag_shift=1.0, leaf=256, eta=1.0, tol=1e-8, far_samples=1024,
              near_samples=64)
    bt = B.H2Batch.forest([p / l for p, l in zip(P, ells)], **kw)
    st = bt.stats()
    assert st["mode"] == "forest" and st["groups"] == 2 and sorted(st["group_systems"]) == [3, 3]
    b = [W.uniform_rhs(n, 80 + k) for k, n in enumerate(ns)]
    X, rel, its, sec = bt.run("fp16", b, target=1e-10, max_iters=200)
    print(f"forest batch: {sec:.3f} s, relres {[f'{r:.1e}' for r in rel]}, steps {its}")
    for k in range(len(ns)):
        assert rel[k] <= 1e-10
        # the same system alone (scaled points, l = 1; its own ranks, so
        # the two H^2 matrices differ at the compression's level), FP64
        S = B.H2Solver.build(P[k] / ells[k], **kw)
        S.factor("fp64")
        xs, _, _ = S.solve(b[k], target=1e-12, max_iters=200)
        e = np.linalg.norm(X[k] - xs) / np.linalg.norm(xs)
        S.close()
        # and against the unscaled points with its own l: the same matrix up
        # to the construction's rounding, so the residual stays at the
        # approximation level (a length scale left out gives O(1))
        S = B.H2Solver.build(P[k], kernel="gaussian", ell=ells[k], diag_shift=1.0, leaf=256, eta=1.0, tol=1e-8,
                             far_samples=1024, near_samples=64)
        r = np.linalg.norm(b[k] - S.matvec(X[k])) / np.linalg.norm(b[k])
        S.close()
        print(f"  system {k}: vs its own FP64 solve {e:.2e}; residual against the unscaled instance {r:.2e}")
        assert e <= 1e-3 and r <= 1e-3
    bt.close()


def test_fp64_leaf_release(B):
    """H2_OPT_FP64_LEAF = 0 frees the FP64 leaf blocks: the FP16 path gives
    the same refined solution as before (it reads only the FP32 pair and
    FP16 copies; same steps, same x to 1e-12), and everything that needs the
    FP64 blocks returns H2_ERR_STATE instead of reading freed memory."""
    P = W.cube_points(4096, 120)
    b = W.uniform_rhs(4096, 121)
    S = B.H2Solver.build(P, **KW)
    S.factor("fp16")
    x0, r0, i0 = S.solve(b, target=1e-10, max_iters=100)
    S.set_option("fp64_leaf", 0)
    S.factor("fp16")
    x1, r1, i1 = S.solve(b, target=1e-10, max_iters=100)
    assert i1 == i0 and np.abs(x0 - x1).max() <= 1e-12 * np.abs(x0).max()
    y = S.matvec_arith(x1, "fp32_pair")
    assert np.linalg.norm(y - b) <= 1e-9 * np.linalg.norm(b)
    for call in (lambda: S.factor("fp64"), lambda: S.factor("bf16"), lambda: S.matvec(b),
                 lambda: S.set_option("fp64_leaf", 1)):
        with pytest.raises(B.H2Error) as ei:
            call()
        assert ei.value.status == -7
    S.close()


def test_release_factorization(B):
    """h2_release_factorization frees the factorization's arrays (a forest
    batch does so after each group's solve): a solve then reports
    H2_ERR_STATE, and a new factorization gives the same solution."""
    P = W.cube_points(4096, 130)
    b = W.uniform_rhs(4096, 131)
    S = B.H2Solver.build(P, **KW)
    S.factor("fp16")
    x0, _, i0 = S.solve(b, target=1e-10, max_iters=100)
    S.release_factorization()
    with pytest.raises(B.H2Error) as ei:
        S.solve(b, target=1e-10, max_iters=100)
    assert ei.value.status == -7
    S.factor("fp16")
    x1, _, i1 = S.solve(b, target=1e-10, max_iters=100)
    assert i1 == i0 and np.abs(x0 - x1).max() <= 1e-12 * np.abs(x0).max()
    S.close()
