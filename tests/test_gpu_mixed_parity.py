"""GPU parity of the mixed-precision path (FP16/BF16 factorizations) against
the FP64 oracle, kernel by kernel, on the same H^2 instance (h2_import).

What each test pins, and the bound it uses:
  * one ULV application (Eq. 24-31 and its mirror) after a 16-bit
    factorization, element by element against the oracle's FP64
    solve_parallel: the factors differ from the FP64 ones by the rounding of
    the 16-bit operands (unit roundoff u16 = 2^-11 for FP16, 2^-8 for BF16),
    grown by the conditioning of the substitution, so the bound is a fixed
    multiple of u16 times max |x|;
  * the inverses (Ahat_ii^RR)^-1 of the mixed factorization against
    numpy.linalg.inv of the same FP32 blocks, and (FP64 elimination, the
    H2_OPT_RR_LU_FP64 option) the pivot sequence against LAPACK getrf on the
    same input;
  * the leaf self Schur update Ahat_ii^SS -= Ahat_ii^SR (Ahat_ii^RR)^-1
    Ahat_ii^RS (Eq. 21) against the same formula in FP64 on the library's own
    FP32 bases and quadrants;
  * the FP32 H^2 matvec of the inner solver and the FP32-pair matvec of the
    refinement residual against the oracle's FP64 matvec, element by
    element, relative to the row sums s = |A_H2| |x| (the absolute terms of
    each product sum): c u32 s for FP32 (u32 = 2^-24) and c 2^-46 s for the
    FP32 pairs;
  * the refined solve: the number of preconditioner applications of the
    mixed refinement is bounded by the FP64 one's plus a small margin.
Cases: cube8192_yukawa (L = 5) and cube32768_yukawa (L = 7: levels with few
boxes, per-level row splitting, the upper-pair projection over six levels).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W

pytestmark = pytest.mark.gpu

U16 = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
U32 = 2.0 ** -24

# name: (n, leaf, far_samples, near_samples, seed, kernel, parameters)
YUKAWA = ("yukawa_eps", dict(diag_shift=1.0))
CASES = {
    "cube8192_yukawa": (8192, 256, 1024, 64, 5) + YUKAWA,
    "cube32768_yukawa": (32768, 256, 1024, 64, 5) + YUKAWA,
    # a Gaussian kernel exp(-r^2 / 0.0225) + 0.01 on the diagonal, leaf 256,
    # rank 128: the RR blocks are far from diagonal, so the self Schur update
    # of Eq. 21 is 9 - 51 % of the result
    "cube4096_gauss": (4096, 256, 512, 64, 7, "gaussian", dict(ell=0.15, diag_shift=0.01)),
}
MAIN = ["cube8192_yukawa", "cube32768_yukawa"]

_cache = {}


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding
    return binding


def oracle_case(name):
    if name in _cache:
        return _cache[name]
    from oracle import ulv
    from oracle.construct import construct
    from oracle.instance import flatten
    from oracle.kernels import Kernel
    n, leaf, fs, ns, seed, kern, kw = CASES[name]
    P = W.cube_points(n, seed)
    H = construct(P, Kernel(kern, **kw), leaf, 1.0, 1e-10 if kern == "yukawa_eps" else 1e-8, 0, fs, ns)
    F = ulv.factor(H)
    b = W.uniform_rhs(n, seed + 100)
    _cache[name] = (H, F, flatten(H), b)
    return _cache[name]


def solver(B, name):
    H, F, flat, b = oracle_case(name)
    n, leaf, fs, ns, seed, kern, kw = CASES[name]
    return B.H2Solver.from_instance(flat, kernel=kern, leaf=leaf, eta=1.0, tol=H["tol"], far_samples=fs,
                                    near_samples=ns, **kw)


def abs_instance(H):
    """The instance with every stored array replaced by its absolute value:
    its matvec with |x| gives the row sums of the absolute product terms."""
    Ha = dict(H)
    Ha["A"] = {k: np.abs(v) for k, v in H["A"].items()}
    Ha["X"] = [None if v is None else np.abs(v) for v in H["X"]]
    Ha["S"] = [{k: np.abs(v) for k, v in d.items()} for d in H["S"]]
    return Ha


@pytest.mark.parametrize("rr", [1, 0])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("name", MAIN)
def test_mixed_ulv_apply_elementwise(B, name, prec, rr):
    """x = ULV^-1 b with the 16-bit factorization against the oracle's FP64
    Eq. 24-31: |x - x_ref|_i <= 8 u16 max|x_ref| for every i (measured:
    3.2 - 4.3 u16 on both cases, FP16 and BF16)."""
    from oracle import ulv
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    S.set_option("rr_lu_fp64", rr)
    S.factor(prec)
    x = S.ulv_apply(b)
    x_ref = ulv.solve_parallel(F, H, b)
    err = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    print(f"\n{name} {prec} rr_lu_fp64={rr}: max|x - x_ref| / max|x_ref| = {err:.3e} ({err / U16[prec]:.2f} u16)")
    assert err <= 8 * U16[prec], err
    S.close()


@pytest.mark.parametrize("name", MAIN)
def test_streamed_box_steps_elementwise(B, name):
    """The streamed per-box substitution kernels (bulk-copy ring, persistent
    CTAs; H2_OPT_BOX_STREAM = 2 puts them on every level of these shapes,
    1 only on levels with a box per SM; off by default) against the oracle's FP64
    Eq. 24-31, with the bound of the row-split kernels (8 u16), and against
    the row-split kernels on the same factorization (FP32 sums grouped
    differently: 1e-5 of max|x|)."""
    from oracle import ulv
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    S.factor("fp16")
    try:
        S.set_option("box_stream", 0)
        x0 = S.ulv_apply(b)
        S.set_option("box_stream", 2)
        x2 = S.ulv_apply(b)
        _, rel, its = S.solve(b, target=1e-10, max_iters=100)
    finally:
        S.set_option("box_stream", 0)  # the library's default
    x_ref = ulv.solve_parallel(F, H, b)
    e_ref = np.abs(x2 - x_ref).max() / np.abs(x_ref).max()
    e_rs = np.abs(x2 - x0).max() / np.abs(x0).max()
    print(f"\n{name}: streamed vs oracle {e_ref:.3e} ({e_ref / U16['fp16']:.2f} u16), vs row-split {e_rs:.2e}; "
          f"refined {rel:.2e} in {its}")
    assert e_ref <= 8 * U16["fp16"] and e_rs <= 1e-5 and rel <= 1e-10
    S.close()


@pytest.mark.parametrize("rr", [1, 0])
@pytest.mark.parametrize("name", MAIN)
def test_mixed_inverses_and_pivots(B, name, rr):
    """(Ahat_ii^RR)^-1 of the FP16 factorization against numpy's inverse of
    the same FP32 blocks, at every level and at the root.  FP64 LU (rr = 1):
    the pivots are LAPACK getrf's on that input and the inverse is the FP64
    one rounded to FP32 (relative error <= 8 u32; measured 0.6 u32).  FP32
    Gauss-Jordan (rr = 0): relative error <= 2 R u32 cond(Ahat_ii^RR), the
    n u backward-error bound of elimination (measured up to 1.1 R u32 at
    cond 1.9)."""
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    S.set_option("rr_lu_fp64", rr)
    S.factor("fp16")
    worst = 0.0
    for l in range(H["L"], 0, -1):
        D, K = H["D"][l], H["K"][l]
        R, nb = D - K, 1 << l
        if R == 0:
            continue
        Ah = S.export("Ahat", l).reshape(-1, D, D).astype(np.float64)
        Ainv = S.export("Ainv", l).reshape(nb, R, R).astype(np.float64)
        piv = S.export("piv", l).reshape(nb, R)
        for i in range(nb):
            q = H["near"][l].index((i, i))
            RR = Ah[q][:R, :R]
            ref = np.linalg.inv(RR)
            e = np.linalg.norm(Ainv[i] - ref) / np.linalg.norm(ref)
            worst = max(worst, e)
            if rr:
                assert (piv[i] == sla.lu_factor(RR)[1]).all(), (l, i)
                assert e <= 8 * U32, (l, i, e)
            else:
                assert e <= 2 * R * U32 * np.linalg.cond(RR), (l, i, e)
    D0 = H["D"][0]
    print(f"\n{name} rr_lu_fp64={rr}: worst relative inverse error {worst:.3e}")
    root_inv = S.export("root_inv", 0).reshape(D0, D0).astype(np.float64)
    assert np.all(np.isfinite(root_inv))
    S.close()


def test_mixed_schur_update_leaf(B):
    """Eq. 21's self Schur update at the leaf level of the FP16
    factorization: the stored SS quadrant of Ahat_ii equals
    (U_i^T A_ii U_i)^SS - SR (RR)^-1 RS, evaluated in FP64 from the library's
    FP32 bases and its own RR, RS, SR quadrants, to the 16-bit rounding of
    the projection (4e-3 relative, the leaf projection test's bound).  The
    update runs on the tensor cores (16-bit (Ahat_ii^RR)^-1 and Z^T, FP32
    accumulation); on this Gaussian case it is 9 - 51 % of the result, so
    leaving it out or applying it with a wrong sign fails the bound."""
    name = "cube4096_gauss"
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    S.factor("fp16")
    st = S.stats()
    assert st["tensor_cores"] is True and st["schur_tensor_cores"] is True
    L = H["L"]
    D, K = H["D"][L], H["K"][L]
    R, nb = D - K, 1 << L
    U = S.export("U", L).reshape(nb, D, D).astype(np.float64)  # U[i] = U_i^T
    Ah = S.export("Ahat", L).reshape(-1, D, D).astype(np.float64)
    ratios = []
    for i in range(nb):
        q = H["near"][L].index((i, i))
        proj = U[i] @ H["A"][(i, i)] @ U[i].T
        blk = Ah[q]
        upd = blk[R:, :R] @ np.linalg.solve(blk[:R, :R], blk[:R, R:])
        ref = proj[R:, R:] - upd
        err = np.linalg.norm(blk[R:, R:] - ref) / np.linalg.norm(ref)
        ratios.append(np.linalg.norm(upd) / np.linalg.norm(ref))
        assert err <= 4e-3, (i, err)
    print(f"\n{name}: |Schur update| / |SS| in [{min(ratios):.2e}, {max(ratios):.2e}]")
    assert max(ratios) >= 10 * 4e-3
    S.close()


@pytest.mark.parametrize("name", MAIN)
def test_fp32_matvec_elementwise(B, name):
    """The inner solver's FP32 H^2 matvec (symmetric leaf storage, all
    levels' couplings in one launch, leaf products on a second stream)
    against the oracle's FP64 matvec: |y - y_ref|_i <= 4 u32 s_i (measured
    at most 0.5 u32)."""
    from oracle import ulv
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    Ha = abs_instance(H)
    for seed in (0, 1):
        x = W.uniform_rhs(H["N"], 500 + seed)
        y = S.matvec_arith(x, "fp32")
        y_ref = ulv.matvec(H, x)
        s = ulv.matvec(Ha, np.abs(x))
        c = (np.abs(y - y_ref) / s).max() / U32
        print(f"\n{name}: FP32 matvec max |y - y_ref| / s = {c:.2f} u32")
        assert c <= 4, c
    S.close()


@pytest.mark.parametrize("name", MAIN)
def test_fp32_pair_residual_elementwise(B, name):
    """The mixed refinement's residual matvec (FP32-pair arithmetic) against
    the oracle's FP64 matvec: |y - y_ref|_i <= 2^-46 s_i (the pair
    arithmetic's error per product sum; measured at most 0.16 2^-46, which
    includes the FP64 evaluation's own rounding); on a refined solution the
    residuals b - A_H2 x agree to 5e-14 ||b|| in norm, 2000 times below the
    1e-10 stopping threshold the residual decides (measured 1.2e-14, with
    the bases, couplings and leaf sums in FP32 pairs as well)."""
    from oracle import ulv
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    Ha = abs_instance(H)
    x = W.uniform_rhs(H["N"], 600)
    y = S.matvec_arith(x, "fp32_pair")
    y_ref = ulv.matvec(H, x)
    s = ulv.matvec(Ha, np.abs(x))
    c = (np.abs(y - y_ref) / s).max()
    print(f"\n{name}: FP32-pair matvec max |y - y_ref| / s = {c:.3e} ({c / 2.0 ** -46:.2f} x 2^-46)")
    assert c <= 2.0 ** -46, c
    y64 = S.matvec_arith(x, "fp64")
    assert (np.abs(y64 - y_ref) / s).max() <= 2.0 ** -48
    S.factor("fp16")
    xs, rel, its = S.solve(b, target=1e-11, max_iters=100)
    r_df = b - S.matvec_arith(xs, "fp32_pair")
    r_ref = b - ulv.matvec(H, xs)
    d = np.linalg.norm(r_df - r_ref) / np.linalg.norm(b)
    print(f"{name}: ||r_pair - r_ref|| / ||b|| = {d:.3e}, relres {rel:.2e}")
    assert d <= 5e-14, d
    S.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("name", MAIN)
def test_mixed_iterations_bounded(B, name, prec):
    """Refinement to 1e-11: the mixed path (16-bit factorization, FP32 inner
    FGMRES, FP64 residual and update) needs at most the FP64 path's
    preconditioner applications plus 2 (measured: plus 0 or 1), and its
    solution matches the oracle's refined one."""
    from oracle import ulv
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    S.factor("fp64")
    x64, r64, n64 = S.solve(b, target=1e-11, max_iters=100)
    S.factor(prec)
    x, r, n = S.solve(b, target=1e-11, max_iters=100)
    print(f"\n{name} {prec}: preconditioner applications fp64 {n64}, mixed {n}")
    assert r <= 1e-11 and r64 <= 1e-11
    assert n <= n64 + 2, (n, n64)
    x_ref, _, _ = ulv.refine_gmres(F, H, b, 1e-11, 60, 30)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-8
    S.close()


def test_residual_fp64_option(B):
    """H2_OPT_RESIDUAL_FP64: the mixed refinement with its residual in FP64
    instructions reaches the same solution as with FP32 pairs."""
    H, F, flat, b = oracle_case("cube8192_yukawa")
    S = solver(B, "cube8192_yukawa")
    S.factor("fp16")
    xa, ra, na = S.solve(b, target=1e-11, max_iters=100)
    S.set_option("residual_fp64", 1)
    xb, rb, nb_ = S.solve(b, target=1e-11, max_iters=100)
    assert ra <= 1e-11 and rb <= 1e-11
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xb) <= 1e-9
    S.close()


def test_bounded_wait_gives_timeout_and_context_survives(B):
    """A bounded device wait that nothing completes gives up after its limit
    and the library reports H2_ERR_TIMEOUT; the context stays usable (a
    matvec afterwards equals one before)."""
    H, F, flat, b = oracle_case("cube8192_yukawa")
    S = solver(B, "cube8192_yukawa")
    y0 = S.matvec(b)
    st = B.h2_wait_selftest(S.ctx, 1_000_000)
    assert st == -6, st
    assert "gave up" in B.h2_last_error(S.ctx)
    assert np.array_equal(S.matvec(b), y0)
    S.factor("fp16")
    x, r, its = S.solve(b, target=1e-10, max_iters=100)
    assert r <= 1e-10
    S.close()


@pytest.mark.parametrize("rr", [0, 1])
def test_cluster_inverse_root256(B, rr):
    """A root block of dimension 256 (every level at rank 128 from the
    fixed-rank GPU construction, so D_0 = 2 K_1 = 256): its inverse comes
    from the Gauss-Jordan elimination split over a thread-block cluster
    (FP32: 4 CTAs; FP64 with H2_OPT_RR_LU_FP64: 8 CTAs).  Against numpy's
    inverse of the same FP32 root block: FP64 elimination, relative error
    <= 8 u32 and LAPACK getrf's pivots; FP32, <= 2 R u32 cond.  The refined
    solve then reaches 1e-10."""
    n = 8192
    P = W.cube_points(n, 81)
    S = B.H2Solver.build_gpu(P, None, 0, kernel="laplace_eps", leaf=256, tol=1e-8, far_samples=1024,
                             near_samples=64)
    D0 = S.stats()["levels"][0]["D"]
    assert D0 == 256
    S.set_option("rr_lu_fp64", rr)
    S.factor("fp16")
    A0 = S.export("A", 0).reshape(D0, D0).astype(np.float64)
    inv = S.export("root_inv", 0).reshape(D0, D0).astype(np.float64)
    piv = S.export("root_piv", 0)
    ref = np.linalg.inv(A0)
    e = np.linalg.norm(inv - ref) / np.linalg.norm(ref)
    cond = np.linalg.cond(A0)
    print(f"\nroot 256, rr_lu_fp64={rr}: relative inverse error {e:.3e} ({e / U32:.1f} u32), cond {cond:.2e}")
    if rr:
        assert (piv == sla.lu_factor(A0)[1]).all()
        assert e <= 8 * U32
    else:
        assert e <= 2 * D0 * U32 * cond
    _, rel, its = S.solve(W.uniform_rhs(n, 83), target=1e-10, max_iters=100)
    assert rel <= 1e-10
    S.close()


def test_autotune_choices_and_parity(B):
    """h2_autotune times the three GEMM forms and the 24 launch-shape
    combinations of the substitution on this instance and keeps the fastest
    of each; the context is left factored, its ULV application still meets
    the oracle bound (8 u16) and the refined solve reaches 1e-10.  The
    process-wide settings go back to the library's defaults afterwards."""
    from oracle import ulv
    name = "cube32768_yukawa"
    H, F, flat, b = oracle_case(name)
    S = solver(B, name)
    try:
        t = S.autotune("fp16")
        print(f"\nautotune: form {t['tc_kernel']} (factor s {t['factor_s']}), pair {t['pair_ctas_per_sm']}, "
              f"box {t['box_ctas_per_sm']}, streamed {t['box_stream']}, graphs {t['graphs']}: {t['subst_ms']:.3f} ms")
        assert t["tc_kernel"] in (0, 1, 2) and t["factor_s"][t["tc_kernel"]] == min(t["factor_s"])
        assert len(t["tried"]) == 24 and all(r[4] > 0 for r in t["tried"])
        assert abs(t["subst_ms"] - min(r[4] for r in t["tried"])) <= 1e-6 * t["subst_ms"] + 1e-9
        x = S.ulv_apply(b)
        x_ref = ulv.solve_parallel(F, H, b)
        assert np.abs(x - x_ref).max() <= 8 * U16["fp16"] * np.abs(x_ref).max()
        _, rel, _ = S.solve(b, target=1e-10, max_iters=100)
        assert rel <= 1e-10
    finally:
        for opt, val in (("tc_kernel", 2), ("pair_ctas", 3), ("box_ctas", 1), ("box_stream", 0), ("graphs", 1)):
            S.set_option(opt, val)
    S.close()
