"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties one part of the oracle to something the paper or the
mathematics fixes: closed forms, textbook routines, an exact-rank kernel for
which the method must be exact, invariants (orthogonality, basis rotation, the
H^2 block partition), and the convergence of the refinement.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dense, ulv
from oracle.construct import construct, id_basis, interpolative_decomposition
from oracle.kernels import Kernel
from oracle.tree import build_tree, interaction_lists, box_geometry


# ---------------------------------------------------------------- kernels ---
def test_kernel_closed_forms():
    """Eq. 35, Eq. 36 and the softened variants at hand-checked distances."""
    P = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    idx = np.arange(3)
    lap = Kernel("laplace_paper").matrix(P, idx, idx)
    assert lap[0, 0] == 1e3 and lap[0, 1] == 0.5 and lap[0, 2] == 1.0
    assert lap[1, 2] == pytest.approx(1.0 / math.sqrt(5.0), rel=1e-15)
    yuk = Kernel("yukawa_paper").matrix(P, idx, idx)
    assert yuk[1, 1] == 1e3
    assert yuk[0, 2] == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert yuk[0, 1] == pytest.approx(math.exp(-2.0) / 2.0, rel=1e-15)
    le = Kernel("laplace_eps", eps=1e-3).matrix(P, idx, idx)
    assert le[0, 0] == pytest.approx(1000.0, rel=1e-15)
    assert le[0, 1] == pytest.approx(1.0 / 2.001, rel=1e-15)
    ye = Kernel("yukawa_eps", eps=1e-3, diag_shift=1.0).matrix(P, idx, idx)
    assert ye[2, 2] == pytest.approx(1001.0, rel=1e-15)
    assert ye[0, 2] == pytest.approx(math.exp(-1.0) / 1.001, rel=1e-15)
    g = Kernel("gaussian", ell=0.5, diag_shift=1e-2).matrix(P, idx, idx)
    assert g[0, 0] == pytest.approx(1.01, rel=1e-15)
    assert g[0, 2] == pytest.approx(math.exp(-4.0), rel=1e-15)
    pq = Kernel("poly2_test", diag_shift=3.0).matrix(P, idx, idx)
    assert pq[1, 1] == pytest.approx(25.0 + 3.0 * 5.0)  # (1 + 4)^2 + d (1 + 4)
    assert pq[1, 2] == pytest.approx(1.0)             # (1 + 0)^2
    assert np.allclose(pq, pq.T) and np.allclose(lap, lap.T)


def test_poly2_blocks_have_rank_10():
    P = W.cube_points(200, 3)
    K = Kernel("poly2_test")
    M = K.matrix(P, np.arange(100), np.arange(100, 200))
    s = np.linalg.svd(M, compute_uv=False)
    assert s[9] > 1e-8 * s[0] and s[10] < 1e-12 * s[0]


# ------------------------------------------------------------------- tree ---
@pytest.mark.parametrize("n,leaf", [(1000, 64), (2048, 64), (777, 50), (64, 64), (65, 64)])
def test_tree_partition(n, leaf):
    P = W.cube_points(n, 7)
    perm, ranges = build_tree(P, leaf)
    L = len(ranges) - 1
    assert sorted(perm.tolist()) == list(range(n))
    sizes = np.diff(ranges[L])
    assert sizes.max() <= leaf and sizes.max() - sizes.min() <= 1
    assert L == (0 if n <= leaf else math.ceil(math.log2(n / leaf)))
    for l in range(L):
        # children 2i, 2i+1 split box i; the split is a median cut along the
        # longest axis of the box's bounding box
        for i in range(1 << l):
            a, m, b = ranges[l + 1][2 * i], ranges[l + 1][2 * i + 1], ranges[l + 1][2 * i + 2]
            assert a == ranges[l][i] and b == ranges[l][i + 1]
            assert m - a == (b - a) // 2
            X = P[perm[a:b]]
            ax = int(np.argmax(X.max(0) - X.min(0)))
            assert P[perm[a:m], ax].max() <= P[perm[m:b], ax].min()


@pytest.mark.parametrize("eta", [0.0, 1.0, 2.0])
def test_lists_partition_every_entry_once(eta):
    """Every (point, point) entry lies in exactly one block: a near block of
    the leaf level or a far block of exactly one level (the H^2 partition)."""
    n, leaf = 600, 40
    P = W.cube_points(n, 11)
    perm, ranges = build_tree(P, leaf)
    near, far = interaction_lists(P, perm, ranges, eta)
    L = len(ranges) - 1
    cover = np.zeros((n, n), dtype=np.int32)
    for (i, j) in near[L]:
        cover[ranges[L][i]:ranges[L][i + 1], ranges[L][j]:ranges[L][j + 1]] += 1
    for l in range(1, L + 1):
        c, R = box_geometry(P, perm, ranges[l])
        for (i, j) in far[l]:
            # brute-force admissibility
            assert i != j and np.linalg.norm(c[i] - c[j]) > eta * (R[i] + R[j])
            cover[ranges[l][i]:ranges[l][i + 1], ranges[l][j]:ranges[l][j + 1]] += 1
        for (i, j) in near[l]:
            assert i == j or not np.linalg.norm(c[i] - c[j]) > eta * (R[i] + R[j])
    assert (cover == 1).all()
    if eta == 0.0:
        for l in range(1, L + 1):  # HSS: only the diagonal is near
            assert near[l] == [(i, i) for i in range(1 << l)]


@pytest.mark.parametrize("eta", [0.0, 1.0, 2.0])
def test_lists_closed_under_transposition(eta):
    """Admissibility is symmetric in the two boxes, so every level's near and
    far lists hold (j, i) with (i, j): the library's symmetric storage and
    upper-pair projection pair each block with its mirror."""
    n, leaf = 600, 40
    P = W.cube_points(n, 11)
    perm, ranges = build_tree(P, leaf)
    near, far = interaction_lists(P, perm, ranges, eta)
    for l in range(1, len(ranges)):
        assert set(near[l]) == {(j, i) for (i, j) in near[l]}
        assert set(far[l]) == {(j, i) for (i, j) in far[l]}


def test_projected_blocks_of_symmetric_kernel_are_mirrors():
    """For a symmetric kernel every projected block is its mirror's
    transpose, Ahat_ji = Ahat_ij^T and Shat_ji = Shat_ij^T, on every level
    (the identity behind projecting the pairs i <= j only), while a
    non-symmetric change of one block breaks it."""
    P = W.cube_points(800, 4)
    H = construct(P, Kernel("yukawa_eps", diag_shift=1.0), 50, 1.0, 1e-8, 0, 256, 32)
    F = ulv.factor(H)
    for l in range(1, H["L"] + 1):
        A = F["Ahat"][l]
        for (i, j) in H["near"][l]:
            if i < j:
                scale = max(np.abs(A[(i, j)]).max(), 1e-300)
                assert np.abs(A[(j, i)] - A[(i, j)].T).max() <= 1e-12 * scale, (l, i, j)
        S = F["Shat"][l]
        for (i, j) in H["far"][l]:
            if i < j:
                scale = max(np.abs(S[(i, j)]).max(), 1e-300)
                assert np.abs(S[(j, i)] - S[(i, j)].T).max() <= 1e-12 * scale, (l, i, j)
    # the check is not vacuous: an off-diagonal block is not symmetric itself
    L = H["L"]
    (i, j) = next(p for p in H["near"][L] if p[0] < p[1])
    assert np.abs(F["Ahat"][L][(i, j)] - F["Ahat"][L][(i, j)].T).max() > 1e-6


# ------------------------------------------------------------ dense / LU ---
def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(0)
    for n in (1, 5, 33):
        A = rng.standard_normal((n, n))
        b = rng.standard_normal(n)
        assert np.allclose(dense.lu_solve(A, b), np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)
    # a case that needs pivoting
    A = np.array([[0.0, 1.0], [1.0, 1.0]])
    assert np.allclose(dense.lu_solve(A, np.array([1.0, 2.0])), [1.0, 1.0])


# --------------------------------------------------------------------- ID ---
def test_id_exact_on_low_rank_matrix():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((40, 7)) @ rng.standard_normal((7, 90))
    piv, R = interpolative_decomposition(M)
    X = id_basis(piv, R, 7)
    assert np.allclose(X[piv[:7]], np.eye(7))
    assert np.linalg.norm(M - X @ M[piv[:7]]) <= 1e-11 * np.linalg.norm(M)
    # fewer samples (columns) than rows still gives an n x k basis
    M2 = rng.standard_normal((30, 5))
    piv2, R2 = interpolative_decomposition(M2)
    assert R2.shape == (30, 30) and id_basis(piv2, R2, 5).shape == (30, 5)


def _poly2(n, leaf, eta=1.0, seed=1, shift=1.0, tol=1e-10):
    P = W.cube_points(n, seed)
    return construct(P, Kernel("poly2_test", diag_shift=shift), leaf, eta, tol, 0, 0, 0)


def test_exact_rank_kernel_ranks():
    H = _poly2(512, 64)
    assert all(H["K"][l] == 10 for l in range(1, H["L"] + 1))
    A = dense.dense_matrix(H["points"], H["kernel"])
    assert np.linalg.norm(dense.assemble_h2(H) - A) <= 1e-13 * np.linalg.norm(A)


# ------------------------------------------------------- complement bases ---
def test_complement_bases_orthogonal_and_span():
    P = W.cube_points(2048, 1)
    H = construct(P, Kernel("laplace_eps"), 64, 1.0, 1e-6, 0, 256, 32)
    U, T, _ = ulv.complement_bases(H)
    for l in range(1, H["L"] + 1):
        K = H["K"][l]
        for i in range(1 << l):
            Ui = U[l][i]
            assert np.abs(Ui.T @ Ui - np.eye(len(Ui))).max() <= 1e-13
            Xo = H["X"][l][i]
            if l < H["L"]:
                Kc = H["K"][l + 1]
                Xo = sla.block_diag(T[l + 1][2 * i], T[l + 1][2 * i + 1]) @ Xo
            # X = U^S T, and the redundant part is orthogonal to span(X)
            assert np.linalg.norm(Ui[:, -K:] @ T[l][i] - Xo) <= 1e-13 * np.linalg.norm(Xo)
            assert np.linalg.norm(Ui[:, :-K].T @ Xo) <= 1e-13 * np.linalg.norm(Xo)


# ------------------------------------------------------ whole pipeline ---
@pytest.mark.parametrize("n,leaf,eta", [(512, 64, 1.0), (1000, 64, 1.0), (700, 32, 0.0), (300, 40, 2.0)])
def test_exact_rank_pipeline_equals_dense_solve(n, leaf, eta):
    """On the rank-10 kernel the composite basis is exact, every term Eq. 21
    drops is zero and Eq. 31 equals Algorithm 3: the ULV solve must equal
    the dense solve to rounding."""
    H = _poly2(n, leaf, eta)
    F = ulv.factor(H)
    b = W.uniform_rhs(n, 2)
    A = dense.dense_matrix(H["points"], H["kernel"])
    xd = dense.lu_solve(A, b)
    for solver in (ulv.solve_parallel, ulv.solve_naive):
        x = solver(F, H, b)
        assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)
    for l, (drop, rr) in ulv.dropped_fill_norms(F).items():
        assert drop <= 1e-12 and rr <= 1e-12
    # the self Schur update (Algorithm 2, Eq. 21) is not trivial on this kernel
    lv = H["L"]
    R = H["D"][lv] - H["K"][lv]
    Aii = F["Ahat"][lv][(0, 0)]
    assert np.linalg.norm(Aii[:R, R:]) > 1e-3 * np.linalg.norm(Aii)


def test_dense_path_single_box():
    P = W.cube_points(50, 4)
    H = construct(P, Kernel("laplace_eps"), 64, 1.0, 1e-10)
    assert H["L"] == 0
    F = ulv.factor(H)
    b = W.uniform_rhs(50, 5)
    xd = np.linalg.solve(dense.dense_matrix(P, H["kernel"]), b)
    assert np.allclose(ulv.solve_parallel(F, H, b), xd, rtol=1e-12, atol=1e-14)


def test_parallel_vs_naive_differ_only_by_dropped_terms():
    P = W.cube_points(2048, 1)
    H = construct(P, Kernel("laplace_eps"), 64, 1.0, 1e-10, 0, 256, 32)
    F = ulv.factor(H)
    b = W.uniform_rhs(2048, 2)
    xp, xn = ulv.solve_parallel(F, H, b), ulv.solve_naive(F, H, b)
    rel = np.linalg.norm(xp - xn) / np.linalg.norm(xn)
    drop = max(rr for (_, rr) in ulv.dropped_fill_norms(F).values())
    assert 0 < rel <= 100 * drop


def test_basis_rotation_invariance():
    """The factorization depends only on the skeleton and redundant
    subspaces: rotating U^R and U^S inside themselves leaves x unchanged."""
    P = W.cube_points(1024, 3)
    H = construct(P, Kernel("laplace_eps"), 64, 1.0, 1e-6, 0, 256, 32)
    U, T, Shat = ulv.complement_bases(H)
    rng = np.random.default_rng(9)
    U2 = [None] + [u.copy() for u in U[1:]]
    T2 = [None] + [t.copy() for t in T[1:]]
    for l in range(1, H["L"] + 1):
        K, D = H["K"][l], H["D"][l]
        for i in range(1 << l):
            Qr = np.linalg.qr(rng.standard_normal((D - K, D - K)))[0]
            Qs = np.linalg.qr(rng.standard_normal((K, K)))[0]
            U2[l][i][:, :D - K] = U[l][i][:, :D - K] @ Qr
            U2[l][i][:, D - K:] = U[l][i][:, D - K:] @ Qs
            T2[l][i] = Qs.T @ T[l][i]
    # the children's coordinates change with Qs, so rebuild the parent bases
    # from the rotated T: X_p^orth = blockdiag(T2) X_p, whose span is rotated
    # consistently; recompute U and Shat level by level on top of T2.
    Hr = dict(H)
    U3, T3, S3 = [None] * (H["L"] + 1), [None] * (H["L"] + 1), [dict() for _ in range(H["L"] + 1)]
    for l in range(H["L"], 0, -1):
        K, D = H["K"][l], H["D"][l]
        U3[l] = np.zeros_like(U[l])
        T3[l] = np.zeros_like(T[l])
        for i in range(1 << l):
            Xo = H["X"][l][i]
            if l < H["L"]:
                Xo = sla.block_diag(T3[l + 1][2 * i], T3[l + 1][2 * i + 1]) @ Xo
            Q, Rf = np.linalg.qr(Xo, mode="complete")
            Qr = np.linalg.qr(rng.standard_normal((D - K, D - K)))[0]
            Qs = np.linalg.qr(rng.standard_normal((K, K)))[0]
            U3[l][i] = np.hstack([Q[:, K:] @ Qr, Q[:, :K] @ Qs])
            T3[l][i] = Qs.T @ Rf[:K, :K]
        for (i, j), Sij in H["S"][l].items():
            S3[l][(i, j)] = T3[l][i] @ Sij @ T3[l][j].T
    b = W.uniform_rhs(1024, 4)
    x1 = ulv.solve_parallel(ulv.factor(H), H, b)
    x2 = ulv.solve_parallel(ulv.factor(Hr, (U3, T3, S3)), Hr, b)
    assert np.linalg.norm(x1 - x2) <= 1e-11 * np.linalg.norm(x1)


# ------------------------------------------------------- matvec / refine ---
@pytest.mark.parametrize("n,leaf,eta", [(1000, 64, 1.0), (700, 32, 0.0)])
def test_matvec_equals_assembled_h2(n, leaf, eta):
    P = W.sphere_points(n, 5)
    H = construct(P, Kernel("laplace_eps"), leaf, eta, 1e-6, 0, 128, 16)
    x = W.uniform_rhs(n, 6)
    Ah = dense.assemble_h2(H)
    y = ulv.matvec(H, x)
    assert np.linalg.norm(y - Ah @ x) <= 1e-13 * np.linalg.norm(Ah @ x)
    if eta > 0:  # HSS at a capped rank is a poor approximation (Section 6.3)
        A = dense.dense_matrix(P, H["kernel"])
        assert np.linalg.norm(Ah - A) <= 1e-3 * np.linalg.norm(A)


def test_refinement_reaches_target_and_dense_solution():
    wl = W.workload("cube2048_laplace")
    P = wl.points()
    H = construct(P, Kernel(wl.kernel), wl.leaf, wl.eta, wl.tol, 0, 512, 64)
    F = ulv.factor(H)
    b = wl.rhs()
    x, hist = ulv.refine(F, H, b, 1e-10, 30)
    assert hist[-1] <= 1e-10 and len(hist) <= 12
    assert all(hist[k + 1] < hist[k] for k in range(len(hist) - 1))
    A = dense.dense_matrix(P, H["kernel"])
    xd = np.linalg.solve(A, b)
    err_h2 = np.linalg.norm(dense.assemble_h2(H) - A) / np.linalg.norm(A)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 100 * err_h2


def test_gmres_refinement_matches_plain_refinement():
    """FGMRES-based refinement reaches the same solution as plain refinement
    with no more preconditioner applications; on the exact-rank kernel one
    application suffices."""
    wl = W.workload("cube2048_laplace")
    P = wl.points()
    H = construct(P, Kernel(wl.kernel), wl.leaf, wl.eta, wl.tol, 0, 512, 64)
    F = ulv.factor(H)
    b = wl.rhs()
    x1, h1 = ulv.refine(F, H, b, 1e-11, 40)
    x2, h2, its = ulv.refine_gmres(F, H, b, 1e-11, 40, 30)
    assert h2[-1] <= 1e-11 and its <= len(h1) - 1
    assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x1)
    Hp = _poly2(512, 64)
    Fp = ulv.factor(Hp)
    bp = W.uniform_rhs(512, 3)
    xp, hp, itp = ulv.refine_gmres(Fp, Hp, bp, 1e-11, 10, 5)
    assert itp == 1 and hp[-1] <= 1e-11


def test_residual_tracks_tolerance():
    """With no rank cap and no sampling, the dense residual ||Ax - b|| / ||b||
    of the refined H^2 solution falls with the truncation tolerance and stays
    below it (sphere surface)."""
    n = 1024
    P = W.sphere_points(n, 8)
    kern = Kernel("laplace_eps")
    A = dense.dense_matrix(P, kern)
    b = W.uniform_rhs(n, 9)
    tols = (1e-2, 1e-4, 1e-6, 1e-8)
    res = []
    for tol in tols:
        H = construct(P, kern, 64, 1.0, tol, 10 ** 6, 0, 0)
        F = ulv.factor(H)
        x, hist = ulv.refine(F, H, b, 1e-13, 40)
        assert hist[-1] <= 1e-13
        res.append(np.linalg.norm(A @ x - b) / np.linalg.norm(b))
    assert all(res[k + 1] < res[k] for k in range(len(res) - 1))
    assert all(r <= t for r, t in zip(res, tols))


def test_hss_needs_higher_rank_than_h2():
    """Section 6.3: at the same tolerance, eta = 0 (HSS) needs higher ranks
    than eta = 1 (H^2)."""
    P = W.sphere_points(2048, 12)
    kern = Kernel("laplace_eps")
    h2 = construct(P, kern, 128, 1.0, 1e-6, 128, 0, 0)
    hss = construct(P, kern, 128, 0.0, 1e-6, 128, 0, 0)
    L = h2["L"]
    assert max(hss["ranks"][L]) > max(h2["ranks"][L]) or np.mean(hss["ranks"][L]) > np.mean(h2["ranks"][L])


def test_prefactor_basis_bounds_dropped_fill():
    """Section 3.4, Eq. 21-23: with the close-field term G(B_i, S_C)
    G(S_C, S_C)^-1 in the composite matrix, the Schur fill-ins the
    factorization drops (Eq. 10-12, the terms Eq. 21 sets to zero) fall with
    the truncation tolerance, and one ULV application (no refinement) is the
    dense solve to within the tolerance.  With the term left out (the plain
    H^2 basis of Fig. 7) the dropped fill-ins stay at the 1e-2 level whatever
    the tolerance.  Real kernel (1/(r+1e-3) on a sphere), no rank cap, no
    sampling."""
    n = 1024
    P = W.sphere_points(n, 8)
    kern = Kernel("laplace_eps")
    A = dense.dense_matrix(P, kern)
    b = W.uniform_rhs(n, 9)
    xd = np.linalg.solve(A, b)

    def run(tol, prefactor):
        H = construct(P, kern, 64, 1.0, tol, 10 ** 6, 0, 0, prefactor=prefactor)
        F = ulv.factor(H)
        drop = max(v[0] for v in ulv.dropped_fill_norms(F).values())
        x = ulv.solve_parallel(F, H, b)
        return drop, np.linalg.norm(x - xd) / np.linalg.norm(xd)

    tols = (1e-3, 1e-5, 1e-7)
    got = [run(t, True) for t in tols]
    for (drop, err), tol in zip(got, tols):
        assert drop <= 0.5 * tol, (tol, drop)
        assert err <= tol, (tol, err)
    assert got[0][0] > got[1][0] > got[2][0]
    drop_far, err_far = run(1e-7, False)
    assert drop_far >= 1e4 * got[2][0] and drop_far >= 1e-3
    assert err_far >= 1e3 * got[2][1]


def test_prefactor_term_scales_with_inverse_diagonal():
    """The close-field content of Eq. 22-23 is A_ji A_ii^-1.  With a diagonal
    shift of 1e6 (A_ii^-1 ~ 1e-6 I) that content lies far below the far
    field's at tol 1e-3 and 1e-5, so the leaf ranks equal those of the
    far-field-only basis exactly; with the plain diagonal (1e3) the
    pre-factorization basis needs strictly more rank.  (A close-field term
    without the inverse would keep the block at full weight and raise the
    ranks in the shifted case too.)"""
    P = W.sphere_points(1024, 8)
    for tol in (1e-3, 1e-5):
        for shift, same in ((1e6, True), (0.0, False)):
            kern = Kernel("laplace_eps", diag_shift=shift)
            Hp = construct(P, kern, 64, 1.0, tol, 10 ** 6, 0, 0, prefactor=True)
            Hf = construct(P, kern, 64, 1.0, tol, 10 ** 6, 0, 0, prefactor=False)
            L = Hp["L"]
            if same:
                assert list(Hp["ranks"][L]) == list(Hf["ranks"][L]), (tol, shift)
            else:
                assert max(Hp["ranks"][L]) > max(Hf["ranks"][L]), (tol, shift)
