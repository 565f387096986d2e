"""H^2 construction with the pre-factorization (composite) basis (oracle; FP64).

Algorithm 1 (Section 3.5), level by level from the leaves to level 1:

  * For every box i, sample its far field S_F and its close field S_C, and
    row-compress the composite matrix
        M_i = [ G(B_i, S_F) | G(B_i, S_C^(j)) G(S_C^(j), S_C^(j))^-1  for each close j != i ]
    by an interpolative decomposition (ID).  The far part is the ordinary H^2
    low-rank content (Fig. 7); the close part approximates A_ji A_ii^-1, the
    factorization basis of Eq. 22-23 (Fig. 8).  Box i itself is left out of
    the close part: G(B_i, B_i) G(B_i, B_i)^-1 is the identity, which has full
    rank.  One solve per close box follows the A_ji A_ii^-1 form of
    Section 3.4.
  * The ID is a column-pivoted QR of M_i^T: M_i^T P = Q R.  The first k pivots
    are the skeleton SK_i and X_i = P [I; (R_11^-1 R_12)^T] is the basis, so
    that M_i ~= X_i M_i[SK_i, :].
  * Dense near blocks G(B_i, B_j) at the leaf level and couplings
    S_ij = G(SK_i, SK_j) for far pairs.
  * The points of box i at level l-1 are the skeletons (SK_2i, SK_2i+1).

Readings of what the paper leaves open:
  * Rank: k_i = #{t : |R_tt| > tol * |R_11|}.  Following the constant-rank
    batches of Section 4.1 (and the constant rank of Section 5), every box of
    a level keeps the same rank K_l = max_i k_i, capped by max_rank (0 means
    half the level's box dimension, so no level grows past the leaf size) and
    by the smallest box of the level.
  * Sampling: the far field of box i is every point outside the union of its
    near boxes (at any level, in original coordinates).  A sample of size s
    from a list of length n takes entries floor(t * n / s), t = 0..s-1, of the
    list in tree order; s = min(n, far_samples) for the far field and
    s = min(n_j, near_samples) for each close box j.  A sample size <= 0 means
    no sampling.  This rule is not fixed by the paper ("parity unpinned").
  * Leaf padding: every leaf block is padded to D_L = max leaf size.  Padded
    rows of X are zero, padded diagonal entries of A_ii are 1 and all other
    padded entries 0 (the padding of Section 4.1, written directly).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .kernels import Kernel
from .tree import build_tree, interaction_lists


def stride_sample(idx: np.ndarray, s: int) -> np.ndarray:
    n = len(idx)
    if s <= 0 or s >= n:
        return idx
    t = np.arange(s, dtype=np.int64)
    return idx[(t * n) // s]


def interpolative_decomposition(M: np.ndarray):
    """Column-pivoted QR of M^T.  Returns (piv, R) with M^T[:, piv] = Q R."""
    n = M.shape[0]
    MT = M.T
    if MT.shape[0] < n:  # fewer samples than rows: pad with zero rows
        MT = np.vstack([MT, np.zeros((n - MT.shape[0], n))])
    R, piv = sla.qr(MT, mode="r", pivoting=True)
    return piv, R[:n, :]


def id_basis(piv: np.ndarray, R: np.ndarray, k: int) -> np.ndarray:
    """X = P [I; (R_11^-1 R_12)^T], shape (n, k)."""
    n = R.shape[1]
    R11 = R[:k, :k]
    R12 = R[:k, k:]
    d = np.abs(np.diag(R11))
    if k == 0:
        T = np.zeros((0, n))
    elif d.min() > 0.0:
        T = sla.solve_triangular(R11, R12, lower=False)
    else:
        # R_11 singular (the level rank exceeds this box's rank): a
        # least-squares solution of R_11 T = R_12 keeps the ID exact.
        T = sla.lstsq(R11, R12)[0]
    X = np.zeros((n, k))
    X[piv[:k], :] = np.eye(k)
    X[piv[k:], :] = T.T
    return X


def construct(points: np.ndarray, kernel: Kernel, leaf: int, eta: float, tol: float,
              max_rank: int = 0, far_samples: int = 1024, near_samples: int = 64, prefactor: bool = True):
    """Algorithm 1.  prefactor=False leaves the close-field part out of M_i
    (the plain H^2 basis of Fig. 7, without the fill-in content of Eq. 22-23);
    the tests use it to show what the pre-factorization term contributes."""
    points = np.ascontiguousarray(points, dtype=np.float64)
    N = len(points)
    perm, ranges = build_tree(points, leaf)
    near, far = interaction_lists(points, perm, ranges, eta)
    L = len(ranges) - 1

    leaf_sizes = np.diff(ranges[L])
    D = [0] * (L + 1)
    K = [0] * (L + 1)
    D[L] = int(leaf_sizes.max()) if N else 0
    box_pts = [None] * (L + 1)
    box_pts[L] = [perm[ranges[L][i]:ranges[L][i + 1]] for i in range(1 << L)]
    X = [None] * (L + 1)
    SK = [None] * (L + 1)
    S = [dict() for _ in range(L + 1)]
    ranks = [None] * (L + 1)

    for l in range(L, 0, -1):
        nb = 1 << l
        nbrs = [[] for _ in range(nb)]
        for (i, j) in near[l]:
            nbrs[i].append(j)
        pivs, Rs, ks = [], [], []
        for i in range(nb):
            Pi = box_pts[l][i]
            # far field: every point outside the near boxes of i (tree order)
            mask = np.ones(N, dtype=bool)
            for j in nbrs[i]:
                mask[ranges[l][j]:ranges[l][j + 1]] = False
            SF = stride_sample(perm[mask], far_samples)
            parts = [kernel.matrix(points, Pi, SF)]
            for j in nbrs[i]:
                if j == i or not prefactor:
                    continue
                SC = stride_sample(box_pts[l][j], near_samples)
                Acc = kernel.matrix(points, SC, SC)
                Bic = kernel.matrix(points, Pi, SC)
                parts.append(sla.solve(Acc, Bic.T).T)  # G(B_i,S_C) G(S_C,S_C)^-1 (G symmetric)
            M = np.hstack(parts)
            piv, R = interpolative_decomposition(M)
            dg = np.abs(np.diag(R))
            k = int(np.sum(dg > tol * dg[0])) if len(dg) and dg[0] > 0 else 0
            pivs.append(piv)
            Rs.append(R)
            ks.append(k)
        cap = max_rank if max_rank > 0 else D[l] // 2
        nmin = min(len(p) for p in box_pts[l])
        K[l] = max(1, min(max(ks), cap, nmin)) if nmin > 0 else 0
        ranks[l] = ks
        X[l] = np.zeros((nb, D[l], K[l]))
        SK[l] = np.zeros((nb, K[l]), dtype=np.int64)
        for i in range(nb):
            Xi = id_basis(pivs[i], Rs[i], K[l])
            X[l][i, :Xi.shape[0], :] = Xi
            SK[l][i] = box_pts[l][i][pivs[i][:K[l]]]
        for (i, j) in far[l]:
            S[l][(i, j)] = kernel.matrix(points, SK[l][i], SK[l][j])
        # points of the parent boxes: the children's skeletons
        box_pts[l - 1] = [np.concatenate([SK[l][2 * p], SK[l][2 * p + 1]]) for p in range(nb // 2)]
        D[l - 1] = 2 * K[l]
    if L == 0:
        D[0] = N

    # dense near blocks of the leaf level, padded to D_L
    A = {}
    for (i, j) in near[L]:
        Pi, Pj = box_pts[L][i], box_pts[L][j]
        blk = np.zeros((D[L], D[L]))
        blk[:len(Pi), :len(Pj)] = kernel.matrix(points, Pi, Pj)
        if i == j:
            for t in range(len(Pi), D[L]):
                blk[t, t] = 1.0
        A[(i, j)] = blk

    return dict(points=points, kernel=kernel, N=N, L=L, leaf=leaf, eta=eta, tol=tol,
                perm=perm, ranges=ranges, near=near, far=far, D=D, K=K,
                box_pts=box_pts, X=X, SK=SK, S=S, A=A, ranks=ranks)
