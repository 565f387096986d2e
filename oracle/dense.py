"""Dense reference pieces (oracle; FP64).

  dense_matrix   the full kernel matrix G(P, P) in original point order
  lu_solve       textbook Gaussian elimination with partial pivoting (row
                 interchanges choose the largest |pivot| in the column), written
                 out so that a test can compare it with numpy.linalg.solve
  assemble_h2    the H^2 matrix A_H2 written out densely: leaf near blocks plus,
                 for every far pair (i, j) of level l, E_i S_ij E_j^T with the
                 expanded nested basis E (E_i = X_i at the leaves,
                 E_p = blockdiag(E_2p, E_2p+1) X_p above them)
"""
from __future__ import annotations

import numpy as np


def dense_matrix(points: np.ndarray, kernel) -> np.ndarray:
    idx = np.arange(len(points))
    return kernel.matrix(points, idx, idx)


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = np.array(A, dtype=np.float64, copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    n = A.shape[0]
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0.0:
            raise np.linalg.LinAlgError("singular matrix")
        if p != k:
            A[[k, p]] = A[[p, k]]
            x[[k, p]] = x[[p, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
        x[k + 1:] -= A[k + 1:, k][:, None] * x[k] if x.ndim > 1 else A[k + 1:, k] * x[k]
    for k in range(n - 1, -1, -1):
        x[k] = (x[k] - A[k, k + 1:] @ x[k + 1:]) / A[k, k]
    return x


def assemble_h2(H) -> np.ndarray:
    N, L = H["N"], H["L"]
    D, K = H["D"], H["K"]
    rg = H["ranges"]
    perm = H["perm"]
    At = np.zeros((N, N))  # tree order
    if L == 0:
        At[:, :] = H["A"][(0, 0)][:N, :N]
    else:
        for (i, j), blk in H["A"].items():
            ni, nj = rg[L][i + 1] - rg[L][i], rg[L][j + 1] - rg[L][j]
            At[rg[L][i]:rg[L][i + 1], rg[L][j]:rg[L][j + 1]] = blk[:ni, :nj]
        E = [None] * (L + 1)
        E[L] = [H["X"][L][i][:rg[L][i + 1] - rg[L][i]] for i in range(1 << L)]
        for l in range(L - 1, 0, -1):
            E[l] = []
            for p in range(1 << l):
                a, b = E[l + 1][2 * p], E[l + 1][2 * p + 1]
                Bd = np.zeros((a.shape[0] + b.shape[0], a.shape[1] + b.shape[1]))
                Bd[:a.shape[0], :a.shape[1]] = a
                Bd[a.shape[0]:, a.shape[1]:] = b
                E[l].append(Bd @ H["X"][l][p])
        for l in range(1, L + 1):
            for (i, j), Sij in H["S"][l].items():
                At[rg[l][i]:rg[l][i + 1], rg[l][j]:rg[l][j + 1]] = E[l][i] @ Sij @ E[l][j].T
    out = np.zeros((N, N))
    out[np.ix_(perm, perm)] = At
    return out
