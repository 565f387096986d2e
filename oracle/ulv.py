"""Level-by-level H^2-ULV factorization and substitution (oracle; FP64).

Notation (per level l): nb_l = 2^l boxes, box dimension D_l, skeleton rank
K_l, redundant size R_l = D_l - K_l.  Box i's full basis is the orthogonal
U_i = [U_i^R  U_i^S] (Eq. 7), so U_i^-1 = U_i^T.  A projected block
Ahat_ij = U_i^T A_ij U_j splits into the RR, RS, SR and SS parts of Eq. 7
(rows R first, then S).

Steps, in the order of Algorithm 4 (partial-pivot LU in place of the paper's
Cholesky; for symmetric positive definite blocks both give the same solution):

  complement_bases  Eq. 6-7: QR of the skeleton basis gives U_i and T_i with
                    X_i = U_i^S T_i.  Above the leaves the basis lives in the
                    children's skeleton coordinates:
                    X_p^orth = blockdiag(T_2p, T_2p+1) X_p  (from
                    A ~= X_c S X_d^T = U_c^S (T_c S T_d^T) U_d^S^T).
  factor            for l = L..1:
                      Ahat_ij = U_i^T A_ij U_j for every near pair        (Alg. 2: projection)
                      P_i L_i U_i' = Ahat_ii^RR                          (Alg. 2: RR LU)
                      Z_i = (Ahat_ii^RR)^-1 Ahat_ii^RS                   (Alg. 2: RS solve)
                      Ahat_ii^SS -= Ahat_ii^SR Z_i                       (Alg. 2: Schur, Eq. 21)
                      Shat_ij = T_i S_ij T_j^T for every far pair        (Alg. 2: couplings)
                      merge the children's SS / Shat blocks into the
                      parent's near blocks                               (Alg. 2: merge)
                    then LU of the root block                            (Alg. 2: root)
                    Every fill-in other than the self Schur update is
                    dropped, as Eq. 10-12 / Eq. 21 state.
  solve_naive       Algorithm 3 (block triangular solve with the factors,
                    serial within a level) and its mirror image.
  solve_parallel    the product form of L^-1 of Eq. 24-31: triangular solves
                    only on the diagonal blocks, matrix-vector products for
                    the off-diagonal blocks; the backward pass is its mirror
                    image (Section 3.7 gives only the forward pass).
  matvec            y = A_H2 x with the nested ID bases (upward pass,
                    couplings, downward pass, dense near blocks).
  refine            iterative refinement: r = b - A_H2 x, x += ULV^-1 r.

With LU factors Ahat_ii^RR = P_i L_i U'_i the lower factor blocks are
L(r)_ij = Ahat_ij^RR U'_j^-1 (i > j), L(s)_ij = Ahat_ij^SR U'_j^-1, and the
upper ones U(r)_ij = (P_i L_i)^-1 Ahat_ij^RR (i < j),
U(s)_ij = (P_i L_i)^-1 Ahat_ij^RS (Eq. 32 with the LU split).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------
# a1: complement bases (Eq. 6-7)
# ----------------------------------------------------------------------------
def complement_bases(H):
    """Return (U, T, Shat): U[l] (nb, D, D) = [U^R U^S], T[l] (nb, K, K),
    Shat[l] dict of far-pair couplings in orthogonal coordinates."""
    L = H["L"]
    U = [None] * (L + 1)
    T = [None] * (L + 1)
    Shat = [dict() for _ in range(L + 1)]
    for l in range(L, 0, -1):
        nb, D, K = 1 << l, H["D"][l], H["K"][l]
        U[l] = np.zeros((nb, D, D))
        T[l] = np.zeros((nb, K, K))
        for i in range(nb):
            Xi = H["X"][l][i]
            if l < L:
                Kc = H["K"][l + 1]
                Tc = np.zeros((2 * Kc, 2 * Kc))
                Tc[:Kc, :Kc] = T[l + 1][2 * i]
                Tc[Kc:, Kc:] = T[l + 1][2 * i + 1]
                Xi = Tc @ Xi
            Q, Rf = np.linalg.qr(Xi, mode="complete")
            U[l][i] = np.hstack([Q[:, K:], Q[:, :K]])
            T[l][i] = Rf[:K, :K]
        for (i, j), Sij in H["S"][l].items():
            Shat[l][(i, j)] = T[l][i] @ Sij @ T[l][j].T
    return U, T, Shat


# ----------------------------------------------------------------------------
# factorization (Algorithm 2 / 4 with LU)
# ----------------------------------------------------------------------------
def factor(H, bases=None):
    """Factor the H^2 matrix H.  ``bases`` = (U, T, Shat) overrides the
    complement bases (used to check basis-rotation invariance)."""
    L = H["L"]
    U, T, Shat = complement_bases(H) if bases is None else bases
    F = dict(U=U, T=T, Shat=Shat, Ahat=[None] * (L + 1), lu=[None] * (L + 1), L=L,
             D=H["D"], K=H["K"], near=H["near"], far=H["far"])
    A = dict(H["A"])  # the current level's near blocks
    for l in range(L, 0, -1):
        nb, D, K = 1 << l, H["D"][l], H["K"][l]
        R = D - K
        Ahat = {}
        for (i, j) in H["near"][l]:
            Ahat[(i, j)] = U[l][i].T @ A[(i, j)] @ U[l][j]
        lus = []
        for i in range(nb):
            Aii = Ahat[(i, i)]
            P, Lo, Up = sla.lu(Aii[:R, :R])
            lus.append((P, Lo, Up))
            if R and K:
                Y = sla.solve_triangular(Lo, P.T @ Aii[:R, R:], lower=True, unit_diagonal=True)
                Z = sla.solve_triangular(Up, Y, lower=False)
                Aii[R:, R:] = Aii[R:, R:] - Aii[R:, :R] @ Z
        F["Ahat"][l] = Ahat
        F["lu"][l] = lus
        # merge into the parent's near blocks
        nearset = set(H["near"][l])
        A = {}
        for (p, q) in H["near"][l - 1]:
            blk = np.zeros((2 * K, 2 * K))
            for a in (0, 1):
                for b in (0, 1):
                    c, d = 2 * p + a, 2 * q + b
                    sub = Ahat[(c, d)][R:, R:] if (c, d) in nearset else Shat[l][(c, d)]
                    blk[a * K:(a + 1) * K, b * K:(b + 1) * K] = sub
            A[(p, q)] = blk
    F["root"] = sla.lu(A[(0, 0)]) if A[(0, 0)].size else None
    F["root_A"] = A[(0, 0)]
    return F


# ----------------------------------------------------------------------------
# helpers for the triangular pieces of the LU of Ahat_ii^RR = P L U'
# ----------------------------------------------------------------------------
def _solve_PL(lu, v):
    P, Lo, _ = lu
    return sla.solve_triangular(Lo, P.T @ v, lower=True, unit_diagonal=True)


def _solve_U(lu, v):
    return sla.solve_triangular(lu[2], v, lower=False)


def _root_solve(F, v):
    if F["root"] is None:
        return v
    P, Lo, Up = F["root"]
    return sla.solve_triangular(Up, sla.solve_triangular(Lo, P.T @ v, lower=True, unit_diagonal=True))


def to_tree(H, b):
    """Original order -> padded leaf-box vector (nb_L * D_L)."""
    L, D = H["L"], H["D"][H["L"]]
    rg = H["ranges"][L]
    out = np.zeros(((1 << L) * D,) + b.shape[1:])
    bt = b[H["perm"]]
    for i in range(1 << L):
        n = rg[i + 1] - rg[i]
        out[i * D:i * D + n] = bt[rg[i]:rg[i + 1]]
    return out


def from_tree(H, v):
    L, D = H["L"], H["D"][H["L"]]
    rg = H["ranges"][L]
    bt = np.zeros((H["N"],) + v.shape[1:])
    for i in range(1 << L):
        n = rg[i + 1] - rg[i]
        bt[rg[i]:rg[i + 1]] = v[i * D:i * D + n]
    out = np.zeros_like(bt)
    out[H["perm"]] = bt
    return out


def _nbrs(pairs, nb):
    out = [[] for _ in range(nb)]
    for (i, j) in pairs:
        out[i].append(j)
    return out


# ----------------------------------------------------------------------------
# substitution: naive (Algorithm 3 and its mirror)
# ----------------------------------------------------------------------------
def solve_naive(F, H, b):
    L = F["L"]
    vec = to_tree(H, b)
    ys = [None] * (L + 1)
    for l in range(L, 0, -1):
        nb, D, K = 1 << l, F["D"][l], F["K"][l]
        R = D - K
        U, Ah, lus = F["U"][l], F["Ahat"][l], F["lu"][l]
        nbr = _nbrs(F["near"][l], nb)
        c = [U[i].T @ vec[i * D:(i + 1) * D] for i in range(nb)]     # Alg. 3: c_i = U_i^T b_i
        bR = [ci[:R].copy() for ci in c]
        bS = [ci[R:].copy() for ci in c]
        for i in range(nb):                                           # Alg. 3: redundant parts
            bR[i] = _solve_PL(lus[i], bR[i])
            ui = _solve_U(lus[i], bR[i])                              # U'_ii^-1 y_i
            for j in nbr[i]:
                if j > i:
                    bR[j] = bR[j] - Ah[(j, i)][:R, :R] @ ui           # L(r)_ji y_i
            for j in nbr[i]:
                bS[j] = bS[j] - Ah[(j, i)][R:, :R] @ ui               # L(s)_ji y_i
        ys[l] = bR
        vec = np.concatenate(bS) if K else np.zeros(0)                # Alg. 3: skeletons to the parent
    xs = _root_solve(F, vec)
    for l in range(1, L + 1):
        nb, D, K = 1 << l, F["D"][l], F["K"][l]
        R = D - K
        U, Ah, lus = F["U"][l], F["Ahat"][l], F["lu"][l]
        nbr = _nbrs(F["near"][l], nb)
        xS = [xs[i * K:(i + 1) * K] for i in range(nb)]
        w = []
        for i in range(nb):
            t = np.zeros(R)
            for j in nbr[i]:
                t = t + Ah[(i, j)][:R, R:] @ xS[j]
            w.append(ys[l][i] - _solve_PL(lus[i], t))                 # y - U(s) x^S
        xR = [None] * nb
        for i in range(nb - 1, -1, -1):
            xR[i] = _solve_U(lus[i], w[i])
            for j in nbr[i]:
                if j < i:
                    w[j] = w[j] - _solve_PL(lus[j], Ah[(j, i)][:R, :R] @ xR[i])   # U(r)_ji x_i
        xs = np.concatenate([U[i] @ np.concatenate([xR[i], xS[i]]) for i in range(nb)])
    return from_tree(H, xs)


# ----------------------------------------------------------------------------
# substitution: parallel product form (Eq. 24-31 and its mirror)
# ----------------------------------------------------------------------------
def forward_parallel(F, vec, l):
    """One level of the forward pass: returns (y, s) per box, s = the S part
    passed to the parent."""
    nb, D, K = 1 << l, F["D"][l], F["K"][l]
    R = D - K
    U, Ah, lus = F["U"][l], F["Ahat"][l], F["lu"][l]
    nbr = _nbrs(F["near"][l], nb)
    c = [U[i].T @ vec[i * D:(i + 1) * D] for i in range(nb)]
    u = [_solve_U(lus[i], _solve_PL(lus[i], c[i][:R])) for i in range(nb)]  # (Ahat_ii^RR)^-1 b_i^R
    y, v = [], []
    for i in range(nb):
        bi = c[i][:R].copy()
        for j in nbr[i]:
            if j < i:
                bi = bi - Ah[(i, j)][:R, :R] @ u[j]        # -L(r)_ij L_jj^-1 b_j  (Eq. 31)
        y.append(_solve_PL(lus[i], bi))                   # L_ii^-1 (...)
        v.append(_solve_U(lus[i], y[i]))
    s = []
    for i in range(nb):
        si = c[i][R:].copy()
        for j in nbr[i]:
            si = si - Ah[(i, j)][R:, :R] @ v[j]            # -L(s)_ij y_j
        s.append(si)
    return y, s


def backward_parallel(F, y, xs, l):
    nb, D, K = 1 << l, F["D"][l], F["K"][l]
    R = D - K
    U, Ah, lus = F["U"][l], F["Ahat"][l], F["lu"][l]
    nbr = _nbrs(F["near"][l], nb)
    xS = [xs[i * K:(i + 1) * K] for i in range(nb)]
    w = []
    for i in range(nb):
        t = np.zeros(R)
        for j in nbr[i]:
            t = t + Ah[(i, j)][:R, R:] @ xS[j]
        w.append(y[i] - _solve_PL(lus[i], t))              # y - U(s) x^S
    om = [_solve_U(lus[i], w[i]) for i in range(nb)]       # U'_jj^-1 w_j
    out = []
    for i in range(nb):
        q = np.zeros(R)
        for j in nbr[i]:
            if j > i:
                q = q + Ah[(i, j)][:R, :R] @ om[j]
        xR = _solve_U(lus[i], w[i] - _solve_PL(lus[i], q))  # mirror of Eq. 31
        out.append(U[i] @ np.concatenate([xR, xS[i]]))
    return np.concatenate(out)


def solve_parallel(F, H, b):
    L = F["L"]
    vec = to_tree(H, b)
    ys = [None] * (L + 1)
    for l in range(L, 0, -1):
        ys[l], s = forward_parallel(F, vec, l)
        vec = np.concatenate(s) if F["K"][l] else np.zeros(0)
    xs = _root_solve(F, vec)
    for l in range(1, L + 1):
        xs = backward_parallel(F, ys[l], xs, l)
    return from_tree(H, xs)


# ----------------------------------------------------------------------------
# H^2 matrix-vector product (FP64), the operator the refinement targets
# ----------------------------------------------------------------------------
def matvec(H, x):
    L = H["L"]
    xt = to_tree(H, x)
    if L == 0:
        return from_tree(H, H["A"][(0, 0)] @ xt)
    xhat = [None] * (L + 1)
    D, K = H["D"], H["K"]
    xhat[L] = [H["X"][L][i].T @ xt[i * D[L]:(i + 1) * D[L]] for i in range(1 << L)]
    for l in range(L - 1, 0, -1):
        xhat[l] = [H["X"][l][p].T @ np.concatenate([xhat[l + 1][2 * p], xhat[l + 1][2 * p + 1]])
                   for p in range(1 << l)]
    yhat = [None] * (L + 1)
    for l in range(1, L + 1):
        yhat[l] = [np.zeros(K[l]) for _ in range(1 << l)]
        for (i, j), Sij in H["S"][l].items():
            yhat[l][i] = yhat[l][i] + Sij @ xhat[l][j]
    for l in range(1, L):
        for p in range(1 << l):
            t = H["X"][l][p] @ yhat[l][p]
            yhat[l + 1][2 * p] = yhat[l + 1][2 * p] + t[:K[l + 1]]
            yhat[l + 1][2 * p + 1] = yhat[l + 1][2 * p + 1] + t[K[l + 1]:]
    y = np.zeros_like(xt)
    for i in range(1 << L):
        y[i * D[L]:(i + 1) * D[L]] = H["X"][L][i] @ yhat[L][i]
    for (i, j) in H["near"][L]:
        y[i * D[L]:(i + 1) * D[L]] += H["A"][(i, j)] @ xt[j * D[L]:(j + 1) * D[L]]
    return from_tree(H, y)


def refine(F, H, b, target=1e-10, max_iters=50, solver=solve_parallel):
    """Iterative refinement: x_0 = 0; r = b - A_H2 x; x += ULV^-1 r until
    ||r|| / ||b|| <= target.  Returns (x, history of relative residuals)."""
    x = np.zeros_like(b)
    nb_ = np.linalg.norm(b)
    r = b.copy()
    hist = [1.0]
    for _ in range(max_iters):
        x = x + solver(F, H, r)
        r = b - matvec(H, x)
        hist.append(float(np.linalg.norm(r) / nb_))
        if hist[-1] <= target:
            break
    return x, hist


def refine_gmres(F, H, b, target=1e-10, max_iters=100, restart=30, solver=solve_parallel):
    """GMRES-based iterative refinement: restarted, right-preconditioned
    flexible GMRES on A_H2 x = b with the ULV factorization as the
    preconditioner (z_j = ULV^-1 v_j, w = A_H2 z_j), modified Gram-Schmidt
    and Givens rotations; after each cycle x += Z y and the true residual
    r = b - A_H2 x is recomputed in FP64.  max_iters counts preconditioner
    applications.  Returns (x, relative residual after every cycle, total
    preconditioner applications)."""
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    beta = bn
    hist = [1.0]
    its = 0
    while its < max_iters and beta > target * bn:
        m = min(restart, max_iters - its)
        V = [r / beta]
        Z = []
        Hs = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            Z.append(solver(F, H, V[j]))
            w = matvec(H, Z[j])
            for i in range(j + 1):
                Hs[i, j] = w @ V[i]
                w = w - Hs[i, j] * V[i]
            Hs[j + 1, j] = np.linalg.norm(w)
            V.append(w / Hs[j + 1, j] if Hs[j + 1, j] > 0 else w)
            for i in range(j):  # previous rotations
                t = cs[i] * Hs[i, j] + sn[i] * Hs[i + 1, j]
                Hs[i + 1, j] = -sn[i] * Hs[i, j] + cs[i] * Hs[i + 1, j]
                Hs[i, j] = t
            d = np.hypot(Hs[j, j], Hs[j + 1, j])
            cs[j], sn[j] = Hs[j, j] / d, Hs[j + 1, j] / d
            Hs[j, j] = d
            Hs[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            its += 1
            if abs(g[j + 1]) <= target * bn:
                break
        y = sla.solve_triangular(Hs[:k, :k], g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - matvec(H, x)
        beta = np.linalg.norm(r)
        hist.append(float(beta / bn))
    return x, hist, its


# ----------------------------------------------------------------------------
# Eq. 21 diagnostics: the size of the fill-ins the factorization drops
# ----------------------------------------------------------------------------
def dropped_fill_norms(F):
    """Per level, the largest dropped Schur fill-in of Eq. 10-12,
    ||Ahat_ji^SR (Ahat_ii^RR)^-1 Ahat_ik^RS|| over (j, k) != (i, i), and the
    largest dropped RR fill-in ||Ahat_ji^RR (Ahat_ii^RR)^-1 Ahat_ik^RR||
    (j, k != i), both relative to the largest ||Ahat_jj|| of the level."""
    out = {}
    for l in range(F["L"], 0, -1):
        nb, D, K = 1 << l, F["D"][l], F["K"][l]
        R = D - K
        Ah = F["Ahat"][l]
        nbr = _nbrs(F["near"][l], nb)
        scale = max(np.linalg.norm(Ah[(i, i)], 2) for i in range(nb))
        dropped, rr = 0.0, 0.0
        for i in range(nb):
            if R == 0:
                continue
            Ainv = np.linalg.inv(Ah[(i, i)][:R, :R])
            for j in nbr[i]:
                for k in nbr[i]:
                    if K and (j, k) != (i, i):
                        C = Ah[(j, i)][R:, :R] @ Ainv @ Ah[(i, k)][:R, R:]
                        dropped = max(dropped, np.linalg.norm(C, 2))
                    if j != i and k != i:
                        Crr = Ah[(j, i)][:R, :R] @ Ainv @ Ah[(i, k)][:R, :R]
                        rr = max(rr, np.linalg.norm(Crr, 2))
        out[l] = (dropped / scale, rr / scale)
    return out
