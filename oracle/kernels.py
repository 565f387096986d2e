"""Kernel functions G(x, y) that generate the dense matrix (oracle; FP64).

Eq. 35 (Section 6.2): Laplace, A_ii = 1e3, A_ij = 1/r_ij.
Eq. 36 (Section 6.4): Yukawa, A_ii = 1e3, A_ij = exp(-r_ij)/r_ij.
The workloads also use softened forms 1/(r+eps) and exp(-r)/(r+eps), whose
value at r = 0 is 1/eps (= 1e3 for eps = 1e-3, matching the paper's diagonal),
a Gaussian covariance exp(-r^2/ell^2), and the test kernel (1 + x.y)^2, whose
off-diagonal blocks all have rank <= 10.  The test kernel's diagonal adds
diag_shift * (1 + |x|^2): a point-dependent term, so the projected diagonal
blocks have non-zero RS/SR parts and the self Schur update is exercised while
every fill-in Eq. 21 drops is still exactly zero.

Entries are indexed by point index: entry (a, b) uses the kernel's diagonal
value when a == b (the same point), and the off-diagonal formula otherwise.
The diagonal value is f(0) + diag_shift for the softened kernels and the
Gaussian, f(x, x) + diag_shift * (1 + |x|^2) for the test kernel, and
1e3 + diag_shift for the paper's Eq. 35 / Eq. 36.
"""
from __future__ import annotations

import numpy as np

KINDS = ("laplace_eps", "yukawa_eps", "gaussian", "laplace_paper", "yukawa_paper", "poly2_test")


class Kernel:
    def __init__(self, kind: str, eps: float = 1e-3, ell: float = 1.0, diag_shift: float = 0.0):
        if kind not in KINDS:
            raise ValueError(f"unknown kernel {kind!r}")
        self.kind = kind
        self.eps = float(eps)
        self.ell = float(ell)
        self.diag_shift = float(diag_shift)

    def off(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        """Off-diagonal formula f(x, y) for all pairs, shape (len(X), len(Y))."""
        if self.kind == "poly2_test":
            return (1.0 + X @ Y.T) ** 2
        d = X[:, None, :] - Y[None, :, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        if self.kind == "laplace_eps":
            return 1.0 / (r + self.eps)
        if self.kind == "yukawa_eps":
            return np.exp(-r) / (r + self.eps)
        if self.kind == "gaussian":
            return np.exp(-(r * r) / (self.ell * self.ell))
        with np.errstate(divide="ignore", invalid="ignore"):
            if self.kind == "laplace_paper":
                return 1.0 / r
            return np.exp(-r) / r  # yukawa_paper

    def diag(self, X: np.ndarray) -> np.ndarray:
        """Diagonal values A_aa for the points X, shape (len(X),)."""
        if self.kind in ("laplace_paper", "yukawa_paper"):
            return np.full(len(X), 1e3 + self.diag_shift)
        if self.kind == "laplace_eps":
            return np.full(len(X), 1.0 / self.eps + self.diag_shift)
        if self.kind == "yukawa_eps":
            return np.full(len(X), 1.0 / self.eps + self.diag_shift)
        if self.kind == "gaussian":
            return np.full(len(X), 1.0 + self.diag_shift)
        q = 1.0 + np.sum(X * X, axis=1)  # poly2_test
        return q * q + self.diag_shift * q

    def matrix(self, points: np.ndarray, I: np.ndarray, J: np.ndarray) -> np.ndarray:
        """G(P[I], P[J]) with the diagonal value wherever I[a] == J[b]."""
        I = np.asarray(I, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        M = self.off(points[I], points[J])
        same = I[:, None] == J[None, :]
        if same.any():
            a, b = np.nonzero(same)
            M[a, b] = self.diag(points[I[a]])
        return M
