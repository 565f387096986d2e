"""Seeded synthetic inputs for the H^2-ULV solver.

This module only draws random numbers. It contains none of the solver's
arithmetic, so the oracle (``oracle/``) and the GPU path
(``paper_2502_02395_gb300``) can both use it without sharing any part of the
method.

The point sets are stand-ins for the geometries the paper measures on:
  * points on a unit-sphere surface, for the paper's Laplace sphere test
    (Section 6.2; the paper spaces the points evenly, we draw them uniformly
    at random on the surface);
  * points uniform in the unit cube, the volume case behind the Yukawa and
    Laplace-kernel workloads (Section 6.4 uses hemoglobin surface meshes, which
    are not available here; a random volume set is the harder case for
    compression).
All generators use NumPy's PCG64 ``default_rng(seed)`` and return float64.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "batch_systems",
    "cube_points",
    "sphere_points",
    "uniform_rhs",
    "Workload",
    "WORKLOADS",
    "workload",
]


def cube_points(n: int, seed: int) -> np.ndarray:
    """``n`` points uniform in the unit cube [0,1]^3, shape (n, 3), float64."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 3))


def sphere_points(n: int, seed: int) -> np.ndarray:
    """``n`` points uniform on the unit sphere surface (normalised Gaussians)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def uniform_rhs(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand side entries uniform in [-1, 1]; shape (n,) or (n, nrhs)."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=(n, nrhs))
    return b[:, 0].copy() if nrhs == 1 else b


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named problem: geometry, kernel and solver parameters.

    ``kernel`` is one of ``laplace_eps`` (1/(r+eps), diagonal 1/eps),
    ``yukawa_eps`` (exp(-r)/(r+eps), diagonal 1/eps + diag_shift),
    ``gaussian``, ``laplace_paper`` (Eq. 35), ``yukawa_paper`` (Eq. 36) and
    ``poly2_test`` ((1 + x.y)^2 + diag_shift on the diagonal; every
    off-diagonal block has rank <= 10).
    """

    name: str
    n: int
    geometry: str  # "cube" | "sphere"
    point_seed: int
    rhs_seed: int
    kernel: str
    leaf: int
    eta: float
    tol: float
    max_rank: int = 0  # 0: the default cap (half the box dimension)
    eps: float = 1e-3
    ell: float = 1.0
    diag_shift: float = 0.0
    far_samples: int = 1024
    near_samples: int = 64

    def points(self) -> np.ndarray:
        if self.geometry == "cube":
            return cube_points(self.n, self.point_seed)
        if self.geometry == "sphere":
            return sphere_points(self.n, self.point_seed)
        raise ValueError(self.geometry)

    def rhs(self, nrhs: int = 1) -> np.ndarray:
        return uniform_rhs(self.n, self.rhs_seed, nrhs)


# The solver configurations the library is measured and tested on.
WORKLOADS = {
    # 2048 points in the unit cube, 1/(r+1e-3), leaf 64, eta 1, tol 1e-10.
    "cube2048_laplace": Workload("cube2048_laplace", 2048, "cube", 1, 2,
                                 "laplace_eps", 64, 1.0, 1e-10),
    # Its compressing twin (tol 1e-4), where elimination really drops terms.
    "cube2048_laplace_tol4": Workload("cube2048_laplace_tol4", 2048, "cube", 1, 2,
                                      "laplace_eps", 64, 1.0, 1e-4),
    # 65536 points on the unit sphere, 1/(r+1e-3), leaf 256, tol 1e-8, FP64.
    "sphere65536_laplace": Workload("sphere65536_laplace", 65536, "sphere", 3, 4,
                                    "laplace_eps", 256, 1.0, 1e-8),
    # An eighth-size version of the next one: small-case profiler captures
    # (a few GB on the device, leaf blocks still larger than L2).
    "cube32768_yukawa": Workload("cube32768_yukawa", 32768, "cube", 5, 6,
                                 "yukawa_eps", 256, 1.0, 1e-10, diag_shift=1.0),
    # A quarter-size version of the next one (profiling captures).
    "cube65536_yukawa": Workload("cube65536_yukawa", 65536, "cube", 5, 6,
                                 "yukawa_eps", 256, 1.0, 1e-10, diag_shift=1.0),
    # 262144 points in the unit cube, Yukawa exp(-r)/(r+1e-3) + 1 on the
    # diagonal, leaf 256, eta 1, tol 1e-10 with the default rank cap.
    "cube262144_yukawa": Workload("cube262144_yukawa", 262144, "cube", 5, 6,
                                  "yukawa_eps", 256, 1.0, 1e-10, diag_shift=1.0),
    # 2^20 points in the unit cube, 1/(r+1e-3), leaf 256, eta 1, tol 1e-8:
    # the learned rank predictor against the plain rank-revealing build.
    "cube1048576_laplace": Workload("cube1048576_laplace", 1048576, "cube", 9, 10,
                                    "laplace_eps", 256, 1.0, 1e-8),
}


def rank_training_sets():
    """The problems whose plain-compression ranks train the rank predictor:
    (points, parameters) for cube 2048 / 1/(r+1e-3) / leaf 64 at tolerances
    1e-4 .. 1e-10, sphere 65536 / 1/(r+1e-3) / leaf 256 at 1e-6 and 1e-8, and
    cube 262144 / Yukawa + 1 / leaf 256 at 1e-8 and 1e-10 (far / near
    samples 1024 / 64 throughout)."""
    sets = []
    for tol in (1e-4, 1e-6, 1e-8, 1e-10):
        sets.append((cube_points(2048, 1), dict(kernel="laplace_eps", leaf=64, tol=tol)))
    for tol in (1e-6, 1e-8):
        sets.append((sphere_points(65536, 3), dict(kernel="laplace_eps", leaf=256, tol=tol)))
    for tol in (1e-8, 1e-10):
        sets.append((cube_points(262144, 5), dict(kernel="yukawa_eps", leaf=256, tol=tol, diag_shift=1.0)))
    return [(P, dict(far_samples=1024, near_samples=64, **kw)) for P, kw in sets]


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def batch_systems(count: int = 64, seed: int = 100, n_min: int = 4096, n_max: int = 65536):
    """A batch of independent Gaussian-covariance systems of uneven size:
    N_s = round(exp(U[ln n_min, ln n_max])) and length scale
    l_s ~ U[0.05, 0.5] (both drawn from `seed`), points uniform in the unit
    cube with seed 1000 + s, right-hand side seed 2000 + s, leaf 256 when
    N_s >= 16384 else 128.  Returns a list of dicts (n, ell, leaf,
    point_seed, rhs_seed, shift); kernel exp(-r^2 / l^2) with `shift` added
    to the diagonal (1.0: with 1e-2 the H^2-ULV preconditioner of the
    FP64 oracle itself stalls for l around 0.1 - 0.4), tolerance 1e-8."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), count))).astype(int)
    ells = rng.uniform(0.05, 0.5, count)
    return [dict(n=int(n), ell=float(e), leaf=256 if n >= 16384 else 128, point_seed=1000 + s, rhs_seed=2000 + s,
                 shift=1.0) for s, (n, e) in enumerate(zip(ns, ells))]
