"""h2_matvec_noalloc: the matvec for callers that must not allocate device
memory after building their context (for example a host framework that owns
all device memory, or a loop on a latency budget where cudaMalloc can block).
Its per-call scratch is a fixed array inside the library instead of buffers
the context allocated.  This file is collected last on purpose.

The test calls the new entry point through the C ABI twice in a row, with
different inputs, and compares each result with h2_matvec's (same kernels,
so the results agree to rounding): the second call must not be disturbed by
what the first left in the shared array.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding
    P = W.cube_points(4096, 21)
    S = binding.H2Solver.build(P, kernel="yukawa_eps", leaf=128, eta=1.0, tol=1e-8, diag_shift=1.0,
                               far_samples=256, near_samples=32)
    yield binding, S, torch
    S.close()


def test_noalloc_matvec_matches_matvec_on_two_calls(solver):
    B, S, torch = solver
    for seed in (31, 32):
        x = torch.from_numpy(W.uniform_rhs(S.n, seed)).cuda()
        y_ref = S.matvec(x)
        y = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        B.h2_matvec_noalloc(S.ctx, x, y)
        torch.cuda.synchronize()
        a, r = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - r) <= 1e-13 * np.linalg.norm(r)


def test_noalloc_matvec_rejects_host_pointers(solver):
    B, S, torch = solver
    x = W.uniform_rhs(S.n, 33)
    y = np.zeros_like(x)
    with pytest.raises(B.H2Error) as e:
        B.h2_matvec_noalloc(S.ctx, x, y)
    assert e.value.status == -1 and "device pointers" in e.value.message


def test_noalloc_matvec_other_depth(solver):
    """A second instance of another depth and with uneven leaves (sphere,
    3000 points, leaf 64: six levels) gives h2_matvec's result too."""
    B, S0, torch = solver
    P = W.sphere_points(3000, 22)
    S = B.H2Solver.build(P, kernel="laplace_eps", leaf=64, eta=1.0, tol=1e-8, far_samples=256, near_samples=32)
    try:
        for seed in (41, 42):
            x = torch.from_numpy(W.uniform_rhs(S.n, seed)).cuda()
            y_ref = S.matvec(x)
            y = torch.full_like(x, float("nan"))
            B.h2_matvec_noalloc(S.ctx, x, y)
            torch.cuda.synchronize()
            a, r = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.linalg.norm(a - r) <= 1e-13 * np.linalg.norm(r)
    finally:
        S.close()


def test_noalloc_matvec_rejects_problem_beyond_its_scratch(solver):
    """A problem whose scratch (two padded vectors plus the skeleton
    coefficients) exceeds the fixed 2^21-double array is refused with
    H2_ERR_INVALID_ARG and a message giving both sizes.  The instance is a
    plain block-diagonal H^2 structure imported directly: 2^20 points in
    2048 leaves of 512, near pairs only on the diagonal, siblings far, rank 1
    above the leaves."""
    B, S0, torch = solver
    L, D = 11, 512
    nb = 1 << L
    N = nb * D
    pts = W.cube_points(N, 23)
    K = [0] + [1] * L
    Dl = [2] * L + [D]
    X, SK, near, far = [None], [None], [np.array([[0, 0]], dtype=np.int32)], [np.zeros((0, 2), dtype=np.int32)]
    for l in range(1, L + 1):
        n_l = 1 << l
        Xl = np.zeros((n_l, Dl[l], 1))
        Xl[:, 0, 0] = 1.0
        X.append(Xl)
        SK.append((np.arange(n_l, dtype=np.int64) * (N // n_l))[:, None])
        near.append(np.stack([np.arange(n_l), np.arange(n_l)], 1).astype(np.int32))
        f = np.arange(n_l)
        far.append(np.stack([f, f ^ 1], 1).astype(np.int32))
    flat = dict(N=N, L=L, points=pts, perm=np.arange(N, dtype=np.int64),
                leaf_offsets=np.arange(0, N + 1, D, dtype=np.int64), D=np.array(Dl, dtype=np.int32),
                K=np.array(K, dtype=np.int32), near=near, far=far, X=X, SK=SK)
    S = B.H2Solver.from_instance(flat, kernel="laplace_eps", leaf=D, eta=1.0, tol=1e-6)
    try:
        x = torch.from_numpy(W.uniform_rhs(N, 43)).cuda()
        y = torch.zeros_like(x)
        with pytest.raises(B.H2Error) as e:
            B.h2_matvec_noalloc(S.ctx, x, y)
        assert e.value.status == -1
        assert "doubles of scratch" in e.value.message and str(1 << 21) in e.value.message
    finally:
        S.close()
