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
