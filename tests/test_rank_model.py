"""The learned rank predictor: the oracle's FP64 network against the
mathematics (CPU), and the library's BF16 training kernels against the
oracle (GPU)."""
import numpy as np
import pytest

from oracle import mlp


def _net(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, mlp.N_PARAMS)
    X = rng.normal(0.0, 1.0, (40, mlp.N_IN))
    y = rng.uniform(0.0, 1.0, 40)
    return theta, X, y


def test_oracle_gradient_matches_central_differences():
    """The chain-rule gradient of the oracle's loss equals central finite
    differences of the loss (FP64, step 1e-6) to 1e-6 relative, on every
    parameter group."""
    theta, X, y = _net(1)
    loss, g = mlp.loss_and_grad(theta, X, y)
    assert abs(loss - np.mean((mlp.forward(theta, X) - y) ** 2)) <= 1e-14 * loss
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 300, replace=False), [mlp.N_PARAMS - 1]])
    h = 1e-6
    fd = np.empty(len(idx))
    for t, k in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[t] = (mlp.loss_and_grad(tp, X, y)[0] - mlp.loss_and_grad(tm, X, y)[0]) / (2 * h)
    assert np.abs(fd - g[idx]).max() <= 1e-6 * np.abs(g).max()


def test_oracle_gradient_closed_form_for_constant_network():
    """With zero weights and biases except b3 the network outputs b3 for
    every input: the loss is mean((b3 - y)^2), its derivative in b3 is
    2 mean(b3 - y) and every other gradient entry is 0."""
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = 0.25
    _, X, y = _net(3)
    loss, g = mlp.loss_and_grad(theta, X, y)
    assert abs(loss - np.mean((0.25 - y) ** 2)) <= 1e-15
    assert abs(g[-1] - 2 * np.mean(0.25 - y)) <= 1e-15
    assert np.all(g[:-1] == 0.0)


def test_oracle_parameter_layout():
    p = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=np.float64))
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1
    assert p["W1"][1, 0] == 16 and p["b1"][0] == 1024 and p["b3"][0] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(p), np.arange(mlp.N_PARAMS))


# ---------------------------------------------------------------- GPU ---
def _bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as floats."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding
    return binding


GROUPS = (("W1", 0, 1024), ("b1", 1024, 1088), ("W2", 1088, 5184), ("b2", 5184, 5248), ("w3", 5248, 5312),
          ("b3", 5312, 5313))


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [11, 12])
def test_gpu_gradient_matches_oracle(B, seed):
    """The training kernels' loss and gradient against the oracle's FP64
    chain rule on the same BF16-valued weights and inputs.  The kernels
    round the hidden activations to BF16 (unit roundoff 2^-9) and sum in
    FP32, so each parameter group agrees to a few 2^-9 in relative norm;
    the bound is 2^-5."""
    rng = np.random.default_rng(seed)
    theta = _bf16(rng.normal(0.0, 0.25, mlp.N_PARAMS))
    X = _bf16(rng.normal(0.0, 1.0, (300, mlp.N_IN)))
    y = rng.uniform(0.0, 1.0, 300).astype(np.float32)
    m = B.h2_rank_model_create(1)
    try:
        B.h2_rank_model_set_weights(m, theta)
        loss, g = B.h2_rank_model_grad(m, X, y)
    finally:
        B.h2_rank_model_destroy(m)
    loss_ref, g_ref = mlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(loss - loss_ref) <= 2.0 ** -7 * loss_ref
    for name, a, b in GROUPS:
        e = np.linalg.norm(g[a:b] - g_ref[a:b]) / np.linalg.norm(g_ref[a:b])
        print(f"seed {seed} {name}: relative gradient error {e:.2e}")
        assert e <= 2.0 ** -5, (name, e)


def _training_set(B):
    """Ranks of the plain compression on the three solver workloads
    (workloads.rank_training_sets)."""
    import workloads as W
    F, Y = [], []
    for pts, kw in W.rank_training_sets():
        f, y, _ = B.h2_rank_data(B.make_params(**kw), pts)
        F.append(f)
        Y.append(y)
    return np.concatenate(F), np.concatenate(Y)


@pytest.fixture(scope="module")
def trained(B):
    F, Y = _training_set(B)
    m = B.h2_rank_model_create(7)
    loss0 = float(np.mean((B.h2_rank_model_predict(m, F) - Y) ** 2))
    loss = B.h2_rank_model_train(m, F, Y, steps=1500, lr=3e-3)
    yield m, F, Y, loss0, loss
    B.h2_rank_model_destroy(m)


@pytest.mark.gpu
def test_gpu_training_fits_the_plain_ranks(B, trained):
    """Full-batch Adam on the GPU drives the loss down and the trained
    network reproduces the training ranks k / n to a few percent."""
    m, F, Y, loss0, loss = trained
    pred = B.h2_rank_model_predict(m, F)
    mae = float(np.mean(np.abs(pred - Y)))
    print(f"training loss {loss0:.3e} -> {loss:.3e}, mean |k/n error| {mae:.3f} on {len(Y)} boxes")
    assert loss <= 0.1 * loss0
    assert mae <= 0.05


@pytest.mark.gpu
def test_gpu_predicted_layout_and_build_gain(B, trained):
    """What the trained network gains over the method without it, on a
    held-out problem shaped like the large workload (cube, 1/(r+1e-3),
    leaf 256, tol 1e-8): (1) the whole batch layout (every level's rank)
    comes from features and one inference per level, with no compression
    pass, and matches the plain build's ranks; (2) h2_build_predicted
    compresses with sketches sized by those ranks, faster than the plain
    rank-revealing pass, with few plain fallbacks; (3) the resulting H^2
    matrix reproduces exactly evaluated rows of A within a factor 4 of the
    plain build's error (sketched skeletons at the capped ranks are somewhat
    worse than a pivoted QR of the whole composite matrix), and the refined
    solve reaches 1e-10."""
    import time

    import workloads as W
    from oracle.kernels import Kernel
    m = trained[0]
    n = 65536
    P = W.cube_points(n, 71)
    kw = dict(kernel="laplace_eps", leaf=256, tol=1e-8, far_samples=1024, near_samples=64)
    prm = B.make_params(**kw)
    t0 = time.perf_counter()
    plan = B.h2_plan(prm, P)
    t_plan = time.perf_counter() - t0
    t0 = time.perf_counter()
    lay = B.h2_plan_predicted(prm, P, m)
    t_lay = time.perf_counter() - t0
    K_plain = [lv["K"] for lv in plan["levels"]]
    K_lay = [lv["K"] for lv in lay["levels"]]
    nb = [lv["nb"] for lv in plan["levels"]]
    print(f"layout: plain pass {t_plan:.2f} s (compression {plan['compress_s']:.2f} s), predicted {t_lay:.3f} s; "
          f"K plain {K_plain}, predicted {K_lay}")
    # levels with at least 16 boxes within 10 % (the few boxes of the top
    # levels give the regression little to go on; the build corrects them)
    assert all(abs(a - b) <= max(4, 0.1 * a) for a, b, c in zip(K_plain, K_lay, nb) if c >= 16)
    assert t_lay <= 0.2 * t_plan

    S0 = B.H2Solver.build(P, **kw)
    Sp = B.H2Solver.build_predicted(P, m, **kw)
    Sg = B.H2Solver.build_gpu(P, m, 0, **kw)
    c0, cp, cg = S0.stats()["construction"], Sp.stats()["construction"], Sg.stats()["construction"]
    print(f"compression: plain {c0['compress_s']:.2f} s, predicted (host sketches) {cp['compress_s']:.2f} s, "
          f"predicted (GPU sketches) {cg['compress_s']:.2f} s; fallback boxes {cp['fallback_boxes']} / "
          f"{cg['fallback_boxes']}, levels {cp['fallback_levels']} / {cg['fallback_levels']}; K {cp['K']} / {cg['K']}")
    assert cp["compress_s"] <= 0.8 * c0["compress_s"]
    assert cg["compress_s"] <= 0.5 * c0["compress_s"]
    assert cp["fallback_levels"] <= 1 and cg["fallback_levels"] <= 1
    # accuracy of A_H2 against exact rows of A (256 sampled rows)
    rng = np.random.default_rng(3)
    rows = rng.choice(n, 256, replace=False)
    x = W.uniform_rhs(n, 72)
    exact = Kernel("laplace_eps").matrix(P, rows, np.arange(n)) @ x
    e0 = np.linalg.norm(S0.matvec(x)[rows] - exact) / np.linalg.norm(exact)
    ep = np.linalg.norm(Sp.matvec(x)[rows] - exact) / np.linalg.norm(exact)
    eg = np.linalg.norm(Sg.matvec(x)[rows] - exact) / np.linalg.norm(exact)
    print(f"sampled-row error of A_H2: plain {e0:.2e}, predicted {ep:.2e}, predicted on the GPU {eg:.2e}")
    assert ep <= max(4 * e0, 1e-8) and eg <= max(4 * e0, 1e-8)
    for S in (S0, Sp, Sg):
        S.factor("fp16")
        _, rel, its = S.solve(W.uniform_rhs(n, 73), target=1e-10, max_iters=100)
        assert rel <= 1e-10
    for S in (S0, Sp, Sg):
        S.close()
