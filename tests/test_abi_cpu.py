"""The C-ABI library on a machine without a GPU: it loads, exports every
symbol include/h2ulv.h declares, and its host-side construction (tree, near
and far lists, ranks) agrees with the oracle's independent implementation of
the same rules."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2502_02395_gb300 import build as bld
    bld.build()
    from paper_2502_02395_gb300 import binding
    return binding


def declared_functions():
    src = open(os.path.join(ROOT, "include", "h2ulv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h2_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(B):
    names = declared_functions()
    assert len(names) >= 12
    L = ctypes.CDLL(B.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(B.EXPORTED) == names


def test_library_binds_every_symbol_at_load(B):
    """With immediate binding every symbol the library references resolves
    at load time (a template launcher used but never instantiated would only
    fail at its first call otherwise)."""
    ctypes.CDLL(B.LIB_PATH, mode=os.RTLD_NOW)


@pytest.mark.parametrize("n,leaf,eta,geom", [(2048, 64, 1.0, "cube"), (1000, 64, 1.0, "cube"),
                                             (3000, 100, 0.0, "sphere"), (777, 50, 2.0, "cube")])
def test_plan_lists_match_oracle(B, n, leaf, eta, geom):
    from oracle.tree import build_tree, interaction_lists
    P = W.cube_points(n, 3) if geom == "cube" else W.sphere_points(n, 3)
    plan = B.h2_plan(B.make_params("laplace_eps", leaf=leaf, eta=eta, tol=1e-6, far_samples=256,
                                   near_samples=32), P)
    perm, ranges = build_tree(P, leaf)
    near, far = interaction_lists(P, perm, ranges, eta)
    assert plan["L"] == len(ranges) - 1
    for lv in plan["levels"]:
        l = lv["l"]
        assert lv["NP"] == len(near[l]) and lv["FP"] == len(far[l])
        assert lv["nb"] == 1 << l
    assert plan["levels"][-1]["D"] == int(np.diff(ranges[-1]).max())


def test_plan_ranks_match_oracle_construction(B):
    """The library's streamed-QR ID and the oracle's LAPACK pivoted QR pick
    the same level ranks (same tolerance rule, same sampling rule)."""
    from oracle.construct import construct
    from oracle.kernels import Kernel
    P = W.sphere_points(4096, 5)
    kw = dict(leaf=128, eta=1.0, tol=1e-6, max_rank=0, far_samples=512, near_samples=32)
    plan = B.h2_plan(B.make_params("laplace_eps", **kw), P)
    H = construct(P, Kernel("laplace_eps"), kw["leaf"], kw["eta"], kw["tol"], kw["max_rank"],
                  kw["far_samples"], kw["near_samples"])
    for lv in plan["levels"][1:]:
        assert abs(lv["K"] - H["K"][lv["l"]]) <= 1, (lv, H["K"])
    assert abs(plan["levels"][-1]["rank_max"] - max(H["ranks"][H["L"]])) <= 1


def test_plan_poly2_exact_rank(B):
    P = W.cube_points(1000, 1)
    plan = B.h2_plan(B.make_params("poly2_test", leaf=64, tol=1e-10, far_samples=0, near_samples=0,
                                   diag_shift=1.0), P)
    assert all(lv["K"] == 10 for lv in plan["levels"][1:])


@pytest.mark.parametrize("bad", ["tol", "eta", "leaf", "nan", "kernel", "n0"])
def test_plan_rejects_bad_input(B, bad):
    P = W.cube_points(100, 1)
    kw = dict(leaf=32, tol=1e-6)
    if bad == "tol":
        kw["tol"] = 0.0
    if bad == "eta":
        kw["eta"] = -1.0
    if bad == "leaf":
        kw["leaf"] = 0
    if bad == "nan":
        P = P.copy()
        P[5, 1] = np.nan
    kern = 17 if bad == "kernel" else "laplace_eps"
    if bad == "n0":
        P = P[:0]
    with pytest.raises(B.H2Error) as ei:
        B.h2_plan(B.make_params(kern, **kw), P)
    assert ei.value.status == -1


def test_single_box_plan(B):
    P = W.cube_points(40, 2)
    plan = B.h2_plan(B.make_params("laplace_eps", leaf=64), P)
    assert plan["L"] == 0 and plan["levels"][0]["D"] == 40


def test_memory_limit_gives_oom_before_any_launch(B):
    """h2_set_memory_limit: an instance whose device arrays exceed the cap is
    refused with H2_ERR_OOM after the host construction and before any CUDA
    call (so this runs on a machine without a GPU); the message names the
    bytes needed and the cap."""
    P = W.cube_points(2048, 3)
    prm = B.make_params("laplace_eps", leaf=64, tol=1e-6, far_samples=256, near_samples=32)
    plan = B.h2_plan(prm, P)
    B.h2_set_memory_limit(1 << 20)
    try:
        with pytest.raises(B.H2Error) as e:
            B.h2_build(prm, P)
        assert e.value.status == -2
        assert "memory limit is 1048576" in e.value.message
        need = float(e.value.message.split("about ")[1].split(" ")[0])
        assert need >= plan["device_bytes_build"]
    finally:
        B.h2_set_memory_limit(0)


def test_forest_depth_checks_before_any_device_work():
    """h2_tree_depth, and h2_build_forest's refusal of systems of different
    depths or of depth 0, are host checks made before any CUDA call."""
    import ctypes
    from paper_2502_02395_gb300 import binding as bd
    assert bd.h2_tree_depth(4096, 256) == 4 and bd.h2_tree_depth(4097, 256) == 5
    assert bd.h2_tree_depth(256, 256) == 0 and bd.h2_tree_depth(0, 256) == -1
    rng = np.random.default_rng(0)
    for ns in ([3000, 5000], [200, 300]):
        with pytest.raises(bd.H2Error) as ei:
            bd.h2_build_forest(bd.make_params(leaf=256), [rng.random((n, 3)) for n in ns])
        assert ei.value.status == -1 and "depth" in ei.value.message
