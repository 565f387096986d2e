"""ctypes binding of the C ABI declared in include/h2ulv.h.

The module-level functions carry the C names (h2_build, h2_plan, h2_import,
h2_factor, h2_solve, h2_solve_many, h2_ulv_apply, h2_matvec, h2_matvec_many,
h2_matvec_noalloc, h2_matvec_arith, h2_set_option, h2_wait_selftest,
h2_set_memory_limit, the rank predictor's h2_rank_data / h2_rank_model_* /
h2_plan_predicted / h2_build_predicted / h2_build_gpu, h2_set_refinement, h2_set_stream, h2_stats, h2_export,
h2_last_error, h2_destroy) and only marshal arguments: every step
of the computation runs in the library.  ``H2Solver`` wraps a context.

Vectors may be NumPy float64 arrays (host) or CUDA torch float64 tensors
(device); the library tells the two apart.  The library must have been built
(``paper_2502_02395_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libh2ulv.so")

KERNELS = {"laplace_eps": 0, "yukawa_eps": 1, "gaussian": 2, "laplace_paper": 3,
           "yukawa_paper": 4, "poly2_test": 5}
PRECS = {"fp64": 0, "fp16": 1, "bf16": 2}
STATUS = {0: "H2_OK", -1: "H2_ERR_INVALID_ARG", -2: "H2_ERR_OOM", -3: "H2_ERR_SINGULAR",
          -4: "H2_ERR_NOT_CONVERGED", -5: "H2_ERR_CUDA", -6: "H2_ERR_TIMEOUT", -7: "H2_ERR_STATE"}

# every symbol include/h2ulv.h declares
EXPORTED = ("h2_build", "h2_plan", "h2_import", "h2_factor", "h2_release_factorization", "h2_solve", "h2_solve_many", "h2_ulv_apply",
            "h2_matvec", "h2_matvec_many", "h2_matvec_noalloc", "h2_matvec_arith", "h2_set_option",
            "h2_wait_selftest", "h2_autotune", "h2_set_memory_limit", "h2_rank_data", "h2_rank_model_create",
            "h2_rank_model_set_weights", "h2_rank_model_get_weights", "h2_rank_model_grad", "h2_rank_model_train",
            "h2_rank_model_predict", "h2_rank_model_last_error", "h2_rank_model_destroy", "h2_plan_predicted",
            "h2_build_predicted", "h2_build_gpu", "h2_tree_depth", "h2_build_forest", "h2_batch_create",
            "h2_batch_create_forest", "h2_batch_run", "h2_batch_tune",
            "h2_batch_stats", "h2_batch_last_error", "h2_batch_destroy",
            "h2_set_refinement", "h2_set_stream", "h2_stats", "h2_export", "h2_last_error", "h2_destroy")
OPTIONS = {"rr_lu_fp64": 0, "residual_fp64": 1, "graphs": 2, "tc_kernel": 3, "fp64_leaf": 4, "box_stream": 5,
           "pair_ctas": 6, "box_ctas": 7}
ARITH = {"fp64": 0, "fp32": 1, "fp32_pair": 2}


class H2Error(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Params(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("eps", ctypes.c_double), ("ell", ctypes.c_double),
                ("diag_shift", ctypes.c_double), ("leaf_size", ctypes.c_int32), ("eta", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_rank", ctypes.c_int32), ("far_samples", ctypes.c_int32),
                ("near_samples", ctypes.c_int32)]


_P = ctypes.c_void_p


class Instance(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("L", ctypes.c_int32), ("points", _P), ("perm", _P),
                ("leaf_offsets", _P), ("D", _P), ("K", _P), ("n_near", _P), ("near", _P),
                ("n_far", _P), ("far", _P), ("X", _P), ("SK", _P)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2502_02395_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "h2_build": (i32, [pp, vp, vp, i64]),
            "h2_plan": (i32, [vp, vp, i64, ctypes.c_char_p, ctypes.c_size_t]),
            "h2_import": (i32, [pp, vp, vp]),
            "h2_factor": (i32, [vp, i32]),
            "h2_release_factorization": (i32, [vp]),
            "h2_solve": (i32, [vp, vp, vp, dbl, i32, vp, vp]),
            "h2_solve_many": (i32, [vp, vp, vp, i32, dbl, i32, vp, vp]),
            "h2_matvec_many": (i32, [vp, vp, vp, i32]),
            "h2_ulv_apply": (i32, [vp, vp, vp]),
            "h2_matvec": (i32, [vp, vp, vp]),
            "h2_matvec_noalloc": (i32, [vp, vp, vp]),
            "h2_set_refinement": (i32, [vp, i32, i32]),
            "h2_set_option": (i32, [vp, i32, i64]),
            "h2_matvec_arith": (i32, [vp, vp, vp, i32]),
            "h2_wait_selftest": (i32, [vp, i64]),
            "h2_autotune": (i32, [vp, i32, ctypes.c_char_p, ctypes.c_size_t]),
            "h2_set_memory_limit": (i32, [ctypes.c_uint64]),
            "h2_rank_data": (i32, [vp, vp, i64, vp, vp, vp, i64, vp]),
            "h2_rank_model_create": (i32, [pp, ctypes.c_uint64]),
            "h2_rank_model_set_weights": (i32, [vp, vp]),
            "h2_rank_model_get_weights": (i32, [vp, vp, vp, vp]),
            "h2_rank_model_grad": (i32, [vp, vp, vp, i64, vp, vp]),
            "h2_rank_model_train": (i32, [vp, vp, vp, i64, i32, ctypes.c_float, vp]),
            "h2_rank_model_predict": (i32, [vp, vp, i64, vp]),
            "h2_rank_model_last_error": (ctypes.c_char_p, [vp]),
            "h2_rank_model_destroy": (None, [vp]),
            "h2_plan_predicted": (i32, [vp, vp, i64, vp, ctypes.c_char_p, ctypes.c_size_t]),
            "h2_build_predicted": (i32, [pp, vp, vp, i64, vp]),
            "h2_build_gpu": (i32, [pp, vp, vp, i64, vp, i32]),
            "h2_tree_depth": (i32, [i64, i32]),
            "h2_build_forest": (i32, [pp, vp, vp, vp, i32]),
            "h2_batch_create": (i32, [pp, vp, vp, i32]),
            "h2_batch_create_forest": (i32, [pp, vp, vp, vp, vp, i32]),
            "h2_batch_run": (i32, [vp, i32, vp, vp, dbl, i32, vp, vp, vp]),
            "h2_batch_tune": (i32, [vp, i32, vp, vp, dbl, i32, vp]),
            "h2_batch_stats": (i32, [vp, ctypes.c_char_p, ctypes.c_size_t]),
            "h2_batch_last_error": (ctypes.c_char_p, [vp]),
            "h2_batch_destroy": (None, [vp]),
            "h2_set_stream": (i32, [vp, vp]),
            "h2_stats": (i32, [vp, ctypes.c_char_p, ctypes.c_size_t]),
            "h2_export": (i32, [vp, ctypes.c_char_p, i32, vp, ctypes.c_size_t, vp, vp]),
            "h2_last_error": (ctypes.c_char_p, [vp]),
            "h2_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """Address of a NumPy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _check(st: int, ctx=None):
    if st != 0:
        msg = lib().h2_last_error(ctx)
        raise H2Error(st, msg.decode() if msg else "")


def make_params(kernel="laplace_eps", leaf=256, eta=1.0, tol=1e-10, max_rank=0, far_samples=1024,
                near_samples=64, eps=1e-3, ell=1.0, diag_shift=0.0) -> Params:
    return Params(KERNELS[kernel] if isinstance(kernel, str) else int(kernel), eps, ell, diag_shift, leaf,
                  eta, tol, max_rank, far_samples, near_samples)


# ------------------------------------------------------------ C names ---
def h2_build(params: Params, points: np.ndarray):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    out = ctypes.c_void_p()
    st = lib().h2_build(ctypes.byref(out), ctypes.byref(params), _ptr(pts), len(pts))
    _check(st, None)
    return out


def h2_plan(params: Params, points: np.ndarray) -> dict:
    pts = np.ascontiguousarray(points, dtype=np.float64)
    buf = ctypes.create_string_buffer(1 << 20)
    st = lib().h2_plan(ctypes.byref(params), _ptr(pts), len(pts), buf, len(buf))
    _check(st, None)
    return json.loads(buf.value.decode())


def h2_import(params: Params, flat: dict):
    """flat: the dict of arrays oracle.instance.flatten produces."""
    L = int(flat["L"])
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    def ptrs(lst, dt):
        vals = [arr(a, dt) if a is not None else 0 for a in lst]
        a = (ctypes.c_void_p * len(vals))(*vals)
        keep.append(a)
        return ctypes.cast(a, ctypes.c_void_p)

    inst = Instance()
    inst.N = int(flat["N"])
    inst.L = L
    inst.points = arr(flat["points"], np.float64)
    inst.perm = arr(flat["perm"], np.int64)
    inst.leaf_offsets = arr(flat["leaf_offsets"], np.int64)
    inst.D = arr(flat["D"], np.int32)
    inst.K = arr(flat["K"], np.int32)
    inst.n_near = arr([len(a) for a in flat["near"]], np.int64)
    inst.near = ptrs([np.asarray(a).reshape(-1, 2) for a in flat["near"]], np.int32)
    inst.n_far = arr([len(a) for a in flat["far"]], np.int64)
    inst.far = ptrs([np.asarray(a).reshape(-1, 2) if len(a) else np.zeros((0, 2)) for a in flat["far"]],
                    np.int32)
    inst.X = ptrs([None] + [flat["X"][l] for l in range(1, L + 1)], np.float64)
    inst.SK = ptrs([None] + [flat["SK"][l] for l in range(1, L + 1)], np.int64)
    out = ctypes.c_void_p()
    st = lib().h2_import(ctypes.byref(out), ctypes.byref(params), ctypes.byref(inst))
    _check(st, None)
    return out


def h2_factor(ctx, prec: str | int = "fp64"):
    _check(lib().h2_factor(ctx, PRECS[prec] if isinstance(prec, str) else prec), ctx)


def h2_solve(ctx, b, x, target=1e-10, max_iters=50, check=True):
    rel = ctypes.c_double()
    its = ctypes.c_int32()
    st = lib().h2_solve(ctx, _ptr(b), _ptr(x), target, max_iters, ctypes.byref(rel), ctypes.byref(its))
    if check:
        _check(st, ctx)
    return st, rel.value, its.value


def h2_solve_many(ctx, B, X, target=1e-10, max_iters=50, check=True):
    """B, X: nrhs x N (one right-hand side per row, contiguous)."""
    nrhs = int(B.shape[0])
    rel = (ctypes.c_double * max(nrhs, 1))()
    its = (ctypes.c_int32 * max(nrhs, 1))()
    st = lib().h2_solve_many(ctx, _ptr(B), _ptr(X), nrhs, target, max_iters, ctypes.cast(rel, ctypes.c_void_p),
                             ctypes.cast(its, ctypes.c_void_p))
    if check:
        _check(st, ctx)
    return st, list(rel)[:nrhs], list(its)[:nrhs]


def h2_matvec_many(ctx, X, Y):
    _check(lib().h2_matvec_many(ctx, _ptr(X), _ptr(Y), int(X.shape[0])), ctx)


def h2_ulv_apply(ctx, b, x):
    _check(lib().h2_ulv_apply(ctx, _ptr(b), _ptr(x)), ctx)


def h2_matvec(ctx, x, y):
    _check(lib().h2_matvec(ctx, _ptr(x), _ptr(y)), ctx)


def h2_matvec_noalloc(ctx, x, y):
    """y = A_H2 x with x, y CUDA tensors; the library allocates nothing for
    this call (its scratch is a fixed array inside the library)."""
    _check(lib().h2_matvec_noalloc(ctx, _ptr(x), _ptr(y)), ctx)


def h2_set_refinement(ctx, method: str | int = "auto", restart: int = 30):
    """method: "ir" (0), "gmres" (1, FP64 FGMRES), "nested" (2, FP64 outer /
    FP32 inner FGMRES) or "auto" (3)."""
    m = {"ir": 0, "gmres": 1, "nested": 2, "auto": 3}.get(method, method)
    _check(lib().h2_set_refinement(ctx, int(m), int(restart)), ctx)


def h2_set_option(ctx, option: str | int, value: int):
    """option: "rr_lu_fp64" (0), "residual_fp64" (1) or "graphs" (2); value 0 or 1."""
    _check(lib().h2_set_option(ctx, OPTIONS.get(option, option), int(value)), ctx)


def h2_matvec_arith(ctx, x, y, arith: str | int = "fp64"):
    """y = A_H2 x in "fp64" (0), "fp32" (1) or "fp32_pair" (2) arithmetic."""
    _check(lib().h2_matvec_arith(ctx, _ptr(x), _ptr(y), ARITH.get(arith, arith)), ctx)


def h2_wait_selftest(ctx, timeout_ns: int):
    """Returns the raw status (-6, H2_ERR_TIMEOUT, when the wait gave up)."""
    return lib().h2_wait_selftest(ctx, int(timeout_ns))


def h2_set_memory_limit(nbytes: int):
    _check(lib().h2_set_memory_limit(int(nbytes)), None)


# ------------------------------------------------------ rank predictor ---
RANK_FEATURES = 16
RANK_PARAMS = 5313


def _check_model(st: int, m):
    if st != 0:
        msg = lib().h2_rank_model_last_error(m) if m else lib().h2_last_error(None)
        raise H2Error(st, msg.decode() if msg else "")


def h2_rank_data(params: Params, points: np.ndarray):
    """Features (nbox x 16), targets k_i / n_i and levels of every box from
    the plain compression (host only)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    nbox = ctypes.c_int64()
    st = lib().h2_rank_data(ctypes.byref(params), _ptr(pts), len(pts), None, None, None, 0, ctypes.byref(nbox))
    if st not in (0, -1):
        _check(st, None)
    n = nbox.value
    F = np.zeros((n, RANK_FEATURES), dtype=np.float32)
    y = np.zeros(n, dtype=np.float32)
    lv = np.zeros(n, dtype=np.int32)
    _check(lib().h2_rank_data(ctypes.byref(params), _ptr(pts), len(pts), _ptr(F), _ptr(y), _ptr(lv), n,
                              ctypes.byref(nbox)), None)
    return F, y, lv


def h2_rank_model_create(seed: int = 0):
    out = ctypes.c_void_p()
    _check_model(lib().h2_rank_model_create(ctypes.byref(out), int(seed)), None)
    return out


def h2_rank_model_set_weights(m, theta):
    t = np.ascontiguousarray(theta, dtype=np.float32)
    _check_model(lib().h2_rank_model_set_weights(m, _ptr(t)), m)


def h2_rank_model_get_weights(m):
    t = np.zeros(RANK_PARAMS, dtype=np.float32)
    mean = np.zeros(RANK_FEATURES, dtype=np.float32)
    istd = np.zeros(RANK_FEATURES, dtype=np.float32)
    _check_model(lib().h2_rank_model_get_weights(m, _ptr(t), _ptr(mean), _ptr(istd)), m)
    return t, mean, istd


def h2_rank_model_grad(m, inputs, targets):
    X = np.ascontiguousarray(inputs, dtype=np.float32)
    y = np.ascontiguousarray(targets, dtype=np.float32)
    g = np.zeros(RANK_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check_model(lib().h2_rank_model_grad(m, _ptr(X), _ptr(y), len(y), ctypes.byref(loss), _ptr(g)), m)
    return float(loss.value), g


def h2_rank_model_train(m, feats, targets, steps=2000, lr=3e-3):
    X = np.ascontiguousarray(feats, dtype=np.float32)
    y = np.ascontiguousarray(targets, dtype=np.float32)
    loss = ctypes.c_float()
    _check_model(lib().h2_rank_model_train(m, _ptr(X), _ptr(y), len(y), int(steps), float(lr), ctypes.byref(loss)), m)
    return float(loss.value)


def h2_rank_model_predict(m, feats):
    X = np.ascontiguousarray(feats, dtype=np.float32)
    out = np.zeros(len(X), dtype=np.float32)
    _check_model(lib().h2_rank_model_predict(m, _ptr(X), len(X), _ptr(out)), m)
    return out


def h2_rank_model_destroy(m):
    lib().h2_rank_model_destroy(m)


def h2_plan_predicted(params: Params, points: np.ndarray, m) -> dict:
    pts = np.ascontiguousarray(points, dtype=np.float64)
    buf = ctypes.create_string_buffer(1 << 20)
    _check(lib().h2_plan_predicted(ctypes.byref(params), _ptr(pts), len(pts), m, buf, len(buf)), None)
    return json.loads(buf.value.decode())


def h2_build_predicted(params: Params, points: np.ndarray, m):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib().h2_build_predicted(ctypes.byref(out), ctypes.byref(params), _ptr(pts), len(pts), m), None)
    return out


def h2_build_gpu(params: Params, points: np.ndarray, m=None, gs_sweeps: int = 0):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib().h2_build_gpu(ctypes.byref(out), ctypes.byref(params), _ptr(pts), len(pts), m, int(gs_sweeps)), None)
    return out


def h2_tree_depth(n: int, leaf: int) -> int:
    return int(lib().h2_tree_depth(int(n), int(leaf)))


def _point_arrays(points_list):
    pts = [np.ascontiguousarray(P, dtype=np.float64) for P in points_list]
    ptrs = (ctypes.c_void_p * len(pts))(*[P.ctypes.data for P in pts])
    ns = (ctypes.c_int64 * len(pts))(*[len(P) for P in pts])
    return pts, ptrs, ns


def h2_build_forest(params: Params, points_list):
    """One instance over several systems of one tree depth (h2_build_forest)."""
    pts, ptrs, ns = _point_arrays(points_list)
    out = ctypes.c_void_p()
    _check(lib().h2_build_forest(ctypes.byref(out), ctypes.byref(params), ctypes.cast(ptrs, ctypes.c_void_p),
                                 ctypes.cast(ns, ctypes.c_void_p), len(pts)), None)
    return out


# ------------------------------------------------------------- batches ---
class H2Batch:
    """Independent systems factored and solved by the library's worker pool:
    H2Batch(solvers) over H2Solver objects (one context per system), or
    H2Batch.forest(points_list, **params) (the systems grouped by tree depth,
    each group one instance whose levels are single launches over all of
    its systems)."""

    def __init__(self, solvers=None, _handle=None, _count=0):
        if _handle is not None:
            self.solvers, self.count, self.b = [], _count, _handle
            return
        self.solvers = list(solvers)
        n = self.count = len(self.solvers)
        self._ctx = (ctypes.c_void_p * n)(*[s.ctx.value if hasattr(s.ctx, "value") else s.ctx for s in self.solvers])
        self._n = (ctypes.c_int64 * n)(*[s.n for s in self.solvers])
        out = ctypes.c_void_p()
        _check(lib().h2_batch_create(ctypes.byref(out), ctypes.cast(self._ctx, ctypes.c_void_p),
                                     ctypes.cast(self._n, ctypes.c_void_p), n), None)
        self.b = out

    @classmethod
    def forest(cls, points_list, leaves=None, **kw):
        """Systems grouped by (leaf size, tree depth); leaves: one leaf size
        per system (None: the `leaf` parameter for all)."""
        pts, ptrs, ns = _point_arrays(points_list)
        lv = None if leaves is None else (ctypes.c_int32 * len(pts))(*[int(v) for v in leaves])
        out = ctypes.c_void_p()
        params = make_params(**kw)
        _check(lib().h2_batch_create_forest(ctypes.byref(out), ctypes.byref(params), ctypes.cast(ptrs, ctypes.c_void_p),
                                            ctypes.cast(ns, ctypes.c_void_p),
                                            None if lv is None else ctypes.cast(lv, ctypes.c_void_p), len(pts)), None)
        return cls(_handle=out, _count=len(pts))

    def _ptrs(self, arrs):
        a = (ctypes.c_void_p * len(arrs))(*[_ptr(x).value for x in arrs])
        return a

    def _err(self, st):
        if st != 0:
            m = lib().h2_batch_last_error(self.b)
            raise H2Error(st, m.decode() if m else "")

    def run(self, prec="fp16", B=None, target=1e-10, max_iters=100, check=True):
        """Factor all systems (prec None: keep) and solve each for B[i];
        returns (X list, relres, iters, seconds).  check=False: a system
        that stops above the target does not raise (see relres)."""
        n = self.count
        p = -1 if prec is None else PRECS[prec]
        rel = (ctypes.c_double * n)()
        its = (ctypes.c_int32 * n)()
        sec = ctypes.c_double()
        X = None
        if B is not None:
            X = [np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape) for b in B]
            pb, px = self._ptrs(B), self._ptrs(X)
            st = lib().h2_batch_run(self.b, p, ctypes.cast(pb, ctypes.c_void_p), ctypes.cast(px, ctypes.c_void_p),
                                    target, max_iters, ctypes.cast(rel, ctypes.c_void_p),
                                    ctypes.cast(its, ctypes.c_void_p), ctypes.byref(sec))
        else:
            st = lib().h2_batch_run(self.b, p, None, None, target, max_iters, None, None, ctypes.byref(sec))
        if check or st != -4:
            self._err(st)
        return X, list(rel), list(its), sec.value

    def tune(self, prec="fp16", B=None, target=1e-10, max_iters=100, check=True):
        X = [np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape) for b in B]
        pb, px = self._ptrs(B), self._ptrs(X)
        w = ctypes.c_int32()
        st = lib().h2_batch_tune(self.b, PRECS[prec], ctypes.cast(pb, ctypes.c_void_p), ctypes.cast(px, ctypes.c_void_p),
                                 target, max_iters, ctypes.byref(w))
        if check or st != -4:
            self._err(st)
        return w.value

    def stats(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 14)
        self._err(lib().h2_batch_stats(self.b, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if self.b:
            lib().h2_batch_destroy(self.b)
            self.b = None


def h2_set_stream(ctx, stream):
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().h2_set_stream(ctx, ctypes.c_void_p(int(handle) if handle else 0)), ctx)


def h2_stats(ctx) -> dict:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().h2_stats(ctx, buf, len(buf)), ctx)
    return json.loads(buf.value.decode())


def h2_export(ctx, name: str, level: int = 0) -> np.ndarray:
    cnt = ctypes.c_size_t()
    es = ctypes.c_int32()
    _check(lib().h2_export(ctx, name.encode(), level, None, 0, ctypes.byref(cnt), ctypes.byref(es)), ctx)
    dt = {("perm", 8): np.int64, ("piv", 4): np.int32, ("root_piv", 4): np.int32}.get(
        (name, es.value), np.float64 if es.value == 8 else np.float32)
    out = np.empty(cnt.value, dtype=dt)
    _check(lib().h2_export(ctx, name.encode(), level, _ptr(out), out.nbytes, ctypes.byref(cnt),
                           ctypes.byref(es)), ctx)
    return out


def h2_last_error(ctx=None) -> str:
    m = lib().h2_last_error(ctx)
    return m.decode() if m else ""


def h2_destroy(ctx):
    lib().h2_destroy(ctx)


# ------------------------------------------------------------ wrapper ---
class H2Solver:
    """A factorizable H^2 instance on the current CUDA device."""

    def __init__(self, ctx, n: int):
        self.ctx = ctx
        self.n = n

    @classmethod
    def build(cls, points, **kw):
        return cls(h2_build(make_params(**kw), points), len(points))

    @classmethod
    def build_predicted(cls, points, model, **kw):
        """h2_build with the ranks laid out by a trained rank model."""
        return cls(h2_build_predicted(make_params(**kw), points, model), len(points))

    @classmethod
    def build_gpu(cls, points, model=None, gs_sweeps=0, **kw):
        """h2_build with the compression on the GPU (ranks from the model, or
        each level's cap when model is None)."""
        return cls(h2_build_gpu(make_params(**kw), points, model, gs_sweeps), len(points))

    @classmethod
    def build_forest(cls, points_list, **kw):
        """Several systems of one tree depth as one block-diagonal instance;
        vectors are the systems' vectors concatenated."""
        return cls(h2_build_forest(make_params(**kw), points_list), int(sum(len(P) for P in points_list)))

    @classmethod
    def from_instance(cls, flat: dict, **kw):
        return cls(h2_import(make_params(**kw), flat), int(flat["N"]))

    def factor(self, prec="fp64"):
        h2_factor(self.ctx, prec)

    def release_factorization(self):
        _check(lib().h2_release_factorization(self.ctx), self.ctx)

    def solve(self, b, target=1e-10, max_iters=50, x=None):
        if x is None:
            x = np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape)
        st, rel, its = h2_solve(self.ctx, b, x, target, max_iters)
        return x, rel, its

    def solve_many(self, B, target=1e-10, max_iters=50):
        """One row of B per right-hand side; returns (X, relres list, iteration list)."""
        if isinstance(B, np.ndarray):
            B = np.ascontiguousarray(B, dtype=np.float64)
        else:
            B = B.contiguous()
        X = np.zeros_like(B) if isinstance(B, np.ndarray) else B.new_zeros(B.shape)
        st, rel, its = h2_solve_many(self.ctx, B, X, target, max_iters)
        return X, rel, its

    def matvec_many(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64) if isinstance(X, np.ndarray) else X.contiguous()
        Y = np.zeros_like(X) if isinstance(X, np.ndarray) else X.new_zeros(X.shape)
        h2_matvec_many(self.ctx, X, Y)
        return Y

    def ulv_apply(self, b):
        x = np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape)
        h2_ulv_apply(self.ctx, b, x)
        return x

    def matvec(self, x):
        y = np.zeros_like(x) if isinstance(x, np.ndarray) else x.new_zeros(x.shape)
        h2_matvec(self.ctx, x, y)
        return y

    def set_stream(self, stream):
        h2_set_stream(self.ctx, stream)

    def set_option(self, option, value):
        h2_set_option(self.ctx, option, value)

    def autotune(self, prec="fp16") -> dict:
        """h2_autotune: measure and keep the fastest kernel forms and launch
        shapes on this instance; the context is left factored in prec."""
        buf = ctypes.create_string_buffer(1 << 14)
        _check(lib().h2_autotune(self.ctx, PRECS[prec], buf, len(buf)), self.ctx)
        return json.loads(buf.value.decode())

    def matvec_arith(self, x, arith="fp64"):
        y = np.zeros_like(x) if isinstance(x, np.ndarray) else x.new_zeros(x.shape)
        h2_matvec_arith(self.ctx, x, y, arith)
        return y

    def set_refinement(self, method="auto", restart=30):
        h2_set_refinement(self.ctx, method, restart)

    def stats(self) -> dict:
        return h2_stats(self.ctx)

    def export(self, name, level=0):
        return h2_export(self.ctx, name, level)

    def close(self):
        if self.ctx:
            h2_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
