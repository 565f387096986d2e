"""The FP32-pair dot product behind the mixed refinement's FP64 residual
(each FP64 entry m held as fl32(m) + fl32(m - fl32(m)), products split
exactly, running sums kept as an FP32 pair by an error-free two-sum), written
out here with NumPy float32 operations and checked against exact rational
arithmetic: the sum comes out to about 2^-46 of sum |m x|, where plain FP32
gives about 2^-24.  The sums across lanes and warps are formed the same way
(pairs added by the two-sum, one conversion to FP64 at the end).  This pins
the arithmetic the residual kernels use; the GPU tests compare those kernels
with the FP64 matvec."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def split(v):
    h = f32(v)
    return h, f32(v - np.float64(h))


def fma32(a, b, c):
    # a*b is exact in FP64 for FP32 inputs; one rounding of the FP64 sum
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def pair_dot(m, x):
    H, L = f32(0), f32(0)
    for mi, xi in zip(m, x):
        mh, ml = split(mi)
        xh, xl = split(xi)
        p = f32(mh * xh)
        e = f32(np.float64(mh) * np.float64(xh) - np.float64(p))  # exact product error
        small = fma32(mh, xl, fma32(ml, xh, e))
        s = f32(H + p)
        bb = f32(s - H)
        err = f32(f32(H - f32(s - bb)) + f32(p - bb))
        H = s
        L = f32(L + f32(small + err))
    return np.float64(H) + np.float64(L)


def test_pair_dot_reaches_fp64_level():
    rng = np.random.default_rng(3)
    for n in (16, 64, 256):
        m = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
        x = rng.standard_normal(n)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(m, x))
        scale = float(np.sum(np.abs(m * x)))
        got = pair_dot(m, x)
        assert abs(Fraction(float(got)) - exact) <= Fraction(2.0 ** -44) * Fraction(scale), n
        # plain FP32 is far coarser: the pin would catch a dropped term
        plain = float(np.dot(m.astype(f32), x.astype(f32)))
        assert abs(Fraction(plain) - exact) > Fraction(2.0 ** -40) * Fraction(scale), n


def test_pair_dot_without_low_parts_fails():
    """Dropping the low words (a plausible slip) costs the FP64 accuracy."""
    rng = np.random.default_rng(5)
    m, x = rng.standard_normal(128), rng.standard_normal(128)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(m, x))
    scale = float(np.sum(np.abs(m * x)))
    hi_only = pair_dot(m.astype(f32).astype(np.float64), x.astype(f32).astype(np.float64))
    assert abs(Fraction(float(hi_only)) - exact) > Fraction(2.0 ** -40) * Fraction(scale)


def pair_acc(m, x):
    """The running FP32 pair (H, L) of pair_dot, before any FP64 step."""
    H, L = f32(0), f32(0)
    for mi, xi in zip(m, x):
        mh, ml = split(mi)
        xh, xl = split(xi)
        p = f32(mh * xh)
        e = f32(np.float64(mh) * np.float64(xh) - np.float64(p))
        small = fma32(mh, xl, fma32(ml, xh, e))
        H, L = pair_add(H, L, p, small)
    return H, L


def pair_add(H, L, h, l, keep_error=True):
    """(H, L) + (h, l): the two-sum of the high words, its error joining the
    low words (the kernels' df_add)."""
    s = f32(H + h)
    bb = f32(s - H)
    err = f32(f32(H - f32(s - bb)) + f32(h - bb)) if keep_error else f32(0)
    return s, f32(L + f32(l + err))


def pair_tree(m, x, lanes=32, keep_error=True):
    """The dot product as the residual kernels now form it: each lane's pair
    over a strided share of the entries, the lanes added pairwise by a
    butterfly in pair arithmetic, one conversion to FP64 at the end."""
    parts = [pair_acc(m[k::lanes], x[k::lanes]) for k in range(lanes)]
    while len(parts) > 1:
        half = len(parts) // 2
        parts = [pair_add(*parts[k], *parts[k + half], keep_error=keep_error) for k in range(half)]
    H, L = parts[0]
    return np.float64(H) + np.float64(L)


def test_pair_tree_reduction_keeps_fp64_level():
    """Adding the lanes' pairs in pair arithmetic (no FP64 instruction until
    the result) stays at the pair arithmetic's accuracy; a two-sum that drops
    its error term (a plausible slip) falls to FP32 accuracy."""
    rng = np.random.default_rng(7)
    for n in (256, 1024):
        m = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
        x = rng.standard_normal(n)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(m, x))
        scale = Fraction(float(np.sum(np.abs(m * x))))
        got = pair_tree(m, x)
        assert abs(Fraction(float(got)) - exact) <= Fraction(2.0 ** -44) * scale, n
        sloppy = pair_tree(m, x, keep_error=False)
        assert abs(Fraction(float(sloppy)) - exact) > Fraction(2.0 ** -40) * scale, n
