"""The compensated dot product the substrate kernels accumulate with (Dot2
of Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
Comput. 26(6), 2005), emulated step by step in float32 on the host: on sums
of large weights it lands within about one float32 rounding of the exact
value, where plain float32 accumulation drifts by many.  This pins the
method the kernels follow; the GPU tests pin the kernels themselves."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    z = f32(s - a)
    return s, f32(f32(a - f32(s - z)) + f32(b - z))


def two_prod(x, w):
    p = f32(x * w)
    # x*w - p is exact in float64 (both factors have 24-bit significands)
    # and representable in float32, so this is the FMA's result
    return p, f32(np.float64(x) * np.float64(w) - np.float64(p))


def dot2(xs, ws):
    s, c = f32(0), f32(0)
    for x, w in zip(xs, ws):
        p, pe = two_prod(x, w)
        s, e = two_sum(s, p)
        c = f32(c + f32(e + pe))
    return f32(s + c)


def naive(xs, ws):
    s = f32(0)
    for x, w in zip(xs, ws):
        s = f32(np.float64(x) * np.float64(w) + np.float64(s))      # one FMA: a single rounding
    return s


def exact(xs, ws):
    return float(sum(Fraction(float(x)) * Fraction(float(w)) for x, w in zip(xs, ws)))


def test_dot2_is_within_a_rounding_of_the_exact_sum():
    rng = np.random.default_rng(0)
    worst_dot2 = worst_naive = 0.0
    for _ in range(300):
        xs = rng.standard_normal(64).astype(np.float32)
        ws = (rng.standard_normal(64) * 8.0).astype(np.float32)     # large weights, as CPPN blocks carry
        ref = exact(xs, ws)
        ulp = float(np.spacing(f32(abs(ref)))) if ref else float(np.spacing(f32(1e-30)))
        worst_dot2 = max(worst_dot2, abs(float(dot2(xs, ws)) - ref) / ulp)
        worst_naive = max(worst_naive, abs(float(naive(xs, ws)) - ref) / ulp)
    assert worst_dot2 <= 1.0                 # correctly rounded or one ulp off
    assert worst_naive > 4.0 * max(worst_dot2, 0.5)


def test_dot2_with_cancellation():
    # terms that cancel to a small result: the plain sum loses the digits,
    # the compensated one keeps them
    xs = np.array([1.0, 1.0, -1.0, 1.0], dtype=np.float32)
    ws = np.array([1e8, 1.0, 1e8, 3.0e-3], dtype=np.float32)
    assert abs(float(dot2(xs, ws)) - exact(xs, ws)) <= float(np.spacing(f32(1.003)))
    assert abs(float(naive(xs, ws)) - exact(xs, ws)) > 0.5
