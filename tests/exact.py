"""Exact-rational helpers for pinning FP32/FP64 arithmetic in the tests.

round_f32 rounds an exact rational to the nearest float32 (ties to even), so a
single correctly-rounded FP32 operation can be replayed as
round_f32(exact result of the operation on the float32 operands)."""
from fractions import Fraction

import numpy as np


def F(x):
    return Fraction(float(x))


def round_f32(q: Fraction) -> np.float32:
    if q == 0:
        return np.float32(0.0)
    c = np.float32(float(q))  # within one float32 ulp of the exact value
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        if not np.isfinite(cand):
            continue
        err = abs(Fraction(float(cand)) - q)
        if best is None or err < best[0] or (err == best[0] and int(cand.view(np.uint32)) % 2 == 0):
            best = (err, cand)
    return np.float32(best[1])


def f32_add(a, b):
    return round_f32(F(a) + F(b))


def f32_sub(a, b):
    return round_f32(F(a) - F(b))


def f32_mul(a, b):
    return round_f32(F(a) * F(b))


def f32_div(a, b):
    return round_f32(F(a) / F(b))


def f32_fma(a, b, c):
    return round_f32(F(a) * F(b) + F(c))


def f32_sqrt(a):
    # sqrt of a float32 correctly rounded in binary64, then to binary32, is the
    # correctly rounded binary32 square root (53 >= 2*24 + 2).
    return np.float32(np.sqrt(np.float64(np.float32(a))))
