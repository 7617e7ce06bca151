"""Exact rational evaluation of the direct-search map f, for pinning the oracle.

Independent of the oracle's C code: each operation is carried out on Python
Fractions and rounded to the nearest float32/float64 (ties to even) by an
explicit comparison of the exact value against its neighbouring floats.
"""
from fractions import Fraction

import numpy as np


def round_nearest(q, dtype):
    """Round the rational q to the nearest value of dtype, ties to even."""
    dtype = np.dtype(dtype).type
    if q == 0:
        return dtype(0.0)
    c = dtype(float(q))  # a candidate within a couple of ulps
    if not np.isfinite(c):
        return c
    best = None
    cands = [c, np.nextafter(c, dtype(np.inf)), np.nextafter(c, dtype(-np.inf))]
    for _ in range(2):
        cands += [np.nextafter(x, dtype(np.inf)) for x in cands] + [np.nextafter(x, dtype(-np.inf)) for x in cands]
    cands = sorted(set(float(x) for x in cands if np.isfinite(x)))
    for x in cands:
        d = abs(Fraction(x) - q)
        if best is None or d < best[0]:
            best = (d, x)
        elif d == best[0]:
            # tie: keep the one with an even last significand bit
            bits = np.array([x], dtype=dtype).view(np.uint32 if dtype == np.float32 else np.uint64)[0]
            if int(bits) & 1 == 0:
                best = (d, x)
    return dtype(best[1])


def trunc_u32(v):
    v = float(v)
    if not (v > 0.0):
        return 0
    if v >= 4294967296.0:
        return 0xFFFFFFFF
    return int(v)


def f_plain(H, X0, z, dtype):
    """trunc(m(H * m(z - X0))) with each operation rounded once."""
    D = round_nearest(Fraction(float(z)) - Fraction(float(X0)), dtype)
    return trunc_u32(round_nearest(Fraction(float(H)) * Fraction(float(D)), dtype))


def f_fma(H, W, z, dtype):
    """trunc(m(H z - W)) with a single rounding."""
    return trunc_u32(round_nearest(Fraction(float(H)) * Fraction(float(z)) - Fraction(float(W)), dtype))


def mul(a, b, dtype):
    return round_nearest(Fraction(float(a)) * Fraction(float(b)), dtype)


def add(a, b, dtype):
    return round_nearest(Fraction(float(a)) + Fraction(float(b)), dtype)
