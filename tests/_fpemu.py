"""Exact IEEE-754 helpers in numpy for checking a learned index on the CPU.

Independent of both the oracle and the CUDA library.  Used to recompute, from
an index's stored parameters, the leaf each key is routed to and each key's
prediction error, bit for bit as correctly rounded hardware computes them:

  u64_to_f32   uint64 -> float32, round to nearest even (integer arithmetic)
  fma32        float32 a*x+b with one rounding (exact product in float64,
               TwoSum for the addition, explicit fix of the single
               double-rounding case: a float64 sum that lands exactly on a
               float32 midpoint while the exact sum does not)

The helpers are themselves pinned against exact rational arithmetic
(`fractions.Fraction`) in tests/test_fpemu.py.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

_U = np.uint64


def u64_to_f32(x: np.ndarray) -> np.ndarray:
    """Correctly rounded uint64 -> float32."""
    x = np.asarray(x, dtype=np.uint64)
    out = np.empty(x.shape, dtype=np.float32)
    small = x < _U(1 << 24)
    out[small] = x[small].astype(np.float32)        # exact
    big = ~small
    if np.any(big):
        v = x[big]
        # bit length via float64 exponent of v (v < 2^64); correct it exactly
        k = np.floor(np.log2(v.astype(np.float64))).astype(np.int64)
        k = np.where((k < 63) & ((v >> (k + 1).astype(np.uint64)) > 0), k + 1, k)
        k = np.where((v >> k.astype(np.uint64)) == 0, k - 1, k)
        shift = (k - 23).astype(np.uint64)
        q = v >> shift
        rem = v - (q << shift)
        half = _U(1) << (shift - _U(1))
        up = (rem > half) | ((rem == half) & ((q & _U(1)) == _U(1)))
        q = q + up.astype(np.uint64)
        out[big] = np.ldexp(q.astype(np.float64), shift.astype(np.int64)).astype(np.float32)
    return out


def _two_sum(a: np.ndarray, b: np.ndarray):
    s = a + b
    bb = s - a
    err = (a - (s - bb)) + (b - bb)
    return s, err


def fma32(a, x, b) -> np.ndarray:
    """float32 fused multiply-add, correctly rounded (round to nearest even)."""
    a = np.asarray(a, dtype=np.float32).astype(np.float64)
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    b = np.asarray(b, dtype=np.float32).astype(np.float64)
    p = a * x                                  # exact: 24 + 24 bits <= 53
    s, t = _two_sum(p, b)                      # s + t == p + b exactly
    r = s.astype(np.float32)
    # neighbours of s on the float32 grid and their midpoint (exact in f64)
    r64 = r.astype(np.float64)
    other = np.where(r64 <= s, np.nextafter(r, np.float32(np.inf)),
                     np.nextafter(r, np.float32(-np.inf))).astype(np.float64)
    mid = (r64 + other) * 0.5
    on_mid = (s == mid) & (t != 0.0)
    if np.any(on_mid):
        up = t > 0
        lo = np.minimum(r64, other)
        hi = np.maximum(r64, other)
        fixed = np.where(up, hi, lo).astype(np.float32)
        r = np.where(on_mid, fixed, r)
    return r


def round_fraction_f32(q: Fraction) -> np.float32:
    """Round an exact rational to float32 (nearest, ties to even); normal range."""
    if q == 0:
        return np.float32(0.0)
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    # q in [2^e, 2^(e+1)); significand with 23 fraction bits
    scaled = q * Fraction(2) ** (23 - e)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return np.float32(sign * float(Fraction(m) * Fraction(2) ** (e - 23)))


def round_fraction_f64(q: Fraction) -> float:
    """Python's float(Fraction) is correctly rounded (nearest, ties to even)."""
    return float(q)


def fma64_exact(a: float, x: float, b: float) -> float:
    """float64 fused multiply-add via exact rationals (slow; small inputs)."""
    return round_fraction_f64(Fraction(a) * Fraction(x) + Fraction(b))


def leaf_of_f32(keys: np.ndarray, a0: np.float32, b0: np.float32, L: int) -> np.ndarray:
    """Single-precision root: clamp(floor(fmaf(a0, float(x), b0)), 0, L-1)."""
    fx = u64_to_f32(keys)
    v = np.floor(fma32(np.full(fx.shape, a0, np.float32), fx,
                       np.full(fx.shape, b0, np.float32)).astype(np.float64))
    v = np.where(np.isnan(v), -1.0, v)
    return np.clip(v, 0, L - 1).astype(np.int64)


def leaf_pred_f32(keys: np.ndarray, base: np.ndarray, a: np.ndarray,
                  b: np.ndarray) -> np.ndarray:
    """Single-precision leaf prediction floor(fmaf(a, D, b)), D = x - base
    signed and rounded to float32, clamped to [-2^40, 2^40]."""
    keys = np.asarray(keys, np.uint64)
    base = np.asarray(base, np.uint64)
    ge = keys >= base
    d = np.where(ge, keys - base, base - keys)
    df = u64_to_f32(d)
    df = np.where(ge, df, -df).astype(np.float32)
    v = np.floor(fma32(a, df, b).astype(np.float64))
    return np.clip(v, -(2.0 ** 40), 2.0 ** 40).astype(np.int64)
