"""Exact IEEE-754 helpers in numpy for checking a learned index on the CPU.

Independent of both the oracle and the CUDA library.  Used to recompute, from
an index's stored parameters, the leaf each key is routed to and each key's
prediction error, bit for bit as correctly rounded hardware computes them:

  u64_to_f32   uint64 -> float32, round to nearest even (integer arithmetic)
  fma32        float32 a*x+b with one rounding (exact product in float64,
               TwoSum for the addition, explicit fix of the single
               double-rounding case: a float64 sum that lands exactly on a
               float32 midpoint while the exact sum does not)
  u64_to_f64   uint64 -> float64, round to nearest even (integer arithmetic)
  floor_fma64  floor(fma(a, x, b)) in float64 with one rounding: the exact
               value a*x + b as an unevaluated sum (Dekker's exact product
               by Veltkamp splitting, TwoSum), its floor decided from that
               sum; the rare elements whose value lies within a few units in
               the last place of an integer (where the one rounding of the
               hardware fma can move the floor) are recomputed with exact
               rationals

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


# --------------------------------------------------------------- float64 --

def u64_to_f64(x: np.ndarray) -> np.ndarray:
    """Correctly rounded uint64 -> float64 (integer arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    out = np.empty(x.shape, dtype=np.float64)
    small = x < _U(1 << 53)
    out[small] = x[small].astype(np.float64)        # exact
    big = ~small
    if np.any(big):
        v = x[big]
        hi32 = (v >> _U(32)).astype(np.float64)      # exact (< 2^32)
        k = np.floor(np.log2(hi32)).astype(np.int64) + 32
        k = np.where((k < 63) & ((v >> (k + 1).astype(np.uint64)) > 0), k + 1, k)
        k = np.where((v >> k.astype(np.uint64)) == 0, k - 1, k)
        shift = (k - 52).astype(np.uint64)
        q = v >> shift
        rem = v - (q << shift)
        half = _U(1) << (shift - _U(1))
        up = (rem > half) | ((rem == half) & ((q & _U(1)) == _U(1)))
        q = q + up.astype(np.uint64)
        out[big] = np.ldexp(q.astype(np.float64), shift.astype(np.int64))
    return out


def _split(a: np.ndarray):
    c = 134217729.0 * a                         # 2^27 + 1 (Veltkamp)
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a: np.ndarray, b: np.ndarray):
    """p + e == a * b exactly (Dekker), no fma needed; finite, no underflow."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _ulp(v: np.ndarray) -> np.ndarray:
    v = np.abs(v)
    return np.nextafter(v, np.inf) - v


def floor_fma64(a, x, b) -> np.ndarray:
    """floor(fma(a, x, b)) for float64 arrays, as float64 (NaN stays NaN).

    fma rounds the exact value a*x + b once to float64; its floor differs
    from the floor of the exact value only where the exact value lies within
    half a unit in the last place below an integer.  The exact value is
    carried as s + w (+ a residual far below ulp(s)); elements whose floor
    that sum cannot settle are recomputed with exact rationals."""
    a = np.asarray(a, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    a, x, b = np.broadcast_arrays(a, x, b)
    with np.errstate(over="ignore", invalid="ignore"):
        p, e = _two_prod(a, x)
        s1, t1 = _two_sum(p, b)                  # s1 + t1 == p + b
        w1 = t1 + e                              # error <= 2^-53 |t1 + e|
        s, w = _two_sum(s1, w1)                  # s + w == s1 + w1, |w| <= ulp(s)/2
        k = np.floor(s)
        fl = np.where((s == k) & (w < 0), k - 1, k)
        # distance to the integer above, and how close the one rounding of
        # the fma (half an ulp) or the residual could bring the value to it
        gap_up = (fl + 1 - s) - w
        gap_dn = (s - fl) + w
        tol = 4 * _ulp(np.abs(s) + 1.0) + (np.abs(t1) + np.abs(e)) * 2.0 ** -50
        unsure = (gap_up <= tol) | (gap_dn <= tol) | ~np.isfinite(p) | ~np.isfinite(e)
    out = fl.astype(np.float64)
    out[np.isnan(a) | np.isnan(x) | np.isnan(b)] = np.nan
    idx = np.flatnonzero(unsure & ~(np.isnan(a) | np.isnan(x) | np.isnan(b)))
    for i in idx:
        ai, xi, bi = float(a.flat[i]), float(x.flat[i]), float(b.flat[i])
        try:
            v = float(Fraction(ai) * Fraction(xi) + Fraction(bi))
        except OverflowError:
            v = np.inf if (Fraction(ai) * Fraction(xi) + Fraction(bi)) > 0 else -np.inf
        out.flat[i] = np.floor(v)
    return out


def leaf_of_f64(keys: np.ndarray, a0: float, b0: float, L: int) -> np.ndarray:
    """Double-precision root: clamp(floor(fma(a0, double(x), b0)), 0, L-1)."""
    fx = u64_to_f64(keys)
    v = floor_fma64(np.float64(a0), fx, np.float64(b0))
    v = np.where(np.isnan(v), -1.0, v)
    return np.clip(v, 0, L - 1).astype(np.int64)


def leaf_pred_f64(keys: np.ndarray, base: np.ndarray, a: np.ndarray,
                  b: np.ndarray) -> np.ndarray:
    """Double-precision leaf prediction floor(fma(a, D, b)), D = x - base
    signed and rounded to float64, clamped to [-2^40, 2^40]."""
    keys = np.asarray(keys, np.uint64)
    base = np.asarray(base, np.uint64)
    ge = keys >= base
    d = np.where(ge, keys - base, base - keys)
    df = u64_to_f64(d)
    df = np.where(ge, df, -df)
    v = floor_fma64(np.asarray(a, np.float64), df, np.asarray(b, np.float64))
    return np.clip(v, -(2.0 ** 40), 2.0 ** 40).astype(np.int64)
