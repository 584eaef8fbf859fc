"""Pins for the exact IEEE helpers against rational arithmetic."""
from fractions import Fraction

import numpy as np

from tests import _fpemu as fe


def _f32_exact(v) -> Fraction:
    return Fraction(float(np.float32(v)))


def test_u64_to_f32_matches_rational_rounding():
    rng = np.random.default_rng(1)
    vals = list(rng.integers(0, 2**63, 2000, dtype=np.uint64))
    vals += [np.uint64(v) for v in (0, 1, 2**24 - 1, 2**24, 2**24 + 1, 2**24 + 2,
                                     2**24 + 3, 2**25 + 2, 2**25 + 6, 2**63,
                                     2**63 + 2**39, 2**64 - 1, 2**53 + 1)]
    vals = np.array(vals, dtype=np.uint64)
    got = fe.u64_to_f32(vals)
    for v, g in zip(vals, got):
        assert g == fe.round_fraction_f32(Fraction(int(v))), int(v)


def test_fma32_matches_rational_rounding_random():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(3000).astype(np.float32)
    x = (rng.standard_normal(3000) * 1e6).astype(np.float32)
    b = (rng.standard_normal(3000) * 1e3).astype(np.float32)
    got = fe.fma32(a, x, b)
    for ai, xi, bi, g in zip(a, x, b, got):
        want = fe.round_fraction_f32(_f32_exact(ai) * _f32_exact(xi) + _f32_exact(bi))
        assert g == want


def test_fma32_double_rounding_cases():
    # Exact sum just above a float32 midpoint, float64 sum on the midpoint:
    # a*x = 2^-24 (1 + 2^-32) (641 * 6700417 = 2^32 + 1), b = 1.
    a = np.float32(641 * 2.0 ** -28)
    x = np.float32(6700417 * 2.0 ** -28)
    got = fe.fma32(np.array([a]), np.array([x]), np.array([np.float32(1.0)]))[0]
    assert got == np.float32(1.0 + 2.0 ** -23)
    # Exact sum just below a midpoint whose tie would round up:
    # a*x = 2^-24 - 2^-70, b = 1 + 2^-23.
    a = np.float32(1.0 + 2.0 ** -23)
    x = np.float32(2.0 ** -24 * (1.0 - 2.0 ** -23))
    b = np.float32(1.0 + 2.0 ** -23)
    got = fe.fma32(np.array([a]), np.array([x]), np.array([b]))[0]
    assert got == np.float32(1.0 + 2.0 ** -23)
    # exact midpoint with no residual: ties to even
    got = fe.fma32(np.array([np.float32(1.0)]), np.array([np.float32(2.0 ** -24)]),
                   np.array([np.float32(1.0)]))[0]
    assert got == np.float32(1.0)
