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


def test_u64_to_f64_matches_rational_rounding():
    rng = np.random.default_rng(3)
    vals = list(rng.integers(0, 2**64 - 1, 3000, dtype=np.uint64, endpoint=True))
    vals += [np.uint64(v) for v in (0, 1, 2**53 - 1, 2**53, 2**53 + 1, 2**53 + 2, 2**53 + 3,
                                     2**54 + 2, 2**54 + 6, 2**63, 2**63 + 2**10,
                                     2**63 + 2**10 + 1, 2**64 - 1, 2**64 - 2**11)]
    vals = np.array(vals, dtype=np.uint64)
    got = fe.u64_to_f64(vals)
    for v, g in zip(vals, got):
        assert g == float(Fraction(int(v))), int(v)


def _floor_fma64_exact(a, x, b):
    return float(np.floor(float(Fraction(float(a)) * Fraction(float(x)) + Fraction(float(b)))))


def test_floor_fma64_matches_rational_rounding_random():
    rng = np.random.default_rng(4)
    k = 4000
    a = rng.standard_normal(k) * 10.0 ** rng.integers(-12, 3, k)
    x = rng.standard_normal(k) * 10.0 ** rng.integers(0, 19, k)
    b = rng.standard_normal(k) * 10.0 ** rng.integers(-3, 12, k)
    got = fe.floor_fma64(a, x, b)
    for ai, xi, bi, g in zip(a, x, b, got):
        assert g == _floor_fma64_exact(ai, xi, bi), (ai, xi, bi)


def test_floor_fma64_near_integers_and_cancellation():
    """Values within an ulp of an integer (where the one rounding of fma
    decides the floor), and products cancelled by the addend."""
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(1500):
        k = float(rng.integers(-2**20, 2**20))
        x = float(rng.integers(1, 2**60))
        a = k / x                                    # a*x within an ulp or so of k
        for da in (-2, -1, 0, 1, 2):
            aa = float(np.nextafter(a, np.inf)) if da > 0 else a
            for _ in range(abs(da) - 1 if da else 0):
                aa = float(np.nextafter(aa, np.inf if da > 0 else -np.inf))
            for b in (0.0, 0.5, -0.5, float(np.nextafter(0.0, 1.0)), 2.0 ** -60):
                cases.append((aa, x, b))
        # cancellation: a*x ~ -b with a large product
        big = float(rng.integers(2**40, 2**52))
        cases.append((big / x, x, -big + float(rng.integers(-3, 4))))
    a, x, b = (np.array(c, dtype=np.float64) for c in zip(*cases))
    got = fe.floor_fma64(a, x, b)
    for ai, xi, bi, g in zip(a, x, b, got):
        assert g == _floor_fma64_exact(ai, xi, bi), (ai, xi, bi)
    # an exact product one half-ulp below an integer: fma rounds up to it
    a = np.array([1.0 - 2.0 ** -53])
    assert fe.floor_fma64(a, np.array([1.0]), np.array([0.0]))[0] == 0.0
    x = np.array([3.0])
    a = np.array([(1.0 - 2.0 ** -53) / 3.0])
    assert fe.floor_fma64(a, x, np.array([0.0]))[0] == _floor_fma64_exact(a[0], 3.0, 0.0)


def test_floor_fma64_single_rounding_case():
    # a*x = 1 - 2^-60 rounds to 1 on its own; with b = -1 the fused result
    # is -2^-60 (floor -1) while a rounded product would give 0
    a = np.array([1.0 + 2.0 ** -30])
    x = np.array([1.0 - 2.0 ** -30])
    b = np.array([-1.0])
    assert fe.floor_fma64(a, x, b)[0] == -1.0 == _floor_fma64_exact(a[0], x[0], b[0])


def _as_gpu_dict(rmi):
    return {"root": rmi.root_dep, "leaf_lo": rmi.leaf_lo, "leaf_ab": rmi.leaf_dep, "err": rmi.err}


def test_tight_checks_accept_the_oracle_index_and_reject_a_planted_bound():
    """The fp32 and fp64 recomputations of leaves and error bounds agree
    with the oracle, which evaluates the models with the C library's fmaf /
    fma: two independent routes to the same integers.  A bound moved by one
    and a leaf boundary moved by one key are rejected."""
    import oracle
    from tests import _validate
    rng = np.random.default_rng(9)
    rels = [
        np.unique(rng.integers(0, 2**63, 60000, dtype=np.uint64)),
        np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(60000))).astype(np.uint64)),
        np.unique(np.concatenate([rng.integers(2**62, 2**62 + 10**6, 30000, dtype=np.uint64),
                                  np.array([0, 2**64 - 1], dtype=np.uint64)])),
        np.sort(rng.integers(0, 5000, 60000, dtype=np.uint64)),   # duplicates
    ]
    for R in rels:
        for fp64 in (False, True):
            for L in (1, 64, 4096):
                g = _as_gpu_dict(oracle.rmi_fit(R, L, fp64=fp64))
                (_validate.check_f64_tight if fp64 else _validate.check_f32_tight)(R, g)
    R = rels[1]
    for fp64 in (False, True):
        check = _validate.check_f64_tight if fp64 else _validate.check_f32_tight
        ora = oracle.rmi_fit(R, 256, fp64=fp64)
        nz = np.flatnonzero(np.diff(ora.leaf_lo) > 0)
        bad = _as_gpu_dict(ora)
        bad["err"] = ora.err.copy()
        bad["err"][nz[3], 1] += 1                     # window one key too wide
        try:
            check(R, bad)
            raise RuntimeError("a widened bound passed")
        except AssertionError:
            pass
        bad = _as_gpu_dict(ora)
        bad["leaf_lo"] = ora.leaf_lo.copy()
        bad["leaf_lo"][nz[5]] += 1                    # a key routed to the wrong leaf
        try:
            check(R, bad)
            raise RuntimeError("a moved leaf boundary passed")
        except AssertionError:
            pass
