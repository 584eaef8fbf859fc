"""Pins of the oracle's RadixSpline (Section 2.D) and of the learned hash
index that uses it as the hash function (Section 3.C, RSHASH-INLJ).

  * the error guarantee: every distinct key's predicted position lies
    within eps (plus the floor) of the position of its first copy, checked
    with exact integers against the data;
  * greediness: every spline segment that does not end a chunk is maximal:
    stretching it to the next CDF point would put some point between them
    more than eps away from the line (exact rationals);
  * spline points are CDF points, strictly increasing, with the first and
    last key of every chunk; exactly linear keys give one segment per chunk;
  * the radix table: all spline points in [table[b], table[b+1]) have
    prefix b, and the table starts at 0 and ends at the number of points;
  * predictions are monotone, 0 below the smallest key and n above the
    largest;
  * the hash table: the closed form slot_d = d + max_{e<=d}(4 h_e - e);
    joins through it equal the sort-merge join and brute force;
  * planted mistakes (a spline position moved past eps, two positions
    swapped, a lost last point) are caught.
"""
import zlib
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _relation(kind, rng, n):
    if kind == "uniform":
        return np.unique(rng.integers(0, 2**63, n, dtype=np.uint64))
    if kind == "lognormal":
        return np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    if kind == "seqh":
        keys = np.cumsum(1 + (rng.random(n) < 0.1)).astype(np.uint64)
        return np.repeat(keys, rng.integers(1, 6, n))
    if kind == "extremes":
        return np.unique(np.concatenate([rng.integers(0, 2**64 - 1, n, dtype=np.uint64,
                                                      endpoint=True),
                                         np.array([0, 2**64 - 1], dtype=np.uint64)]))
    raise ValueError(kind)


def _cdf(R):
    vals, first = np.unique(R, return_index=True)
    return vals, first


def _line_y(x0, y0, x1, y1, x):
    return Fraction(int(y0)) + Fraction(int(x) - int(x0)) * (int(y1) - int(y0)) / (int(x1) - int(x0))


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "seqh", "extremes"])
@pytest.mark.parametrize("eps,chunk", [(0, 0), (2, 64), (16, 1024), (64, 0)])
def test_error_guarantee_and_spline_points(kind, eps, chunk):
    rng = np.random.default_rng(zlib.crc32(f"{kind}{eps}{chunk}".encode()))
    R = _relation(kind, rng, 3000)
    rs = oracle.rs_build(R, eps=eps, chunk=chunk, rbits=10)
    vals, first = _cdf(R)
    D = vals.size
    # spline points are CDF points, strictly increasing, chunk ends included
    idx = np.searchsorted(vals, rs.sx)
    assert np.array_equal(vals[idx], rs.sx) and np.array_equal(first[idx], rs.sy)
    assert np.all(np.diff(rs.sx.astype(np.float64)) > 0) or rs.sx.size <= 1
    c = chunk or D
    ends = sorted({0, D - 1} | set(range(0, D, c)) | {min(D, a + c) - 1 for a in range(0, D, c)})
    assert set(ends) <= set(idx.tolist())
    # error guarantee, exact: floor(line) within [first - eps - 1, first + eps]
    pred = oracle.rs_predict(rs, vals).astype(np.int64)
    assert np.all(pred >= first - eps - 1) and np.all(pred <= first + eps)
    # and the unfloored line within eps of every CDF point (exact rationals)
    for i in range(rs.sx.size - 1):
        a, b = idx[i], idx[i + 1]
        for d in range(a + 1, b, max(1, (b - a) // 7)):
            y = _line_y(rs.sx[i], rs.sy[i], rs.sx[i + 1], rs.sy[i + 1], vals[d])
            assert abs(y - int(first[d])) <= eps


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "seqh"])
def test_segments_are_maximal(kind):
    """Greedy corridor: a segment ends only where it must."""
    rng = np.random.default_rng(7)
    R = _relation(kind, rng, 1500)
    eps, chunk = 4, 0
    rs = oracle.rs_build(R, eps=eps, chunk=chunk, rbits=8)
    vals, first = _cdf(R)
    idx = np.searchsorted(vals, rs.sx)
    for i in range(rs.sx.size - 1):
        a, b = int(idx[i]), int(idx[i + 1])
        if b + 1 >= vals.size:
            continue
        # the line from spline point a to the CDF point after b misses some point by > eps
        t = b + 1
        worst = max(abs(_line_y(vals[a], first[a], vals[t], first[t], vals[d]) - int(first[d]))
                    for d in range(a + 1, t))
        assert worst > eps, (i, a, b)


def test_linear_keys_give_one_segment_per_chunk():
    R = (np.arange(5000, dtype=np.uint64) * np.uint64(7) + np.uint64(11))
    assert oracle.rs_build(R, eps=0, chunk=0).sx.size == 2
    assert oracle.rs_build(R, eps=0, chunk=1000).sx.size == 10
    assert np.array_equal(oracle.rs_predict(oracle.rs_build(R, eps=0, chunk=0), R),
                          np.arange(5000, dtype=np.uint64))


@pytest.mark.parametrize("rbits", [1, 6, 12])
def test_radix_table_and_monotone_predictions(rbits):
    rng = np.random.default_rng(rbits)
    R = _relation("lognormal", rng, 4000)
    rs = oracle.rs_build(R, eps=8, chunk=256, rbits=rbits)
    S = rs.sx.size
    t = rs.table
    assert t[0] == 0 and t[-1] == S and np.all(np.diff(t.astype(np.int64)) >= 0)
    pref = (rs.sx - rs.sx[0]) >> np.uint64(rs.shift)
    for b in range(t.size - 1):
        assert np.all(pref[t[b]:t[b + 1]] == b)
    assert int(pref[-1]) < (1 << rbits)
    X = np.sort(np.concatenate([R, rng.integers(0, 2**50, 3000, dtype=np.uint64),
                                np.array([0, 2**64 - 1], dtype=np.uint64)]))
    p = oracle.rs_predict(rs, X)
    assert np.all(np.diff(p.astype(np.int64)) >= 0)
    assert np.all(p[X < R[0]] == 0) and np.all(p[X > R[-1]] == R.size)


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "seqh"])
@pytest.mark.parametrize("spk", [1, 4, 8])
def test_rs_hash_table_closed_form_and_joins(kind, spk):
    rng = np.random.default_rng(31 + spk)
    R = _relation(kind, rng, 5000)
    rs = oracle.rs_build(R, eps=16, chunk=512, rbits=10)
    h = oracle.rs_lhash_build(R, rs, spk)
    vals, first = _cdf(R)
    D = vals.size
    B = max(1, (spk * D + 3) // 4)
    assert h.D == D and h.B == B and np.array_equal(h.first, np.append(first, R.size))
    hb = oracle.rs_predict(rs, vals).astype(np.int64) * B // (R.size + 1)
    slot = np.arange(D) + np.maximum.accumulate(4 * hb - np.arange(D))
    assert np.array_equal(h.keys[slot], vals) and np.array_equal(h.pos[slot], np.arange(D))
    S = np.concatenate([R[rng.integers(0, R.size, 3000)], rng.integers(0, 2**63, 2000,
                                                                         dtype=np.uint64)])
    lo, hi, t = oracle.rs_lhash_join(R, h, S)
    lo2, hi2, t2 = oracle.join_ranges(R, S)
    assert t == t2 and np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    small = S[:60]
    want = oracle.brute_force_join(R[:400], small)
    h2 = oracle.rs_lhash_build(R[:400], oracle.rs_build(R[:400], eps=3, chunk=64, rbits=5), spk)
    lo3, hi3, _ = oracle.rs_lhash_join(R[:400], h2, small)
    got = [(r, j) for j in range(small.size) for r in range(int(lo3[j]), int(hi3[j]))]
    assert sorted(got) == sorted(want)


def test_planted_mistakes_are_caught():
    """Splines with a wrong position (a spline point's y moved past eps, two
    positions swapped) or a lost last point break the error guarantee or
    the range checks above."""
    rng = np.random.default_rng(3)
    R = _relation("lognormal", rng, 3000)
    vals, first = _cdf(R)
    eps = 4
    rs = oracle.rs_build(R, eps=eps, chunk=0, rbits=8)

    def within(sp):
        pred = oracle.rs_predict(sp, vals).astype(np.int64)
        return bool(np.all(pred >= first - eps - 1) and np.all(pred <= first + eps))

    assert within(rs)
    for i in range(1, rs.sx.size - 1, max(1, rs.sx.size // 8)):
        sy = rs.sy.copy()
        sy[i] += eps + 2
        assert not within(oracle.RadixSpline(eps, 0, 8, rs.sx, sy, rs.table, rs.shift, rs.n))
    sy = rs.sy.copy()
    sy[[1, 2]] = sy[[2, 1]]
    assert not within(oracle.RadixSpline(eps, 0, 8, rs.sx, sy, rs.table, rs.shift, rs.n))
    # dropping the last point: the largest keys are predicted at n
    bad = oracle.RadixSpline(eps, 0, 8, rs.sx[:-1], rs.sy[:-1], rs.table, rs.shift, rs.n)
    assert oracle.rs_predict(bad, vals[-1:])[0] == R.size != first[-1]
