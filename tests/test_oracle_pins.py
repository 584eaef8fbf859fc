"""Pins for the CPU oracle against what the paper and the mathematics fix.

The oracle is pinned to things other than itself:
  * the nested-loop definition of the join (brute force, tiny inputs);
  * a library binary search (numpy.searchsorted) per probe;
  * the closed form |J| = sum_k mult_R(k) * mult_S(k) from two histograms;
  * hand-derived fixtures under tests/golden/ (each cites its passage);
  * exact rational least squares for the model fits;
  * invariants of the two-level RMI (Section 2.D): every key of R lies
    inside its leaf's error window, the windows are the exact min/max of the
    errors, leaves are contiguous ranges, linear keys give errors in [-1, 1];
  * the learned lookup returns the same [lb, ub) as the sort-merge join.
A few tests plant a mistake in a copy of the oracle's output and check that
the comparison used by the pins rejects it.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import _fpemu as fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pairs_as_list(p):
    return [(int(r), int(s)) for r, s in p]


def _rand_case(rng, n, m, alphabet):
    R = np.sort(rng.integers(0, alphabet, n, dtype=np.uint64)) if n else np.zeros(0, np.uint64)
    S = rng.integers(0, alphabet, m, dtype=np.uint64) if m else np.zeros(0, np.uint64)
    return R, S


# ------------------------------------------------------------------- join --

@pytest.mark.parametrize("seed", range(150))
def test_join_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 60))
    m = int(rng.integers(0, 60))
    alphabet = [2, 5, 30, 1000, 2**64 - 1][seed % 5]
    R, S = _rand_case(rng, n, m, alphabet)
    got = _pairs_as_list(oracle.join_pairs(R, S))
    want = oracle.brute_force_join(R, S)
    assert got == want


def test_join_extreme_and_equal_keys_brute_force():
    top = np.uint64(2**64 - 1)
    cases = [
        (np.array([0, 0, 0, 0], np.uint64), np.array([0, 0, 0], np.uint64)),
        (np.array([top, top], np.uint64), np.array([top, 0, top], np.uint64)),
        (np.array([0, 1, top], np.uint64), np.array([top, 1, 0, 2], np.uint64)),
        (np.zeros(0, np.uint64), np.array([1, 2], np.uint64)),
        (np.array([1, 2], np.uint64), np.zeros(0, np.uint64)),
        (np.zeros(0, np.uint64), np.zeros(0, np.uint64)),
    ]
    for R, S in cases:
        assert _pairs_as_list(oracle.join_pairs(R, S)) == oracle.brute_force_join(R, S)


def test_join_ranges_match_library_binary_search():
    rng = np.random.default_rng(7)
    for alphabet in (50, 10**6, 2**63):
        R, S = _rand_case(rng, 20000, 30000, alphabet)
        lo, hi, total = oracle.join_ranges(R, S)
        assert np.array_equal(lo, np.searchsorted(R, S, side="left").astype(np.uint64))
        assert np.array_equal(hi, np.searchsorted(R, S, side="right").astype(np.uint64))
        assert total == int(np.sum(hi - lo))


def test_join_total_closed_form_from_histograms():
    rng = np.random.default_rng(8)
    R, S = _rand_case(rng, 50000, 70000, 3000)
    _, _, total = oracle.join_ranges(R, S)
    kr, cr = np.unique(R, return_counts=True)
    ks, cs = np.unique(S, return_counts=True)
    common, ir, is_ = np.intersect1d(kr, ks, return_indices=True)
    assert total == int(np.sum(cr[ir].astype(np.int64) * cs[is_].astype(np.int64)))


def test_join_self_join_unique_is_identity():
    R = np.unique(np.random.default_rng(9).integers(0, 2**63, 5000, dtype=np.uint64))
    p = oracle.join_pairs(R, R)
    assert np.array_equal(p[:, 0], np.arange(R.size)) and np.array_equal(p[:, 1], np.arange(R.size))


def test_join_rejects_unsorted_R():
    with pytest.raises(oracle.OracleError):
        oracle.join_ranges(np.array([3, 1], np.uint64), np.array([1], np.uint64))


def _read_join_golden(name):
    R = S = None
    pairs = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "R":
                R = np.array([int(t) for t in tok[1:]], dtype=np.uint64)
            elif tok[0] == "S":
                S = np.array([int(t) for t in tok[1:]], dtype=np.uint64)
            else:
                pairs.append((int(tok[0]), int(tok[1])))
    return R, S, pairs


@pytest.mark.parametrize("name", ["join_small.txt", "join_extremes.txt"])
def test_join_golden(name):
    R, S, pairs = _read_join_golden(name)
    assert _pairs_as_list(oracle.join_pairs(R, S)) == pairs


def test_planted_mistakes_are_caught():
    """Corrupt copies of a correct result must fail the pins' comparisons."""
    rng = np.random.default_rng(10)
    R, S = _rand_case(rng, 40, 40, 6)
    good = _pairs_as_list(oracle.join_pairs(R, S))
    want = oracle.brute_force_join(R, S)
    assert good == want and len(good) > 2
    dropped = good[:-1]
    off_by_one = [(r + 1, s) if k == 0 else (r, s) for k, (r, s) in enumerate(good)]
    transposed = [(s, r) for r, s in good]
    for bad in (dropped, off_by_one, transposed):
        assert bad != want
    # the histogram closed form catches a dropped pair too
    kr, cr = np.unique(R, return_counts=True)
    ks, cs = np.unique(S, return_counts=True)
    _, ir, is_ = np.intersect1d(kr, ks, return_indices=True)
    assert len(dropped) != int(np.sum(cr[ir] * cs[is_]))


# -------------------------------------------------------------------- RMI --

def _exact_lsq(x, y):
    k = len(x)
    if k == 0:
        return Fraction(0), Fraction(0)
    mx = sum(x, Fraction(0)) / k
    my = sum(y, Fraction(0)) / k
    sxx = sum(((xi - mx) ** 2 for xi in x), Fraction(0))
    sxy = sum(((xi - mx) * (yi - my) for xi, yi in zip(x, y)), Fraction(0))
    a = sxy / sxx if sxx > 0 else Fraction(0)
    if a < 0:
        a = Fraction(0)
    return a, my - a * mx


def _read_rmi_golden():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "rmi_small.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"leaves": []}
                cases.append(cur)
            elif tok[0] == "R":
                cur["R"] = np.array([int(t) for t in tok[1:]], dtype=np.uint64)
            elif tok[0] == "L":
                cur["L"] = int(tok[1])
            elif tok[0] == "root":
                cur["root"] = [Fraction(t) for t in tok[1:]]
            elif tok[0] == "leaf_lo":
                cur["leaf_lo"] = [int(t) for t in tok[1:]]
            elif tok[0] == "leaf":
                cur["leaves"].append((Fraction(tok[1]), Fraction(tok[2]), int(tok[3]), int(tok[4])))
    return cases


@pytest.mark.parametrize("fp64", [False, True])
def test_rmi_golden(fp64):
    for c in _read_rmi_golden():
        m = oracle.rmi_fit(c["R"], c["L"], fp64=fp64)
        for got, want in zip(m.root_fit, c["root"]):
            assert abs(Fraction(float(got)) - want) <= Fraction(1, 10**12) * (1 + abs(want))
        assert list(m.leaf_lo) == c["leaf_lo"]
        for l, (a, b, elo, ehi) in enumerate(c["leaves"]):
            assert abs(Fraction(float(m.leaf_fit[l, 0])) - a) <= Fraction(1, 10**12)
            assert abs(Fraction(float(m.leaf_fit[l, 1])) - b) <= Fraction(1, 10**12)
            assert (m.err[l, 0], m.err[l, 1]) == (elo, ehi)


@pytest.mark.parametrize("seed", range(6))
def test_rmi_fits_match_exact_least_squares(seed):
    rng = np.random.default_rng(100 + seed)
    n, L = 300, [1, 3, 8, 32, 64, 300][seed]
    R = np.sort(rng.integers(0, [2**20, 2**40, 2**63][seed % 3], n, dtype=np.uint64))
    m = oracle.rmi_fit(R, L, fp64=True)
    xs = [Fraction(float(np.float64(v))) for v in R]   # keys as doubles
    ys = [Fraction(float(np.float64(i) * L / n)) for i in range(n)]
    a0, b0 = _exact_lsq(xs, ys)
    scale = max(abs(float(a0)) * float(R[-1]), 1.0)
    assert abs(float(m.root_fit[0]) - float(a0)) * float(R[-1]) <= 1e-9 * scale
    assert abs(float(m.root_fit[1]) - float(b0)) <= 1e-9 * max(scale, abs(float(b0)))
    for l in range(L):
        lo, hi = int(m.leaf_lo[l]), int(m.leaf_lo[l + 1])
        if hi - lo < 2:
            continue
        x = [Fraction(int(R[i]) - int(R[lo])) for i in range(lo, hi)]
        y = [Fraction(i - lo) for i in range(lo, hi)]
        a, b = _exact_lsq(x, y)
        span = float(x[-1]) if x[-1] else 1.0
        assert abs(float(m.leaf_fit[l, 0]) - float(a)) * span <= 1e-9 * (hi - lo)
        assert abs(float(m.leaf_fit[l, 1]) - float(b)) <= 1e-9 * (hi - lo)


def _check_rmi_invariants(R, m):
    n, L = R.size, m.L
    lo = m.leaf_lo.astype(np.int64)
    assert lo[0] == 0 and lo[L] == n and np.all(np.diff(lo) >= 0)
    if not m.fp64 and n:
        # independent recomputation of the root with exact float32 emulation
        leaf = fe.leaf_of_f32(R, np.float32(m.root_dep[0]), np.float32(m.root_dep[1]), L)
        assert np.array_equal(leaf, np.repeat(np.arange(L), np.diff(lo)))
        # and of every key's error with the deployed leaf parameters
        owner = leaf
        base = R[lo[owner]]
        pred = fe.leaf_pred_f32(R, base, m.leaf_dep[owner, 0].astype(np.float32),
                                m.leaf_dep[owner, 1].astype(np.float32))
        err = np.arange(n) - lo[owner] - pred
        for l in range(L):
            e = err[lo[l]:lo[l + 1]]
            if e.size:
                assert (m.err[l, 0], m.err[l, 1]) == (e.min(), e.max())
            else:
                assert (m.err[l, 0], m.err[l, 1]) == (0, 0)
    # every key of R inside its window, found exactly
    for i in range(0, n, max(1, n // 2000)):
        q = oracle.rmi_lookup(R, m, int(R[i]))
        assert q["w_lo"] <= i < q["w_hi"] or q["lb"] <= i < q["ub"]
        assert q["lb"] <= i < q["ub"]


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "clusters"])
def test_rmi_invariants(kind, fp64):
    rng = np.random.default_rng(11)
    n = 20000
    if kind == "uniform":
        R = np.sort(rng.integers(0, 2**63, n, dtype=np.uint64))
    elif kind == "lognormal":
        R = np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    elif kind == "dups":
        R = np.sort(rng.integers(0, 500, n, dtype=np.uint64))
    else:   # tight clusters far apart: collapse under float32
        c = rng.integers(0, 2**62, 8, dtype=np.uint64)
        R = np.sort((c[rng.integers(0, 8, n)] + rng.integers(0, 1000, n).astype(np.uint64)))
    for L in (1, 37, 1024, 3 * n):
        m = oracle.rmi_fit(R, L, fp64=fp64)
        _check_rmi_invariants(R, m)


def test_rmi_linear_keys_have_unit_errors():
    for c, d, k, L in ((3, 5, 100, 64), (1, 0, 50, 10), (1000, 7, 33, 128)):
        n = k * L
        R = (np.arange(n, dtype=np.uint64) * np.uint64(c) + np.uint64(d))
        for fp64 in (False, True):
            m = oracle.rmi_fit(R, L, fp64=fp64)
            assert m.err[:, 0].min() >= -1 and m.err[:, 1].max() <= 1


@pytest.mark.parametrize("fp64", [False, True])
def test_rmi_lookup_equals_sort_merge(fp64):
    rng = np.random.default_rng(12)
    R = np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(30000))).astype(np.uint64))
    R = np.sort(np.concatenate([R, R[::7], R[::13]]))     # duplicates too
    S = np.concatenate([rng.choice(R, 3000),
                        rng.integers(0, int(R[-1]) * 2, 3000, dtype=np.uint64),
                        np.array([0, 1, int(R[0]) - 1, int(R[-1]) + 1, 2**64 - 1], np.uint64)])
    assert S.dtype == np.uint64
    lo, hi, _ = oracle.join_ranges(R, S)
    for L in (1, 100, 4096):
        m = oracle.rmi_fit(R, L, fp64=fp64)
        for j in range(S.size):
            q = oracle.rmi_lookup(R, m, int(S[j]))
            assert (q["lb"], q["ub"]) == (lo[j], hi[j])
            assert q["w_lo"] <= q["lb"] <= q["ub"] <= q["w_hi"]


def test_rmi_degenerate_inputs():
    for R in (np.zeros(0, np.uint64), np.array([5], np.uint64),
              np.full(100, 42, np.uint64), np.array([0, 2**64 - 1], np.uint64)):
        for L in (1, 2, 1000):
            for fp64 in (False, True):
                m = oracle.rmi_fit(R, L, fp64=fp64)
                assert m.leaf_lo[0] == 0 and m.leaf_lo[L] == R.size
                for x in list(R[:3]) + [0, 7, 2**64 - 1]:
                    q = oracle.rmi_lookup(R, m, int(x))
                    assert q["lb"] == np.searchsorted(R, np.uint64(x), "left")
                    assert q["ub"] == np.searchsorted(R, np.uint64(x), "right")
    with pytest.raises(oracle.OracleError):
        oracle.rmi_fit(np.array([2, 1], np.uint64), 4)


def test_unsorted_join_equals_nested_loops_and_histograms():
    """The sort-based join of two unsorted relations (Section 4): equal to the
    nested-loop definition on small inputs (duplicates on both sides,
    extreme keys, empty sides) and to the histogram closed form on larger
    ones."""
    rng = np.random.default_rng(77)
    for t in range(60):
        n, m = int(rng.integers(0, 120)), int(rng.integers(0, 120))
        R = rng.integers(0, 25, n).astype(np.uint64)
        S = rng.integers(0, 25, m).astype(np.uint64)
        if t % 7 == 0:
            R[: n // 3] = np.uint64(2**64 - 1)
        got = oracle.join_pairs_unsorted(R, S)
        want = sorted((j, i) for i, j in oracle.brute_force_join(R, S))
        assert [(int(s), int(r)) for r, s in got] == want
    R = rng.integers(0, 5000, 200000).astype(np.uint64)
    S = rng.integers(0, 6000, 150000).astype(np.uint64)
    got = oracle.join_pairs_unsorted(R, S)
    cr = np.bincount(R.astype(np.int64), minlength=6000)
    cs = np.bincount(S.astype(np.int64), minlength=6000)
    assert got.shape[0] == int(np.sum(cr * cs))
    assert np.all(R[got[:, 0]] == S[got[:, 1]])
