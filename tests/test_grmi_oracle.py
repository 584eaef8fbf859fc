"""Pins for the oracle's gapped RMI (Section 3.A).

The gapped arrays and the GRMI lookup are pinned to things other than the
oracle's own code:
  * closed form of model-based insertion: inserting sorted keys, each at its
    predicted slot or right after the previous key, puts key i at
        slot_i = i + max_{j <= i} (pslot_j - j),
    and a slot s then holds the payload #{i : slot_i < s}; the predicted
    slots come from an independent float32 emulation of the model
    (tests/_fpemu.py) or from exact rational arithmetic for float64;
  * a model that predicts every key exactly (keys base + 8 i, one leaf)
    places key i at (1 + gaps) * i and finds every key with one load;
  * the lookup returns the same match ranges as the sort-merge join (the
    definition, itself pinned by test_oracle_pins.py) and, on tiny inputs,
    as the nested-loop definition;
  * the exponential search reads at most max(1, 2 ceil(log2(d + 1))) keys for
    a key of R placed d slots after its prediction.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import _fpemu as fe

TOP = np.uint64(2**64 - 1)


def _pslot_f32(R, m, gaps):
    """Predicted slot of every key of R with the float32 model, emulated."""
    n = R.size
    lo = m.leaf_lo.astype(np.int64)
    leaf = fe.leaf_of_f32(R, np.float32(m.root_dep[0]), np.float32(m.root_dep[1]), m.L)
    lo_k, hi_k = lo[leaf], lo[leaf + 1]
    pred = fe.leaf_pred_f32(R, R[np.minimum(lo_k, n - 1)], m.leaf_dep[leaf, 0].astype(np.float32),
                            m.leaf_dep[leaf, 1].astype(np.float32))
    p = np.clip(lo_k + pred, lo_k, hi_k)
    return p * (1 + gaps)


def _pslot_f64_exact(R, m, gaps):
    """Same with the float64 model, each fused multiply-add exactly rounded."""
    lo = m.leaf_lo.astype(np.int64)
    out = []
    for x in R:
        x = int(x)
        v = math.floor(fe.fma64_exact(float(m.root_dep[0]), float(x), float(m.root_dep[1])))
        leaf = 0 if not v >= 0 else min(int(v), m.L - 1)
        a, b = lo[leaf], lo[leaf + 1]
        p = a
        if b > a:
            base = int(R[a])
            d = float(x - base) if x >= base else -float(base - x)
            w = math.floor(fe.fma64_exact(float(m.leaf_dep[leaf, 0]), d, float(m.leaf_dep[leaf, 1])))
            p = a + max(-(2**40), min(2**40, w))
        out.append(min(max(p, a), b) * (1 + gaps))
    return np.array(out, dtype=np.int64)


def _closed_form_arrays(R, pslot, gaps):
    n = R.size
    i = np.arange(n, dtype=np.int64)
    slot = i + np.maximum.accumulate(pslot - i) if n else np.zeros(0, np.int64)
    C = max((1 + gaps) * n, int(slot[-1]) + 1 if n else 0)
    s = np.arange(C + 1, dtype=np.int64)
    pos = np.searchsorted(slot, s, side="left")          # keys placed before slot s
    keys = np.where(pos[:C] < n, R[np.minimum(pos[:C], max(n - 1, 0))] if n else TOP, TOP)
    return slot, keys.astype(np.uint64), pos.astype(np.uint32)


def _datasets(rng):
    n = 6000
    yield "uniform", np.sort(rng.integers(0, 2**63, n, dtype=np.uint64))
    yield "lognormal", np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    yield "dups", np.sort(rng.integers(0, 700, n, dtype=np.uint64))
    c = rng.integers(0, 2**62, 6, dtype=np.uint64)
    yield "clusters", np.sort(c[rng.integers(0, 6, n)] + rng.integers(0, 5000, n).astype(np.uint64))


@pytest.mark.parametrize("gaps", [0, 1, 4])
def test_insertion_matches_closed_form_f32(gaps):
    rng = np.random.default_rng(21)
    for kind, R in _datasets(rng):
        for L in (1, 13, 512):
            m = oracle.rmi_fit(R, L, fp64=False)
            g = oracle.grmi_build(R, m, gaps)
            pslot = _pslot_f32(R, m, gaps)
            slot, keys, pos = _closed_form_arrays(R, pslot, gaps)
            assert np.array_equal(g.slot_of_key.astype(np.int64), slot), (kind, L)
            assert np.array_equal(g.keys, keys), (kind, L)
            assert np.array_equal(g.pos, pos), (kind, L)
            assert np.all(slot >= pslot)


def test_insertion_matches_closed_form_f64_exact():
    rng = np.random.default_rng(22)
    R = np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(300))).astype(np.uint64))
    for L in (1, 9):
        m = oracle.rmi_fit(R, L, fp64=True)
        for gaps in (0, 4):
            g = oracle.grmi_build(R, m, gaps)
            slot, keys, pos = _closed_form_arrays(R, _pslot_f64_exact(R, m, gaps), gaps)
            assert np.array_equal(g.slot_of_key.astype(np.int64), slot)
            assert np.array_equal(g.keys, keys) and np.array_equal(g.pos, pos)


def test_exact_model_places_every_key_at_its_prediction():
    n = 5000
    R = np.uint64(1000) + np.arange(n, dtype=np.uint64) * np.uint64(8)
    for fp64 in (False, True):
        m = oracle.rmi_fit(R, 1, fp64=fp64)
        assert m.err[0, 0] == 0 and m.err[0, 1] == 0
        for gaps in (0, 1, 4):
            g = oracle.grmi_build(R, m, gaps)
            assert np.array_equal(g.slot_of_key, np.arange(n, dtype=np.uint64) * (1 + gaps))
            assert g.keys.size == (1 + gaps) * n
            lo, hi, total, loads = oracle.grmi_join(R, g, R)
            assert total == n and np.array_equal(lo, np.arange(n))
            # the lower bound is found with one load; the upper bound at the next slot
            assert np.all(loads <= 3)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("gaps", [0, 2, 4])
def test_lookup_equals_sort_merge(fp64, gaps):
    rng = np.random.default_rng(23 + gaps)
    for kind, R in _datasets(rng):
        S = np.concatenate([rng.choice(R, 2000), rng.integers(0, 2**64 - 1, 500, dtype=np.uint64),
                            rng.integers(0, int(R[-1]) + 2, 1500, dtype=np.uint64),
                            np.array([0, 1, int(R[0]) - 1 if R[0] else 0, int(R[-1]) + 1, TOP],
                                     np.uint64)])
        want_lo, want_hi, want_total = oracle.join_ranges(R, S)
        for L in (1, 64, 2048):
            g = oracle.grmi_build(R, oracle.rmi_fit(R, L, fp64=fp64), gaps)
            lo, hi, total, _ = oracle.grmi_join(R, g, S)
            assert total == want_total, (kind, L)
            assert np.array_equal(lo, want_lo) and np.array_equal(hi, want_hi), (kind, L)


@pytest.mark.parametrize("seed", range(60))
def test_lookup_matches_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(0, 40)), int(rng.integers(0, 40))
    alphabet = [3, 50, 2**64 - 1][seed % 3]
    R = np.sort(rng.integers(0, alphabet, n, dtype=np.uint64))
    S = rng.integers(0, alphabet, m, dtype=np.uint64)
    want = oracle.brute_force_join(R, S)
    for L in (1, 5):
        for gaps in (0, 3):
            g = oracle.grmi_build(R, oracle.rmi_fit(R, L, fp64=bool(seed % 2)), gaps)
            lo, hi, total, _ = oracle.grmi_join(R, g, S)
            got = [(i, j) for j in range(m) for i in range(int(lo[j]), int(hi[j]))]
            assert got == want and total == len(want)


def test_extreme_and_degenerate_relations():
    cases = [np.zeros(0, np.uint64), np.array([5], np.uint64), np.full(50, 42, np.uint64),
             np.array([0, TOP], np.uint64), np.array([0, 0, 1, TOP, TOP], np.uint64)]
    S = np.array([0, 1, 5, 42, 43, 2**63, TOP], np.uint64)
    for R in cases:
        for fp64 in (False, True):
            for gaps in (0, 4):
                g = oracle.grmi_build(R, oracle.rmi_fit(R, 3, fp64=fp64), gaps)
                assert g.pos[-1] == R.size and g.keys.size >= (1 + gaps) * R.size
                lo, hi, _, _ = oracle.grmi_join(R, g, S)
                assert np.array_equal(lo, np.searchsorted(R, S, "left"))
                assert np.array_equal(hi, np.searchsorted(R, S, "right"))


def test_search_cost_bound_for_keys_of_R():
    rng = np.random.default_rng(24)
    R = np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(20000))).astype(np.uint64))
    m = oracle.rmi_fit(R, 256, fp64=False)
    g = oracle.grmi_build(R, m, 4)
    pslot = _pslot_f32(R, m, 4)
    disp = g.slot_of_key.astype(np.int64) - pslot
    bound = np.maximum(1, 2 * np.ceil(np.log2(disp + 1)).astype(np.int64))
    lo, hi, total, loads = oracle.grmi_join(R, g, R)
    assert total == R.size and np.array_equal(lo, np.arange(R.size))
    keys = g.keys
    for i in range(0, R.size, 53):
        # the lower-bound search alone, walked by hand: q, q+1, q+3, ... then bisection
        x, q = R[i], int(pslot[i])
        cnt, off, a, b = 0, 0, q, keys.size
        while q + off < keys.size:
            cnt += 1
            if keys[q + off] >= x:
                b = q + off
                break
            a = q + off + 1
            off = 2 * off + 1
        while a < b:
            mid = (a + b) // 2
            cnt += 1
            if keys[mid] >= x:
                b = mid
            else:
                a = mid + 1
        assert g.pos[a] == i
        assert cnt <= bound[i]
        assert cnt < loads[i]          # the oracle also searched the upper bound


def test_planted_mistakes_are_caught():
    """Plausible wrong readings give arrays or answers that the pins reject."""
    rng = np.random.default_rng(25)
    R = np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(3000))).astype(np.uint64))
    m = oracle.rmi_fit(R, 16, fp64=False)
    g = oracle.grmi_build(R, m, 4)
    pslot = _pslot_f32(R, m, 4)
    i = np.arange(R.size)
    # insertion that ignores the previous key's slot (collisions overwrite)
    assert not np.array_equal(g.slot_of_key.astype(np.int64), np.maximum(pslot, i))
    # gaps filled with a copy of the previous key instead of the next one
    filled = np.zeros(g.keys.size, bool)
    filled[g.slot_of_key.astype(np.int64)] = True
    prev_fill = g.keys.copy()
    gaps = np.flatnonzero(~filled & (g.pos[:-1] > 0))
    prev_fill[gaps] = R[g.pos[gaps].astype(np.int64) - 1]
    assert not np.array_equal(prev_fill, g.keys)
    # a lookup that trusts the predicted slot without the exponential search
    lo, _, _, _ = oracle.grmi_join(R, g, R)
    naive = g.pos[np.minimum(pslot, g.keys.size)]
    assert not np.array_equal(naive, lo)
