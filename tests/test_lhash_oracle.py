"""Pins for the oracle's learned hash index (Section 3.C).

  * closed form of the table: distinct keys in key order, key d hashed to
    bucket h_d = p_d * B // (n + 1) and placed by linear probing, i.e. at
        slot_d = d + max_{e <= d} (4 h_e - e),
    a slot s holding payload #{d : slot_d < s}; p_d comes from the
    independent float32 emulation of the model (tests/_fpemu.py); first[d]
    is the first position of key d (numpy.unique);
  * evenly spaced keys (base + 8 i, one leaf: an exact model) stay in their
    hashed bucket: all but one are found with one slot read;
  * lookups equal the sort-merge join's ranges (duplicates, misses, extreme
    keys) and, on tiny inputs, the nested-loop definition;
  * planted wrong readings are rejected.
"""
import numpy as np
import pytest

import oracle
from tests import _fpemu as fe

TOP = np.uint64(2**64 - 1)


def _pred_f32(R, keys, m):
    """RMI prediction p(x) clamped to the leaf's positions (float32 model)."""
    n = R.size
    lo = m.leaf_lo.astype(np.int64)
    leaf = fe.leaf_of_f32(keys, np.float32(m.root_dep[0]), np.float32(m.root_dep[1]), m.L)
    a, b = lo[leaf], lo[leaf + 1]
    pred = fe.leaf_pred_f32(keys, R[np.minimum(a, n - 1)], m.leaf_dep[leaf, 0].astype(np.float32),
                            m.leaf_dep[leaf, 1].astype(np.float32))
    return np.where(b > a, np.clip(a + pred, a, b), a)


def _closed_form(R, m, spk):
    n = R.size
    dkey, first = np.unique(R, return_index=True)
    D = dkey.size
    B = max(1, (spk * D + 3) // 4)
    p = _pred_f32(R, dkey, m).astype(object)
    h = np.array([int(v) * B // (n + 1) for v in p], dtype=np.int64)
    d = np.arange(D, dtype=np.int64)
    slot = d + np.maximum.accumulate(4 * h - d) if D else np.zeros(0, np.int64)
    C = max(4 * B, int(slot[-1]) + 1 if D else 0)
    pos = np.searchsorted(slot, np.arange(C + 1), side="left")
    keys = np.where(pos[:C] < D, dkey[np.minimum(pos[:C], max(D - 1, 0))] if D else TOP, TOP)
    return slot, h, keys.astype(np.uint64), pos.astype(np.uint32), \
        np.append(first, n).astype(np.uint32), D, B


def _datasets(rng):
    n = 8000
    yield "uniform", np.sort(rng.integers(0, 2**63, n, dtype=np.uint64))
    yield "lognormal", np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    yield "dups", np.sort(rng.integers(0, 900, n, dtype=np.uint64))
    holes = np.flatnonzero(rng.random(3 * n) > 0.1).astype(np.uint64)[:n]     # sequential with holes
    yield "seq_holes", np.sort(np.repeat(holes[: n // 4], rng.integers(1, 8, n // 4)))


@pytest.mark.parametrize("spk", [1, 2, 4, 8])
def test_table_matches_closed_form(spk):
    rng = np.random.default_rng(51 + spk)
    for kind, R in _datasets(rng):
        for L in (1, 17, 1024):
            m = oracle.rmi_fit(R, L, fp64=False)
            h = oracle.lhash_build(R, m, spk)
            slot, hb, keys, pos, first, D, B = _closed_form(R, m, spk)
            assert (h.D, h.B) == (D, B), kind
            assert np.array_equal(h.keys, keys), (kind, L)
            assert np.array_equal(h.pos, pos), (kind, L)
            assert np.array_equal(h.first, first), (kind, L)
            assert np.all(slot >= 4 * hb)


def test_exact_model_keys_stay_in_their_bucket():
    n = 6000
    R = np.uint64(500) + np.arange(n, dtype=np.uint64) * np.uint64(8)
    for fp64 in (False, True):
        m = oracle.rmi_fit(R, 1, fp64=fp64)
        h = oracle.lhash_build(R, m, 4)
        lo, hi, total, loads = oracle.lhash_join(R, h, R)
        assert total == n and np.array_equal(lo, np.arange(n))
        # h(x_i) = i n // (n + 1) = max(i - 1, 0): keys 0 and 1 share bucket 0, every
        # other key has a bucket of its own, so no lookup leaves its bucket
        assert np.all(loads <= 2) and np.count_nonzero(loads == 1) == n - 1


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("spk", [1, 4])
def test_lookup_equals_sort_merge(fp64, spk):
    rng = np.random.default_rng(61 + spk)
    for kind, R in _datasets(rng):
        S = np.concatenate([rng.choice(R, 2500), rng.integers(0, 2**64 - 1, 500, dtype=np.uint64),
                            rng.integers(0, int(R[-1]) + 2, 1500, dtype=np.uint64),
                            np.array([0, 1, int(R[-1]) + 1, TOP], np.uint64)])
        want_lo, want_hi, want_total = oracle.join_ranges(R, S)
        for L in (1, 64, 4096):
            h = oracle.lhash_build(R, oracle.rmi_fit(R, L, fp64=fp64), spk)
            lo, hi, total, _ = oracle.lhash_join(R, h, S)
            assert total == want_total, (kind, L)
            assert np.array_equal(lo, want_lo) and np.array_equal(hi, want_hi), (kind, L)


@pytest.mark.parametrize("seed", range(40))
def test_lookup_matches_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n, mm = int(rng.integers(0, 40)), int(rng.integers(0, 40))
    alphabet = [3, 50, 2**64 - 1][seed % 3]
    R = np.sort(rng.integers(0, alphabet, n, dtype=np.uint64))
    S = rng.integers(0, alphabet, mm, dtype=np.uint64)
    want = oracle.brute_force_join(R, S)
    for L in (1, 5):
        for spk in (1, 4):
            h = oracle.lhash_build(R, oracle.rmi_fit(R, L, fp64=bool(seed % 2)), spk)
            lo, hi, total, _ = oracle.lhash_join(R, h, S)
            got = [(i, j) for j in range(mm) for i in range(int(lo[j]), int(hi[j]))]
            assert got == want and total == len(want)


def test_extreme_and_degenerate_relations():
    S = np.array([0, 1, 5, 42, 43, 2**63, TOP], np.uint64)
    for R in (np.zeros(0, np.uint64), np.array([5], np.uint64), np.full(50, 42, np.uint64),
              np.array([0, TOP], np.uint64), np.array([0, 0, 1, TOP, TOP], np.uint64)):
        for fp64 in (False, True):
            h = oracle.lhash_build(R, oracle.rmi_fit(R, 3, fp64=fp64), 4)
            assert h.pos[-1] == h.D and h.first[-1] == R.size
            lo, hi, _, _ = oracle.lhash_join(R, h, S)
            assert np.array_equal(lo, np.searchsorted(R, S, "left"))
            assert np.array_equal(hi, np.searchsorted(R, S, "right"))


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(71)
    R = np.sort(rng.integers(0, 3000, 20000, dtype=np.uint64))
    m = oracle.rmi_fit(R, 8, fp64=False)
    h = oracle.lhash_build(R, m, 4)
    slot, hb, keys, pos, first, D, B = _closed_form(R, m, 4)
    # placement without linear probing (keys hashed to one bucket overwrite each other)
    assert not np.array_equal(slot, 4 * hb)
    # a hash that forgets the + 1 (p = n would address bucket B, past the table)
    n = R.size
    p = _pred_f32(R, np.unique(R), m).astype(np.int64)
    assert np.any(p * B // n != p * B // (n + 1))
    # a lookup that reads only the hashed bucket's first slot misses keys
    dkey = np.unique(R)
    direct = h.keys[np.minimum(4 * hb, h.keys.size - 1)]
    assert not np.array_equal(direct, dkey)
