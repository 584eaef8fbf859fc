"""Property-based pins of the oracle (CPU only; hypothesis draws the cases):
for arbitrary small relations, key ranges, leaf counts, gap and slot counts,
  * the sort-merge join equals the nested-loop definition;
  * the learned lookups (RMI bounded search, gapped RMI, learned hash) give
    the same match ranges as the sort-merge join;
  * |J| equals the sum over keys of mult_R(k) * mult_S(k).
"""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

_keys = st.one_of(st.integers(0, 20), st.integers(0, 2**64 - 1), st.integers(10**9, 10**9 + 40))


@settings(max_examples=200, deadline=None)
@given(st.lists(_keys, max_size=40), st.lists(_keys, max_size=40))
def test_sort_merge_equals_nested_loops(R, S):
    R = np.sort(np.array(R, dtype=np.uint64))
    S = np.array(S, dtype=np.uint64)
    got = [(int(r), int(s)) for r, s in oracle.join_pairs(R, S)]
    assert got == oracle.brute_force_join(R, S)
    vals, mr = np.unique(R, return_counts=True)
    ms = {int(v): c for v, c in zip(*np.unique(S, return_counts=True))}
    assert len(got) == sum(int(c) * ms.get(int(v), 0) for v, c in zip(vals, mr))


@settings(max_examples=150, deadline=None)
@given(st.lists(_keys, min_size=0, max_size=60), st.lists(_keys, max_size=40),
       st.integers(1, 70), st.booleans(), st.integers(0, 6), st.integers(1, 8))
def test_learned_lookups_equal_sort_merge(R, S, L, fp64, gaps, spk):
    R = np.sort(np.array(R, dtype=np.uint64))
    S = np.array(S, dtype=np.uint64)
    lo, hi, total = oracle.join_ranges(R, S)
    m = oracle.rmi_fit(R, L, fp64=fp64)
    for j, x in enumerate(S):
        q = oracle.rmi_lookup(R, m, int(x))
        assert (q["lb"], q["ub"]) == (lo[j], hi[j])
    g = oracle.grmi_build(R, m, gaps)
    glo, ghi, gtot, _ = oracle.grmi_join(R, g, S)
    assert gtot == total and np.array_equal(glo, lo) and np.array_equal(ghi, hi)
    h = oracle.lhash_build(R, m, spk)
    hlo, hhi, htot, _ = oracle.lhash_join(R, h, S)
    assert htot == total and np.array_equal(hlo, lo) and np.array_equal(hhi, hi)
