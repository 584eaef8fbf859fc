"""Full-size parity: the three single-GPU workloads at their real sizes, in
the launch configuration bench.py times (default execution paths).

  uniform_1m        2^20 x 2^20, fp64 model, L = 4096: every pair compared
                    with the oracle.
  lognormal_100m    100M x 400M, L = 2^20, fp32 and fp64 models: properties
                    that hold at any size (|J| = number of generated hits,
                    the matched probes are exactly the generated hits, every
                    pair has equal keys), both precisions give the same pairs,
                    and 2^20 sampled probes compared with the oracle.
  dup_seqh_50m      50M rows x 200M probes (~6.2e9 pairs), L = 2^18: counts
                    equal the generated multiplicities, |J| equals their sum,
                    every pair has equal keys and the pairs of each probe are
                    its contiguous run of R; 2^18 sampled probes compared with
                    the oracle's ranges.
"""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


def test_uniform_1m_full_parity():
    lj = _lj()
    w = datagen.uniform_1m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    pairs = torch.empty((w.S.size, 2), dtype=torch.int32, device="cuda")
    total = lj.join_emit(idx, Sd, pairs)
    assert total == w.meta["expected_pairs"] == w.S.size
    got = pairs[:total].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.join_pairs(w.R, w.S))


def _pairs_equal_keys(Rd, Sd, pairs, total, chunk=1 << 28):
    """Every pair (r, s) has R[r] == S[s]; s non-decreasing across the list."""
    prev_s = -1
    for a in range(0, total, chunk):
        p = pairs[a:min(total, a + chunk)].to(torch.int64) & 0xFFFFFFFF
        r, s = p[:, 0], p[:, 1]
        assert torch.equal(Rd[r], Sd[s])
        assert bool((s[1:] >= s[:-1]).all()) and int(s[0]) >= prev_s
        prev_s = int(s[-1])


def test_lognormal_100m_full_properties_and_samples():
    lj = _lj()
    w = datagen.lognormal_100m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    m = w.S.size
    hits = w.meta["hits"]
    results = {}
    for prec in ("fp32", "fp64"):
        idx = lj.rmi_build(Rd, w.leaves, prec)
        pairs = torch.empty((m, 2), dtype=torch.int32, device="cuda")
        total = lj.join_emit(idx, Sd, pairs)
        assert total == hits
        _pairs_equal_keys(Rd, Sd, pairs, total)
        s_idx = pairs[:total, 1].to(torch.int64) & 0xFFFFFFFF
        assert bool((s_idx[1:] > s_idx[:-1]).all())          # unique R: one pair per probe
        mask = torch.zeros(m, dtype=torch.bool, device="cuda")
        mask[s_idx] = True
        assert torch.equal(mask.cpu(), torch.from_numpy(w.meta["hit_mask"]))
        results[prec] = (pairs[:total].clone(), idx.stats()["mean_window"])
        del pairs
    # results stay exact whatever precision the model runs at
    assert torch.equal(results["fp32"][0], results["fp64"][0])
    # sampled probes against the oracle
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(m, 1 << 20, replace=False))
    lo, hi, _ = oracle.join_ranges(w.R, w.S[sample])
    p = results["fp32"][0].cpu().numpy().view(np.uint32)
    r_of_s = np.full(m, -1, dtype=np.int64)
    r_of_s[p[:, 1]] = p[:, 0]
    got = r_of_s[sample]
    want = np.where(hi > lo, lo.astype(np.int64), -1)
    assert np.array_equal(got, want)


def test_dup_seqh_50m_full_properties_and_samples():
    lj = _lj()
    w = datagen.dup_seqh_50m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    assert idx.stats()["unique"] == 0
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    total = lj.join_count(idx, Sd, counts=counts, offsets=offsets)
    assert total == w.meta["expected_pairs"]
    # counts equal the generated multiplicity of each probe's key
    _, vals_pos = np.unique(w.R, return_index=True)
    mult = np.diff(np.append(vals_pos, w.R.size))
    key_rank = np.searchsorted(w.R[vals_pos], w.S)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), mult[key_rank])
    pairs = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    assert lj.join_emit(idx, Sd, pairs, offsets=offsets) == total
    _pairs_equal_keys(Rd, Sd, pairs, total)
    # sampled probes: their pairs are exactly the oracle's range of R
    rng = np.random.default_rng(6)
    sample = np.sort(rng.choice(m, 1 << 18, replace=False))
    lo, hi, _ = oracle.join_ranges(w.R, w.S[sample])
    off = offsets.cpu().numpy()
    assert np.array_equal(off[sample + 1] - off[sample], (hi - lo).astype(np.int64))
    for k in range(0, sample.size, 4096):
        j = sample[k]
        a, b = int(off[j]), int(off[j + 1])
        blk = pairs[a:b].cpu().numpy().view(np.uint32)
        assert np.array_equal(blk[:, 0], np.arange(lo[k], hi[k], dtype=np.uint32))
        assert np.all(blk[:, 1] == j)


def test_lognormal_100m_gapped_full():
    """Gapped RMI (Section 3.A, 4 gaps per key, the paper's default) at full
    size: the 500M-slot arrays equal the oracle's model-based insertion slot
    for slot, and the join through the exponential search has the workload's
    properties and matches the oracle on 2^20 sampled probes."""
    lj = _lj()
    w = datagen.lognormal_100m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, "fp32")
    st = lj.grmi_build(idx, 4)
    keys, pos = lj.grmi_export(idx)
    want = oracle.grmi_build(w.R, oracle.rmi_fit(w.R, w.leaves, fp64=False), 4)
    assert st["slots"] == want.keys.size
    assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
    del keys, pos
    pairs = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    total = lj.join_emit(idx, Sd, pairs)
    assert total == w.meta["hits"]
    _pairs_equal_keys(Rd, Sd, pairs, total)
    s_idx = pairs[:total, 1].to(torch.int64) & 0xFFFFFFFF
    mask = torch.zeros(m, dtype=torch.bool, device="cuda")
    mask[s_idx] = True
    assert torch.equal(mask.cpu(), torch.from_numpy(w.meta["hit_mask"]))
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(m, 1 << 20, replace=False))
    lo, hi, _ = oracle.grmi_join(w.R, want, w.S[sample])[:3]
    lo2, hi2, _ = oracle.join_ranges(w.R, w.S[sample])
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    p = pairs[:total].cpu().numpy().view(np.uint32)
    r_of_s = np.full(m, -1, dtype=np.int64)
    r_of_s[p[:, 1]] = p[:, 0]
    assert np.array_equal(r_of_s[sample], np.where(hi > lo, lo.astype(np.int64), -1))


def test_dup_seqh_50m_gapped_counts_and_samples():
    lj = _lj()
    w = datagen.dup_seqh_50m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    lj.grmi_build(idx, 4)
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    total = lj.join_count(idx, Sd, counts=counts, offsets=offsets)
    assert total == w.meta["expected_pairs"]
    _, vals_pos = np.unique(w.R, return_index=True)
    mult = np.diff(np.append(vals_pos, w.R.size))
    key_rank = np.searchsorted(w.R[vals_pos], w.S)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), mult[key_rank])
    # emit a sampled slice of probes through the two-pass path and check them
    rng = np.random.default_rng(8)
    sample = np.sort(rng.choice(m, 1 << 16, replace=False))
    Ss = _dev(w.S[sample])
    off_s = torch.empty(sample.size + 1, dtype=torch.int64, device="cuda")
    tot_s = lj.join_count(idx, Ss, offsets=off_s)
    pairs = torch.empty((tot_s, 2), dtype=torch.int32, device="cuda")
    assert lj.join_emit(idx, Ss, pairs, offsets=off_s) == tot_s
    got = pairs.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.join_pairs(w.R, w.S[sample]))


def test_dup_seqh_50m_learned_hash():
    """Learned hash index (Section 3.C, 4 slots per distinct key) on the
    duplicate workload: the table equals the oracle's, counts equal the
    generated multiplicities, sampled probes' pairs equal the oracle's."""
    lj = _lj()
    w = datagen.dup_seqh_50m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    lj.lhash_build(idx, 4)
    keys, pos = lj.grmi_export(idx)
    want = oracle.lhash_build(w.R, oracle.rmi_fit(w.R, w.leaves, fp64=False), 4)
    assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
    assert np.array_equal(lj.lhash_export_first(idx), want.first)
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    total = lj.join_count(idx, Sd, counts=counts)
    assert total == w.meta["expected_pairs"]
    _, vals_pos = np.unique(w.R, return_index=True)
    mult = np.diff(np.append(vals_pos, w.R.size))
    assert np.array_equal(counts.cpu().numpy().astype(np.int64),
                          mult[np.searchsorted(w.R[vals_pos], w.S)])
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(m, 1 << 16, replace=False))
    Ss = _dev(w.S[sample])
    first = torch.empty(sample.size, dtype=torch.int32, device="cuda")
    off = torch.empty(sample.size + 1, dtype=torch.int64, device="cuda")
    tot_s = lj.join_locate(idx, Ss, first, offsets=off)
    pairs = torch.empty((tot_s, 2), dtype=torch.int32, device="cuda")
    assert lj.join_expand(first, off, pairs) == tot_s
    assert np.array_equal(pairs.cpu().numpy().view(np.uint32), oracle.join_pairs(w.R, w.S[sample]))
