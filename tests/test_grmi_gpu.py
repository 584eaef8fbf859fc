"""GPU parity of the gapped RMI (Section 3.A) against the CPU oracle.

  * the gapped key and payload arrays built on the GPU equal the oracle's
    model-based insertion slot for slot (fp32 and fp64 models, unique and
    duplicated keys, 0 to 8 gaps per key, sizes spanning several build tiles
    of 2048 keys with a ragged tail), and so do the displacement statistics;
  * joins through the exponential search equal the oracle's join pair for
    pair: single join (unique R, one call), two-pass join with duplicates,
    host-resident S, misaligned S, misses below and above R, keys 0 and
    2^64-1, empty and one-key relations;
  * grmi_drop returns to the bounded search with the same results; the paths
    that do not take gapped indexes reject them.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOP = np.uint64(2**64 - 1)


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


def dev(a: np.ndarray):
    assert a.dtype == np.uint64, a.dtype
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _relation(kind, n, rng):
    if kind == "uniform":
        return np.unique(rng.integers(0, 2**63, n, dtype=np.uint64))
    if kind == "lognormal":
        return np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    if kind == "dups":
        return np.sort(rng.integers(0, max(2, n // 6), n, dtype=np.uint64))
    c = rng.integers(0, 2**62, 5, dtype=np.uint64)       # float32-collapsing clusters
    return np.sort(c[rng.integers(0, 5, n)] + rng.integers(0, 3000, n).astype(np.uint64))


def _probes(R, m, rng):
    hits = R[rng.integers(0, R.size, m // 2)] if R.size else np.zeros(0, np.uint64)
    top = int(R[-1]) if R.size else 2**40
    miss = rng.integers(0, top + 2 if top < 2**63 else 2**63, m - hits.size, dtype=np.uint64)
    S = np.concatenate([hits, miss, np.array([0, 1, TOP], np.uint64)])
    rng.shuffle(S)
    return S


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "clusters"])
@pytest.mark.parametrize("gaps", [0, 1, 4, 8])
def test_gapped_arrays_match_oracle(kind, prec, gaps):
    lj = _lj()
    rng = np.random.default_rng(100 + gaps)
    R = _relation(kind, 3 * 2048 + 777, rng)
    for L in (1, 37, 2048):
        idx = lj.rmi_build(dev(R), L, prec)
        st = lj.grmi_build(idx, gaps)
        keys, pos = lj.grmi_export(idx)
        m = oracle.rmi_fit(R, L, fp64=prec == "fp64")
        want = oracle.grmi_build(R, m, gaps)
        assert st["slots"] == want.keys.size and st["gaps"] == gaps
        assert np.array_equal(keys, want.keys), (kind, L)
        assert np.array_equal(pos, want.pos), (kind, L)
        pslot = np.array([oracle.grmi_pslot(R, m, gaps, int(x)) for x in R], dtype=np.int64)
        disp = want.slot_of_key.astype(np.int64) - pslot
        assert st["max_disp"] == disp.max()
        assert st["mean_disp"] == pytest.approx(disp.mean(), rel=1e-12, abs=1e-12)


def _join(lj, idx, S_dev, m):
    unique = bool(idx.stats()["unique"])
    if unique:
        pairs = torch.full((max(m, 1), 2), -1, dtype=torch.int32, device="cuda")
        total = lj.join_emit(idx, S_dev, pairs)
    else:
        offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        total = lj.join_count(idx, S_dev, None, offsets)
        pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
        assert lj.join_emit(idx, S_dev, pairs, offsets=offsets) == total
    return pairs[:total].cpu().numpy().view(np.uint32), total


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "clusters"])
def test_gapped_join_matches_oracle(kind, prec):
    lj = _lj()
    rng = np.random.default_rng(7)
    R = _relation(kind, 20000, rng)
    S = _probes(R, 3 * 4096 + 1234, rng)
    want = oracle.join_pairs(R, S)
    for L in (1, 64, 4096):
        for gaps in (0, 4):
            idx = lj.rmi_build(dev(R), L, prec)
            lj.grmi_build(idx, gaps)
            for misalign in (False, True):
                Sd = dev(np.concatenate([np.zeros(1, np.uint64), S]))[1:] if misalign else dev(S)
                got, total = _join(lj, idx, Sd, S.size)
                assert total == want.shape[0], (kind, L, gaps)
                assert np.array_equal(got, want), (kind, L, gaps, misalign)
            # counts and offsets of the two-pass path as well
            counts = torch.empty(S.size, dtype=torch.int32, device="cuda")
            offsets = torch.empty(S.size + 1, dtype=torch.int64, device="cuda")
            lj.join_count(idx, dev(S), counts, offsets)
            lo, hi, _ = oracle.join_ranges(R, S)
            assert np.array_equal(counts.cpu().numpy().astype(np.int64), (hi - lo).astype(np.int64))


def test_gapped_degenerate_relations():
    lj = _lj()
    S = np.array([0, 1, 5, 42, 43, 2**63, TOP, 5, 42], np.uint64)
    for R in (np.zeros(0, np.uint64), np.array([5], np.uint64), np.full(50, 42, np.uint64),
              np.array([0, TOP], np.uint64), np.array([0, 0, 1, TOP, TOP], np.uint64)):
        for prec in ("fp32", "fp64"):
            for L in (1, 3):
                Rd = dev(R) if R.size else torch.zeros(0, dtype=torch.int64, device="cuda")
                idx = lj.rmi_build(Rd, L, prec)
                lj.grmi_build(idx, 4)
                keys, pos = lj.grmi_export(idx)
                want = oracle.grmi_build(R, oracle.rmi_fit(R, L, fp64=prec == "fp64"), 4)
                assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
                got, total = _join(lj, idx, dev(S), S.size)
                assert np.array_equal(got, oracle.join_pairs(R, S))
                got, total = _join(lj, idx, torch.zeros(0, dtype=torch.int64, device="cuda"), 0)
                assert total == 0


def test_gapped_host_join_and_drop():
    lj = _lj()
    rng = np.random.default_rng(8)
    R = _relation("lognormal", 50000, rng)
    S = _probes(R, 3 * 65536 + 4321, rng)
    want = oracle.join_pairs(R, S)
    idx = lj.rmi_build(dev(R), 512, "fp32")
    lj.grmi_build(idx, 4)
    out = np.zeros((S.size, 2), dtype=np.uint32)
    old = lj.lj_get_option("host_chunk")
    lj.lj_set_option("host_chunk", 65536)        # several chunks, ragged tail
    try:
        total = lj.join_host(idx, S, out)
    finally:
        lj.lj_set_option("host_chunk", old)
    assert total == want.shape[0] and np.array_equal(out[:total], want)
    # rebuild with other gaps, then drop: the bounded search gives the same pairs
    lj.grmi_build(idx, 1)
    assert lj.grmi_stats(idx)["gaps"] == 1
    got, _ = _join(lj, idx, dev(S), S.size)
    assert np.array_equal(got, want)
    lj.grmi_drop(idx)
    with pytest.raises(lj.LJoinError) as e:
        lj.grmi_stats(idx)
    assert e.value.code == -9
    got, _ = _join(lj, idx, dev(S), S.size)
    assert np.array_equal(got, want)


def test_gapped_rejections():
    lj = _lj()
    R = np.arange(1, 5001, dtype=np.uint64) * np.uint64(3)
    S = dev(R[::2])
    idx = lj.rmi_build(dev(R), 16, "fp32")
    with pytest.raises(lj.LJoinError) as e:
        lj.grmi_build(idx, 17)
    assert e.value.code == -1
    lj.grmi_build(idx, 4)
    pairs = torch.empty((S.numel(), 2), dtype=torch.int32, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.join_batch([idx], [S], [pairs])
    assert e.value.code == -1
    with pytest.raises(lj.LJoinError) as e:
        lj.join_count_noalloc(idx, S)
    assert e.value.code == -1
    # the index itself still joins
    assert lj.join_emit(idx, S, pairs) == S.numel()
