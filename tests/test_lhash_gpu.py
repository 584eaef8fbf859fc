"""GPU parity of the learned hash index (Section 3.C) against the CPU oracle.

  * the table built on the GPU (keys, payloads, first positions of the
    distinct keys) equals the oracle's slot for slot, for four key
    distributions (incl. duplicates and sequential keys with holes), fp32 and
    fp64 models, 1 to 8 slots per distinct key, sizes spanning several build
    tiles of 2048 keys with a ragged tail;
  * joins through the hash lookups equal the oracle's pairs: unique R in one
    call, duplicates through join_count + join_emit and join_locate +
    join_expand, host-resident S, misaligned S, degenerate relations;
  * rebuilding as a gapped RMI or dropping the table keeps the results.
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
    holes = np.flatnonzero(rng.random(2 * n) > 0.1).astype(np.uint64)
    return np.sort(np.repeat(holes[: n // 4], rng.integers(1, 8, n // 4)))[:n]


def _probes(R, m, rng):
    hits = R[rng.integers(0, R.size, m // 2)] if R.size else np.zeros(0, np.uint64)
    top = int(R[-1]) if R.size else 2**40
    miss = rng.integers(0, top + 2 if top < 2**63 else 2**63, m - hits.size, dtype=np.uint64)
    S = np.concatenate([hits, miss, np.array([0, 1, TOP], np.uint64)])
    rng.shuffle(S)
    return S


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "seq_holes"])
@pytest.mark.parametrize("spk", [1, 4, 8])
def test_table_matches_oracle(kind, prec, spk):
    lj = _lj()
    rng = np.random.default_rng(200 + spk)
    R = _relation(kind, 3 * 2048 + 901, rng)
    for L in (1, 37, 2048):
        idx = lj.rmi_build(dev(R), L, prec)
        st = lj.lhash_build(idx, spk)
        keys, pos = lj.grmi_export(idx)
        first = lj.lhash_export_first(idx)
        want = oracle.lhash_build(R, oracle.rmi_fit(R, L, fp64=prec == "fp64"), spk)
        assert st["kind"] == 1 and st["gaps"] == spk and st["distinct"] == want.D
        assert st["slots"] == want.keys.size
        assert np.array_equal(keys, want.keys), (kind, L)
        assert np.array_equal(pos, want.pos), (kind, L)
        assert np.array_equal(first, want.first), (kind, L)


def _join(lj, idx, S_dev, m, how):
    if how == "direct":
        pairs = torch.full((max(m, 1), 2), -1, dtype=torch.int32, device="cuda")
        total = lj.join_emit(idx, S_dev, pairs)
    elif how == "two_pass":
        offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        total = lj.join_count(idx, S_dev, None, offsets)
        pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
        assert lj.join_emit(idx, S_dev, pairs, offsets=offsets) == total
    else:
        offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        first = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        total = lj.join_locate(idx, S_dev, first[:m], None, offsets)
        pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
        assert lj.join_expand(first[:m], offsets, pairs) == total
    return pairs[:total].cpu().numpy().view(np.uint32), total


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "seq_holes"])
def test_join_matches_oracle(kind, prec):
    lj = _lj()
    rng = np.random.default_rng(9)
    R = _relation(kind, 20000, rng)
    S = _probes(R, 3 * 4096 + 777, rng)
    want = oracle.join_pairs(R, S)
    unique = np.unique(R).size == R.size
    for L in (1, 64, 4096):
        for spk in (1, 4):
            idx = lj.rmi_build(dev(R), L, prec)
            lj.lhash_build(idx, spk)
            for how in (["direct"] if unique else []) + ["two_pass", "locate"]:
                for misalign in (False, True):
                    Sd = (dev(np.concatenate([np.zeros(1, np.uint64), S]))[1:] if misalign
                          else dev(S))
                    got, total = _join(lj, idx, Sd, S.size, how)
                    assert total == want.shape[0], (kind, L, spk, how)
                    assert np.array_equal(got, want), (kind, L, spk, how, misalign)


def test_degenerate_relations_and_host_join():
    lj = _lj()
    S = np.array([0, 1, 5, 42, 43, 2**63, TOP, 5, 42], np.uint64)
    for R in (np.zeros(0, np.uint64), np.array([5], np.uint64), np.full(50, 42, np.uint64),
              np.array([0, TOP], np.uint64), np.array([0, 0, 1, TOP, TOP], np.uint64)):
        for prec in ("fp32", "fp64"):
            Rd = dev(R) if R.size else torch.zeros(0, dtype=torch.int64, device="cuda")
            idx = lj.rmi_build(Rd, 3, prec)
            lj.lhash_build(idx, 4)
            keys, pos = lj.grmi_export(idx)
            want = oracle.lhash_build(R, oracle.rmi_fit(R, 3, fp64=prec == "fp64"), 4)
            assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
            assert np.array_equal(lj.lhash_export_first(idx), want.first)
            got, _ = _join(lj, idx, dev(S), S.size, "two_pass")
            assert np.array_equal(got, oracle.join_pairs(R, S))
    rng = np.random.default_rng(10)
    R = _relation("seq_holes", 60000, rng)
    S = _probes(R, 3 * 65536 + 99, rng)
    want = oracle.join_pairs(R, S)
    idx = lj.rmi_build(dev(R), 512, "fp32")
    lj.lhash_build(idx, 4)
    old = lj.lj_get_option("host_chunk")
    lj.lj_set_option("host_chunk", 65536)
    try:
        out = np.zeros((want.shape[0], 2), dtype=np.uint32)
        assert lj.join_host(idx, S, out) == want.shape[0]
        assert np.array_equal(out, want)
    finally:
        lj.lj_set_option("host_chunk", old)
    # a gapped RMI in its place, then no table at all: the same pairs
    lj.grmi_build(idx, 4)
    assert lj.grmi_stats(idx)["kind"] == 0
    assert np.array_equal(_join(lj, idx, dev(S), S.size, "locate")[0], want)
    lj.grmi_drop(idx)
    assert np.array_equal(_join(lj, idx, dev(S), S.size, "locate")[0], want)
    with pytest.raises(lj.LJoinError) as e:
        lj.lhash_export_first(idx)
    assert e.value.code == -9
    with pytest.raises(lj.LJoinError) as e:
        lj.lhash_build(idx, 0)
    assert e.value.code == -1


@pytest.mark.parametrize("kind", ["lognormal", "seq_holes"])
def test_index_autotune_keeps_results(kind):
    """The autotuner times the four lookup structures and keeps the fastest;
    whichever it keeps, the join equals the oracle's."""
    lj = _lj()
    rng = np.random.default_rng(12)
    R = _relation(kind, 200000, rng)
    S = _probes(R, 300000, rng)
    want = oracle.join_pairs(R, S)
    idx = lj.rmi_build(dev(R), 2048, "fp32")
    choice, ns = lj.index_autotune(idx, dev(S[: 1 << 17]))
    assert choice in lj._native.LOOKUPS and set(ns) == set(lj._native.LOOKUPS)
    assert all(v > 0 for v in ns.values())
    assert ns[choice] == min(ns.values())
    for how in ("two_pass", "locate"):
        got, total = _join(lj, idx, dev(S), S.size, how)
        assert np.array_equal(got, want), (choice, how)
