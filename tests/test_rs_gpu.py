"""GPU parity of the RadixSpline hash index (RSHASH-INLJ: the learned hash
of Section 3.C with a RadixSpline, Section 2.D, as the hash) against the
CPU oracle.

  * the spline (keys and positions of its points), the radix table and the
    prefix shift built on the GPU equal the oracle's, for four key
    distributions (incl. duplicates and sequential keys with holes), several
    error bounds and radix widths, sizes spanning several passes of 1024
    distinct keys with a ragged tail;
  * the hash table (keys, payloads, first positions) equals the oracle's
    slot for slot;
  * joins through it equal the oracle's pairs on every path (direct,
    two-pass, located ranges, host-resident S), incl. degenerate relations;
  * the index autotuner may pick it, and results stay exact.
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
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _relation(kind, n, rng):
    if kind == "uniform":
        return np.unique(rng.integers(0, 2**63, n, dtype=np.uint64))
    if kind == "lognormal":
        return np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    if kind == "dups":
        return np.sort(rng.integers(0, max(2, n // 6), n, dtype=np.uint64))
    if kind == "extremes":
        return np.unique(np.concatenate([rng.integers(0, 2**64 - 1, n, dtype=np.uint64,
                                                      endpoint=True), np.array([0, TOP], dtype=np.uint64)]))
    holes = np.flatnonzero(rng.random(2 * n) > 0.1).astype(np.uint64)
    return np.sort(np.repeat(holes[: n // 4], rng.integers(1, 8, n // 4)))[:n]


def _probes(R, m, rng):
    hits = R[rng.integers(0, R.size, m // 2)] if R.size else np.zeros(0, np.uint64)
    top = int(R[-1]) if R.size else 2**40
    miss = rng.integers(0, top + 2 if top < 2**63 else 2**63, m - hits.size, dtype=np.uint64)
    S = np.concatenate([hits, miss, np.array([0, 1, TOP], np.uint64)])
    rng.shuffle(S)
    return S


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "seq_holes", "extremes"])
@pytest.mark.parametrize("eps,rbits", [(0, 4), (16, 18), (64, 10)])
def test_spline_and_radix_table_match_oracle(kind, eps, rbits):
    lj = _lj()
    rng = np.random.default_rng(400 + eps + rbits)
    R = _relation(kind, 5 * 1024 + 333, rng)
    idx = lj.rmi_build(dev(R), 256, "fp32")
    lj.lhash_build_rs(idx, 4, eps, rbits)
    got = lj.rs_export(idx)
    want = oracle.rs_build(R, eps=eps, chunk=1024, rbits=rbits)
    assert got["count"] == want.sx.size
    assert np.array_equal(got["sx"], want.sx) and np.array_equal(got["sy"], want.sy)
    assert got["shift"] == want.shift
    assert np.array_equal(lj.rs_export_table(idx, rbits), want.table)


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "seq_holes"])
@pytest.mark.parametrize("spk", [1, 4, 8])
def test_hash_table_matches_oracle(kind, spk):
    lj = _lj()
    rng = np.random.default_rng(500 + spk)
    R = _relation(kind, 3 * 2048 + 901, rng)
    idx = lj.rmi_build(dev(R), 64, "fp64")
    st = lj.lhash_build_rs(idx, spk, 16, 12)
    h = oracle.rs_lhash_build(R, oracle.rs_build(R, eps=16, chunk=1024, rbits=12), spk)
    keys, pos = lj.grmi_export(idx)
    assert st["kind"] == 2 and st["distinct"] == h.D and st["slots"] == h.keys.size
    assert np.array_equal(keys, h.keys) and np.array_equal(pos, h.pos)
    assert np.array_equal(lj.lhash_export_first(idx), h.first)


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "dups", "seq_holes", "extremes"])
def test_joins_through_rs_hash_match_oracle(kind):
    lj = _lj()
    rng = np.random.default_rng(600)
    R = _relation(kind, 20000, rng)
    S = _probes(R, 30000, rng)
    Rd, Sd = dev(R), dev(S)
    idx = lj.rmi_build(Rd, 512, "fp32")
    lj.lhash_build_rs(idx, 4, 8, 14)
    want = oracle.join_pairs(R, S)
    lo, hi, _ = oracle.join_ranges(R, S)
    # counts and offsets
    counts = torch.empty(S.size, dtype=torch.int32, device="cuda")
    offsets = torch.empty(S.size + 1, dtype=torch.int64, device="cuda")
    total = lj.join_count(idx, Sd, counts=counts, offsets=offsets)
    assert total == want.shape[0]
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), (hi - lo).astype(np.int64))
    pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
    # two-pass emit
    assert lj.join_emit(idx, Sd, pairs, offsets=offsets) == total
    assert np.array_equal(pairs[:total].cpu().numpy().view(np.uint32), want)
    # located ranges + expansion
    first = torch.empty(S.size, dtype=torch.int32, device="cuda")
    pairs.fill_(-1)
    assert lj.join_locate(idx, Sd, first, offsets=offsets) == total
    lj.join_expand(first, offsets, pairs)
    assert np.array_equal(pairs[:total].cpu().numpy().view(np.uint32), want)
    # direct path (unique R)
    if kind in ("uniform", "lognormal", "extremes"):
        pairs.fill_(-1)
        assert lj.join_emit(idx, Sd, pairs) == total
        assert np.array_equal(pairs[:total].cpu().numpy().view(np.uint32), want)
    # S in host memory through join_host
    P = np.zeros((max(total, 1), 2), dtype=np.uint32)
    assert lj.join_host(idx, S, P) == total
    assert np.array_equal(P[:total], want)


@pytest.mark.parametrize("R", [np.zeros(0, np.uint64), np.array([7], np.uint64),
                               np.full(100, 5, np.uint64), np.array([0, TOP], np.uint64)])
def test_degenerate_relations(R):
    lj = _lj()
    S = np.array([0, 5, 7, 8, TOP, 5], dtype=np.uint64)
    Rd = dev(R) if R.size else torch.zeros(0, dtype=torch.int64, device="cuda")
    idx = lj.rmi_build(Rd, 1, "fp32")
    lj.lhash_build_rs(idx, 4, 0, 3)
    want = oracle.join_pairs(R, S)
    off = torch.empty(S.size + 1, dtype=torch.int64, device="cuda")
    t = lj.join_count(idx, dev(S), offsets=off)
    p = torch.empty((max(t, 1), 2), dtype=torch.int32, device="cuda")
    lj.join_emit(idx, dev(S), p, offsets=off)
    assert t == want.shape[0]
    assert np.array_equal(p[:t].cpu().numpy().view(np.uint32), want)


def test_autotuner_can_choose_it_and_stays_exact():
    lj = _lj()
    rng = np.random.default_rng(700)
    R = _relation("seq_holes", 200000, rng)
    S = _probes(R, 1 << 18, rng)
    idx = lj.rmi_build(dev(R), 4096, "fp32")
    choice, ns = lj.index_autotune(idx, dev(S))
    assert set(ns) == {"rmi", "rmi_bucketed", "grmi", "lhash", "rmi_sortmerge", "rshash",
                       "rmi_levels"}
    assert all(v > 0 for v in ns.values())
    off = torch.empty(S.size + 1, dtype=torch.int64, device="cuda")
    t = lj.join_count(idx, dev(S), offsets=off)
    p = torch.empty((max(t, 1), 2), dtype=torch.int32, device="cuda")
    lj.join_emit(idx, dev(S), p, offsets=off)
    assert np.array_equal(p[:t].cpu().numpy().view(np.uint32), oracle.join_pairs(R, S))
