"""GPU parity: the CUDA path against the CPU oracle, element by element.

Every test runs on the four execution paths of the probe (fused
single-pass kernel, pipeline in S order, in bucketed probe order, in learned
sort-merge order).
Join results are compared exactly (the pairs are a set, and both sides write
them in the same canonical order: s_idx ascending, r_idx ascending).  Index
builds are compared through tests/_validate.py.  Sizes span several probe
tiles (2048 probes each) plus a ragged tail, and cover the degenerate cases
of the method: empty inputs, one key, one leaf, more leaves than keys, all
keys equal, keys 0 and 2^64-1, float32-collapsing clusters, misses below
the minimum and above the maximum, misaligned S.
"""
import zlib

import numpy as np
import pytest

import oracle
from tests import _validate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOP = np.uint64(2**64 - 1)


PATHS = {   # path: (single_pass_max, probe_buckets, fused_max, fused_groups, key_levels)
    "single_pass": (1 << 40, 0, 0, 1, 0),
    "pipeline": (0, 0, 0, 1, 1),           # key-level descent (levels_search_kernel)
    "pipeline_halving": (0, 0, 0, 1, 0),   # halving (probe_search_kernel)
    "bucketed": (0, 1, 0, 1, 0),
    "sortmerge": (0, 2, 0, 1, 0),
    "fused": (0, 0, 1 << 22, 1, 1),        # fused kernel with the key-level descent
    "fused_g4": (0, 0, 1 << 22, 1, 0),     # ... halving over 4-key groups
    "fused_halving": (0, 0, 1 << 22, 0, 0),
}
_OPTS = ("single_pass_max", "probe_buckets", "fused_max", "fused_groups", "key_levels")


@pytest.fixture(params=sorted(PATHS), autouse=True)
def probe_path(request):
    """Run every test on each execution path of the probe: the single-pass
    kernel; the pipeline in S order (key-level descent or halving), in
    bucketed probe order and in learned sort-merge order; the fused
    cooperative kernel of small unique batches (key-level descent, halving
    over 4-key groups, plain halving).  The options apply to the indexes the
    test builds."""
    import paper_2111_08824_gb300 as lj
    old = [lj.lj_get_option(k) for k in _OPTS]
    for k, v in zip(_OPTS, PATHS[request.param]):
        lj.lj_set_option(k, v)
    yield request.param
    for k, v in zip(_OPTS, old):
        lj.lj_set_option(k, v)


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


def dev(a: np.ndarray):
    assert a.dtype == np.uint64, a.dtype
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int64)).cuda()


def gpu_join(R, S, L, prec="fp32", path="auto", misalign=False):
    lj = _lj()
    Rd = dev(R)
    if misalign:
        Sfull = dev(np.concatenate([np.zeros(1, np.uint64), S]))
        Sd = Sfull[1:]
    else:
        Sd = dev(S)
    idx = lj.rmi_build(Rd, L, prec)
    unique = bool(idx.stats()["unique"])
    if path == "auto":
        path = "fused" if unique else "two_pass"
    m = S.size
    if path == "fused":
        pairs = torch.full((max(m, 1), 2), -1, dtype=torch.int32, device="cuda")
        total = lj.join_emit(idx, Sd, pairs)
        counts = offsets = None
    else:
        offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        counts = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        total = lj.join_count(idx, Sd, counts, offsets)
        pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
        written = lj.join_emit(idx, Sd, pairs, offsets=offsets)
        assert written == total
        counts = counts[:m].cpu().numpy().view(np.uint32)
        offsets = offsets.cpu().numpy().view(np.uint64)
    torch.cuda.synchronize()
    out = pairs[:total].cpu().numpy().view(np.uint32)
    return out, total, counts, offsets, idx


def check_against_oracle(R, S, L, prec="fp32", path="auto", misalign=False):
    got, total, counts, offsets, idx = gpu_join(R, S, L, prec, path, misalign)
    lo, hi, want_total = oracle.join_ranges(R, S)
    assert total == want_total
    want = oracle.join_pairs(R, S)
    assert np.array_equal(got, want)
    if counts is not None:
        assert np.array_equal(counts.astype(np.uint64), hi - lo)
        assert offsets[0] == 0 and np.array_equal(np.diff(offsets.astype(np.int64)),
                                                  (hi - lo).astype(np.int64))
    return idx


def _probe_mix(rng, R, m):
    """Hits, near misses, misses below/above the range, extremes."""
    parts = []
    if R.size:
        parts.append(R[rng.integers(0, R.size, m // 2)])
        near = R[rng.integers(0, R.size, m // 4)]
        parts.append(near + np.uint64(1))
    parts.append(rng.integers(0, 2**64 - 1, m - sum(p.size for p in parts), dtype=np.uint64,
                              endpoint=True))
    S = np.concatenate(parts + [np.array([0, 1, TOP, TOP - np.uint64(1)], np.uint64)])
    rng.shuffle(S)
    return S


def _relation(kind, rng, n):
    if kind == "uniform":
        return np.unique(rng.integers(0, 2**63, n, dtype=np.uint64))
    if kind == "lognormal":
        return np.unique(np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64))
    if kind == "clusters":   # tight clusters far apart: collapse under float32
        c = rng.integers(0, 2**62, 16, dtype=np.uint64)
        return np.unique(c[rng.integers(0, 16, n)] + rng.integers(0, 5000, n).astype(np.uint64))
    if kind == "extremes":
        keys = rng.integers(0, 2**64 - 1, n, dtype=np.uint64, endpoint=True)
        return np.unique(np.concatenate([keys, np.array([0, TOP], np.uint64)]))
    raise ValueError(kind)


# ------------------------------------------------------------------ joins --

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "clusters", "extremes"])
@pytest.mark.parametrize("path", ["fused", "two_pass"])
def test_join_unique_parity(kind, path, prec):
    rng = np.random.default_rng(zlib.crc32(f"{kind}{path}{prec}".encode()))
    R = _relation(kind, rng, 60000)
    S = _probe_mix(rng, R, 2048 * 5 + 37)
    for L in (1, 512, 100000):
        check_against_oracle(R, S, L, prec, path)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_join_duplicates_parity(prec):
    rng = np.random.default_rng(21)
    R = np.sort(np.concatenate([rng.integers(0, 5000, 40000, dtype=np.uint64),
                                np.full(300, 777, np.uint64),
                                np.array([0, 0, TOP, TOP], np.uint64)]))
    S = np.concatenate([R[rng.integers(0, R.size, 6000)],
                        rng.integers(0, 6000, 4000, dtype=np.uint64),
                        np.array([TOP, 0, 777], np.uint64)])
    for L in (1, 64, 5000, 100000):
        check_against_oracle(R, S, L, prec, "two_pass")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("dups", [False, True])
def test_locate_and_expand_parity(dups, prec):
    """join_locate's first positions and counts, and join_expand's pairs,
    against the oracle's ranges and pairs (unique and duplicated R)."""
    rng = np.random.default_rng(31 + dups)
    R = (np.sort(rng.integers(0, 4000, 120000, dtype=np.uint64)) if dups
         else _relation("lognormal", rng, 120000))
    S = _probe_mix(rng, R, 3 * 4096 + 555)
    lj = _lj()
    idx = lj.rmi_build(dev(R), 2000, prec)
    m = S.size
    first = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    total = lj.join_locate(idx, dev(S), first, counts, offsets)
    lo, hi, want_total = oracle.join_ranges(R, S)
    assert total == want_total
    c = counts.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(c, hi - lo)
    f = first.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(f[c > 0], lo[c > 0])
    pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
    assert lj.join_expand(first, offsets, pairs) == total
    assert np.array_equal(pairs[:total].cpu().numpy().view(np.uint32), oracle.join_pairs(R, S))
    # an output that is not 32-byte aligned takes the pair-at-a-time path
    shifted = torch.full((total + 1, 2), -1, dtype=torch.int32, device="cuda")[1:]
    assert lj.join_expand(first, offsets, shifted) == total
    assert np.array_equal(shifted.cpu().numpy().view(np.uint32), oracle.join_pairs(R, S))
    # too little room: reported, the first `capacity` pairs written
    if total > 1:
        small = torch.full((total // 2, 2), -1, dtype=torch.int32, device="cuda")
        with pytest.raises(lj.LJoinError) as e:
            lj.join_expand(first, offsets, small)
        assert e.value.code == -5
        assert np.array_equal(small.cpu().numpy().view(np.uint32),
                              oracle.join_pairs(R, S)[: total // 2])
    # empty S
    e0 = torch.zeros(0, dtype=torch.int64, device="cuda")
    off0 = torch.empty(1, dtype=torch.int64, device="cuda")
    assert lj.join_locate(idx, e0, first[:0], None, off0) == 0
    assert lj.join_expand(first[:0], off0, pairs) == 0


def test_join_many_chunks_ragged():
    """More probes than one bucketing chunk (2^22), with a ragged tail."""
    rng = np.random.default_rng(41)
    R = np.sort(rng.integers(0, 3 * 10**6, 2 * 10**6, dtype=np.uint64))    # duplicates
    S = rng.integers(0, 3 * 10**6 + 10, (1 << 22) + 12345, dtype=np.uint64)
    # a third of the probes on a few hot keys: buckets far above 1024 probes
    hot = rng.random(S.size) < 0.33
    S[hot] = R[rng.integers(0, 5, hot.sum()) * 1000]
    check_against_oracle(R, S, 20000, "fp32", "two_pass")
    Ru = np.unique(R)
    check_against_oracle(Ru, S, 20000, "fp32", "fused")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_join_unique_sizes_across_the_grid(prec):
    """Batch sizes from one probe to 2^22 - 2 against one unique R: one
    block, several groups of 32 blocks, a full grid of resident blocks with
    several rounds per thread, odd sizes (a block whose last probe has no
    partner) -- on every probe path, the fused kernel included."""
    rng = np.random.default_rng(43)
    R = np.unique(rng.integers(0, 2**63, 1 << 20, dtype=np.uint64))
    check_against_oracle(R, R[7:8], 4096, prec, "fused")             # one probe
    for m in (3, 513, 65537, 1048583, (1 << 22) - 6):                 # + 4 extreme keys
        S = _probe_mix(rng, R, m)
        check_against_oracle(R, S, 4096, prec, "fused")


def test_join_misaligned_S_uses_scalar_loads():
    rng = np.random.default_rng(22)
    R = _relation("uniform", rng, 30000)
    S = _probe_mix(rng, R, 2048 * 3 + 5)
    for path in ("fused", "two_pass"):
        check_against_oracle(R, S, 2048, "fp32", path, misalign=True)


@pytest.mark.parametrize("case", ["empty_R", "empty_S", "both_empty", "one_key", "all_equal",
                                  "leaves_gg_n", "self_join", "below_above"])
def test_join_degenerate(case):
    rng = np.random.default_rng(23)
    if case == "empty_R":
        R, S, L = np.zeros(0, np.uint64), rng.integers(0, 100, 5000, dtype=np.uint64), 16
    elif case == "empty_S":
        R, S, L = np.arange(100, dtype=np.uint64), np.zeros(0, np.uint64), 16
    elif case == "both_empty":
        R, S, L = np.zeros(0, np.uint64), np.zeros(0, np.uint64), 1
    elif case == "one_key":
        R, S, L = np.array([42], np.uint64), np.array([41, 42, 43, 42], np.uint64), 4
    elif case == "all_equal":
        R, S, L = np.full(3000, 9, np.uint64), np.array([9, 8, 9, 10] * 500, np.uint64), 64
    elif case == "leaves_gg_n":
        R = np.unique(rng.integers(0, 2**40, 500, dtype=np.uint64))
        S, L = _probe_mix(rng, R, 3000), 1 << 20
    elif case == "self_join":
        R = _relation("lognormal", rng, 50000)
        S, L = R.copy(), 3000
    else:
        R = np.arange(1000, 2000, dtype=np.uint64) * np.uint64(7)
        S, L = np.array([0, 6999, 14000, TOP, 7000, 13993], np.uint64), 10
    for path in ("auto", "two_pass"):
        for prec in ("fp32", "fp64"):
            check_against_oracle(R, S, L, prec, path)


def test_error_codes():
    lj = _lj()
    with pytest.raises(lj.LJoinError) as e:
        lj.rmi_build(dev(np.array([3, 2, 1], np.uint64)), 4)
    assert e.value.code == -4                     # LJ_E_UNSORTED
    with pytest.raises(lj.LJoinError) as e:
        lj.rmi_build(dev(np.array([1, 2], np.uint64)), 0)
    assert e.value.code == -1                     # LJ_E_INVAL
    R = np.array([1, 1, 2], np.uint64)
    idx = lj.rmi_build(dev(R), 2)
    pairs = torch.empty((8, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.join_emit(idx, dev(np.array([1], np.uint64)), pairs)
    assert e.value.code == -8                     # LJ_E_NOTUNIQUE
    # capacity overflow is reported, the first `capacity` pairs are written
    R = np.arange(100, dtype=np.uint64)
    idx = lj.rmi_build(dev(R), 8)
    small = torch.full((10, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.join_emit(idx, dev(R), small)
    assert e.value.code == -5                     # LJ_E_CAPACITY
    got = small.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, np.stack([np.arange(10), np.arange(10)], 1).astype(np.uint32))
    # the error word is cleared: the next call succeeds
    full = torch.empty((100, 2), dtype=torch.int32, device="cuda")
    assert lj.join_emit(idx, dev(R), full) == 100


def test_join_host_chunked_duplicates_and_capacity():
    """Host join over several chunks (copy-outs overlapping the next chunk),
    with duplicate keys, pinned and pageable S, and too little room."""
    import torch as _t
    lj = _lj()
    rng = np.random.default_rng(25)
    R = np.sort(rng.integers(0, 20000, 150000, dtype=np.uint64))
    S = rng.integers(0, 21000, 5 * 65536 + 321, dtype=np.uint64)
    want = oracle.join_pairs(R, S)
    idx = lj.rmi_build(dev(R), 2048, "fp32")
    old = lj.lj_get_option("host_chunk")
    lj.lj_set_option("host_chunk", 65536)
    try:
        pinned = _t.from_numpy(S.view(np.int64)).pin_memory().numpy().view(np.uint64)
        for S_in in (S, pinned):
            pairs = np.zeros((want.shape[0], 2), np.uint32)
            assert lj.join_host(idx, S_in, pairs) == want.shape[0]
            assert np.array_equal(pairs, want)
        small = np.zeros((want.shape[0] // 3, 2), np.uint32)
        with pytest.raises(lj.LJoinError) as e:
            lj.join_host(idx, S, small)
        assert e.value.code == -5
        assert np.array_equal(small, want[: small.shape[0]])
    finally:
        lj.lj_set_option("host_chunk", old)


def test_join_host_matches_device_path():
    lj = _lj()
    rng = np.random.default_rng(24)
    R = _relation("lognormal", rng, 80000)
    S = _probe_mix(rng, R, 50000)
    idx = lj.rmi_build(dev(R), 4096, "fp32")
    want = oracle.join_pairs(R, S)
    pairs = np.zeros((S.size, 2), np.uint32)
    total = lj.join_host(idx, S, pairs)
    assert total == want.shape[0] and np.array_equal(pairs[:total], want)
    Rd = np.sort(np.concatenate([R, R[::3]]))
    idx2 = lj.rmi_build(dev(Rd), 4096, "fp32")
    want2 = oracle.join_pairs(Rd, S)
    pairs2 = np.zeros((want2.shape[0], 2), np.uint32)
    total2 = lj.join_host(idx2, S, pairs2)
    assert total2 == want2.shape[0] and np.array_equal(pairs2, want2)
