"""Full-size parity: the three single-GPU workloads at their real sizes, in
the launch configuration bench.py times (default execution paths), every
probe compared with the oracle (the CPU sort-merge join, run on chunks of S
on every host core).

  uniform_1m        2^20 x 2^20, L = 4096: every pair compared with the
                    oracle's pairs, fp64 (the workload's model) and fp32.
  lognormal_100m    100M x 400M, L = 2^20, fp32 and fp64 models: the pairs of
                    every probe equal the oracle's (each hit j gives exactly
                    (lo_j, j), in s order), and join_count's counts and
                    offsets equal the oracle's for all 400M probes.
  dup_seqh_50m      50M rows x 200M probes (~6.2e9 pairs), L = 2^18: the
                    located range (first match, count) and the offset of every
                    probe equal the oracle's; every one of the ~6.2e9 emitted
                    pairs, through join_expand and through the two-pass
                    join_emit, is checked on the device against the oracle's
                    ranges: the pair at output position q is (lo_s + q -
                    off_s, s) for the one probe s with off_s <= q < off_s+1.
  gapped RMI, learned hash and RadixSpline hash at full size: their arrays
                    equal the oracle's, and their joins give the oracle's
                    ranges for every probe.
  lsj_uniform_100m  the learned sort-merge join of two unsorted 100M-key
                    relations: every pair equals the oracle's.
"""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_CHUNK = 1 << 25            # probes per host-side comparison chunk
_PCHUNK = 1 << 27           # pairs per device-side comparison chunk


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


class _Cached:
    """A workload, its device copies and the oracle's ranges (computed once)."""

    def __init__(self, w):
        self.w = w
        self.Rd, self.Sd = _dev(w.R), _dev(w.S)
        self._ranges = None

    def ranges(self):
        if self._ranges is None:
            lo, hi, total = oracle.join_ranges_mt(self.w.R, self.w.S)
            self._ranges = (lo, hi, total)
        return self._ranges


@pytest.fixture(scope="module")
def lognormal():
    c = _Cached(datagen.lognormal_100m(seed=0))
    yield c
    del c.Rd, c.Sd
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def dup():
    c = _Cached(datagen.dup_seqh_50m(seed=0))
    yield c
    del c.Rd, c.Sd
    torch.cuda.empty_cache()


def _unique_pairs_equal_oracle(pairs, total, lo, hi):
    """Direct path on a unique R: the pairs are (lo_j, j) for every hit j,
    in s order (compared chunk by chunk of probes)."""
    done = 0
    for a in range(0, lo.size, _CHUNK):
        b = min(lo.size, a + _CHUNK)
        hit = hi[a:b] > lo[a:b]
        js = np.flatnonzero(hit) + a
        want = np.stack([lo[a:b][hit].astype(np.uint32), js.astype(np.uint32)], axis=1)
        got = pairs[done:done + js.size].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), f"pairs of probes [{a}, {b})"
        done += js.size
    assert total == done


def _pairs_equal_ranges_on_device(pairs, total, lo, off):
    """Every pair at output position q is (lo_s + q - off_s, s) for the one
    probe s with off_s <= q < off_{s+1} (lo, off: the oracle's, on the host)."""
    lo_d = torch.from_numpy(lo.view(np.int64)).cuda()
    off_d = torch.from_numpy(off).cuda()
    for a in range(0, total, _PCHUNK):
        b = min(total, a + _PCHUNK)
        p = pairs[a:b].to(torch.int64) & 0xFFFFFFFF
        r, s = p[:, 0], p[:, 1]
        q = torch.arange(a, b, dtype=torch.int64, device="cuda")
        o = off_d[s]
        assert bool(((o <= q) & (q < off_d[s + 1])).all()), f"s labels of pairs [{a}, {b})"
        assert torch.equal(r, lo_d[s] + (q - o)), f"r of pairs [{a}, {b})"
        del p, r, s, q, o
    del lo_d, off_d


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uniform_1m_full_parity(prec):
    lj = _lj()
    w = datagen.uniform_1m(seed=0)
    Rd, Sd = _dev(w.R), _dev(w.S)
    idx = lj.rmi_build(Rd, w.leaves, prec)
    pairs = torch.empty((w.S.size, 2), dtype=torch.int32, device="cuda")
    want = oracle.join_pairs(w.R, w.S)
    names = ("single_pass_max", "fused_max", "fused_groups")
    old = [lj.lj_get_option(k) for k in names]
    # the bench's default (fused cooperative kernel, 4-key groups), the fused
    # kernel with bisection, the pipeline and the single-pass kernel
    for spm, fmax, groups in ((0, old[1], 1), (0, old[1], 0), (0, 0, 1), (1 << 40, 0, 1)):
        lj.lj_set_option("single_pass_max", spm)
        lj.lj_set_option("fused_max", fmax)
        lj.lj_set_option("fused_groups", groups)
        try:
            pairs.fill_(-1)
            total = lj.join_emit(idx, Sd, pairs)
        finally:
            for k, v in zip(names, old):
                lj.lj_set_option(k, v)
        assert total == w.meta["expected_pairs"] == w.S.size
        assert np.array_equal(pairs[:total].cpu().numpy().view(np.uint32), want)


def test_lognormal_100m_full_parity(lognormal):
    lj = _lj()
    w, Rd, Sd = lognormal.w, lognormal.Rd, lognormal.Sd
    m = w.S.size
    lo, hi, total_o = lognormal.ranges()
    assert total_o == w.meta["hits"] and int((hi - lo).max()) == 1
    # which probes hit is fixed by the generator: the oracle agrees
    assert np.array_equal(hi > lo, w.meta["hit_mask"])
    pairs = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    for prec in ("fp32", "fp64"):   # results stay exact whatever the model precision
        idx = lj.rmi_build(Rd, w.leaves, prec)
        pairs.fill_(-1)
        total = lj.join_emit(idx, Sd, pairs)
        _unique_pairs_equal_oracle(pairs, total, lo, hi)
    # counts and offsets of the count pass (fp32 index), all probes
    del pairs
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    assert lj.join_count(idx, Sd, counts=counts, offsets=offsets) == total_o
    for a in range(0, m, _CHUNK):
        b = min(m, a + _CHUNK)
        c_o = (hi[a:b] - lo[a:b]).astype(np.int64)
        assert np.array_equal(counts[a:b].cpu().numpy().astype(np.int64), c_o)
        off = offsets[a:b + 1].cpu().numpy()
        assert np.array_equal(np.diff(off), c_o)
    assert int(offsets[0]) == 0 and int(offsets[m]) == total_o


def test_dup_seqh_50m_full_parity(dup):
    lj = _lj()
    w, Rd, Sd = dup.w, dup.Rd, dup.Sd
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    assert idx.stats()["unique"] == 0
    lo, hi, total_o = dup.ranges()
    assert total_o == w.meta["expected_pairs"]
    cnt_o = (hi - lo).astype(np.int64)
    off_o = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(cnt_o, out=off_o[1:])
    first = torch.empty(m, dtype=torch.int32, device="cuda")
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    total = lj.join_locate(idx, Sd, first, counts=counts, offsets=offsets)
    assert total == total_o
    hit = cnt_o > 0
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), cnt_o)
    assert np.array_equal(first.cpu().numpy().view(np.uint32)[hit], lo[hit].astype(np.uint32))
    assert np.array_equal(offsets.cpu().numpy(), off_o)
    pairs = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    assert lj.join_expand(first, offsets, pairs) == total          # the bench's path
    _pairs_equal_ranges_on_device(pairs, total, lo, off_o)
    pairs.fill_(-1)
    assert lj.join_emit(idx, Sd, pairs, offsets=offsets) == total  # two-pass emit
    _pairs_equal_ranges_on_device(pairs, total, lo, off_o)


def test_lognormal_100m_gapped_full(lognormal):
    """Gapped RMI (Section 3.A, 4 gaps per key, the paper's default) at full
    size: the 500M-slot arrays equal the oracle's model-based insertion slot
    for slot, and the join through the exponential search gives the oracle's
    result for every probe."""
    lj = _lj()
    w, Rd, Sd = lognormal.w, lognormal.Rd, lognormal.Sd
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, "fp32")
    st = lj.grmi_build(idx, 4)
    keys, pos = lj.grmi_export(idx)
    want = oracle.grmi_build(w.R, oracle.rmi_fit(w.R, w.leaves, fp64=False), 4)
    assert st["slots"] == want.keys.size
    assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
    del keys, pos
    # the oracle's own gapped lookup agrees with its sort-merge on a sample
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(m, 1 << 18, replace=False))
    glo, ghi, _ = oracle.grmi_join(w.R, want, w.S[sample])[:3]
    lo, hi, _ = lognormal.ranges()
    assert np.array_equal(glo, lo[sample]) and np.array_equal(ghi, hi[sample])
    del want
    pairs = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    total = lj.join_emit(idx, Sd, pairs)
    _unique_pairs_equal_oracle(pairs, total, lo, hi)


def test_dup_seqh_50m_gapped_full(dup):
    lj = _lj()
    w, Rd, Sd = dup.w, dup.Rd, dup.Sd
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    lj.grmi_build(idx, 4)
    lo, hi, total_o = dup.ranges()
    first = torch.empty(m, dtype=torch.int32, device="cuda")
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    total = lj.join_locate(idx, Sd, first, counts=counts)
    assert total == total_o
    cnt_o = (hi - lo).astype(np.int64)
    hit = cnt_o > 0
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), cnt_o)
    assert np.array_equal(first.cpu().numpy().view(np.uint32)[hit], lo[hit].astype(np.uint32))


def test_dup_seqh_50m_learned_hash_full(dup):
    """Learned hash index (Section 3.C, 4 slots per distinct key) on the
    duplicate workload: the table equals the oracle's; the located range of
    every probe and every emitted pair equal the oracle's."""
    lj = _lj()
    w, Rd, Sd = dup.w, dup.Rd, dup.Sd
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    lj.lhash_build(idx, 4)
    keys, pos = lj.grmi_export(idx)
    want = oracle.lhash_build(w.R, oracle.rmi_fit(w.R, w.leaves, fp64=False), 4)
    assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
    assert np.array_equal(lj.lhash_export_first(idx), want.first)
    del keys, pos, want
    lo, hi, total_o = dup.ranges()
    cnt_o = (hi - lo).astype(np.int64)
    off_o = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(cnt_o, out=off_o[1:])
    first = torch.empty(m, dtype=torch.int32, device="cuda")
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    total = lj.join_locate(idx, Sd, first, counts=counts, offsets=offsets)
    assert total == total_o
    hit = cnt_o > 0
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), cnt_o)
    assert np.array_equal(first.cpu().numpy().view(np.uint32)[hit], lo[hit].astype(np.uint32))
    assert np.array_equal(offsets.cpu().numpy(), off_o)
    pairs = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    assert lj.join_expand(first, offsets, pairs) == total
    _pairs_equal_ranges_on_device(pairs, total, lo, off_o)


def test_dup_seqh_50m_rs_hash_full(dup):
    """RadixSpline hash index (RSHASH-INLJ, eps 16, 18 radix bits, 4 slots per
    distinct key) on the duplicate workload: spline, radix table and hash
    table equal the oracle's; the located range of every probe and every
    emitted pair equal the oracle's."""
    lj = _lj()
    w, Rd, Sd = dup.w, dup.Rd, dup.Sd
    m = w.S.size
    idx = lj.rmi_build(Rd, w.leaves, w.precision)
    lj.lhash_build_rs(idx, 4, 16, 18)
    rs = oracle.rs_build(w.R, eps=16, chunk=1024, rbits=18)
    got = lj.rs_export(idx)
    assert np.array_equal(got["sx"], rs.sx) and np.array_equal(got["sy"], rs.sy)
    assert np.array_equal(lj.rs_export_table(idx, 18), rs.table)
    want = oracle.rs_lhash_build(w.R, rs, 4)
    keys, pos = lj.grmi_export(idx)
    assert np.array_equal(keys, want.keys) and np.array_equal(pos, want.pos)
    del keys, pos, want
    lo, hi, total_o = dup.ranges()
    cnt_o = (hi - lo).astype(np.int64)
    off_o = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(cnt_o, out=off_o[1:])
    first = torch.empty(m, dtype=torch.int32, device="cuda")
    counts = torch.empty(m, dtype=torch.int32, device="cuda")
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    assert lj.join_locate(idx, Sd, first, counts=counts, offsets=offsets) == total_o
    hit = cnt_o > 0
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), cnt_o)
    assert np.array_equal(first.cpu().numpy().view(np.uint32)[hit], lo[hit].astype(np.uint32))
    pairs = torch.empty((total_o, 2), dtype=torch.int32, device="cuda")
    assert lj.join_expand(first, offsets, pairs) == total_o
    _pairs_equal_ranges_on_device(pairs, total_o, lo, off_o)


def test_lsj_uniform_100m_full_parity():
    """The learned sort-merge join (Section 4) of the bench's two unsorted
    100M-key relations: every pair equals the oracle's (the sort-based join
    of unsorted relations).  S is drawn from the unique R, so each probe j
    has exactly one match: the pairs are compared probe by probe."""
    lj = _lj()
    w = datagen.lsj_uniform_100m(seed=0)
    n, m = w.R.size, w.S.size
    # the oracle's unsorted join (oracle.join_pairs_unsorted), with the
    # sort-merge ranges taken on every host core: R sorted with its
    # positions, each probe's range in it, mapped back to R's positions
    perm = np.argsort(w.R, kind="stable")
    lo, hi, total = oracle.join_ranges_mt(w.R[perm], w.S)
    assert total == m == w.meta["expected_pairs"] and np.all(hi - lo == 1)
    want_r = perm[lo.astype(np.int64)].astype(np.uint32)
    Rd, Sd = _dev(w.R), _dev(w.S)
    pairs = torch.full((m, 2), -1, dtype=torch.int32, device="cuda")
    assert lj.lsj_join(Rd, Sd, pairs) == m
    got = pairs.cpu().numpy().view(np.uint32)
    s_idx = got[:, 1].astype(np.int64)
    assert np.array_equal(np.bincount(s_idx, minlength=m), np.ones(m, np.int64))
    r_of_s = np.empty(m, np.uint32)
    r_of_s[s_idx] = got[:, 0]
    assert np.array_equal(r_of_s, want_r)
    del Rd, Sd, pairs
    torch.cuda.empty_cache()
