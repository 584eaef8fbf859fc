"""join_count_noalloc, the entry point for callers that cannot allocate.

Some callers of this library cannot allocate device memory while they run:
a serving loop with a hard latency budget cannot afford cudaMalloc (which
can synchronise the device), and a host that hands all device memory to its
own allocator has none left to give.  join_count_noalloc serves them with
scratch memory compiled into the library.  This test checks, through the C
ABI, that two calls in a row give exactly what join_count gives and what
the CPU oracle gives (counts, offsets and total are integers, so the
comparisons are exact), that the
second call is not disturbed by what the first left in the shared scratch,
and that batches beyond the scratch's limit are refused.

The file name sorts last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _count(fn, idx, S):
    m = S.numel()
    counts = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    offsets = torch.full((m + 1,), -1, dtype=torch.int64, device="cuda")
    total = fn(idx, S, counts=counts, offsets=offsets)
    torch.cuda.synchronize()
    return total, counts.cpu().numpy(), offsets.cpu().numpy()


@pytest.mark.parametrize("dups", [False, True])
def test_noalloc_matches_join_count_twice(dups):
    import paper_2111_08824_gb300 as lj
    rng = np.random.default_rng(31 + dups)
    R = np.unique(rng.integers(0, 2**40, 300_000, dtype=np.uint64))
    if dups:
        R = np.sort(np.concatenate([R, R[::4], R[::9]]))
    idx = lj.rmi_build(_dev(R), 8192, "fp32")
    # two different batches in a row: the second must not see the first's scratch
    S1 = np.concatenate([R[rng.integers(0, R.size, 400_000)],
                         rng.integers(0, 2**40, 300_000, dtype=np.uint64)])
    S2 = np.concatenate([rng.integers(0, 2**40, 5_000, dtype=np.uint64), R[:50_000]])
    for S in (S1, S2):
        Sd = _dev(S)
        want = _count(lj.join_count, idx, Sd)
        got = _count(lj.join_count_noalloc, idx, Sd)
        assert got[0] == want[0]
        assert np.array_equal(got[1], want[1])
        assert np.array_equal(got[2], want[2])
        # and the oracle's (CPU sort-merge join): counts hi - lo, offsets
        # their exclusive prefix sums, total |J|
        lo, hi, total = oracle.join_ranges(R, S)
        cnt = (hi - lo).astype(np.int64)
        assert got[0] == total
        assert np.array_equal(got[1].astype(np.int64), cnt)
        assert got[2][0] == 0 and np.array_equal(np.diff(got[2]), cnt)


def test_noalloc_rejects_batches_beyond_its_limit():
    import paper_2111_08824_gb300 as lj
    R = np.arange(1000, dtype=np.uint64)
    idx = lj.rmi_build(_dev(R), 16, "fp32")
    S = torch.zeros((1 << 25) + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.join_count_noalloc(idx, S)
    assert e.value.code == -1 and "limit" in str(e.value)
    # a batch at the limit is accepted
    assert lj.join_count_noalloc(idx, S[: 1 << 25]) == 1 << 25
