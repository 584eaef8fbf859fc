"""GPU parity of the learned sort-merge join (L-SJ, Section 4) of two
unsorted relations against the CPU oracle (the sort-based join of
oracle.join_pairs_unsorted, itself pinned to nested loops).

The pairs are compared as sets (sorted by (s, r)): L-SJ writes them grouped
by R's sorted chunks.  Cases: unique and duplicate keys on both sides,
uniform / lognormal / clustered / sequential keys, extreme keys 0 and
2^64-1, sizes below and above the 16,384-key sample and the 2048-key
partitions with ragged tails, a heavily skewed relation (one key repeated
beyond a shared-memory partition: the global-memory sort), empty sides, and
a capacity overflow.  Two runs give the same pairs in the same order.
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
    if a.size == 0:
        return torch.zeros(0, dtype=torch.int64, device="cuda")
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _keys(kind, n, rng):
    if kind == "uniform":
        return rng.integers(0, 2**63, n, dtype=np.uint64)
    if kind == "lognormal":
        return np.rint(1e9 * np.exp(2 * rng.standard_normal(n))).astype(np.uint64)
    if kind == "clustered":
        c = rng.integers(0, 2**62, 64, dtype=np.uint64).astype(np.float64)
        return np.maximum(0, np.rint(c[rng.integers(0, 64, n)] + 1e6 * rng.standard_normal(n))
                          ).astype(np.uint64)
    if kind == "seq":
        return rng.permutation(np.arange(n, dtype=np.uint64) * np.uint64(3))
    if kind == "extremes":
        # keys 0 and 2^64-1 repeated (at most 2000 copies each, so that the
        # largest case stays at a few million pairs)
        k = rng.integers(0, 2**64 - 1, n, dtype=np.uint64, endpoint=True)
        c = min(n // 10, 2000)
        k[:c] = TOP
        k[c: 2 * c] = 0
        return rng.permutation(k)
    raise ValueError(kind)


def _check(lj, R, S):
    want = oracle.join_pairs_unsorted(R, S)
    pairs = torch.full((max(want.shape[0], 1), 2), -1, dtype=torch.int32, device="cuda")
    total = lj.lsj_join(dev(R), dev(S), pairs)
    assert total == want.shape[0]
    got = pairs[:total].cpu().numpy().view(np.uint32)
    order = np.lexsort((got[:, 0], got[:, 1]))
    assert np.array_equal(got[order], want)
    return got


@pytest.mark.parametrize("kind", ["uniform", "lognormal", "clustered", "seq", "extremes"])
@pytest.mark.parametrize("n,m", [(1000, 3000), (50_000, 20_000), (300_001, 411_111)])
def test_lsj_matches_oracle(kind, n, m):
    lj = _lj()
    rng = np.random.default_rng(n + m)
    R = _keys(kind, n, rng)
    # S: half draws from R (hits, duplicates on both sides), half fresh keys
    S = np.concatenate([R[rng.integers(0, n, m // 2)], _keys(kind, m - m // 2, rng)])
    S = rng.permutation(S)
    _check(lj, R, S)


def test_lsj_duplicates_and_skew():
    lj = _lj()
    rng = np.random.default_rng(9)
    R = rng.permutation(np.concatenate([np.full(20_000, 77, np.uint64),        # > one partition
                                        rng.integers(0, 10**6, 100_000).astype(np.uint64)]))
    S = rng.permutation(np.concatenate([np.full(50, 77, np.uint64),
                                        rng.integers(0, 10**6, 60_000).astype(np.uint64)]))
    a = _check(lj, R, S)
    b = _check(lj, R, S)
    assert np.array_equal(a, b)                                                # deterministic


@pytest.mark.parametrize("n,m", [(0, 100), (100, 0), (1, 1), (0, 0)])
def test_lsj_degenerate(n, m):
    lj = _lj()
    rng = np.random.default_rng(3)
    R = rng.integers(0, 5, n).astype(np.uint64)
    S = rng.integers(0, 5, m).astype(np.uint64)
    _check(lj, R, S)


def test_lsj_capacity_overflow_is_reported():
    lj = _lj()
    R = np.full(100, 5, np.uint64)
    S = np.full(100, 5, np.uint64)
    pairs = torch.empty((10, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.lsj_join(dev(R), dev(S), pairs)
    assert e.value.code == -5                                                  # LJ_E_CAPACITY
