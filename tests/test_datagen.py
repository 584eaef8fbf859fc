"""The device generator draws the same raw splitmix64 numbers as the numpy one."""
import numpy as np
import pytest

import datagen
from datagen import device as dg

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("seed,stream,start,count", [(0, 1, 0, 1000), (7, 5, 123456, 5000),
                                                     (2**40 + 3, 9, 0, 777)])
def test_torch_and_numpy_draws_are_bit_identical(seed, stream, start, count):
    a = datagen.rand_u64(seed, stream, start, count)
    b = dg.t_rand_u64(seed, stream, start, count, "cpu").numpy().view(np.uint64)
    assert np.array_equal(a, b)
    assert np.array_equal(datagen.bounded(a, 1000003),
                          dg.t_bounded(torch.from_numpy(a.view(np.int64)), 1000003).numpy())
    assert np.array_equal(datagen.u01(a), dg.t_u01(torch.from_numpy(a.view(np.int64))).numpy())


def test_batched_workload_shapes_cpu():
    w = dg.batched_workload(k=12, seed=1, device="cpu", scale=1 / 256)
    assert len(w) == 12
    for j in w:
        R, S = j["R"], j["S"]
        assert R.dtype == torch.int64 and S.numel() == j["m"]
        Ru = R.numpy().view(np.uint64)
        assert np.all(np.diff(Ru.astype(np.float64)) >= 0) and np.unique(Ru).size == Ru.size
    assert {j["dist"] for j in dg.batched_workload(k=30, seed=2, device="cpu", scale=1 / 1024)} \
        == set(dg.DISTRIBUTIONS)


def test_duplicate_multiplicity_readings():
    """"Zipf(1.2) capped at 64": clipped, P(64) ~ 0.39 and mean ~ 31; truncated
    to 1..64, mean ~ 10 (closed forms of the two distributions)."""
    import math
    import datagen
    s, cap = 1.2, 64
    clip = datagen.zipf_clipped_table(s, cap)
    trunc = datagen.zipf_truncated_table(s, cap)
    k = np.arange(1, cap + 1)
    mean = lambda cdf: float(np.sum(np.diff(np.concatenate([[0.0], cdf])) * k))
    z = datagen.zeta(math.inf, s)
    assert abs((1 - clip[-2]) - (z - np.sum(np.arange(1, cap) ** -s)) / z) < 1e-9
    assert 0.37 < 1 - clip[-2] < 0.41 and 29 < mean(clip) < 33
    assert abs(mean(trunc) - np.sum(k ** (1 - s)) / np.sum(k ** -s)) < 1e-9
    assert 9.5 < mean(trunc) < 10.5 and trunc[-1] == 1.0
    for reading, lo, hi in (("clip", 28, 34), ("truncate", 9, 11)):
        R, vals, mult = datagen.dup_seqh(200_000, 3, reading=reading)
        assert R.size == 200_000 and np.all(np.diff(R.astype(np.int64)) >= 0)
        assert mult.min() >= 1 and mult.max() <= cap and lo < mult.mean() < hi
        assert np.array_equal(np.repeat(vals, mult), R)
