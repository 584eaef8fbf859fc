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
