"""GPU parity of the RMI build (Section 2.D: root least squares, leaf
assignment, per-leaf least squares, min/max errors) against the CPU oracle.
The build does not depend on the probe path, so these tests run once (the
join tests of test_parity_gpu.py run on every probe path)."""
import zlib

import numpy as np
import pytest

import oracle
from tests import _validate
from tests.test_parity_gpu import _lj, _relation, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# ------------------------------------------------------------ index build --

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["uniform", "lognormal", "clusters", "extremes"])
@pytest.mark.parametrize("L", [1, 7, 4096, 300000])
def test_rmi_build_parity(kind, L, prec):
    rng = np.random.default_rng(zlib.crc32(f"{kind}{L}{prec}".encode()))
    R = _relation(kind, rng, 100000)
    lj = _lj()
    idx = lj.rmi_build(dev(R), L, prec)
    gpu = lj.rmi_export(idx)
    ora = oracle.rmi_fit(R, L, fp64=(prec == "fp64"))
    _validate.compare_index(R, gpu, ora, fp64=(prec == "fp64"))
    st = idx.stats()
    assert st["unique"] == 1 and st["n"] == R.size and st["leaves"] == L


def test_rmi_build_with_duplicates_parity():
    rng = np.random.default_rng(5)
    R = np.sort(rng.integers(0, 3000, 200000, dtype=np.uint64))
    lj = _lj()
    for prec in ("fp32", "fp64"):
        idx = lj.rmi_build(dev(R), 1000, prec)
        assert idx.stats()["unique"] == 0
        _validate.compare_index(R, lj.rmi_export(idx), oracle.rmi_fit(R, 1000, prec == "fp64"),
                                prec == "fp64")


def test_rmi_build_is_deterministic():
    rng = np.random.default_rng(6)
    R = _relation("lognormal", rng, 300000)
    lj = _lj()
    a = lj.rmi_export(lj.rmi_build(dev(R), 5000, "fp32"))
    b = lj.rmi_export(lj.rmi_build(dev(R), 5000, "fp32"))
    for k in a:
        assert np.array_equal(a[k], b[k])
