"""Validity checks of a learned index built on the GPU (test-side helpers).

A GPU build and the oracle's build may differ in the last bit of a
least-squares parameter (their sums run in different orders), and then
both are valid indexes.  These helpers therefore compare what is unique
and check that the rest is valid:
  * parameters against the oracle's, within a relative tolerance;
  * leaf ranges and error bounds exactly, wherever the deployed parameters
    are bit-identical to the oracle's;
  * every key's leaf and every leaf's error bounds recomputed from the
    GPU's own deployed parameters with exact IEEE emulation
    (tests/_fpemu.py), in the model's precision: bounds must be exact
    (tight and covering).
"""
from __future__ import annotations

import numpy as np

from tests import _fpemu as fe


def compare_index(R: np.ndarray, gpu: dict, ora, fp64: bool) -> dict:
    L = ora.L
    n = R.size
    lo_g = gpu["leaf_lo"].astype(np.int64)
    lo_o = ora.leaf_lo.astype(np.int64)
    assert lo_g[0] == 0 and lo_g[L] == n and np.all(np.diff(lo_g) >= 0)
    # least-squares root within tolerance (a0 * key spans [0, L))
    span = float(R[-1]) if n else 1.0
    assert abs(gpu["root"][0] - ora.root_dep[0]) * span <= 1e-5 * max(L, 1) + 1e-30
    assert abs(gpu["root"][1] - ora.root_dep[1]) <= 1e-5 * max(L, 1) + abs(ora.root_dep[1]) * 1e-6
    report = {"root_identical": bool(np.array_equal(gpu["root"], ora.root_dep))}
    if report["root_identical"]:
        assert np.array_equal(lo_g, lo_o), "same root parameters must give the same leaves"
        same = np.all(gpu["leaf_ab"] == ora.leaf_dep, axis=1)
        report["leaves_identical"] = int(same.sum())
        report["leaves"] = L
        # where parameters agree bit for bit the error bounds must agree exactly
        assert np.array_equal(gpu["err"][same], ora.err[same])
        # where they do not, both parameters are still within rounding
        # distance of the oracle's least-squares fit: the slope relative to
        # itself (times the leaf's key span, i.e. in positions), the
        # intercept in positions
        sizes = np.diff(lo_o)
        rel = 1e-9 if fp64 else 1e-6
        for l in np.flatnonzero(~same):
            k = max(int(sizes[l]), 1)
            a_g, b_g = gpu["leaf_ab"][l]
            a_o, b_o = ora.leaf_fit[l]
            span = float(R[lo_o[l + 1] - 1] - R[lo_o[l]]) if sizes[l] else 0.0
            assert abs(a_g - a_o) <= rel * abs(a_o) + 1e-6 * k / max(span, 1.0), ("slope", l)
            assert abs(b_g - b_o) <= 1e-4 * k + 1e-6, ("intercept", l)
    if n:
        (check_f64_tight if fp64 else check_f32_tight)(R, gpu)
    return report


def check_f32_tight(R: np.ndarray, gpu: dict):
    """Recompute leaves and error bounds from the GPU's own fp32 parameters."""
    L = gpu["leaf_ab"].shape[0]
    lo = gpu["leaf_lo"].astype(np.int64)
    n = R.size
    leaf = fe.leaf_of_f32(R, np.float32(gpu["root"][0]), np.float32(gpu["root"][1]), L)
    assert np.array_equal(leaf, np.repeat(np.arange(L), np.diff(lo))), "leaf ranges"
    base = R[lo[leaf]]
    a = gpu["leaf_ab"][leaf, 0].astype(np.float32)
    b = gpu["leaf_ab"][leaf, 1].astype(np.float32)
    err = np.arange(n, dtype=np.int64) - lo[leaf] - fe.leaf_pred_f32(R, base, a, b)
    sizes = np.diff(lo)
    nz = sizes > 0
    emin = np.minimum.reduceat(err, lo[:-1][nz]) if nz.any() else np.zeros(0, np.int64)
    emax = np.maximum.reduceat(err, lo[:-1][nz]) if nz.any() else np.zeros(0, np.int64)
    assert np.array_equal(gpu["err"][nz, 0], emin), "e_lo must be the exact minimum"
    assert np.array_equal(gpu["err"][nz, 1], emax), "e_hi must be the exact maximum"
    assert np.all(gpu["err"][~nz] == 0)


def check_f64_tight(R: np.ndarray, gpu: dict):
    """Recompute leaves and error bounds from the GPU's own fp64 parameters
    (exact fma emulation: tests/_fpemu.floor_fma64)."""
    L = gpu["leaf_ab"].shape[0]
    lo = gpu["leaf_lo"].astype(np.int64)
    n = R.size
    leaf = fe.leaf_of_f64(R, float(gpu["root"][0]), float(gpu["root"][1]), L)
    assert np.array_equal(leaf, np.repeat(np.arange(L), np.diff(lo))), "leaf ranges"
    base = R[lo[leaf]]
    a = gpu["leaf_ab"][leaf, 0].astype(np.float64)
    b = gpu["leaf_ab"][leaf, 1].astype(np.float64)
    err = np.arange(n, dtype=np.int64) - lo[leaf] - fe.leaf_pred_f64(R, base, a, b)
    sizes = np.diff(lo)
    nz = sizes > 0
    emin = np.minimum.reduceat(err, lo[:-1][nz]) if nz.any() else np.zeros(0, np.int64)
    emax = np.maximum.reduceat(err, lo[:-1][nz]) if nz.any() else np.zeros(0, np.int64)
    assert np.array_equal(gpu["err"][nz, 0], emin), "e_lo must be the exact minimum"
    assert np.array_equal(gpu["err"][nz, 1], emax), "e_hi must be the exact maximum"
    assert np.all(gpu["err"][~nz] == 0)
