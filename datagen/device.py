"""Device-side (torch) generation of the large multi-relation workloads.

Same counter-based splitmix64 streams as `datagen` (bit-identical raw draws,
checked by tests/test_datagen.py), with the distribution transforms done in
torch on whichever device the caller picks, so the 4096-join batched workload
(about 2e9 inner and 7e9 outer keys) and the served relations can be produced
in seconds on the GPU.  Float transforms (log, exp, cos) may round differently
from numpy's; every test feeds the same arrays to the CUDA path and to the
oracle, so this never matters for parity.  Holds none of the join's arithmetic.

  batched_workload   k independent (R, S): |R| log-uniform in [2^10, 2^22],
                     |S| log-uniform in [2^10, 2^24], each pair's keys from
                     uniform / lognormal(0, 2) / clustered (64 Gaussian
                     clusters, sigma 1e6, centres uniform in [0, 2^62)); R
                     deduplicated and sorted; S half uniform draws from R,
                     half fresh draws of R's distribution (chance hits allowed).
"""
from __future__ import annotations

import math

import numpy as np

from . import (ST_BATCH_DIST, ST_BATCH_SIZES, ST_CLUSTER, ST_R_KEYS, ST_S_COIN, ST_S_HIT,
               ST_S_MISS, _stream_key, rand_u64)

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _i64(c: int) -> int:
    """uint64 constant as the int64 with the same bits."""
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(z, k: int):
    """Logical right shift of an int64 tensor viewed as uint64."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def t_rand_u64(seed: int, stream: int, start: int, count: int, device):
    """splitmix64 outputs start..start+count-1 as int64 tensors (uint64 bits)."""
    import torch
    key = _i64(int(_stream_key(seed, stream)))
    z = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = z * _i64(_GAMMA) + key
    z = z ^ _srl(z, 30)
    z = z * _i64(_M1)
    z = z ^ _srl(z, 27)
    z = z * _i64(_M2)
    z = z ^ _srl(z, 31)
    return z


def t_u01(bits):
    return _srl(bits, 11).double() * (1.0 / 9007199254740992.0)


def t_u01_open(bits):
    return (_srl(bits, 11).double() + 1.0) * (1.0 / 9007199254740992.0)


def t_bounded(bits, n: int):
    """Integers in [0, n), n < 2^32 (multiply-shift on the top 32 bits)."""
    return _srl(_srl(bits, 32) * n, 32)


def t_normal(seed: int, stream: int, start: int, count: int, device):
    import torch
    u1 = t_u01_open(t_rand_u64(seed, stream, start, count, device))
    u2 = t_u01(t_rand_u64(seed, stream + 1000, start, count, device))
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


DISTRIBUTIONS = ("uniform", "lognormal", "clustered")


def _keys(dist: str, seed: int, stream: int, count: int, device):
    """`count` raw keys of a distribution (not deduplicated), int64 bits."""
    import torch
    if dist == "uniform":
        return _srl(t_rand_u64(seed, stream, 0, count, device), 1)
    if dist == "lognormal":
        z = t_normal(seed, stream, 0, count, device)
        return torch.round(1e9 * torch.exp(2.0 * z)).to(torch.int64)
    if dist == "clustered":
        centres = _srl(t_rand_u64(seed, ST_CLUSTER, 0, 64, device), 2).double()
        which = t_bounded(t_rand_u64(seed, stream + 100, 0, count, device), 64)
        z = t_normal(seed, stream, 0, count, device)
        v = torch.clamp(centres[which] + 1e6 * z, min=0.0)
        return torch.round(v).to(torch.int64)
    raise ValueError(dist)


def log_uniform_sizes(seed: int, stream: int, k: int, lo: int, hi: int) -> np.ndarray:
    from . import u01
    u = u01(rand_u64(seed, stream, 0, k))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def batched_workload(k: int = 4096, seed: int = 0, device="cuda", n_range=(1 << 10, 1 << 22),
                     m_range=(1 << 10, 1 << 24), scale: float = 1.0):
    """List of dicts {R, S, dist, n, m} with R sorted unique and S as described
    above (int64 tensors holding uint64 keys).  `scale` shrinks both size
    ranges (tests use small batches)."""
    import torch
    from . import u01
    n_sizes = log_uniform_sizes(seed, ST_BATCH_SIZES, k, max(1, int(n_range[0] * scale)),
                                max(2, int(n_range[1] * scale)))
    m_sizes = log_uniform_sizes(seed, ST_BATCH_SIZES + 50, k, max(1, int(m_range[0] * scale)),
                                max(2, int(m_range[1] * scale)))
    dists = (u01(rand_u64(seed, ST_BATCH_DIST, 0, k)) * 3).astype(np.int64)
    out = []
    for j in range(k):
        sj = seed * 1_000_003 + j
        dist = DISTRIBUTIONS[int(dists[j])]
        R = torch.unique(_keys(dist, sj, ST_R_KEYS, int(n_sizes[j]), device))   # sorted
        m = int(m_sizes[j])
        coin = t_u01(t_rand_u64(sj, ST_S_COIN, 0, m, device)) < 0.5
        hit_idx = t_bounded(t_rand_u64(sj, ST_S_HIT, 0, m, device), R.numel())
        fresh = _keys(dist, sj, ST_S_MISS, m, device)
        S = torch.where(coin, R[hit_idx], fresh)
        out.append({"R": R.contiguous(), "S": S.contiguous(), "dist": dist, "n": R.numel(), "m": m})
    return out
