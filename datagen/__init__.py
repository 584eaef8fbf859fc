"""Seeded synthetic workloads for the learned indexed nested loop join.

This module is shared by the tests, the benchmark and the oracle checks. It
holds no part of the join or of the learned index: it only draws the inner
relation R (sorted uint64 keys) and the outer relation S (uint64 probe keys).

Every random number comes from one counter-based generator, the splitmix64
sequence (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i of stream `k` under seed `s` is
mix(key(s, k) + (i + 1) * 0x9E3779B97F4A7C15), where mix is the splitmix64
finaliser. Results depend only on (seed, stream, counter), never on chunking
or thread count.

Workload shapes follow the synthetic datasets of the paper's evaluation
(Section 6.A: sequential with holes, uniform, lognormal), at the sizes and
parameters of the five workloads this library is measured on:

  uniform_1m        R = 1M unique keys uniform in [0, 2^63); S = 1M keys drawn
                    with replacement from R (every probe matches once).
  lognormal_100m    R = 100M unique keys round(1e9 * LogNormal(0, 2)); S = 400M
                    keys, half Zipf(0.99) over R's ranks (rank 1 = smallest
                    key), half true misses uniform in [min R, max R].
  dup_seqh_50m      R = 50M rows, sequential keys with 10% holes, each key
                    repeated min(Zipf(1.2), 64) times; S = 200M keys uniform
                    over R's distinct keys.
  batched / served  see `batched_workload` and `served_relations`.
  lsj_uniform_100m  unsorted relations for the sort-based join: R = 100M
                    distinct uniform keys in random order; S = 100M draws
                    from R (every probe matches once), in random order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_U64 = np.uint64
_GAMMA = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)
_STREAM_MUL = _U64(0xD1B54A32D192ED03)
_CHUNK = 1 << 24

# Stream ids: each distribution parameter draws from its own stream.
ST_R_KEYS, ST_R_NORM2, ST_S_COIN, ST_S_HIT, ST_S_MISS = 1, 2, 3, 4, 5
ST_HOLES, ST_MULT, ST_BATCH_SIZES, ST_BATCH_DIST, ST_CLUSTER = 6, 7, 8, 9, 10
ST_ARRIVAL = 11
ST_SHUFFLE_R, ST_SHUFFLE_S = 12, 13


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser, in place on a uint64 array (wrapping arithmetic)."""
    z ^= z >> _U64(30)
    z *= _M1
    z ^= z >> _U64(27)
    z *= _M2
    z ^= z >> _U64(31)
    return z


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.array([(seed & 0xFFFFFFFFFFFFFFFF)], dtype=_U64)
        k ^= _U64(stream) * _STREAM_MUL
        return _mix(k)[0]


def rand_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream (uint64)."""
    key = _stream_key(seed, stream)
    out = np.empty(count, dtype=_U64)
    with np.errstate(over="ignore"):
        for c0 in range(0, count, _CHUNK):
            c1 = min(count, c0 + _CHUNK)
            z = np.arange(start + c0 + 1, start + c1 + 1, dtype=_U64)
            z *= _GAMMA
            z += key
            out[c0:c1] = _mix(z)
    return out


def u01_open(bits: np.ndarray) -> np.ndarray:
    """Map uint64 draws to doubles in (0, 1] (53-bit resolution)."""
    return ((bits >> _U64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def u01(bits: np.ndarray) -> np.ndarray:
    """Map uint64 draws to doubles in [0, 1)."""
    return (bits >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def bounded(bits: np.ndarray, n: int) -> np.ndarray:
    """Map uint64 draws to integers in [0, n), n < 2^32 (multiply-shift)."""
    assert 0 < n <= 0xFFFFFFFF
    with np.errstate(over="ignore"):
        return ((bits >> _U64(32)) * _U64(n)) >> _U64(32)


def normal(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Standard normal draws by Box-Muller on two counter streams."""
    u1 = u01_open(rand_u64(seed, stream, start, count))
    u2 = u01(rand_u64(seed, stream + 1000, start, count))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _unique_in_draw_order(vals: np.ndarray, want: int) -> np.ndarray | None:
    """First `want` distinct values of `vals` in draw order, or None if short."""
    uniq, first = np.unique(vals, return_index=True)
    if uniq.size < want:
        return None
    first.sort()
    return vals[first[:want]]


def _draw_unique(draw, n: int) -> np.ndarray:
    """Draw until n distinct keys exist; keep the first n in draw order."""
    count = n + max(16, n // 64)
    while True:
        vals = draw(count)
        got = _unique_in_draw_order(vals, n)
        if got is not None:
            got.sort()
            return got
        count = count * 2


# --------------------------------------------------------------------------
# Zipf samplers
# --------------------------------------------------------------------------

def zeta(n: float, theta: float, exact_terms: int = 100000) -> float:
    """sum_{i=1..n} i^-theta (n may be inf for theta > 1), Euler-Maclaurin tail."""
    k = int(min(n, exact_terms))
    i = np.arange(1, k + 1, dtype=np.float64)
    s = float(np.sum(i ** -theta))
    if n <= exact_terms:
        return s
    # tail sum_{i=k+1..n} f(i) with f(x) = x^-theta
    a = float(k)

    def f(x):
        return x ** -theta

    def fp(x):
        return -theta * x ** (-theta - 1)

    if math.isinf(n):
        integral = a ** (1 - theta) / (theta - 1)
        return s + integral - f(a) / 2 - fp(a) / 12
    b = float(n)
    if theta == 1.0:
        integral = math.log(b / a)
    else:
        integral = (b ** (1 - theta) - a ** (1 - theta)) / (1 - theta)
    return s + integral + (f(b) - f(a)) / 2 + (fp(b) - fp(a)) / 12


class ZipfGray:
    """Bounded Zipf(theta) over ranks 1..n by the method of Gray et al.,
    "Quickly generating billion-record synthetic databases", SIGMOD 1994."""

    def __init__(self, n: int, theta: float):
        self.n, self.theta = n, theta
        self.alpha = 1.0 / (1.0 - theta)
        self.zetan = zeta(n, theta)
        zeta2 = 1.0 + 0.5 ** theta
        self.eta = (1.0 - (2.0 / n) ** (1.0 - theta)) / (1.0 - zeta2 / self.zetan)

    def ranks(self, u: np.ndarray) -> np.ndarray:
        uz = u * self.zetan
        base = np.maximum(self.eta * u - self.eta + 1.0, 0.0)
        r = 1.0 + np.floor(self.n * base ** self.alpha)
        r = np.where(uz < 1.0 + 0.5 ** self.theta, 2.0, r)
        r = np.where(uz < 1.0, 1.0, r)
        return np.clip(r, 1, self.n).astype(np.int64)


def zipf_clipped_table(s: float, cap: int) -> np.ndarray:
    """CDF over k = 1..cap of an unbounded Zipf(s) whose draws are clipped at
    cap (all mass of k >= cap sits on cap)."""
    z = zeta(math.inf, s)
    k = np.arange(1, cap, dtype=np.float64)
    p = k ** -s / z
    cdf = np.concatenate([np.cumsum(p), [1.0]])
    return cdf


def zipf_truncated_table(s: float, cap: int) -> np.ndarray:
    """CDF over k = 1..cap of a Zipf(s) truncated to support 1..cap (mass
    renormalised over the support)."""
    k = np.arange(1, cap + 1, dtype=np.float64)
    p = k ** -s
    cdf = np.cumsum(p / p.sum())
    cdf[-1] = 1.0
    return cdf


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    R: np.ndarray               # sorted uint64
    S: np.ndarray               # uint64
    leaves: int
    precision: str              # "fp32" | "fp64"
    meta: dict = field(default_factory=dict)


def uniform_unique(n: int, seed: int, bits: int = 63) -> np.ndarray:
    """n distinct keys uniform in [0, 2^bits), sorted."""
    shift = _U64(64 - bits)
    return _draw_unique(lambda c: rand_u64(seed, ST_R_KEYS, 0, c) >> shift, n)


def uniform_1m(seed: int = 0, n: int = 1 << 20, m: int | None = None,
               leaves: int = 4096) -> Workload:
    """R: n unique uniform 63-bit keys; S: m draws with replacement from R.
    The default sizes are 1M = 2^20 keys on each side."""
    m = n if m is None else m
    R = uniform_unique(n, seed)
    idx = bounded(rand_u64(seed, ST_S_HIT, 0, m), n) if n else np.zeros(0, np.uint64)
    S = R[idx.astype(np.int64)] if n else np.zeros(m, np.uint64)
    return Workload("uniform_1m", R, S, leaves, "fp64",
                    {"expected_pairs": m if n else 0})


def lognormal_keys(n: int, seed: int, sigma: float = 2.0,
                   scale: float = 1e9) -> np.ndarray:
    """n distinct keys round(scale * exp(sigma * N(0,1))), sorted."""
    def draw(c):
        z = normal(seed, ST_R_KEYS, 0, c)
        return np.rint(scale * np.exp(sigma * z)).astype(np.uint64)
    return _draw_unique(draw, n)


def _true_misses(R: np.ndarray, seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """count keys uniform in [lo, hi] none of which occurs in R (redrawn)."""
    span = _U64(hi - lo + 1) if hi - lo + 1 < (1 << 64) else None
    out = np.empty(count, dtype=_U64)
    todo = np.arange(count, dtype=np.int64)
    start = 0
    while todo.size:
        b = rand_u64(seed, ST_S_MISS, start, todo.size)
        start += todo.size
        cand = (b % span + _U64(lo)) if span is not None else b
        pos = np.searchsorted(R, cand)
        hit = (pos < R.size) & (R[np.minimum(pos, R.size - 1)] == cand)
        out[todo[~hit]] = cand[~hit]
        todo = todo[hit]
    return out


def lognormal_100m(seed: int = 0, n: int = 100_000_000, m: int = 400_000_000,
                   leaves: int = 1 << 20, hit_frac: float = 0.5,
                   theta: float = 0.99, precision: str = "fp32") -> Workload:
    """R: n unique lognormal(0, 2) keys scaled by 1e9; S: per probe a coin
    chooses a Zipf(theta) hit over R's ranks or a true miss."""
    R = lognormal_keys(n, seed)
    coin = u01(rand_u64(seed, ST_S_COIN, 0, m)) < hit_frac
    hits_j = np.flatnonzero(coin)
    miss_j = np.flatnonzero(~coin)
    S = np.empty(m, dtype=_U64)
    zg = ZipfGray(n, theta)
    rank = zg.ranks(u01(rand_u64(seed, ST_S_HIT, 0, hits_j.size)))
    S[hits_j] = R[rank - 1]
    S[miss_j] = _true_misses(R, seed, miss_j.size, int(R[0]), int(R[-1]))
    return Workload("lognormal_100m", R, S, leaves, precision,
                    {"hits": int(hits_j.size), "expected_pairs": int(hits_j.size),
                     "hit_mask": coin})


def dup_seqh(rows: int, seed: int, skip_p: float = 0.1, s: float = 1.2,
             cap: int = 64, reading: str = "clip") -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Sequential keys from 0 with each value skipped with probability
    skip_p; each kept value repeated min(Zipf(s), cap) times ("clip": an
    unbounded Zipf clipped at cap) or a Zipf truncated to 1..cap times
    ("truncate"); truncated to `rows` rows. Returns (R sorted, distinct keys,
    multiplicity per key)."""
    if reading not in ("clip", "truncate"):
        raise ValueError(reading)
    cdf = zipf_clipped_table(s, cap) if reading == "clip" else zipf_truncated_table(s, cap)
    keep_p = 1.0 - skip_p
    mean_mult = float(np.sum(np.diff(np.concatenate([[0.0], cdf])) *
                             np.arange(1, cap + 1)))
    V = int(rows / (keep_p * mean_mult) * 1.1) + 64
    while True:
        keep = u01(rand_u64(seed, ST_HOLES, 0, V)) >= skip_p
        vals = np.flatnonzero(keep).astype(np.uint64)
        u = u01(rand_u64(seed, ST_MULT, 0, V))[keep]
        mult = (np.searchsorted(cdf, u, side="right") + 1).astype(np.int64)
        mult = np.minimum(mult, cap)
        csum = np.cumsum(mult)
        if csum.size and csum[-1] >= rows:
            break
        V *= 2
    last = int(np.searchsorted(csum, rows, side="left"))
    vals = vals[: last + 1]
    mult = mult[: last + 1].copy()
    mult[-1] -= int(csum[last] - rows)
    R = np.repeat(vals, mult)
    return R, vals, mult


def dup_seqh_50m(seed: int = 0, rows: int = 50_000_000, m: int = 200_000_000,
                 leaves: int = 1 << 18, reading: str = "clip") -> Workload:
    """R: duplicated sequential-with-holes keys; S: uniform over distinct keys.
    `reading` picks how "Zipf(1.2) capped at 64" is read: "clip" (an unbounded
    draw clipped at 64, mean multiplicity ~31) or "truncate" (support 1..64,
    mean ~10)."""
    R, vals, mult = dup_seqh(rows, seed, reading=reading)
    pick = bounded(rand_u64(seed, ST_S_HIT, 0, m), vals.size).astype(np.int64)
    S = vals[pick]
    expected = int(np.sum(mult[pick], dtype=np.int64))
    return Workload("dup_seqh_50m", R, S, leaves, "fp32",
                    {"expected_pairs": expected, "distinct": int(vals.size),
                     "zipf_reading": reading})


def clustered_keys(n: int, seed: int, clusters: int = 64,
                   sigma: float = 1e6) -> np.ndarray:
    """n distinct keys from `clusters` Gaussian clusters (std sigma) with
    centres uniform in [0, 2^62), sorted."""
    centres = (rand_u64(seed, ST_CLUSTER, 0, clusters) >> _U64(2)).astype(np.float64)

    def draw(c):
        which = bounded(rand_u64(seed, ST_R_KEYS + 100, 0, c), clusters).astype(np.int64)
        z = normal(seed, ST_R_KEYS, 0, c)
        v = np.maximum(centres[which] + sigma * z, 0.0)
        return np.rint(v).astype(np.uint64)
    return _draw_unique(draw, n)


WORKLOADS = {
    "uniform_1m": uniform_1m,
    "lognormal_100m": lognormal_100m,
    "dup_seqh_50m": dup_seqh_50m,
}


def lsj_uniform_100m(seed: int = 0, n: int = 100_000_000, m: int = 100_000_000) -> Workload:
    """Unsorted R (n distinct uniform 63-bit keys, shuffled) and S (m draws
    from R with replacement, so every key of S matches exactly once).  The
    shuffle orders the keys by a splitmix64 draw per position."""
    R = uniform_unique(n, seed)[np.argsort(rand_u64(seed, ST_SHUFFLE_R, 0, n), kind="stable")]
    S = R[bounded(rand_u64(seed, ST_S_HIT, 0, m), n).astype(np.int64)] if n else \
        np.zeros(0, np.uint64)
    return Workload("lsj_uniform_100m", R, S, 0, "fp32", {"expected_pairs": m if n else 0})
