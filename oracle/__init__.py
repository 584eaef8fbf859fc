"""CPU oracle for the learned indexed nested loop join.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the library itself.  It
shares no code with the CUDA implementation and does not import it.

The arithmetic lives in `ljoin_oracle.c` (plain C, built with gcc); this
module compiles it on first use and wraps it for numpy arrays.  It also
carries `brute_force_join`, the nested-loop definition of the join in pure
Python, used only on tiny inputs to pin the C sort-merge.

Functions and the passages they follow (Sabek and Kraska, "The Case for
Learned In-Memory Joins"):
  join_ranges / join_pairs   Section 2.A (indexed nested loop join) and
                             Section 6.B (duplicates return all matches);
                             join_ranges_mt runs join_ranges on chunks of S
                             on every host core
  rmi_fit / rmi_lookup       Section 2.D (two-level RMI with per-leaf
                             min/max error bounds and a bounded search)
  grmi_build / grmi_join     Section 3.A (gapped RMI: model-based insertion
                             into gapped key and payload arrays, lookup by
                             exponential search from the predicted slot)
  lhash_build / lhash_join   Section 3.C (learned hash index: the CDF model as
                             an order-preserving hash into a table of 4-slot
                             buckets with linear probing)
  rs_build / rs_predict      Section 2.D (RadixSpline: greedy error-bounded
                             spline over the CDF, radix table over key
                             prefixes, interpolation between spline points)
  rs_lhash_build / _join     Section 3.C with a RadixSpline as the hash
                             (the paper's RSHASH-INLJ)
  join_pairs_unsorted        Section 4 (sort-based join of two unsorted
                             relations): J = {(i, j) : R[i] == S[j]} with i, j
                             positions in the relations as given
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ljoin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libljoin_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            U64 = ctypes.c_uint64
            lib.lj_oracle_is_sorted.argtypes = [P, U64]
            lib.lj_oracle_is_sorted.restype = ctypes.c_int
            lib.lj_oracle_join_ranges.argtypes = [P, U64, P, U64, P, P]
            lib.lj_oracle_join_ranges.restype = ctypes.c_int64
            lib.lj_oracle_join_pairs.argtypes = [P, U64, P, U64, P, U64]
            lib.lj_oracle_join_pairs.restype = ctypes.c_int64
            lib.lj_oracle_rmi_fit.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int,
                                              P, P, P, P, P, P]
            lib.lj_oracle_rmi_fit.restype = ctypes.c_int
            lib.lj_oracle_rmi_lookup.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int,
                                                 P, P, P, P, U64, P, P, P, P]
            lib.lj_oracle_rmi_lookup.restype = ctypes.c_uint32
            lib.lj_oracle_grmi_pslot.argtypes = [P, ctypes.c_uint32, ctypes.c_int, P, P, P,
                                                 ctypes.c_uint32, U64]
            lib.lj_oracle_grmi_pslot.restype = U64
            lib.lj_oracle_grmi_build.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int, P, P, P,
                                                 ctypes.c_uint32, P, P, U64, P]
            lib.lj_oracle_grmi_build.restype = ctypes.c_int64
            lib.lj_oracle_grmi_join_ranges.argtypes = [P, ctypes.c_uint32, ctypes.c_int, P, P,
                                                       P, ctypes.c_uint32, P, P, U64, P, U64,
                                                       P, P, P]
            lib.lj_oracle_grmi_join_ranges.restype = ctypes.c_int64
            lib.lj_oracle_lhash_build.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int, P, P, P,
                                                  ctypes.c_uint32, P, P, U64, P, P, P]
            lib.lj_oracle_lhash_build.restype = ctypes.c_int64
            lib.lj_oracle_lhash_join_ranges.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int, P,
                                                        P, P, U64, P, P, U64, P, U64, P, U64, P,
                                                        P, P]
            lib.lj_oracle_lhash_join_ranges.restype = ctypes.c_int64
            lib.lj_oracle_rs_build.argtypes = [P, U64, ctypes.c_uint32, U64, ctypes.c_uint32,
                                               P, P, U64, P, P]
            lib.lj_oracle_rs_build.restype = ctypes.c_int64
            lib.lj_oracle_rs_predict_many.argtypes = [P, P, U64, U64, P, U64, P]
            lib.lj_oracle_rs_predict_many.restype = None
            lib.lj_oracle_rs_lhash_build.argtypes = [P, U64, P, P, U64, ctypes.c_uint32, P, P,
                                                     U64, P, P, P]
            lib.lj_oracle_rs_lhash_build.restype = ctypes.c_int64
            lib.lj_oracle_rs_lhash_join_ranges.argtypes = [P, U64, P, P, U64, U64, P, P, U64,
                                                           P, U64, P, U64, P, P]
            lib.lj_oracle_rs_lhash_join_ranges.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _u64(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype != np.uint64:
        if a.dtype.kind not in "iu" or (a.size and a.min() < 0):
            raise TypeError(f"keys must be unsigned 64-bit integers, got {a.dtype}")
        a = a.astype(np.uint64)
    return np.ascontiguousarray(a)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


class OracleError(ValueError):
    pass


def is_sorted(R) -> bool:
    R = _u64(R)
    return bool(_load().lj_oracle_is_sorted(_ptr(R), R.size))


def join_ranges(R, S) -> tuple[np.ndarray, np.ndarray, int]:
    """Per-probe match ranges [lo_j, hi_j) into sorted R, and |J|."""
    R, S = _u64(R), _u64(S)
    lo = np.zeros(S.size, dtype=np.uint64)
    hi = np.zeros(S.size, dtype=np.uint64)
    total = _load().lj_oracle_join_ranges(_ptr(R), R.size, _ptr(S), S.size,
                                          _ptr(lo), _ptr(hi))
    if total == -1:
        raise OracleError("R is not sorted non-decreasing")
    if total < 0:
        raise MemoryError("oracle ran out of memory")
    return lo, hi, int(total)


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:          # not Linux
        return os.cpu_count() or 1


def join_ranges_mt(R, S, threads: int | None = None, chunk: int = 1 << 20
                   ) -> tuple[np.ndarray, np.ndarray, int]:
    """join_ranges over contiguous chunks of S on `threads` host threads (all
    cores by default).  Each chunk is one unchanged call of the C sort-merge
    (ctypes releases the GIL during the call), writing its slice of lo / hi;
    per-probe ranges do not depend on the chunking."""
    from concurrent.futures import ThreadPoolExecutor
    R, S = _u64(R), _u64(S)
    threads = threads or host_threads()
    lo = np.zeros(S.size, dtype=np.uint64)
    hi = np.zeros(S.size, dtype=np.uint64)
    lib = _load()
    if S.size and not lib.lj_oracle_is_sorted(_ptr(R), R.size):
        raise OracleError("R is not sorted non-decreasing")
    chunk = max(1 << 14, min(chunk, -(-S.size // (4 * threads))))   # >= 4 chunks per thread
    bounds = [(a, min(S.size, a + chunk)) for a in range(0, S.size, chunk)]

    def one(ab):
        a, b = ab
        t = lib.lj_oracle_join_ranges(_ptr(R), R.size, _ptr(S[a:b]), b - a,
                                      _ptr(lo[a:b]), _ptr(hi[a:b]))
        if t < 0:
            raise MemoryError("oracle ran out of memory") if t == -2 else OracleError("unsorted R")
        return t

    if threads <= 1 or len(bounds) <= 1:
        total = sum(one(ab) for ab in bounds)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            total = sum(ex.map(one, bounds))
    return lo, hi, int(total)


def join_pairs(R, S, cap: int | None = None) -> np.ndarray:
    """All (r_idx, s_idx) pairs, s ascending then r ascending, as (k, 2) uint32."""
    R, S = _u64(R), _u64(S)
    lib = _load()
    if cap is None:
        _, _, cap = join_ranges(R, S)
    out = np.zeros((max(cap, 1), 2), dtype=np.uint32)
    total = lib.lj_oracle_join_pairs(_ptr(R), R.size, _ptr(S), S.size, _ptr(out), cap)
    if total == -1:
        raise OracleError("R is not sorted non-decreasing")
    if total < 0:
        raise MemoryError("oracle ran out of memory")
    return out[: min(total, cap)]


def brute_force_join(R, S) -> list[tuple[int, int]]:
    """Nested loops over every (i, j): the definition of J(R, S). Tiny inputs."""
    R = [int(v) for v in R]
    S = [int(v) for v in S]
    return [(i, j) for j in range(len(S)) for i in range(len(R)) if R[i] == S[j]]


@dataclass
class RMI:
    """A fitted two-level linear RMI (oracle side)."""
    L: int
    fp64: bool
    root_fit: np.ndarray   # (2,) float64: least-squares (a0, b0)
    root_dep: np.ndarray   # (2,) deployed (a0, b0)
    leaf_lo: np.ndarray    # (L+1,) uint64
    leaf_fit: np.ndarray   # (L, 2) float64
    leaf_dep: np.ndarray   # (L, 2) deployed
    err: np.ndarray        # (L, 2) int64: (e_lo, e_hi)


def rmi_fit(R, L: int, fp64: bool = False) -> RMI:
    R = _u64(R)
    root_fit = np.zeros(2)
    root_dep = np.zeros(2)
    leaf_lo = np.zeros(L + 1, dtype=np.uint64)
    leaf_fit = np.zeros((L, 2))
    leaf_dep = np.zeros((L, 2))
    err = np.zeros((L, 2), dtype=np.int64)
    rc = _load().lj_oracle_rmi_fit(_ptr(R), R.size, L, int(fp64), _ptr(root_fit),
                                   _ptr(root_dep), _ptr(leaf_lo), _ptr(leaf_fit),
                                   _ptr(leaf_dep), _ptr(err))
    if rc == -1:
        raise OracleError("R is not sorted or L == 0")
    if rc < 0:
        raise MemoryError("oracle ran out of memory")
    return RMI(L, fp64, root_fit, root_dep, leaf_lo, leaf_fit, leaf_dep, err)


def rmi_lookup(R, rmi: RMI, x: int) -> dict:
    """Learned lookup of one key: leaf, window [w_lo, w_hi) and [lb, ub)."""
    R = _u64(R)
    out = [ctypes.c_uint64() for _ in range(4)]
    leaf = _load().lj_oracle_rmi_lookup(
        _ptr(R), R.size, rmi.L, int(rmi.fp64), _ptr(rmi.root_dep), _ptr(rmi.leaf_lo),
        _ptr(rmi.leaf_dep), _ptr(rmi.err), int(x), *[ctypes.byref(o) for o in out])
    lb, ub, wl, wh = (o.value for o in out)
    return {"leaf": int(leaf), "lb": lb, "ub": ub, "w_lo": wl, "w_hi": wh}


@dataclass
class GRMI:
    """Gapped arrays of a GRMI (oracle side): C slots of keys, C+1 payloads
    (positions in R; pos[C] = n), and the slot every key of R took."""
    rmi: RMI
    gaps: int
    keys: np.ndarray       # (C,) uint64
    pos: np.ndarray        # (C+1,) uint32
    slot_of_key: np.ndarray  # (n,) uint64


def grmi_pslot(R, rmi: RMI, gaps: int, x: int) -> int:
    """Predicted slot of one key (before clamping to the array length)."""
    R = _u64(R)
    return int(_load().lj_oracle_grmi_pslot(_ptr(R), rmi.L, int(rmi.fp64), _ptr(rmi.root_dep),
                                            _ptr(rmi.leaf_lo), _ptr(rmi.leaf_dep), gaps, int(x)))


def grmi_build(R, rmi: RMI, gaps: int) -> GRMI:
    """Model-based insertion of sorted R into the gapped arrays."""
    R = _u64(R)
    lib = _load()
    args = (_ptr(R), R.size, rmi.L, int(rmi.fp64), _ptr(rmi.root_dep), _ptr(rmi.leaf_lo),
            _ptr(rmi.leaf_dep), gaps)
    C = lib.lj_oracle_grmi_build(*args, None, None, 0, None)
    if C == -1:
        raise OracleError("R is not sorted non-decreasing")
    if C < 0:
        raise MemoryError("oracle ran out of memory")
    keys = np.zeros(C, dtype=np.uint64)
    pos = np.zeros(C + 1, dtype=np.uint32)
    slot = np.zeros(R.size, dtype=np.uint64)
    rc = lib.lj_oracle_grmi_build(*args, _ptr(keys), _ptr(pos), C, _ptr(slot))
    if rc != C:
        raise OracleError(f"gapped build failed ({rc})")
    return GRMI(rmi, gaps, keys, pos, slot)


def grmi_join(R, g: GRMI, S) -> tuple[np.ndarray, np.ndarray, int, np.ndarray]:
    """Per-probe match ranges [lo_j, hi_j) found through the GRMI, |J|, and
    the number of keys each probe's searches read."""
    R, S = _u64(R), _u64(S)
    lo = np.zeros(S.size, dtype=np.uint64)
    hi = np.zeros(S.size, dtype=np.uint64)
    loads = np.zeros(S.size, dtype=np.uint64)
    r = g.rmi
    total = _load().lj_oracle_grmi_join_ranges(
        _ptr(R), r.L, int(r.fp64), _ptr(r.root_dep), _ptr(r.leaf_lo), _ptr(r.leaf_dep), g.gaps,
        _ptr(g.keys), _ptr(g.pos), g.keys.size, _ptr(S), S.size, _ptr(lo), _ptr(hi), _ptr(loads))
    return lo, hi, int(total), loads


@dataclass
class LHash:
    """Learned hash index (oracle side): C slots of keys, C+1 payloads
    (distinct-key ranks; pos[C] = D), first[D+1] positions in R, B buckets."""
    rmi: RMI
    spk: int
    keys: np.ndarray      # (C,) uint64
    pos: np.ndarray       # (C+1,) uint32
    first: np.ndarray     # (D+1,) uint32
    D: int
    B: int


def lhash_build(R, rmi: RMI, spk: int) -> LHash:
    R = _u64(R)
    lib = _load()
    args = (_ptr(R), R.size, rmi.L, int(rmi.fp64), _ptr(rmi.root_dep), _ptr(rmi.leaf_lo),
            _ptr(rmi.leaf_dep), spk)
    D, B = ctypes.c_uint64(), ctypes.c_uint64()
    C = lib.lj_oracle_lhash_build(*args, None, None, 0, None, ctypes.byref(D), ctypes.byref(B))
    if C == -1:
        raise OracleError("R is not sorted non-decreasing")
    if C < 0:
        raise MemoryError("oracle ran out of memory")
    keys = np.zeros(C, dtype=np.uint64)
    pos = np.zeros(C + 1, dtype=np.uint32)
    first = np.zeros(D.value + 1, dtype=np.uint32)
    rc = lib.lj_oracle_lhash_build(*args, _ptr(keys), _ptr(pos), C, _ptr(first), None, None)
    if rc != C:
        raise OracleError(f"hash build failed ({rc})")
    return LHash(rmi, spk, keys, pos, first, D.value, B.value)


def lhash_join(R, h: LHash, S) -> tuple[np.ndarray, np.ndarray, int, np.ndarray]:
    """Per-probe match ranges through the learned hash index, |J|, and the
    number of table slots each lookup read."""
    R, S = _u64(R), _u64(S)
    lo = np.zeros(S.size, dtype=np.uint64)
    hi = np.zeros(S.size, dtype=np.uint64)
    loads = np.zeros(S.size, dtype=np.uint64)
    r = h.rmi
    total = _load().lj_oracle_lhash_join_ranges(
        _ptr(R), R.size, r.L, int(r.fp64), _ptr(r.root_dep), _ptr(r.leaf_lo), _ptr(r.leaf_dep),
        h.B, _ptr(h.keys), _ptr(h.pos), h.keys.size, _ptr(h.first), h.D, _ptr(S), S.size,
        _ptr(lo), _ptr(hi), _ptr(loads))
    return lo, hi, int(total), loads


@dataclass
class RadixSpline:
    """RadixSpline of a sorted R (oracle side): S spline points (sx, sy),
    radix table (2^rbits + 1 entries) over (key - sx[0]) >> shift."""
    eps: int
    chunk: int
    rbits: int
    sx: np.ndarray        # (S,) uint64
    sy: np.ndarray        # (S,) uint32
    table: np.ndarray     # (2^rbits + 1,) uint32
    shift: int
    n: int


def rs_build(R, eps: int = 32, chunk: int = 1024, rbits: int = 18) -> RadixSpline:
    R = _u64(R)
    lib = _load()
    shift = ctypes.c_uint32()
    S = lib.lj_oracle_rs_build(_ptr(R), R.size, eps, chunk, rbits, None, None, 0, None,
                               ctypes.byref(shift))
    if S == -1:
        raise OracleError("R is not sorted non-decreasing")
    if S < 0:
        raise MemoryError("oracle ran out of memory")
    sx = np.zeros(S, dtype=np.uint64)
    sy = np.zeros(S, dtype=np.uint32)
    table = np.zeros((1 << rbits) + 1, dtype=np.uint32)
    rc = lib.lj_oracle_rs_build(_ptr(R), R.size, eps, chunk, rbits, _ptr(sx), _ptr(sy), S,
                                _ptr(table), ctypes.byref(shift))
    if rc != S:
        raise OracleError(f"RadixSpline build failed ({rc})")
    return RadixSpline(eps, chunk, rbits, sx, sy, table, int(shift.value), int(R.size))


def rs_predict(rs: RadixSpline, X) -> np.ndarray:
    """Predicted position of every key of X (uint64)."""
    X = _u64(X)
    out = np.zeros(X.size, dtype=np.uint64)
    _load().lj_oracle_rs_predict_many(_ptr(rs.sx), _ptr(rs.sy), rs.sx.size, rs.n, _ptr(X),
                                      X.size, _ptr(out))
    return out


@dataclass
class RSHash:
    """Learned hash index with a RadixSpline as the hash (oracle side)."""
    rs: RadixSpline
    spk: int
    keys: np.ndarray      # (C,) uint64
    pos: np.ndarray       # (C+1,) uint32
    first: np.ndarray     # (D+1,) uint32
    D: int
    B: int


def rs_lhash_build(R, rs: RadixSpline, spk: int) -> RSHash:
    R = _u64(R)
    lib = _load()
    args = (_ptr(R), R.size, _ptr(rs.sx), _ptr(rs.sy), rs.sx.size, spk)
    D, B = ctypes.c_uint64(), ctypes.c_uint64()
    C = lib.lj_oracle_rs_lhash_build(*args, None, None, 0, None, ctypes.byref(D),
                                     ctypes.byref(B))
    if C == -1:
        raise OracleError("R is not sorted non-decreasing")
    if C < 0:
        raise MemoryError("oracle ran out of memory")
    keys = np.zeros(C, dtype=np.uint64)
    pos = np.zeros(C + 1, dtype=np.uint32)
    first = np.zeros(D.value + 1, dtype=np.uint32)
    rc = lib.lj_oracle_rs_lhash_build(*args, _ptr(keys), _ptr(pos), C, _ptr(first), None, None)
    if rc != C:
        raise OracleError(f"hash build failed ({rc})")
    return RSHash(rs, spk, keys, pos, first, D.value, B.value)


def rs_lhash_join(R, h: RSHash, S) -> tuple[np.ndarray, np.ndarray, int]:
    """Per-probe match ranges through the RadixSpline hash index and |J|."""
    R, S = _u64(R), _u64(S)
    lo = np.zeros(S.size, dtype=np.uint64)
    hi = np.zeros(S.size, dtype=np.uint64)
    rs = h.rs
    total = _load().lj_oracle_rs_lhash_join_ranges(
        _ptr(R), R.size, _ptr(rs.sx), _ptr(rs.sy), rs.sx.size, h.B, _ptr(h.keys), _ptr(h.pos),
        h.keys.size, _ptr(h.first), h.D, _ptr(S), S.size, _ptr(lo), _ptr(hi))
    return lo, hi, int(total)


def join_pairs_unsorted(R, S) -> np.ndarray:
    """The join of two unsorted relations (Section 4's learned sort-merge join
    computes it): all (i, j) with R[i] == S[j], i and j positions in R and S
    as given, ordered by j then i, as (k, 2) uint32.  R is sorted with its
    positions (numpy's stable sort: equal keys keep their order), then the
    sort-merge join above gives each probe's run of R."""
    R, S = _u64(R), _u64(S)
    perm = np.argsort(R, kind="stable")
    lo, hi, total = join_ranges(R[perm], S)
    out = np.zeros((total, 2), dtype=np.uint32)
    cnt = (hi - lo).astype(np.int64)
    j = np.repeat(np.arange(S.size, dtype=np.int64), cnt)
    first = np.repeat(lo.astype(np.int64), cnt)
    start = np.repeat(np.cumsum(cnt) - cnt, cnt)
    r_sorted = first + (np.arange(total, dtype=np.int64) - start)
    out[:, 0] = perm[r_sorted]
    out[:, 1] = j
    return out
