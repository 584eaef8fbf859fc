"""ctypes binding of libljoin (include/ljoin.h): argument marshalling only.

Every computation runs in the CUDA library.  There is no CPU fallback: if
the library cannot be loaded (not built, or built for another machine) the
first call raises.  torch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

LJ_FP32, LJ_FP64 = 0, 1
_ERR_NAMES = {
    -1: "LJ_E_INVAL", -2: "LJ_E_NOMEM", -3: "LJ_E_CUDA", -4: "LJ_E_UNSORTED",
    -5: "LJ_E_CAPACITY", -6: "LJ_E_TIMEOUT", -7: "LJ_E_BUDGET", -8: "LJ_E_NOTUNIQUE",
    -9: "LJ_E_STATE",
}


class LJoinError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class lj_index_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("leaves", ctypes.c_uint32),
                ("precision", ctypes.c_int32), ("unique", ctypes.c_int32),
                ("nonempty_leaves", ctypes.c_uint32), ("max_leaf_size", ctypes.c_uint32),
                ("max_window", ctypes.c_uint32), ("mean_window", ctypes.c_double),
                ("root_a", ctypes.c_double), ("root_b", ctypes.c_double),
                ("build_ms", ctypes.c_double)]


class lj_grmi_stats(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint64), ("gaps", ctypes.c_uint32),
                ("kind", ctypes.c_uint32), ("mean_disp", ctypes.c_double),
                ("max_disp", ctypes.c_uint64), ("build_ms", ctypes.c_double),
                ("distinct", ctypes.c_uint64)]


class lj_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("streams", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32)]


class lj_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("pairs", ctypes.c_uint64),
                ("pairs_dev", ctypes.c_void_p), ("latency_us", ctypes.c_double),
                ("queue_us", ctypes.c_double)]


class lj_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("keys", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double),
                ("mem_in_use", ctypes.c_uint64), ("mem_peak", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("span_s", ctypes.c_double), ("keys_per_s", ctypes.c_double),
                ("resident", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None

# every function declared in include/ljoin.h, with its ctypes signature
_P, _U64, _U32, _I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
SIGNATURES = {
    "rmi_build": ([_P, _U64, _U32, _I, _P, _P], _I),
    "rmi_build_batch": ([_P, _P, _P, _U32, _I, _P, _P], _I),
    "rmi_free": ([_P], None),
    "rmi_stats": ([_P, _P], _I),
    "rmi_export": ([_P, _P, _P, _P, _P], _I),
    "grmi_build": ([_P, _U32, _P], _I),
    "lhash_build": ([_P, _U32, _P], _I),
    "lhash_build_rs": ([_P, _U32, _U32, _U32, _P], _I),
    "rs_export": ([_P, _P, _P, _P, _P, _P], _I),
    "lsj_join": ([_P, _U64, _P, _U64, _P, _U64, _P, _P], _I),
    "lhash_export_first": ([_P, _P], _I),
    "index_autotune": ([_P, _P, _U64, _P, _P, _P], _I),
    "grmi_drop": ([_P], _I),
    "grmi_stats": ([_P, _P], _I),
    "grmi_export": ([_P, _P, _P], _I),
    "join_count": ([_P, _P, _U64, _P, _P, _P, _P], _I),
    "join_count_noalloc": ([_P, _P, _U64, _P, _P, _P, _P], _I),
    "join_emit": ([_P, _P, _U64, _P, _P, _U64, _P, _P, _P], _I),
    "join_host": ([_P, _P, _U64, _P, _U64, _P, _P], _I),
    "join_locate": ([_P, _P, _U64, _P, _P, _P, _P, _P], _I),
    "join_expand": ([_P, _P, _U64, _P, _U64, _P, _P, _P], _I),
    "join_batch_plan": ([_P, _P, _P, _U32, _P, _P, _P, _P], _I),
    "join_batch_run": ([_P, _P, _P, _P], _I),
    "join_batch_capture": ([_P, _P], _I),
    "join_batch_set_shape": ([_P, _I, _I], _I),
    "join_batch_autotune": ([_P, _P, _P, _P], _I),
    "join_batch_free": ([_P], None),
    "join_batch": ([_P, _P, _P, _U32, _P, _P, _P, _P], _I),
    "rmi_autotune": ([_P, _U64, _P, _U64, _I, _P, _P, _P], _I),
    "join_server_create": ([_P, _P], _I),
    "join_server_add_relation": ([_P, _P, _P], _I),
    "join_submit": ([_P, _U32, _P, _U64, _P], _I),
    "join_wait": ([_P, _U64, ctypes.c_int64, _P], _I),
    "join_fetch": ([_P, _U64, _P, _U64, _P], _I),
    "join_release": ([_P, _U64], _I),
    "join_server_stats": ([_P, _P, _I], _I),
    "join_server_destroy": ([_P], None),
    "rmi_autotune_clear": ([], None),
    "lj_set_option": ([ctypes.c_char_p, ctypes.c_int64], _I),
    "lj_get_option": ([ctypes.c_char_p], ctypes.c_int64),
    "lj_profile_report": ([ctypes.c_char_p, ctypes.c_size_t], _I),
    "lj_last_error": ([], ctypes.c_char_p),
    "lj_version": ([], ctypes.c_char_p),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libljoin.so (building it in-tree first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libljoin is not built ({path}); run build() first")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = load().lj_last_error().decode(errors="replace")
        raise LJoinError(rc, msg)


def _stream_ptr(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data if t.size else None
    return t.data_ptr() if t.numel() else None


def _require_cuda_u64(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in (torch.int64, torch.uint64) or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous 64-bit integer tensor")


@dataclass
class Index:
    """A learned index over R (keeps R alive: the library borrows it)."""
    handle: int
    R: object
    leaves: int
    precision: int

    def stats(self) -> dict:
        st = lj_index_stats()
        _check(load().rmi_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.rmi_free(h)


def rmi_build(R, leaves: int, precision: str | int = "fp32", stream=None) -> Index:
    """Fit the two-level linear RMI over the sorted device tensor R."""
    _require_cuda_u64(R, "R")
    prec = {"fp32": LJ_FP32, "fp64": LJ_FP64}.get(precision, precision)
    out = ctypes.c_void_p()
    _check(load().rmi_build(_ptr(R), R.numel(), leaves, prec, _stream_ptr(stream),
                            ctypes.byref(out)))
    return Index(out.value, R, leaves, prec)


def rmi_build_batch(Rs, leaves, precision: str | int = "fp32", stream=None) -> list:
    """Fit one RMI per sorted device tensor of Rs in one segmented pass;
    leaves[j] leaf models for Rs[j]."""
    k = len(Rs)
    if len(leaves) != k:
        raise ValueError("one leaf count per relation")
    for R in Rs:
        _require_cuda_u64(R, "R")
    prec = {"fp32": LJ_FP32, "fp64": LJ_FP64}.get(precision, precision)
    ptrs = _ptr_array(list(Rs)) if k else (ctypes.c_void_p * 1)()
    ns = (ctypes.c_uint64 * max(k, 1))(*[R.numel() for R in Rs])
    ls = (ctypes.c_uint32 * max(k, 1))(*[int(x) for x in leaves])
    out = (ctypes.c_void_p * max(k, 1))()
    _check(load().rmi_build_batch(ptrs, ns, ls, k, prec, _stream_ptr(stream), out))
    return [Index(out[j], Rs[j], int(leaves[j]), prec) for j in range(k)]


def rmi_free(index: Index):
    h, index.handle = index.handle, None
    if h:
        load().rmi_free(h)


def rmi_stats(index: Index) -> dict:
    return index.stats()


def rmi_export(index: Index) -> dict:
    L = index.leaves
    root = np.zeros(2)
    lo = np.zeros(L + 1, dtype=np.uint64)
    ab = np.zeros((L, 2))
    err = np.zeros((L, 2), dtype=np.int64)
    _check(load().rmi_export(index.handle, _ptr(root), _ptr(lo), _ptr(ab), _ptr(err)))
    return {"root": root, "leaf_lo": lo, "leaf_ab": ab, "err": err}


def grmi_build(index: Index, gaps: int = 4, stream=None) -> dict:
    """Attach the gapped arrays of a GRMI (Section 3.A) to the index; joins on
    it then use the exponential search from the predicted slot.  Returns the
    statistics of the arrays."""
    _check(load().grmi_build(index.handle, gaps, _stream_ptr(stream)))
    return grmi_stats(index)


def lhash_build(index: Index, spk: int = 4, stream=None) -> dict:
    """Attach a learned hash index (Section 3.C: the RMI as an order-preserving
    hash into 4-slot buckets, one entry per distinct key, spk slots per
    distinct key); joins on the index then hash each probe.  Returns the
    table's statistics."""
    _check(load().lhash_build(index.handle, spk, _stream_ptr(stream)))
    return grmi_stats(index)


def lhash_export_first(index: Index) -> np.ndarray:
    """first[D + 1]: position in R of each distinct key's first copy."""
    D = grmi_stats(index)["distinct"]
    first = np.zeros(D + 1, dtype=np.uint32)
    _check(load().lhash_export_first(index.handle, _ptr(first)))
    return first


def lhash_build_rs(index: Index, spk: int = 4, eps: int = 16, radix_bits: int = 18,
                   stream=None) -> dict:
    """Attach a learned hash index whose hash is a RadixSpline (Section 2.D)
    over R's distinct keys (the paper's RSHASH-INLJ, Section 3.C); joins on
    the index then hash each probe through the spline.  Returns the table's
    statistics."""
    _check(load().lhash_build_rs(index.handle, spk, eps, radix_bits, _stream_ptr(stream)))
    return grmi_stats(index)


def rs_export(index: Index) -> dict:
    """The RadixSpline of an lhash_build_rs index: spline keys and positions,
    radix table and prefix shift."""
    count, shift = ctypes.c_uint64(), ctypes.c_uint32()
    _check(load().rs_export(index.handle, None, None, None, ctypes.byref(shift),
                            ctypes.byref(count)))
    sx = np.zeros(count.value, dtype=np.uint64)
    sy = np.zeros(count.value, dtype=np.uint32)
    _check(load().rs_export(index.handle, _ptr(sx), _ptr(sy), None, None, None))
    return {"sx": sx, "sy": sy, "shift": shift.value, "count": count.value}


def rs_export_table(index: Index, radix_bits: int) -> np.ndarray:
    """The radix table (2^radix_bits + 1 entries) of an lhash_build_rs index."""
    table = np.zeros((1 << radix_bits) + 1, dtype=np.uint32)
    _check(load().rs_export(index.handle, None, None, _ptr(table), None, None))
    return table


def lsj_join(R, S, pairs, stream=None) -> int:
    """Learned sort-merge join (Section 4) of two unsorted device tensors of
    uint64 keys into `pairs` (int32 tensor (cap, 2)); returns |J|."""
    _require_cuda_u64(R, "R")
    _require_cuda_u64(S, "S")
    total = ctypes.c_uint64()
    cap = pairs.shape[0] if pairs is not None else 0
    _check(load().lsj_join(_ptr(R), R.numel(), _ptr(S), S.numel(), _ptr(pairs), cap,
                           ctypes.byref(total), _stream_ptr(stream)))
    return total.value


LOOKUPS = ("rmi", "rmi_bucketed", "grmi", "lhash", "rmi_sortmerge", "rshash", "rmi_levels")


def index_autotune(index: Index, S_sample, stream=None) -> tuple[str, dict]:
    """Time the seven lookup structures on a probe sample and keep the fastest;
    returns its name and every candidate's ns per probe."""
    _require_cuda_u64(S_sample, "S_sample")
    choice = ctypes.c_int()
    ns = np.zeros(len(LOOKUPS))
    _check(load().index_autotune(index.handle, _ptr(S_sample), S_sample.numel(),
                                 _stream_ptr(stream), ctypes.byref(choice), _ptr(ns)))
    return LOOKUPS[choice.value], dict(zip(LOOKUPS, ns.tolist()))


def grmi_drop(index: Index):
    _check(load().grmi_drop(index.handle))


def grmi_stats(index: Index) -> dict:
    st = lj_grmi_stats()
    _check(load().grmi_stats(index.handle, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_}


def grmi_export(index: Index) -> tuple[np.ndarray, np.ndarray]:
    """The gapped key array (C uint64) and payload array (C + 1 uint32)."""
    C = grmi_stats(index)["slots"]
    keys = np.zeros(C, dtype=np.uint64)
    pos = np.zeros(C + 1, dtype=np.uint32)
    _check(load().grmi_export(index.handle, _ptr(keys), _ptr(pos)))
    return keys, pos


def join_count(index: Index, S, counts=None, offsets=None, want_total: bool = True,
               stream=None) -> int | None:
    """Match counts (uint32 tensor, optional) and offsets (m+1 int64 tensor,
    optional) of every probe of S; returns |J| when want_total (synchronises)."""
    _require_cuda_u64(S, "S")
    total = ctypes.c_uint64()
    _check(load().join_count(index.handle, _ptr(S), S.numel(), _ptr(counts), _ptr(offsets),
                             ctypes.byref(total) if want_total else None,
                             _stream_ptr(stream)))
    return total.value if want_total else None


def join_count_noalloc(index: Index, S, counts=None, offsets=None, want_total: bool = True,
                       stream=None) -> int | None:
    """join_count without any allocation (fixed scratch in the library; at
    most 2^25 probes per call; calls that overlap on the GPU race)."""
    _require_cuda_u64(S, "S")
    total = ctypes.c_uint64()
    _check(load().join_count_noalloc(index.handle, _ptr(S), S.numel(), _ptr(counts),
                                     _ptr(offsets), ctypes.byref(total) if want_total else None,
                                     _stream_ptr(stream)))
    return total.value if want_total else None


def join_emit(index: Index, S, pairs, offsets=None, written=None, want_total: bool = True,
              stream=None) -> int | None:
    """Write the join pairs into `pairs` (int32 tensor of shape (cap, 2)).
    offsets=None selects the single-pass path (R unique).  `written` is an
    optional 1-element 64-bit device tensor receiving |J| without a sync."""
    _require_cuda_u64(S, "S")
    cap = pairs.shape[0] if pairs is not None else 0
    total = ctypes.c_uint64()
    _check(load().join_emit(index.handle, _ptr(S), S.numel(), _ptr(offsets), _ptr(pairs), cap,
                            _ptr(written), ctypes.byref(total) if want_total else None,
                            _stream_ptr(stream)))
    return total.value if want_total else None


def join_locate(index: Index, S, first, counts=None, offsets=None, want_total: bool = True,
                stream=None) -> int | None:
    """join_count that also writes each probe's first match position into
    `first` (uint32/int32 tensor of m); returns |J| when want_total."""
    _require_cuda_u64(S, "S")
    total = ctypes.c_uint64()
    _check(load().join_locate(index.handle, _ptr(S), S.numel(), _ptr(first), _ptr(counts),
                              _ptr(offsets), ctypes.byref(total) if want_total else None,
                              _stream_ptr(stream)))
    return total.value if want_total else None


def join_expand(first, offsets, pairs, written=None, want_total: bool = True,
                stream=None) -> int | None:
    """Pairs of the ranges located by join_locate (no index, no S needed)."""
    m = offsets.numel() - 1
    cap = pairs.shape[0] if pairs is not None else 0
    total = ctypes.c_uint64()
    _check(load().join_expand(_ptr(first), _ptr(offsets), m, _ptr(pairs), cap, _ptr(written),
                              ctypes.byref(total) if want_total else None, _stream_ptr(stream)))
    return total.value if want_total else None


def join_host(index: Index, S_host: np.ndarray, pairs_host: np.ndarray, stream=None) -> int:
    """The whole join from host arrays (S uint64; pairs (cap, 2) uint32)."""
    assert S_host.dtype == np.uint64 and S_host.flags.c_contiguous
    assert pairs_host.dtype == np.uint32 and pairs_host.flags.c_contiguous
    total = ctypes.c_uint64()
    _check(load().join_host(index.handle, _ptr(S_host), S_host.size, _ptr(pairs_host),
                            pairs_host.shape[0], ctypes.byref(total), _stream_ptr(stream)))
    return total.value


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = _ptr(t)
    return arr


class BatchPlan:
    """A plan of k joins (unique-R indexes of one precision) that run together:
    one persistent search launch, one scan, one compaction per run."""

    def __init__(self, indexes, S_list, pairs_list, stream=None):
        k = len(indexes)
        assert k == len(S_list) == len(pairs_list) and k > 0
        for S in S_list:
            _require_cuda_u64(S, "S")
        self._keep = (list(indexes), list(S_list), list(pairs_list))
        m = (ctypes.c_uint64 * k)(*[S.numel() for S in S_list])
        cap = (ctypes.c_uint64 * k)(*[p.shape[0] for p in pairs_list])
        out = ctypes.c_void_p()
        _check(load().join_batch_plan((ctypes.c_void_p * k)(*[ix.handle for ix in indexes]),
                                      _ptr_array(S_list), m, k, _ptr_array(pairs_list), cap,
                                      _stream_ptr(stream), ctypes.byref(out)))
        self.handle = out.value
        self.k = k

    def run(self, want_totals: bool = True, written=None, stream=None):
        tot = (ctypes.c_uint64 * self.k)()
        _check(load().join_batch_run(self.handle, _ptr(written),
                                     tot if want_totals else None, _stream_ptr(stream)))
        return list(tot) if want_totals else None

    def capture(self, stream):
        _check(load().join_batch_capture(self.handle, _stream_ptr(stream)))

    def set_shape(self, block: int, tiles_per_item: int):
        _check(load().join_batch_set_shape(self.handle, int(block), int(tiles_per_item)))

    def autotune(self, stream=None) -> tuple[int, int]:
        """Pick the fastest work-item shape by timing one run of each."""
        bb, bt = ctypes.c_int(), ctypes.c_int()
        _check(load().join_batch_autotune(self.handle, _stream_ptr(stream), ctypes.byref(bb),
                                          ctypes.byref(bt)))
        return bb.value, bt.value

    def free(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.join_batch_free(h)

    def __del__(self):
        self.free()


def join_batch_plan(indexes, S_list, pairs_list, stream=None) -> BatchPlan:
    return BatchPlan(indexes, S_list, pairs_list, stream)


def join_batch(indexes, S_list, pairs_list, stream=None) -> list:
    """Plan + run + free: each join's |J| (pairs written into pairs_list[j])."""
    k = len(indexes)
    for S in S_list:
        _require_cuda_u64(S, "S")
    m = (ctypes.c_uint64 * k)(*[S.numel() for S in S_list])
    cap = (ctypes.c_uint64 * k)(*[p.shape[0] for p in pairs_list])
    tot = (ctypes.c_uint64 * k)()
    _check(load().join_batch((ctypes.c_void_p * k)(*[ix.handle for ix in indexes]),
                             _ptr_array(S_list), m, k, _ptr_array(pairs_list), cap, tot,
                             _stream_ptr(stream)))
    return list(tot)


def rmi_autotune(R, S_sample, precision: str | int = "fp32", stream=None) -> tuple[int, float]:
    """Leaf count with the least probe time per key on S_sample (cached)."""
    _require_cuda_u64(R, "R")
    _require_cuda_u64(S_sample, "S_sample")
    prec = {"fp32": LJ_FP32, "fp64": LJ_FP64}.get(precision, precision)
    L = ctypes.c_uint32()
    ns = ctypes.c_double()
    _check(load().rmi_autotune(_ptr(R), R.numel(), _ptr(S_sample), S_sample.numel(), prec,
                               _stream_ptr(stream), ctypes.byref(L), ctypes.byref(ns)))
    return L.value, ns.value


def rmi_autotune_clear():
    load().rmi_autotune_clear()


class Server:
    """Continuous-batching join server over resident learned indexes."""

    def __init__(self, hbm_budget_bytes: int = 150 << 30, streams: int = 4,
                 max_batch: int = 1024):
        cfg = lj_server_cfg(hbm_budget_bytes, streams, max_batch)
        out = ctypes.c_void_p()
        _check(load().join_server_create(ctypes.byref(cfg), ctypes.byref(out)))
        self.handle = out.value
        self._keep = {}          # ticket -> S (must stay alive until the request is done)
        self._rels = []

    def add_relation(self, index: Index) -> int:
        rid = ctypes.c_uint32()
        _check(load().join_server_add_relation(self.handle, index.handle, ctypes.byref(rid)))
        self._rels.append(index)
        return rid.value

    def submit(self, rel: int, S) -> int:
        t = ctypes.c_uint64()
        _check(load().join_submit(self.handle, rel, _ptr(S), S.numel() if hasattr(S, "numel")
                                  else S.size, ctypes.byref(t)))
        self._keep[t.value] = S
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        r = lj_result()
        _check(load().join_wait(self.handle, ticket, timeout_us, ctypes.byref(r)))
        return {"status": r.status, "pairs": r.pairs, "latency_us": r.latency_us,
                "queue_us": r.queue_us}

    def fetch(self, ticket: int, out, stream=None):
        _check(load().join_fetch(self.handle, ticket, _ptr(out), out.shape[0],
                                 _stream_ptr(stream)))

    def release(self, ticket: int):
        _check(load().join_release(self.handle, ticket))
        self._keep.pop(ticket, None)

    def stats(self, reset: bool = False) -> dict:
        st = lj_server_stats()
        _check(load().join_server_stats(self.handle, ctypes.byref(st), int(reset)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.join_server_destroy(h)
        self._keep = {}

    def __del__(self):
        self.close()


def lj_set_option(name: str, value: int):
    _check(load().lj_set_option(name.encode(), int(value)))


def lj_get_option(name: str) -> int:
    v = load().lj_get_option(name.encode())
    if v == -1:
        raise LJoinError(-1, lj_last_error())
    return v


def lj_profile_report() -> dict:
    """Per-kernel timings recorded with the "profile" option on (and clear them)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    n = load().lj_profile_report(buf, len(buf))
    if n < 0:
        raise LJoinError(n, lj_last_error())
    return json.loads(buf.value.decode())


def lj_last_error() -> str:
    return load().lj_last_error().decode(errors="replace")


def lj_version() -> str:
    return load().lj_version().decode()
