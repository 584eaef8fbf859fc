#!/usr/bin/env python3
"""Benchmark of the learned indexed nested loop join (RMI-INLJ) on GB300.

One step = one pass of the probe path over the whole outer relation S with
the learned index of R resident on the device (the index is built before
the timed region, as the paper measures joins: Section 3.A / 6.A); the
build is timed separately and reported as build_ms.

Default workload (lognormal_100m): R = 100M unique keys
round(1e9 * LogNormal(0, 2)), sorted; S = 400M keys, half Zipf(0.99) hits
over R's ranks, half true misses uniform in [min R, max R]; two-level
linear RMI with 2^20 leaves, single-precision model evaluation.

--index grmi probes through a gapped RMI (Section 3.A) built on the same
RMI (--gaps per key) instead of the bounded search in R.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
(sort-merge join) on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import datagen  # noqa: E402

WORKLOADS = {
    "lognormal_100m": dict(fn=datagen.lognormal_100m, kw={}),
    "uniform_1m": dict(fn=datagen.uniform_1m, kw={}),
    "dup_seqh_50m": dict(fn=datagen.dup_seqh_50m, kw={}),
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.path = gpu_index, None, None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="lj_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("LJ_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def reduce_max(value: float, dist, device) -> float:
    """Max of a per-rank value over all ranks (the slowest rank's time)."""
    if not dist:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, units_per_rank: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in the step."""
    return world * units_per_rank / (ms_per_step / 1e3)


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def run_reference(args, rank, world):
    """CPU oracle (sort-merge) on bounded samples of the same workload, on
    every host core (chunks of S on parallel threads)."""
    import oracle
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    wl = w["fn"](seed=args.seed, **_overrides(args))
    m_s = min(wl.S.size, args.ref_sample)
    oracle.build()
    cores = oracle.host_threads()
    times = []
    for step in range(args.warmup + args.steps):
        off = (step * m_s) % max(1, wl.S.size - m_s + 1)
        S = wl.S[off:off + m_s]
        t0 = time.perf_counter()
        oracle.join_ranges_mt(wl.R, S, threads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = m_s * args.steps / t
    line = {
        "impl": "reference", "metric": "probe_keys_per_s", "value": value, "unit": "keys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": _config(args, wl),
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": cores, "kind": "oracle",
                         "cpu": _cpu_model(),
                         "sample": f"{m_s} probes of S per step against the full R, "
                                   f"{cores} threads"},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _overrides(args) -> dict:
    kw = dict(WORKLOADS[args.workload]["kw"])
    if args.n is not None:
        kw["rows" if args.workload == "dup_seqh_50m" else "n"] = args.n
    if args.m is not None:
        kw["m"] = args.m
    if args.leaves is not None:
        kw["leaves"] = args.leaves
    if args.workload == "dup_seqh_50m":
        kw["reading"] = args.dup_reading
    return kw


L2_FLUSH_BYTES = 512 << 20          # written between steps when the inputs fit in L2


def _small(wl) -> bool:
    """Inputs below twice the L2 (126 MB) get an L2 flush before every timed
    step; larger ones evict themselves."""
    return wl.S.nbytes + wl.R.nbytes < (256 << 20)


def _config(args, wl):
    l2 = ("L2 flushed before every step (%d MB written, outside the timed events)"
          % (L2_FLUSH_BYTES >> 20) if _small(wl) else "inputs larger than L2")
    return {"workload": wl.name, "n": int(wl.R.size), "m": int(wl.S.size),
            "leaves": int(wl.leaves), "precision": wl.precision, "seed": args.seed,
            "index": {"rmi": "rmi", "grmi": f"grmi, {args.gaps} gaps per key",
                      "lhash": f"learned hash, {args.gaps} slots per distinct key",
                      "rshash": f"RadixSpline hash (eps {args.rs_eps}, {args.rs_bits} radix "
                                f"bits), {args.gaps} slots per distinct key",
                      "auto": "chosen by index_autotune"}[args.index],
            "probe_order": ["as given", "bucketed", "learned sort-merge"][args.probe_buckets],
            "l2": l2 + " (S = %.3f GB, R = %.3f GB)" % (wl.S.nbytes / 1e9, wl.R.nbytes / 1e9)}


KERNEL_SOURCES = ("device_common.cuh", "probe_core.cuh", "probe.cu")


def _ncu_traffic(kernel: str, args) -> float | None:
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources for this workload (the default
    lognormal_100m sizes), else None."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if (not os.path.exists(p) or args.workload != "lognormal_100m"
            or any(v is not None for v in (args.n, args.m, args.leaves))):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2111_08824_gb300", "csrc")
    for name in KERNEL_SOURCES:           # the files the probe kernels are built from
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    if d.get("csrc_sha256") != h.hexdigest():
        return None
    return d.get("kernels", {}).get(kernel, {}).get("dram_bytes_per_launch")


def cpu_baseline(wl, sample: int, sample_1t: int) -> dict:
    """The oracle (sort-merge) as it stands, on every host core and on one
    thread, over bounded samples of S against the full R."""
    import oracle
    oracle.build()
    cores = oracle.host_threads()
    m_s = min(sample, wl.S.size)
    t0 = time.perf_counter()
    oracle.join_ranges_mt(wl.R, wl.S[:m_s], threads=cores)
    dt = time.perf_counter() - t0
    m1 = min(sample_1t, wl.S.size)
    t0 = time.perf_counter()
    oracle.join_ranges(wl.R, wl.S[:m1])
    dt1 = time.perf_counter() - t0
    return {"value": m_s / dt, "unit": "keys/s", "cores": cores, "kind": "oracle",
            "cpu": _cpu_model(),
            "sample": f"first {m_s} probes of S against the full R ({dt:.2f} s on {cores} threads)",
            "one_thread": {"value": m1 / dt1, "unit": "keys/s",
                           "sample": f"first {m1} probes of S ({dt1:.2f} s)"}}


def uniform_1m_record(reps: int = 200) -> dict:
    """The 1M x 1M uniform workload (L = 4096) as a latency case: the inputs
    fit in L2, so L2 is flushed before every rep and each rep is timed alone
    (CUDA events around the call on the launch stream; median of `reps`).
    Both model precisions; the default fused cooperative kernel, the
    search-compaction pipeline and the single-pass look-back kernel;
    roofline on the algorithmic bytes of the pass."""
    import torch

    import paper_2111_08824_gb300 as lj
    w = datagen.uniform_1m(seed=0)
    n, m, L = w.R.size, w.S.size, w.leaves
    Rd = torch.from_numpy(w.R.view(np.int64)).cuda()
    Sd = torch.from_numpy(w.S.view(np.int64)).cuda()
    pairs = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    written = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    peak, _ = _peaks()

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sorted(a.elapsed_time(b) for a, b in evs)

    out = {"workload": "uniform_1m", "n": n, "m": m, "leaves": L,
           "timing": f"L2 flushed ({L2_FLUSH_BYTES >> 20} MB written) before each rep, "
                     f"median of {reps} reps, CUDA events around the call"}
    empty = torch.zeros(1, device="cuda")
    out["event_floor_us"] = 1e3 * statistics.median(timed(lambda: empty.add_(1), reps))
    names = ("single_pass_max", "fused_max")
    old = [lj.lj_get_option(k) for k in names]
    for prec in ("fp64", "fp32"):
        idx = lj.rmi_build(Rd, L, prec)
        rec = 64 if prec == "fp64" else 32
        # fused: the default path (one cooperative kernel); pipeline: search,
        # compaction; single_pass: lookups + decoupled look-back in one kernel
        for name, spm, fmax in (("fused", 0, old[1]), ("pipeline", 0, 0),
                                ("single_pass", 1 << 40, 0)):
            lj.lj_set_option("single_pass_max", spm)
            lj.lj_set_option("fused_max", fmax)

            def step():
                lj.join_emit(idx, Sd, pairs, written=written, want_total=False)
            for _ in range(5):
                step()
            total = int(lj.join_emit(idx, Sd, pairs))
            ts = timed(step, reps)
            lj.lj_profile_report()
            lj.lj_set_option("profile", 1)
            timed(step, 20)
            lj.lj_set_option("profile", 0)
            kern = lj.lj_profile_report()
            med = statistics.median(ts)
            alg = 8 * m + 8 * n + 8 * total + rec * L
            out[f"{prec}_{name}"] = {
                "us_median": 1e3 * med, "us_min": 1e3 * ts[0],
                "probe_keys_per_s": m / (med / 1e3), "pairs": total,
                "roofline": {"bound": "hbm", "alg_bytes": alg,
                             "achieved": alg / (med / 1e3) / 1e9, "peak": peak,
                             "frac": alg / (med / 1e3) / 1e9 / peak, "unit": "GB/s"},
                "kernels_us": {k: 1e3 * v["total_ms"] / v["launches"] for k, v in kern.items()},
                "mean_window": idx.stats()["mean_window"]}
    for k, v in zip(names, old):
        lj.lj_set_option(k, v)
    del Rd, Sd, pairs, flush
    torch.cuda.empty_cache()
    return out


def run_lsj(args, rank, world, dist):
    """Learned sort-merge join (Section 4) of two unsorted relations: one step
    = the whole join (sampled models, partitioning and sorting of both
    relations, chunked merge-join, pairs written)."""
    import torch

    import paper_2111_08824_gb300 as lj
    n = args.n or 100_000_000
    m = args.m or 100_000_000
    wl = datagen.lsj_uniform_100m(seed=args.seed + 1000 * rank, n=n, m=m)
    Rd = torch.from_numpy(wl.R.view(np.int64)).cuda()
    Sd = torch.from_numpy(wl.S.view(np.int64)).cuda()
    total = wl.meta["expected_pairs"]
    pairs = torch.empty((max(total, 1), 2), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        assert lj.lsj_join(Rd, Sd, pairs) == total
    lj.lj_profile_report()
    lj.lj_set_option("profile", 1)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lj.lsj_join(Rd, Sd, pairs)
    e1.record(stream)
    torch.cuda.synchronize()
    lj.lj_set_option("profile", 0)
    kernels = lj.lj_profile_report()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), dist, "cuda") / args.steps
    peak, peak_kind = _peaks()
    # algorithmic bytes per launch (one launch per relation: the average of
    # R and S): the histogram reads a key and writes its partition; the
    # scatter reads both and writes (key, position); the sort reads and
    # writes each (key, position) once; the join passes read R's and S's
    # sorted (key, position) and the write pass writes the pairs
    half = (n + m) / 2
    alg = {"lsj_hist_kernel": 12 * half, "lsj_scatter_kernel": 24 * half,
           "lsj_sort_kernel": 24 * half, "lsj_join_count_kernel": 12 * (n + m),
           "lsj_join_write_kernel": 12 * (n + m) + 8 * total}
    dom = max((k for k in kernels if k in alg), key=lambda k: kernels[k]["total_ms"])
    dom_ms = kernels[dom]["total_ms"] / kernels[dom]["launches"]
    pass_bytes = 8 * (n + m) + 8 * total
    return {
        "metric": "join_tuples_per_s", "value": world * (n + m) / (ms / 1e3), "unit": "tuples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 keys", "data": "synthetic",
        "config": {"workload": "lsj_uniform_100m", "n": n, "m": m, "seed": args.seed,
                   "l2": "inputs larger than L2"},
        "pairs": total, "pairs_per_s": world * total / (ms / 1e3),
        "roofline": {"bound": "hbm", "kernel": dom, "alg_bytes_per_launch": alg[dom],
                     "launch_ms": dom_ms,
                     "achieved": alg[dom] / (dom_ms / 1e3) / 1e9, "peak": peak,
                     "frac": alg[dom] / (dom_ms / 1e3) / 1e9 / peak, "unit": "GB/s",
                     "peak_kind": peak_kind + " copy bandwidth (hbm_gbs)", "traffic": None},
        "roofline_pass": {"alg_bytes": pass_bytes,
                          "frac": pass_bytes / (ms / 1e3) / 1e9 / peak},
        "kernels": kernels, "gpu_launches": sum(k["launches"] for k in kernels.values()),
        "clocks": clk,
    }


def run_batched(args, rank, world, dist):
    """4096 uneven joins: per-join launches of the plain probe vs one batched
    plan run vs the same run replayed from a CUDA graph (same GPU, same data)."""
    import torch

    import paper_2111_08824_gb300 as lj
    from datagen import device as dg
    t0 = time.perf_counter()
    joins = dg.batched_workload(k=args.joins, seed=args.seed + 1000 * rank, device="cuda",
                                scale=args.scale)
    gen_s = time.perf_counter() - t0
    lj.rmi_autotune_clear()
    t0 = time.perf_counter()
    leaves = [lj.rmi_autotune(j["R"], j["S"][: 1 << 16])[0] for j in joins]
    tune_s = time.perf_counter() - t0
    # every relation's index in one segmented build; the same indexes built
    # one call each, for comparison (identical results, see the tests)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = lj.rmi_build_batch([j["R"] for j in joins], leaves, "fp32")
    build_batch_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    one_by_one = [lj.rmi_build(j["R"], L, "fp32") for j, L in zip(joins, leaves)]
    build_seq_s = time.perf_counter() - t0
    del one_by_one
    S_list = [j["S"] for j in joins]
    pairs = [torch.empty((max(j["m"], 1), 2), dtype=torch.int32, device="cuda") for j in joins]
    m_total = sum(j["m"] for j in joins)
    n_total = sum(j["n"] for j in joins)
    stream = torch.cuda.Stream()
    plan = lj.join_batch_plan(idx, S_list, pairs)
    with torch.cuda.stream(stream):
        shape = plan.autotune(stream=stream)
    totals = plan.run()
    pairs_total = sum(totals)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def per_join():
        for ix, S, p in zip(idx, S_list, pairs):
            lj.join_emit(ix, S, p, want_total=False, stream=stream)

    ms_per_join = timed(per_join, max(1, args.steps // 4))
    ms_batch = timed(lambda: plan.run(want_totals=False, stream=stream), args.steps)
    plan.capture(stream)
    lj.lj_profile_report()
    ms_graph = timed(lambda: plan.run(want_totals=False, stream=stream), args.steps)
    assert plan.run(stream=stream) == totals
    line = {
        "metric": "probe_keys_per_s", "value": world * m_total / (ms_graph / 1e3), "unit": "keys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 keys, f32 model", "data": "synthetic (generated on the device)",
        "config": {"workload": "batched_4096", "joins": len(joins), "sum_n": n_total,
                   "sum_m": m_total, "scale": args.scale, "seed": args.seed,
                   "leaves": "autotuned per R", "l2": "inputs larger than L2"},
        "pairs": pairs_total,
        "per_join_launches": {"ms_per_step": ms_per_join, "keys_per_s": m_total / (ms_per_join / 1e3)},
        "batched_run": {"ms_per_step": ms_batch, "keys_per_s": m_total / (ms_batch / 1e3)},
        "graph_replay": {"ms_per_step": ms_graph, "keys_per_s": m_total / (ms_graph / 1e3)},
        "speedup_vs_per_join": ms_per_join / ms_graph,
        "gen_s": gen_s, "leaf_count_tuning_s": tune_s,
        "index_build": {"batched_s": build_batch_s, "one_call_per_relation_s": build_seq_s,
                        "speedup": build_seq_s / build_batch_s},
        "leaves_chosen": sorted(set(leaves)), "sum_leaves": int(sum(leaves)),
        "tile_shape_chosen": {"block": shape[0], "tiles_per_item": shape[1]},
        "gpu_launches": 3 * args.steps,
    }
    del plan, pairs, idx, joins
    torch.cuda.empty_cache()
    return line


def run_served(args, rank, world, dist):
    """64 resident relations, Poisson arrivals; continuous-batching server vs
    a plain per-request probe fed by the same arrival times."""
    import queue
    import threading

    import torch

    import paper_2111_08824_gb300 as lj
    from datagen import device as dg
    t0 = time.perf_counter()
    rels = dg.batched_workload(k=64, seed=args.seed + 77, device="cuda",
                               n_range=(1 << 20, 1 << 26), m_range=(2, 4), scale=args.scale)
    lj.rmi_autotune_clear()
    idx = []
    for j in rels:
        R = j["R"]
        L, _ = lj.rmi_autotune(R, R[torch.randint(0, R.numel(), (1 << 16,), device="cuda")])
        idx.append(lj.rmi_build(R, L, "fp32"))
    # a pool of requests, replayed in order: relation uniform, m log-uniform
    # in [2^10, 2^23], 70% keys drawn from the relation, 30% fresh 62-bit keys
    rng = np.random.default_rng(args.seed + 5)
    pool = []
    for q in range(args.joins if args.joins != 4096 else 1024):
        r = int(rng.integers(0, len(rels)))
        m = int(np.exp(rng.uniform(np.log(1 << 10), np.log(1 << 23))) * args.scale) or 1
        R = rels[r]["R"]
        g = torch.Generator(device="cuda").manual_seed(args.seed * 1000 + q)
        hits = R[torch.randint(0, R.numel(), (m,), device="cuda", generator=g)]
        miss = torch.randint(0, 2**62, (m,), device="cuda", generator=g)
        coin = torch.rand(m, device="cuda", generator=g) < 0.7
        pool.append((r, torch.where(coin, hits, miss).contiguous()))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    n_req = int(args.rate * args.duration)
    gaps = rng.exponential(1.0 / args.rate, n_req)

    def serve(rate_gaps):
        srv = lj.Server(hbm_budget_bytes=150 << 30, streams=4, max_batch=256)
        rids = [srv.add_relation(ix) for ix in idx]
        tickets = queue.Queue()
        done_keys = [0]

        def waiter():
            while True:
                t = tickets.get()
                if t is None:
                    return
                res = srv.wait(t)
                done_keys[0] += res["pairs"]
                srv.release(t)

        th = threading.Thread(target=waiter)
        th.start()
        start = time.perf_counter()
        nxt = start
        for q, gap in enumerate(rate_gaps):
            nxt += gap
            dt = nxt - time.perf_counter()
            if dt > 0:
                time.sleep(dt)          # releases the GIL for the other thread
            r, S = pool[q % len(pool)]
            tickets.put(srv.submit(rids[r], S))
        tickets.put(None)
        th.join()
        st = srv.stats()
        srv.close()
        return st

    def plain(rate_gaps):
        """Each request alone with join_emit on one stream, in arrival order."""
        work = queue.Queue()
        lat = []
        keys = [0]
        bufs = {}

        def worker():
            while True:
                item = work.get()
                if item is None:
                    return
                t_arr, q = item
                r, S = pool[q % len(pool)]
                p = bufs.get(q % len(pool))
                if p is None:
                    p = bufs[q % len(pool)] = torch.empty((max(S.numel(), 1), 2),
                                                          dtype=torch.int32, device="cuda")
                lj.join_emit(idx[r], S, p)
                keys[0] += S.numel()
                lat.append((time.perf_counter() - t_arr) * 1e6)

        th = threading.Thread(target=worker)
        th.start()
        start = time.perf_counter()
        nxt = start
        for q, gap in enumerate(rate_gaps):
            nxt += gap
            dt = nxt - time.perf_counter()
            if dt > 0:
                time.sleep(dt)          # releases the GIL for the other thread
            work.put((time.perf_counter(), q))
        work.put(None)
        th.join()
        span = time.perf_counter() - start
        lat.sort()
        return {"p50_us": lat[len(lat) // 2], "p99_us": lat[int(0.99 * (len(lat) - 1))],
                "keys_per_s": keys[0] / span, "completed": len(lat)}

    # warm-up both paths on a few requests
    serve(gaps[:64])
    plain(gaps[:64])
    s_srv = serve(gaps)
    s_plain = plain(gaps)
    # saturation: all requests at once (closed batch), both paths
    burst = np.zeros(min(n_req, 4 * len(pool)))
    sat_srv = serve(burst)
    sat_plain = plain(burst)
    line = {
        "metric": "served_p99_latency_us", "value": s_srv["p99_us"], "unit": "us",
        "n_gpus": world, "steps": n_req, "warmup": 64, "ms_per_step": s_srv["mean_us"] / 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 keys, f32 model", "data": "synthetic (generated on the device)",
        "config": {"workload": "served_64", "relations": len(rels),
                   "sum_n": int(sum(j["n"] for j in rels)), "rate_per_s": args.rate,
                   "duration_s": args.duration, "requests": n_req, "pool": len(pool),
                   "hbm_budget_gb": 150, "streams": 4, "scale": args.scale},
        "server": {k: s_srv[k] for k in ("p50_us", "p99_us", "mean_us", "keys_per_s",
                                          "completed", "batches", "mean_batch", "mem_peak")},
        "plain_per_request": s_plain,
        "saturation": {"server": {k: sat_srv[k] for k in ("p50_us", "p99_us", "keys_per_s",
                                                           "mean_batch")},
                       "plain_per_request": sat_plain},
        "setup_s": setup_s,
    }
    del pool, idx, rels
    torch.cuda.empty_cache()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lognormal_100m",
                    choices=sorted(WORKLOADS) + ["batched_4096", "served_64", "lsj_uniform_100m"])
    ap.add_argument("--rate", type=float, default=2000.0, help="served workload: requests/s")
    ap.add_argument("--duration", type=float, default=5.0, help="served workload: seconds")
    ap.add_argument("--joins", type=int, default=4096, help="batched workload: number of joins")
    ap.add_argument("--scale", type=float, default=1.0, help="batched workload: size scale")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=1 << 27)
    ap.add_argument("--cpu-sample-1t", type=int, default=1 << 23)
    ap.add_argument("--ref-sample", type=int, default=1 << 25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="skip the uniform_1m, batched and served records of the default line")
    ap.add_argument("--n", type=int, default=None, help="override |R| (profiling runs)")
    ap.add_argument("--m", type=int, default=None, help="override |S| (profiling runs)")
    ap.add_argument("--leaves", type=int, default=None, help="override L (profiling runs)")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"],
                    help="override the workload's model precision")
    ap.add_argument("--index", default="rmi", choices=["rmi", "grmi", "lhash", "rshash", "auto"],
                    help="rmi: bounded search in R; grmi: gapped RMI (exponential search); "
                         "lhash: learned hash index; rshash: learned hash with a RadixSpline "
                         "as the hash; auto: index_autotune on 2^22 probes")
    ap.add_argument("--rs-eps", type=int, default=16, help="rshash: spline error bound")
    ap.add_argument("--rs-bits", type=int, default=18, help="rshash: radix table bits")
    ap.add_argument("--gaps", type=int, default=4,
                    help="grmi: gaps per key; lhash: slots per distinct key")
    ap.add_argument("--dup-reading", default="clip", choices=["clip", "truncate"],
                    help="dup_seqh_50m: Zipf(1.2) multiplicity clipped at 64, or truncated to 1..64")
    ap.add_argument("--probe-buckets", type=int, default=0, choices=[0, 1, 2],
                    help="1: probes looked up in bucketed order; 2: learned sort-merge order "
                         "(option probe_buckets)")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    rank, world, local, dist = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return

    import torch

    import paper_2111_08824_gb300 as lj
    torch.cuda.set_device(local)
    if args.workload in ("served_64", "batched_4096", "lsj_uniform_100m"):
        fn = {"served_64": run_served, "batched_4096": run_batched,
              "lsj_uniform_100m": run_lsj}[args.workload]
        line = fn(args, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    w = WORKLOADS[args.workload]
    # weak scaling: every rank probes its own S (seeded by rank) against the
    # replicated R; no collective on the data path.
    wl = w["fn"](seed=args.seed + 1000 * rank, **_overrides(args))
    if args.precision:
        wl.precision = args.precision
    n, m, L = wl.R.size, wl.S.size, wl.leaves

    Rd = torch.from_numpy(wl.R.view(np.int64)).cuda()
    Sd = torch.from_numpy(wl.S.view(np.int64)).cuda()
    idx = lj.rmi_build(Rd, L, wl.precision)
    st = idx.stats()
    unique = bool(st["unique"])
    # precision variants: windows re-measured under each model precision
    windows = {}
    other = None                                 # the index in the other precision
    for prec in ("fp32", "fp64"):
        if prec != wl.precision:
            other = lj.rmi_build(Rd, L, prec)
        s2 = st if prec == wl.precision else other.stats()
        windows[prec] = {"mean_window": s2["mean_window"], "max_window": s2["max_window"],
                         "build_ms": s2["build_ms"]}
    lj.lj_set_option("probe_buckets", args.probe_buckets)
    autotune = None
    if args.index == "auto":
        choice, ns = lj.index_autotune(idx, Sd[: min(m, 1 << 22)])
        autotune = {"choice": choice, "ns_per_probe": ns, "sample": min(m, 1 << 22)}
    grmi = (lj.grmi_build(idx, args.gaps) if args.index == "grmi"
            else lj.lhash_build(idx, args.gaps) if args.index == "lhash"
            else lj.lhash_build_rs(idx, args.gaps, args.rs_eps, args.rs_bits)
            if args.index == "rshash" else None)
    if autotune and autotune["choice"] in ("grmi", "lhash", "rshash"):
        grmi = lj.grmi_stats(idx)
    stream = torch.cuda.current_stream()

    if unique:
        pairs = torch.empty((m, 2), dtype=torch.int32, device="cuda")
        written = torch.zeros(1, dtype=torch.int64, device="cuda")

        def step():
            lj.join_emit(idx, Sd, pairs, written=written, want_total=False)
        launches_per_step = 1
    else:
        # duplicates: locate each probe's range of R (count pass), then expand
        # the ranges into pairs without searching again
        offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
        first = torch.empty(m, dtype=torch.int32, device="cuda")
        total0 = lj.join_locate(idx, Sd, first, offsets=offsets)
        pairs = torch.empty((max(total0, 1), 2), dtype=torch.int32, device="cuda")

        def step():
            lj.join_locate(idx, Sd, first, offsets=offsets, want_total=False)
            lj.join_expand(first, offsets, pairs, want_total=False)
        launches_per_step = 2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    total = lj.join_emit(idx, Sd, pairs) if unique else lj.join_count(idx, Sd)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)                              # let the sampler start before the timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    lj.lj_profile_report()                       # drop earlier records
    lj.lj_set_option("profile", 1)               # per-kernel events on the launch stream
    if _small(wl):
        # inputs fit in L2: flush it before each step, time the steps alone
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        local_ms = sum(a.elapsed_time(b) for a, b in evs)
    else:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            step()
        t_end.record(stream)
        torch.cuda.synchronize()
        local_ms = t_start.elapsed_time(t_end)
    lj.lj_set_option("profile", 0)
    kernels = lj.lj_profile_report()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = reduce_max(local_ms, dist, "cuda")
    ms_per_step = elapsed_ms / args.steps
    value = weak_value(world, m, ms_per_step)

    # ---- end to end through the C ABI with host buffers (pinned): S is read
    # in place by the GPU, pairs are copied out while the next chunk is probed
    S_host = torch.from_numpy(wl.S.view(np.int64)).pin_memory()
    P_host = torch.empty((max(total, 1), 2), dtype=torch.int32).pin_memory()
    S_np = S_host.numpy().view(np.uint64)
    P_np = P_host.numpy().view(np.uint32)
    e2e_s = None
    if args.e2e_steps > 0:
        for _ in range(2):
            lj.join_host(idx, S_np, P_np)      # warm-up (first touches of the pinned buffers)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            got = lj.join_host(idx, S_np, P_np)
            times.append(time.perf_counter() - t0)
            assert got == total
        e2e_s = statistics.median(times)

    # ---- roofline of the dominant kernel (algorithmic bytes per launch)
    peak, peak_kind = _peaks()
    alg = {
        # S, R once, leaves, 4-B result (+ 4-B first match when locating duplicates)
        "probe_search_kernel": 8 * m + 8 * n + 32 * L + 4 * m + (0 if unique else 4 * m),
        # the same join searched by descending R's key levels
        "levels_search_kernel": 8 * m + 8 * n + 32 * L + 4 * m + (0 if unique else 4 * m),
        # small unique batches: lookups and pairs in one kernel
        "probe_fused_kernel": 8 * m + 8 * n + 32 * L + 8 * total,
        "gapped_search_kernel": 8 * m + 8 * n + 32 * L + 4 * m,  # the same join, gapped index
        "hash_search_kernel": 8 * m + 8 * n + 32 * L + 4 * m + (0 if unique else 4 * m),
        "rs_hash_search_kernel": 8 * m + 8 * n + 4 * m + (0 if unique else 4 * m),
        "scan_kernel": 4 * m + (8 * total if unique else 8 * (m + 1)),
        "probe_single_pass_kernel": 8 * m + 8 * n + 32 * L + 8 * total,
        "emit_kernel": 8 * m + 8 * n + 32 * L + 8 * (m + 1) + 8 * total,
        "expand_kernel": 4 * m + 8 * (m + 1) + 8 * total,    # first, offsets, pairs
        # the join's bytes again, plus the bucketed copy of S written and read
        "bucketed_search_kernel": 8 * m + 8 * n + 32 * L + 4 * m + (0 if unique else 4 * m),
        "sortmerge_kernel": 8 * m + 8 * n + 32 * L + 4 * m + (0 if unique else 4 * m),
    }
    dom = max((k for k in kernels if k in alg), key=lambda k: kernels[k]["total_ms"])
    dom_ms = kernels[dom]["total_ms"] / kernels[dom]["launches"]
    achieved = alg[dom] / (dom_ms / 1e3) / 1e9
    pass_bytes = 8 * m + 8 * n + 8 * total + 32 * L
    traffic = _ncu_traffic(dom, args)
    line = {
        "metric": "probe_keys_per_s", "value": value, "unit": "keys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 keys, f32 model" if wl.precision == "fp32" else "u64 keys, f64 model",
        "data": "synthetic", "config": _config(args, wl),
        "pairs": int(total), "pairs_per_s": world * total / (ms_per_step / 1e3),
        "paper_metric_tuples_per_s": world * (n + m) / (ms_per_step / 1e3),
        "build_ms": st["build_ms"], "mean_window": st["mean_window"],
        "max_window": st["max_window"], "windows_by_precision": windows,
        "grmi": grmi,
        "index_autotune": autotune,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind + " copy bandwidth (hbm_gbs)",
                     "kernel": dom, "alg_bytes_per_launch": alg[dom],
                     "launch_ms": dom_ms},
        "roofline_pass": {"alg_bytes": pass_bytes, "achieved": pass_bytes / (ms_per_step / 1e3) / 1e9,
                          "frac": pass_bytes / (ms_per_step / 1e3) / 1e9 / peak},
        "kernels": kernels,
        "e2e": None if e2e_s is None else {
            "value": world * m / e2e_s, "unit": "keys/s", "h2d_bytes_per_step": 8 * m,
            "d2h_bytes_per_step": 8 * total,
            "note": "median of the timed join_host calls; S pinned on the host and read in "
                    "place over NVLink-C2C, pairs copied out"},
        "gpu_launches": sum(k["launches"] for k in kernels.values()),
        "clocks": clk,
    }
    # the same probe pass with the other model precision (same inputs, same
    # pipeline): FP32-model vs FP64-model probe
    if unique and args.index == "rmi" and other is not None:
        def step_other():
            lj.join_emit(other, Sd, pairs, written=written, want_total=False)
        for _ in range(args.warmup):
            step_other()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if _small(wl):
            flush.fill_(1)
        e0.record(stream)
        for _ in range(args.steps):
            step_other()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_o = e0.elapsed_time(e1) / args.steps
        assert int(lj.join_emit(other, Sd, pairs)) == total
        prec_o = "fp64" if wl.precision == "fp32" else "fp32"
        line[prec_o + "_model_probe"] = {
            "ms_per_step": ms_o, "value": world * m / (ms_o / 1e3), "unit": "keys/s",
            "roofline_pass": {"alg_bytes": pass_bytes,
                              "frac": pass_bytes / (ms_o / 1e3) / 1e9 / peak},
            "mean_window": windows[prec_o]["mean_window"],
            "max_window": windows[prec_o]["max_window"]}
    del other
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample, args.cpu_sample_1t)
    # the other workloads' records (one GPU): the 1M x 1M latency case, the
    # batched and the served workloads, each measured against its baseline
    if world == 1 and args.workload == "lognormal_100m" and not args.no_subrecords:
        del idx, pairs, Rd, Sd
        torch.cuda.empty_cache()
        sub = argparse.Namespace(**vars(args))
        sub.joins, sub.scale, sub.seed = 4096, 1.0, args.seed
        sub_lsj = argparse.Namespace(**vars(sub))
        sub_lsj.steps, sub_lsj.warmup, sub_lsj.n, sub_lsj.m = 5, 3, None, None
        line["configs"] = {"uniform_1m": uniform_1m_record(),
                           "batched_4096": run_batched(sub, rank, world, dist),
                           "served_64": run_served(sub, rank, world, dist),
                           "lsj_uniform_100m": run_lsj(sub_lsj, rank, world, dist)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
