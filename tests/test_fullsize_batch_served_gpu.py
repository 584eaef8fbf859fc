"""Full-size parity of the batched and the served workloads, built exactly as
bench.py builds them (device generator, leaf count per relation from
rmi_autotune, single-precision models), compared with the oracle (the CPU
sort-merge join) on every host core.

  batched_4096   all 4096 joins of one plan (tuned work-item shape), launched
                 directly and replayed from a CUDA graph: every join's |J| and
                 every one of its pairs equal the oracle's for that join
                 alone (about 7.5e9 probes in all).
  served_64      the 64 resident relations (2^20 .. 2^26 keys) and a mix of
                 256 requests (2^10 .. 2^23 keys, 70% hits) submitted at once
                 to a server with the 150 GB budget and 4 slots: each
                 request's pairs equal join_emit's for it alone and the
                 oracle's.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from datagen import device as dg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _want_pairs(R, S):
    """The oracle's pairs of a join on a unique R: (lo_j, j) for every hit."""
    lo, hi, total = oracle.join_ranges(R, S)
    hit = hi > lo
    return np.stack([lo[hit].astype(np.uint32), np.flatnonzero(hit).astype(np.uint32)], axis=1)


def test_batched_4096_full_parity():
    lj = _lj()
    joins = dg.batched_workload(k=4096, seed=0, device="cuda")
    lj.rmi_autotune_clear()
    idx = []
    for j in joins:
        L, _ = lj.rmi_autotune(j["R"], j["S"][: 1 << 16])
        idx.append(lj.rmi_build(j["R"], L, "fp32"))
    pairs = [torch.empty((max(j["m"], 1), 2), dtype=torch.int32, device="cuda") for j in joins]
    plan = lj.join_batch_plan(idx, [j["S"] for j in joins], pairs)
    plan.autotune()
    for p in pairs:
        p.fill_(-1)
    totals = plan.run()
    stream = torch.cuda.Stream()
    plan.capture(stream)
    replay = plan.run(stream=stream)
    torch.cuda.synchronize()
    assert replay == totals

    def check(i):
        R, S = _u64(joins[i]["R"]), _u64(joins[i]["S"])
        want = _want_pairs(R, S)
        got = pairs[i][: totals[i]].cpu().numpy().view(np.uint32)
        return i, totals[i] == want.shape[0] and np.array_equal(got, want)

    with ThreadPoolExecutor(max_workers=oracle.host_threads()) as ex:
        bad = [i for i, ok in ex.map(check, range(len(joins))) if not ok]
    assert not bad, f"joins differing from the oracle: {bad[:20]}"


def test_served_64_full_mix_parity():
    lj = _lj()
    rels = dg.batched_workload(k=64, seed=77, device="cuda", n_range=(1 << 20, 1 << 26),
                               m_range=(2, 4))
    lj.rmi_autotune_clear()
    idx = []
    for j in rels:
        R = j["R"]
        L, _ = lj.rmi_autotune(R, R[torch.randint(0, R.numel(), (1 << 16,), device="cuda")])
        idx.append(lj.rmi_build(R, L, "fp32"))
    rng = np.random.default_rng(5)
    reqs = []
    for q in range(256):
        r = int(rng.integers(0, len(rels)))
        m = int(np.exp(rng.uniform(np.log(1 << 10), np.log(1 << 23))))
        R = rels[r]["R"]
        g = torch.Generator(device="cuda").manual_seed(1000 + q)
        hits = R[torch.randint(0, R.numel(), (m,), device="cuda", generator=g)]
        miss = torch.randint(0, 2**62, (m,), device="cuda", generator=g)
        coin = torch.rand(m, device="cuda", generator=g) < 0.7
        reqs.append((r, torch.where(coin, hits, miss).contiguous()))
    torch.cuda.synchronize()
    srv = lj.Server(hbm_budget_bytes=150 << 30, streams=4, max_batch=256)
    results = []
    try:
        rids = [srv.add_relation(ix) for ix in idx]
        tickets = [srv.submit(rids[r], S) for r, S in reqs]
        for t, (r, S) in zip(tickets, reqs):
            res = srv.wait(t, timeout_us=120_000_000)
            assert res["status"] == 0
            out = torch.empty((max(res["pairs"], 1), 2), dtype=torch.int32, device="cuda")
            srv.fetch(t, out)
            torch.cuda.synchronize()
            srv.release(t)
            got = out[: res["pairs"]]
            alone = torch.empty((max(S.numel(), 1), 2), dtype=torch.int32, device="cuda")
            n_alone = lj.join_emit(idx[r], S, alone)
            assert n_alone == res["pairs"] and torch.equal(got, alone[:n_alone])
            results.append(got.cpu().numpy().view(np.uint32))
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["rejected"] == 0
    finally:
        srv.close()
    host_R = {r: _u64(rels[r]["R"]) for r in {r for r, _ in reqs}}

    def check(q):
        r, S = reqs[q]
        return q, np.array_equal(results[q], _want_pairs(host_R[r], _u64(S)))

    with ThreadPoolExecutor(max_workers=oracle.host_threads()) as ex:
        bad = [q for q, ok in ex.map(check, range(len(reqs))) if not ok]
    assert not bad, f"requests differing from the oracle: {bad[:20]}"
