"""Serving with continuous batching: each request's result is exactly what
join_emit gives for it alone (and what the oracle gives), whatever else is in
flight; admission respects the HBM budget; waits time out cleanly."""
import threading
import time

import numpy as np
import pytest

import oracle
from datagen import device as dg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


def _relations(lj, k=4, seed=8):
    joins = dg.batched_workload(k=k, seed=seed, device="cuda", scale=1 / 8)
    rels = [j["R"] for j in joins]
    idx = [lj.rmi_build(R, max(1, R.numel() // 64), "fp32") for R in rels]
    return rels, idx


def _request(R, m, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    hits = R[torch.randint(0, R.numel(), (m,), device="cuda", generator=g)]
    miss = torch.randint(0, 2**62, (m,), device="cuda", generator=g)
    coin = torch.rand(m, device="cuda", generator=g) < 0.7
    return torch.where(coin, hits, miss).contiguous()


def _alone(lj, idx, S):
    p = torch.empty((max(S.numel(), 1), 2), dtype=torch.int32, device="cuda")
    t = lj.join_emit(idx, S, p)
    return p[:t].cpu()


def test_results_alone_equal_results_in_the_mix():
    lj = _lj()
    rels, idx = _relations(lj)
    srv = lj.Server(hbm_budget_bytes=8 << 30, streams=4, max_batch=64)
    try:
        rids = [srv.add_relation(ix) for ix in idx]
        rng = np.random.default_rng(9)
        reqs = []
        for q in range(160):
            r = int(rng.integers(0, len(rels)))
            m = int(np.exp(rng.uniform(np.log(1000), np.log(200_000))))
            reqs.append((r, _request(rels[r], m, 100 + q)))
        torch.cuda.synchronize()
        # submit from two threads with jitter, so batches form and overlap
        tickets = [None] * len(reqs)

        def client(part):
            for q in part:
                tickets[q] = srv.submit(rids[reqs[q][0]], reqs[q][1])
                time.sleep(float(rng.uniform(0, 2e-4)))

        th = [threading.Thread(target=client, args=(list(range(i, len(reqs), 2)),)) for i in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for q, (r, S) in enumerate(reqs):
            res = srv.wait(tickets[q], timeout_us=30_000_000)
            assert res["status"] == 0
            out = torch.empty((max(res["pairs"], 1), 2), dtype=torch.int32, device="cuda")
            srv.fetch(tickets[q], out)
            torch.cuda.synchronize()
            got = out[: res["pairs"]].cpu()
            assert torch.equal(got, _alone(lj, idx[r], S))
            if q % 20 == 0:   # and the oracle, on a few
                want = oracle.join_pairs(rels[r].cpu().numpy().view(np.uint64),
                                         S.cpu().numpy().view(np.uint64))
                assert np.array_equal(got.numpy().view(np.uint32), want)
            srv.release(tickets[q])
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["batches"] >= 1
        assert st["p99_us"] >= st["p50_us"] > 0
        # only the registered relations stay charged once every request is released
        assert st["mem_in_use"] == st["resident"] == sum(
            R.numel() * 8 + ix.leaves * 32 for R, ix in zip(rels, idx))
    finally:
        srv.close()


def test_budget_admission_rejection_and_timeout():
    lj = _lj()
    rels, idx = _relations(lj, k=1, seed=10)
    resident = rels[0].numel() * 8 + idx[0].leaves * 32   # keys + fp32 leaf records
    # a relation larger than the budget is refused
    small = lj.Server(hbm_budget_bytes=resident - 1, streams=1, max_batch=8)
    try:
        with pytest.raises(lj.LJoinError) as e:
            small.add_relation(idx[0])
        assert e.value.code == -7                           # LJ_E_BUDGET
    finally:
        small.close()
    # room for the relation and one 300k-probe request at a time
    budget = resident + 12 * 300_000 + 4096
    srv = lj.Server(hbm_budget_bytes=budget, streams=2, max_batch=8)
    try:
        rid = srv.add_relation(idx[0])
        assert srv.stats()["resident"] == resident
        with pytest.raises(lj.LJoinError) as e:
            srv.submit(rid, _request(rels[0], 400_000, 1))
        assert e.value.code == -7                           # LJ_E_BUDGET
        a = _request(rels[0], 300_000, 2)
        b = _request(rels[0], 300_000, 3)
        ta, tb = srv.submit(rid, a), srv.submit(rid, b)
        assert srv.wait(ta, timeout_us=30_000_000)["status"] == 0
        # b cannot be admitted while a holds the budget (a is not released yet)
        with pytest.raises(lj.LJoinError) as e:
            srv.wait(tb, timeout_us=2000)
        assert e.value.code == -6                           # LJ_E_TIMEOUT
        srv.release(ta)
        res = srv.wait(tb, timeout_us=30_000_000)
        out = torch.empty((max(res["pairs"], 1), 2), dtype=torch.int32, device="cuda")
        srv.fetch(tb, out)
        torch.cuda.synchronize()
        assert torch.equal(out[: res["pairs"]].cpu(), _alone(lj, idx[0], b))
        srv.release(tb)
        st = srv.stats()
        assert st["rejected"] == 1 and st["completed"] == 2 and st["mem_peak"] <= budget
    finally:
        srv.close()


def test_gapped_and_hash_relations_are_served_alone_and_exactly():
    """Relations with a gapped RMI, a learned hash (RMI or RadixSpline as the
    hash) and none, served together: requests to the first three run alone
    with join_emit's kernels, the others in batches; every result equals
    join_emit's for the request alone and the oracle's, and the arrays are
    charged to the budget while the relations are registered."""
    lj = _lj()
    rels, idx = _relations(lj, k=4, seed=19)
    lj.grmi_build(idx[0], 4)
    lj.lhash_build(idx[1], 4)
    lj.lhash_build_rs(idx[2], 4, 16, 18)
    srv = lj.Server(hbm_budget_bytes=8 << 30, streams=3, max_batch=32)
    try:
        rids = [srv.add_relation(ix) for ix in idx]
        plain = rels[3].numel() * 8 + idx[3].leaves * 32
        st = srv.stats()
        # the gapped and hash arrays are part of the resident bytes
        assert st["resident"] > sum(R.numel() * 8 + ix.leaves * 32 for R, ix in zip(rels, idx))
        assert st["resident"] > plain
        rng = np.random.default_rng(23)
        reqs = []
        for q in range(64):
            r = int(rng.integers(0, len(rels)))
            m = int(np.exp(rng.uniform(np.log(500), np.log(100_000))))
            reqs.append((r, _request(rels[r], m, 700 + q)))
        torch.cuda.synchronize()
        tickets = [srv.submit(rids[r], S) for r, S in reqs]
        for q, (r, S) in enumerate(reqs):
            res = srv.wait(tickets[q], timeout_us=30_000_000)
            assert res["status"] == 0
            out = torch.empty((max(res["pairs"], 1), 2), dtype=torch.int32, device="cuda")
            srv.fetch(tickets[q], out)
            torch.cuda.synchronize()
            got = out[: res["pairs"]].cpu()
            assert torch.equal(got, _alone(lj, idx[r], S))
            want = oracle.join_pairs(rels[r].cpu().numpy().view(np.uint64),
                                     S.cpu().numpy().view(np.uint64))
            assert np.array_equal(got.numpy().view(np.uint32), want)
            srv.release(tickets[q])
        st = srv.stats()
        assert st["completed"] == len(reqs)
        assert st["mem_in_use"] == st["resident"]
    finally:
        srv.close()
