"""Batched joins (one plan, three launches for all joins) against the oracle.

Every join of a batch must give exactly the pairs the oracle gives for that
join alone, whatever the tile shape, whether the run is launched directly or
replayed from a CUDA graph, and whatever leaf count the autotuner picks.
"""
import numpy as np
import pytest

import oracle
from datagen import device as dg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lj():
    import paper_2111_08824_gb300 as lj
    return lj


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _build(lj, joins, leaves_of=lambda n: max(1, n // 64)):
    return [lj.rmi_build(j["R"], leaves_of(j["R"].numel()), "fp32") for j in joins]


def _check_all(joins, pairs, totals):
    for j, p, t in zip(joins, pairs, totals):
        want = oracle.join_pairs(_u64(j["R"]), _u64(j["S"]))
        assert t == want.shape[0]
        got = p[:t].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)


def _workload(k=40, seed=3, scale=1 / 64):
    joins = dg.batched_workload(k=k, seed=seed, device="cuda", scale=scale)
    # edge cases: an empty S, a misaligned S (odd offset), a single probe
    joins[0]["S"] = joins[0]["S"][:0]
    s1 = joins[1]["S"]
    joins[1]["S"] = torch.cat([s1[:1], s1])[1:]
    joins[2]["S"] = joins[2]["S"][:1]
    return joins


def test_batch_matches_oracle_per_join():
    lj = _lj()
    joins = _workload()
    idx = _build(lj, joins)
    pairs = [torch.full((max(j["S"].numel(), 1), 2), -1, dtype=torch.int32, device="cuda")
             for j in joins]
    plan = lj.join_batch_plan(idx, [j["S"] for j in joins], pairs)
    totals = plan.run()
    _check_all(joins, pairs, totals)
    block, tiles = plan.autotune()
    assert block in (128, 256) and tiles in (1, 4, 8)
    # a further run on the same plan (tuned shape) gives the same result
    for p in pairs:
        p.fill_(-1)
    assert plan.run() == totals
    _check_all(joins, pairs, totals)


@pytest.mark.parametrize("block,tiles", [(128, 1), (128, 4), (128, 8), (256, 1), (256, 4),
                                         (256, 8)])
def test_batch_graph_replay_and_tile_shapes(block, tiles):
    lj = _lj()
    joins = _workload(k=24, seed=4)
    idx = _build(lj, joins)
    pairs = [torch.full((max(j["S"].numel(), 1), 2), -1, dtype=torch.int32, device="cuda")
             for j in joins]
    plan = lj.join_batch_plan(idx, [j["S"] for j in joins], pairs)
    plan.set_shape(block, tiles)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    plan.capture(stream)
    for _ in range(2):
        for p in pairs:
            p.fill_(-1)
        torch.cuda.synchronize()
        totals = plan.run(stream=stream)
        _check_all(joins, pairs, totals)


def test_batch_one_shot_and_capacity():
    lj = _lj()
    joins = _workload(k=10, seed=5)
    idx = _build(lj, joins)
    pairs = [torch.full((max(j["S"].numel(), 1), 2), -1, dtype=torch.int32, device="cuda")
             for j in joins]
    totals = lj.join_batch(idx, [j["S"] for j in joins], pairs)
    _check_all(joins, pairs, totals)
    # one join with too little room: reported, its first `capacity` pairs written
    big = max(range(len(joins)), key=lambda q: totals[q])
    small = [p if q != big else p[: totals[big] // 2] for q, p in enumerate(pairs)]
    with pytest.raises(lj.LJoinError) as e:
        lj.join_batch(idx, [j["S"] for j in joins], small)
    assert e.value.code == -5


def test_batch_rejects_duplicate_R_and_mixed_precision():
    lj = _lj()
    R = torch.tensor([1, 1, 2], dtype=torch.int64, device="cuda")
    S = torch.tensor([1, 2], dtype=torch.int64, device="cuda")
    p = torch.empty((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.join_batch([lj.rmi_build(R, 2)], [S], [p])
    assert e.value.code == -8
    Ru = torch.tensor([1, 2, 3], dtype=torch.int64, device="cuda")
    with pytest.raises(lj.LJoinError) as e:
        lj.join_batch([lj.rmi_build(Ru, 2, "fp32"), lj.rmi_build(Ru, 2, "fp64")], [S, S], [p, p])
    assert e.value.code == -1


def test_autotuner_choice_does_not_change_results():
    lj = _lj()
    lj.rmi_autotune_clear()
    joins = dg.batched_workload(k=6, seed=6, device="cuda", scale=1 / 16)
    for j in joins:
        R, S = j["R"], j["S"]
        lj.rmi_autotune_clear()
        L, ns = lj.rmi_autotune(R, S[: 1 << 15])
        assert L >= 256 and (L & (L - 1)) == 0 and ns > 0
        assert lj.rmi_autotune(R, S[: 1 << 15]) == (L, -1.0)     # cached
        want = oracle.join_pairs(_u64(R), _u64(S))
        for leaves in {L, 256, max(1, R.numel() // 8)}:
            idx = lj.rmi_build(R, leaves, "fp32")
            pairs = torch.empty((max(S.numel(), 1), 2), dtype=torch.int32, device="cuda")
            t = lj.join_emit(idx, S, pairs)
            assert np.array_equal(pairs[:t].cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_index_build_is_bit_identical(prec):
    """rmi_build_batch (one segmented pass over all relations) gives, for
    every relation, exactly the index rmi_build gives for it alone: root,
    leaf ranges, deployed parameters and error bounds; and each index also
    passes the oracle's checks (tests/_validate.py)."""
    from tests import _validate
    lj = _lj()
    joins = dg.batched_workload(k=24, seed=12, device="cuda", scale=1 / 32)
    Rs = [j["R"] for j in joins]
    Rs[3] = Rs[3][:0]                                   # an empty relation
    Rs[5] = Rs[5][:1]                                   # a single key
    Rs[7] = torch.sort(torch.cat([Rs[7], Rs[7][::3]]))[0]   # duplicates
    leaves = [max(1, R.numel() // 48) for R in Rs]
    leaves[0] = 1
    leaves[1] = 1 << 14                                 # far more leaves than keys
    batch = lj.rmi_build_batch(Rs, leaves, prec)
    for R, L, b in zip(Rs, leaves, batch):
        one = lj.rmi_build(R, L, prec)
        ea, eb = lj.rmi_export(one), lj.rmi_export(b)
        for key in ea:
            assert np.array_equal(ea[key], eb[key]), key
        sa, sb = one.stats(), b.stats()
        for key in ("unique", "nonempty_leaves", "max_leaf_size", "max_window", "mean_window"):
            assert sa[key] == sb[key], key
        if R.numel():
            Rh = _u64(R)
            _validate.compare_index(Rh, eb, oracle.rmi_fit(Rh, L, prec == "fp64"), prec == "fp64")
    # the batch's indexes join exactly like indexes built alone
    S = joins[2]["S"]
    p1 = torch.empty((S.numel(), 2), dtype=torch.int32, device="cuda")
    t1 = lj.join_emit(batch[2], S, p1)
    assert np.array_equal(p1[:t1].cpu().numpy().view(np.uint32),
                          oracle.join_pairs(_u64(Rs[2]), _u64(S)))
    # freeing indexes of a batch in any order keeps the others usable
    del batch[0:2]
    assert lj.join_emit(batch[0], S, p1) == t1


def test_batched_index_build_rejects_an_unsorted_relation():
    lj = _lj()
    joins = dg.batched_workload(k=3, seed=13, device="cuda", scale=1 / 64)
    Rs = [j["R"] for j in joins]
    bad = Rs[1].clone()
    bad[0], bad[-1] = Rs[1][-1], Rs[1][0]
    with pytest.raises(lj.LJoinError) as e:
        lj.rmi_build_batch([Rs[0], bad, Rs[2]], [16, 16, 16], "fp32")
    assert e.value.code == -4          # LJ_E_UNSORTED
