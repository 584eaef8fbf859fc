"""Failure detection on the device without a GPU fault: a bounded wait that
runs out.

The single-pass probe kernel takes each tile's output offset by a decoupled
look-back over its predecessors' published states.  The test hook
"fault_skip_tiles" launches the kernel without its leading tile, so that
tile's state is never published (a flag that nothing sets); with the wait
bound "lookback_polls" lowered, the next tiles give up after a few hundred
polls, record LJ_E_TIMEOUT in the error word and finish.  The calls must
report LJ_E_TIMEOUT, nothing may trap or hang, and the context must stay
usable: afterwards the same joins give the oracle's result.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = -6   # LJ_E_TIMEOUT


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_lookback_wait_runs_out_and_reports_timeout():
    import paper_2111_08824_gb300 as lj
    rng = np.random.default_rng(21)
    R = np.unique(rng.integers(0, 2**50, 400_000, dtype=np.uint64))
    S = np.concatenate([R[rng.integers(0, R.size, 15_000)],
                        rng.integers(0, 2**50, 5_000, dtype=np.uint64)])   # ~10 tiles
    idx = lj.rmi_build(_dev(R), 2048, "fp32")
    Sd = _dev(S)
    lo, hi, want = oracle.join_ranges(R, S)
    names = ("lookback_polls", "fault_skip_tiles", "single_pass_max")
    old = {k: lj.lj_get_option(k) for k in names}
    try:
        lj.lj_set_option("lookback_polls", 256)
        lj.lj_set_option("fault_skip_tiles", 1)
        lj.lj_set_option("single_pass_max", 1 << 40)
        with pytest.raises(lj.LJoinError) as e:
            lj.join_count(idx, Sd)
        assert e.value.code == TIMEOUT
        with pytest.raises(lj.LJoinError) as e:
            lj.join_count_noalloc(idx, Sd)
        assert e.value.code == TIMEOUT
        # an asynchronous call's timeout is reported by the next call with a total
        lj.join_count_noalloc(idx, Sd, want_total=False)
        lj.lj_set_option("fault_skip_tiles", 0)
        with pytest.raises(lj.LJoinError) as e:
            lj.join_count_noalloc(idx, Sd)
        assert e.value.code == TIMEOUT
        # once reported, the error is cleared: the next calls are clean
        assert lj.join_count_noalloc(idx, Sd) == want
        assert lj.join_count(idx, Sd) == want
        # the fused kernel's grid-wide barrier: a skipped block never arrives,
        # the other blocks' bounded waits run out
        lj.lj_set_option("fault_skip_tiles", 1)
        pairs = torch.empty((S.size, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(lj.LJoinError) as e:
            lj.join_emit(idx, Sd, pairs)
        assert e.value.code == TIMEOUT
        lj.lj_set_option("fault_skip_tiles", 0)
        assert lj.join_emit(idx, Sd, pairs) == want
    finally:
        for k, v in old.items():
            lj.lj_set_option(k, v)
    # the context is still usable: the full join equals the oracle's
    counts = torch.empty(S.size, dtype=torch.int32, device="cuda")
    assert lj.join_count(idx, Sd, counts=counts) == want
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), (hi - lo).astype(np.int64))
    pairs = torch.empty((S.size, 2), dtype=torch.int32, device="cuda")
    total = lj.join_emit(idx, Sd, pairs)
    assert np.array_equal(pairs[:total].cpu().numpy().view(np.uint32), oracle.join_pairs(R, S))
