"""The bench's multi-rank path on CPU: world size 2 over gloo (127.0.0.1).

Each rank reports its own elapsed time; the job time is the slowest rank's,
and the whole-job value counts every rank's units (weak scaling: each rank
probes its own S against its replica of the index, with no collective on the
data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    os.environ["LJ_BENCH_BACKEND"] = "gloo"
    import bench
    r, w, local, d = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    elapsed = 10.0 + 5.0 * rank          # rank 1 is slower
    worst = bench.reduce_max(elapsed, d, "cpu")
    out[rank] = (worst, bench.weak_value(w, 1000, worst))
    d.barrier()
    d.destroy_process_group()


def test_two_rank_max_time_and_weak_value():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (15.0, 2 * 1000 / 0.015)


def test_single_rank_has_no_collective():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.weak_value(1, 400, 2.0) == 200000.0
