"""The multi-GPU path of bench.py is replicas only (every rank solves its own
mirror, no collective on the data path); the only exchange is the whole-job
aggregation of the timing.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, loc = bench.dist_setup()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        # rank-local figures differ: the job takes the slowest rank's time
        # and the applies of all ranks
        t_max, applies = bench.aggregate_over_ranks(1.5 + r, 100 * (r + 1), dist, torch.device("cpu"))
        out[r] = (w, r, loc, t_max, applies)
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_the_slowest_rank_and_all_applies():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (w, rr, loc, t_max, applies) in res.items():
        assert (w, rr, loc) == (2, r, r)
        assert t_max == 2.5          # max(1.5, 2.5)
        assert applies == 300.0      # 100 + 200
