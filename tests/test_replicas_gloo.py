"""Multi-GPU path of bench.py on CPU: the solve needs no exchange between GPUs, so N
ranks run independent replicas; the job time is the maximum over ranks (gloo,
world size 2, no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r measured (r + 1) seconds for its replica and 10 (r + 1) ms end to end
    t, e = bench.max_over_ranks([1.0 + rank, 0.01 * (1 + rank)], dist, "cpu")
    out[rank] = (t, e, bench.job_throughput(5, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, e, v = res[r]
        assert t == 2.0 and abs(e - 0.02) < 1e-15       # slowest rank sets the job time
        assert v == pytest.approx(2 * 5 / 2.0)           # all ranks' solves / slowest time


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_throughput(10, 1, 2.0) == 5.0
