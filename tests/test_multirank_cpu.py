"""The multi-GPU path of bench.py on CPU ranks (gloo, world_size 2): every
rank runs its own replica with its own seed, the timing is the slowest
rank's, and the reported value counts all replicas' pair-updates."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_local = 0.25 + 0.5 * rank  # rank 1 is the slow one
    t_max = bench.max_over_ranks(t_local, dist)
    value = bench.whole_job_value(1000.0, 10, world, t_max)
    q.put((rank, t_max, value, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0.75, 0.75]  # both see the slowest rank's time
    assert out[0][2] == pytest.approx(1000.0 * 10 * 2 / 0.75)
    assert out[0][3] != out[1][3]  # independent replicas


def test_single_rank_is_local_time():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_value(10.0, 3, 1, 2.0) == 15.0
