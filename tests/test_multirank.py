"""Multi-rank host logic of the bench (replicas): two gloo ranks on CPU.

Rays are independent and every GPU replicates the grid, so N GPUs run N
replicas with no data-path collective; the only cross-rank step is the
max-over-ranks reduction of the step time behind the whole-job throughput.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mean_ms, rate = bench.combine_ranks(10.0 * (rank + 1), 1000, world)  # rank 1 is the slow one
    q.put((rank, mean_ms, rate, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mean_ms, rate, env in out:
        assert mean_ms == pytest.approx(20.0)
        assert rate == pytest.approx(2 * 1000 / 0.020)
        assert env == (rank, 0, 2)


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(5.0, 100, 1) == (5.0, 100 / 0.005)
