"""The N > 1 benchmark path on CPU: two gloo ranks, the barrier, the max of the
timed region over ranks and the whole-job value of independent replicas."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_env()
    assert (w, r, lr) == (world, rank, rank)
    bench.barrier(world)
    # rank r "took" 100 + 10 r ms for 50 steps
    mx = bench.max_over_ranks(torch, 100.0 + 10.0 * rank, world)
    out[rank] = (mx, bench.replica_steps_per_s(world, 50, mx))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    mx, sps = out[0]
    assert mx == 110.0
    assert sps == pytest.approx(2 * 50 / 0.110)
