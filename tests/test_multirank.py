"""The benchmark's multi-process host logic with two gloo ranks on the CPU:
replicas that share nothing on the data path, the barrier, the maximum of
the ranks' times, and the split of independent designs over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(None, backend="gloo")
    assert (w, r) == (world, rank)
    bench.barrier(w)
    out[rank] = bench.max_over_ranks(1.5 + rank, w)
    mine = bench.shard(range(11), r, w)
    out[world + rank] = sum(mine)
    out[2 * world + rank] = len(mine)
    dist.destroy_process_group()


def test_two_ranks_max_and_shard():
    world = 2
    out = mp.get_context("spawn").Array("d", 3 * world)
    port = _free_port()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    assert out[0] == out[1] == 2.5              # max over the ranks' values
    assert out[2] + out[3] == sum(range(11))      # every design on exactly one rank
    assert (out[4], out[5]) == (6, 5)           # 0,2,4,6,8,10 and 1,3,5,7,9
