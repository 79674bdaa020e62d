"""The multi-GPU path of the benchmark runs independent replicas (the step has no
exchange): whole-job time = max over ranks, samples = sum over ranks.  Checked
with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    maxes, sums = bench.reduce_over_ranks([10.0 + rank, 20.0 - rank], [1000 * (rank + 1), 7], "cpu")
    out[rank] = (maxes, sums)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        maxes, sums = out[r]
        assert maxes == [11.0, 20.0]
        assert sums == [3000.0, 14.0]
