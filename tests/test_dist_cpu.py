"""The multi-rank bench path on CPU: two gloo ranks, one replica each.

bench.py reports the slowest rank's time and the units all ranks processed
(weak scaling, no data-path collective); the reference arm runs on rank 0
only and the other ranks leave at once.
"""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    t, u = bench.aggregate(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world, torch.device("cpu"))
    ws, r, local = bench.dist_env()

    class A:
        steps, warmup, gpus, scale = 1, 0, world, 20
    ref_rc = bench.run_reference(A()) if rank != 0 else None
    dist.barrier()
    out[rank] = (t, u, ws, r, ref_rc)
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29000 + os.getpid() % 1000
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0][:4] == (15.0, 3000.0, 2, 0)
    assert out[1][:4] == (15.0, 3000.0, 2, 1)
    assert out[1][4] == 0          # the reference arm does no work off rank 0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 7.0, 1, None) == (12.5, 7.0)
