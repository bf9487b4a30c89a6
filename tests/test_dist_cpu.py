"""The multi-rank bench path on CPU: two gloo ranks, one replica each.

bench.py reports the slowest rank's time and the units all ranks processed
(weak scaling, no data-path collective); the reference arm runs on rank 0
only and the other ranks leave at once.
"""
import os
import sys

import numpy as np
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
    mgr = mp.get_context("spawn").Manager()
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


# ---------------------------------------------------------------- independent graphs sharded by graph
class _OracleWorker:
    """Per-rank stand-in for the CUDA multi-graph handle: one CPU oracle
    graph per owned graph (O4), no kernels."""

    def __init__(self, ns, ms, edges):
        import oracle
        off = np.concatenate([[0], np.cumsum(ms)])
        self.gs = [oracle.OracleGraph(int(n), edges[off[i]:off[i + 1]], mode=oracle.SUPERIOR)
                   for i, n in enumerate(ns)]

    def update(self, op, counts, edges):
        off = np.concatenate([[0], np.cumsum(counts)])
        return [(g.insert_edges if op == 0 else g.delete_edges)(edges[off[i]:off[i + 1]])
                for i, g in enumerate(self.gs)]

    def cores(self):
        return [g.cores() for g in self.gs]


def _shard_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1612_09368_gb300 import shard
    from synth import workloads
    w = workloads.ba_many(24, rounds=1, nmax_exp=3.6, bmax_exp=2.5)
    s = shard.Shard(w["ns"], np.diff(w["eoff"]), w["edges"], rank, world, make_worker=_OracleWorker)
    pi = s.insert(w["kins"][0], w["ins"][0])
    pd = s.delete(w["kdel"][0], w["dele"][0])
    got = s.gather()
    out[rank] = (s.owned.tolist(), pi.tolist(), pd.tolist(), got)
    dist.destroy_process_group()


def test_sharded_graphs_two_ranks_gloo():
    """24 BA graphs split over two gloo ranks: each graph is owned by exactly
    one rank, the edge loads balance, every rank applies only its graphs'
    batches, and rank 0's gathered cores equal O1 on every graph's expected
    edge set."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1612_09368_gb300 import shard
    from synth import workloads
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    mp.spawn(_shard_main, args=(2, port, out), nprocs=2, join=True)
    w = workloads.ba_many(24, rounds=1, nmax_exp=3.6, bmax_exp=2.5)
    ms = np.diff(w["eoff"])
    owned0, owned1 = out[0][0], out[1][0]
    assert sorted(owned0 + owned1) == list(range(24)) and not set(owned0) & set(owned1)
    loads = [ms[owned0].sum(), ms[owned1].sum()]
    assert max(loads) - min(loads) <= ms.max()
    for o, pi, pd in (out[0][:3], out[1][:3]):
        assert pi == [int(w["kins"][0][i]) for i in o] and pd == [int(w["kdel"][0][i]) for i in o]
    got = out[0][3]
    assert out[1][3] is None and sorted(got) == list(range(24))
    io = np.concatenate([[0], np.cumsum(w["kins"][0])])
    do = np.concatenate([[0], np.cumsum(w["kdel"][0])])
    key = lambda e: set(map(tuple, np.sort(np.asarray(e).reshape(-1, 2), 1).tolist()))
    for i in range(24):
        k = key(w["edges"][w["eoff"][i]:w["eoff"][i + 1]]) | key(w["ins"][0][io[i]:io[i + 1]])
        k -= key(w["dele"][0][do[i]:do[i + 1]])
        exp = oracle.bz(int(w["ns"][i]), np.array(sorted(k), np.int32).reshape(-1, 2))
        assert (got[i] == exp).all(), i


def test_partition_is_balanced_and_deterministic():
    sys.path.insert(0, ROOT)
    from paper_1612_09368_gb300 import shard
    rng = np.random.default_rng(3)
    w = rng.integers(1, 10 ** 6, 512)
    for world in (1, 2, 4, 8):
        parts = shard.partition(w, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(512))
        loads = [w[p].sum() for p in parts]
        assert max(loads) - min(loads) <= w.max()
        assert all((a == b).all() for a, b in zip(parts, shard.partition(w, world)))
