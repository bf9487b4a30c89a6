"""Independent graphs sharded across GPUs, one process per GPU.

A many-graph workload (graphs that share no edge, such as the 512
Barabasi-Albert graphs or the serving graphs) splits by graph: every rank
owns a subset of the graphs, keeps them in ONE multi-graph handle on its own
GPU and applies their update batches without any communication, since the
core numbers of a graph depend on that graph alone (Section III,
Definitions 1-2).  Per-graph results meet on the host only when asked
(``Shard.gather``: a gather of Python objects to rank 0).  A single graph
does not shard (an iteration of Algorithms 1 / 5 is one global step with
data-dependent waves), so there is no device-side collective anywhere.

Only argument marshalling and bookkeeping live here; the per-rank worker
is the CUDA library's multi-graph handle (``CudaWorker``).
"""
from __future__ import annotations

import numpy as np

from . import CM_OP_DELETE, CM_OP_INSERT, CoreGraph


def partition(weights, world: int) -> list:
    """Graphs -> ranks: largest first onto the least-loaded rank (ties to
    the lower rank), so every rank gets about the same number of edges.
    Deterministic; returns, per rank, its graph indices in increasing order."""
    w = np.asarray(weights, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(len(w), dtype=np.int64)
    for i in np.argsort(-w, kind="stable"):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += w[i]
    return [np.nonzero(owner == r)[0] for r in range(world)]


def select(counts, edges, owned):
    """The batches of the owned graphs out of a per-graph concatenation:
    (their counts, their edges concatenated in owned order)."""
    counts = np.asarray(counts, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(counts)])
    e = np.asarray(edges).reshape(-1, 2)
    parts = [e[off[i]:off[i + 1]] for i in owned]
    sub = np.concatenate(parts) if parts else np.zeros((0, 2), e.dtype)
    return counts[owned], np.ascontiguousarray(sub, dtype=np.int32)


class CudaWorker:
    """The owned graphs in one multi-graph handle on this process's GPU."""

    def __init__(self, ns, ms, edges, **opts):
        import torch
        self.ns = np.asarray(ns, dtype=np.int32)
        self.g = CoreGraph(None, torch.from_numpy(np.ascontiguousarray(edges, dtype=np.int32)).cuda(),
                           multi=(self.ns, np.asarray(ms, dtype=np.int64)), **opts)
        self.bases = self.g.bases()

    def update(self, op, counts, edges):
        return self.g.update_multi(op, counts, edges)

    def cores(self):
        c = self.g.cores()
        return [c[b:b + n] for b, n in zip(self.bases, self.ns)]

    def close(self):
        self.g.close()


class Shard:
    """This rank's part of a many-graph workload.  ns / ms: vertices and
    edges of every graph; edges: all graphs' edge lists (local ids)
    concatenated in graph order.  make_worker(ns, ms, edges) builds the
    per-rank worker (default: CudaWorker)."""

    def __init__(self, ns, ms, edges, rank: int, world: int, make_worker=None, **opts):
        self.ns = np.asarray(ns, dtype=np.int32)
        self.ms = np.asarray(ms, dtype=np.int64)
        self.rank, self.world = rank, world
        self.owned = partition(self.ms, world)[rank]
        _, sub = select(self.ms, edges, self.owned)
        make = make_worker or CudaWorker
        self.worker = make(self.ns[self.owned], self.ms[self.owned], sub, **opts)

    def update(self, op, counts, edges):
        """One batch per graph of the whole workload (counts for every
        graph, edges concatenated in graph order); applies the owned graphs'
        batches and returns their applied counts (owned order)."""
        c, sub = select(counts, edges, self.owned)
        return np.asarray(self.worker.update(op, c, sub), dtype=np.int64)

    def insert(self, counts, edges):
        return self.update(CM_OP_INSERT, counts, edges)

    def delete(self, counts, edges):
        return self.update(CM_OP_DELETE, counts, edges)

    def cores(self) -> dict:
        return {int(i): c for i, c in zip(self.owned, self.worker.cores())}

    def gather(self, group=None):
        """Every graph's core numbers on rank 0 ({graph: cores}), None on
        the other ranks.  Host objects through torch.distributed; nothing
        on the device path."""
        import torch.distributed as dist
        mine = {i: np.asarray(c) for i, c in self.cores().items()}
        if self.world == 1:
            return mine
        out = [None] * self.world if self.rank == 0 else None
        dist.gather_object(mine, out, dst=0, group=group)
        if self.rank != 0:
            return None
        allc = {}
        for part in out:
            allc.update(part)
        return allc

    def close(self):
        close = getattr(self.worker, "close", None)
        if close:
            close()
