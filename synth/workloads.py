"""Named synthetic workloads (inputs only).

Each recipe returns the initial graph and the update batches, drawn from
seeded SplitMix64 streams named (config, graph, round, purpose).  The graph
families are those of the paper's synthetic experiments (Section VII:
Erdos-Renyi, Barabasi-Albert, R-MAT) plus a grid with shortcuts.  The SNAP
graphs of the paper's real-world experiments are not available; these
inputs stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (ARRIVAL, DELETE, GRAPH, INSERT, PREFERENTIAL, UNIFORM, VDELETE, VINSERT, DynGraph, ba, er, rmat,
               static_sample_delete, static_sample_insert, stream, uniform)
from . import grid as _grid
from . import ba_many as _ba_many

EDGE_UNIFORM = PREFERENTIAL   # "a uniform random existing edge" is the degree-proportional delete law


@dataclass
class Round:
    ins: np.ndarray                    # (k, 2) new edges
    dele: np.ndarray                   # (k, 2) existing edges
    vnbrs: np.ndarray                  # (count, degree) neighbours of new vertices
    vdel: np.ndarray                   # ids of deleted vertices
    vdel_edges: int = 0                # edges incident to them when deleted
    first_new_id: int = 0

    def edge_updates(self) -> int:
        return len(self.ins) + len(self.dele) + int(self.vnbrs.size) + self.vdel_edges


@dataclass
class Workload:
    name: str
    n: int
    edges: np.ndarray
    rounds: list = field(default_factory=list)
    params: dict = field(default_factory=dict)
    final: DynGraph | None = None


def er_small(cfg: int = 1) -> Workload:
    """ER G(n=10,000, m=50,000); one batch of 1,000 uniform new edges, then
    1,000 uniform existing edges deleted."""
    n, m = 10000, 50000
    e = er(n, m, stream(cfg, 0, 0, GRAPH))
    d = DynGraph(n, e)
    ins = d.sample_insert(1000, UNIFORM, stream(cfg, 0, 0, INSERT))
    d.apply(0, ins)
    dl = d.sample_delete(1000, EDGE_UNIFORM, stream(cfg, 0, 0, DELETE))
    d.apply(1, dl)
    w = Workload("er-10k-50k", n, e, params={"n": n, "m": m, "insert": 1000, "delete": 1000})
    w.rounds.append(Round(ins, dl, np.zeros((0, 8), np.int32), np.zeros(0, np.int32)))
    w.final = d
    return w


def rmat_rounds(rounds: int, scale: int = 20, edge_factor: int = 16, ins: int = 10 ** 4, dele: int = 10 ** 4,
                vins: int = 100, vdeg: int = 8, vdel: int = 100, cfg: int = 2) -> Workload:
    """R-MAT (a,b,c,d) = (.57,.19,.19,.05), 2^scale vertices, edge_factor *
    2^scale samples, symmetrised and deduplicated, ids permuted.  Each round:
    `ins` uniform new edges, `dele` uniform existing edges, `vins` new
    vertices of degree `vdeg` (uniform live neighbours) and `vdel` uniform
    live vertices deleted, in that order."""
    e = rmat(scale, edge_factor, stream(cfg, 0, 0, GRAPH))
    n = 1 << scale
    d = DynGraph(n, e)
    w = Workload(f"rmat{scale}-rounds", n, e, params={
        "scale": scale, "edge_factor": edge_factor, "insert_per_round": ins, "delete_per_round": dele,
        "vertex_insert_per_round": vins, "vertex_degree": vdeg, "vertex_delete_per_round": vdel})
    for r in range(rounds):
        a = d.sample_insert(ins, UNIFORM, stream(cfg, 0, r, INSERT))
        d.apply(0, a)
        b = d.sample_delete(dele, EDGE_UNIFORM, stream(cfg, 0, r, DELETE))
        d.apply(1, b)
        first = d.n
        nb = d.add_vertices(vins, vdeg, stream(cfg, 0, r, VINSERT)) if vins else np.zeros((0, vdeg), np.int32)
        m_before = d.m
        vd = d.delete_vertices(vdel, stream(cfg, 0, r, VDELETE)) if vdel else np.zeros(0, np.int32)
        w.rounds.append(Round(a, b, nb, vd, m_before - d.m, first))
    w.final = d
    return w


def rmat_sweep(scale: int = 24, edge_factor: int = 16, sizes=(10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6), cfg: int = 3,
               ops=("insert", "delete"), laws=(UNIFORM, PREFERENTIAL)):
    """R-MAT graph plus, per batch size and endpoint law (uniform /
    degree-proportional), an insert batch of new edges and a delete batch of
    existing edges, each drawn against the original graph."""
    from . import csr, static_sample_delete, static_sample_insert
    e = rmat(scale, edge_factor, stream(cfg, 0, 0, GRAPH))
    n = 1 << scale
    c = csr(n, e) if ("delete" in ops and UNIFORM in laws) else None
    batches = {}
    for i, s in enumerate(sizes):
        for law in laws:
            if "insert" in ops:
                batches[("insert", s, law)] = static_sample_insert(n, e, s, law, stream(cfg, 0, 2 * i + law, INSERT))
            if "delete" in ops:
                batches[("delete", s, law)] = static_sample_delete(n, e, s, law, stream(cfg, 0, 2 * i + law, DELETE),
                                                                   c)
    return n, e, batches


def ba_many(ngraphs: int = 512, rounds: int = 1, cfg: int = 4, nmin_exp: float = 3.0, nmax_exp: float = 6.0,
            bmin_exp: float = 1.0, bmax_exp: float = 4.0, frac_insert: float = 0.7):
    """Barabasi-Albert graphs with n log-uniform in [10^nmin_exp,
    10^nmax_exp] and attachment m uniform in {4..16}; per graph and round a
    batch of size log-uniform in [10^bmin_exp, 10^bmax_exp], 70% new
    uniform pairs and 30% uniform existing edges, every round drawn against
    the graph as generated (a round is applied, timed, then undone).
    Returns dict(ns, ms, edges, eoff, ins [rounds], dele [rounds],
    kins [rounds, ng], kdel [rounds, ng])."""
    ns = np.empty(ngraphs, dtype=np.int32)
    ms = np.empty(ngraphs, dtype=np.int32)
    gseeds = np.empty(ngraphs, dtype=np.uint64)
    kins = np.empty((rounds, ngraphs), dtype=np.int64)
    kdel = np.empty((rounds, ngraphs), dtype=np.int64)
    bseeds = np.empty((rounds, ngraphs), dtype=np.uint64)
    for gi in range(ngraphs):
        s = stream(cfg, gi, 0, 5)   # parameters
        ns[gi] = int(10 ** (nmin_exp + (nmax_exp - nmin_exp) * uniform(s, 0)))
        ms[gi] = 4 + int(13 * uniform(s, 1))
        gseeds[gi] = stream(cfg, gi, 0, GRAPH)
        for r in range(rounds):
            sb = stream(cfg, gi, r + 1, 5)
            b = int(10 ** (bmin_exp + (bmax_exp - bmin_exp) * uniform(sb, 0)))
            kins[r, gi] = int(round(frac_insert * b))
            kdel[r, gi] = b - kins[r, gi]
            bseeds[r, gi] = stream(cfg, gi, r + 1, INSERT)
    edges, eoff, ins, dele = _ba_many(ns, ms, gseeds, kins, kdel, bseeds)
    return {"ns": ns, "ms": ms, "edges": edges, "eoff": eoff, "ins": ins, "dele": dele, "kins": kins, "kdel": kdel}


def serving_graphs(cfg: int = 5, scale: int = 22, edge_factor: int = 16, side: int = 2048,
                   shortcut_frac: float = 0.01):
    """The resident graphs of the serving workload: an R-MAT graph and a
    side x side 4-neighbour grid plus shortcut_frac x its edge count of
    uniform random long-range pairs.  Returns [(n, edges), (n, edges)]."""
    e0 = rmat(scale, edge_factor, stream(cfg, 0, 0, GRAPH))
    nshort = int(round(shortcut_frac * 2 * side * (side - 1)))
    e1 = _grid(side, nshort, stream(cfg, 1, 0, GRAPH))
    return [(1 << scale, e0), (side * side, e1)]


def serving_trace(graphs, rate: float, duration_s: float, cfg: int = 5, trace: int = 0, median: float = 200.0,
                  sigma: float = 1.5, lo: int = 10, hi: int = 10 ** 5, frac_insert: float = 0.7):
    """Open-loop request stream: Poisson arrivals at `rate` per second for
    `duration_s`; each request targets a uniform graph, is an insert with
    probability frac_insert, and carries a log-normal number of edges
    (median `median`, log-space deviation `sigma`, clamped to [lo, hi]).
    Inserts are distinct uniform pairs absent from the graph as given and
    deletes distinct uniform edges of it, none shared between requests, so
    the requests of a graph can be applied in any interleaving and each
    applies exactly its edges.  Returns dict(arrival_ns, graph, op, counts,
    edges, off) with `edges` concatenated in request order (local ids)."""
    import math
    s = stream(cfg, 0, trace, ARRIVAL)
    arr, gr, op, cnt = [], [], [], []
    t, i = 0.0, 0
    ng = len(graphs)
    while True:
        t += -math.log(1.0 - uniform(s, 5 * i)) / rate
        if t >= duration_s:
            break
        gr.append(min(ng - 1, int(ng * uniform(s, 5 * i + 1))))
        op.append(0 if uniform(s, 5 * i + 2) < frac_insert else 1)
        u1 = max(uniform(s, 5 * i + 3), 1e-300)
        z = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * uniform(s, 5 * i + 4))
        cnt.append(int(min(hi, max(lo, round(median * math.exp(sigma * z))))))
        arr.append(int(t * 1e9))
        i += 1
    gr = np.array(gr, dtype=np.int32)
    op = np.array(op, dtype=np.int32)
    cnt = np.array(cnt, dtype=np.int64)
    pools = {}
    for gi, (n, e) in enumerate(graphs):
        need_i = int(cnt[(gr == gi) & (op == 0)].sum())
        need_d = int(cnt[(gr == gi) & (op == 1)].sum())
        pi = static_sample_insert(n, e, need_i, UNIFORM, stream(cfg, gi, trace, INSERT))
        pd = static_sample_delete(n, e, need_d, PREFERENTIAL, stream(cfg, gi, trace, DELETE))
        if len(pi) < need_i or len(pd) < need_d:
            raise ValueError("graph too small for the trace's batches")
        pools[(gi, 0)] = [pi, 0]
        pools[(gi, 1)] = [pd, 0]
    off = np.zeros(len(cnt) + 1, dtype=np.int64)
    off[1:] = np.cumsum(cnt)
    edges = np.empty((int(off[-1]), 2), dtype=np.int32)
    for j in range(len(cnt)):
        p = pools[(int(gr[j]), int(op[j]))]
        edges[off[j]:off[j + 1]] = p[0][p[1]:p[1] + cnt[j]]
        p[1] += int(cnt[j])
    return {"arrival_ns": np.array(arr, dtype=np.int64), "graph": gr, "op": op, "counts": cnt, "edges": edges,
            "off": off}
