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

from . import (DELETE, GRAPH, INSERT, PREFERENTIAL, UNIFORM, VDELETE, VINSERT, DynGraph, ba, er, rmat, stream,
               uniform)
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
