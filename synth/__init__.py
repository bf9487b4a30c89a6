"""Seeded synthetic graphs and update streams (inputs only).

This module writes inputs -- edge lists, update batches and vertex ids -- and
nothing else: it computes no core numbers and contains none of the
maintenance method's arithmetic.  Both the CPU oracle and the CUDA library
consume what it produces.  The C source is ``synth.c``; it is compiled on
first use (or by ``build()``) into ``libsynth.so`` next to it.

Randomness is SplitMix64 used counter-wise; every stream is named by a tuple
(config, graph, round, purpose) hashed with a base seed (0 by default).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, i64, dbl = ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            vp = ctypes.c_void_p
            sig = {
                "sy_stream": (u64, [u64, u64, u64, u64, u64]),
                "sy_draw": (u64, [u64, u64]),
                "sy_er": (i64, [i32, i64, u64, _i32p]),
                "sy_rmat": (i64, [i32, i64, dbl, dbl, dbl, u64, i32, _i32p]),
                "sy_ba": (i64, [i32, i32, u64, _i32p]),
                "sy_ba_many": (ctypes.c_int, [i32, _i32p, _i32p, vp, _i64p, _i32p, i32, _i64p, _i64p, vp, _i64p,
                                              _i64p, _i32p, _i32p]),
                "sy_grid": (i64, [i32, i64, u64, _i32p]),
                "sy_dyn_create": (vp, [i32, i64, _i32p]),
                "sy_dyn_free": (None, [vp]),
                "sy_dyn_n": (i32, [vp]),
                "sy_dyn_m": (i64, [vp]),
                "sy_dyn_nlive": (i32, [vp]),
                "sy_dyn_degree": (i32, [vp, i32]),
                "sy_dyn_edges": (i64, [vp, _i32p]),
                "sy_dyn_alive": (None, [vp, _i8p]),
                "sy_dyn_sample_insert": (i64, [vp, i64, i32, u64, _i32p]),
                "sy_dyn_sample_delete": (i64, [vp, i64, i32, u64, _i32p]),
                "sy_dyn_apply": (i64, [vp, i32, _i32p, i64]),
                "sy_dyn_add_vertices": (i64, [vp, i32, i32, u64, _i32p]),
                "sy_dyn_delete_vertices": (i64, [vp, i32, u64, _i32p]),
                "sy_dyn_incident": (i64, [vp, i32, _i32p]),
                "sy_static_sample_insert": (i64, [_i32p, i64, i32, i64, i32, u64, _i32p]),
                "sy_static_sample_delete": (i64, [_i32p, i64, i32, _i64p, _i32p, i64, i32, u64, _i32p]),
                "sy_csr": (ctypes.c_int, [i32, i64, _i32p, _i64p, _i32p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


# purposes of a stream
GRAPH, INSERT, DELETE, VINSERT, VDELETE, PARAM, ARRIVAL = range(7)
# sampling laws
UNIFORM = 0      # insert: uniform endpoints; delete: uniform vertex, then a uniform neighbour
PREFERENTIAL = 1  # insert: degree-proportional endpoints; delete: a uniform random edge


def stream(cfg: int, graph: int = 0, rnd: int = 0, purpose: int = GRAPH, base: int = 0) -> int:
    return int(_L().sy_stream(base, cfg, graph, rnd, purpose))


def draw(seed: int, i: int) -> int:
    return int(_L().sy_draw(seed, i))


def uniform(seed: int, i: int) -> float:
    """i-th U[0,1) draw of a stream (53-bit)."""
    return (draw(seed, i) >> 11) * (1.0 / 9007199254740992.0)


def er(n: int, m: int, seed: int) -> np.ndarray:
    out = np.empty((m, 2), dtype=np.int32)
    got = _L().sy_er(n, m, seed, _p32(out))
    if got != m:
        raise ValueError(f"sy_er failed ({got})")
    return out


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19, permute=True) -> np.ndarray:
    ns = edge_factor << scale
    out = np.empty((ns, 2), dtype=np.int32)
    m = _L().sy_rmat(scale, ns, a, b, c, seed, 1 if permute else 0, _p32(out))
    if m < 0:
        raise ValueError(f"sy_rmat failed ({m})")
    return out[:m].copy() if m < ns // 2 else out[:m]


def ba(n: int, m: int, seed: int) -> np.ndarray:
    cnt = m * (m + 1) // 2 + (n - m - 1) * m
    out = np.empty((cnt, 2), dtype=np.int32)
    got = _L().sy_ba(n, m, seed, _p32(out))
    if got != cnt:
        raise ValueError(f"sy_ba failed ({got})")
    return out


def ba_edge_count(n: int, m: int) -> int:
    """Edges of ba(n, m): a clique on m + 1 vertices, then m per vertex."""
    return m * (m + 1) // 2 + (n - m - 1) * m


def ba_many(ns, ms, gseeds, kins, kdel, bseeds):
    """Many BA graphs and per-graph batches (see sy_ba_many).  kins, kdel,
    bseeds: arrays [rounds, ngraphs].  Returns (edges [sum m, 2] in graph
    order with local ids, eoff [ng+1], ins [rounds] list of arrays, del
    [rounds] list of arrays), round r's arrays holding every graph's batch
    in graph order."""
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    ng = len(ns)
    kins = np.ascontiguousarray(kins, dtype=np.int64).reshape(-1, ng)
    kdel = np.ascontiguousarray(kdel, dtype=np.int64).reshape(-1, ng)
    rounds = kins.shape[0]
    gs = np.ascontiguousarray(gseeds, dtype=np.uint64)
    bs = np.ascontiguousarray(bseeds, dtype=np.uint64).reshape(-1)
    ecount = np.array([ba_edge_count(int(n), int(m)) for n, m in zip(ns, ms)], dtype=np.int64)
    eoff = np.zeros(ng + 1, dtype=np.int64)
    eoff[1:] = np.cumsum(ecount)
    ioff = np.zeros(rounds * ng + 1, dtype=np.int64)
    ioff[1:] = np.cumsum(kins.reshape(-1))
    doff = np.zeros(rounds * ng + 1, dtype=np.int64)
    doff[1:] = np.cumsum(kdel.reshape(-1))
    edges = np.empty((int(eoff[-1]), 2), dtype=np.int32)
    ins = np.empty((int(ioff[-1]), 2), dtype=np.int32)
    dele = np.empty((int(doff[-1]), 2), dtype=np.int32)
    rc = _L().sy_ba_many(ng, _p32(ns), _p32(ms), gs.ctypes.data, eoff.ctypes.data_as(_i64p), _p32(edges), rounds,
                         kins.ctypes.data_as(_i64p), kdel.ctypes.data_as(_i64p), bs.ctypes.data,
                         ioff.ctypes.data_as(_i64p), doff.ctypes.data_as(_i64p), _p32(ins), _p32(dele))
    if rc != 0:
        raise RuntimeError(f"sy_ba_many failed ({rc})")
    ins_r = [ins[ioff[r * ng]: ioff[(r + 1) * ng]] for r in range(rounds)]
    del_r = [dele[doff[r * ng]: doff[(r + 1) * ng]] for r in range(rounds)]
    return edges, eoff, ins_r, del_r


def grid(side: int, nshort: int, seed: int) -> np.ndarray:
    cnt = 2 * side * (side - 1) + nshort
    out = np.empty((cnt, 2), dtype=np.int32)
    got = _L().sy_grid(side, nshort, seed, _p32(out))
    if got != cnt:
        raise ValueError(f"sy_grid failed ({got})")
    return out


def csr(n: int, edges: np.ndarray):
    """(row_off int64[n+1], adj int32[2m]) listing every edge in both rows."""
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    row_off = np.empty(n + 1, dtype=np.int64)
    adj = np.empty(2 * len(e), dtype=np.int32)
    if _L().sy_csr(n, len(e), _p32(e), row_off.ctypes.data_as(_i64p), _p32(adj)) != 0:
        raise MemoryError("sy_csr")
    return row_off, adj


def static_sample_insert(n: int, edges: np.ndarray, count: int, law: int, seed: int) -> np.ndarray:
    """New edges for a large static graph (no dynamic model needed)."""
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    out = np.empty((count, 2), dtype=np.int32)
    got = _L().sy_static_sample_insert(_p32(e), len(e), n, count, law, seed, _p32(out))
    if got < 0:
        raise MemoryError("sy_static_sample_insert")
    return out[:got].copy()


def static_sample_delete(n: int, edges: np.ndarray, count: int, law: int, seed: int, csr_=None) -> np.ndarray:
    """Existing edges of a large static graph; law UNIFORM needs csr_ = csr(n, edges)."""
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    out = np.empty((count, 2), dtype=np.int32)
    ro, ad = (None, None) if csr_ is None else csr_
    got = _L().sy_static_sample_delete(_p32(e), len(e), n, None if ro is None else ro.ctypes.data_as(_i64p),
                                       None if ad is None else _p32(ad), count, law, seed, _p32(out))
    if got < 0:
        raise MemoryError("sy_static_sample_delete")
    return out[:got].copy()


class DynGraph:
    """Evolving vertex/edge set used to draw update batches: new edges are
    absent from the current graph, existing ones present, and inserted
    vertices receive the ids an append-only dense numbering gives them."""

    def __init__(self, n: int, edges: np.ndarray):
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        self._h = _L().sy_dyn_create(n, len(e), _p32(e))
        if not self._h:
            raise MemoryError("sy_dyn_create")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().sy_dyn_free(h)
            self._h = None

    @property
    def n(self) -> int:
        return int(_L().sy_dyn_n(self._h))

    @property
    def m(self) -> int:
        return int(_L().sy_dyn_m(self._h))

    @property
    def nlive(self) -> int:
        return int(_L().sy_dyn_nlive(self._h))

    def degree(self, v: int) -> int:
        return int(_L().sy_dyn_degree(self._h, v))

    def edges(self) -> np.ndarray:
        out = np.empty((self.m, 2), dtype=np.int32)
        _L().sy_dyn_edges(self._h, _p32(out))
        return out

    def alive(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int8)
        _L().sy_dyn_alive(self._h, out.ctypes.data_as(_i8p))
        return out.astype(bool)

    def sample_insert(self, count: int, law: int, seed: int) -> np.ndarray:
        out = np.empty((count, 2), dtype=np.int32)
        got = _L().sy_dyn_sample_insert(self._h, count, law, seed, _p32(out))
        return out[:got].copy()

    def sample_delete(self, count: int, law: int, seed: int) -> np.ndarray:
        out = np.empty((count, 2), dtype=np.int32)
        got = _L().sy_dyn_sample_delete(self._h, count, law, seed, _p32(out))
        return out[:got].copy()

    def apply(self, op: int, edges: np.ndarray) -> int:
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        return int(_L().sy_dyn_apply(self._h, op, _p32(e), len(e)))

    def add_vertices(self, count: int, degree: int, seed: int) -> np.ndarray:
        """Returns (count, degree) neighbour ids; the new ids are n .. n+count-1."""
        out = np.empty((count, degree), dtype=np.int32)
        got = _L().sy_dyn_add_vertices(self._h, count, degree, seed, _p32(out))
        if got < 0:
            raise ValueError("not enough live vertices")
        return out

    def delete_vertices(self, count: int, seed: int) -> np.ndarray:
        out = np.empty(count, dtype=np.int32)
        got = _L().sy_dyn_delete_vertices(self._h, count, seed, _p32(out))
        return out[:got].copy()

    def incident(self, v: int) -> np.ndarray:
        out = np.empty((max(self.degree(v), 0), 2), dtype=np.int32)
        _L().sy_dyn_incident(self._h, v, _p32(out))
        return out
