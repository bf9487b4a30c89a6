"""CPU oracle for k-core maintenance -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The CUDA library neither calls
it nor shares code with it.  The arithmetic lives in ``oracle.c`` (plain,
sequential C); this file compiles it and exposes it through ctypes.

  bz(n, edges)            O1  Batagelj-Zaversnik peeling (the [O(m)] algorithm
                              the paper cites in Section I)
  brute(n, edges)         O2  max over vertex subsets of the minimum induced
                              degree (Section III, Defs. 1-2), n <= 20
  OracleGraph(mode=0)     O3  sequential single-edge traversal, Section V
                              Algorithms 3-4 and Section VI Algorithms 6-7
                              with one edge per call
  OracleGraph(mode=1)     O4  superior-edge-set iterations, Algorithms 1, 2, 5

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, brute force, invariants of
Lemmas 1-4); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_libs: dict = {}

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)

SEQUENTIAL = 0   # O3
SUPERIOR = 1     # O4
INSERT, DELETE = 0, 1


def lib_path(plant: int = 0) -> str:
    return os.path.join(_HERE, "liboracle.so" if plant == 0 else f"liboracle_plant{plant}.so")


def build(plant: int = 0, force: bool = False) -> str:
    """Compile oracle.c (plain C, -O2).  plant > 0 builds a variant with one
    planted mistake, used only by the tests that show the pins catch it."""
    out = lib_path(plant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", f"-DPLANT={plant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def load(plant: int = 0):
    with _lock:
        if plant in _libs:
            return _libs[plant]
        lib = ctypes.CDLL(build(plant))
        i32, i64, u64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        sig = {
            "or_fmix64": (u64, [u64]),
            "or_bz": (ctypes.c_int, [i32, i64, _i32p, _i32p]),
            "or_bz_trusted": (ctypes.c_int, [i32, i64, _i32p, _i32p]),
            "or_brute": (ctypes.c_int, [i32, i64, _i32p, _i32p]),
            "or_create": (vp, [i32, i64, _i32p, _i32p]),
            "or_create_simple": (vp, [i32, i64, _i32p, _i32p]),
            "or_apply_structure": (None, [vp, i32, _i32p, i64]),
            "or_set_cores": (None, [vp, _i32p]),
            "or_free": (None, [vp]),
            "or_n": (i32, [vp]),
            "or_m": (i64, [vp]),
            "or_get_cores": (None, [vp, _i32p]),
            "or_edges": (i64, [vp, _i32p]),
            "or_last_iterations": (i64, [vp]),
            "or_last_log": (i64, [vp, _i64p, i64]),
            "or_update_edges": (i64, [vp, i32, _i32p, i64, i32]),
            "or_insert_vertices": (i64, [vp, i32, _i64p, _i32p, i32]),
            "or_delete_vertices": (i64, [vp, i32, _i32p, i32]),
            "or_batch_begin": (i64, [vp, i32, _i32p, i64]),
            "or_batch_step": (i32, [vp, _i32p, _i64p, _i32p, _i64p]),
            "or_set_selection": (None, [vp, i32, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[plant] = lib
        return lib


def _e(edges) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))


def _p32(a):
    return a.ctypes.data_as(_i32p)


def fmix64(x: int, plant: int = 0) -> int:
    return int(load(plant).or_fmix64(x & 0xFFFFFFFFFFFFFFFF))


def bz(n: int, edges, plant: int = 0, trusted: bool = False) -> np.ndarray:
    e = _e(edges)
    core = np.empty(n, dtype=np.int32)
    f = load(plant).or_bz_trusted if trusted else load(plant).or_bz
    rc = f(n, len(e), _p32(e), _p32(core))
    if rc != 0:
        raise ValueError(f"or_bz rejected the graph ({rc})")
    return core


def brute(n: int, edges, plant: int = 0) -> np.ndarray:
    e = _e(edges)
    core = np.empty(max(n, 1), dtype=np.int32)
    rc = load(plant).or_brute(n, len(e), _p32(e), _p32(core))
    if rc != 0:
        raise ValueError(f"or_brute rejected the graph ({rc})")
    return core[:n]


class OracleError(RuntimeError):
    pass


class OracleGraph:
    """Dynamic graph with core numbers maintained by O3 (mode 0) or O4 (mode 1)."""

    def __init__(self, n: int, edges, cores=None, mode: int = SUPERIOR, plant: int = 0,
                 select_order: int = 0, select_rounds: int = 0, simple: bool = False):
        """select_order / select_rounds: the variants of reading R1 for O4
        (1 = canonical-key order instead of its fmix64; R > 0 = at most R
        claim rounds per iteration).  simple: the caller guarantees the edge
        list is simple (no self-loop, no repeated pair), which skips the
        per-edge membership test of construction (unchecked)."""
        self._L = load(plant)
        e = _e(edges)
        c = None if cores is None else np.ascontiguousarray(cores, dtype=np.int32)
        mk = self._L.or_create_simple if simple else self._L.or_create
        self._h = mk(n, len(e), _p32(e), None if c is None else _p32(c))
        if not self._h:
            raise MemoryError("or_create")
        self.mode = mode
        self._L.or_set_selection(self._h, int(select_order), int(select_rounds))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_free(h)
            self._h = None

    @property
    def n(self) -> int:
        return int(self._L.or_n(self._h))

    @property
    def m(self) -> int:
        return int(self._L.or_m(self._h))

    def cores(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        self._L.or_get_cores(self._h, _p32(out))
        return out

    def edges(self) -> np.ndarray:
        out = np.empty((self.m, 2), dtype=np.int32)
        self._L.or_edges(self._h, _p32(out))
        return out

    def _chk(self, rc):
        if rc < 0:
            raise OracleError(f"oracle call failed ({rc})")
        return int(rc)

    def insert_edges(self, edges, mode=None) -> int:
        e = _e(edges)
        return self._chk(self._L.or_update_edges(self._h, INSERT, _p32(e), len(e), self.mode if mode is None else mode))

    def delete_edges(self, edges, mode=None) -> int:
        e = _e(edges)
        return self._chk(self._L.or_update_edges(self._h, DELETE, _p32(e), len(e), self.mode if mode is None else mode))

    def insert_vertices(self, nbr_lists, mode=None) -> int:
        lens = [len(x) for x in nbr_lists]
        off = np.zeros(len(lens) + 1, dtype=np.int64)
        off[1:] = np.cumsum(lens)
        nb = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.int32) for x in nbr_lists])
                                  if lens and off[-1] else np.zeros(0, dtype=np.int32))
        rc = self._L.or_insert_vertices(self._h, len(lens), off.ctypes.data_as(_i64p), _p32(nb),
                                        self.mode if mode is None else mode)
        return self._chk(rc)

    def delete_vertices(self, ids, mode=None) -> int:
        a = np.ascontiguousarray(ids, dtype=np.int32)
        return self._chk(self._L.or_delete_vertices(self._h, len(a), _p32(a), self.mode if mode is None else mode))

    def restore(self, op: int, edges, cores) -> None:
        """Puts the graph back into a saved state: applies `edges` to the
        structure only (op INSERT adds them, DELETE removes them; each must
        be absent, resp. present) and overwrites the cores with `cores`, the
        saved core numbers of that state.  No maintenance runs."""
        e = _e(edges)
        c = np.ascontiguousarray(cores, dtype=np.int32)
        if len(c) != self.n:
            raise ValueError("cores must cover every vertex")
        self._L.or_apply_structure(self._h, int(op), _p32(e), len(e))
        self._L.or_set_cores(self._h, _p32(c))

    def last_iterations(self) -> int:
        return int(self._L.or_last_iterations(self._h))

    def last_log(self) -> np.ndarray:
        cnt = int(self._L.or_last_log(self._h, None, 0))
        out = np.empty((max(cnt, 1), 2), dtype=np.int64)
        self._L.or_last_log(self._h, out.ctypes.data_as(_i64p), cnt)
        return out[:cnt]

    # stepper for per-iteration invariant checks
    def batch_begin(self, op: int, edges) -> int:
        e = _e(edges)
        self._bcap = self._chk(self._L.or_batch_begin(self._h, op, _p32(e), len(e)))
        return self._bcap

    def batch_step(self):
        """Runs one superior-edge-set iteration; returns (selected pairs,
        changed vertices) or None when no edges remain."""
        cap = getattr(self, "_bcap", 0) + 8
        sel = np.empty((cap, 2), dtype=np.int32)
        chg = np.empty(self.n + 1, dtype=np.int32)
        ns = ctypes.c_int64(0)
        nc = ctypes.c_int64(0)
        r = self._L.or_batch_step(self._h, _p32(sel), ctypes.byref(ns), _p32(chg), ctypes.byref(nc))
        if r == 0:
            return None
        return sel[: ns.value].copy(), chg[: nc.value].copy()
