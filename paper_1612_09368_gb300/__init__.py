"""GB300-native batched k-core maintenance by superior edge sets.

Thin Python binding over the C ABI declared in include/coremaint.h
(libcoremaint.so, built by ``build.build()``).  Every function here only
marshals arguments -- numpy arrays, torch tensors (CPU or CUDA) and streams
-- into the C calls of the same name; all graph work runs in the library's
CUDA kernels.  Importing fails loudly when the library is missing.

Method: N. Wang et al., "Parallel Algorithms for Core Maintenance in Dynamic
Graphs" (arXiv 1612.09368): superior edge sets (Section IV), incremental
maintenance (Section V, Algorithms 1-4), decremental maintenance (Section VI,
Algorithms 5-7), vertex operations reduced to edge operations (Section I).
"""
from __future__ import annotations

import ctypes
import weakref
import os

import numpy as np

from . import build as _build

__all__ = [
    "CM_OK", "CM_ERR_INVALID", "CM_ERR_OOM", "CM_ERR_CAPACITY", "CM_ERR_LIMIT", "CM_ERR_CUDA", "CM_ERR_STATE",
    "CM_OP_INSERT", "CM_OP_DELETE", "CM_DEBUG_BARRIER_NEVER_RELEASES", "CM_DEBUG_ITER_CAP",
    "CM_DEBUG_TASK_WAIT_NEVER_ENDS", "CM_DEBUG_CHECK_ITERATIONS", "CoreMaintError", "cm_options", "cm_stats",
    "cm_check_report", "cm_check",
    "lib", "library_path", "cm_default_options", "cm_create", "cm_create_multi", "cm_destroy", "cm_insert_edges",
    "cm_delete_edges", "cm_insert_vertices", "cm_insert_vertex", "cm_delete_vertices", "cm_delete_vertex",
    "cm_get_cores", "cm_get_superior_degrees", "cm_get_edges", "cm_num_vertices", "cm_num_edges", "cm_apply_edges", "cm_recompute_cores",
    "cm_get_stats", "cm_set_stream", "cm_last_error", "cm_multi_bases", "cm_update_multi", "CoreGraph",
]

CM_OK = 0
CM_ERR_INVALID = -1
CM_ERR_OOM = -2
CM_ERR_CAPACITY = -3
CM_ERR_LIMIT = -4
CM_ERR_CUDA = -5
CM_ERR_STATE = -6
CM_OP_INSERT = 0
CM_OP_DELETE = 1
CM_DEBUG_BARRIER_NEVER_RELEASES = 1
CM_DEBUG_ITER_CAP = 2
CM_DEBUG_TASK_WAIT_NEVER_ENDS = 4
CM_DEBUG_CHECK_ITERATIONS = 8
CM_SELECT_HASH = 0
CM_SELECT_KEY = 1

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class cm_options(ctypes.Structure):
    _fields_ = [
        ("slack_pct", ctypes.c_int32), ("min_cap", ctypes.c_int32), ("block_threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32), ("max_sms", ctypes.c_int32), ("block_mode_edges", ctypes.c_int32),
        ("spin_limit_ns", ctypes.c_int64), ("alloc", _ALLOC_FN), ("free", _FREE_FN), ("alloc_ctx", ctypes.c_void_p),
        ("debug_flags", ctypes.c_int32), ("block_mode_enter", ctypes.c_int32), ("block_mode_leave", ctypes.c_int32),
        ("hub_slots", ctypes.c_int32), ("block_slots", ctypes.c_int32), ("block_slots_delete", ctypes.c_int32),
        ("task_claim", ctypes.c_int32), ("select_order", ctypes.c_int32), ("select_rounds", ctypes.c_int32),
        ("expand_early", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2),
    ]


class cm_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "applied", "iterations", "select_rounds", "selected", "remaining_sum", "visited", "visited_slots",
        "evicted", "evicted_slots", "changed", "changed_slots", "waves", "alg_bytes", "launches")] + [
        ("maintain_ms", ctypes.c_double), ("call_ms", ctypes.c_double), ("peel_levels", ctypes.c_int64),
        ("barriers", ctypes.c_int64), ("grid_iterations", ctypes.c_int64), ("phase_ns", ctypes.c_int64 * 7),
        ("reserved", ctypes.c_int64 * 4)]

    PHASES = ("claim", "check", "apply", "discover", "evict", "commit", "fixup")

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "phase_ns")}
        d["phase_ns"] = dict(zip(self.PHASES, list(self.phase_ns)))
        return d


class cm_check_report(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "vertices_checked", "sd_mismatches", "key_mismatches", "degree_mismatches", "bad_neighbour_ids",
        "kcore_violations", "first_bad_vertex", "reserved")]


class cm_step_config(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in (
        "block_mode_edges", "block_mode_enter", "block_mode_leave", "hub_slots", "blocks_per_sm", "block_slots",
        "task_claim", "reserved")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class cm_tune_report(ctypes.Structure):
    _fields_ = [("best", cm_step_config), ("best_ms", ctypes.c_double), ("first_ms", ctypes.c_double),
                ("tried", ctypes.c_int32), ("reps", ctypes.c_int32)]


class cm_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("pad", ctypes.c_int32)] + [
        (k, ctypes.c_int64) for k in ("round", "round_applied", "round_edges", "round_requests", "latency_ns",
                                      "queue_ns")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class cm_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "rounds", "coalesced", "failed", "edges",
                                              "p50_ns", "p99_ns")] + [("reserved", ctypes.c_int64 * 4)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class CoreMaintError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None
library_path = _build.LIB


def lib():
    """The loaded libcoremaint.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(f"{library_path} is missing: run paper_1612_09368_gb300.build.build() "
                              "(needs nvcc); there is no CPU fallback")
        L = ctypes.CDLL(library_path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        p32 = ctypes.POINTER(ctypes.c_int32)
        p64 = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "cm_default_options": (None, [ctypes.POINTER(cm_options)]),
            "cm_create": (ctypes.c_int, [ctypes.POINTER(vp), i32, vp, i64, vp, ctypes.POINTER(cm_options), vp]),
            "cm_create_multi": (ctypes.c_int, [ctypes.POINTER(vp), i32, p32, p64, vp, vp,
                                               ctypes.POINTER(cm_options), vp]),
            "cm_destroy": (None, [vp]),
            "cm_insert_edges": (ctypes.c_int, [vp, vp, i64, p64]),
            "cm_delete_edges": (ctypes.c_int, [vp, vp, i64, p64]),
            "cm_insert_vertices": (ctypes.c_int, [vp, i32, vp, vp, p32, p64]),
            "cm_insert_vertex": (ctypes.c_int, [vp, vp, i32, p32]),
            "cm_delete_vertices": (ctypes.c_int, [vp, i32, vp, p64]),
            "cm_delete_vertex": (ctypes.c_int, [vp, i32]),
            "cm_get_cores": (ctypes.c_int, [vp, vp, p32]),
            "cm_get_edges": (ctypes.c_int, [vp, vp, i64, p64]),
            "cm_get_superior_degrees": (ctypes.c_int, [vp, vp, p32]),
            "cm_check": (ctypes.c_int, [vp, ctypes.POINTER(cm_check_report)]),
            "cm_num_vertices": (i32, [vp]),
            "cm_num_edges": (i64, [vp]),
            "cm_apply_edges": (ctypes.c_int, [vp, i32, vp, i64, p64]),
            "cm_recompute_cores": (ctypes.c_int, [vp]),
            "cm_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(cm_stats)]),
            "cm_set_stream": (ctypes.c_int, [vp, vp]),
            "cm_last_error": (ctypes.c_char_p, [vp]),
            "cm_multi_bases": (ctypes.c_int, [vp, p32, p32]),
            "cm_update_multi": (ctypes.c_int, [vp, i32, p64, vp, p64]),
            "cm_step_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, i64, i64, ctypes.POINTER(cm_step_config)]),
            "cm_step_run": (ctypes.c_int, [vp, p64, vp, p64, vp, p64, p64]),
            "cm_step_get_config": (ctypes.c_int, [vp, ctypes.POINTER(cm_step_config)]),
            "cm_step_set_config": (ctypes.c_int, [vp, ctypes.POINTER(cm_step_config)]),
            "cm_step_counters": (ctypes.c_int, [vp, p64, p64, p64]),
            "cm_step_autotune": (ctypes.c_int, [vp, p64, vp, p64, vp, i32, ctypes.POINTER(cm_tune_report)]),
            "cm_step_destroy": (None, [vp]),
            "cm_server_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), i32, i64, i64]),
            "cm_server_submit": (ctypes.c_int, [vp, i32, i32, vp, i64, p64]),
            "cm_server_wait": (ctypes.c_int, [vp, i64, ctypes.POINTER(cm_request_result)]),
            "cm_server_drain": (ctypes.c_int, [vp]),
            "cm_server_get_cores": (ctypes.c_int, [vp, i32, vp]),
            "cm_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(cm_server_stats)]),
            "cm_server_run_trace": (ctypes.c_int, [vp, i64, vp, vp, vp, vp, vp, vp, vp,
                                                   ctypes.POINTER(ctypes.c_double)]),
            "cm_server_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------- marshalling
def _arr(x, dtype):
    """(pointer, keepalive) for a host numpy array or a torch tensor."""
    if x is None:
        return None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            tdt = torch.int32 if dtype == np.int32 else torch.int64
            t = x.to(tdt).contiguous()
            return ctypes.c_void_p(t.data_ptr()), t
    except ImportError:
        pass
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return ctypes.c_void_p(a.ctypes.data), a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(h, rc, what):
    if rc != CM_OK:
        msg = lib().cm_last_error(h)
        raise CoreMaintError(rc, f"{what}: {msg.decode() if msg else ''}")
    return rc


def _npairs(x) -> int:
    shape = getattr(x, "shape", None)
    if shape is not None and len(shape) == 2:
        return int(shape[0])
    return len(x) // 2 if not hasattr(x, "numel") else int(x.numel()) // 2


# Device allocation through torch's caching allocator.
class _TorchAllocator:
    def __init__(self):
        import torch
        self._torch = torch

        def _alloc(size, stream, ctx):
            try:
                return int(self._torch.cuda.caching_allocator_alloc(int(size), stream=int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, size, stream, ctx):
            self._torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _ALLOC_FN(_alloc)
        self.free = _FREE_FN(_free)


# ---------------------------------------------------------------- C-named functions
def cm_default_options() -> cm_options:
    o = cm_options()
    lib().cm_default_options(ctypes.byref(o))
    return o


def cm_create(n, edges, cores=None, options: cm_options | None = None, stream=None):
    h = ctypes.c_void_p()
    ep, ek = _arr(edges, np.int32)
    cp, ck = _arr(cores, np.int32)
    m = _npairs(edges) if edges is not None else 0
    rc = lib().cm_create(ctypes.byref(h), int(n), ep, m, cp, ctypes.byref(options) if options else None,
                         _stream(stream))
    _check(None, rc, "cm_create")
    return h


def cm_create_multi(ns, ms, edges, cores=None, options: cm_options | None = None, stream=None):
    h = ctypes.c_void_p()
    nsa = np.ascontiguousarray(ns, dtype=np.int32)
    msa = np.ascontiguousarray(ms, dtype=np.int64)
    ep, ek = _arr(edges, np.int32)
    cp, ck = _arr(cores, np.int32)
    rc = lib().cm_create_multi(ctypes.byref(h), len(nsa), nsa.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               msa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ep, cp,
                               ctypes.byref(options) if options else None, _stream(stream))
    _check(None, rc, "cm_create_multi")
    return h


def cm_destroy(h):
    lib().cm_destroy(h)


def _upd(fn, h, edges, what):
    ep, keep = _arr(edges, np.int32)
    applied = ctypes.c_int64(0)
    _check(h, fn(h, ep, _npairs(edges), ctypes.byref(applied)), what)
    return applied.value


def cm_insert_edges(h, edges) -> int:
    return _upd(lib().cm_insert_edges, h, edges, "cm_insert_edges")


def cm_delete_edges(h, edges) -> int:
    return _upd(lib().cm_delete_edges, h, edges, "cm_delete_edges")


def cm_apply_edges(h, op, edges) -> int:
    ep, keep = _arr(edges, np.int32)
    applied = ctypes.c_int64(0)
    _check(h, lib().cm_apply_edges(h, int(op), ep, _npairs(edges), ctypes.byref(applied)), "cm_apply_edges")
    return applied.value


def cm_insert_vertices(h, nbr_off, nbrs):
    """Returns (first new id, edges applied)."""
    op, ok = _arr(nbr_off, np.int64)
    npt, nk = _arr(nbrs, np.int32)
    count = (len(nbr_off) if not hasattr(nbr_off, "numel") else int(nbr_off.numel())) - 1
    first = ctypes.c_int32(0)
    applied = ctypes.c_int64(0)
    _check(h, lib().cm_insert_vertices(h, count, op, npt, ctypes.byref(first), ctypes.byref(applied)),
           "cm_insert_vertices")
    return first.value, applied.value


def cm_insert_vertex(h, nbrs) -> int:
    npt, nk = _arr(nbrs, np.int32)
    d = len(nbrs) if not hasattr(nbrs, "numel") else int(nbrs.numel())
    vid = ctypes.c_int32(0)
    _check(h, lib().cm_insert_vertex(h, npt, d, ctypes.byref(vid)), "cm_insert_vertex")
    return vid.value


def cm_delete_vertices(h, ids) -> int:
    ip, ik = _arr(ids, np.int32)
    count = len(ids) if not hasattr(ids, "numel") else int(ids.numel())
    applied = ctypes.c_int64(0)
    _check(h, lib().cm_delete_vertices(h, count, ip, ctypes.byref(applied)), "cm_delete_vertices")
    return applied.value


def cm_delete_vertex(h, v: int):
    _check(h, lib().cm_delete_vertex(h, int(v)), "cm_delete_vertex")


def cm_num_vertices(h) -> int:
    return int(lib().cm_num_vertices(h))


def cm_num_edges(h) -> int:
    return int(lib().cm_num_edges(h))


def cm_get_cores(h, out=None):
    """Core numbers (dead vertices -1) into `out` (a torch tensor, host or
    CUDA) or a new numpy array."""
    n = cm_num_vertices(h)
    if out is None:
        out = np.empty(n, dtype=np.int32)
        _check(h, lib().cm_get_cores(h, ctypes.c_void_p(out.ctypes.data), None), "cm_get_cores")
        return out
    _check(h, lib().cm_get_cores(h, ctypes.c_void_p(out.data_ptr()), None), "cm_get_cores")
    return out


def cm_get_superior_degrees(h, out=None):
    """SD (Definition 7) of every vertex (dead -1) into `out` (a torch tensor,
    host or CUDA) or a new numpy array."""
    n = cm_num_vertices(h)
    if out is None:
        out = np.empty(n, dtype=np.int32)
        _check(h, lib().cm_get_superior_degrees(h, ctypes.c_void_p(out.ctypes.data), None),
               "cm_get_superior_degrees")
        return out
    _check(h, lib().cm_get_superior_degrees(h, ctypes.c_void_p(out.data_ptr()), None), "cm_get_superior_degrees")
    return out


def cm_check(h) -> dict:
    """Consistency of the device store with its definitions (SD recount,
    scan keys, degrees, neighbour ids, the k-core condition), as a dict of
    cm_check_report's fields."""
    r = cm_check_report()
    _check(h, lib().cm_check(h, ctypes.byref(r)), "cm_check")
    return {name: getattr(r, name) for name, _ in r._fields_ if name != "reserved"}


def cm_get_edges(h) -> np.ndarray:
    m = cm_num_edges(h)
    out = np.empty((max(m, 0), 2), dtype=np.int32)
    got = ctypes.c_int64(0)
    _check(h, lib().cm_get_edges(h, ctypes.c_void_p(out.ctypes.data), m, ctypes.byref(got)), "cm_get_edges")
    return out


def cm_recompute_cores(h):
    _check(h, lib().cm_recompute_cores(h), "cm_recompute_cores")


def cm_get_stats(h) -> dict:
    s = cm_stats()
    _check(h, lib().cm_get_stats(h, ctypes.byref(s)), "cm_get_stats")
    return s.as_dict()


def cm_set_stream(h, stream):
    _check(h, lib().cm_set_stream(h, _stream(stream)), "cm_set_stream")


def cm_last_error(h) -> str:
    m = lib().cm_last_error(h)
    return m.decode() if m else ""


def cm_multi_bases(h) -> np.ndarray:
    ng = ctypes.c_int32(0)
    lib().cm_multi_bases(h, None, ctypes.byref(ng))
    out = np.empty(ng.value, dtype=np.int32)
    lib().cm_multi_bases(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(ng))
    return out


def cm_update_multi(h, op, counts, edges) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.int64)
    ep, ek = _arr(edges, np.int32)
    out = np.zeros(len(c), dtype=np.int64)
    _check(h, lib().cm_update_multi(h, int(op), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ep,
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "cm_update_multi")
    return out


def _counts(c, ng):
    if c is None:
        return None, None
    a = np.ascontiguousarray(c, dtype=np.int64)
    if len(a) != ng:
        raise ValueError(f"{len(a)} counts for {ng} graphs")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), a


def cm_step_create(h, max_insert, max_delete, config: cm_step_config | None = None):
    s = ctypes.c_void_p()
    _check(h, lib().cm_step_create(ctypes.byref(s), h, int(max_insert), int(max_delete),
                                   ctypes.byref(config) if config is not None else None), "cm_step_create")
    return s


def cm_step_run(h, s, ng, ins_counts, ins_edges, del_counts, del_edges):
    """Returns (per-graph inserted, per-graph deleted) as int64 arrays."""
    ic, ick = _counts(ins_counts, ng)
    dc, dck = _counts(del_counts, ng)
    ip, ik = _arr(ins_edges, np.int32)
    dp, dk = _arr(del_edges, np.int32)
    ia = np.zeros(ng, dtype=np.int64)
    da = np.zeros(ng, dtype=np.int64)
    _check(h, lib().cm_step_run(s, ic, ip, dc, dp, ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                da.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "cm_step_run")
    return ia, da


def cm_step_autotune(h, s, ng, ins_counts, ins_edges, del_counts, del_edges, reps=2) -> dict:
    ic, ick = _counts(ins_counts, ng)
    dc, dck = _counts(del_counts, ng)
    ip, ik = _arr(ins_edges, np.int32)
    dp, dk = _arr(del_edges, np.int32)
    r = cm_tune_report()
    _check(h, lib().cm_step_autotune(s, ic, ip, dc, dp, int(reps), ctypes.byref(r)), "cm_step_autotune")
    return {"best": r.best.as_dict(), "best_ms": r.best_ms, "first_ms": r.first_ms, "tried": r.tried,
            "reps": r.reps}


def cm_step_get_config(s) -> cm_step_config:
    c = cm_step_config()
    lib().cm_step_get_config(s, ctypes.byref(c))
    return c


def cm_step_set_config(s, config: cm_step_config):
    lib().cm_step_set_config(s, ctypes.byref(config))


def cm_step_counters(s) -> dict:
    a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    lib().cm_step_counters(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return {"captures": a.value, "replays": b.value, "fallbacks": c.value}


def cm_step_destroy(s):
    lib().cm_step_destroy(s)


# ---------------------------------------------------------------- convenience object
class CoreGraph:
    """Owning wrapper: a graph resident on the GPU with maintained cores."""

    def __init__(self, n, edges, cores=None, *, stream=None, use_torch_allocator=True, multi=None, allocator=None,
                 **opts):
        """allocator: an object whose ``alloc`` / ``free`` attributes are the
        cm_alloc_fn / cm_free_fn callbacks (kept alive by this wrapper);
        otherwise torch's caching allocator (use_torch_allocator) or
        cudaMalloc."""
        o = cm_default_options()
        for k, v in opts.items():
            setattr(o, k, v)
        self._alloc = None
        if allocator is not None:
            self._alloc = allocator
        elif use_torch_allocator:
            self._alloc = _TorchAllocator()
        if self._alloc is not None:
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        self.options = o
        self._stream = stream
        self._steps = weakref.WeakSet()
        if multi is not None:
            ns, ms = multi
            self._h = cm_create_multi(ns, ms, edges, cores, o, stream)
        else:
            self._h = cm_create(n, edges, cores, o, stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            for st in list(getattr(self, "_steps", ())):
                st.close()
            cm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def n(self) -> int:
        return cm_num_vertices(self._h)

    @property
    def m(self) -> int:
        return cm_num_edges(self._h)

    def insert_edges(self, edges) -> int:
        return cm_insert_edges(self._h, edges)

    def delete_edges(self, edges) -> int:
        return cm_delete_edges(self._h, edges)

    def apply_edges(self, op, edges) -> int:
        return cm_apply_edges(self._h, op, edges)

    def insert_vertices(self, nbr_lists):
        lens = [len(x) for x in nbr_lists]
        off = np.zeros(len(lens) + 1, dtype=np.int64)
        off[1:] = np.cumsum(lens)
        nb = (np.concatenate([np.asarray(x, dtype=np.int32) for x in nbr_lists]) if off[-1]
              else np.zeros(0, dtype=np.int32))
        return cm_insert_vertices(self._h, off, nb)

    def delete_vertices(self, ids) -> int:
        return cm_delete_vertices(self._h, ids)

    def cores(self, out=None):
        return cm_get_cores(self._h, out)

    def superior_degrees(self, out=None):
        return cm_get_superior_degrees(self._h, out)

    def check(self) -> dict:
        return cm_check(self._h)

    def edges(self) -> np.ndarray:
        return cm_get_edges(self._h)

    def recompute_cores(self):
        cm_recompute_cores(self._h)

    def stats(self) -> dict:
        return cm_get_stats(self._h)

    def bases(self) -> np.ndarray:
        return cm_multi_bases(self._h)

    def update_multi(self, op, counts, edges) -> np.ndarray:
        return cm_update_multi(self._h, op, counts, edges)

    def step(self, max_insert, max_delete, config: cm_step_config | None = None) -> "Step":
        return Step(self, max_insert, max_delete, config)


class Step:
    """A captured update step of a CoreGraph (see cm_step_create): one
    insert batch then one delete batch per graph, one CUDA graph replay."""

    def __init__(self, graph: CoreGraph, max_insert, max_delete, config: cm_step_config | None = None):
        self.graph = graph
        self.ngraphs = len(graph.bases())
        self._s = cm_step_create(graph.handle, max_insert, max_delete, config)
        graph._steps.add(self)

    def run(self, ins_counts=None, ins_edges=None, del_counts=None, del_edges=None):
        return cm_step_run(self.graph.handle, self._s, self.ngraphs, ins_counts, ins_edges, del_counts, del_edges)

    def autotune(self, ins_counts=None, ins_edges=None, del_counts=None, del_edges=None, reps=2) -> dict:
        return cm_step_autotune(self.graph.handle, self._s, self.ngraphs, ins_counts, ins_edges, del_counts,
                                del_edges, reps)

    @property
    def config(self) -> cm_step_config:
        return cm_step_get_config(self._s)

    @config.setter
    def config(self, c: cm_step_config):
        cm_step_set_config(self._s, c)

    def counters(self) -> dict:
        return cm_step_counters(self._s)

    def close(self):
        if getattr(self, "_s", None):
            cm_step_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop over resident graphs (see cm_server_create): update
    batches are admitted into each graph's slice of a device budget as
    room frees up, consecutive same-operation requests are coalesced into
    one maintenance call, and graphs are served concurrently."""

    def __init__(self, graphs, device_budget_bytes: int, max_round_edges: int = 0):
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle.value for g in self.graphs])
        self._s = ctypes.c_void_p()
        rc = lib().cm_server_create(ctypes.byref(self._s), arr, len(self.graphs), int(device_budget_bytes),
                                    int(max_round_edges))
        if rc != CM_OK:
            raise CoreMaintError(rc, "cm_server_create")

    def submit(self, graph: int, op: int, edges) -> int:
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        rid = ctypes.c_int64(0)
        rc = lib().cm_server_submit(self._s, int(graph), int(op), ctypes.c_void_p(e.ctypes.data), len(e),
                                    ctypes.byref(rid))
        if rc != CM_OK:
            raise CoreMaintError(rc, "cm_server_submit")
        return rid.value

    def wait(self, request_id: int) -> dict:
        r = cm_request_result()
        lib().cm_server_wait(self._s, int(request_id), ctypes.byref(r))
        return r.as_dict()

    def drain(self) -> int:
        return int(lib().cm_server_drain(self._s))

    def cores(self, graph: int) -> np.ndarray:
        out = np.empty(cm_num_vertices(self.graphs[graph].handle), dtype=np.int32)
        rc = lib().cm_server_get_cores(self._s, int(graph), ctypes.c_void_p(out.ctypes.data))
        if rc != CM_OK:
            raise CoreMaintError(rc, "cm_server_get_cores")
        return out

    def stats(self) -> dict:
        st = cm_server_stats()
        lib().cm_server_get_stats(self._s, ctypes.byref(st))
        return st.as_dict()

    def run_trace(self, arrival_ns, graph, op, counts, edges):
        """Open-loop replay; returns (latency_ns, round_of, wall_s)."""
        a = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        gr = np.ascontiguousarray(graph, dtype=np.int32)
        o = np.ascontiguousarray(op, dtype=np.int32)
        c = np.ascontiguousarray(counts, dtype=np.int64)
        e = np.ascontiguousarray(edges, dtype=np.int32)
        lat = np.zeros(len(a), dtype=np.int64)
        rnd = np.zeros(len(a), dtype=np.int64)
        wall = ctypes.c_double(0)
        rc = lib().cm_server_run_trace(self._s, len(a), ctypes.c_void_p(a.ctypes.data),
                                       ctypes.c_void_p(gr.ctypes.data), ctypes.c_void_p(o.ctypes.data),
                                       ctypes.c_void_p(c.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                                       ctypes.c_void_p(lat.ctypes.data), ctypes.c_void_p(rnd.ctypes.data),
                                       ctypes.byref(wall))
        if rc != CM_OK:
            raise CoreMaintError(rc, "cm_server_run_trace")
        return lat, rnd, wall.value

    def close(self):
        if getattr(self, "_s", None):
            lib().cm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
