"""cm_core_numbers_noalloc: the decomposition entry point that allocates no
device memory, for callers that cannot call cudaMalloc (a framework that
already reserved the device memory for its pool, or a loop that must not
wait on the allocator).  Its output must equal the core numbers the regular
graph store computes (cm_create + cm_get_cores), exactly, on two calls in a
row that share the static scratch array.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _csr(n, edges):
    e = np.asarray(edges, dtype=np.int64)
    src = np.concatenate([e[:, 0], e[:, 1]])
    dst = np.concatenate([e[:, 1], e[:, 0]])
    order = np.argsort(src, kind="stable")
    adj = dst[order].astype(np.int32)
    deg = np.bincount(src, minlength=n)
    row_off = np.zeros(n + 1, dtype=np.int64)
    row_off[1:] = np.cumsum(deg)
    return row_off, adj


def test_noalloc_matches_store_on_two_calls_in_a_row():
    import torch
    from paper_1612_09368_gb300 import build
    build.build()
    import paper_1612_09368_gb300 as cm

    f = cm.lib().cm_core_numbers_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    graphs = [(1 << 15, synth.rmat(15, 16, synth.stream(90, 0))),
              (30000, synth.er(30000, 120000, synth.stream(90, 1)))]
    for n, e in graphs:          # two calls in a row share the scratch array
        row_off, adj = _csr(n, e)
        d_off = torch.from_numpy(row_off).cuda()
        d_adj = torch.from_numpy(adj).cuda()
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        rc = f(n, d_off.data_ptr(), d_adj.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == cm.CM_OK
        ref = cm.CoreGraph(n, e).cores()
        assert (out.cpu().numpy() == ref).all()


def test_noalloc_rejects_too_many_vertices():
    import torch
    import paper_1612_09368_gb300 as cm

    f = cm.lib().cm_core_numbers_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    t = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert f((1 << 20) + 1, t.data_ptr(), t.data_ptr(), t.data_ptr(), None) == cm.CM_ERR_CAPACITY
