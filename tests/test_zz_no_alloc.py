"""cm_core_numbers_noalloc: the decomposition entry point that allocates no
device memory, for callers that cannot call cudaMalloc (a framework that
already reserved the device memory for its own pool, or a loop that must not
wait on the allocator, since cudaMalloc / cudaFree may synchronise the
device).  Its output must equal, exactly, both the core numbers the regular
graph store computes (cm_create + cm_get_cores) and the CPU oracle's
Batagelj-Zaversnik peeling, on calls in a row that share the static scratch
array.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def noalloc():
    import torch
    from paper_1612_09368_gb300 import build
    build.build()
    import paper_1612_09368_gb300 as cm

    f = cm.lib().cm_core_numbers_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    torch.cuda.set_device(0)
    return cm, f


def _run(f, n, row_off, adj, stream):
    import torch
    d_off = torch.from_numpy(row_off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    rc = f(n, d_off.data_ptr(), d_adj.data_ptr(), out.data_ptr(), stream.cuda_stream)
    return rc, out.cpu().numpy()


def test_noalloc_matches_store_and_oracle_on_calls_in_a_row(noalloc):
    import torch
    cm, f = noalloc
    stream = torch.cuda.current_stream()
    graphs = [(1 << 15, synth.rmat(15, 16, synth.stream(90, 0))),
              (30000, synth.er(30000, 120000, synth.stream(90, 1))),
              (1 << 20, synth.rmat(20, 16, synth.stream(90, 2)))]   # n at the documented maximum
    for n, e in graphs:          # calls in a row share the scratch array
        row_off, adj = _csr(n, e)
        rc, got = _run(f, n, row_off, adj, stream)
        assert rc == cm.CM_OK
        assert (got == cm.CoreGraph(n, e).cores()).all()
        assert (got == oracle.bz(n, e)).all()


def test_noalloc_allocates_nothing(noalloc):
    """After a first call (which looks up the scratch array's address), a
    call changes neither torch's allocated bytes nor the device's free
    memory."""
    import torch
    cm, f = noalloc
    n = 1 << 14
    e = synth.rmat(14, 16, synth.stream(90, 3))
    row_off, adj = _csr(n, e)
    d_off = torch.from_numpy(row_off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    assert f(n, d_off.data_ptr(), d_adj.data_ptr(), out.data_ptr(), s.cuda_stream) == cm.CM_OK
    torch.cuda.synchronize()
    a0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert f(n, d_off.data_ptr(), d_adj.data_ptr(), out.data_ptr(), s.cuda_stream) == cm.CM_OK
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0
    assert torch.cuda.mem_get_info()[0] == free0
    assert (out.cpu().numpy() == oracle.bz(n, e)).all()


def test_noalloc_rejects_bad_arguments(noalloc):
    import torch
    cm, f = noalloc
    t = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert f((1 << 20) + 1, t.data_ptr(), t.data_ptr(), t.data_ptr(), None) == cm.CM_ERR_CAPACITY
    assert f(-1, t.data_ptr(), t.data_ptr(), t.data_ptr(), None) == cm.CM_ERR_INVALID
    assert f(3, None, t.data_ptr(), t.data_ptr(), None) == cm.CM_ERR_INVALID
    host = np.zeros(4, dtype=np.int32)          # host memory is refused, not read
    assert f(3, t.data_ptr(), host.ctypes.data, t.data_ptr(), None) == cm.CM_ERR_INVALID
    assert f(0, None, None, None, None) == cm.CM_OK
    # the device is still usable
    n, e = 2000, synth.er(2000, 8000, synth.stream(90, 4))
    rc, got = _run(f, n, *_csr(n, e), torch.cuda.current_stream())
    assert rc == cm.CM_OK and (got == oracle.bz(n, e)).all()
