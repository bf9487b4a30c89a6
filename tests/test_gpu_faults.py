"""Failure handling of the library, with no GPU fault ever caused.

* A device allocation that fails (the caller's allocator callback returns
  NULL at the N-th request) makes the call return CM_ERR_OOM with the graph
  exactly as before -- edges, cores and superior degrees -- and the same
  call succeeds once memory is available again.
* A maintenance call whose iteration cap is forced to one, and a grid-mode
  search whose task queue can never become quiescent, stop within their
  limits with CM_ERR_LIMIT (the handle is poisoned, the device stays
  usable).
Core numbers are checked against the CPU oracle throughout."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cm():
    import torch
    from paper_1612_09368_gb300 import build
    build.build()
    import paper_1612_09368_gb300 as cm
    torch.cuda.set_device(0)
    return cm


class FailingAllocator:
    """Device memory from torch's caching allocator; the request numbered
    `fail_at` (counting from 1 since the allocator was made) gets NULL."""

    def __init__(self, cm):
        import torch
        self.count = 0
        self.fail_at = None
        self.failed = 0

        def _alloc(size, stream, ctx):
            self.count += 1
            if self.fail_at is not None and self.count == self.fail_at:
                self.failed += 1
                return None
            return int(torch.cuda.caching_allocator_alloc(int(size), stream=int(stream or 0)))

        def _free(ptr, size, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = cm._ALLOC_FN(_alloc)
        self.free = cm._FREE_FN(_free)


def _keys(e):
    e = np.asarray(e, dtype=np.int64).reshape(-1, 2)
    return np.sort((np.minimum(e[:, 0], e[:, 1]) << 32) | np.maximum(e[:, 0], e[:, 1]))


def _state(g):
    return g.n, _keys(g.edges()), g.cores().copy(), g.superior_degrees().copy()


def _same(a, b):
    return a[0] == b[0] and all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))


def test_allocation_failure_leaves_the_graph_unchanged(cm):
    n = 3000
    e = synth.ba(n, 4, synth.stream(80))
    ins = synth.static_sample_insert(n, e, 20000, synth.PREFERENTIAL, synth.stream(80, 0, 0, synth.INSERT))
    dele = synth.static_sample_delete(n, e, 4000, synth.PREFERENTIAL, synth.stream(80, 0, 0, synth.DELETE))
    rng = np.random.default_rng(80)
    nv = 2500            # more new vertices than the vertex arrays' headroom: they must grow
    vnb = [rng.choice(n, 12, replace=False).tolist() for _ in range(nv)]
    vdel = np.arange(0, 60, dtype=np.int32)
    def ins_vertices(g):
        first, applied = g.insert_vertices(vnb)
        return applied

    def ins_vertices_ref(r):
        r.insert_vertices(vnb)
        return nv * 12           # every edge of a new vertex is new

    # (name, call, oracle call, allocations the call makes at least): the
    # insert grows the batch buffers, the edge index, the adjacency pool and
    # the task queue; the delete that follows it needs no new memory; a
    # vertex insertion grows the vertex arrays; a vertex deletion stages ids
    ops = [("insert", lambda g: g.insert_edges(ins), lambda r: r.insert_edges(ins), 3),
           ("delete", lambda g: g.delete_edges(dele), lambda r: r.delete_edges(dele), 0),
           ("insert vertices", ins_vertices, ins_vertices_ref, 1),
           ("delete vertices", lambda g: g.delete_vertices(vdel), lambda r: r.delete_vertices(vdel), 1)]
    for j, (name, run, run_ref, least) in enumerate(ops):
        failures = 0
        for nth in range(1, 64):
            alloc = FailingAllocator(cm)
            g = cm.CoreGraph(n, e, allocator=alloc)
            ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
            for _, prev, prev_ref, _ in ops[:j]:    # the state the op starts from
                prev(g)
                prev_ref(ref)
            before = _state(g)
            alloc.fail_at = alloc.count + nth
            try:
                got = run(g)
                ok = True
            except cm.CoreMaintError as ex:
                assert ex.code == cm.CM_ERR_OOM, (name, nth, ex)
                ok = False
            alloc.fail_at = None
            if ok:                                  # past the op's last allocation
                assert alloc.failed == 0
                g.close()
                break
            failures += 1
            assert _same(_state(g), before), f"{name}: allocation {nth} failed and the graph changed"
            assert run(g) == run_ref(ref), (name, nth)      # the same call, memory available again
            assert (g.cores() == ref.cores()).all(), (name, nth)
            g.close()
        assert failures >= least, f"{name}: only {failures} allocations failed"


def test_iteration_cap_returns_limit(cm):
    """A batch that needs several iterations (chords from one vertex of a
    cycle: every edge is constrained at that vertex, so one is selected per
    iteration) stops with CM_ERR_LIMIT when the cap is one iteration."""
    n = 200
    cyc = np.array([(i, (i + 1) % n) for i in range(n)], np.int32)
    chords = np.array([(0, j) for j in range(10, 60)], np.int32)
    g = cm.CoreGraph(n, cyc, debug_flags=cm.CM_DEBUG_ITER_CAP)
    with pytest.raises(cm.CoreMaintError) as ei:
        g.insert_edges(chords)
    assert ei.value.code == cm.CM_ERR_LIMIT
    with pytest.raises(cm.CoreMaintError) as ei:
        g.cores()
    assert ei.value.code == cm.CM_ERR_STATE
    g.close()
    g = cm.CoreGraph(n, cyc)
    ref = oracle.OracleGraph(n, cyc, mode=oracle.SUPERIOR)
    assert g.insert_edges(chords) == ref.insert_edges(chords)
    assert g.stats()["iterations"] == ref.last_iterations() > 1
    assert (g.cores() == ref.cores()).all()


def test_task_queue_wait_limit_returns_error(cm):
    """A grid-mode search that can never become quiescent (a task is counted
    that nobody queues): every warp's wait on the queue runs out after the
    handle's wait limit and the call returns CM_ERR_LIMIT; the device keeps
    working."""
    n = 4000
    e = synth.er(n, 16000, synth.stream(81))
    ins = synth.static_sample_insert(n, e, 500, synth.UNIFORM, synth.stream(81, 0, 0, synth.INSERT))
    g = cm.CoreGraph(n, e, spin_limit_ns=50_000_000, debug_flags=cm.CM_DEBUG_TASK_WAIT_NEVER_ENDS)
    t0 = time.time()
    with pytest.raises(cm.CoreMaintError) as ei:
        g.insert_edges(ins)
    assert ei.value.code == cm.CM_ERR_LIMIT
    assert time.time() - t0 < 30
    with pytest.raises(cm.CoreMaintError) as ei:
        g.cores()
    assert ei.value.code == cm.CM_ERR_STATE
    g.close()
    g = cm.CoreGraph(n, e)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    assert g.insert_edges(ins) == ref.insert_edges(ins)
    assert (g.cores() == ref.cores()).all()
