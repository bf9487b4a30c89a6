"""The store's consistency check (cm_check) and the debug mode that runs it
after every superior-edge-set iteration.  The check recounts SD (Section IV,
Definition 7) from scratch for every vertex and tests the scan keys, the
degrees, the neighbour ids and the k-core condition (Definition 1: a vertex
of core k has at least k neighbours of core >= k).  All of it must hold
after creation, after each batch, and after every iteration of insert,
delete and vertex-operation calls; the debug mode must reach the oracle's
cores and iteration counts."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

COUNTS = ("sd_mismatches", "key_mismatches", "degree_mismatches", "bad_neighbour_ids", "kcore_violations")


@pytest.fixture(scope="module")
def cm():
    import torch
    from paper_1612_09368_gb300 import build
    build.build()
    import paper_1612_09368_gb300 as cm
    torch.cuda.set_device(0)
    return cm


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _clean(report, n, what=""):
    assert report["vertices_checked"] == n, (what, report)
    for k in COUNTS:
        assert report[k] == 0, (what, k, report)
    assert report["first_bad_vertex"] == -1, (what, report)


def _graphs():
    rng = np.random.default_rng(900)
    iu = np.triu_indices(400, 1)
    keep = rng.random(len(iu[0])) < 0.05
    yield "random", 400, np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int32)
    yield "rmat", 1 << 13, synth.rmat(13, 16, synth.stream(901))
    yield "ba", 20000, synth.ba(20000, 6, synth.stream(902))


def test_check_after_create_and_batches(cm):
    for name, n, e in _graphs():
        g = cm.CoreGraph(n, _dev(e))
        _clean(g.check(), n, f"{name} create")
        ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
        for law in (synth.UNIFORM, synth.PREFERENTIAL):
            ins = synth.static_sample_insert(n, ref.edges(), 2000, law, synth.stream(903, n, law, synth.INSERT))
            assert g.insert_edges(_dev(ins)) == ref.insert_edges(ins)
            _clean(g.check(), n, f"{name} insert law {law}")
            dl = synth.static_sample_delete(n, ref.edges(), 2000, synth.PREFERENTIAL,
                                            synth.stream(903, n, law, synth.DELETE))
            assert g.delete_edges(_dev(dl)) == ref.delete_edges(dl)
            _clean(g.check(), n, f"{name} delete law {law}")
        assert (g.cores() == ref.cores()).all(), name


def test_debug_mode_checks_every_iteration(cm):
    """Degree-proportional batches need several iterations; in the debug
    mode each one ends its own launch pair and the store is checked before
    the next (a failed check fails the call), with the normal mode's
    iteration counts and the oracle's cores."""
    for name, n, e in _graphs():
        g = cm.CoreGraph(n, _dev(e), debug_flags=cm.CM_DEBUG_CHECK_ITERATIONS)
        ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
        for law in (synth.PREFERENTIAL, synth.UNIFORM):
            ins = synth.static_sample_insert(n, ref.edges(), 3000, law, synth.stream(904, n, law, synth.INSERT))
            assert g.insert_edges(_dev(ins)) == ref.insert_edges(ins)
            st = g.stats()
            assert st["iterations"] == ref.last_iterations(), (name, law)
            assert st["launches"] >= 2 * st["iterations"], (name, st)   # one launch pair per iteration at least
            assert (g.cores() == ref.cores()).all(), (name, law)
            dl = synth.static_sample_delete(n, ref.edges(), 3000, synth.PREFERENTIAL,
                                            synth.stream(904, n, law, synth.DELETE))
            assert g.delete_edges(_dev(dl)) == ref.delete_edges(dl)
            st = g.stats()
            assert st["iterations"] == ref.last_iterations(), (name, law)
            assert (g.cores() == ref.cores()).all(), (name, law)
        _clean(g.check(), n, name)


def test_debug_mode_vertex_operations(cm):
    """Vertex insertions (new vertices, then their edges) and deletions
    (pinned vertices whose edges go) under the per-iteration check."""
    rng = np.random.default_rng(905)
    n = 600
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < 0.03
    e = np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int32)
    g = cm.CoreGraph(n, _dev(e), debug_flags=cm.CM_DEBUG_CHECK_ITERATIONS)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    alive = np.ones(n, bool)
    for r in range(3):
        nl = [rng.choice(np.nonzero(alive)[0], 8, replace=False).tolist() for _ in range(20)]
        first, _ = g.insert_vertices(nl)
        assert first == ref.insert_vertices(nl) == len(alive)
        assert g.stats()["iterations"] == ref.last_iterations()
        alive = np.concatenate([alive, np.ones(20, bool)])
        assert (g.cores() == ref.cores()).all(), r
        deg = np.bincount(ref.edges().ravel(), minlength=len(alive))
        dead = np.argsort(-np.where(alive, deg, -1))[:5].astype(np.int32)   # the largest live hubs
        assert g.delete_vertices(dead) == ref.delete_vertices(dead)
        alive[dead] = False
        assert (g.cores() == ref.cores()).all(), r
        _clean(g.check(), len(alive), f"round {r}")
    # a checkpoint with deleted vertices (core -1) resumes into a consistent store
    g2 = cm.CoreGraph(len(alive), _dev(g.edges()), _dev(g.cores()))
    _clean(g2.check(), len(alive), "resumed")
    assert (g2.cores() == ref.cores()).all()
