"""CUDA path against the CPU oracle, through the C ABI.

Core numbers are integers with one correct answer (Section III, Definitions
1-2), so every comparison is bit-exact.  The iteration count of a batch is
compared with the oracle's superior-edge-set procedure (O4), which selects
with the same priority rule, so it must match exactly too.
"""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _rand_graph(rng, n, p):
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int32)


def sd_recount(n, edges, cores):
    """SD (Section IV, Definition 7) from scratch: for every vertex the number
    of neighbours whose core is at least its own; -1 for dead vertices."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    cu, cv = cores[e[:, 0]], cores[e[:, 1]]
    sd = np.bincount(e[:, 0][cv >= cu], minlength=n) + np.bincount(e[:, 1][cu >= cv], minlength=n)
    return np.where(cores < 0, -1, sd).astype(np.int32)


def _check_same(g, ref, what=""):
    gc = g.cores()
    rc = ref.cores()
    assert gc.shape == rc.shape, what
    bad = np.nonzero(gc != rc)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} cores differ, first {bad[:8]} gpu {gc[bad[:8]]} ref {rc[bad[:8]]}"
    # the superior degrees the library keeps beside the cores (Definition 7)
    sd = g.superior_degrees()
    exp = sd_recount(len(rc), ref.edges(), rc)
    bad = np.nonzero(sd != exp)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} SD differ, first {bad[:8]} gpu {sd[bad[:8]]} recount {exp[bad[:8]]}"


# ---------------------------------------------------------------- decomposition
@pytest.mark.parametrize("kind", ["er", "rmat", "ba", "grid", "empty", "k50"])
def test_create_peel_matches_bz(cm, kind):
    if kind == "er":
        n, e = 3000, synth.er(3000, 12000, synth.stream(10))
    elif kind == "rmat":
        e = synth.rmat(13, 16, synth.stream(11))
        n = 1 << 13
    elif kind == "ba":
        n, e = 5000, synth.ba(5000, 7, synth.stream(12))
    elif kind == "grid":
        n, e = 60 * 60, synth.grid(60, 40, synth.stream(13))
    elif kind == "empty":
        n, e = 100, np.zeros((0, 2), np.int32)
    else:
        n = 50
        e = np.array([(i, j) for i in range(n) for j in range(i + 1, n)], np.int32)
    g = cm.CoreGraph(n, _dev(e) if len(e) else e)
    ref = oracle.bz(n, e)
    assert (g.cores() == ref).all()
    assert g.m == len(e)
    got = g.edges()
    assert set(map(tuple, np.sort(got, 1).tolist())) == set(map(tuple, np.sort(e, 1).tolist()))
    # host input and given cores give the same store
    g2 = cm.CoreGraph(n, e, cores=ref)
    assert (g2.cores() == ref).all()


def test_create_drops_repeats_and_loops(cm):
    e = np.array([[0, 1], [1, 0], [2, 2], [1, 2], [0, 1], [2, 0]], np.int32)
    g = cm.CoreGraph(4, e)
    assert g.m == 3
    assert g.cores().tolist() == [2, 2, 2, 0]


# ---------------------------------------------------------------- batches vs oracle
@pytest.mark.parametrize("seed", range(6))
def test_random_batches_small(cm, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 300))
    e = _rand_graph(rng, n, rng.uniform(0.02, 0.2))
    g = cm.CoreGraph(n, _dev(e) if len(e) else e)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    _check_same(g, ref, "create")
    for b in range(8):
        cur = ref.edges()
        if b % 2 == 0 or len(cur) == 0:
            k = int(rng.integers(1, 4 * n))
            batch = rng.integers(0, n, (k, 2)).astype(np.int32)
            batch = np.concatenate([batch, batch[: k // 5, ::-1], np.array([[3, 3]], np.int32)])
            got = g.insert_edges(_dev(batch))
            exp = ref.insert_edges(batch)
        else:
            k = int(rng.integers(1, len(cur) + 1))
            batch = cur[rng.permutation(len(cur))[:k]]
            batch = np.concatenate([batch, batch[: k // 3, ::-1], np.array([[0, 1]], np.int32)])
            got = g.delete_edges(batch)          # host input path
            exp = ref.delete_edges(batch)
        assert got == exp
        s = g.stats()
        assert s["iterations"] == ref.last_iterations(), (b, s["iterations"], ref.last_iterations())
        assert s["selected"] == exp
        _check_same(g, ref, f"batch {b}")
        assert g.m == ref.m


@pytest.mark.parametrize("order,rounds", [(1, 0), (0, 1), (0, 2), (1, 1)])
def test_selection_variants(cm, order, rounds):
    """The selection variants of reading R1 (Section IV, Definition 6 and
    Algorithm 2): canonical-key order instead of its fmix64, and claim
    rounds capped per iteration.  The cores equal the oracle's after every
    batch and the iteration counts equal O4's under the same variant, on
    small graphs and on a 20,000-vertex BA graph (one core level)."""
    rng = np.random.default_rng(200 + 10 * order + rounds)
    opts = dict(select_order=order, select_rounds=rounds)
    for trial in range(3):
        n = int(rng.integers(50, 400))
        e = _rand_graph(rng, n, rng.uniform(0.02, 0.15))
        g = cm.CoreGraph(n, _dev(e), **opts)
        ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR, **opts)
        for b in range(6):
            cur = ref.edges()
            if b % 2 == 0 or len(cur) == 0:
                batch = rng.integers(0, n, (int(rng.integers(1, 4 * n)), 2)).astype(np.int32)
                got, exp = g.insert_edges(_dev(batch)), ref.insert_edges(batch)
            else:
                batch = cur[rng.permutation(len(cur))[: int(rng.integers(1, len(cur) + 1))]]
                got, exp = g.delete_edges(_dev(batch)), ref.delete_edges(batch)
            assert got == exp
            assert g.stats()["iterations"] == ref.last_iterations(), (trial, b)
            _check_same(g, ref, f"variant {order}/{rounds} trial {trial} batch {b}")
    n = 20000
    e = synth.ba(n, 6, synth.stream(21))
    dyn = synth.DynGraph(n, e)
    g = cm.CoreGraph(n, _dev(e), **opts)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR, **opts)
    ins = dyn.sample_insert(3000, synth.PREFERENTIAL, synth.stream(21, 0, 0, synth.INSERT))
    g.insert_edges(_dev(ins))
    ref.insert_edges(ins)
    assert g.stats()["iterations"] == ref.last_iterations()
    _check_same(g, ref, "BA insert")


@pytest.mark.parametrize("early", [1, -1])
def test_expand_early_variants(cm, early):
    """The insert search's frontier vertices visiting their candidates in
    the CSD pass (1: always) or only after their support is known (-1: the
    paper's order, Algorithm 3) reach the oracle's cores, SD and iteration
    counts, on a random graph, an R-MAT graph with hubs and a single-level BA
    graph."""
    rng = np.random.default_rng(300 + early)
    graphs = [(400, _rand_graph(rng, 400, 0.05)), (1 << 13, synth.rmat(13, 16, synth.stream(301))),
              (20000, synth.ba(20000, 6, synth.stream(302)))]
    for n, e in graphs:
        g = cm.CoreGraph(n, _dev(e), expand_early=early)
        ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
        for law in (synth.UNIFORM, synth.PREFERENTIAL):
            ins = synth.static_sample_insert(n, ref.edges(), 3000, law, synth.stream(303, n, law, synth.INSERT))
            assert g.insert_edges(_dev(ins)) == ref.insert_edges(ins)
            assert g.stats()["iterations"] == ref.last_iterations()
            _check_same(g, ref, f"early {early} n {n} law {law}")


def test_cfg_er_insert_then_delete_full_size(cm):
    """ER G(n=10,000, m=50,000), 1,000 new edges inserted, then 1,000 existing
    edges deleted; cores checked after each batch (the small workload)."""
    n, m = 10000, 50000
    e = synth.er(n, m, synth.stream(1, 0, 0, synth.GRAPH))
    dyn = synth.DynGraph(n, e)
    g = cm.CoreGraph(n, _dev(e))
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    ins = dyn.sample_insert(1000, synth.UNIFORM, synth.stream(1, 0, 0, synth.INSERT))
    assert g.insert_edges(_dev(ins)) == ref.insert_edges(ins) == 1000
    assert g.stats()["iterations"] == ref.last_iterations()
    _check_same(g, ref, "insert")
    dyn.apply(0, ins)
    assert (g.cores() == oracle.bz(n, dyn.edges())).all()
    dl = dyn.sample_delete(1000, synth.PREFERENTIAL, synth.stream(1, 0, 0, synth.DELETE))
    assert g.delete_edges(_dev(dl)) == ref.delete_edges(dl) == 1000
    assert g.stats()["iterations"] == ref.last_iterations()
    _check_same(g, ref, "delete")
    dyn.apply(1, dl)
    assert (g.cores() == oracle.bz(n, dyn.edges())).all()


def test_sequential_oracle_agrees(cm):
    """The paper's sequential single-edge traversal (O3) reaches the same
    cores as the batched GPU call."""
    n = 4000
    e = synth.rmat(12, 8, synth.stream(20))
    n = 1 << 12
    dyn = synth.DynGraph(n, e)
    g = cm.CoreGraph(n, _dev(e))
    seq = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL)
    for r in range(3):
        ins = dyn.sample_insert(500, synth.PREFERENTIAL, synth.stream(20, 0, r, synth.INSERT))
        g.insert_edges(_dev(ins))
        seq.insert_edges(ins)
        dyn.apply(0, ins)
        _check_same(g, seq, f"insert {r}")
        dl = dyn.sample_delete(500, synth.UNIFORM, synth.stream(20, 0, r, synth.DELETE))
        g.delete_edges(_dev(dl))
        seq.delete_edges(dl)
        dyn.apply(1, dl)
        _check_same(g, seq, f"delete {r}")


def test_single_level_graph(cm):
    """Barabasi-Albert graphs put every vertex at one core level, the paper's
    worst case for level parallelism (Section VII): all work is in one level."""
    n = 20000
    e = synth.ba(n, 6, synth.stream(21))
    dyn = synth.DynGraph(n, e)
    g = cm.CoreGraph(n, _dev(e))
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    ins = dyn.sample_insert(3000, synth.PREFERENTIAL, synth.stream(21, 0, 0, synth.INSERT))
    g.insert_edges(_dev(ins))
    ref.insert_edges(ins)
    assert g.stats()["iterations"] == ref.last_iterations()
    _check_same(g, ref, "BA insert")
    dl = dyn.sample_delete(3000, synth.UNIFORM, synth.stream(21, 0, 0, synth.DELETE))
    dyn.apply(0, ins)
    dl = dyn.sample_delete(3000, synth.UNIFORM, synth.stream(21, 0, 1, synth.DELETE))
    g.delete_edges(_dev(dl))
    ref.delete_edges(dl)
    assert g.stats()["iterations"] == ref.last_iterations()
    _check_same(g, ref, "BA delete")


# ---------------------------------------------------------------- vertex operations
def test_vertex_insert_delete(cm):
    rng = np.random.default_rng(7)
    n = 500
    e = _rand_graph(rng, n, 0.03)
    g = cm.CoreGraph(n, _dev(e))
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    alive = np.ones(n, bool)
    for r in range(5):
        nl = [rng.choice(np.nonzero(alive)[0], 8, replace=False).tolist() for _ in range(20)]
        nl[5].append(g.n)            # a neighbour that is another new vertex of the same call
        first, applied = g.insert_vertices(nl)
        rf = ref.insert_vertices(nl)
        assert first == rf == len(alive)
        assert g.stats()["iterations"] == ref.last_iterations()
        alive = np.concatenate([alive, np.ones(20, bool)])
        _check_same(g, ref, f"vinsert {r}")
        dead = rng.choice(np.nonzero(alive)[0], 7, replace=False)
        dead = np.concatenate([dead, dead[:2]])          # repeats allowed
        got = g.delete_vertices(dead.astype(np.int32))
        exp = ref.delete_vertices(dead)
        assert got == exp
        alive[dead] = False
        _check_same(g, ref, f"vdelete {r}")
        assert (g.cores()[~alive] == -1).all()
    v = cm.cm_insert_vertex(g.handle, np.array([0, 1, 2], np.int32)) if alive[:3].all() else None
    if v is not None:
        assert v == g.n - 1
        cm.cm_delete_vertex(g.handle, v)
        assert g.cores()[v] == -1


def test_vertex_delete_hubs_and_neighbours(cm):
    """Deleting hubs, hubs that share neighbours, and adjacent vertices in
    one call: the deleted vertices are pinned while their edges go, so the
    call needs far fewer iterations than one edge per hub per iteration,
    and the cores are those of the graph without them."""
    scale = 13
    n = 1 << scale
    e = synth.rmat(scale, 16, synth.stream(44))
    g = cm.CoreGraph(n, _dev(e))
    deg = np.bincount(e.ravel(), minlength=n)
    hubs = np.argsort(-deg)[:6]
    nb = e[e[:, 0] == hubs[0], 1][:3]                      # neighbours of the largest hub
    dead = np.unique(np.concatenate([hubs, nb, [7, 8, 9]])).astype(np.int32)
    got = g.delete_vertices(dead)
    keep = ~np.isin(e, dead).any(1)
    assert got == int((~keep).sum())
    exp = oracle.bz(n, e[keep])
    c = g.cores()
    assert (c[dead] == -1).all()
    alive = np.setdiff1d(np.arange(n), dead)
    assert (c[alive] == exp[alive]).all()
    assert (g.superior_degrees() == sd_recount(n, e[keep], c)).all()
    assert g.stats()["iterations"] < deg[hubs[0]] // 4
    # the graph keeps working after it
    ref = oracle.OracleGraph(n, e[keep], mode=oracle.SUPERIOR)
    dl = synth.static_sample_delete(n, e[keep], 2000, synth.PREFERENTIAL, synth.stream(45))
    assert g.delete_edges(_dev(dl)) == ref.delete_edges(dl)
    assert (g.cores()[alive] == ref.cores()[alive]).all()


# ---------------------------------------------------------------- edge cases
def test_edge_cases(cm):
    n = 40
    e = np.array([(i, (i + 1) % n) for i in range(n)], np.int32)   # a cycle: all cores 2
    g = cm.CoreGraph(n, e)
    assert (g.cores() == 2).all()
    assert g.insert_edges(np.zeros((0, 2), np.int32)) == 0          # empty batch
    assert g.insert_edges(e) == 0                                   # all present
    assert g.delete_edges(np.array([[0, 5], [7, 7]], np.int32)) == 0  # absent + self-loop
    assert g.insert_edges(np.array([[4, 4]], np.int32)) == 0        # self-loop only
    before = g.cores().copy()
    m0 = g.m
    with pytest.raises(cm.CoreMaintError) as ei:
        g.insert_edges(np.array([[0, 2], [1, n]], np.int32))        # id out of range
    assert ei.value.code == cm.CM_ERR_INVALID
    with pytest.raises(cm.CoreMaintError):
        g.delete_edges(np.array([[0, 1], [-1, 3]], np.int32))
    assert (g.cores() == before).all() and g.m == m0                # unchanged
    g.delete_vertices(np.array([3], np.int32))
    with pytest.raises(cm.CoreMaintError) as ei:
        g.insert_edges(np.array([[3, 10]], np.int32))               # dead vertex
    assert ei.value.code == cm.CM_ERR_INVALID
    with pytest.raises(cm.CoreMaintError) as ei:
        g.delete_edges(np.array([[5, 6], [3, 4]], np.int32))        # a delete naming a dead vertex
    assert ei.value.code == cm.CM_ERR_INVALID
    assert g.m == m0 - 2                                            # vertex 3's two edges went, nothing else
    with pytest.raises(cm.CoreMaintError):
        g.delete_vertices(np.array([3], np.int32))                  # already dead
    with pytest.raises(cm.CoreMaintError):
        g.insert_vertices([[0, 1, 10**6]])                          # bad neighbour
    assert g.n == n
    # a chord makes a 3-core only where the degrees allow: check against BZ
    alive = np.ones(n, bool)
    alive[3] = False
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    ref.delete_vertices([3])
    chords = np.array([[0, 20], [10, 30], [0, 10], [20, 30]], np.int32)
    g.insert_edges(chords)
    ref.insert_edges(chords)
    _check_same(g, ref, "chords")


def test_hub_overflow_relocation(cm):
    """A batch that adds far more edges to one vertex than its slack holds
    exercises relocation; a later delete batch leaves holes behind."""
    n = 3000
    e = synth.er(n, 6000, synth.stream(30))
    g = cm.CoreGraph(n, _dev(e))
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    hub = 17
    others = np.setdiff1d(np.arange(n), [hub])[:2500]
    batch = np.stack([np.full(len(others), hub), others], 1).astype(np.int32)
    batch = np.concatenate([batch, synth.er(n, 3000, synth.stream(31))])
    g.insert_edges(_dev(batch))
    ref.insert_edges(batch)
    _check_same(g, ref, "hub insert")
    assert g.stats()["iterations"] == ref.last_iterations()
    cur = ref.edges()
    dl = cur[np.random.default_rng(3).permutation(len(cur))[:4000]]
    g.delete_edges(_dev(dl))
    ref.delete_edges(dl)
    _check_same(g, ref, "hub delete")
    again = np.stack([np.full(1500, hub), others[:1500]], 1).astype(np.int32)
    g.insert_edges(_dev(again))
    ref.insert_edges(again)
    _check_same(g, ref, "hub reinsert")
    got = np.sort(g.edges(), 1)
    exp = np.sort(ref.edges(), 1)
    assert set(map(tuple, got.tolist())) == set(map(tuple, exp.tolist()))


@pytest.mark.parametrize("grid_only", [True, False])
def test_hub_chunked_scans(cm, grid_only):
    """Vertices with at least hub_slots slots are scanned by every block in
    chunks of 2048 slots (frontier sums, expansion, both evictions); with a
    low threshold most of an R-MAT graph's upper shells take that path, and
    its largest lists span several chunks."""
    scale = 14
    n = 1 << scale
    e = synth.rmat(scale, 16, synth.stream(40))
    rng = np.random.default_rng(40)
    stars = [np.stack([np.full(5000, h), rng.choice(n, 5000, replace=False)], 1) for h in (5, 77, 901)]
    e = np.concatenate([e] + stars).astype(np.int32)
    e = np.unique(np.sort(e, 1), axis=0)
    e = e[e[:, 0] != e[:, 1]]
    opts = {"hub_slots": 256}
    if grid_only:
        opts["block_mode_edges"] = -1
    g = cm.CoreGraph(n, _dev(e), **opts)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    deg = np.bincount(e.ravel(), minlength=n)
    assert deg.max() > 2 * 2048
    cur = e
    for b, (op, law, k) in enumerate([(0, synth.UNIFORM, 3000), (0, synth.PREFERENTIAL, 3000),
                                      (1, synth.PREFERENTIAL, 4000), (1, synth.UNIFORM, 4000),
                                      (0, synth.PREFERENTIAL, 20000), (1, synth.PREFERENTIAL, 20000)]):
        if op == 0:
            batch = synth.static_sample_insert(n, cur, k, law, synth.stream(41, 0, b))
            got, exp = g.insert_edges(_dev(batch)), ref.insert_edges(batch)
        else:
            batch = synth.static_sample_delete(n, cur, k, law, synth.stream(42, 0, b), synth.csr(n, cur))
            got, exp = g.delete_edges(_dev(batch)), ref.delete_edges(batch)
        assert got == exp
        assert g.stats()["iterations"] == ref.last_iterations(), b
        _check_same(g, ref, f"batch {b}")
        cur = ref.edges()
    assert (g.cores() == oracle.bz(n, cur)).all()


def test_structure_apply_then_repeel(cm):
    """The full re-peel comparator: apply the batch to the structure only,
    then recompute every core by GPU peeling."""
    n = 1 << 12
    e = synth.rmat(12, 16, synth.stream(40))
    dyn = synth.DynGraph(n, e)
    g = cm.CoreGraph(n, _dev(e))
    ins = dyn.sample_insert(2000, synth.UNIFORM, synth.stream(40, 0, 0, synth.INSERT))
    assert g.apply_edges(cm.CM_OP_INSERT, _dev(ins)) == 2000
    with pytest.raises(cm.CoreMaintError) as ei:
        g.cores()
    assert ei.value.code == cm.CM_ERR_STATE
    g.recompute_cores()
    dyn.apply(0, ins)
    assert (g.cores() == oracle.bz(n, dyn.edges())).all()
    dl = dyn.sample_delete(2000, synth.PREFERENTIAL, synth.stream(40, 0, 0, synth.DELETE))
    g.apply_edges(cm.CM_OP_DELETE, _dev(dl))
    g.recompute_cores()
    dyn.apply(1, dl)
    assert (g.cores() == oracle.bz(n, dyn.edges())).all()
    # maintenance continues correctly after a recompute
    ins2 = dyn.sample_insert(1000, synth.UNIFORM, synth.stream(40, 0, 1, synth.INSERT))
    g.insert_edges(_dev(ins2))
    dyn.apply(0, ins2)
    assert (g.cores() == oracle.bz(n, dyn.edges())).all()


# ---------------------------------------------------------------- many graphs in one handle
def test_multi_graph_one_launch(cm):
    rng = np.random.default_rng(5)
    ng = 24
    ns, ms, parts = [], [], []
    for i in range(ng):
        n = int(10 ** rng.uniform(2, 3.5))
        mm = int(rng.integers(2, 7))
        e = synth.ba(n, mm, synth.stream(50, i))
        ns.append(n)
        ms.append(len(e))
        parts.append(e)
    g = cm.CoreGraph(None, _dev(np.concatenate(parts)), multi=(ns, ms))
    bases = g.bases()
    assert bases.tolist() == np.concatenate([[0], np.cumsum(ns)[:-1]]).tolist()
    refs = [oracle.OracleGraph(ns[i], parts[i], mode=oracle.SUPERIOR) for i in range(ng)]
    dyns = [synth.DynGraph(ns[i], parts[i]) for i in range(ng)]
    # the union with global ids: priorities hash global keys, so the union's
    # oracle run gives the exact iteration count of the fused call
    union = oracle.OracleGraph(int(sum(ns)), np.concatenate([p + b for p, b in zip(parts, bases)]),
                               mode=oracle.SUPERIOR)
    for op in (0, 1):
        batches = []
        for i in range(ng):
            b = int(10 ** rng.uniform(1, 2.5))
            if op == 0:
                batches.append(dyns[i].sample_insert(b, synth.UNIFORM, synth.stream(51, i)))
            else:
                batches.append(dyns[i].sample_delete(b, synth.UNIFORM, synth.stream(52, i)))
        counts = [len(b) for b in batches]
        per = g.update_multi(op, counts, _dev(np.concatenate(batches)))
        for i in range(ng):
            exp = refs[i].insert_edges(batches[i]) if op == 0 else refs[i].delete_edges(batches[i])
            dyns[i].apply(op, batches[i])
            assert per[i] == exp
        glob = np.concatenate([b + bases[i] for i, b in enumerate(batches)])
        (union.insert_edges if op == 0 else union.delete_edges)(glob)
        assert g.stats()["iterations"] == union.last_iterations()
        assert (g.cores() == union.cores()).all()
        c = g.cores()
        for i in range(ng):
            assert (c[bases[i]: bases[i] + ns[i]] == refs[i].cores()).all(), (op, i)


# ---------------------------------------------------------------- bounded waits
def test_barrier_wait_limit_returns_error(cm):
    """A grid barrier that can never complete (it waits for one block more
    than the launch has) must end in CM_ERR_LIMIT within its wait limit,
    with the device still usable afterwards."""
    import time

    n = 500
    e = synth.er(n, 1500, synth.stream(60))
    g = cm.CoreGraph(n, _dev(e), spin_limit_ns=50_000_000,
                     debug_flags=cm.CM_DEBUG_BARRIER_NEVER_RELEASES)
    t0 = time.time()
    with pytest.raises(cm.CoreMaintError) as ei:
        g.insert_edges(np.array([[0, 1], [2, 3]], np.int32) if True else None)
    assert ei.value.code == cm.CM_ERR_LIMIT
    assert time.time() - t0 < 30
    with pytest.raises(cm.CoreMaintError) as ei:
        g.cores()
    assert ei.value.code == cm.CM_ERR_STATE
    g.close()
    g2 = cm.CoreGraph(n, _dev(e))
    assert (g2.cores() == oracle.bz(n, e)).all()


def test_torch_allocator_and_device_outputs(cm):
    import torch
    n = 1000
    e = synth.er(n, 4000, synth.stream(70))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = cm.CoreGraph(n, _dev(e), stream=s, use_torch_allocator=True)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        g.cores(out)
    s.synchronize()
    assert (out.cpu().numpy() == oracle.bz(n, e)).all()
    g2 = cm.CoreGraph(n, e, use_torch_allocator=False)
    assert (g2.cores() == oracle.bz(n, e)).all()


def test_readme_quick_start(cm):
    """The quick-start example: a triangle with a pendant becomes K4 after two
    inserts (cores 3), then deleting vertex 3 leaves the triangle (cores 2)
    and a dead vertex (-1)."""
    import torch
    edges = torch.tensor([[0, 1], [1, 2], [2, 0], [2, 3]], dtype=torch.int32).cuda()
    G = cm.CoreGraph(4, edges)
    assert G.cores().tolist() == [2, 2, 2, 1]
    assert G.insert_edges(torch.tensor([[3, 0], [3, 1]], dtype=torch.int32).cuda()) == 2
    assert G.cores().tolist() == [3, 3, 3, 3]
    G.delete_vertices(torch.tensor([3], dtype=torch.int32).cuda())
    assert G.cores().tolist() == [2, 2, 2, -1]
