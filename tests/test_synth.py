"""The seeded input generators: determinism and the structural properties
each workload recipe promises (distinct edges, no self-loops, absent/present
edges for insert/delete batches, append-only vertex ids)."""
import numpy as np

import synth


def _keys(e):
    e = np.asarray(e, dtype=np.int64)
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    return lo << 32 | hi


def test_er_distinct_and_deterministic():
    a = synth.er(1000, 5000, synth.stream(1))
    b = synth.er(1000, 5000, synth.stream(1))
    assert (a == b).all() and len(np.unique(_keys(a))) == 5000
    assert (a[:, 0] != a[:, 1]).all() and a.min() >= 0 and a.max() < 1000


def test_rmat_canonical_unique():
    e = synth.rmat(12, 8, synth.stream(2))
    assert (e[:, 0] < e[:, 1]).all()
    k = _keys(e)
    assert (np.diff(k) > 0).all() and e.max() < 4096
    # skewed degrees: the top vertex is far above the mean
    deg = np.bincount(e.ravel(), minlength=4096)
    assert deg.max() > 10 * deg.mean()


def test_ba_and_grid_counts():
    e = synth.ba(2000, 5, synth.stream(3))
    assert len(e) == 5 * 6 // 2 + (2000 - 6) * 5 and len(np.unique(_keys(e))) == len(e)
    g = synth.grid(50, 40, synth.stream(4))
    assert len(g) == 2 * 50 * 49 + 40 and len(np.unique(_keys(g))) == len(g)


def test_dyn_streams():
    e = synth.er(500, 2000, synth.stream(5))
    d = synth.DynGraph(500, e)
    cur = set(_keys(e).tolist())
    for law in (synth.UNIFORM, synth.PREFERENTIAL):
        ins = d.sample_insert(300, law, synth.stream(5, 0, law, synth.INSERT))
        k = _keys(ins)
        assert len(ins) == 300 and len(set(k.tolist())) == 300 and not (set(k.tolist()) & cur)
        dl = d.sample_delete(300, law, synth.stream(5, 0, law, synth.DELETE))
        k = _keys(dl)
        assert len(set(k.tolist())) == 300 and set(k.tolist()) <= cur
    assert d.apply(0, ins) == 300 and d.m == 2300
    nb = d.add_vertices(4, 6, synth.stream(5, 0, 0, synth.VINSERT))
    assert d.n == 504 and nb.shape == (4, 6) and nb.max() < 500
    dead = d.delete_vertices(3, synth.stream(5, 0, 0, synth.VDELETE))
    al = d.alive()
    assert (~al[dead]).all() and all(d.degree(int(v)) == 0 for v in dead)


def test_ba_many_graphs_and_batches():
    """Each generated graph equals the single-graph BA generator with its
    seed; each round's inserts are distinct pairs absent from its graph and
    its deletes distinct edges of it, laid out round by round in graph
    order."""
    from synth import workloads
    w = workloads.ba_many(12, rounds=2, nmax_exp=3.6)
    ns, ms, e, eoff = w["ns"], w["ms"], w["edges"], w["eoff"]
    assert ((ms >= 4) & (ms <= 16)).all() and ((ns >= 1000) & (ns < 10 ** 3.6)).all()
    for r in range(2):
        io = do = 0
        for i in range(12):
            g = e[eoff[i]:eoff[i + 1]]
            if r == 0:
                assert (g == synth.ba(int(ns[i]), int(ms[i]), synth.stream(4, i, 0, synth.GRAPH))).all()
            ki, kd = int(w["kins"][r, i]), int(w["kdel"][r, i])
            assert 10 <= ki + kd <= 10 ** 4 and abs(ki - 0.7 * (ki + kd)) <= 1
            E = set(map(tuple, np.sort(g, 1).tolist()))
            a = set(map(tuple, np.sort(w["ins"][r][io:io + ki], 1).tolist()))
            d = set(map(tuple, np.sort(w["dele"][r][do:do + kd], 1).tolist()))
            assert len(a) == ki and len(d) == kd
            assert not (a & E) and d <= E
            assert all(u != v and 0 <= u < ns[i] and 0 <= v < ns[i] for u, v in a)
            io += ki
            do += kd
        assert io == len(w["ins"][r]) and do == len(w["dele"][r])


def test_serving_trace_recipe():
    """The serving trace keeps its stated recipe: Poisson arrivals at the
    given rate, a uniform graph, 70% inserts, log-normal sizes with median
    200 clamped to [10, 10^5]; inserts are absent distinct pairs, deletes
    present distinct edges, and no edge belongs to two requests of a graph."""
    from synth import workloads
    n = 200000
    e = synth.er(n, 2000000, synth.stream(77))
    tr = workloads.serving_trace([(n, e), (n, e)], 2000.0, 1.0)
    arr, gr, op, cnt = tr["arrival_ns"], tr["graph"], tr["op"], tr["counts"]
    k = len(cnt)
    assert abs(k - 2000) < 5 * 2000 ** 0.5                       # Poisson count
    assert (np.diff(arr) >= 0).all() and arr[-1] < 1e9
    assert abs((gr == 0).mean() - 0.5) < 0.05 and abs((op == 0).mean() - 0.7) < 0.05
    assert cnt.min() >= 10 and cnt.max() <= 10 ** 5 and 150 < np.median(cnt) < 260
    assert tr["off"][-1] == cnt.sum() and len(tr["edges"]) == cnt.sum()
    have = set(((e[:, 0].astype(np.int64) << 32) | e[:, 1]).tolist())
    have |= set(((e[:, 1].astype(np.int64) << 32) | e[:, 0]).tolist())
    for g in (0, 1):
        seen = set()
        for j in np.nonzero(gr == g)[0]:
            x = tr["edges"][tr["off"][j]:tr["off"][j + 1]].astype(np.int64)
            keys = np.minimum(x[:, 0], x[:, 1]) << 32 | np.maximum(x[:, 0], x[:, 1])
            ks = set(keys.tolist())
            assert len(ks) == len(keys) and not (ks & seen)
            seen |= ks
            present = np.array([int(q) in have for q in keys])
            assert present.all() if op[j] == 1 else not present.any()


def test_rmat_rounds_recipe():
    """Each round of the rounds workload, replayed on a plain edge set:
    inserts are distinct absent pairs, deletes distinct present edges, new
    vertices get ids in order and distinct live neighbours, deleted vertices
    are live and take their edges with them; the replay ends on the
    generator's own final graph."""
    from synth import workloads
    w = workloads.rmat_rounds(3, scale=12, ins=500, dele=500, vins=10, vdeg=8, vdel=10)
    key = lambda u, v: (min(int(u), int(v)), max(int(u), int(v)))
    edges = {key(u, v) for u, v in w.edges}
    alive = set(range(w.n))
    nxt = w.n
    for r in w.rounds:
        ins = [key(u, v) for u, v in r.ins]
        assert len(set(ins)) == len(ins) and all(u != v and u in alive and v in alive for u, v in ins)
        assert not (set(ins) & edges)
        edges |= set(ins)
        dl = [key(u, v) for u, v in r.dele]
        assert len(set(dl)) == len(dl) and set(dl) <= edges
        edges -= set(dl)
        assert r.first_new_id == nxt
        for i, nb in enumerate(r.vnbrs):
            v = nxt + i
            assert len(set(nb.tolist())) == len(nb) and all(int(x) in alive or nxt <= x < v for x in nb)
            edges |= {key(v, x) for x in nb}
        alive |= set(range(nxt, nxt + len(r.vnbrs)))
        nxt += len(r.vnbrs)
        before = len(edges)
        for v in r.vdel.tolist():
            assert v in alive
            alive.discard(v)
            edges = {e for e in edges if v not in e}
        assert before - len(edges) == r.vdel_edges
    assert edges == {key(u, v) for u, v in w.final.edges()}


def test_sweep_batch_laws():
    """The sweep's batches: inserts are distinct absent pairs and deletes
    distinct present edges under both endpoint laws.  Degree-proportional
    insert endpoints have a far higher mean degree than uniform ones; for
    deletes the "uniform" law picks a uniform vertex and then a uniform
    neighbour (itself degree-biased), so the gap to uniform random edges is
    smaller but still there."""
    from synth import workloads
    n, e, batches = workloads.rmat_sweep(scale=14, sizes=(3000,))
    key = lambda a: set(map(tuple, np.sort(a, 1).tolist()))
    have = key(e)
    deg = np.bincount(e.ravel(), minlength=n)
    mean_deg = {}
    for (op, size, law), b in batches.items():
        ks = key(b)
        assert len(ks) == len(b) == size and (b[:, 0] != b[:, 1]).all()
        assert (ks <= have) if op == "delete" else not (ks & have)
        mean_deg[(op, law)] = deg[b.ravel()].mean()
    assert mean_deg[("insert", synth.PREFERENTIAL)] > 4 * mean_deg[("insert", synth.UNIFORM)], mean_deg
    assert mean_deg[("delete", synth.PREFERENTIAL)] > 1.1 * mean_deg[("delete", synth.UNIFORM)], mean_deg
