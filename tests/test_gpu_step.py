"""Captured update steps (one CUDA graph replay applies every graph's insert
batch, then every graph's delete batch) against the oracle, and the
autotuner that times schedules on a saved copy of the graph.

The superior-edge-set procedure (Algorithms 1 and 5) is deterministic given
the selection priorities, so the oracle run on the disjoint union (global
ids) gives the step's exact iteration count; core numbers are compared
bit-exactly per graph.
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


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.Stream()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _many(seed, ng, lo=2.0, hi=3.5):
    rng = np.random.default_rng(seed)
    ns, ms, parts = [], [], []
    for i in range(ng):
        n = int(10 ** rng.uniform(lo, hi))
        m = int(rng.integers(2, 9))
        e = synth.ba(n, m, synth.stream(60 + seed, i))
        ns.append(n)
        ms.append(len(e))
        parts.append(e)
    return rng, ns, ms, parts


def _batches(rng, dyns, seed, step, frac_ins=0.7, lo=1.0, hi=2.7):
    ins, dele = [], []
    for i, d in enumerate(dyns):
        b = int(10 ** rng.uniform(lo, hi))
        k_ins = int(round(frac_ins * b))
        a = d.sample_insert(k_ins, synth.UNIFORM, synth.stream(seed, i, step, synth.INSERT))
        d.apply(0, a)
        x = d.sample_delete(b - k_ins, synth.UNIFORM, synth.stream(seed, i, step, synth.DELETE))
        d.apply(1, x)
        ins.append(a)
        dele.append(x)
    return ins, dele


def test_step_matches_oracle_over_replays(cm, stream):
    rng, ns, ms, parts = _many(1, 20)
    ng = len(ns)
    g = cm.CoreGraph(None, _dev(np.concatenate(parts)), multi=(ns, ms), stream=stream)
    bases = g.bases()
    union = oracle.OracleGraph(int(sum(ns)), np.concatenate([p + b for p, b in zip(parts, bases)]),
                               mode=oracle.SUPERIOR)
    dyns = [synth.DynGraph(ns[i], parts[i]) for i in range(ng)]
    st = g.step(20000, 20000)
    for step in range(5):
        ins, dele = _batches(rng, dyns, 70, step)
        ci, cd = [len(a) for a in ins], [len(x) for x in dele]
        gi = np.concatenate([a + bases[i] for i, a in enumerate(ins)])
        gd = np.concatenate([x + bases[i] for i, x in enumerate(dele)])
        # host input on even steps, device input on odd ones
        src = (lambda a: a) if step % 2 == 0 else _dev
        pi, pd = st.run(ci, src(np.concatenate(ins)), cd, src(np.concatenate(dele)))
        assert pi.tolist() == ci and pd.tolist() == cd
        assert union.insert_edges(gi) == sum(ci)
        it_ins = union.last_iterations()
        assert union.delete_edges(gd) == sum(cd)
        it_del = union.last_iterations()
        s = g.stats()
        assert s["iterations"] == it_ins + it_del, step
        assert s["applied"] == sum(ci) + sum(cd)
        assert (g.cores() == union.cores()).all(), step
        assert g.m == union.m
    c = g.cores()
    for i in range(ng):
        assert (c[bases[i]: bases[i] + ns[i]] == oracle.bz(ns[i], dyns[i].edges())).all(), i
    cnt = st.counters()
    assert cnt["replays"] == 5 and cnt["fallbacks"] == 0
    assert 1 <= cnt["captures"] <= 5


def test_step_with_selection_variant(cm, stream):
    """A captured step on a handle created with a selection variant
    (canonical-key order, one claim round per iteration) matches the
    oracle's superior-edge-set procedure under the same variant, iteration
    count included."""
    rng, ns, ms, parts = _many(3, 8)
    ng = len(ns)
    opts = dict(select_order=cm.CM_SELECT_KEY, select_rounds=1)
    g = cm.CoreGraph(None, _dev(np.concatenate(parts)), multi=(ns, ms), stream=stream, **opts)
    bases = g.bases()
    union = oracle.OracleGraph(int(sum(ns)), np.concatenate([p + b for p, b in zip(parts, bases)]),
                               mode=oracle.SUPERIOR, **opts)
    dyns = [synth.DynGraph(ns[i], parts[i]) for i in range(ng)]
    st = g.step(20000, 20000)
    for step in range(3):
        ins, dele = _batches(rng, dyns, 70, step)
        ci, cd = [len(a) for a in ins], [len(x) for x in dele]
        gi = np.concatenate([a + bases[i] for i, a in enumerate(ins)])
        gd = np.concatenate([x + bases[i] for i, x in enumerate(dele)])
        st.run(ci, _dev(np.concatenate(ins)), cd, _dev(np.concatenate(dele)))
        union.insert_edges(gi)
        it_ins = union.last_iterations()
        union.delete_edges(gd)
        it_del = union.last_iterations()
        assert g.stats()["iterations"] == it_ins + it_del, step
        assert (g.cores() == union.cores()).all(), step


def test_step_single_graph_and_errors(cm, stream):
    n = 4000
    e = synth.er(n, 16000, synth.stream(80))
    g = cm.CoreGraph(n, _dev(e), stream=stream)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    dyn = synth.DynGraph(n, e)
    st = g.step(3000, 3000)
    a = dyn.sample_insert(2000, synth.UNIFORM, synth.stream(81))
    dyn.apply(0, a)
    x = dyn.sample_delete(1500, synth.PREFERENTIAL, synth.stream(82))
    dyn.apply(1, x)
    pi, pd = st.run([len(a)], a, [len(x)], x)
    assert (pi[0], pd[0]) == (ref.insert_edges(a), ref.delete_edges(x)) == (2000, 1500)
    assert (g.cores() == ref.cores()).all()
    before = g.cores().copy()
    m0 = g.m
    # an id out of range in the delete batch: nothing changes
    bad = np.array([[0, 1], [2, n + 5]], np.int32)
    good = dyn.sample_insert(10, synth.UNIFORM, synth.stream(83))
    with pytest.raises(cm.CoreMaintError) as ei:
        st.run([len(good)], good, [2], bad)
    assert ei.value.code == cm.CM_ERR_INVALID
    assert "delete batch" in str(ei.value)
    assert g.m == m0 and (g.cores() == before).all()
    # above capacity: refused before anything runs
    big = dyn.sample_insert(3001, synth.UNIFORM, synth.stream(84))
    with pytest.raises(cm.CoreMaintError) as ei:
        st.run([len(big)], big, None, None)
    assert ei.value.code == cm.CM_ERR_CAPACITY
    # insert-only and delete-only steps
    pi, pd = st.run([len(good)], good, None, None)
    assert pi[0] == ref.insert_edges(good) and pd[0] == 0
    dyn.apply(0, good)
    pi, pd = st.run(None, None, [len(good)], good)
    assert pd[0] == ref.delete_edges(good)
    dyn.apply(1, good)
    assert (g.cores() == ref.cores()).all()


def test_step_pool_short_falls_back(cm, stream):
    """No slack and a batch that piles edges on a few vertices: the step's
    relocations do not fit the pool, the replay changes nothing and both
    phases run on the ordinary path; the next replay is captured again."""
    n = 3000
    e = synth.er(n, 6000, synth.stream(90))
    g = cm.CoreGraph(n, _dev(e), stream=stream, slack_pct=0, min_cap=4)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    st = g.step(20000, 20000)
    hubs = [3, 4, 5, 6]
    others = np.setdiff1d(np.arange(n), hubs)
    a = np.concatenate([np.stack([np.full(2000, h), others[:2000]], 1) for h in hubs]).astype(np.int32)
    x = ref.edges()[:500]
    pi, pd = st.run([len(a)], a, [len(x)], x)
    assert pi[0] == ref.insert_edges(a) and pd[0] == ref.delete_edges(x)
    assert (g.cores() == ref.cores()).all()
    assert st.counters()["fallbacks"] == 1
    b = np.stack([np.full(300, 7), others[100:400]], 1).astype(np.int32)
    pi, pd = st.run([len(b)], b, None, None)
    assert pi[0] == ref.insert_edges(b)
    assert (g.cores() == ref.cores()).all()
    assert st.counters()["captures"] >= 2


def test_autotune_leaves_graph_unchanged(cm, stream):
    rng, ns, ms, parts = _many(3, 12, 2.5, 3.5)
    ng = len(ns)
    g = cm.CoreGraph(None, _dev(np.concatenate(parts)), multi=(ns, ms), stream=stream)
    bases = g.bases()
    union = oracle.OracleGraph(int(sum(ns)), np.concatenate([p + b for p, b in zip(parts, bases)]),
                               mode=oracle.SUPERIOR)
    dyns = [synth.DynGraph(ns[i], parts[i]) for i in range(ng)]
    ins, dele = _batches(rng, dyns, 95, 0)
    ci, cd = [len(a) for a in ins], [len(x) for x in dele]
    st = g.step(sum(ci), sum(cd))
    c0 = g.cores().copy()
    e0 = set(map(tuple, np.sort(g.edges(), 1).tolist()))
    rep = st.autotune(ci, np.concatenate(ins), cd, np.concatenate(dele), reps=1)
    assert rep["tried"] == 16 and rep["best_ms"] > 0 and rep["best_ms"] <= rep["first_ms"]
    assert (g.cores() == c0).all()
    assert set(map(tuple, np.sort(g.edges(), 1).tolist())) == e0
    assert st.config.as_dict() == rep["best"]
    # the tuned step still computes the same result
    pi, pd = st.run(ci, np.concatenate(ins), cd, np.concatenate(dele))
    union.insert_edges(np.concatenate([a + bases[i] for i, a in enumerate(ins)]))
    union.delete_edges(np.concatenate([x + bases[i] for i, x in enumerate(dele)]))
    assert (g.cores() == union.cores()).all()
    assert pi.tolist() == ci and pd.tolist() == cd
