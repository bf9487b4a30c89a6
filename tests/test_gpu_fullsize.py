"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (default options, grid + single-block modes,
task-queue search, pinned vertex deletion, captured steps, serving).

Core numbers are unique (Section III, Definitions 1-2), so after each call
the library's cores must equal the oracle's Batagelj-Zaversnik peeling (O1)
of the expected graph, bit for bit.  These tests take minutes (graphs of up
to 260M edges) and are marked slow as well as gpu.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def _keys(e):
    e = np.asarray(e, dtype=np.int64).reshape(-1, 2)
    return np.sort((np.minimum(e[:, 0], e[:, 1]) << 32) | np.maximum(e[:, 0], e[:, 1]))


def _pairs(keys):
    return np.stack([keys >> 32, keys & 0xFFFFFFFF], 1).astype(np.int32)


def _sd_recount(n, e, cores):
    """SD (Definition 7): neighbours with core >= the vertex's; dead -1."""
    e = np.asarray(e, dtype=np.int64)
    cu, cv = cores[e[:, 0]], cores[e[:, 1]]
    sd = np.bincount(e[:, 0][cv >= cu], minlength=n) + np.bincount(e[:, 1][cu >= cv], minlength=n)
    return np.where(cores < 0, -1, sd).astype(np.int32)


def _check_against_bz(g, n_alive_mask=None, expected_keys=None):
    """The library's cores against O1; the edge set is the library's own
    unless the expected one is given (then the two must be equal)."""
    n = g.n
    e = g.edges()
    if expected_keys is not None:
        assert np.array_equal(_keys(e), expected_keys)
        e = _pairs(expected_keys)
    exp = oracle.bz(n, e, trusted=True)
    got = g.cores()
    assert (g.superior_degrees() == _sd_recount(n, e, np.where(got < 0, -1, exp))).all()
    if n_alive_mask is None:
        assert (got == exp).all(), np.nonzero(got != exp)[0][:8]
    else:
        alive = n_alive_mask
        assert (got[~alive] == -1).all()
        bad = np.nonzero((got != exp) & alive)[0]
        assert len(bad) == 0, (bad[:8], got[bad[:8]], exp[bad[:8]])
    return e


def test_rmat20_rounds_full_size(cm):
    """Three rounds of the bench's default workload (R-MAT scale 20):
    10^4 inserts, 10^4 deletes, 100 vertex inserts of degree 8, 100 vertex
    deletes per round; cores checked after every call, and the final edge
    set and live vertices against the generator's own model."""
    w = workloads.rmat_rounds(3, scale=20)
    g = cm.CoreGraph(w.n, _dev(w.edges))
    assert (g.cores() == oracle.bz(w.n, w.edges, trusted=True)).all()
    alive = np.ones(w.n, bool)
    for r in w.rounds:
        assert g.insert_edges(_dev(r.ins)) == len(r.ins)
        _check_against_bz(g, alive)
        assert g.delete_edges(_dev(r.dele)) == len(r.dele)
        _check_against_bz(g, alive)
        first, applied = g.insert_vertices([list(x) for x in r.vnbrs])
        assert first == r.first_new_id and applied == r.vnbrs.size
        alive = np.concatenate([alive, np.ones(len(r.vnbrs), bool)])
        _check_against_bz(g, alive)
        assert g.delete_vertices(_dev(r.vdel)) == r.vdel_edges
        alive[r.vdel] = False
        e = _check_against_bz(g, alive)
    assert np.array_equal(_keys(e), _keys(w.final.edges()))
    assert np.array_equal(alive, w.final.alive().astype(bool))


def test_rmat24_batches_full_size(cm):
    """R-MAT scale 24 (260M edges): a degree-proportional insert batch of
    10^5 edges, then a delete batch of 10^5 uniform random edges; after
    each, the library's whole edge set must equal the expected one (the
    generated graph plus the inserts, minus the deletes) and its cores O1
    on that expected set, with SD equal to its recount."""
    n, e, batches = workloads.rmat_sweep(scale=24, sizes=(10 ** 5,), ops=("insert", "delete"),
                                         laws=(synth.PREFERENTIAL,))
    ins = batches[("insert", 10 ** 5, synth.PREFERENTIAL)]
    dele = batches[("delete", 10 ** 5, synth.PREFERENTIAL)]
    g = cm.CoreGraph(n, _dev(e))
    keys = _keys(e)
    del e
    assert g.insert_edges(_dev(ins)) == len(ins)
    keys = np.union1d(keys, _keys(ins))
    _check_against_bz(g, expected_keys=keys)
    assert g.delete_edges(_dev(dele)) == len(dele)
    keys = np.setdiff1d(keys, _keys(dele), assume_unique=True)
    _check_against_bz(g, expected_keys=keys)


def test_ba512_captured_step_full_size(cm):
    """The 512-graph Barabasi-Albert workload, one captured step (every
    graph's inserts then deletes); 24 graphs of the union checked against
    O1 on their own expected edge sets, and the applied counts."""
    import torch
    w = workloads.ba_many(512, rounds=1)
    ns, eoff = w["ns"], w["eoff"]
    g = cm.CoreGraph(None, _dev(w["edges"]), multi=(ns, np.diff(eoff)), stream=torch.cuda.Stream())
    kins, kdel = w["kins"][0], w["kdel"][0]
    st = g.step(int(kins.sum()), int(kdel.sum()))
    pi, pd = st.run(kins, _dev(w["ins"][0]), kdel, _dev(w["dele"][0]))
    assert (pi == kins).all() and (pd == kdel).all()
    cores = g.cores()
    bases = g.bases()
    io = np.concatenate([[0], np.cumsum(kins)])
    do = np.concatenate([[0], np.cumsum(kdel)])
    rng = np.random.default_rng(0)
    for i in sorted(rng.choice(512, 24, replace=False)):
        keys = _keys(w["edges"][eoff[i]:eoff[i + 1]])
        keys = np.union1d(keys, _keys(w["ins"][0][io[i]:io[i + 1]]))
        keys = np.setdiff1d(keys, _keys(w["dele"][0][do[i]:do[i + 1]]), assume_unique=True)
        exp = oracle.bz(int(ns[i]), _pairs(keys), trusted=True)
        assert (cores[bases[i]: bases[i] + ns[i]] == exp).all(), i


def test_serving_full_size(cm):
    """The serving workload's resident graphs (R-MAT scale 22 and the 2048^2
    grid with shortcuts) under a short open-loop trace; afterwards each
    graph holds the cores of its requests applied one by one."""
    import torch
    graphs = workloads.serving_graphs()
    tr = workloads.serving_trace(graphs, 2000, 0.5)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    hs = [cm.CoreGraph(n, _dev(e), stream=torch.cuda.Stream(), max_sms=sms // 2) for n, e in graphs]
    with cm.Server(hs, 1 << 30, max_round_edges=1 << 20) as srv:
        srv.run_trace(tr["arrival_ns"], tr["graph"], tr["op"], tr["counts"], tr["edges"])
        assert srv.drain() == 0
        st = srv.stats()
        assert st["failed"] == 0 and st["edges"] == int(tr["counts"].sum())
        got = [srv.cores(0), srv.cores(1)]
    for gi, (n, e) in enumerate(graphs):
        keys = _keys(e)
        sel = tr["graph"] == gi
        ins = [tr["edges"][tr["off"][j]:tr["off"][j + 1]] for j in np.nonzero(sel & (tr["op"] == 0))[0]]
        dl = [tr["edges"][tr["off"][j]:tr["off"][j + 1]] for j in np.nonzero(sel & (tr["op"] == 1))[0]]
        if ins:
            keys = np.union1d(keys, _keys(np.concatenate(ins)))
        if dl:
            keys = np.setdiff1d(keys, _keys(np.concatenate(dl)), assume_unique=True)
        assert (got[gi] == oracle.bz(n, _pairs(keys), trusted=True)).all(), gi
