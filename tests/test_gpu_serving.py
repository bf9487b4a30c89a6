"""Serving loop: resident graphs, admission by a device budget, coalescing
of consecutive same-operation requests, graphs served concurrently.

A graph's core numbers are a function of its edge set (Definitions 1-2),
and coalescing keeps each graph's requests in submission order, so after
a trace every graph must hold the cores of applying its requests one by
one -- served alone or mixed with another graph's traffic, with a roomy
or a tight budget.  Compared exactly with the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads

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
def setup():
    graphs = workloads.serving_graphs(scale=12, side=64)
    tr = workloads.serving_trace(graphs, 600, 0.4, median=20, hi=300)
    # expected final cores: each graph's requests applied one by one
    exp = []
    for gi, (n, e) in enumerate(graphs):
        ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
        for j in np.nonzero(tr["graph"] == gi)[0]:
            b = tr["edges"][tr["off"][j]:tr["off"][j + 1]]
            got = ref.insert_edges(b) if tr["op"][j] == 0 else ref.delete_edges(b)
            assert got == tr["counts"][j]
        exp.append(ref.cores())
        assert (exp[-1] == oracle.bz(n, ref.edges())).all()
    return graphs, tr, exp


def _handles(cm, graphs, which, share_sms=True):
    import torch
    props = torch.cuda.get_device_properties(0)
    hs = []
    for gi in which:
        n, e = graphs[gi]
        opts = {"max_sms": props.multi_processor_count // 2} if share_sms else {}
        hs.append(cm.CoreGraph(n, e, stream=torch.cuda.Stream(), **opts))
    return hs


def _sub(tr, keep, remap):
    idx = np.nonzero(keep)[0]
    edges = np.concatenate([tr["edges"][tr["off"][j]:tr["off"][j + 1]] for j in idx])
    return (tr["arrival_ns"][idx], np.array([remap[g] for g in tr["graph"][idx]], np.int32), tr["op"][idx],
            tr["counts"][idx], edges)


@pytest.mark.parametrize("budget", [1 << 26, 3 * 300 * 16])
def test_alone_equals_mix(cm, setup, budget):
    graphs, tr, exp = setup
    # graph 0 alone
    hs = _handles(cm, graphs, [0])
    with cm.Server(hs, budget) as srv:
        lat, rnd, wall = srv.run_trace(*_sub(tr, tr["graph"] == 0, {0: 0}))
        assert srv.drain() == 0
        alone = srv.cores(0)
        st = srv.stats()
        assert st["failed"] == 0 and st["completed"] == int((tr["graph"] == 0).sum())
        assert (lat > 0).all() and (rnd >= 0).all()
    assert (alone == exp[0]).all()
    # both graphs, mixed
    hs = _handles(cm, graphs, [0, 1])
    with cm.Server(hs, 2 * budget) as srv:
        lat, rnd, wall = srv.run_trace(tr["arrival_ns"], tr["graph"], tr["op"], tr["counts"], tr["edges"])
        assert srv.drain() == 0
        mix = [srv.cores(0), srv.cores(1)]
        st = srv.stats()
        assert st["edges"] == int(tr["counts"].sum())
        assert st["rounds"] + st["coalesced"] == st["completed"] == len(tr["counts"])
    assert (mix[0] == alone).all() and (mix[0] == exp[0]).all()
    assert (mix[1] == exp[1]).all()


def test_coalescing_and_invalid_request(cm, setup):
    """Requests queued together are merged per graph and per operation; a
    request naming a vertex out of range fails alone, its round-mates are
    applied."""
    graphs, tr, exp = setup
    n, e = graphs[1]
    hs = _handles(cm, graphs, [1], share_sms=False)
    ref = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR)
    new = synth.static_sample_insert(n, e, 400, synth.UNIFORM, synth.stream(77))
    with cm.Server(hs, 1 << 24) as srv:
        ids = [srv.submit(0, 0, new[40 * i: 40 * i + 40]) for i in range(5)]
        bad = srv.submit(0, 0, np.array([[1, n + 3]], np.int32))
        ids += [srv.submit(0, 0, new[200 + 40 * i: 240 + 40 * i]) for i in range(5)]
        dl = srv.submit(0, 1, new[:100])
        res = [srv.wait(i) for i in ids]
        rb = srv.wait(bad)
        rd = srv.wait(dl)
        assert all(r["status"] == 0 for r in res)
        assert rb["status"] == cm.CM_ERR_INVALID
        assert rd["status"] == 0 and rd["round_applied"] == 100
        ref.insert_edges(new[:400])
        ref.delete_edges(new[:100])
        assert (srv.cores(0) == ref.cores()).all()
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 12
    with pytest.raises(cm.CoreMaintError):
        with cm.Server(hs, 128) as srv:
            srv.submit(0, 0, new)   # larger than the graph's insert ring
