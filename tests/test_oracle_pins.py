"""The CPU oracle against closed forms, brute force, golden fixtures and the
invariants of Section IV (see tests/pins.py for what pins what)."""
import pytest

import pins


@pytest.mark.parametrize("check", pins.ALL, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(0)


def test_simple_construction_and_restore_match_the_checked_path():
    """or_create_simple builds the same graph and cores as or_create on a
    simple edge list, and restore() (structure-only undo plus saved cores)
    returns a graph to the state that O3 maintenance left it in before."""
    import numpy as np
    import oracle
    import synth

    n = 3000
    e = synth.er(n, 15000, synth.stream(91, 0, 0, synth.GRAPH))
    a = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL)
    b = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL, simple=True)
    assert (a.cores() == b.cores()).all() and (a.cores() == oracle.bz(n, e)).all()
    key = lambda x: np.sort(np.sort(x, 1)[:, 0].astype(np.int64) << 32 | np.sort(x, 1)[:, 1])
    assert (key(a.edges()) == key(b.edges())).all()
    c0 = b.cores()
    ins = synth.static_sample_insert(n, e, 400, synth.PREFERENTIAL, synth.stream(91, 0, 0, synth.INSERT))
    assert b.insert_edges(ins) == len(ins)
    assert (b.cores() == oracle.bz(n, np.concatenate([e, ins]))).all() and not (b.cores() == c0).all()
    b.restore(oracle.DELETE, ins, c0)
    assert (b.cores() == c0).all() and (key(b.edges()) == key(e)).all()
    dl = synth.static_sample_delete(n, e, 400, synth.UNIFORM, synth.stream(91, 0, 0, synth.DELETE))
    assert b.delete_edges(dl) == len(dl)
    b.restore(oracle.INSERT, dl, c0)
    assert (b.cores() == c0).all() and (key(b.edges()) == key(e)).all()
    assert a.insert_edges(ins) == len(ins) and b.insert_edges(ins) == len(ins)
    assert (b.cores() == a.cores()).all()
