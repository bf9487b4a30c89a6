"""Checks that pin the CPU oracle to facts outside itself.

Each check takes ``plant``: 0 runs it against the real oracle; a positive
value runs it against an oracle build with one planted mistake (see the
PLANT switches in oracle/oracle.c), where at least one check must fail.

What pins what:
  * brute force (O2)      closed forms of textbook graphs (complete graphs,
                          cycles, paths, stars, complete bipartite graphs).
  * BZ peeling (O1)       brute force on every graph with <= 6 vertices and on
                          random graphs up to 14 vertices; closed forms at
                          larger sizes (grids, K_n, trees, Barabasi-Albert
                          graphs whose every core equals m).
  * traversal (O3) and    BZ after every single edge / every batch, the
    batched method (O4)   golden fixtures, and per-iteration invariants of
                          Section IV: selection is a superior edge set
                          (Definition 6 (ii) at every level) and maximal,
                          cores move by at most one per iteration (Lemmas 3-4)
                          and only at the levels of the selected edges
                          (Lemmas 1-2 (ii)), insertion never lowers and
                          deletion never raises a core, and the number of
                          iterations is at most 2*Delta_B - 1.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _canon(edges):
    return {(min(u, v), max(u, v)) for u, v in np.asarray(edges).reshape(-1, 2) if u != v}


# ---------------------------------------------------------------- closed forms
def complete(n):
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def path(n):
    return [(i, i + 1) for i in range(n - 1)]


def star(n):
    return [(0, i) for i in range(1, n)]


def kab(a, b):
    return [(i, a + j) for i in range(a) for j in range(b)]


def grid(r, c):
    e = []
    for i in range(r):
        for j in range(c):
            v = i * c + j
            if j + 1 < c:
                e.append((v, v + 1))
            if i + 1 < r:
                e.append((v, v + c))
    return e


def check_brute_closed_forms(plant=0):
    for n in range(1, 9):
        assert (oracle.brute(n, complete(n), plant) == n - 1).all(), f"K{n}"
    for n in range(3, 11):
        assert (oracle.brute(n, cycle(n), plant) == 2).all(), f"C{n}"
        assert (oracle.brute(n, path(n), plant) == 1).all(), f"P{n}"
        assert (oracle.brute(n, star(n), plant) == 1).all(), f"S{n}"
    for a in range(1, 5):
        for b in range(1, 5):
            assert (oracle.brute(a + b, kab(a, b), plant) == min(a, b)).all(), f"K{a},{b}"
    assert (oracle.brute(5, [], plant) == 0).all()


def check_bz_closed_forms(plant=0):
    for n in (2, 5, 17, 40):
        assert (oracle.bz(n, complete(n), plant) == n - 1).all()
    for n in (3, 100, 1001):
        assert (oracle.bz(n, cycle(n), plant) == 2).all()
    assert (oracle.bz(2000, path(2000), plant) == 1).all()
    for r, c in ((2, 2), (7, 9), (40, 40)):
        assert (oracle.bz(r * c, grid(r, c), plant) == 2).all()
    for a, b in ((3, 7), (6, 6), (1, 9)):
        assert (oracle.bz(a + b, kab(a, b), plant) == min(a, b)).all()
    rng = np.random.default_rng(11)
    n = 3000                                         # random recursive tree: every core is 1
    tree = [(int(rng.integers(0, v)), v) for v in range(1, n)]
    assert (oracle.bz(n, tree, plant) == 1).all()
    # Barabasi-Albert with a seed clique K_{m+1}: each vertex has m earlier
    # neighbours, so the whole graph is an m-core and removing vertices in
    # reverse order shows no (m+1)-core exists: every core is m.
    import synth
    for n, m in ((500, 3), (3000, 8)):
        e = synth.ba(n, m, synth.stream(99, n, m))
        assert (oracle.bz(n, e, plant) == m).all()
    # a disjoint union keeps each part's cores; an isolated vertex has core 0
    e = complete(6) + [(6 + u, 6 + v) for u, v in cycle(5)]
    assert oracle.bz(12, e, plant).tolist() == [5] * 6 + [2] * 5 + [0]


def check_bz_vs_brute_exhaustive(plant=0, nmax=6):
    for n in range(1, nmax + 1):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            b = oracle.brute(n, e, plant)
            z = oracle.bz(n, e, plant)
            assert (b == z).all(), (n, e, b, z)


def check_bz_vs_brute_random(plant=0, trials=300, seed=3):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(7, 15))
        p = rng.uniform(0.1, 0.7)
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        assert (oracle.brute(n, e, plant) == oracle.bz(n, e, plant)).all(), (n, e)


# ---------------------------------------------------------------- golden fixtures
def load_golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vals = line.split()
            d[k] = [int(x) for x in vals]
    d["n"] = d["n"][0]
    d["edges"] = np.array(d.get("edges", []), dtype=np.int32).reshape(-1, 2)
    return d


def golden_names():
    return sorted(x for x in os.listdir(GOLDEN) if x.endswith(".txt"))


def check_golden(plant=0):
    for name in golden_names():
        g = load_golden(name)
        n, e = g["n"], g["edges"]
        assert oracle.bz(n, e, plant).tolist() == g["cores"], name
        if n <= 20:
            assert oracle.brute(n, e, plant).tolist() == g["cores"], name
        for mode in (oracle.SEQUENTIAL, oracle.SUPERIOR):
            og = oracle.OracleGraph(n, e, mode=mode, plant=plant)
            assert og.cores().tolist() == g["cores"], name
            if "insert" in g:
                og.insert_edges(np.array(g["insert"]).reshape(-1, 2))
                assert og.cores().tolist() == g["cores_after_insert"], (name, mode)
            if "delete" in g:
                og.delete_edges(np.array(g["delete"]).reshape(-1, 2))
                assert og.cores().tolist() == g["cores_after_delete"], (name, mode)


# ---------------------------------------------------------------- maintenance vs BZ
def _rand_graph(rng, n, p):
    return [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]


def check_o3_every_edge(plant=0, trials=12, seed=5):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(10, 60))
        e = _rand_graph(rng, n, rng.uniform(0.05, 0.3))
        og = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL, plant=plant)
        cur = _canon(e)
        for _ in range(60):
            before = og.cores()
            if rng.random() < 0.5 or not cur:
                u, v = (int(x) for x in rng.integers(0, n, 2))
                if u == v:
                    continue
                og.insert_edges([(u, v)])
                cur.add((min(u, v), max(u, v)))
                d = og.cores() - before
                assert d.min() >= 0 and d.max() <= 1, "single insert moves a core by at most one"
            else:
                u, v = list(cur)[int(rng.integers(0, len(cur)))]
                og.delete_edges([(v, u)])
                cur.discard((u, v))
                d = og.cores() - before
                assert d.max() <= 0 and d.min() >= -1, "single delete moves a core by at most one"
            assert (og.cores() == oracle.bz(n, sorted(cur), plant)).all(), (t, n)


def _constrained(core, u, v):
    k = min(core[u], core[v])
    return [x for x in (u, v) if core[x] == k], k


def run_batch_with_invariants(og, op, batch, plant=0, maximal=True, log=None):
    """Runs one O4 batch through the stepper and asserts the per-iteration
    invariants; returns the number of iterations.  maximal=False for a
    selection whose claim rounds are capped (the set is a superior edge set
    but need not be maximal).  log: a list that receives each iteration's
    selected edges."""
    cur = _canon(og.edges())
    seen, rem = set(), []
    for u, v in np.asarray(batch).reshape(-1, 2):
        u, v = int(u), int(v)
        key = (min(u, v), max(u, v))
        if u == v or key in seen:
            continue
        seen.add(key)
        if (op == oracle.INSERT) == (key in cur):
            continue
        rem.append(key)
    cnt = og.batch_begin(op, batch)
    assert cnt == len(rem)
    inc = {}
    for u, v in rem:
        inc[u] = inc.get(u, 0) + 1
        inc[v] = inc.get(v, 0) + 1
    delta_b = max(inc.values()) if inc else 0
    remset = set(rem)
    iters = 0
    while True:
        before = og.cores()
        r = og.batch_step()
        if r is None:
            break
        iters += 1
        sel, chg = r
        selk = _canon(sel)
        assert len(selk) == len(sel) and selk <= remset, "selected edges come from the remaining batch"
        taken, levels = {}, set()
        for u, v in selk:
            cons, k = _constrained(before, u, v)
            levels.add(k)
            for x in cons:
                assert x not in taken, "Definition 6 (ii): one edge per constrained endpoint"
                taken[x] = (u, v)
        assert selk, "every iteration selects an edge"
        if log is not None:
            log.append([tuple(int(x) for x in e) for e in sel])
        remset -= selk
        for u, v in (remset if maximal else ()):
            cons, _ = _constrained(before, u, v)
            assert any(x in taken for x in cons), "selection is maximal"
        after = og.cores()
        d = after - before
        if op == oracle.INSERT:
            assert d.min() >= 0 and d.max() <= 1, "Lemma 3"
        else:
            assert d.max() <= 0 and d.min() >= -1, "Lemma 4"
        moved = set(np.nonzero(d)[0].tolist())
        assert moved == set(chg.tolist())
        for x in moved:
            assert before[x] in levels, "Lemmas 1-2 (ii): only vertices at a selected level change"
    assert not remset
    if maximal:
        assert iters <= max(2 * delta_b - 1, 0), (iters, delta_b)
    return iters


def check_o4_batches(plant=0, trials=10, seed=7):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(12, 80))
        e = _rand_graph(rng, n, rng.uniform(0.05, 0.25))
        og = oracle.OracleGraph(n, e, mode=oracle.SUPERIOR, plant=plant)
        for b in range(6):
            cur = _canon(og.edges())
            if b % 2 == 0:
                k = int(rng.integers(1, 3 * n))
                batch = rng.integers(0, n, (k, 2))
                # sprinkle repeats, reversed repeats and self-loops
                batch = np.concatenate([batch, batch[: k // 4, ::-1], np.array([[1, 1]])])
                run_batch_with_invariants(og, oracle.INSERT, batch, plant)
            else:
                lst = sorted(cur)
                k = int(rng.integers(0, len(lst) + 1))
                idx = rng.permutation(len(lst))[:k]
                batch = np.array([lst[i] for i in idx] + [(0, n - 1)], dtype=np.int32).reshape(-1, 2)
                run_batch_with_invariants(og, oracle.DELETE, batch, plant)
            assert (og.cores() == oracle.bz(n, og.edges(), plant)).all(), (t, b)


def check_selection_order_worked_examples(plant=0):
    """Worked examples of the selection variants, derived by hand.
    (1) K5 on 0..4 (core 4) and an isolated vertex 5: inserting 5-0 .. 5-4
    (giving K6, core 5) constrains vertex 5 in every edge, so each
    iteration selects one edge, in
    increasing priority: by key (0,5), (1,5), ..., (4,5); by fmix64 of the
    key in that order.  (2) Four isolated vertices and the inserted path
    0-1, 1-2, 2-3 in key order: the claim rounds select (0,1) in round one
    and (2,3) in round two, then (1,2) in the next iteration -- two
    iterations; capped at one round per iteration, three: (0,1), then (1,2)
    (vertex 2 is its only constrained endpoint once 1 has core 1), then
    (2,3)."""
    k5 = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    batch = np.array([(5, 3), (5, 0), (5, 4), (5, 1), (5, 2)], dtype=np.int32)
    for order in (0, 1):
        for rounds in (0, 1):
            og = oracle.OracleGraph(6, k5, mode=oracle.SUPERIOR, plant=plant, select_order=order,
                                    select_rounds=rounds)
            got = []
            run_batch_with_invariants(og, oracle.INSERT, batch, plant, maximal=rounds == 0, log=got)
            keys = [(x, 5) for x in range(5)]
            if order == 0:
                keys.sort(key=lambda e: oracle.fmix64((e[0] << 32) | e[1], plant))
            assert [sorted(map(tuple, map(sorted, it))) for it in got] == [[k] for k in keys], (order, rounds, got)
            assert (og.cores() == 5).all()   # K6
    path = np.array([(2, 3), (0, 1), (1, 2)], dtype=np.int32)
    for rounds, want in ((0, [[(0, 1), (2, 3)], [(1, 2)]]), (1, [[(0, 1)], [(1, 2)], [(2, 3)]]),
                         (2, [[(0, 1), (2, 3)], [(1, 2)]])):
        og = oracle.OracleGraph(4, np.zeros((0, 2), np.int32), mode=oracle.SUPERIOR, plant=plant, select_order=1,
                                select_rounds=rounds)
        got = []
        run_batch_with_invariants(og, oracle.INSERT, path, plant, maximal=rounds != 1, log=got)
        assert [sorted(tuple(sorted(e)) for e in it) for it in got] == want, (rounds, got)
        assert (og.cores() == np.array([1, 1, 1, 1])).all()


def check_selection_variants(plant=0, trials=6, seed=11):
    """Every selection variant reaches the cores of O1 after every batch, and
    claim rounds run to the end select, iteration by iteration, exactly the
    greedy pass's sets (the least-priority-first maximal set)."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(12, 70))
        e = _rand_graph(rng, n, rng.uniform(0.05, 0.25))
        for order in (0, 1):
            gs = {r: oracle.OracleGraph(n, e, mode=oracle.SUPERIOR, plant=plant, select_order=order,
                                        select_rounds=r) for r in (0, 1, 2, 1 << 20)}
            for b in range(4):
                cur = _canon(gs[0].edges())
                if b % 2 == 0:
                    batch = rng.integers(0, n, (int(rng.integers(1, 3 * n)), 2)).astype(np.int32)
                    op = oracle.INSERT
                else:
                    lst = sorted(cur)
                    idx = rng.permutation(len(lst))[: int(rng.integers(0, len(lst) + 1))]
                    batch = np.array([lst[i] for i in idx] + [(0, n - 1)], dtype=np.int32).reshape(-1, 2)
                    op = oracle.DELETE
                logs, its = {}, {}
                for r, og in gs.items():
                    logs[r] = []
                    its[r] = run_batch_with_invariants(og, op, batch, plant, maximal=r in (0, 1 << 20), log=logs[r])
                canon = {r: [sorted(tuple(sorted(x)) for x in it) for it in lg] for r, lg in logs.items()}
                assert canon[1 << 20] == canon[0], (t, order, b)
                # (a capped selection need not take more iterations: a maximal
                # set is not always the best next step)
                ref = oracle.bz(n, gs[0].edges(), plant)
                for r, og in gs.items():
                    assert (og.cores() == ref).all(), (t, order, b, r)


def check_vertex_ops(plant=0, seed=9):
    rng = np.random.default_rng(seed)
    for mode in (oracle.SEQUENTIAL, oracle.SUPERIOR):
        n = 50
        e = _rand_graph(rng, n, 0.12)
        og = oracle.OracleGraph(n, e, mode=mode, plant=plant)
        alive = np.ones(n, dtype=bool)
        for r in range(4):
            nl = [rng.choice(np.nonzero(alive)[0], 5, replace=False).tolist() for _ in range(3)]
            nl[2].append(og.n)          # a new vertex may connect to an earlier new one
            first = og.insert_vertices(nl)
            assert first == len(alive)
            alive = np.concatenate([alive, np.ones(3, dtype=bool)])
            dead = rng.choice(np.nonzero(alive)[0], 2, replace=False)
            og.delete_vertices(dead)
            alive[dead] = False
            c = og.cores()
            assert (c[~alive] == -1).all()
            ref = oracle.bz(og.n, og.edges(), plant)
            assert (c[alive] == ref[alive]).all() and (ref[~alive] == 0).all()


def check_fmix64(plant=0):
    # fmix64 must be a bijection (priorities distinct): invert it explicitly.
    c1, c2 = 0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53
    i1, i2 = pow(c1, -1, 1 << 64), pow(c2, -1, 1 << 64)
    M = (1 << 64) - 1

    def inv(y):
        y ^= y >> 33
        y = (y * i2) & M
        y ^= y >> 33
        y = (y * i1) & M
        y ^= y >> 33
        return y

    rng = np.random.default_rng(1)
    xs = [0, 1, M] + [int(x) for x in rng.integers(0, 1 << 62, 2000, dtype=np.int64)]
    for x in xs:
        assert inv(oracle.fmix64(x, plant)) == x
    assert oracle.fmix64(0, plant) == 0


ALL = [check_brute_closed_forms, check_bz_closed_forms, check_bz_vs_brute_exhaustive,
       check_bz_vs_brute_random, check_golden, check_o3_every_edge, check_o4_batches,
       check_selection_order_worked_examples, check_selection_variants, check_vertex_ops, check_fmix64]
