"""Host-side pieces of bench.py that need no GPU: the kernel code hash that
decides whether the committed DRAM-traffic capture still applies, and the
--options parser."""
import json
import os

import bench


def test_code_hash_ignores_comments_only():
    src = "int f(int x) {  // doubles\n    /* the\n       body */ return 2 * x;\n}\n\n"
    assert bench._code_only(src) == "int f(int x) {\n     return 2 * x;\n}"
    assert bench._code_only(src) == bench._code_only(src.replace("doubles", "twice"))
    assert bench._code_only(src) != bench._code_only(src.replace("2 * x", "3 * x"))


def test_traffic_applies_only_to_the_captured_kernel(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "maintain_traffic.json")) as f:
        stored = json.load(f)
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: stored["source_sha"])
    for name, w in stored["workloads"].items():
        assert bench.kernel_traffic(name) == w["dram_bytes_per_launch"]
    assert bench.kernel_traffic("no-such-workload") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    for name in stored["workloads"]:
        assert bench.kernel_traffic(name) is None


def test_options_parser():
    class A:
        options = "hub_slots=512, task_claim=2"
    assert bench.handle_options(A()) == {"hub_slots": 512, "task_claim": 2}
    A.options = None
    assert bench.handle_options(A()) == {}


def test_sweep_o3_estimate_weights_cases_by_size():
    """The CPU baseline of the sweep extrapolates per (operation, law) rates
    to every case: total edges over the sum of size / rate."""
    import numpy as np
    sizes = (10, 100)
    batches = {(op, s, law): np.zeros((s, 2), np.int32) for op in bench.SWEEP_OPS for s in sizes
               for law, _ in bench.SWEEP_LAWS}
    rates = {("insert", 0): (10, 1.0), ("insert", 1): (1, 10.0), ("delete", 0): (100, 1.0), ("delete", 1): (50, 1.0)}
    value, t = bench.o3_estimate(rates, batches, sizes, bench.SWEEP_OPS)
    exp_t = 110 / 10.0 + 110 / 0.1 + 110 / 100.0 + 110 / 50.0
    assert abs(t - exp_t) < 1e-9 and abs(value - 440 / exp_t) < 1e-9


def test_sweep_o3_rates_restore_the_oracle_graph():
    """o3_law_rates times O3 on batch prefixes and leaves the oracle graph
    exactly as it found it (edges and cores)."""
    import numpy as np
    import oracle
    from synth import workloads
    n, e, batches = workloads.rmat_sweep(scale=12, sizes=(50, 200))
    og = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL, simple=True)
    c0, m0 = og.cores(), og.m
    offsets = {}
    r = bench.o3_law_rates(og, batches, (50, 200), bench.SWEEP_OPS, 0.01, offsets)
    assert set(r) == {(op, law) for op in bench.SWEEP_OPS for law, _ in bench.SWEEP_LAWS}
    assert all(d >= 1 for d, t in r.values()) and all(offsets[k] == r[k][0] for k in r)
    assert (og.cores() == c0).all() and og.m == m0
    assert (og.cores() == oracle.bz(n, e)).all()


def test_reference_arm_prints_one_line_on_a_small_sweep():
    """The reference arm (the oracle on host cores) on a small R-MAT sweep:
    one JSON line carrying the sweep's metric, its own CPU baseline and an
    e2e record, with no GPU needed."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "12", "--sizes", "100,1000",
                        "--steps", "1", "--warmup", "1", "--ref-budget", "0.2"],
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))), capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["config"]["workload"] == "rmat12-sweep"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
