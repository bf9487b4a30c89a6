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
