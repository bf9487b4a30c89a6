"""Benchmark: batched k-core maintenance on one or more GB300s.

Workload (one "step" = one round of the R-MAT scale-20 stream): R-MAT
(a,b,c,d) = (.57,.19,.19,.05), 2^20 vertices, 16 * 2^20 sampled edges
(symmetrised, deduplicated, ids permuted); each round inserts 10^4 uniform
new edges, deletes 10^4 uniform existing edges, inserts 100 vertices of
degree 8 and deletes 100 uniform live vertices, each as one batched call.

value: edge updates applied per second over K timed rounds, inputs already
in device memory, device time by CUDA events on the handle's stream, L2
flushed (256 MiB write) before every round.  e2e: the same metric through
host (pinned) buffers, copies inside the timed region, and the full core
array read back after every round.  roofline: the maintenance kernel's
algorithmic bytes over its event-timed duration against the measured HBM
copy bandwidth.  cpu_baseline / --impl reference: the CPU oracle (the
paper's sequential single-edge traversal) on a bounded prefix of the
same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: torchrun, one rank per GPU, every rank runs its own replica.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge updates/sec (insert & delete)"
UNIT = "edge updates/s"
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("cm_iterate.cu", "cm_vertex.cuh", "cm_common.cuh", "cm_launch.h")


def _code_only(src: str) -> str:
    """C++ source without comments and blank lines (a comment edit does not
    change the compiled kernel)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_sha() -> str:
    """Hash of the maintenance kernel's code (the kernel file and the headers
    it includes, comments removed), to tell whether a stored ncu capture is
    current."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1612_09368_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def kernel_traffic(workload: str):
    """DRAM bytes per launch (one maintenance call) of the maintenance kernel
    on `workload`, from the committed ncu summary, only if the kernel source
    is unchanged since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "maintain_traffic.json")) as f:
            t = json.load(f)
        if kernel_source_sha() != t.get("source_sha"):
            return None
        w = t.get("workloads", {}).get(workload)
        return None if w is None else w.get("dram_bytes_per_launch")
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sms, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sms)}


def nvtx(push: bool):
    """Brackets a measured maintenance call with an NVTX range named
    "maintenance call" (a no-op unless a profiler listens)."""
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push("maintenance call")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def handle_options(args) -> dict:
    """cm_options fields given as --options name=value,... (defaults otherwise)."""
    out = {}
    for kv in filter(None, (args.options or "").split(",")):
        k, v = kv.split("=")
        out[k.strip()] = int(v)
    return out


def aggregate(t_ms: float, units: float, ws: int, device):
    """Whole-job numbers over the ranks of a multi-GPU run: the slowest
    rank's timed region and the units every rank processed (each rank runs
    its own replica, so per-rank work is fixed as ranks are added)."""
    if ws <= 1:
        return t_ms, units
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms], device=device, dtype=torch.float64)
    uu = torch.tensor([units], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


def make_workload(args, rounds):
    from synth import workloads
    return workloads.rmat_rounds(rounds, scale=args.scale)


def config_of(w, args):
    c = {"workload": w.name, **w.params, "vertices": w.n, "initial_edges": int(len(w.edges)),
         "l2": "flushed before every step (256 MiB write)", "parallelism": "replicas"}
    if handle_options(args):
        c["options"] = handle_options(args)
    return c


# ---------------------------------------------------------------- CPU oracle leg
def cpu_oracle_rate(w, budget_s: float):
    """Edges/s of the paper's sequential single-edge traversal (oracle O3) on
    a prefix of round 0's insert and delete batches, ~budget_s seconds."""
    import oracle
    og = oracle.OracleGraph(w.n, w.edges, mode=oracle.SEQUENTIAL)
    done, t_used = 0, 0.0
    for r in w.rounds:
        t0 = time.perf_counter()
        done += og.insert_edges(r.ins)
        done += og.delete_edges(r.dele)
        og.insert_vertices(r.vnbrs.tolist())
        done += r.vnbrs.size
        done += og.delete_vertices(r.vdel)
        t_used += time.perf_counter() - t0
        if t_used >= budget_s:
            break
    return done / t_used, done, t_used


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args, 8)
    per = []
    total_edges = 0
    total_t = 0.0
    budget = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for s in range(args.warmup + args.steps):
        rate, edges, t = cpu_oracle_rate(w, budget)
        if s >= args.warmup:
            per.append(rate)
            total_edges += edges
            total_t += t
    value = total_edges / total_t if total_t else 0.0
    sample = (f"whole rounds from round 0 of {w.name} until ~{budget:.0f} s per step, "
              "oracle O3 sequential single-edge traversal, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": config_of(w, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU leg
def run_round(g, r, dev_inputs, cm):
    """One step: the four batched calls of a round.  Returns (edge updates,
    stats of each call)."""
    ins, dele, off, nb, vd = dev_inputs
    st = []
    a = g.insert_edges(ins)
    st.append(g.stats())
    b = g.delete_edges(dele)
    st.append(g.stats())
    first, c = cm.cm_insert_vertices(g.handle, off, nb)
    st.append(g.stats())
    d = g.delete_vertices(vd)
    st.append(g.stats())
    return a + b + c + d, st


SWEEP_OPS = ("insert", "delete")
SWEEP_LAWS = ((0, "uniform"), (1, "degree-proportional"))


def sweep_cases(batches):
    """The sweep's cases in a fixed order: by batch size, then operation,
    then endpoint law."""
    return sorted(batches.items(), key=lambda x: (x[0][1], SWEEP_OPS.index(x[0][0]), x[0][2]))


def sweep_config(args, n, m, sizes, ops):
    laws = [nm for _, nm in SWEEP_LAWS if nm.split("-")[0] in args.laws.split(",")]
    c = {"workload": f"rmat{args.scale}-sweep", "scale": args.scale, "edge_factor": 16,
         "rmat_abcd": [0.57, 0.19, 0.19, 0.05], "vertices": n, "initial_edges": m, "batch_sizes": list(sizes),
         "operations": list(ops), "laws": laws,
         "cases_per_step": len(sizes) * len(ops) * len(laws),
         "step": "every case once: its batch applied by one maintenance call, then undone untimed",
         "l2": "flushed before every timed call (256 MiB write)", "parallelism": "replicas"}
    if handle_options(args):
        c["options"] = handle_options(args)
    return c


def sweep_inputs(args):
    from synth import workloads
    sizes = tuple(int(x) for x in args.sizes.split(","))
    ops = tuple(args.ops.split(","))
    t0 = time.time()
    laws = tuple(law for law, nm in SWEEP_LAWS if nm.split("-")[0] in args.laws.split(","))
    n, e, batches = workloads.rmat_sweep(scale=args.scale, sizes=sizes, ops=ops, laws=laws)
    return n, e, batches, sizes, ops, time.time() - t0


def o3_law_rates(og, batches, sizes, ops, budget_s, offsets=None):
    """The paper's sequential single-edge traversal (oracle O3) timed on a
    prefix of the largest batch of every (operation, law), one edge per call,
    until budget_s seconds per pair (at least one edge); the graph is put
    back (structure undone, saved cores restored, untimed) after each.  O3
    handles a batch one edge at a time, so its cost per edge depends on the
    endpoint law and not on the batch size.  offsets: per pair, where in the
    batch the prefix starts (the next call continues after it)."""
    import oracle
    c0 = og.cores()
    out = {}
    for op in ops:
        for law, _ in SWEEP_LAWS:
            if (op, max(sizes), law) not in batches:
                continue
            b = batches[(op, max(sizes), law)]
            start = 0 if offsets is None else offsets.get((op, law), 0) % len(b)
            fwd = og.insert_edges if op == "insert" else og.delete_edges
            done, t = 0, 0.0
            while (done == 0 or t < budget_s) and start + done < len(b):
                t0 = time.perf_counter()
                fwd(b[start + done:start + done + 1])
                t += time.perf_counter() - t0
                done += 1
            og.restore(oracle.DELETE if op == "insert" else oracle.INSERT, b[start:start + done], c0)
            if offsets is not None:
                offsets[(op, law)] = start + done
            out[(op, law)] = (done, t)
    return out


def o3_estimate(rates, batches, sizes, ops):
    """Edge updates/s the O3 traversal would reach on the whole sweep step:
    every case's batch size over its (operation, law) rate, summed."""
    edges = t = 0.0
    for op in ops:
        for law, _ in SWEEP_LAWS:
            if (op, law) not in rates:
                continue
            done, secs = rates[(op, law)]
            for sz in sizes:
                k = len(batches[(op, sz, law)])
                edges += k
                t += k * secs / done
    return edges / t, t


def run_sweep(args):
    """R-MAT scale-24 batch sweep (the HBM-roofline workload, the default):
    per batch size (10^3..10^6), operation and endpoint law (uniform or
    degree-proportional), one maintenance call applies the batch (timed with
    CUDA events on the handle's stream, L2 flushed before) and the batch is
    undone untimed, so every case starts from the generated graph.  A step
    is one pass over the 16 cases."""
    import torch
    import paper_1612_09368_gb300 as cm
    from paper_1612_09368_gb300 import build as libbuild

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    libbuild.build()
    K, W = args.steps, args.warmup
    n, e, batches, sizes, ops, gen_s = sweep_inputs(args)
    cases = sweep_cases(batches)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    g = cm.CoreGraph(n, torch.from_numpy(e).to(dev), stream=stream, **handle_options(args))
    create = g.stats()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    peak, peak_kind = load_peaks()
    dbat = [torch.from_numpy(b).to(dev) for _, b in cases]

    def one_pass(timed_into=None, inputs=dbat):
        for j, ((op, size, law), _) in enumerate(cases):
            fwd = g.insert_edges if op == "insert" else g.delete_edges
            inv = g.delete_edges if op == "insert" else g.insert_edges
            flush.fill_(j)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            nvtx(True)      # a profiler can keep the launches of the measured calls apart
            applied = fwd(inputs[j])
            nvtx(False)
            a1.record(stream)
            a1.synchronize()
            st = g.stats()
            if timed_into is not None:
                timed_into.append((j, a0.elapsed_time(a1), applied, st))
            inv(dbat[j])

    for _ in range(W):
        one_pass()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    torch.cuda.synchronize()
    recs = []
    step_ms = []
    for s in range(K):
        before = len(recs)
        one_pass(recs)
        step_ms.append(sum(r[1] for r in recs[before:]))
    torch.cuda.synchronize()
    clocks = clk.stop()
    if ws > 1:
        dist.barrier()
    t_ms = sum(step_ms)
    units = sum(r[2] for r in recs)
    t_ms_all, units_all = aggregate(t_ms, units, ws, dev)
    value = units_all / (t_ms_all / 1000.0)
    alg = sum(r[3]["alg_bytes"] for r in recs)
    maint = sum(r[3]["maintain_ms"] for r in recs)
    calls = sum(1 for r in recs if r[3]["maintain_ms"] > 0)
    launches = sum(r[3]["launches"] for r in recs)
    achieved = alg / (maint / 1000.0) / 1e9 if maint > 0 else 0.0

    # e2e: the same pass through host (pinned) batches -- the library copies
    # each in inside the timed call -- and the full core array read back to
    # host memory at the end of the step
    e2e = None
    if not args.no_e2e:
        hbat = [torch.from_numpy(b).pin_memory() for _, b in cases]
        cores_h = torch.empty(n, dtype=torch.int32).pin_memory()
        e_ms, e_units = 0.0, 0
        for _ in range(args.e2e_steps):
            rec = []
            one_pass(rec, inputs=hbat)
            flush.fill_(99)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            g.cores(cores_h)
            a1.record(stream)
            a1.synchronize()
            e_ms += sum(r[1] for r in rec) + a0.elapsed_time(a1)
            e_units += sum(r[2] for r in rec)
        e2e = {"value": e_units / (e_ms / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(b.numel() * 4 for b in hbat)),
               "d2h_bytes_per_step": int(4 * n + 8 * len(cases)), "steps": args.e2e_steps,
               "note": "host batches copied in by each call; the core array read back once per step"}

    # per case: median call time over the timed steps, its roofline, and the
    # re-peel comparator (apply the batch to the structure, full GPU peel)
    per_case = []
    for j, ((op, size, law), b) in enumerate(cases):
        rs = [r for r in recs if r[0] == j]
        call_ms = statistics.median(r[1] for r in rs)
        st = rs[-1][3]
        a_gbs = st["alg_bytes"] / (st["maintain_ms"] / 1000.0) / 1e9 if st["maintain_ms"] else 0.0
        row = {"op": op, "batch": size, "law": SWEEP_LAWS[law][1], "applied": rs[-1][2], "call_ms": call_ms,
               "call_ms_min": min(r[1] for r in rs), "call_ms_max": max(r[1] for r in rs),
               "edge_updates_per_s": rs[-1][2] / (call_ms / 1000.0), "iterations": st["iterations"],
               "grid_iterations": st["grid_iterations"], "maintain_ms": st["maintain_ms"],
               "alg_bytes": st["alg_bytes"], "achieved_gbs": a_gbs, "frac": a_gbs / peak,
               "visited": st["visited"], "visited_slots": st["visited_slots"], "evicted": st["evicted"],
               "evicted_slots": st["evicted_slots"], "changed": st["changed"], "waves": st["waves"],
               "select_rounds": st["select_rounds"], "launches": st["launches"],
               "phase_ms": {k: v / 1e6 for k, v in st["phase_ns"].items()}}
        if rank == 0 and not args.no_repeel:
            flush.fill_(7)
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            g.apply_edges(cm.CM_OP_INSERT if op == "insert" else cm.CM_OP_DELETE, dbat[j])
            g.recompute_cores()
            r1.record(stream)
            r1.synchronize()
            rp = r0.elapsed_time(r1)
            pst = g.stats()
            pg = pst["alg_bytes"] / (pst["maintain_ms"] / 1000.0) / 1e9 if pst["maintain_ms"] else 0.0
            g.apply_edges(cm.CM_OP_DELETE if op == "insert" else cm.CM_OP_INSERT, dbat[j])
            g.recompute_cores()
            row.update({"repeel_ms": rp, "speedup_vs_repeel": rp / call_ms, "peel_levels": pst["peel_levels"],
                        "peel_subwaves": pst["waves"], "peel_barriers": pst["barriers"],
                        "peel_phase_ms": {"scan": pst["phase_ns"]["claim"] / 1e6,
                                          "subwaves": pst["phase_ns"]["check"] / 1e6,
                                          "chunks": pst["phase_ns"]["apply"] / 1e6},
                        "peel_ms": pst["maintain_ms"], "peel_alg_bytes": pst["alg_bytes"], "peel_gbs": pg,
                        "peel_frac": pg / peak})
        per_case.append(row)
    repeel = None
    if per_case and "repeel_ms" in per_case[0]:
        pk = [r for r in per_case]
        small = [r["speedup_vs_repeel"] for r in pk if r["batch"] <= 10 ** 4]
        repeel = {"repeel_ms_median": statistics.median(r["repeel_ms"] for r in pk),
                  "speedup_min_small_batches": min(small) if small else None,
                  "speedup_median": statistics.median(r["speedup_vs_repeel"] for r in pk),
                  "peel_roofline": {"peel_and_sd_ms": statistics.median(r["peel_ms"] for r in pk),
                                    "alg_bytes": statistics.median(r["peel_alg_bytes"] for r in pk),
                                    "achieved_gbs": statistics.median(r["peel_gbs"] for r in pk),
                                    "frac": statistics.median(r["peel_frac"] for r in pk),
                                    "levels": statistics.median(r["peel_levels"] for r in pk)}}
    g.close()
    del dbat, flush
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = sweep_cpu_baseline(args, n, e, batches, sizes, ops)

    if rank == 0:
        traffic = kernel_traffic(f"rmat{args.scale}-sweep")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": t_ms_all / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic", "config": sweep_config(args, n, int(len(e)), sizes, ops),
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                             "kernel": "maintain_kernel (grid and single-block launches of one maintenance call)",
                             "launch_unit": "one maintenance call", "calls": calls,
                             "alg_bytes_total": alg, "maintain_ms_total": maint,
                             "alg_bytes_per_launch": alg / max(1, calls), "avg_launch_ms": maint / max(1, calls)},
                "cpu_baseline": cpu, "repeel": repeel,
                "detail": {"step_ms": {"min": min(step_ms), "median": statistics.median(step_ms),
                                       "max": max(step_ms)},
                           "generation_s": gen_s, "create_ms": create["call_ms"],
                           "create_peel_levels": create["peel_levels"], "units": units_all, "cases": per_case}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def sweep_cpu_baseline(args, n, e, batches, sizes, ops):
    """cpu_baseline of the sweep: oracle O3 on prefixes of every (operation,
    law), extrapolated to the whole step (see o3_law_rates)."""
    import oracle
    og = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL, simple=True)
    per = max(0.5, args.cpu_budget / (len(ops) * len(SWEEP_LAWS)))
    rates = o3_law_rates(og, batches, sizes, ops, per)
    value, est_s = o3_estimate(rates, batches, sizes, ops)
    sampled = {f"{op}/{SWEEP_LAWS[law][1]}": {"edges": d, "seconds": t, "edges_per_s": d / t}
               for (op, law), (d, t) in rates.items()}
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle O3 (sequential single-edge traversal, 1 thread) on a prefix of the largest batch "
                       f"of every operation and law, ~{per:.1f} s each (at least one edge), graph restored after "
                       "each; the step's rate is every case's size over its (operation, law) rate, summed"),
            "estimated_step_s": est_s, "sampled": sampled}


def run_reference_sweep(args):
    """--impl reference on the sweep: oracle O3 on the host, each step a
    bounded sample of every (operation, law), continuing down the batch from
    step to step; value = the step's edge updates/s extrapolated from the
    sampled rates (o3_estimate), ms_per_step = the time actually spent."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    n, e, batches, sizes, ops, gen_s = sweep_inputs(args)
    og = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL, simple=True)
    per = max(0.25, args.ref_budget / (len(ops) * len(SWEEP_LAWS)))
    offsets = {}
    pooled = {}
    step_s = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = o3_law_rates(og, batches, sizes, ops, per, offsets)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            step_s.append(dt)
            for k, (d, t) in r.items():
                pd, pt = pooled.get(k, (0, 0.0))
                pooled[k] = (pd + d, pt + t)
    value, est_s = o3_estimate(pooled, batches, sizes, ops)
    sample = (f"oracle O3 (sequential single-edge traversal, 1 thread): per step a prefix of the largest batch of "
              f"every operation and law, ~{per:.2f} s each (at least one edge), continuing down the batch from step "
              "to step, graph restored after each; value = the step's edge updates/s extrapolated from the "
              "pooled rates (every case's size over its rate)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(step_s) / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": sweep_config(args, n, int(len(e)), sizes, ops),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "detail": {"estimated_full_step_s": est_s, "generation_s": gen_s,
                       "sampled": {f"{op}/{SWEEP_LAWS[law][1]}": {"edges": d, "seconds": t}
                                   for (op, law), (d, t) in pooled.items()}}}
    print(json.dumps(line), flush=True)
    return 0


def shard_workload(w, rank, world):
    """The part of a many-graph workload (ba_many's dict) that one rank owns
    under the library's partition of graphs over ranks."""
    from paper_1612_09368_gb300.shard import partition, select
    ms = np.diff(w["eoff"])
    own = partition(ms, world)[rank]
    _, edges = select(ms, w["edges"], own)
    out = {"ns": w["ns"][own], "ms": w["ms"][own], "edges": edges,
           "eoff": np.concatenate([[0], np.cumsum(ms[own])]).astype(np.int64),
           "kins": w["kins"][:, own], "kdel": w["kdel"][:, own], "ins": [], "dele": []}
    for r in range(len(w["ins"])):
        out["ins"].append(select(w["kins"][r], w["ins"][r], own)[1])
        out["dele"].append(select(w["kdel"][r], w["dele"][r], own)[1])
    return out


def run_batched(args):
    """512 independent Barabasi-Albert graphs, each with its own update batch
    (70% inserts, 30% deletes), applied by ONE captured step per round (one
    CUDA graph replay: every graph's inserts, then every graph's deletes),
    with the schedule picked by the library's autotuner; compared with the
    untuned step and with one insert call plus one delete call per graph.
    Every round is undone (untimed) so each starts from the generated graphs."""
    import torch
    import paper_1612_09368_gb300 as cm
    from paper_1612_09368_gb300 import build as libbuild
    from synth import workloads

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    libbuild.build()
    K, W = args.steps, args.warmup
    ncmp = max(1, min(3, K))
    t0 = time.time()
    w = workloads.ba_many(args.graphs, rounds=W + K)
    if ws > 1:   # independent graphs shard by graph: this rank keeps its own, no collective
        w = shard_workload(w, rank, ws)
    gen_s = time.time() - t0
    ns, ms, eoff = w["ns"], w["ms"], w["eoff"]
    ng = len(ns)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(dev)
    peak, peak_kind = load_peaks()
    with torch.cuda.stream(stream):
        g = cm.CoreGraph(None, torch.from_numpy(w["edges"]).to(dev), multi=(ns, np.diff(eoff)), stream=stream,
                         **handle_options(args))
        create = g.stats()
        bases = g.bases()
        kins, kdel = w["kins"], w["kdel"]
        max_i, max_d = int(kins.sum(1).max()), int(kdel.sum(1).max())
        fwd = g.step(max_i, max_d)
        inv = g.step(max_d, max_i)
        dins = [torch.from_numpy(a).to(dev) for a in w["ins"]]
        ddel = [torch.from_numpy(x).to(dev) for x in w["dele"]]
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

        def fwd_run(r, step=fwd):
            return step.run(kins[r], dins[r], kdel[r], ddel[r])

        def undo(r):
            inv.run(kdel[r], ddel[r], kins[r], dins[r])

        def timed(fn):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1), out

        # untuned step (the handle's default schedule) on the warm-up rounds
        untuned_ms = []
        for r in range(W):
            ms_, _ = timed(lambda: fwd_run(r))
            untuned_ms.append(ms_)
            undo(r)
        default_cfg = fwd.config.as_dict()
        t1 = time.time()
        tune = fwd.autotune(kins[0], dins[0], kdel[0], ddel[0], reps=2)
        tune_s = time.time() - t1
        for r in range(W):               # warm-up with the tuned schedule
            fwd_run(r)
            undo(r)
        torch.cuda.synchronize()
        clk = ClockSampler(0)
        clk.start()
        step_ms, applied, maint_ms, alg, iters, launches = [], 0, 0.0, 0, [], 0
        for r in range(W, W + K):
            ms_, (pi, pd) = timed(lambda: fwd_run(r))
            st = g.stats()
            step_ms.append(ms_)
            applied += int(pi.sum() + pd.sum())
            maint_ms += st["maintain_ms"]
            alg += st["alg_bytes"]
            iters.append(st["iterations"])
            launches += st["launches"]
            undo(r)
        clocks = clk.stop()
        t_ms = sum(step_ms)
        value = applied / (t_ms / 1000.0)
        # comparator: one insert call and one delete call per graph
        cmp_ms, cmp_applied = [], 0
        for r in range(W, W + ncmp):
            io = np.concatenate([[0], np.cumsum(kins[r])])
            do = np.concatenate([[0], np.cumsum(kdel[r])])
            gi = [(dins[r][io[i]:io[i + 1]] + int(bases[i])).contiguous() for i in range(ng)]
            gd = [(ddel[r][do[i]:do[i + 1]] + int(bases[i])).contiguous() for i in range(ng)]
            torch.cuda.synchronize()

            def per_graph():
                n_ = 0
                for i in range(ng):
                    n_ += g.insert_edges(gi[i]) + g.delete_edges(gd[i])
                return n_

            ms_, n_ = timed(per_graph)
            cmp_ms.append(ms_)
            cmp_applied += n_
            undo(r)
        cmp_value = cmp_applied / (sum(cmp_ms) / 1000.0)
        # e2e: pinned host batches in, the full core array out, every step
        e2e_ms, e2e_applied = [], 0
        hin = [(torch.from_numpy(w["ins"][r]).pin_memory(), torch.from_numpy(w["dele"][r]).pin_memory())
               for r in range(W, W + ncmp)]
        cores_h = torch.empty(int(g.n), dtype=torch.int32).pin_memory()
        cores_d = torch.empty(int(g.n), dtype=torch.int32, device=dev)
        for j, r in enumerate(range(W, W + ncmp)):
            def e2e_step():
                pi, pd = fwd.run(kins[r], hin[j][0], kdel[r], hin[j][1])
                g.cores(cores_d)
                cores_h.copy_(cores_d, non_blocking=True)
                return int(pi.sum() + pd.sum())
            ms_, n_ = timed(e2e_step)
            e2e_ms.append(ms_)
            e2e_applied += n_
            undo(r)
        e2e_value = e2e_applied / (sum(e2e_ms) / 1000.0)
        counters = fwd.counters()
        untuned_value = float(np.mean([(kins[r].sum() + kdel[r].sum()) / (untuned_ms[r] / 1000.0)
                                       for r in range(W)]))
    achieved = alg / (maint_ms / 1000.0) / 1e9 if maint_ms > 0 else 0.0
    t_ms, units_all = aggregate(t_ms, applied, ws, dev)
    value = units_all / (t_ms / 1000.0)
    if ws > 1:
        dist.destroy_process_group()
        if rank != 0:
            fwd.close()
            inv.close()
            g.close()
            return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"ba{args.graphs}-batched", "graphs": args.graphs, "graphs_on_rank0": ng,
                       "vertices": int(ns.sum()),
                       "initial_edges": int(eoff[-1]), "n_range": [int(ns.min()), int(ns.max())],
                       "attachment_range": [int(ms.min()), int(ms.max())],
                       "batch_per_round": int(kins[W:].sum() / K + kdel[W:].sum() / K),
                       "insert_fraction": 0.7, "l2": "flushed before every step (256 MiB write)",
                       "parallelism": "one captured step per round" if ws == 1 else
                       f"graphs sharded over {ws} ranks (largest first onto the least-loaded rank), "
                       "one captured step per round per rank, no collective"},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int((kins[W:W + ncmp].sum() + kdel[W:W + ncmp].sum()) * 8 / ncmp),
                    "d2h_bytes_per_step": int(g.n) * 4, "steps": ncmp},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "maintain_kernel (both modes, inside the step's loop nodes)"},
            "cpu_baseline": None,
            "one_launch_per_graph": {"value": cmp_value, "unit": UNIT, "ms_per_step": sum(cmp_ms) / ncmp,
                                     "steps": ncmp, "speedup_of_step": value / cmp_value},
            "untuned_step": {"value": untuned_value, "config": default_cfg, "ms": untuned_ms},
            "autotune": {**tune, "seconds": tune_s},
            "step_counters": counters,
            "detail": {"generation_s": gen_s, "create_ms": create["call_ms"], "step_ms": step_ms,
                       "iterations": iters, "maintain_ms_total": maint_ms}}
    print(json.dumps(line), flush=True)
    fwd.close()
    inv.close()
    g.close()
    return 0


def run_serving(args):
    """Serving: an R-MAT scale-22 graph and a 2048 x 2048 grid with 1%
    shortcuts resident on the device, update requests arriving as a Poisson
    stream (70% inserts, log-normal sizes, median 200), served by the
    library's request loop (admission into a device budget, coalescing of
    consecutive same-operation requests, the two graphs on separate streams
    and SM shares).  Sweeps the arrival rate; the headline is the highest
    sustained rate (every request done within 1 s of the last arrival) and
    its p50 / p99 latency.  Times are host-clock, host inputs to results."""
    import torch
    import paper_1612_09368_gb300 as cm
    from paper_1612_09368_gb300 import build as libbuild
    from synth import workloads

    libbuild.build()
    torch.cuda.set_device(0)
    rates = [float(x) for x in args.rates.split(",")]
    D = args.duration
    t0 = time.time()
    graphs = workloads.serving_graphs(scale=args.scale)
    full = workloads.serving_trace(graphs, max(rates), D)
    gen_s = time.time() - t0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    keep_u = np.array([synth_uniform(i) for i in range(len(full["counts"]))])
    clk = ClockSampler(0)
    clk.start()
    rows = []
    for lam in sorted(rates):
        keep = keep_u < lam / max(rates)
        idx = np.nonzero(keep)[0]
        edges = np.concatenate([full["edges"][full["off"][j]:full["off"][j + 1]] for j in idx])
        hs = [cm.CoreGraph(n, torch.from_numpy(e).cuda(), stream=torch.cuda.Stream(),
                           **{"max_sms": sms // 2, **handle_options(args)})
              for n, e in graphs]
        torch.cuda.synchronize()
        with cm.Server(hs, args.budget, max_round_edges=args.max_round) as srv:
            lat, rnd, wall = srv.run_trace(full["arrival_ns"][idx], full["graph"][idx], full["op"][idx],
                                           full["counts"][idx], edges)
            st = srv.stats()
        for h in hs:
            h.close()
        upd = int(full["counts"][idx].sum())
        last_arrival = full["arrival_ns"][idx].max() / 1e9 if len(idx) else 0.0
        rows.append({"rate_req_s": lam, "requests": int(len(idx)), "offered_updates_s": upd / D,
                     "updates_s": upd / wall, "wall_s": wall, "drain_s": wall - last_arrival,
                     "p50_ms": float(np.percentile(lat, 50) / 1e6), "p99_ms": float(np.percentile(lat, 99) / 1e6),
                     "rounds": st["rounds"], "coalesced": st["coalesced"], "failed": st["failed"],
                     "sustained": bool(wall - last_arrival <= 1.0 and st["failed"] == 0)})
        print(json.dumps({"serving_rate": rows[-1]}), file=sys.stderr, flush=True)
    clocks = clk.stop()
    ok = [r for r in rows if r["sustained"]]
    best = max(ok, key=lambda r: r["updates_s"]) if ok else max(rows, key=lambda r: r["updates_s"])

    def near(frac):
        want = frac * best["rate_req_s"]
        return min(rows, key=lambda r: abs(r["rate_req_s"] - want))

    line = {"metric": METRIC + ", p99 ms (serving)", "value": best["updates_s"], "unit": UNIT, "n_gpus": 1,
            "steps": len(rows), "warmup": 0, "ms_per_step": 1000 * best["wall_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serving-rmat22-grid2048", "graphs": [
                {"kind": "rmat", "scale": args.scale, "edge_factor": 16,
                 "vertices": graphs[0][0], "edges": int(len(graphs[0][1]))},
                {"kind": "grid+shortcuts", "side": 2048, "vertices": graphs[1][0], "edges": int(len(graphs[1][1]))}],
                "arrivals": "Poisson", "duration_s": D, "batch": "log-normal median 200, sigma 1.5, [10, 1e5]",
                "insert_fraction": 0.7, "device_budget_bytes": args.budget, "max_round_edges": args.max_round,
                "sm_share": f"{sms // 2} SMs per graph", "timing": "host clock, host inputs to finished rounds"},
            "clocks": clocks,
            "e2e": {"value": best["updates_s"], "unit": UNIT,
                    "h2d_bytes_per_step": int(8 * best["updates_s"] * best["wall_s"]), "d2h_bytes_per_step": 0,
                    "note": "the serving numbers are end-to-end: host batches in, host-clock latency"},
            "gpu_launches": None, "roofline": None, "cpu_baseline": None,
            "serving": {"sustained_rate_req_s": best["rate_req_s"], "p50_ms": best["p50_ms"],
                        "p99_ms": best["p99_ms"], "p50_ms_at_50pct": near(0.5)["p50_ms"],
                        "p99_ms_at_50pct": near(0.5)["p99_ms"], "p50_ms_at_80pct": near(0.8)["p50_ms"],
                        "p99_ms_at_80pct": near(0.8)["p99_ms"], "sweep": rows},
            "detail": {"generation_s": gen_s}}
    print(json.dumps(line), flush=True)
    return 0


def synth_uniform(i: int) -> float:
    """Thinning draw of request i (Poisson thinning keeps each request of the
    densest stream with probability rate / max rate)."""
    import synth
    return synth.uniform(synth.stream(5, 0, 0, synth.PARAM), i)


def run_study(args):
    """Sequential against superior-edge-set processing on the paper's
    synthetic families (Section VII, the scalability experiments): ER, BA
    and R-MAT graphs of average degree 8 with n = 2^15 ... 2^21; per graph
    10^4 uniform new edges inserted, then 10^4 uniform existing edges (of
    the generated graph) deleted.  Per case: the GPU call time and its
    iterations, the iteration bound of the first iteration (the most batch
    edges one vertex constrains at its level, from the cores before the
    batch), and the paper's sequential single-edge traversal (oracle O3,
    one host core) timed on a prefix of the same batch and extrapolated."""
    import torch
    import oracle
    import synth
    import paper_1612_09368_gb300 as cm
    from paper_1612_09368_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scales = [int(x) for x in args.study_scales.split(",")]
    k = 10 ** 4
    rows = []

    def bound(cores, batch):
        c = cores[batch]
        lvl = c.min(1)
        cons = np.concatenate([batch[:, 0][c[:, 0] == lvl], batch[:, 1][c[:, 1] == lvl]])
        return int(np.bincount(cons).max()) if len(cons) else 0

    def o3_rate(n, e, batch, op, budget):
        og = oracle.OracleGraph(n, e, mode=oracle.SEQUENTIAL)
        done, t = 0, 0.0
        while done < len(batch) and t < budget:
            part = batch[done: done + max(50, min(2000, done or 50))]
            t0 = time.perf_counter()
            (og.insert_edges if op == 0 else og.delete_edges)(part)
            t += time.perf_counter() - t0
            done += len(part)
        return done / t, done

    for fam in ("er", "ba", "rmat"):
        for sc in scales:
            n = 1 << sc
            seed = synth.stream(6, sc, 0, synth.GRAPH) + {"er": 0, "ba": 1, "rmat": 2}[fam]
            if fam == "er":
                e = synth.er(n, 4 * n, seed)
            elif fam == "ba":
                e = synth.ba(n, 4, seed)
            else:
                e = synth.rmat(sc, 4, seed)
            ins = synth.static_sample_insert(n, e, k, synth.UNIFORM, synth.stream(6, sc, 1, synth.INSERT))
            # the deletes are edges of the generated graph (none of them inserted above)
            dele = synth.static_sample_delete(n, e, k, synth.PREFERENTIAL, synth.stream(6, sc, 1, synth.DELETE))
            g = cm.CoreGraph(n, torch.from_numpy(e).to(dev))
            c0 = g.cores()
            bi = bound(c0, ins)
            g.insert_edges(torch.from_numpy(ins).to(dev))
            si = g.stats()
            c1 = g.cores()
            bd = bound(c1, dele)
            g.delete_edges(torch.from_numpy(dele).to(dev))
            sd = g.stats()
            c2 = g.cores()
            g.close()
            # cores checked against O1 (Batagelj-Zaversnik) of the expected graphs
            checked = n <= (1 << args.check_max_scale)
            if checked:
                e1 = np.concatenate([e, ins])
                assert (c0 == oracle.bz(n, e, trusted=True)).all(), (fam, sc, "create")
                assert (c1 == oracle.bz(n, e1, trusted=True)).all(), (fam, sc, "insert")
                k1 = (np.minimum(e1[:, 0], e1[:, 1]).astype(np.int64) << 32) | np.maximum(e1[:, 0], e1[:, 1])
                kd = (np.minimum(dele[:, 0], dele[:, 1]).astype(np.int64) << 32) | np.maximum(dele[:, 0], dele[:, 1])
                e2 = e1[~np.isin(k1, kd)]
                assert (c2 == oracle.bz(n, e2, trusted=True)).all(), (fam, sc, "delete")
            ri, ni = o3_rate(n, e, ins, 0, args.study_budget)
            rd, nd = o3_rate(n, e, dele, 1, args.study_budget)
            row = {"family": fam, "n": n, "edges": int(len(e)), "max_core": int(c0.max()),
                   "cores_checked_against_o1": bool(checked),
                   "insert": {"gpu_ms": si["call_ms"], "iterations": si["iterations"], "first_bound": bi,
                              "o3_edges_per_s": ri, "o3_sample": ni,
                              "speedup_vs_o3": (k / ri * 1000.0) / si["call_ms"]},
                   "delete": {"gpu_ms": sd["call_ms"], "iterations": sd["iterations"], "first_bound": bd,
                              "o3_edges_per_s": rd, "o3_sample": nd,
                              "speedup_vs_o3": (k / rd * 1000.0) / sd["call_ms"]}}
            rows.append(row)
            print(json.dumps({"study_case": row}), file=sys.stderr, flush=True)
    line = {"metric": "sequential vs superior-edge-set study (iterations, GPU ms, speedup over the sequential traversal)",
            "workload": "study", "unit": "ms", "n_gpus": 1, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "study-er-ba-rmat", "average_degree": 8, "updates": k, "scales": scales,
                       "o3": f"oracle O3 on one host core, prefix of each batch up to {args.study_budget} s, extrapolated"},
            "study": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_paper_experiments(args):
    """The paper's two efficiency experiments (Section VII, "Performance
    Evaluation"), on an R-MAT graph standing in for its SNAP graphs:
    (1) batch size: P% of the graph's edges (P = 3, 6, 9, 12, 15) chosen
        uniformly are deleted in one call and then inserted back in one
        call (which restores the graph);
    (2) core distribution of the updates: for five core numbers K1 < ... <
        K5 spread over the graph's edge-core distribution, 20% of the edges
        whose core number (the smaller core of the endpoints) is K are
        deleted and inserted back.
    Reported per call: GPU time, time per edge, iterations."""
    import torch
    import synth
    import paper_1612_09368_gb300 as cm
    from paper_1612_09368_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sc = args.scale
    n = 1 << sc
    import oracle
    e = synth.rmat(sc, 16, synth.stream(7, 0, 0, synth.GRAPH))
    g = cm.CoreGraph(n, torch.from_numpy(e).to(dev))
    cores = g.cores()
    check = sc <= args.check_max_scale
    if check:
        assert (cores == oracle.bz(n, e, trusted=True)).all(), "initial cores differ from O1"
    rng = np.random.default_rng(7)

    def cycle(sel):
        b = torch.from_numpy(np.ascontiguousarray(e[sel])).to(dev)
        out = {}
        for name, fn in (("delete", g.delete_edges), ("insert", g.insert_edges)):
            k = fn(b)
            st = g.stats()
            out[name] = {"edges": k, "call_ms": st["call_ms"], "us_per_edge": 1000.0 * st["call_ms"] / max(1, k),
                         "iterations": st["iterations"], "grid_iterations": st["grid_iterations"]}
            if name == "delete" and check:   # the deleted state against O1 of the graph without them
                keep = np.ones(len(e), bool)
                keep[sel] = False
                assert (g.cores() == oracle.bz(n, e[keep], trusted=True)).all(), "cores after the delete differ from O1"
        assert (g.cores() == cores).all(), "a delete then re-insert must restore every core"
        return out

    size_rows = []
    for pct in (3, 6, 9, 12, 15):
        sel = rng.choice(len(e), int(len(e) * pct / 100), replace=False)
        size_rows.append({"percent": pct, **cycle(sel)})
        print(json.dumps({"size_case": size_rows[-1]}), file=sys.stderr, flush=True)
    ecore = np.minimum(cores[e[:, 0]], cores[e[:, 1]])
    levels = np.unique(ecore)
    picks = levels[np.clip((np.array([0.1, 0.3, 0.5, 0.7, 0.9]) * (len(levels) - 1)).round().astype(int), 0,
                           len(levels) - 1)]
    core_rows = []
    for K in picks:
        idx = np.nonzero(ecore == K)[0]
        sel = rng.choice(idx, max(1, int(0.2 * len(idx))), replace=False)
        core_rows.append({"core": int(K), "edges_at_core": int(len(idx)), **cycle(sel)})
        print(json.dumps({"core_case": core_rows[-1]}), file=sys.stderr, flush=True)
    g.close()
    line = {"metric": "paper experiments: time per edge and iterations by batch size and by edge core number",
            "workload": "paper-experiments", "unit": "us/edge", "n_gpus": 1, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"rmat{sc}-paper-experiments", "scale": sc, "edge_factor": 16,
                       "vertices": n, "edges": int(len(e)), "max_core": int(cores.max()),
                       "cores_checked_against_o1": bool(check),
                       "note": "R-MAT stands in for the paper's SNAP graphs; every case deletes then re-inserts"},
            "batch_size": size_rows, "core_distribution": core_rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 10 for the sweep, 100 rounds)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24-sweep", choices=["rmat24-sweep", "rmat20-rounds", "ba512-batched",
                                                                  "serving", "study", "paper-experiments"])
    ap.add_argument("--study-scales", dest="study_scales", default="15,17,19,21")
    ap.add_argument("--study-budget", dest="study_budget", type=float, default=3.0)
    ap.add_argument("--rates", default="500,1000,2000,4000,8000,16000")
    ap.add_argument("--duration", type=float, default=3.0)
    ap.add_argument("--budget", type=int, default=1 << 30)
    ap.add_argument("--max-round", dest="max_round", type=int, default=1 << 20)
    ap.add_argument("--graphs", type=int, default=512)
    ap.add_argument("--options", default="", help="cm_options fields, e.g. block_slots=256,hub_slots=4096")
    ap.add_argument("--scale", type=int, default=None)
    ap.add_argument("--sizes", default="1000,10000,100000,1000000")
    ap.add_argument("--ops", default="insert,delete")
    ap.add_argument("--laws", default="uniform,degree", help="sweep endpoint laws: uniform, degree")
    ap.add_argument("--cpu-budget", dest="cpu_budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", dest="ref_budget", type=float, default=4.0,
                    help="reference arm: seconds of O3 sampling per step")
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-repeel", action="store_true")
    ap.add_argument("--check-max-scale", dest="check_max_scale", type=int, default=22,
                    help="study / paper-experiments: check cores against O1 up to 2^this many vertices")
    args = ap.parse_args()
    if args.scale is None:
        args.scale = {"rmat24-sweep": 24, "serving": 22}.get(args.workload, 20)
    if args.steps is None:
        args.steps = {"rmat24-sweep": 10, "rmat20-rounds": 100}.get(args.workload, 5)
    if args.impl == "reference":
        return run_reference_sweep(args) if args.workload == "rmat24-sweep" else run_reference(args)
    if args.workload == "rmat24-sweep":
        return run_sweep(args)
    if args.workload == "rmat20-rounds":
        return run_rounds(args)
    if args.workload == "ba512-batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "study":
        return run_study(args)
    if args.workload == "paper-experiments":
        return run_paper_experiments(args)
    return 2


def run_rounds(args):
    """R-MAT scale-20 rounds (a secondary workload): each step is one round of
    10^4 uniform new edges inserted, 10^4 uniform existing edges deleted,
    100 vertices of degree 8 inserted and 100 uniform live vertices deleted,
    each as one batched call."""
    import torch
    import paper_1612_09368_gb300 as cm
    from paper_1612_09368_gb300 import build as libbuild

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    libbuild.build()
    K, W = args.steps, args.warmup
    e2e_rounds = 0 if args.no_e2e else min(K, 20)
    w = make_workload(args, W + K + e2e_rounds)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    g = cm.CoreGraph(w.n, torch.from_numpy(w.edges).to(dev), stream=stream, **handle_options(args))

    def to_dev(r):
        off = np.zeros(len(r.vnbrs) + 1, np.int64)
        off[1:] = np.cumsum([r.vnbrs.shape[1]] * len(r.vnbrs))
        return (torch.from_numpy(r.ins).to(dev), torch.from_numpy(r.dele).to(dev), torch.from_numpy(off).to(dev),
                torch.from_numpy(np.ascontiguousarray(r.vnbrs.ravel())).to(dev), torch.from_numpy(r.vdel).to(dev))

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]

    # warm-up rounds
    for s in range(W):
        run_round(g, w.rounds[s], to_dev(w.rounds[s]), cm)
    dev_in = [to_dev(w.rounds[W + s]) for s in range(K)]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    torch.cuda.synchronize()
    units = 0
    maint_ms = 0.0
    alg_bytes = 0
    maint_launches = 0
    launches = 0
    iters = []
    per_call_ms = {"insert": [], "delete": [], "vinsert": [], "vdelete": []}
    per_call_it = {k: [] for k in per_call_ms}
    per_call_grid_it = {k: 0 for k in per_call_ms}
    per_call_bar = {k: 0 for k in per_call_ms}
    per_call_maint = {k: [] for k in per_call_ms}
    per_call_launch = {k: 0 for k in per_call_ms}
    per_call_vol = {k: {"visited": 0, "visited_slots": 0, "evicted": 0, "evicted_slots": 0, "changed": 0,
                        "changed_slots": 0, "waves": 0, "select_rounds": 0} for k in per_call_ms}
    phase_ns = {}
    for s in range(K):
        flush.fill_(s)
        ev0[s].record(stream)
        u, st = run_round(g, w.rounds[W + s], dev_in[s], cm)
        ev1[s].record(stream)
        units += u
        for name, x in zip(per_call_ms, st):
            per_call_ms[name].append(x["call_ms"])
            per_call_it[name].append(x["iterations"])
            per_call_grid_it[name] += x["grid_iterations"]
            per_call_bar[name] += x["barriers"]
            per_call_maint[name].append(x["maintain_ms"])
            per_call_launch[name] += x["launches"]
            for vk in per_call_vol[name]:
                per_call_vol[name][vk] += x[vk]
            for ph, ns in x["phase_ns"].items():
                phase_ns[ph] = phase_ns.get(ph, 0) + ns
            maint_ms += x["maintain_ms"]
            alg_bytes += x["alg_bytes"]
            launches += x["launches"]
            maint_launches += 1 if x["maintain_ms"] > 0 else 0
            iters.append(x["iterations"])
    torch.cuda.synchronize()
    clocks = clk.stop()
    round_ms = [ev0[s].elapsed_time(ev1[s]) for s in range(K)]
    t_ms = sum(round_ms)
    t_ms, units_all = aggregate(t_ms, units, ws, dev)
    value = units_all / (t_ms / 1000.0)

    # e2e: host pinned inputs, copies and the core read-back inside the timed region
    e2e = None
    if e2e_rounds:
        host_in = []
        for s in range(e2e_rounds):
            r = w.rounds[W + K + s]
            off = np.zeros(len(r.vnbrs) + 1, np.int64)
            off[1:] = np.cumsum([r.vnbrs.shape[1]] * len(r.vnbrs))
            host_in.append(tuple(torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
                                 for x in (r.ins, r.dele, off, r.vnbrs.ravel(), r.vdel)))
        out = torch.empty(g.n + 2 * e2e_rounds * 200, dtype=torch.int32).pin_memory()
        h2d = sum(sum(x.numel() * x.element_size() for x in hi) for hi in host_in) / e2e_rounds
        e_units = 0
        e_ms = 0.0
        d2h = 0
        for s in range(e2e_rounds):
            flush.fill_(s)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            u, _ = run_round(g, w.rounds[W + K + s], host_in[s], cm)
            n_now = g.n
            g.cores(out[:n_now])
            a1.record(stream)
            a1.synchronize()
            e_ms += a0.elapsed_time(a1)
            e_units += u
            d2h += 4 * n_now
        e2e = {"value": e_units / (e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h / e2e_rounds)}

    # re-peel comparator: apply 10^4 new edges structurally + full GPU peel,
    # against maintaining the same-size insert batches above
    repeel = None
    if rank == 0:
        from synth import UNIFORM, stream as sstream
        extra = w.final.sample_insert(10 ** 4, UNIFORM, sstream(2, 0, 10 ** 6, 1))
        xin = torch.from_numpy(extra).to(dev)
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        r0.record(stream)
        g.apply_edges(cm.CM_OP_INSERT, xin)
        g.recompute_cores()
        r1.record(stream)
        r1.synchronize()
        rp_ms = r0.elapsed_time(r1)
        mi = statistics.median(per_call_ms["insert"])
        pst = g.stats()
        pk, _ = load_peaks()
        pgbs = pst["alg_bytes"] / (pst["maintain_ms"] / 1000.0) / 1e9 if pst["maintain_ms"] else 0.0
        repeel = {"repeel_ms": rp_ms, "maintain_insert_1e4_ms_median": mi, "speedup": rp_ms / mi,
                  "peel_levels": pst["peel_levels"], "peel_subwaves": pst["waves"],
                  "peel_roofline": {"peel_and_sd_ms": pst["maintain_ms"], "alg_bytes": pst["alg_bytes"],
                                    "achieved_gbs": pgbs, "frac": pgbs / pk if pk else None}}

    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (maint_ms / 1000.0) / 1e9 if maint_ms > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": kernel_traffic(w.name), "peak_kind": peak_kind,
                "kernel": "maintain_kernel",
                "alg_bytes_per_launch": alg_bytes / max(1, maint_launches),
                "avg_launch_ms": maint_ms / max(1, maint_launches)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        rate, edges, t = cpu_oracle_rate(w, args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{edges} edge updates (whole rounds from round 0), {t:.1f} s, "
                         "oracle O3 sequential single-edge traversal, 1 thread"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic", "config": config_of(w, args),
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "cpu_baseline": cpu, "repeel": repeel,
                "detail": {"iterations_per_call_mean": float(np.mean(iters)),
                           "call_ms_median": {k: statistics.median(v) for k, v in per_call_ms.items()},
                           "call_ms_mean": {k: float(np.mean(v)) for k, v in per_call_ms.items()},
                           "iterations_mean": {k: float(np.mean(v)) for k, v in per_call_it.items()},
                           "maintain_ms_median": {k: statistics.median(v) for k, v in per_call_maint.items()},
                           "launches_per_call": {k: v / K for k, v in per_call_launch.items()},
                           "grid_iterations": per_call_grid_it, "barriers": per_call_bar,
                           "volumes": per_call_vol,
                           "phase_ms": {k: v / 1e6 for k, v in phase_ns.items()},
                           "maintain_ms_total": maint_ms, "units": units_all,
                           "round_ms": {"min": min(round_ms), "median": statistics.median(round_ms),
                                        "max": max(round_ms)}}}
        print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
