#!/usr/bin/env python3
"""Benchmark of the GB300 parallel-Louvain path.

One step = one whole run of the method (vertex following, colouring, every
phase's sweeps, modularity, coarse rebuilds) on one synthetic graph already
resident in HBM.  The default workload is the largest single-GPU one: a
Chung-Lu power-law graph of 2^24 vertices and about 2.5e8 edges (every
heuristic on).  ``value`` is edge visits per second of the whole run (the
arcs scanned by all sweep iterations divided by the run's device time);
``edge_visits_per_s_sweep`` divides the same arcs by the sweep time alone.

The default line also carries two sub-records measured in the same process:
``batched`` (4,096 planted-partition graphs of 100-50,000 vertices as one
batch, against the same graphs through 4,096 plain lv_run calls) and
``served`` (2,000 requests arriving as a Poisson stream at 200 per second,
served with continuous batching, against sequential plain solves; p50/p99).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload chunglu24]
  python bench.py --workload planted_batch4096   (the batch alone as the line)
  python bench.py --workload served_mix2000      (the request stream alone)
  python bench.py --impl reference ...   (the serial oracle on host cores)

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the method is single-GPU; replicas only) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge visits/s per sweep (whole run, bit-exact labels)"
UNIT = "edge visits/s"
BYTES_PER_ARC = 12     # col 4 + w 4 + C[col] 4
BYTES_PER_VERTEX = 28  # rowptr 8 + C 4 + k 4 + a,|C| of own community 8 + label write 4
SWEEP_SOURCES = ("lv_sweep.cu", "lv_ops.cuh", "lv_internal.cuh", "lv_engine.cuh")
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the dominant kernel, from ncu captures.  Each entry records the digest of
# the sweep kernel's sources at capture time; when the sources change the
# entry no longer applies and the line reports traffic as null.
MEASURED_TRAFFIC: dict = {
    # sweep_persistent_kernel on chunglu20 (2^20-vertex member of the Chung-Lu
    # family), phase-0 iteration 2: 354,682,368 + 39,672,832 B against
    # 369,528,704 algorithmic (12 x 29,082,750 arcs + 28 x 733,418 vertices);
    # applied to a phase-0 launch of the 2^24-vertex graph by that ratio
    "chunglu24": {"sources": "80dff76642570e5e", "ratio": 394_355_200 / 369_528_704,
                  "scope": "one phase-0 sweep launch, scaled by units from a capture of a "
                           "2^20-vertex Chung-Lu phase-0 launch (ratio 1.067)"},
    # the batched sweep on 512 planted graphs, phase-0 sweep 9 (262 graphs
    # iterating): 261,973,504 + 16,466,688 B against 227,837,952 algorithmic
    # (12 x 16,233,207 arcs + 28 x 1,179,981 vertices)
    "planted_batch4096": {"sources": "80dff76642570e5e",
                          "ratio": 278_440_192 / 227_837_952,
                          "scope": "one phase-0 sweep launch of all 4,096 graphs, scaled by "
                                   "units from a 512-graph capture (ratio 1.22)"},
}
# bounded oracle samples (host-core baseline): the oracle's whole pipeline
# on the same graph, cut after these many phases / iterations
CPU_SAMPLE = {"rmat20": dict(max_phases=1, max_iters=3),
              "planted1k": dict(),
              "rmat16": dict(),
              "chunglu20": dict(max_phases=1, max_iters=3)}
# workloads too large for a whole oracle iteration within the bench: the
# oracle's vertex following once, then its sweep of a block of this many
# phase-0 vertices (ids are shuffled, so a block is a random sample) as one
# class of an uncoloured first iteration; (bench baseline, reference step)
CPU_SWEEP_SAMPLE = {"chunglu24": (1 << 22, 1 << 20)}


def sweep_source_digest() -> str:
    """SHA-256 (first 16 hex digits) of the sweep kernel's source files."""
    import hashlib
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1410_1237_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_entry(workload: str):
    """The ncu traffic record of a workload if it was taken from the current
    sweep sources, else None."""
    e = MEASURED_TRAFFIC.get(workload)
    if e and e.get("sources") == sweep_source_digest():
        return e
    return None


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init_dist(world: int, dev):
    """One process per GPU (torchrun env); NCCL on GPUs, gloo on CPU.  Returns
    the torch.distributed module, or None for a single process."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if dev.type == "cuda":
        dist.init_process_group("nccl", device_id=dev)
    else:
        dist.init_process_group("gloo")
    return dist


def max_over_ranks(x: float, pg, dev) -> float:
    """The largest x over all ranks (the slowest replica sets the job time)."""
    if not pg:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(workload: str, g, prm) -> dict:
    """The oracle as it stands, single-threaded, on a bounded sample."""
    import oracle
    if workload in CPU_SWEEP_SAMPLE:
        count = CPU_SWEEP_SAMPLE[workload][0]
        t0 = time.perf_counter()
        (rp, cl, w), _ = oracle.vertex_following(g.rowptr, g.col, g.w)
        t_vf = time.perf_counter() - t0
        mv, vis, dt = oracle.sweep_sample(rp, cl, w, 0, count)
        return {"value": vis / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{workload}: the oracle's sweep of phase-0 vertices [0, {count}) "
                          f"(of {len(rp) - 1} after its vertex following, {t_vf:.1f} s, not "
                          f"timed) as one class of an uncoloured first iteration; {vis} edge "
                          f"visits, {mv} moves, {dt:.2f} s"}
    sample = dict(CPU_SAMPLE.get(workload, dict(max_phases=1, max_iters=2)))
    t0 = time.perf_counter()
    r = oracle.run(g.rowptr, g.col, g.w, **{**prm, **sample})
    dt = time.perf_counter() - t0
    visits = sum(r.phases[t[0]].arcs for t in r.iters)
    return {"value": visits / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{workload}: {sample_desc(sample)}; {len(r.iters)} iterations, "
                      f"{visits} edge visits, {dt:.2f} s"}


def sample_desc(sample: dict) -> str:
    if not sample:
        return "whole run"
    parts = ["vertex following"]
    if sample.get("coloring", 1):
        parts.append("colouring")
    parts += [f"{k}={v}" for k, v in sample.items() if k != "coloring"]
    if sample.get("coloring", 1) == 0:
        parts.append("phase 0 uncoloured")
    return " + ".join(parts)


def run_reference(args):
    """--impl reference: the serial oracle timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import graphgen
    g, prm = graphgen.workload(args.workload)
    import oracle
    times, visits = [], 0
    if args.workload in CPU_SWEEP_SAMPLE:
        count = CPU_SWEEP_SAMPLE[args.workload][1]
        (rp, cl, w), _ = oracle.vertex_following(g.rowptr, g.col, g.w)
        for step in range(args.warmup + args.steps):
            _, vis, dt = oracle.sweep_sample(rp, cl, w, 0, count)
            if step >= args.warmup:
                times.append(dt)
                visits = vis
        desc = (f"{args.workload}: per step, the oracle's sweep of phase-0 vertices [0, {count}) "
                f"(after its vertex following, done once) as one class of an uncoloured first "
                f"iteration; {visits} edge visits per step")
    else:
        sample = dict(CPU_SAMPLE.get(args.workload, dict(max_phases=1, max_iters=2)))
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            r = oracle.run(g.rowptr, g.col, g.w, **{**prm, **sample})
            dt = time.perf_counter() - t0
            if step >= args.warmup:
                times.append(dt)
                visits = sum(r.phases[t[0]].arcs for t in r.iters)
        desc = f"{args.workload}: {sample_desc(sample)} per step"
    tot = sum(times)
    value = visits * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": args.workload, "n": g.n, "arcs": g.arcs},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


BATCH_METRIC = "batched graphs/s (whole run of every graph, bit-exact labels)"
BATCH_UNIT = "graphs/s"
BATCH_PARAMS = dict(vertex_following=1, coloring=1, color_cutoff=100_000, theta_low=1e-6,
                    theta_high=1e-2)  # the library defaults; no graph reaches the cutoff


def batch_workload(name: str):
    import graphgen
    if name != "planted_batch4096":
        raise SystemExit(f"unknown batch workload {name}")
    return graphgen.planted_batch(num_graphs=4096, nmin=100, nmax=50_000, bmin=2, bmax=200,
                                  intra_deg=12, inter_deg=2, wmax=8, seed=4)


def oracle_graphs_per_s(b, budget_s: float = 15.0) -> tuple[float, str]:
    """The oracle as it stands on graphs of the batch, taken in a seeded random
    order until about budget_s seconds of CPU work."""
    import numpy as np

    import oracle
    order = np.random.default_rng(0).permutation(b.num_graphs)
    t_tot, done, verts = 0.0, 0, 0
    for g in order:
        gr = b.graph(int(g))
        t0 = time.perf_counter()
        oracle.run(gr.rowptr, gr.col, gr.w, **BATCH_PARAMS)
        t_tot += time.perf_counter() - t0
        done += 1
        verts += gr.n
        if t_tot >= budget_s:
            break
    return done / t_tot, (f"{done} of {b.num_graphs} graphs (seeded random order, "
                          f"{verts} vertices), whole run each, {t_tot:.2f} s")


def run_reference_batch(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    b = batch_workload(args.workload)
    vals = []
    desc = ""
    for step in range(args.warmup + args.steps):
        v, desc = oracle_graphs_per_s(b, budget_s=8.0)
        if step >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT,
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * b.num_graphs / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload, "graphs": b.num_graphs, "n": b.n,
                       "arcs": b.arcs},
            "cpu_baseline": {"value": value, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": BATCH_UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_batch(lv, torch, dev, pg, world, local, steps, warmup, plain=True, e2e=True,
                  cpu=True, workload="planted_batch4096") -> dict:
    """The 4,096-graph batch as one handle (one persistent sweep launch per
    batched iteration) against the same graphs run by 4,096 plain lv_run
    calls on resident handles.  Returns the measurements as a dict."""
    import numpy as np
    b = batch_workload(workload)
    stream = torch.cuda.Stream(dev)
    cs = stream.cuda_stream
    with torch.cuda.stream(stream):
        dt = [torch.from_numpy(x).to(dev) for x in (b.gptr, b.rowptr, b.col, b.w)]
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    h = lv.lv_batch_create(b.num_graphs, *dt, stream=cs)
    params = lv.make_params(**BATCH_PARAMS, autotune=1, collect_timing=1)
    for _ in range(warmup):  # the first run also measures the bins of each phase
        lv.lv_batch_run(h, params)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    step_ms, launches, sweep_ms, sweep_bytes, nsweeps = [], 0, 0.0, 0.0, 0
    sweep_arcs = 0
    st0_arcs = st0_n = 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lv.lv_batch_run(h, params)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = lv.lv_batch_get_stats(h)
        launches += st.kernel_launches
        sws = lv.lv_batch_get_sweeps(h)
        st0_arcs, st0_n = (sws[0].arcs, sws[0].vertices) if sws else (0, 0)
        for sw in sws:
            if sw.ms > 0:
                sweep_ms += sw.ms
                sweep_arcs += sw.arcs
                sweep_bytes += BYTES_PER_ARC * sw.arcs + BYTES_PER_VERTEX * sw.vertices
                nsweeps += 1
    torch.cuda.synchronize(dev)
    total_ms = max_over_ranks(sum(step_ms), pg, dev)
    clk = clocks.stop()
    st = lv.lv_batch_get_stats(h)
    batch_labels = np.empty(b.n, dtype=np.int32)
    lv.lv_batch_get_labels(h, -1, -1, batch_labels)
    qs = [lv.lv_batch_get_graph_info(h, g).q for g in range(b.num_graphs)]
    tuning = {r: t for r in range(st.num_phases)
              if (t := lv.lv_batch_get_tuning(h, r)) is not None}
    lv.lv_batch_destroy(h)
    value = whole_job_rate(b.num_graphs * steps, world, total_ms / 1e3)
    peak, peak_src = measured_peak_gbs()
    achieved = (sweep_bytes / (sweep_ms / 1e3) / 1e9) if sweep_ms > 0 else None

    # ---- the same graphs as 4,096 plain runs on resident handles (one pass)
    plain_rec = None
    if plain:
        handles = []
        for g in range(b.num_graphs):
            lo, hi = int(b.gptr[g]), int(b.gptr[g + 1])
            a0, a1 = int(b.rowptr[lo]), int(b.rowptr[hi])
            with torch.cuda.stream(stream):
                rp = dt[1][lo:hi + 1] - a0
                cl = dt[2][a0:a1] - lo
            torch.cuda.synchronize(dev)
            handles.append(lv.lv_graph_create(hi - lo, rp, cl, dt[3][a0:a1], stream=cs))
        p1 = lv.make_params(**BATCH_PARAMS)
        lv.lv_run(handles[0], p1)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
        e0.record(stream)
        for hh in handles:
            lv.lv_run(hh, p1)
        e1.record(stream)
        e1.synchronize()
        plain_ms = e0.elapsed_time(e1)
        same = True
        for g in range(b.num_graphs):  # identical labels, every graph
            one = np.empty(int(b.gptr[g + 1] - b.gptr[g]), dtype=np.int32)
            lv.lv_get_labels(handles[g], -1, one)
            same = same and bool(np.array_equal(one, batch_labels[b.gptr[g]:b.gptr[g + 1]]))
        for hh in handles:
            lv.lv_graph_destroy(hh)
        plain_rec = {"value": b.num_graphs / (plain_ms / 1e3), "unit": BATCH_UNIT,
                     "ms": plain_ms, "launch": "one lv_run per graph, handles resident",
                     "labels_identical_all": same}

    # ---- end to end from pinned host buffers through the batch API
    e2e_rec = None
    if e2e:
        hp = [torch.from_numpy(x).pin_memory() for x in (b.gptr, b.rowptr, b.col, b.w)]
        out = torch.empty(b.n, dtype=torch.int32).pin_memory()
        p2 = lv.make_params(**BATCH_PARAMS)
        times = []
        nwarm = 1
        for i in range(nwarm + steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hh = lv.lv_batch_create(b.num_graphs, *[x.numpy() for x in hp], stream=cs)
            lv.lv_batch_run(hh, p2)
            lv.lv_batch_get_labels(hh, -1, -1, out.numpy())
            lv.lv_batch_destroy(hh)
            t1 = time.perf_counter()
            if i >= nwarm:
                times.append(t1 - t0)
        tt = max_over_ranks(sum(times), pg, dev)
        e2e_rec = {"value": whole_job_rate(b.num_graphs * len(times), world, tt),
                   "unit": BATCH_UNIT,
                   "h2d_bytes_per_step": int(sum(x.nbytes for x in (b.gptr, b.rowptr, b.col,
                                                                     b.w))),
                   "d2h_bytes_per_step": int(4 * b.n), "s_per_step": tt / len(times)}
    del dt, flush
    torch.cuda.empty_cache()

    tr = traffic_entry(workload)
    alg0 = BYTES_PER_ARC * st0_arcs + BYTES_PER_VERTEX * st0_n
    rec = {
        "metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps,
        "config": {"workload": workload, "graphs": b.num_graphs, "n": b.n, "arcs": b.arcs,
                   "params": BATCH_PARAMS,
                   "l2": "input larger than L2 and a 256 MB L2 flush before every step",
                   "phases_max": st.num_phases, "batched_sweeps": st.sweep_launches,
                   "sweeps_from_cuda_graph": st.graph_launches,
                   "iterations_all_graphs": st.total_iterations,
                   "edge_visits_per_step": st.edge_visits,
                   "q_min": min(qs), "q_median": statistics.median(qs),
                   "autotuned_sweep_shape_by_round": tuning},
        "edge_visits_per_s_sweep": (sweep_arcs / (sweep_ms / 1e3)) if sweep_ms > 0 else None,
        "plain_launches": plain_rec,
        "speedup_vs_plain": (value / world / plain_rec["value"]) if plain_rec else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": (tr["ratio"] * alg0) if (tr and st0_arcs) else None,
                     "traffic_scope": tr["scope"] if tr else
                     "null: no ncu capture of the current sweep sources",
                     "algorithmic_bytes_phase0_launch": alg0,
                     "kernel": "batched sweep (persistent launch over all iterating graphs)",
                     "bytes_per_unit": f"{BYTES_PER_ARC} B/arc + {BYTES_PER_VERTEX} B/vertex "
                                       "of the swept graphs",
                     "peak_source": f"{peak_src} MEASURED_PEAKS.json hbm_gbs",
                     "sweeps_timed": nsweeps},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e_rec,
    }
    if cpu and world == 1:
        v, desc = oracle_graphs_per_s(b)
        rec["cpu_baseline"] = {"value": v, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle",
                               "sample": desc}
    return rec


def bench_batch(args, lv, torch, dev, pg, rank, world, local):
    """--workload planted_batch4096: the batch as the line."""
    rec = measure_batch(lv, torch, dev, pg, world, local, args.steps, args.warmup,
                        plain=not args.no_plain, e2e=not args.no_e2e,
                        cpu=not args.no_cpu_baseline, workload=args.workload)
    if rank != 0:
        return 0
    line = {"metric": rec.pop("metric"), "value": rec.pop("value"), "unit": rec.pop("unit"),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": rec.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded generator; same batch on every rank)"}
    rec.pop("steps"), rec.pop("warmup")
    rec["config"]["parallelism"] = f"replicas x{world}"
    line.update(rec)
    print(json.dumps(line), flush=True)
    return 0


SERVED_METRIC = "served graphs/s under Poisson arrivals (whole run per request, bit-exact labels)"
SERVED_PARAMS = dict(vertex_following=1, coloring=1, color_cutoff=100_000, theta_low=1e-6,
                     theta_high=1e-2)  # every heuristic on
SERVED_BUDGET = 120 << 30
SERVED_WORKLOADS = {"served_mix2000": 2000, "served_mix200": 200}


def served_workload(name: str):
    import graphgen
    if name not in SERVED_WORKLOADS:
        raise SystemExit(f"unknown served workload {name}")
    return graphgen.served_stream(num_requests=SERVED_WORKLOADS[name], rate=200.0, seed=5,
                                  workers=min(8, os.cpu_count() or 1))


def pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


def serve_once(lv, reqs):
    """One pass of the request stream through a server: requests are
    submitted at their arrival times by a separate thread; returns per-request
    (labels, info) and the server stats."""
    h = lv.lv_server_create(mem_budget_bytes=SERVED_BUDGET, **SERVED_PARAMS)
    ids = [None] * len(reqs)
    try:
        t0 = time.perf_counter()

        def submitter():
            for i, (a, g) in enumerate(reqs):
                dt = t0 + a - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                ids[i] = lv.lv_server_submit(h, g.rowptr, g.col, g.w)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        for rid in ids:
            lv.lv_server_wait(h, rid, -1.0)
        out = [lv.lv_server_result(h, rid) for rid in ids]
        st = lv.lv_server_get_stats(h)
    finally:
        lv.lv_server_destroy(h)
    return out, st


def oracle_served_sample(reqs, budget_s: float) -> tuple[float, str]:
    """The oracle on the smallest requests of the stream until about
    budget_s seconds of CPU work (whole run each)."""
    import oracle
    order = sorted(range(len(reqs)), key=lambda i: reqs[i][1].arcs)
    t_tot, done = 0.0, 0
    for i in order:
        g = reqs[i][1]
        t0 = time.perf_counter()
        oracle.run(g.rowptr, g.col, g.w, **SERVED_PARAMS)
        t_tot += time.perf_counter() - t0
        done += 1
        if t_tot >= budget_s:
            break
    return done / t_tot, (f"the {done} smallest of {len(reqs)} requests, whole run each, "
                          f"{t_tot:.2f} s")


def run_reference_served(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    reqs = served_workload(args.workload)
    vals, desc = [], ""
    for step in range(args.warmup + args.steps):
        v, desc = oracle_served_sample(reqs, 6.0)
        if step >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": SERVED_METRIC, "value": value, "unit": "graphs/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * len(reqs) / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload, "requests": len(reqs)},
            "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_served(lv, torch, dev, pg, world, local, steps, warmup, cpu=True,
                   workload="served_mix2000") -> dict:
    """The request stream (R-MAT scale 10-20 and planted graphs of 1e3-1e6
    vertices, Poisson arrivals at 200 req/s) served with continuous batching,
    against the same stream solved one request at a time by plain lv_run
    calls in arrival order.  Returns the measurements as a dict."""
    import numpy as np
    reqs = served_workload(workload)
    N = len(reqs)
    in_bytes = int(sum(g.rowptr.nbytes + g.col.nbytes + g.w.nbytes for _, g in reqs))
    out_bytes = int(sum(4 * g.n for _, g in reqs))
    serve_once(lv, reqs[:min(N, 24)])  # warm the library (pool, kernels)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    lat, spans, launches, rounds, sweeps, peak_g = [], [], 0, 0, 0, 0
    results, worker_ms = None, {}
    for step in range(warmup + steps):
        out, st = serve_once(lv, reqs)
        infos = [i for _, i in out]
        if any(i.status != 0 for i in infos):
            raise SystemExit("a served request failed")
        span = (max(i.t_done_ms for i in infos) - min(i.t_submit_ms for i in infos)) / 1e3
        if step >= warmup:
            spans.append(span)
            lat += [i.t_done_ms - i.t_submit_ms for i in infos]
            launches += st.kernel_launches
            rounds, sweeps, peak_g = st.rounds, st.sweeps, st.peak_graphs
            worker_ms = {"admit_thread": st.ms_admit, "append": st.ms_append,
                         "iterate": st.ms_iterate, "rebuild": st.ms_rebuild,
                         "results": st.ms_results}
            results = out
    clk = clocks.stop()
    total_s = max_over_ranks(sum(spans), pg, dev)
    value = whole_job_rate(N * len(spans), world, total_s)

    # ---- the same stream solved one request at a time (FIFO, plain lv_run)
    service = []
    same = True
    p1 = lv.make_params(**SERVED_PARAMS)
    for i, (a, g) in enumerate(reqs):
        t0 = time.perf_counter()
        hh = lv.lv_graph_create(g.n, g.rowptr, g.col, g.w)
        lv.lv_run(hh, p1)
        lab = np.empty(g.n, dtype=np.int32)
        lv.lv_get_labels(hh, -1, lab)
        lv.lv_graph_destroy(hh)
        service.append(time.perf_counter() - t0)
        same = same and bool(np.array_equal(lab, results[i][0]))
    finish, seq_lat = 0.0, []
    for (a, _), sv in zip(reqs, service):
        finish = max(finish, a) + sv
        seq_lat.append(1e3 * (finish - a))
    seq_span = finish - reqs[0][0]
    seq_value = N / seq_span
    rec = {
        "metric": SERVED_METRIC, "value": value, "unit": "graphs/s", "steps": steps,
        "warmup": warmup, "ms_per_step": 1e3 * sum(spans) / len(spans),
        "config": {"workload": workload, "requests": N, "rate_req_s": 200.0,
                   "params": SERVED_PARAMS, "mem_budget_bytes": SERVED_BUDGET,
                   "arcs_total": int(sum(g.arcs for _, g in reqs)),
                   "l2": "inputs larger than L2 (whole stream per step)",
                   "rounds": rounds, "batched_sweeps": sweeps, "peak_resident_requests": peak_g,
                   "worker_ms_last_step": worker_ms},
        "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
        "sequential_plain": {"value": seq_value, "unit": "graphs/s",
                             "latency_ms_p50": pct(seq_lat, 50),
                             "latency_ms_p99": pct(seq_lat, 99),
                             "service_s_total": sum(service),
                             "labels_identical_all": same},
        "speedup_vs_sequential": value / world / seq_value,
        "roofline": None,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes,
                "note": "the served value is end to end: host CSRs in, host labels out"},
    }
    if cpu and world == 1:
        v, desc = oracle_served_sample(reqs, 10.0)
        rec["cpu_baseline"] = {"value": v, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                               "sample": desc}
    return rec


def bench_served(args, lv, torch, dev, pg, rank, world, local):
    """--workload served_mix2000: the request stream as the line."""
    rec = measure_served(lv, torch, dev, pg, world, local, args.steps, args.warmup,
                         cpu=not args.no_cpu_baseline, workload=args.workload)
    if rank != 0:
        return 0
    line = {"metric": rec.pop("metric"), "value": rec.pop("value"), "unit": rec.pop("unit"),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": rec.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded Poisson request stream; same stream on every rank)"}
    rec.pop("steps"), rec.pop("warmup")
    rec["config"]["parallelism"] = f"replicas x{world}"
    line.update(rec)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="chunglu24")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="leave the batched sub-record out of a single-graph line")
    ap.add_argument("--no-served", action="store_true",
                    help="leave the served sub-record out of a single-graph line")
    ap.add_argument("--sub-steps", type=int, default=3,
                    help="timed steps of the batched sub-record (after 2 warm-up steps)")
    args = ap.parse_args()
    batch = args.workload.startswith("planted_batch")
    served = args.workload.startswith("served_")
    if args.impl == "reference":
        if served:
            return run_reference_served(args)
        return run_reference_batch(args) if batch else run_reference(args)

    import torch

    import graphgen
    from paper_1410_1237_gb300 import _build, lv

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print("bench.py needs a CUDA GPU", file=sys.stderr)
        return 2
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = init_dist(world, dev)
    if rank == 0 or world > 1:
        _build.build()
    if pg:
        pg.barrier()
    lv.load()
    if batch or served:
        fn = bench_batch if batch else bench_served
        rc = fn(args, lv, torch, dev, pg, rank, world, local)
        if pg:
            pg.destroy_process_group()
        return rc

    g, prm = graphgen.workload(args.workload)
    stream = torch.cuda.Stream(dev)
    cs = stream.cuda_stream
    with torch.cuda.stream(stream):
        d_rowptr = torch.from_numpy(g.rowptr).to(dev)
        d_col = torch.from_numpy(g.col).to(dev)
        d_w = torch.from_numpy(g.w).to(dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    torch.cuda.synchronize(dev)
    h = lv.lv_graph_create(g.n, d_rowptr, d_col, d_w, stream=cs)
    params = lv.make_params(**prm, collect_timing=1)

    # ---- device-resident steps
    for _ in range(args.warmup):
        lv.lv_run(h, params)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    step_ms, visits, launches, sweep_ms, sweep_bytes, sweeps = [], 0, 0, 0.0, 0.0, 0
    sweep_arcs = 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lv.lv_run(h, params)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = lv.lv_get_stats(h)
        visits = st.edge_visits
        launches += st.kernel_launches
        infos = [lv.lv_get_phase_info(h, p) for p in range(lv.lv_num_phases(h))]
        for it in lv.lv_get_iteration_stats(h):
            if it.ms > 0:
                ph = infos[it.phase]
                sweep_ms += it.ms
                sweep_arcs += it.arcs
                sweep_bytes += BYTES_PER_ARC * ph.arcs + BYTES_PER_VERTEX * ph.n
                sweeps += 1
    torch.cuda.synchronize(dev)
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, pg, dev)
    clk = clocks.stop()
    q = lv.lv_get_modularity(h, -1)[0]
    phases = lv.lv_num_phases(h)
    stats = lv.lv_get_stats(h)
    infos = [lv.lv_get_phase_info(h, p) for p in range(phases)]
    lv.lv_graph_destroy(h)
    del d_rowptr, d_col, d_w, flush
    torch.cuda.empty_cache()

    value = whole_job_rate(visits * args.steps, world, total_ms / 1e3)
    peak, peak_src = measured_peak_gbs()
    achieved = (sweep_bytes / (sweep_ms / 1e3) / 1e9) if sweep_ms > 0 else None

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(x).pin_memory() for x in (g.rowptr, g.col, g.w)]
        out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        p2 = lv.make_params(**prm)
        times = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hh = lv.lv_graph_create(g.n, hp[0].numpy(), hp[1].numpy(), hp[2].numpy(), stream=cs)
            lv.lv_run(hh, p2)
            lv.lv_get_labels(hh, -1, out.numpy())
            lv.lv_graph_destroy(hh)
            t1 = time.perf_counter()
            if i >= args.warmup:
                times.append(t1 - t0)
        tt = sum(times)
        tt = max_over_ranks(tt, pg, dev)
        e2e = {"value": whole_job_rate(visits * len(times), world, tt), "unit": UNIT,
               "h2d_bytes_per_step": int(g.rowptr.nbytes + g.col.nbytes + g.w.nbytes),
               "d2h_bytes_per_step": int(4 * g.n), "s_per_step": tt / len(times)}
        del hp, out

    tr = traffic_entry(args.workload)
    alg0 = BYTES_PER_ARC * infos[0].arcs + BYTES_PER_VERTEX * infos[0].n if infos else 0
    traffic = None
    if tr:
        traffic = tr["bytes"] if "bytes" in tr else tr["ratio"] * alg0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded generator; same graph on every rank)",
        "config": {"workload": args.workload, "n": g.n, "arcs": g.arcs, "two_m": g.two_m,
                   "params": prm, "parallelism": f"replicas x{world}",
                   "l2": "input larger than L2 and a 256 MB L2 flush before every step",
                   "s_to_final_q": total_ms / args.steps / 1e3, "final_q": q,
                   "phases": phases, "iterations": stats.total_iterations,
                   "edge_visits_per_step": visits,
                   "stage_ms_last_step": {"vf": stats.ms_vf, "color": stats.ms_color,
                                          "iterate": stats.ms_iterate,
                                          "rebuild": stats.ms_rebuild},
                   "phase_q": [i.q for i in infos]},
        "s_to_final_q": total_ms / args.steps / 1e3,
        "edge_visits_per_s_sweep": (sweep_arcs / (sweep_ms / 1e3)) if sweep_ms > 0 else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic,
                     "traffic_scope": tr["scope"] if tr else
                     "null: no ncu capture of the current sweep sources",
                     "algorithmic_bytes_phase0_launch": alg0,
                     "kernel": "sweep_persistent_kernel (one launch per iteration, all colour "
                               "classes)",
                     "bytes_per_unit": f"{BYTES_PER_ARC} B/arc + {BYTES_PER_VERTEX} B/vertex",
                     "peak_source": f"{peak_src} MEASURED_PEAKS.json hbm_gbs",
                     "sweeps_timed": sweeps},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1 and rank == 0:
        line["cpu_baseline"] = cpu_baseline(args.workload, g, prm)
    del g
    # sub-records of the batched and served forms (one GPU: replicas add nothing)
    if world == 1 and not args.no_batched:
        line["batched"] = measure_batch(lv, torch, dev, pg, world, local, args.sub_steps, 2,
                                        plain=not args.no_plain, e2e=False,
                                        cpu=not args.no_cpu_baseline)
    if world == 1 and not args.no_served:
        line["served"] = measure_served(lv, torch, dev, pg, world, local, 1, 0,
                                        cpu=not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
