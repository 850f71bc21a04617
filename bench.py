#!/usr/bin/env python3
"""Benchmark of the GB300 parallel-Louvain path.

One step = one whole run of the method (vertex following, colouring, every
phase's sweeps, modularity, coarse rebuilds) on one synthetic graph already
resident in HBM.  The metric is edge visits per second: the arcs scanned by
all sweep iterations of the run divided by the run's device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat20]
  python bench.py --workload planted_batch4096   (4,096 graphs per step: graphs/s,
                                                  against 4,096 plain runs)
  python bench.py --workload served_mix200       (Poisson request stream through the
                                                  server: graphs/s, p50/p99 latency,
                                                  against sequential plain solves)
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
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the dominant kernel, from ncu captures of the current kernels; None where
# no capture applies
MEASURED_TRAFFIC = {
    # sweep_persistent_kernel, rmat20 phase 0 iteration 3 (all 232 classes)
    "rmat20": {"bytes": 335_230_976 + 17_168_128,
               "scope": "one phase-0 sweep launch (iteration 3, 232 colour classes)"},
    # batched sweep: traffic / algorithmic bytes of a 512-graph capture
    # (1,290.2 MB / 914.1 MB), applied to a phase-0 launch of the full batch
    "planted_batch4096": {"ratio": 1290.2 / 914.1,
                          "scope": "one phase-0 sweep launch of all 4,096 graphs, scaled by "
                                   "units from a 512-graph capture"},
}
# bounded oracle samples (host-core baseline): the oracle's whole pipeline
# on the same graph, cut after these many phases / iterations
CPU_SAMPLE = {"rmat20": dict(max_phases=1, max_iters=3),
              "chunglu24": dict(max_phases=1, max_iters=1),
              "planted1k": dict(),
              "rmat16": dict(),
              "chunglu20": dict(max_phases=1, max_iters=3)}


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
    sample = dict(CPU_SAMPLE.get(workload, dict(max_phases=1, max_iters=2)))
    t0 = time.perf_counter()
    r = oracle.run(g.rowptr, g.col, g.w, **prm, **sample)
    dt = time.perf_counter() - t0
    visits = sum(r.phases[t[0]].arcs for t in r.iters)
    desc = "whole run" if not sample else \
        "vertex following + colouring + " + ", ".join(f"{k}={v}" for k, v in sample.items())
    return {"value": visits / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{workload}: {desc}; {len(r.iters)} iterations, {visits} edge visits, "
                      f"{dt:.2f} s"}


def run_reference(args):
    """--impl reference: the serial oracle timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import graphgen
    g, prm = graphgen.workload(args.workload)
    import oracle
    sample = dict(CPU_SAMPLE.get(args.workload, dict(max_phases=1, max_iters=2)))
    times, visits = [], 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.run(g.rowptr, g.col, g.w, **prm, **sample)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            visits = sum(r.phases[t[0]].arcs for t in r.iters)
    tot = sum(times)
    value = visits * len(times) / tot
    desc = "whole run" if not sample else ", ".join(f"{k}={v}" for k, v in sample.items())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": args.workload, "n": g.n, "arcs": g.arcs},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.workload}: {desc}"},
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


def bench_batch(args, lv, torch, dev, pg, rank, world, local):
    """planted_batch4096: the 4,096-graph batch as one handle (one persistent
    sweep launch per batched iteration) against the same graphs run by 4,096
    plain lv_run calls on resident handles."""
    import numpy as np
    b = batch_workload(args.workload)
    stream = torch.cuda.Stream(dev)
    cs = stream.cuda_stream
    with torch.cuda.stream(stream):
        dt = [torch.from_numpy(x).to(dev) for x in (b.gptr, b.rowptr, b.col, b.w)]
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    h = lv.lv_batch_create(b.num_graphs, *dt, stream=cs)
    params = lv.make_params(**BATCH_PARAMS, autotune=1, collect_timing=1)
    for _ in range(args.warmup):  # the first run also measures the bins of each phase
        lv.lv_batch_run(h, params)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    step_ms, launches, sweep_ms, sweep_bytes, nsweeps = [], 0, 0.0, 0.0, 0
    st0_arcs = st0_n = 0
    for _ in range(args.steps):
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
                sweep_bytes += BYTES_PER_ARC * sw.arcs + BYTES_PER_VERTEX * sw.vertices
                nsweeps += 1
    torch.cuda.synchronize(dev)
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, pg, dev)
    clk = clocks.stop()
    st = lv.lv_batch_get_stats(h)
    batch_labels = np.empty(b.n, dtype=np.int32)
    lv.lv_batch_get_labels(h, -1, -1, batch_labels)
    qs = [lv.lv_batch_get_graph_info(h, g).q for g in range(b.num_graphs)]
    lv.lv_batch_destroy(h)
    value = whole_job_rate(b.num_graphs * args.steps, world, total_ms / 1e3)
    peak, peak_src = measured_peak_gbs()
    achieved = (sweep_bytes / (sweep_ms / 1e3) / 1e9) if sweep_ms > 0 else None

    # ---- the same graphs as 4,096 plain runs on resident handles (one pass)
    plain = None
    if not args.no_plain:
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
        for g in range(0, b.num_graphs, 41):  # identical labels, sampled
            one = np.empty(int(b.gptr[g + 1] - b.gptr[g]), dtype=np.int32)
            lv.lv_get_labels(handles[g], -1, one)
            same = same and bool(np.array_equal(one, batch_labels[b.gptr[g]:b.gptr[g + 1]]))
        for hh in handles:
            lv.lv_graph_destroy(hh)
        plain = {"value": b.num_graphs / (plain_ms / 1e3), "unit": BATCH_UNIT,
                 "ms": plain_ms, "launch": "one lv_run per graph, handles resident",
                 "labels_identical_sampled": same}

    # ---- end to end from pinned host buffers through the batch API
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(x).pin_memory() for x in (b.gptr, b.rowptr, b.col, b.w)]
        out = torch.empty(b.n, dtype=torch.int32).pin_memory()
        p2 = lv.make_params(**BATCH_PARAMS)
        times = []
        for i in range(max(1, args.warmup // 2) + args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hh = lv.lv_batch_create(b.num_graphs, *[x.numpy() for x in hp], stream=cs)
            lv.lv_batch_run(hh, p2)
            lv.lv_batch_get_labels(hh, -1, -1, out.numpy())
            lv.lv_batch_destroy(hh)
            t1 = time.perf_counter()
            if i >= max(1, args.warmup // 2):
                times.append(t1 - t0)
        tt = sum(times)
        tt = max_over_ranks(tt, pg, dev)
        e2e = {"value": whole_job_rate(b.num_graphs * len(times), world, tt), "unit": BATCH_UNIT,
               "h2d_bytes_per_step": int(sum(x.nbytes for x in (b.gptr, b.rowptr, b.col, b.w))),
               "d2h_bytes_per_step": int(4 * b.n), "s_per_step": tt / len(times)}

    if rank != 0:
        return 0
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded generator; same batch on every rank)",
        "config": {"workload": args.workload, "graphs": b.num_graphs, "n": b.n, "arcs": b.arcs,
                   "params": BATCH_PARAMS, "parallelism": f"replicas x{world}",
                   "l2": "input larger than L2 and a 256 MB L2 flush before every step",
                   "phases_max": st.num_phases, "batched_sweeps": st.sweep_launches,
                   "sweeps_from_cuda_graph": st.graph_launches,
                   "iterations_all_graphs": st.total_iterations,
                   "edge_visits_per_step": st.edge_visits,
                   "q_min": min(qs), "q_median": statistics.median(qs)},
        "plain_launches": plain,
        "speedup_vs_plain": (value / world / plain["value"]) if plain else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": (MEASURED_TRAFFIC[args.workload]["ratio"] *
                                 (BYTES_PER_ARC * st0_arcs + BYTES_PER_VERTEX * st0_n))
                     if st0_arcs else None,
                     "traffic_scope": MEASURED_TRAFFIC[args.workload]["scope"],
                     "algorithmic_bytes_phase0_launch": BYTES_PER_ARC * st0_arcs +
                     BYTES_PER_VERTEX * st0_n,
                     "kernel": "batched sweep (persistent launch over all iterating graphs)",
                     "bytes_per_unit": f"{BYTES_PER_ARC} B/arc + {BYTES_PER_VERTEX} B/vertex "
                                       "of the swept graphs",
                     "peak_source": f"{peak_src} MEASURED_PEAKS.json hbm_gbs",
                     "sweeps_timed": nsweeps},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1:
        v, desc = oracle_graphs_per_s(b)
        line["cpu_baseline"] = {"value": v, "unit": BATCH_UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line), flush=True)
    return 0


SERVED_METRIC = "served graphs/s under Poisson arrivals (whole run per request, bit-exact labels)"
SERVED_PARAMS = dict(vertex_following=1, coloring=1, color_cutoff=100_000, theta_low=1e-6,
                     theta_high=1e-2)  # every heuristic on
SERVED_BUDGET = 120 << 30


def served_workload(name: str):
    import graphgen
    if name != "served_mix200":
        raise SystemExit(f"unknown served workload {name}")
    return graphgen.served_stream(num_requests=200, rate=200.0, seed=5)


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


def run_reference_served(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    reqs = served_workload(args.workload)
    order = sorted(range(len(reqs)), key=lambda i: reqs[i][1].arcs)  # smallest first: bounded
    vals, desc = [], ""
    for step in range(args.warmup + args.steps):
        t_tot, done = 0.0, 0
        for i in order:
            g = reqs[i][1]
            t0 = time.perf_counter()
            oracle.run(g.rowptr, g.col, g.w, **SERVED_PARAMS)
            t_tot += time.perf_counter() - t0
            done += 1
            if t_tot >= 6.0:
                break
        desc = f"the {done} smallest of {len(reqs)} requests, whole run each, {t_tot:.2f} s"
        if step >= args.warmup:
            vals.append(done / t_tot)
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


def bench_served(args, lv, torch, dev, pg, rank, world, local):
    """served_mix200: 200 requests (R-MAT scale 10-20 and planted graphs of
    1e3-1e6 vertices) arriving as a Poisson stream at 200 req/s, served with
    continuous batching, against the same stream solved one request at a time
    by plain lv_run calls in arrival order."""
    import numpy as np
    reqs = served_workload(args.workload)
    N = len(reqs)
    in_bytes = int(sum(g.rowptr.nbytes + g.col.nbytes + g.w.nbytes for _, g in reqs))
    out_bytes = int(sum(4 * g.n for _, g in reqs))
    serve_once(lv, reqs[:min(N, 24)])  # warm the library (pool, kernels)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    lat, spans, launches, rounds, sweeps, peak_g = [], [], 0, 0, 0, 0
    results = None
    for step in range(args.warmup + args.steps):
        out, st = serve_once(lv, reqs)
        infos = [i for _, i in out]
        if any(i.status != 0 for i in infos):
            raise SystemExit("a served request failed")
        span = (max(i.t_done_ms for i in infos) - min(i.t_submit_ms for i in infos)) / 1e3
        if step >= args.warmup:
            spans.append(span)
            lat += [i.t_done_ms - i.t_submit_ms for i in infos]
            launches += st.kernel_launches
            rounds, sweeps, peak_g = st.rounds, st.sweeps, st.peak_graphs
            worker_ms = {"admit_thread": st.ms_admit, "append": st.ms_append,
                         "iterate": st.ms_iterate, "rebuild": st.ms_rebuild,
                         "results": st.ms_results}
            results = out
    clk = clocks.stop()
    total_s = max_over_ranks(sum(spans), pg, dev if dev.type == "cuda" else dev)
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
    if rank != 0:
        return 0
    line = {
        "metric": SERVED_METRIC, "value": value, "unit": "graphs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(spans) / len(spans),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded Poisson request stream; same stream on every rank)",
        "config": {"workload": args.workload, "requests": N, "rate_req_s": 200.0,
                   "params": SERVED_PARAMS, "mem_budget_bytes": SERVED_BUDGET,
                   "parallelism": f"replicas x{world}", "arcs_total": int(sum(g.arcs for _, g in reqs)),
                   "l2": "inputs larger than L2 (whole stream per step)",
                   "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
                   "rounds": rounds, "batched_sweeps": sweeps, "peak_resident_requests": peak_g,
                   "worker_ms_last_step": worker_ms},
        "sequential_plain": {"value": N / seq_span, "unit": "graphs/s",
                             "latency_ms_p50": pct(seq_lat, 50), "latency_ms_p99": pct(seq_lat, 99),
                             "service_s_total": sum(service),
                             "labels_identical_all": same},
        "speedup_vs_sequential": value / world / (N / seq_span),
        "roofline": None,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes,
                "note": "the served value is end to end: host CSRs in, host labels out"},
    }
    if not args.no_cpu_baseline and world == 1:
        import oracle
        order = sorted(range(N), key=lambda i: reqs[i][1].arcs)
        t_tot, done = 0.0, 0
        for i in order:
            g = reqs[i][1]
            t0 = time.perf_counter()
            oracle.run(g.rowptr, g.col, g.w, **SERVED_PARAMS)
            t_tot += time.perf_counter() - t0
            done += 1
            if t_tot >= 10.0:
                break
        line["cpu_baseline"] = {"value": done / t_tot, "unit": "graphs/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"the {done} smallest of {N} requests, whole run each, "
                                          f"{t_tot:.2f} s"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat20")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args()
    batch = args.workload.startswith("planted_batch")
    served = args.workload.startswith("served_")
    if args.impl == "reference":
        if served:
            return run_reference_served(args)
        return run_reference_batch(args) if batch else run_reference(args)

    import numpy as np
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
                sweep_bytes += BYTES_PER_ARC * ph.arcs + BYTES_PER_VERTEX * ph.n
                sweeps += 1
    torch.cuda.synchronize(dev)
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, pg, dev)
    clk = clocks.stop()
    q = lv.lv_get_modularity(h, -1)[0]
    phases = lv.lv_num_phases(h)
    stats = lv.lv_get_stats(h)
    lv.lv_graph_destroy(h)

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

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0
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
                   "edge_visits_per_step": visits},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": MEASURED_TRAFFIC.get(args.workload, {}).get("bytes"),
                     "traffic_scope": MEASURED_TRAFFIC.get(args.workload, {}).get("scope"),
                     "kernel": "sweep_persistent_kernel (one launch per iteration, all colour "
                               "classes)",
                     "bytes_per_unit": f"{BYTES_PER_ARC} B/arc + {BYTES_PER_VERTEX} B/vertex",
                     "peak_source": f"{peak_src} MEASURED_PEAKS.json hbm_gbs",
                     "sweeps_timed": sweeps},
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, g, prm)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
