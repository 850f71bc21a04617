#!/usr/bin/env python3
"""Benchmark of the GB300 parallel-Louvain path.

One step = one whole run of the method (vertex following, colouring, every
phase's sweeps, modularity, coarse rebuilds) on one synthetic graph already
resident in HBM.  The metric is edge visits per second: the arcs scanned by
all sweep iterations of the run divided by the run's device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat20]
  python bench.py --workload planted_batch4096   (4,096 graphs per step: graphs/s,
                                                  against 4,096 plain runs)
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
        for sw in lv.lv_batch_get_sweeps(h):
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
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
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
    if args.impl == "reference":
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
    if batch:
        rc = bench_batch(args, lv, torch, dev, pg, rank, world, local)
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
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "kernel": "sweep iteration (all class launches of one iteration)",
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
