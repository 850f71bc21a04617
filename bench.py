#!/usr/bin/env python3
"""Benchmark of the GB300 parallel-Louvain path.

One step = one whole run of the method (vertex following, colouring, every
phase's sweeps, modularity, coarse rebuilds) on one synthetic graph already
resident in HBM.  The metric is edge visits per second: the arcs scanned by
all sweep iterations of the run divided by the run's device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat20]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat20")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

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
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    if rank == 0 or world > 1:
        _build.build()
    if pg:
        pg.barrier()
    lv.load()

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
    if pg:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms = float(t.item())
    clk = clocks.stop()
    q = lv.lv_get_modularity(h, -1)[0]
    phases = lv.lv_num_phases(h)
    stats = lv.lv_get_stats(h)
    lv.lv_graph_destroy(h)

    value = world * visits * args.steps / (total_ms / 1e3)
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
        if pg:
            t = torch.tensor([tt], device=dev, dtype=torch.float64)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            tt = float(t.item())
        e2e = {"value": world * visits * len(times) / tt, "unit": UNIT,
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
