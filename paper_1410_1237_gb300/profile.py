"""Stage breakdown of a run: ``python -m paper_1410_1237_gb300.profile [workload] [reps]``.

``workload`` is a named single-graph workload, or ``planted_batch<G>`` for
the planted-partition batch recipe with G graphs (per-sweep records).

Generates a named synthetic workload (see graphgen.WORKLOADS), creates a handle
on device arrays, runs the method ``reps`` times with CUDA-event timing and
prints, for the last run, the per-phase colouring / iteration / rebuild times,
the Jones-Plassmann round count and every iteration's time and moves.  Used as
the driver for ncu captures (its kernels are the library's, launched through
the C ABI).
"""
from __future__ import annotations

import os
import sys
import time


def main(argv: list[str]) -> int:
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import graphgen
    from paper_1410_1237_gb300 import _build, lv

    wl = argv[0] if argv else "rmat20"
    reps = int(argv[1]) if len(argv) > 1 else 2
    _build.build()
    lv.load()
    if wl.startswith("planted_batch"):
        return batch_main(wl, reps, torch, graphgen, lv)
    g, prm = graphgen.workload(wl)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    arrays = [torch.from_numpy(x).to(dev) for x in (g.rowptr, g.col, g.w)]
    torch.cuda.synchronize(dev)
    h = lv.lv_graph_create(g.n, *arrays, stream=stream.cuda_stream)
    params = lv.make_params(**prm, collect_timing=1)
    wall = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        lv.lv_run(h, params)
        wall = time.perf_counter() - t0
    st = lv.lv_get_stats(h)
    print(wl, f"n={g.n} arcs={g.arcs} wall_ms={1e3 * wall:.2f}",
          {f: getattr(st, f) for f, _ in lv.lv_stats._fields_})
    for p in range(lv.lv_num_phases(h)):
        i = lv.lv_get_phase_info(h, p)
        print(f"phase {p} n={i.n} arcs={i.arcs} colours={i.num_colors} rounds={i.color_rounds} "
              f"iters={i.iterations} q={i.q:.6f} ms colour={i.ms_color:.2f} "
              f"iterate={i.ms_iterate:.2f} rebuild={i.ms_rebuild:.2f}")
    for it in lv.lv_get_iteration_stats(h):
        print(f"  iter phase={it.phase} it={it.iter} classes={it.color_steps} moved={it.moved} "
              f"ms={it.ms:.3f}")
    lv.lv_graph_destroy(h)
    return 0


def batch_main(wl: str, reps: int, torch, graphgen, lv) -> int:
    """planted_batch<G>: the planted-partition batch recipe with G graphs."""
    num = int(wl[len("planted_batch"):] or 4096)
    b = graphgen.planted_batch(num_graphs=num)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    arrays = [torch.from_numpy(x).to(dev) for x in (b.gptr, b.rowptr, b.col, b.w)]
    torch.cuda.synchronize(dev)
    h = lv.lv_batch_create(b.num_graphs, *arrays, stream=stream.cuda_stream)
    params = lv.make_params(autotune=1, collect_timing=1)
    wall = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        lv.lv_batch_run(h, params)
        wall = time.perf_counter() - t0
    st = lv.lv_batch_get_stats(h)
    print(wl, f"graphs={b.num_graphs} n={b.n} arcs={b.arcs} wall_ms={1e3 * wall:.2f}",
          {f: getattr(st, f) for f, _ in lv.lv_stats._fields_})
    for sw in lv.lv_batch_get_sweeps(h):
        print(f"  sweep phase={sw.phase} sweep={sw.sweep} graphs={sw.graphs} n={sw.vertices} "
              f"arcs={sw.arcs} moved={sw.moved} ms={sw.ms:.3f}")
    lv.lv_batch_destroy(h)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
