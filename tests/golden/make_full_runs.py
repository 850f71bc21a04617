"""Writes the whole-run oracle records that the full-size parity tests compare
the CUDA path with.  It calls only the seeded generators (graphgen) and the
serial oracle, never the CUDA library:

  python tests/golden/make_full_runs.py [chunglu24] [batch] [served] [--procs P]

* chunglu24_run.txt -- the Chung-Lu graph of 2^24 vertices (every heuristic
  on): a digest of the generated CSR, then per phase the oracle's record
  (vertices, arcs, communities, colouring, iterations, exact numerators) and
  a digest of the labels of the original vertices, then per iteration the
  moves.
* planted_batch4096_runs.txt -- each of the 4,096 planted-partition graphs of
  the batch workload run alone (library defaults): phases, iterations, final
  numerator and a digest of its final labels.
* served_mix2000_runs.txt -- each of the 2,000 requests of the Poisson
  request stream run alone (every heuristic on), as for the batch.

A label digest is the first 16 hex digits of SHA-256 over the int32
little-endian label array; a graph digest the same over rowptr (int64), col
and w (int32) in that order.  Graphs are run in worker processes (each run
serial); the records do not depend on the process count.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# every heuristic on (the library defaults of Sec. 5.1)
PARAMS = dict(vertex_following=1, coloring=1, color_cutoff=100_000, theta_low=1e-6,
              theta_high=1e-2)


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()[:16]


def run_record(g) -> str:
    """'n arcs phases iterations N_final labels_digest' of one whole run."""
    import oracle
    r = oracle.run(g.rowptr, g.col, g.w, **PARAMS)
    return (f"{g.n} {g.arcs} {len(r.phases)} {sum(p.iterations for p in r.phases)} "
            f"{r.phases[-1].N_end} {digest(r.phases[-1].labels)}")


def _batch_one(gi: int) -> tuple[int, str]:
    import graphgen
    g = _BATCH.graph(gi)
    return gi, run_record(g)


def _served_one(i: int) -> tuple[int, str]:
    import graphgen
    g = graphgen.served_request(_SPECS[i])
    return i, f"{_SPECS[i][0]:.9f} {_SPECS[i][1]} " + run_record(g)


_BATCH = None
_SPECS = None


def _one_thread():
    # each worker process generates with one thread: the processes already
    # fill the cores (the generated graphs do not depend on the thread count)
    import graphgen
    graphgen._load().gg_set_threads(1)


def _init_batch():
    global _BATCH
    import graphgen
    _one_thread()
    _BATCH = graphgen.planted_batch(num_graphs=4096, nmin=100, nmax=50_000, bmin=2, bmax=200,
                                    intra_deg=12, inter_deg=2, wmax=8, seed=4)


def _init_served():
    global _SPECS
    import graphgen
    _one_thread()
    _SPECS = graphgen.served_specs(num_requests=2000, rate=200.0, seed=5)


def write_chunglu24():
    import graphgen
    import oracle
    g, prm = graphgen.workload("chunglu24")
    t0 = time.time()
    r = oracle.run(g.rowptr, g.col, g.w, **prm)
    lines = ["# chunglu24: Chung-Lu, 2^24 vertices, gamma 2.1, 30% pendant, 2.5e8 edge draws,",
             "# seed 3; every heuristic on (VF, colouring, theta 1e-2 -> 1e-6).",
             "# Written by tests/golden/make_full_runs.py from the serial oracle",
             f"# ({time.time() - t0:.0f} s of one core).",
             f"graph {g.n} {g.arcs} {digest(g.rowptr, g.col, g.w)}",
             f"vf_n {r.vf_n}",
             f"two_m {r.two_m}",
             "# phase n arcs n_next colored num_colors iterations N_start N_end labels"]
    for i, p in enumerate(r.phases):
        lines.append(f"phase {i} {p.n} {p.arcs} {p.n_next} {int(p.colored)} {p.num_colors} "
                     f"{p.iterations} {p.N_start} {p.N_end} {digest(p.labels)}")
    lines.append("# iter phase iteration moved N")
    for ph, it, mv, N, _ in r.iters:
        lines.append(f"iter {ph} {it} {mv} {N}")
    with open(os.path.join(HERE, "chunglu24_run.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def write_batch(procs: int):
    global _BATCH
    import graphgen
    _BATCH = graphgen.planted_batch(num_graphs=4096, nmin=100, nmax=50_000, bmin=2, bmax=200,
                                    intra_deg=12, inter_deg=2, wmax=8, seed=4)
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(procs, initializer=_init_batch) as pool:
        recs = dict(pool.imap_unordered(_batch_one, range(_BATCH.num_graphs), chunksize=4))
    lines = ["# planted_batch4096: 4,096 planted-partition graphs (n log-uniform in",
             "# [100, 50,000], 2-200 blocks, intra degree 12, inter 2, weights 1-8, graph g",
             "# seeded (4 << 20) + g), each run alone by the serial oracle with the library",
             f"# defaults.  Written by tests/golden/make_full_runs.py ({time.time() - t0:.0f} s).",
             f"batch {_BATCH.num_graphs} {_BATCH.n} {_BATCH.arcs} "
             f"{digest(_BATCH.gptr, _BATCH.rowptr, _BATCH.col, _BATCH.w)}",
             "# graph n arcs phases iterations N_final labels"]
    lines += [f"g {gi} {recs[gi]}" for gi in range(_BATCH.num_graphs)]
    with open(os.path.join(HERE, "planted_batch4096_runs.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def write_served(procs: int):
    _init_served()
    ctx = mp.get_context("spawn")
    t0 = time.time()
    # largest first so the long runs do not come last
    order = sorted(range(len(_SPECS)),
                   key=lambda i: -(_SPECS[i][2][1] << _SPECS[i][2][0] if _SPECS[i][1] == "rmat"
                                   else 14 * _SPECS[i][2][0]))
    with ctx.Pool(procs, initializer=_init_served) as pool:
        recs = dict(pool.imap_unordered(_served_one, order, chunksize=1))
    lines = ["# served_mix2000: 2,000 requests, Poisson arrivals at 200/s (seed 5); each",
             "# request R-MAT (scale 10-20, edge factor 8-16) or planted partition",
             "# (1e3-1e6 vertices), request i seeded (5 << 20) + i, each run alone by the",
             "# serial oracle with every heuristic on.  Written by",
             f"# tests/golden/make_full_runs.py ({time.time() - t0:.0f} s).",
             "# request arrival_s kind n arcs phases iterations N_final labels"]
    lines += [f"r {i} {recs[i]}" for i in range(len(_SPECS))]
    with open(os.path.join(HERE, "served_mix2000_runs.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def main(argv):
    procs = max(1, (os.cpu_count() or 2) - 1)
    if "--procs" in argv:
        procs = int(argv[argv.index("--procs") + 1])
    which = [a for a in argv if a in ("chunglu24", "batch", "served")] or \
        ["chunglu24", "batch", "served"]
    if "batch" in which:
        write_batch(procs)
    if "served" in which:
        write_served(procs)
    if "chunglu24" in which:
        write_chunglu24()


if __name__ == "__main__":
    main(sys.argv[1:])
