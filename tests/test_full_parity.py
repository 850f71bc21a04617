"""Full-size parity: the CUDA path at the workload sizes the bench measures,
against whole-run records of the serial oracle.

The records under tests/golden/ are written by make_full_runs.py beside them,
which calls only the seeded generators and the oracle.  Each record starts
with a digest of the generated input, so a generator change fails here
instead of comparing against stale records.  Compared, exactly:

* chunglu24 (2^24 vertices, 488.7 M arcs, every heuristic on): per phase the
  vertices, arcs, communities, colouring, iteration count, exact numerators
  N_start / N_end and a digest of the labels of every original vertex; per
  iteration the moves and the exact numerator.
* planted_batch4096: every one of the 4,096 graphs of one batched run: its
  phase and iteration counts, final numerator and a digest of its labels.
* served_mix2000: every one of the 2,000 requests of the Poisson stream,
  submitted at their arrival times to one server: the same per-request
  record.
"""
import hashlib
import os
import threading
import time

import numpy as np
import pytest

import graphgen as gg
from conftest import GOLDEN

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

PARAMS = dict(vertex_following=1, coloring=1, color_cutoff=100_000, theta_low=1e-6,
              theta_high=1e-2)


@pytest.fixture(scope="module")
def lv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1237_gb300 import _build, lv as lvmod
    _build.build()
    lvmod.load()
    return lvmod


def digest(*arrays) -> str:
    """First 16 hex digits of SHA-256 over the arrays' little-endian bytes
    (the digest make_full_runs.py writes)."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()[:16]


def records(name: str) -> list:
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def per_graph(recs, key: str) -> dict:
    """{index: (n, arcs, phases, iterations, N_final, labels digest)}"""
    out = {}
    for r in recs:
        if r[0] != key:
            continue
        vals = r[2:] if key == "g" else r[4:]
        out[int(r[1])] = (int(vals[0]), int(vals[1]), int(vals[2]), int(vals[3]), int(vals[4]),
                          vals[5])
    return out


def test_chunglu24_full_run(lv):
    recs = records("chunglu24_run.txt")
    g, prm = gg.workload("chunglu24")
    head = next(r for r in recs if r[0] == "graph")
    assert (g.n, g.arcs, digest(g.rowptr, g.col, g.w)) == (int(head[1]), int(head[2]), head[3])
    assert prm == PARAMS
    res = lv.run(g.rowptr, g.col, g.w, **prm)
    vf_n = int(next(r for r in recs if r[0] == "vf_n")[1])
    assert res.stats["vf_n"] == vf_n
    assert res.two_m == int(next(r for r in recs if r[0] == "two_m")[1])
    want = [r for r in recs if r[0] == "phase"]
    assert len(res.phases) == len(want)
    for p, r in zip(res.phases, want):
        got = (p.n, p.arcs, p.n_next, int(p.colored), p.num_colors, p.iterations, p.N_start,
               p.N_end, digest(p.labels))
        assert got == (int(r[2]), int(r[3]), int(r[4]), int(r[5]), int(r[6]), int(r[7]),
                       int(r[8]), int(r[9]), r[10]), f"phase {r[1]}"
    got_it = [(t[0], t[1], t[3], t[4]) for t in res.iters]
    want_it = [tuple(int(x) for x in r[1:5]) for r in recs if r[0] == "iter"]
    assert got_it == want_it
    # the last phase may end below the previous one's modularity (signed stop
    # test after the moves of Alg. 1); the records hold whichever the oracle got
    assert res.phases[-1].N_end == int(want[-1][9])


def test_planted_batch4096_every_graph(lv):
    torch = pytest.importorskip("torch")
    recs = records("planted_batch4096_runs.txt")
    b = gg.planted_batch(num_graphs=4096, nmin=100, nmax=50_000, bmin=2, bmax=200,
                         intra_deg=12, inter_deg=2, wmax=8, seed=4)
    head = next(r for r in recs if r[0] == "batch")
    assert (b.num_graphs, b.n, b.arcs) == (int(head[1]), int(head[2]), int(head[3]))
    assert digest(b.gptr, b.rowptr, b.col, b.w) == head[4]
    want = per_graph(recs, "g")
    dev = torch.device("cuda:0")
    d = [torch.from_numpy(x).to(dev) for x in (b.gptr, b.rowptr, b.col, b.w)]
    torch.cuda.synchronize()
    h = lv.lv_batch_create(b.num_graphs, *d)
    try:
        lv.lv_batch_run(h, lv.make_params(**PARAMS))
        labels = np.empty(b.n, dtype=np.int32)
        lv.lv_batch_get_labels(h, -1, -1, labels)
        bad = []
        for gi in range(b.num_graphs):
            info = lv.lv_batch_get_graph_info(h, gi)
            lab = labels[b.gptr[gi]:b.gptr[gi + 1]]
            got = (info.n, info.arcs, info.num_phases, info.iterations, info.N_final,
                   digest(lab))
            if got != want[gi]:
                bad.append((gi, got, want[gi]))
        assert not bad, bad[:5]
    finally:
        lv.lv_batch_destroy(h)


def test_served_mix2000_every_request(lv):
    recs = records("served_mix2000_runs.txt")
    want = per_graph(recs, "r")
    arrivals = {int(r[1]): float(r[2]) for r in recs if r[0] == "r"}
    reqs = gg.served_stream(num_requests=2000, rate=200.0, seed=5,
                            workers=min(8, os.cpu_count() or 1))
    assert len(reqs) == len(want) == 2000
    h = lv.lv_server_create(mem_budget_bytes=120 << 30, **PARAMS)
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
        bad = []
        for i, ((a, g), rid) in enumerate(zip(reqs, ids)):
            assert abs(a - arrivals[i]) < 1e-6
            assert lv.lv_server_wait(h, rid, 600.0)
            lab, info = lv.lv_server_result(h, rid)
            got = (info.n, info.arcs, info.num_phases, info.iterations, info.N_final,
                   digest(lab))
            if info.status != 0 or got != want[i]:
                bad.append((i, info.status, got, want[i]))
            lv.lv_server_release(h, rid)
        assert not bad, bad[:5]
        st = lv.lv_server_get_stats(h)
        assert st.completed == len(reqs) and st.failed == 0
    finally:
        lv.lv_server_destroy(h)
