"""Serving with continuous batching vs each request run alone.

Requests of different sizes and shapes are submitted from several threads
while others are on the GPU; every result (labels, exact modularity
numerator, phase and iteration counts) must equal lv_run on that graph alone
with the same parameters, and the oracle on a sample.  Admission limits
(memory budget, slots) change only the scheduling, never a result; an
invalid request fails alone.
"""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

PARAMS = dict(vertex_following=1, coloring=0)


@pytest.fixture(scope="module")
def lv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1237_gb300 import _build, lv as lvmod
    _build.build()
    lvmod.load()
    return lvmod


def request_mix(seed=0, count=24):
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            graphs.append(gg.planted(int(rng.integers(200, 20_000)), int(rng.integers(2, 40)), 0.05,
                                     0.001, 1, 8, seed=1000 + i))
        elif kind == 1:
            graphs.append(gg.rmat(int(rng.integers(8, 15)), int(rng.integers(8, 17)), seed=2000 + i))
        elif kind == 2:
            graphs.append(gg.random_graph(int(rng.integers(20, 300)), 0.05, wmax=5, loops=0.1,
                                          seed=3000 + i))
        else:
            graphs.append(gg.from_edges(3, [(0, 1, 2), (1, 2, 1)]))  # a path: vertex following
    return graphs


def alone(lv, g, **params):
    res = lv.run(g.rowptr, g.col, g.w, **{**PARAMS, **params})
    return res.final_labels, res.phases[-1].N_end, len(res.phases), \
        sum(p.iterations for p in res.phases)


def check(lv, h, rid, g, want):
    lab, info = lv.lv_server_result(h, rid)
    assert info.status == 0
    assert np.array_equal(lab, want[0])
    assert (info.N_final, info.num_phases, info.iterations) == want[1:]
    assert info.t_submit_ms <= info.t_admit_ms <= info.t_done_ms


def submit_threads(lv, h, graphs, nthreads=3, jitter=0.002):
    ids = [None] * len(graphs)

    def work(t):
        rng = np.random.default_rng(t)
        for i in range(t, len(graphs), nthreads):
            time.sleep(float(rng.uniform(0, jitter)))
            ids[i] = lv.lv_server_submit(h, graphs[i].rowptr, graphs[i].col, graphs[i].w)

    th = [threading.Thread(target=work, args=(t,)) for t in range(nthreads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return ids


def test_mix_equals_alone(lv):
    graphs = request_mix(0)
    want = [alone(lv, g) for g in graphs]
    h = lv.lv_server_create(**PARAMS)
    try:
        ids = submit_threads(lv, h, graphs)
        for rid in ids:
            assert lv.lv_server_wait(h, rid, 120.0)
        for rid, g, w in zip(ids, graphs, want):
            check(lv, h, rid, g, w)
        st = lv.lv_server_get_stats(h)
        assert st.completed == len(graphs) and st.failed == 0
        assert st.rounds >= 1 and st.sweeps >= 1
    finally:
        lv.lv_server_destroy(h)
    # a sample against the oracle
    for g, rid in list(zip(graphs, ids))[:6]:
        ref = oracle.run(g.rowptr, g.col, g.w, **PARAMS)
        assert ref.phases[-1].N_end == want[graphs.index(g)][1]


def test_arrivals_while_running_join_later_rounds(lv):
    """Requests submitted while a large one is on the GPU are admitted while
    it runs (the large one on the second lane)."""
    big = gg.planted(1_000_000, 100, 0.0012, 0.000002, 1, 4, seed=77)
    small = request_mix(1, 12)
    want_big = alone(lv, big)
    want = [alone(lv, g) for g in small]
    h = lv.lv_server_create(**PARAMS)
    try:
        rb = lv.lv_server_submit(h, big.rowptr, big.col, big.w)
        # submit the small requests once the large one is admitted (no fixed
        # sleep): its solve on the second lane takes far longer than their
        # admission, which needs only budget and slots
        t_end = time.monotonic() + 60.0
        while lv.lv_server_get_stats(h).admitted < 1 and time.monotonic() < t_end:
            time.sleep(0.001)
        ids = [lv.lv_server_submit(h, g.rowptr, g.col, g.w) for g in small]
        assert lv.lv_server_wait(h, rb, 120.0)
        for rid in ids:
            assert lv.lv_server_wait(h, rid, 120.0)
        check(lv, h, rb, big, want_big)
        for rid, g, w in zip(ids, small, want):
            check(lv, h, rid, g, w)
        done_big = lv.lv_server_result(h, rb)[1].t_done_ms
        assert all(lv.lv_server_result(h, rid)[1].t_admit_ms < done_big for rid in ids)
    finally:
        lv.lv_server_destroy(h)


@pytest.mark.parametrize("limits", [dict(mem_budget_bytes=1), dict(max_graphs=3)])
def test_admission_limits_keep_results(lv, limits):
    graphs = request_mix(2, 10)
    want = [alone(lv, g) for g in graphs]
    h = lv.lv_server_create(**PARAMS, **limits)
    try:
        ids = [lv.lv_server_submit(h, g.rowptr, g.col, g.w) for g in graphs]
        for rid in ids:
            assert lv.lv_server_wait(h, rid, 120.0)
        for rid, g, w in zip(ids, graphs, want):
            check(lv, h, rid, g, w)
        st = lv.lv_server_get_stats(h)
        cap = 1 if "mem_budget_bytes" in limits else 3
        assert st.peak_graphs <= cap
    finally:
        lv.lv_server_destroy(h)


def test_invalid_request_fails_alone(lv):
    good = request_mix(3, 5)
    bad = gg.planted(100, 4, 0.2, 0.01, seed=5)
    w = bad.w.copy()
    w[0] += 1  # breaks symmetry
    empty = gg.from_edges(4, [])
    want = [alone(lv, g) for g in good]
    h = lv.lv_server_create(**PARAMS)
    try:
        ids = [lv.lv_server_submit(h, g.rowptr, g.col, g.w) for g in good[:2]]
        rbad = lv.lv_server_submit(h, bad.rowptr, bad.col, w)
        rempty = lv.lv_server_submit(h, empty.rowptr, empty.col, empty.w)
        ids += [lv.lv_server_submit(h, g.rowptr, g.col, g.w) for g in good[2:]]
        for rid in ids + [rbad, rempty]:
            assert lv.lv_server_wait(h, rid, 120.0)
        with pytest.raises(lv.LVError) as ei:
            lv.lv_server_result(h, rbad)
        assert ei.value.code == -2
        with pytest.raises(lv.LVError) as ei:
            lv.lv_server_result(h, rempty)
        assert ei.value.code == -6
        for rid, g, ww in zip(ids, good, want):
            check(lv, h, rid, g, ww)
        lv.lv_server_release(h, ids[0])
        with pytest.raises(lv.LVError):
            lv.lv_server_result(h, ids[0])
        assert lv.lv_server_get_stats(h).failed == 2
    finally:
        lv.lv_server_destroy(h)


def test_all_heuristics_with_colouring(lv):
    """Every heuristic on: requests that colour a phase (at least color_cutoff
    vertices) are solved on the second lane, the rest are batched; each
    result equals lv_run alone with the same parameters."""
    prm = dict(vertex_following=1, coloring=1, color_cutoff=3000, theta_high=1e-2,
               theta_low=1e-6)
    graphs = [gg.planted(8000, 20, 0.01, 0.0003, 1, 4, seed=41), gg.rmat(13, 12, seed=42)]
    graphs += request_mix(4, 12)
    want = [alone(lv, g, **prm) for g in graphs]
    res0 = lv.run(graphs[0].rowptr, graphs[0].col, graphs[0].w, **prm)
    assert res0.phases[0].colored  # the first request does colour
    h = lv.lv_server_create(**prm)
    try:
        ids = submit_threads(lv, h, graphs)
        for rid in ids:
            assert lv.lv_server_wait(h, rid, 120.0)
        for rid, g, w in zip(ids, graphs, want):
            check(lv, h, rid, g, w)
    finally:
        lv.lv_server_destroy(h)


def test_recursive_vf_requests_take_the_single_graph_lane(lv):
    """With recursive vertex following on, every request is solved by the
    single-graph driver (second lane) and equals lv_run alone."""
    prm = dict(vertex_following=1, coloring=0, vf_recursive=1)
    graphs = [gg.from_edges(3, [(0, 0, 100), (0, 1, 50), (1, 2, 1)]),
              gg.from_edges(4, [(0, 1, 8), (1, 2, 8), (2, 3, 1)])] + request_mix(5, 6)
    want = [alone(lv, g, **prm) for g in graphs]
    h = lv.lv_server_create(**prm)
    try:
        ids = [lv.lv_server_submit(h, g.rowptr, g.col, g.w) for g in graphs]
        for rid in ids:
            assert lv.lv_server_wait(h, rid, 120.0)
        for rid, g, w in zip(ids, graphs, want):
            check(lv, h, rid, g, w)
    finally:
        lv.lv_server_destroy(h)
