"""Batched runs vs the oracle run on each graph alone, through the C ABI.

A batch must give every graph exactly what a run of that graph alone gives:
the same phase count, per-phase sizes, exact modularity numerators, iteration
counts and labels (numbered per graph).  Cases: hand-made graphs mixed with
random ones (self-loops, weights, degree-1 vertices), planted-partition
batches with log-uniform sizes, the full 4,096-graph planted workload on
sampled graphs, parameter edges (max_iters, max_phases, vertex following
off), device-resident input and the error contract.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1237_gb300 import _build, lv as lvmod
    _build.build()
    lvmod.load()
    return lvmod


def run_batch(lv, b, stream=0, **params):
    h = lv.lv_batch_create(b.num_graphs, b.gptr, b.rowptr, b.col, b.w, stream=stream)
    try:
        lv.lv_batch_run(h, lv.make_params(**params))
    except Exception:
        lv.lv_batch_destroy(h)
        raise
    return h


def check_graph(lv, h, b, g, **params):
    """Graph g of the batch against the oracle run on it alone."""
    gr = b.graph(g)
    ref = oracle.run(gr.rowptr, gr.col, gr.w, **params)
    gi = lv.lv_batch_get_graph_info(h, g)
    assert (gi.n, gi.arcs, gi.two_m) == (gr.n, gr.arcs, ref.two_m), g
    assert gi.num_phases == len(ref.phases), (g, gi.num_phases, len(ref.phases))
    for p, ph in enumerate(ref.phases):
        info = lv.lv_batch_get_phase_info(h, g, p)
        got = (info.n, info.arcs, info.n_next, info.N_start, info.N_end, info.iterations)
        want = (ph.n, ph.arcs, ph.n_next, ph.N_start, ph.N_end, ph.iterations)
        assert got == want, (g, p, got, want)
        assert info.q == ph.q
        lab = np.empty(gr.n, dtype=np.int32)
        lv.lv_batch_get_labels(h, g, p, lab)
        assert np.array_equal(lab, ph.labels), (g, p)
    assert gi.N_final == ref.phases[-1].N_end and gi.q == ref.q
    assert gi.iterations == sum(ph.iterations for ph in ref.phases)
    assert gi.n_final == ref.phases[-1].n_next
    return ref


def mixed_graphs(golden):
    graphs = []
    for name in ["two_triangles.txt", "two_k5.txt", "ring3_triangles.txt", "k2_singlet.txt",
                 "k4_minlabel.txt", "star_vf.txt"]:
        fx = golden(name)
        graphs.append(gg.from_edges(fx["n"], fx["edges"]))
    graphs.append(gg.from_edges(1, [(0, 0, 3)]))           # one vertex, a self-loop
    graphs.append(gg.from_edges(2, [(0, 1, 5)]))           # K2
    graphs.append(gg.from_edges(4, [(0, 1, 1), (2, 3, 2)]))  # two K2
    for s in range(6):
        graphs.append(gg.random_graph(40 + 37 * s, 0.08, wmax=5, loops=0.1, seed=100 + s))
    graphs.append(gg.planted(900, 9, 0.1, 0.003, 1, 8, seed=11))
    graphs.append(gg.rmat(10, 8, seed=12))
    return graphs


VARIANTS = [
    dict(vertex_following=1, coloring=0),
    dict(vertex_following=0, coloring=0),
    dict(vertex_following=1, coloring=1),  # cutoff 100,000: no graph here is coloured
    dict(vertex_following=1, coloring=0, max_iters=2),
    dict(vertex_following=1, coloring=0, max_phases=1),
    dict(vertex_following=0, coloring=0, theta_low=1e-2),
]


@pytest.mark.parametrize("vi", range(len(VARIANTS)))
def test_mixed_batch(lv, golden, vi):
    graphs = mixed_graphs(golden)
    b = gg.concat(graphs, "mixed")
    params = VARIANTS[vi]
    h = run_batch(lv, b, **params)
    try:
        for g in range(b.num_graphs):
            check_graph(lv, h, b, g, **params)
        # union labels = per-graph final labels, in union order
        allf = np.empty(b.n, dtype=np.int32)
        lv.lv_batch_get_labels(h, -1, -1, allf)
        for g in range(b.num_graphs):
            one = np.empty(int(b.gptr[g + 1] - b.gptr[g]), dtype=np.int32)
            lv.lv_batch_get_labels(h, g, -1, one)
            assert np.array_equal(allf[b.gptr[g]:b.gptr[g + 1]], one)
        st = lv.lv_batch_get_stats(h)
        tot_it = sum(lv.lv_batch_get_graph_info(h, g).iterations for g in range(b.num_graphs))
        assert st.total_iterations == tot_it
        assert st.num_phases == max(lv.lv_batch_get_graph_info(h, g).num_phases
                                    for g in range(b.num_graphs))
    finally:
        lv.lv_batch_destroy(h)


def test_single_graph_batch(lv):
    g = gg.planted(2000, 20, 0.05, 0.002, 1, 3, seed=21)
    b = gg.concat([g])
    h = run_batch(lv, b)
    try:
        check_graph(lv, h, b, 0)
        res = lv.run(g.rowptr, g.col, g.w)
        lab = np.empty(g.n, dtype=np.int32)
        lv.lv_batch_get_labels(h, 0, -1, lab)
        assert np.array_equal(lab, res.final_labels)
        st = lv.lv_batch_get_stats(h)
        assert st.edge_visits == res.stats["edge_visits"]
        assert st.total_iterations == res.stats["total_iterations"]
    finally:
        lv.lv_batch_destroy(h)


@pytest.mark.parametrize("seed", [7, 8])
def test_planted_batch_all_graphs(lv, seed):
    b = gg.planted_batch(num_graphs=48, nmin=100, nmax=20_000, seed=seed)
    h = run_batch(lv, b)
    try:
        for g in range(b.num_graphs):
            check_graph(lv, h, b, g)
    finally:
        lv.lv_batch_destroy(h)


def test_bins_do_not_change_results(lv):
    b = gg.planted_batch(num_graphs=16, nmin=200, nmax=8_000, seed=9)
    h0 = run_batch(lv, b)
    h1 = run_batch(lv, b, bin_lane_arcs=1, bin_warp_max=16, bin_cta_max=64)
    try:
        a0 = np.empty(b.n, dtype=np.int32)
        a1 = np.empty(b.n, dtype=np.int32)
        lv.lv_batch_get_labels(h0, -1, -1, a0)
        lv.lv_batch_get_labels(h1, -1, -1, a1)
        assert np.array_equal(a0, a1)
        for g in range(0, b.num_graphs, 5):
            check_graph(lv, h1, b, g)
    finally:
        lv.lv_batch_destroy(h0)
        lv.lv_batch_destroy(h1)


def test_device_input_and_determinism(lv):
    import torch
    b = gg.planted_batch(num_graphs=12, nmin=100, nmax=5_000, seed=10)
    dev = torch.device("cuda:0")
    t = [torch.from_numpy(x).to(dev) for x in (b.gptr, b.rowptr, b.col, b.w)]
    torch.cuda.synchronize()
    outs = []
    for _ in range(2):
        h = lv.lv_batch_create(b.num_graphs, *t)
        try:
            lv.lv_batch_run(h)
            out = torch.empty(b.n, dtype=torch.int32, device=dev)
            lv.lv_batch_get_labels(h, -1, -1, out)
            outs.append(out.cpu().numpy())
            check_graph(lv, h, b, 3)
        finally:
            lv.lv_batch_destroy(h)
    assert np.array_equal(outs[0], outs[1])


def test_full_planted_workload_sampled(lv):
    """The 4,096-graph planted workload (log-uniform 100..50,000 vertices):
    sampled graphs (smallest, largest, spread) against the oracle, and the
    per-graph totals against the batch totals."""
    b = gg.planted_batch()
    h = run_batch(lv, b)
    try:
        sizes = np.diff(b.gptr)
        pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
        pick |= set(int(x) for x in np.random.default_rng(0).choice(b.num_graphs, 14, replace=False))
        for g in sorted(pick):
            check_graph(lv, h, b, g)
        st = lv.lv_batch_get_stats(h)
        infos = [lv.lv_batch_get_graph_info(h, g) for g in range(b.num_graphs)]
        assert st.total_iterations == sum(i.iterations for i in infos)
        assert all(i.num_phases >= 1 and -0.5 <= i.q < 1.0 for i in infos)
        allf = np.empty(b.n, dtype=np.int32)
        lv.lv_batch_get_labels(h, -1, -1, allf)
        # labels form a partition numbered 0..n_final-1 inside every graph
        for g in range(0, b.num_graphs, 97):
            seg = allf[b.gptr[g]:b.gptr[g + 1]]
            assert np.array_equal(np.unique(seg), np.arange(infos[g].n_final))
    finally:
        lv.lv_batch_destroy(h)


def test_batch_errors(lv):
    a = gg.planted(50, 5, 0.3, 0.02, seed=1)
    c = gg.planted(60, 6, 0.3, 0.02, seed=2)
    b = gg.concat([a, c])
    E = lv.LVError
    # malformed gptr
    for gp in (np.array([1, 50, 110]), np.array([0, 50, 50, 110]), np.array([0, 60, 110])):
        with pytest.raises(E) as ei:
            lv.lv_batch_create(len(gp) - 1, gp.astype(np.int64), b.rowptr, b.col, b.w)
        assert ei.value.code == -1, gp
    # an arc between graphs
    n = 4
    x = gg.from_edges(n, [(0, 1, 1), (1, 2, 1), (2, 3, 1)])
    with pytest.raises(E) as ei:
        lv.lv_batch_create(2, np.array([0, 2, 4], dtype=np.int64), x.rowptr, x.col, x.w)
    assert ei.value.code == -1
    # a graph without edges
    y = gg.concat([a, gg.from_edges(3, [])])
    with pytest.raises(E) as ei:
        lv.lv_batch_create(2, y.gptr, y.rowptr, y.col, y.w)
    assert ei.value.code == -6
    # the union CSR rules still apply (asymmetric arc)
    bad = b.w.copy()
    bad[0] += 1
    with pytest.raises(E) as ei:
        lv.lv_batch_create(2, b.gptr, b.rowptr, b.col, bad)
    assert ei.value.code == -2
    h = lv.lv_batch_create(2, b.gptr, b.rowptr, b.col, b.w)
    try:
        out = np.empty(b.n, dtype=np.int32)
        with pytest.raises(E) as ei:
            lv.lv_batch_get_labels(h, -1, -1, out)
        assert ei.value.code == -10
        # colouring would apply to a graph of >= cutoff vertices: not batched
        with pytest.raises(E) as ei:
            lv.lv_batch_run(h, lv.make_params(coloring=1, color_cutoff=1))
        assert ei.value.code == -1
        lv.lv_batch_run(h, lv.make_params(coloring=1, color_cutoff=1000))
        assert lv.lv_batch_num_graphs(h) == 2
        with pytest.raises(E) as ei:
            lv.lv_batch_get_phase_info(h, 0, 99)
        assert ei.value.code == -10
        with pytest.raises(E):
            lv.lv_batch_get_graph_info(h, 2)
    finally:
        lv.lv_batch_destroy(h)


def test_autotune_and_graph_capture_keep_results(lv):
    """Bins chosen by timing and sweeps replayed from a captured CUDA graph
    change no result."""
    import torch
    b = gg.planted_batch(num_graphs=40, nmin=20_000, nmax=50_000, seed=12)
    assert b.arcs >= 1 << 22  # large enough to be tuned
    stream = torch.cuda.Stream()  # capture needs a stream other than the legacy default
    runs = {}
    for key, prm in {"plain": dict(autotune=0, graph_capture=0),
                     "tuned": dict(autotune=1, graph_capture=1)}.items():
        h = run_batch(lv, b, stream=stream.cuda_stream, **prm)
        try:
            if key == "tuned":
                lv.lv_batch_run(h, lv.make_params(**prm))  # second run reuses the choice
            lab = np.empty(b.n, dtype=np.int32)
            lv.lv_batch_get_labels(h, -1, -1, lab)
            st = lv.lv_batch_get_stats(h)
            runs[key] = (lab, st.graph_launches, st.sweep_launches)
            if key == "tuned":
                for g in (0, 17, 39):
                    check_graph(lv, h, b, g)
                t = lv.lv_batch_get_tuning(h, 0)  # the first round is large enough
                assert t is not None and t["blocks_per_sm"] in (0, 1)
                assert t["hub_slots_per_arc"] in (0, 4) and 1 <= t["lane_arcs"] <= 8
                assert lv.lv_batch_get_tuning(h, 1000) is None
        finally:
            lv.lv_batch_destroy(h)
    assert np.array_equal(runs["plain"][0], runs["tuned"][0])
    assert runs["plain"][1] == 0
    assert 0 < runs["tuned"][1] <= runs["tuned"][2]


def test_autotune_single_graph(lv):
    g = gg.rmat(18, 16, seed=5)
    assert g.arcs >= 1 << 22
    a = lv.run(g.rowptr, g.col, g.w, coloring=0)
    h = lv.lv_graph_create(g.n, g.rowptr, g.col, g.w)
    try:
        for _ in range(2):
            lv.lv_run(h, lv.make_params(coloring=0, autotune=1))
            res = lv.collect(h, g.n)
            assert len(res.phases) == len(a.phases)
            for x, y in zip(res.phases, a.phases):
                assert (x.N_end, x.iterations) == (y.N_end, y.iterations)
                assert np.array_equal(x.labels, y.labels)
        assert lv.lv_get_tuning(h, 0) is not None
    finally:
        lv.lv_graph_destroy(h)


@pytest.mark.parametrize("shape", [dict(sweep_blocks_per_sm=1), dict(hub_slots_per_arc=4),
                                   dict(hub_slots_per_arc=8, sweep_blocks_per_sm=2),
                                   dict(hub_slots_per_arc=2)])
def test_autotune_shape_knobs_keep_results(lv, shape):
    """Every launch shape the autotuner can choose (sweep blocks per SM, hub
    table slots per arc) gives the same labels, coloured and uncoloured,
    single graph and batch."""
    g, prm = gg.workload("rmat16")
    a = lv.run(g.rowptr, g.col, g.w, **prm)
    r = lv.run(g.rowptr, g.col, g.w, **prm, **shape)
    for x, y in zip(r.phases, a.phases):
        assert (x.N_end, x.iterations) == (y.N_end, y.iterations)
        assert np.array_equal(x.labels, y.labels)
    b = gg.planted_batch(num_graphs=12, nmin=500, nmax=20_000, seed=21)
    runs = []
    for extra in ({}, shape):
        h = run_batch(lv, b, **extra)
        try:
            lab = np.empty(b.n, dtype=np.int32)
            lv.lv_batch_get_labels(h, -1, -1, lab)
            runs.append(lab)
        finally:
            lv.lv_batch_destroy(h)
    assert np.array_equal(runs[0], runs[1])


def test_shape_knobs_validated(lv):
    g = gg.rmat(8, 8, seed=1)
    for bad in (dict(sweep_blocks_per_sm=3), dict(hub_slots_per_arc=3)):
        with pytest.raises(lv.LVError) as e:
            lv.run(g.rowptr, g.col, g.w, **bad)
        assert e.value.code == -1


def test_batch_variants(lv, golden):
    """The absolute-threshold variant in batches (colouring does not batch)."""
    graphs = mixed_graphs(golden)
    b = gg.concat(graphs, "mixed")
    prm = dict(vertex_following=1, coloring=0, abs_threshold=1, max_iters=25)
    h = run_batch(lv, b, **prm)
    try:
        for g in range(b.num_graphs):
            check_graph(lv, h, b, g, **prm)
    finally:
        lv.lv_batch_destroy(h)
