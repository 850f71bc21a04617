"""GPU path vs the serial oracle, through the C ABI.

Labels, exact modularity numerators, iteration and phase counts must be
identical at every phase; with keep_graphs the phase graphs (vertex
following output and every coarse graph) and colourings must be identical
too.  Sizes run from hand-made graphs through several tiles with ragged
tails up to the full R-MAT scale-20 workload; the 2^24-vertex Chung-Lu
workload is checked on its first iterations in full and on invariants and
exact modularity at full length.
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


def compare(lv, g, graphs=True, iters=True, **params):
    res = lv.run(g.rowptr, g.col, g.w, keep_graphs=int(graphs), **params)
    ref = oracle.run(g.rowptr, g.col, g.w, trace=int(graphs), **params)
    assert res.two_m == ref.two_m
    assert np.array_equal(res.vf_map, ref.vf_map)
    assert len(res.phases) == len(ref.phases), ([p.n for p in res.phases], [p.n for p in ref.phases])
    for pi, (a, b) in enumerate(zip(res.phases, ref.phases)):
        assert (a.n, a.arcs, a.n_next) == (b.n, b.arcs, b.n_next), pi
        assert (a.colored, a.num_colors) == (b.colored, b.num_colors), pi
        assert a.N_start == b.N_start, pi
        assert a.N_end == b.N_end, pi
        assert a.iterations == b.iterations, pi
        assert a.q == b.q
        assert np.array_equal(a.labels, b.labels), pi
    if iters:
        got = [(t[0], t[1], t[3], t[4]) for t in res.iters]
        want = [(t[0], t[1], t[2], t[3]) for t in ref.iters]
        assert got == want
    if graphs:
        h = lv.lv_graph_create(g.n, g.rowptr, g.col, g.w)
        try:
            lv.lv_run(h, lv.make_params(keep_graphs=1, **params))
            for pi, b in enumerate(ref.phases):
                rp, col, w = lv.lv_get_phase_graph(h, pi)
                assert np.array_equal(rp, b.graph[0]) and np.array_equal(col, b.graph[1])
                assert np.array_equal(w, b.graph[2])
                if b.colored:
                    assert np.array_equal(lv.lv_get_phase_colors(h, pi, b.n), b.colors)
        finally:
            lv.lv_graph_destroy(h)
    return res, ref


VARIANTS = [
    dict(vertex_following=0, coloring=0),
    dict(vertex_following=1, coloring=0),
    dict(vertex_following=0, coloring=1, color_cutoff=0),
    dict(vertex_following=1, coloring=1, color_cutoff=0, theta_high=1e-2),
]


@pytest.mark.parametrize("name", ["two_triangles.txt", "two_k5.txt", "ring3_triangles.txt",
                                  "k2_singlet.txt", "k4_minlabel.txt", "star_vf.txt",
                                  "zero_gain.txt"])
@pytest.mark.parametrize("vi", range(len(VARIANTS)))
def test_golden_graphs(lv, golden, name, vi):
    fx = golden(name)
    g = gg.from_edges(fx["n"], fx["edges"])
    compare(lv, g, **VARIANTS[vi])


@pytest.mark.parametrize("seed", range(8))
def test_random_small(lv, seed):
    n = [37, 100, 257, 511, 1000, 1537, 2049, 3001][seed]
    g = gg.random_graph(n, min(0.5, 12.0 / n), wmax=1 + seed, loops=0.1 * (seed % 3), seed=seed)
    if g.two_m == 0:
        pytest.skip("empty draw")
    for v in VARIANTS:
        compare(lv, g, **v)


@pytest.mark.parametrize("bins", [(1, 1, 2), (1, 2, 3), (2, 8, 16), (1, 32, 64), (4, 128, 4096),
                                  (8, 256, 4096), (3, 100, 1000)])
def test_every_bin_path(lv, bins):
    # small bin limits push ordinary vertices through the CTA and hub kernels
    g = gg.chunglu(4000, 2.1, 0.7, 16000, 300.0, seed=7)
    la, w_, c = bins
    kw = dict(bin_lane_arcs=la, bin_warp_max=w_, bin_cta_max=c)
    compare(lv, g, vertex_following=1, coloring=1, color_cutoff=0, **kw)
    compare(lv, g, graphs=False, vertex_following=0, coloring=0, **kw)


def test_hub_vertex(lv):
    # a hub of degree 12,000 (> CTA bin) joined to a ring; VF off keeps it
    n = 12001
    edges = [(0, i, 1 + i % 5) for i in range(1, n)] + [(i, i + 1) for i in range(1, n - 1)]
    g = gg.from_edges(n, edges)
    compare(lv, g, vertex_following=0, coloring=0)
    compare(lv, g, vertex_following=1, coloring=1, color_cutoff=0)


def test_planted1k(lv):
    g, prm = gg.workload("planted1k")
    compare(lv, g, **prm)


def test_rmat16(lv):
    g, prm = gg.workload("rmat16")
    compare(lv, g, **prm)


def test_chunglu_small(lv):
    g = gg.chunglu(50_000, 2.1, 0.7, 400_000, 2000.0, seed=3)
    compare(lv, g, vertex_following=1, coloring=1, color_cutoff=10_000, theta_high=1e-2)


def test_rmat20_full(lv):
    g, prm = gg.workload("rmat20")
    compare(lv, g, graphs=False, **prm)


def test_determinism(lv):
    g, prm = gg.workload("rmat16")
    a = lv.run(g.rowptr, g.col, g.w, **prm)
    b = lv.run(g.rowptr, g.col, g.w, bin_lane_arcs=2, bin_warp_max=64, bin_cta_max=512, **prm)
    for x, y in zip(a.phases, b.phases):
        assert np.array_equal(x.labels, y.labels) and x.N_end == y.N_end


def test_device_pointers_and_stream(lv):
    torch = pytest.importorskip("torch")
    g, prm = gg.workload("planted1k")
    dev = torch.device("cuda:0")
    s = torch.cuda.Stream()
    t = [torch.from_numpy(x).to(dev) for x in (g.rowptr, g.col, g.w)]
    torch.cuda.synchronize()
    h = lv.lv_graph_create(g.n, *t, stream=s.cuda_stream)
    try:
        lv.lv_run(h, lv.make_params(**prm))
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
        lv.lv_get_labels(h, -1, out)
        ref = oracle.run(g.rowptr, g.col, g.w, **prm)
        assert np.array_equal(out.cpu().numpy(), ref.final_labels)
        q, num, den = lv.lv_get_modularity(h, -1)
        assert num == ref.phases[-1].N_end and den == ref.two_m ** 2
    finally:
        lv.lv_graph_destroy(h)


@pytest.mark.slow
def test_chunglu24_first_iterations(lv):
    # two iterations of phase 0 in full: labels after them, and each
    # iteration's moves and exact numerator
    g, prm = gg.workload("chunglu24")
    compare(lv, g, graphs=False, max_phases=1, max_iters=2, **prm)


@pytest.mark.slow
def test_chunglu24_full_invariants(lv):
    g, prm = gg.workload("chunglu24")
    res = lv.run(g.rowptr, g.col, g.w, **prm)
    prev = None
    for p in res.phases:
        assert set(np.unique(p.labels).tolist()) == set(range(p.n_next))
        N, tm = oracle.modularity_num(g.rowptr, g.col, g.w, p.labels)
        assert tm == res.two_m and N == p.N_end
        if prev is not None:
            assert p.N_start == prev.N_end
        assert -0.5 <= p.q < 1
        prev = p


# ----------------------------------------------------- heuristic variants
@pytest.mark.parametrize("name", ["two_k5.txt", "ring3_triangles.txt", "star_vf.txt"])
def test_variant_golden_abs_threshold(lv, golden, name):
    fx = golden(name)
    g = gg.from_edges(fx["n"], fx["edges"])
    compare(lv, g, coloring=0, abs_threshold=1, max_iters=30)


def test_variant_abs_threshold_cycles_to_guard(lv):
    # the absolute test 2-cycles on the planted graph until max_iters (R9)
    g, _ = gg.workload("planted1k")
    res, ref = compare(lv, g, graphs=False, coloring=0, abs_threshold=1, max_iters=40)
    assert res.phases[0].iterations == 40


def test_variant_first_phase_colouring(lv):
    g = gg.rmat(16, 8, seed=31)
    res, ref = compare(lv, g, graphs=True, color_cutoff=0, theta_high=0.0, color_phases=1)
    assert res.phases[0].colored and not any(p.colored for p in res.phases[1:])


def _core_graph(case):
    rng = np.random.default_rng(11)
    if case == "clique":  # every vertex in the degree >= 64 core
        n = 80
        return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    if case == "equal_degrees":  # the core ordered by the hash alone
        n, k = 2000, 35
        return gg.from_edges(n, [(i, (i + j) % n) for i in range(n) for j in range(1, k + 1)])
    # hubs joined to each other (a deep core chain) and to leaves, weighted
    hubs, leaves = 200, 100
    edges = [(i, j, int(rng.integers(1, 4))) for i in range(hubs) for j in range(i + 1, hubs)
             if rng.random() < 0.5]
    n = hubs + hubs * leaves
    for h in range(hubs):
        for t in range(leaves):
            edges.append((h, hubs + h * leaves + t, 1))
    edges += [(int(a), int(b), 1) for a, b in rng.integers(hubs, n, size=(3 * n, 2)) if a != b]
    return gg.from_edges(n, edges)


@pytest.mark.parametrize("case", ["clique", "equal_degrees", "hubs"])
def test_colouring_core_without_rounds(lv, case):
    """Graphs whose vertices of degree >= 64 are coloured before the rounds:
    the colourings (and the runs) equal the oracle's."""
    g = _core_graph(case)
    for vf in (0, 1):
        res, ref = compare(lv, g, graphs=True, vertex_following=vf, coloring=1, color_cutoff=0)
        assert res.phases[0].colored


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("graph", ["rmat16", "hubs"])
def test_colour_orders(lv, order, graph):
    """Both colouring priorities (R11) against the oracle: largest degree
    first (its degree core coloured before the rounds) and hash only (no
    core: rounds alone)."""
    g = gg.rmat(16, 8, seed=33) if graph == "rmat16" else _core_graph("hubs")
    res, ref = compare(lv, g, graphs=True, color_cutoff=0, color_order=order)
    assert res.phases[0].colored


def test_variant_colour_phase_theta(lv):
    g = gg.rmat(16, 8, seed=32)
    compare(lv, g, graphs=False, color_cutoff=0, theta_high=1e-4)


# --------------------------------------------- qualitative comparison (Sec. 5)
def test_compare_partitions_against_oracle(lv):
    rng = np.random.default_rng(5)
    for n, ks, kp in [(2, 1, 1), (3, 2, 3), (500, 7, 5), (2000, 40, 3), (1500, 1500, 1)]:
        s = rng.integers(0, ks, size=n).astype(np.int32)
        p = rng.integers(0, kp, size=n).astype(np.int32)
        got = lv.lv_compare_partitions(s, p)
        want = oracle.compare(s, p)
        for key in ("tp", "fp", "fn", "tn", "sp", "se", "oq", "rand"):
            assert got[key] == want[key], (n, key, got[key], want[key])
    assert lv.lv_compare_partitions(np.zeros(0, np.int32), np.zeros(0, np.int32))["rand"] == 1.0
    # labels of any value, negative ones included
    s = np.array([-5, -5, 7, 2**31 - 1, 2**31 - 1], dtype=np.int32)
    p = np.array([0, 1, 1, 3, 3], dtype=np.int32)
    assert lv.lv_compare_partitions(s, p) == oracle.compare(s, p)


def test_compare_partitions_large_device(lv):
    """A phase's labels against the final ones on R-MAT 20 (device arrays),
    against the contingency-table counts computed in numpy."""
    import torch
    g, prm = gg.workload("rmat20")
    res = lv.run(g.rowptr, g.col, g.w, **prm)
    s, p = res.phases[0].labels, res.final_labels
    got = lv.lv_compare_partitions(torch.from_numpy(s).cuda(), torch.from_numpy(p).cuda())
    pairs = lambda x: int((x.astype(np.int64) * (x.astype(np.int64) - 1) // 2).sum())
    _, nij = np.unique(np.stack([s, p], 1), axis=0, return_counts=True)
    tp = pairs(nij)
    assert got["tp"] == tp
    assert got["fn"] == pairs(np.unique(s, return_counts=True)[1]) - tp
    assert got["fp"] == pairs(np.unique(p, return_counts=True)[1]) - tp
    n = len(s)
    assert got["tp"] + got["fp"] + got["fn"] + got["tn"] == n * (n - 1) // 2
    assert got["fn"] == 0  # phase-0 communities nest inside the final ones


# ---------------------------------------------------------------- validation
def _arc(g, i, j):
    """Index of arc (i, j) in the CSR of g."""
    seg = g.col[g.rowptr[i]:g.rowptr[i + 1]]
    k = int(np.searchsorted(seg, j))
    assert seg[k] == j
    return int(g.rowptr[i]) + k


def _drop(g, e):
    rp = g.rowptr.copy()
    rp[int(np.searchsorted(g.rowptr, e, side="right")):] -= 1
    return rp, np.delete(g.col, e), np.delete(g.w, e)


def _validation_cases():
    """Single-defect CSRs around a hub row (pairs of very unequal rows, both
    orders of the defect) and a cycle (pairs of equal rows)."""
    rng = np.random.default_rng(11)
    edges = [(0, v, int(rng.integers(1, 6))) for v in range(1, 1501)]
    edges += [(int(a), int(b), 1) for a, b in rng.integers(1, 1501, size=(3000, 2)) if a != b]
    edges += [(7, 7, 3)]
    hub = gg.from_edges(1501, edges)
    cyc = gg.from_edges(50, [(v, (v + 1) % 50, 1 + v % 3) for v in range(50)])
    cases = [("hub valid", hub.rowptr, hub.col, hub.w), ("cycle valid", cyc.rowptr, cyc.col, cyc.w)]
    for g, tag, i, j in [(hub, "hub row", 0, 5), (hub, "leaf row", 5, 0), (cyc, "tie up", 4, 3),
                         (cyc, "tie down", 3, 4)]:
        e = _arc(g, i, j)
        cases.append((f"{tag}: arc dropped", *_drop(g, e)))
        w = g.w.copy()
        w[e] += 1
        cases.append((f"{tag}: weight differs", g.rowptr, g.col, w))
    e, f = _arc(hub, 0, 9), _arc(hub, 9, 0)
    w = hub.w.copy()
    w[e] = w[f] = 0
    cases.append(("zero weight pair", hub.rowptr, hub.col, w))
    col = hub.col.copy()
    col[e], col[e + 1] = col[e + 1], col[e]
    cases.append(("unsorted row", hub.rowptr, col, hub.w))
    col = hub.col.copy()
    col[_arc(hub, 5, 0)] = 1501
    cases.append(("column out of range", hub.rowptr, col, hub.w))
    col = hub.col.copy()
    col[e + 1] = col[e]
    cases.append(("duplicate in row", hub.rowptr, col, hub.w))
    return cases


def test_validation_codes_match_oracle(lv):
    """lv_graph_create rejects exactly what the oracle rejects, with the same
    status, for one defect at a time (both arcs of a pair between unequal
    rows, and between equal rows)."""
    for name, rp, col, w in _validation_cases():
        want = oracle.validate(rp, col, w)[0]
        try:
            lv.lv_graph_destroy(lv.lv_graph_create(len(rp) - 1, rp, col, w))
            got = 0
        except lv.LVError as err:
            got = err.code
        assert got == want, name
        assert (want == 0) == name.endswith("valid"), name


# ------------------------------------- recursive single-neighbour VF (R23)
def _recursive_vf_graphs():
    from test_oracle_pins import _pendant_graph
    out = [gg.from_edges(3, [(0, 0, 100), (0, 1, 50), (1, 2, 1)]),
           gg.from_edges(4, [(0, 1, 8), (1, 2, 8), (2, 3, 1)]),
           gg.from_edges(6, [(0, 2), (2, 3), (0, 3), (3, 4), (2, 4), (1, 5, 50), (1, 1, 3),
                             (5, 5, 3)])]
    out += [_pendant_graph(s)[0] for s in range(6)]
    return out


@pytest.mark.parametrize("idx", range(9))
def test_variant_recursive_vf_merging_graphs(lv, idx):
    g = _recursive_vf_graphs()[idx]
    compare(lv, g, vertex_following=1, vf_recursive=1, coloring=0)


@pytest.mark.parametrize("wl", ["planted1k", "rmat16"])
def test_variant_recursive_vf_workloads(lv, wl):
    g, prm = gg.workload(wl)
    compare(lv, g, graphs=False, vf_recursive=1, **prm)


def test_recursive_vf_random_looped(lv):
    # a looped random graph with heavy pendant edges: several vertices merge
    rng = np.random.default_rng(9)
    edges = [(i, (i + 1) % 40, 1) for i in range(40)]
    for t in range(30):
        edges.append((40 + t, int(rng.integers(0, 40)), int(rng.integers(1, 60))))
        edges.append((40 + t, 40 + t, int(rng.integers(1, 4))))
    g = gg.from_edges(70, edges)
    ref = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, vf_recursive=1, coloring=0)
    assert ref.vf_n < 70
    compare(lv, g, vertex_following=1, vf_recursive=1, coloring=0)


def test_recursive_vf_is_single_graph_only(lv):
    g = gg.from_edges(3, [(0, 1), (1, 2)])
    gptr = np.array([0, 3], dtype=np.int64)
    h = lv.lv_batch_create(1, gptr, g.rowptr, g.col, g.w)
    try:
        with pytest.raises(lv.LVError) as e:
            lv.lv_batch_run(h, lv.make_params(vf_recursive=1))
        assert e.value.code == -1
    finally:
        lv.lv_batch_destroy(h)
