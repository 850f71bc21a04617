"""Pins of the serial oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: closed
forms of Eq. 3 evaluated by hand (tests/golden), the exact change of the
modularity numerator under single and paired moves (Eqs. 4 and 6), the
worked minimum-label cases of Sec. 4.1, the vertex-following lemma of
Sec. 4.3, brute-force optima on graphs of at most 10 vertices, an
independent colouring routine, and structural invariants.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN_Q = ["two_triangles.txt", "two_k5.txt", "ring3_triangles.txt"]


def _g(fx):
    return gg.from_edges(fx["n"], fx["edges"])


# ------------------------------------------------------------------ Eq. 3
@pytest.mark.parametrize("name", GOLDEN_Q)
def test_q_closed_form(golden, name):
    fx = golden(name)
    g = _g(fx)
    assert oracle.modularity(g.rowptr, g.col, g.w, fx["partition"]) == fx["q"]


@pytest.mark.parametrize("r,s", [(3, 3), (4, 3), (5, 4), (6, 5), (3, 6)])
def test_q_ring_of_cliques(r, s):
    # ring of r cliques K_s joined by single edges; partition = the cliques:
    # Q = l/(l+1) - 1/r with l = s(s-1)/2 (each clique has l edges plus one
    # ring edge per clique), evaluated from Eq. 3 by hand
    edges = []
    for b in range(r):
        base = b * s
        edges += [(base + i, base + j) for i in range(s) for j in range(i + 1, s)]
        edges.append((base + s - 1, ((b + 1) % r) * s))
    g = gg.from_edges(r * s, edges)
    part = [v // s for v in range(r * s)]
    l = s * (s - 1) // 2
    assert oracle.modularity(g.rowptr, g.col, g.w, part) == Fraction(l, l + 1) - Fraction(1, r)


def test_q_singletons_and_single_community():
    g = gg.random_graph(30, 0.2, wmax=5, loops=0.3, seed=4)
    k = np.add.reduceat(g.w.astype(np.int64), g.rowptr[:-1]) if g.arcs else np.zeros(g.n)
    k = np.array([g.w[g.rowptr[i]:g.rowptr[i + 1]].sum() for i in range(g.n)], dtype=np.int64)
    loops = sum(int(g.w[e]) for i in range(g.n) for e in range(g.rowptr[i], g.rowptr[i + 1])
                if g.col[e] == i)
    two_m = int(k.sum())
    # singletons: N = 2m * (sum of self-loops) - sum k_i^2
    N, tm = oracle.modularity_num(g.rowptr, g.col, g.w, np.arange(g.n))
    assert tm == two_m
    assert N == two_m * loops - int((k * k).sum())
    # one community: every arc is intra, a = 2m, N = 2m*2m - (2m)^2 = 0
    N1, _ = oracle.modularity_num(g.rowptr, g.col, g.w, np.zeros(g.n))
    assert N1 == 0


@pytest.mark.parametrize("seed", range(6))
def test_q_bounds(seed):
    rng = np.random.default_rng(seed)
    g = gg.random_graph(25, 0.25, wmax=9, loops=0.2, seed=seed)
    for _ in range(20):
        lab = rng.integers(0, rng.integers(1, 26), size=g.n)
        q = oracle.modularity(g.rowptr, g.col, g.w, lab)
        assert Fraction(-1, 2) <= q < 1


# ------------------------------------------------------------------ Eq. 4
def _move(lab, i, c):
    lab = np.array(lab, dtype=np.int32)
    lab[i] = c
    return lab


@pytest.mark.parametrize("seed", range(8))
def test_gain_is_half_the_numerator_change(seed):
    # Moving i alone from C(i) to c changes N = (2m)^2 Q by exactly 2G, G the
    # scaled gain of Eq. 4.  A dropped term, a wrong sign or a self-loop
    # counted in e_{i->C} breaks this identity.
    rng = np.random.default_rng(100 + seed)
    g = gg.random_graph(18, 0.3, wmax=7, loops=0.4, seed=seed)
    for _ in range(40):
        lab = rng.integers(0, 6, size=g.n).astype(np.int32)
        i = int(rng.integers(0, g.n))
        c = int(rng.integers(0, g.n))
        if c == lab[i]:
            continue
        G = oracle.gain(g.rowptr, g.col, g.w, lab, i, c)
        N0, tm = oracle.modularity_num(g.rowptr, g.col, g.w, lab)
        N1, _ = oracle.modularity_num(g.rowptr, g.col, g.w, _move(lab, i, c))
        assert N1 - N0 == 2 * G
        # and the same gain in the paper's own scaling (Eq. 4)
        m = Fraction(tm, 2)
        k = [int(g.w[g.rowptr[v]:g.rowptr[v + 1]].sum()) for v in range(g.n)]
        row = range(g.rowptr[i], g.rowptr[i + 1])
        e_c = sum(int(g.w[e]) for e in row if g.col[e] != i and lab[g.col[e]] == c)
        e_o = sum(int(g.w[e]) for e in row if g.col[e] != i and lab[g.col[e]] == lab[i])
        a_c = sum(k[v] for v in range(g.n) if lab[v] == c)
        a_o = sum(k[v] for v in range(g.n) if lab[v] == lab[i]) - k[i]
        dq = Fraction(e_c - e_o) / m + Fraction(2 * k[i] * a_o - 2 * k[i] * a_c) / (2 * m) ** 2
        assert dq == Fraction(2 * G, tm * tm)


@pytest.mark.parametrize("seed", range(6))
def test_two_movers_eq6(seed):
    # Eq. 6 (negative-gain scenario): i and j, in two different communities,
    # both move to a third community C(k).  Scaled by (2m)^2:
    #   dN_ij = 2G_i + 2G_j + 2 (2m w(i,j) - k_i k_j)
    rng = np.random.default_rng(200 + seed)
    g = gg.random_graph(16, 0.35, wmax=5, loops=0.3, seed=50 + seed)
    k = [int(g.w[g.rowptr[v]:g.rowptr[v + 1]].sum()) for v in range(g.n)]
    wmap = {}
    for u in range(g.n):
        for e in range(g.rowptr[u], g.rowptr[u + 1]):
            wmap[(u, int(g.col[e]))] = int(g.w[e])
    checked = 0
    for _ in range(200):
        lab = rng.integers(0, 5, size=g.n).astype(np.int32)
        i, j = (int(x) for x in rng.choice(g.n, size=2, replace=False))
        c = int(rng.integers(0, 5))
        if len({int(lab[i]), int(lab[j]), c}) < 3:
            continue
        Gi = oracle.gain(g.rowptr, g.col, g.w, lab, i, c)
        Gj = oracle.gain(g.rowptr, g.col, g.w, lab, j, c)
        N0, tm = oracle.modularity_num(g.rowptr, g.col, g.w, lab)
        lab2 = _move(_move(lab, i, c), j, c)
        N2, _ = oracle.modularity_num(g.rowptr, g.col, g.w, lab2)
        assert N2 - N0 == 2 * Gi + 2 * Gj + 2 * (tm * wmap.get((i, j), 0) - k[i] * k[j])
        checked += 1
    assert checked > 20


# --------------------------------------------------------- Sec. 4.1 cases
def test_k2_singlet_rule(golden):
    fx = golden("k2_singlet.txt")
    g = _g(fx)
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0, trace=1)
    p0 = r.phases[0]
    assert list(p0.iter_labels[0]) == fx["iter1"]
    assert Fraction(p0.N_start, p0.two_m ** 2) == fx["q_start"]
    assert Fraction(r.phases[-1].N_end, r.two_m ** 2) == fx["q"]


def test_zero_gain_does_not_move(golden):
    fx = golden("zero_gain.txt")
    g = _g(fx)
    assert oracle.gain(g.rowptr, g.col, g.w, list(range(fx["n"])), 1, 0) == 0
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0, trace=1)
    p0 = r.phases[0]
    assert r.two_m == 6
    assert list(p0.iter_labels[0]) == fx["iter1"]
    assert Fraction(p0.N_start, p0.two_m ** 2) == fx["q_start"]
    assert Fraction(r.phases[-1].N_end, r.two_m ** 2) == fx["q"]


def test_k4_generalised_min_label(golden):
    fx = golden("k4_minlabel.txt")
    g = _g(fx)
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0, trace=1)
    assert list(r.phases[0].iter_labels[0]) == fx["iter1"]
    assert Fraction(r.phases[-1].N_end, r.two_m ** 2) == fx["q"]


def test_star_vertex_following(golden):
    fx = golden("star_vf.txt")
    g = _g(fx)
    (rp, col, w), m = oracle.vertex_following(g.rowptr, g.col, g.w)
    assert len(rp) - 1 == fx["vf_n"]
    assert list(col) == [0] and list(w) == [fx["vf_loop"]]
    assert list(m) == [0] * 6
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0)
    assert r.vf_n == 1
    assert Fraction(r.phases[-1].N_end, r.two_m ** 2) == fx["q"]


def test_swap_without_singlet_rule_would_oscillate():
    # Sec. 3.2: two singletons joined by an edge would swap forever without
    # the rule; with it the pair merges in one iteration and then stops.
    g = gg.from_edges(2, [(0, 1, 3)])
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0)
    assert r.phases[0].iterations == 2  # one move, then a no-move iteration
    assert list(r.final_labels) == [0, 0]


# ------------------------------------------------------------ Sec. 4.3 VF
def test_vf_cases():
    # path 0-1-2-3: ends merge into 1 and 2, each gets self-loop 2
    g = gg.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    (rp, col, w), m = oracle.vertex_following(g.rowptr, g.col, g.w)
    assert list(rp) == [0, 2, 4] and list(col) == [0, 1, 0, 1] and list(w) == [2, 1, 1, 2]
    assert list(m) == [0, 0, 1, 1]
    # isolated edge: only the smaller id merges (R3); plus a triangle
    g = gg.from_edges(5, [(0, 1, 4), (2, 3), (3, 4), (2, 4)])
    (rp, col, w), m = oracle.vertex_following(g.rowptr, g.col, g.w)
    assert list(m) == [0, 0, 1, 2, 3]
    assert list(col[rp[0]:rp[1]]) == [0] and list(w[rp[0]:rp[1]]) == [8]
    # a degree-one vertex with a self-loop has two entries and is kept
    g = gg.from_edges(3, [(0, 0, 2), (0, 1), (1, 2)])
    (rp, col, w), m = oracle.vertex_following(g.rowptr, g.col, g.w)
    assert len(rp) - 1 == 2 and list(m) == [0, 1, 1]
    # 2m is preserved
    for seed in range(4):
        g = gg.chunglu(2000, 2.1, 0.7, 6000, 50.0, seed=seed)
        (rp, col, w), m = oracle.vertex_following(g.rowptr, g.col, g.w)
        assert int(w.astype(np.int64).sum()) == g.two_m
        assert oracle.validate(rp, col, w)[0] == 0


@pytest.mark.parametrize("seed", range(4))
def test_vf_preserves_modularity_of_expanded_partition(seed):
    # VF is an exact coarsening (R2): Q of any partition of G' equals Q of the
    # partition of G obtained through the VF map.
    rng = np.random.default_rng(seed)
    g = gg.chunglu(300, 2.1, 0.7, 700, 30.0, seed=seed)
    (rp, col, w), m = oracle.vertex_following(g.rowptr, g.col, g.w)
    for _ in range(10):
        lab = rng.integers(0, 12, size=len(rp) - 1).astype(np.int32)
        assert oracle.modularity(rp, col, w, lab) == oracle.modularity(g.rowptr, g.col, g.w,
                                                                      lab[m])


def test_lemma3_fixed_point():
    # Lemma 3: at a no-move fixed point, a single-degree vertex i shares its
    # neighbour's community unless the singlet rule blocks the move (both
    # singletons and the neighbour's label larger).
    hits = 0
    for seed in range(6):
        g = gg.chunglu(400, 2.1, 0.75, 1500, 40.0, seed=seed)
        r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=1, color_cutoff=0,
                       theta_high=0.0, theta_low=-1e300, max_phases=1, max_iters=500, trace=1)
        p = r.phases[0]
        if r.iters[-1][2] != 0:
            continue  # did not reach a fixed point
        C = p.iter_labels[-1]
        size = np.bincount(C, minlength=g.n)
        for i in range(g.n):
            if g.rowptr[i + 1] - g.rowptr[i] == 1 and g.col[g.rowptr[i]] != i:
                j = int(g.col[g.rowptr[i]])
                if C[i] != C[j]:
                    assert size[C[i]] == 1 and size[C[j]] == 1 and C[j] > C[i]
                hits += 1
    assert hits > 50


# ------------------------------------------------------- brute force n<=10
def _set_partitions(n):
    # restricted growth strings
    a = [0] * n

    def rec(i, mx):
        if i == n:
            yield list(a)
            return
        for v in range(mx + 2):
            a[i] = v
            yield from rec(i + 1, max(mx, v))
    if n == 0:
        yield []
        return
    a[0] = 0
    yield from rec(1, 0)


def _brute_best_q(g):
    P = np.array(list(_set_partitions(g.n)), dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    k = np.bincount(src, weights=g.w, minlength=g.n).astype(np.int64)
    two_m = int(k.sum())
    intra = (P[:, src] == P[:, g.col]).astype(np.int64) @ g.w.astype(np.int64)
    onehot = np.zeros((P.shape[0], g.n), dtype=np.int64)
    for v in range(g.n):
        onehot[np.arange(P.shape[0]), P[:, v]] += k[v]
    N = two_m * intra - (onehot ** 2).sum(axis=1)
    best = int(N.max())
    return Fraction(best, two_m * two_m), P[int(N.argmax())]


@pytest.mark.parametrize("name", GOLDEN_Q)
def test_bruteforce_optimum_worked_cases(golden, name):
    fx = golden(name)
    g = _g(fx)
    best, _ = _brute_best_q(g)
    assert best == fx["q"]  # the hand partition is optimal
    for vf, col in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        r = oracle.run(g.rowptr, g.col, g.w, vertex_following=vf, coloring=col, color_cutoff=0)
        q = Fraction(r.phases[-1].N_end, r.two_m ** 2)
        assert q <= best
        assert q == best, (vf, col, q)


@pytest.mark.parametrize("seed", range(10))
def test_bruteforce_upper_bound(seed):
    n = 6 + seed % 4
    g = gg.random_graph(n, 0.45, wmax=4, loops=0.2, seed=300 + seed)
    if g.two_m == 0:
        return
    best, _ = _brute_best_q(g)
    for vf, col in [(0, 0), (1, 1)]:
        r = oracle.run(g.rowptr, g.col, g.w, vertex_following=vf, coloring=col, color_cutoff=0)
        assert Fraction(r.phases[-1].N_end, r.two_m ** 2) <= best


# ------------------------------------------------------------- invariants
def _independent_greedy_colouring(g, seed, order=0):
    # Plain restatement in Python: decreasing (neighbours other than v,
    # h(v^seed), v) -- or (h(v^seed), v) for order 1 -- smallest free colour.
    M = (1 << 64) - 1

    def h(x):
        x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M
        x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M
        return x ^ (x >> 31)

    def d(v):
        return 0 if order == 1 else sum(1 for u in g.col[g.rowptr[v]:g.rowptr[v + 1]] if u != v)
    order = sorted(range(g.n), key=lambda v: (d(v), h(v ^ seed), v), reverse=True)
    col = [-1] * g.n
    for v in order:
        used = {col[u] for u in g.col[g.rowptr[v]:g.rowptr[v + 1]] if u != v and col[u] >= 0}
        c = 0
        while c in used:
            c += 1
        col[v] = c
    return col


def _core_first_colouring(g, seed, T):
    # The GPU's schedule restated in Python: the vertices with at least T
    # neighbours other than themselves, in decreasing priority, each taking
    # the smallest colour free among its coloured neighbours; then rounds
    # over the others (a vertex is ready once its higher-priority neighbours
    # are coloured; a round colours all ready vertices at once).
    M = (1 << 64) - 1

    def h(x):
        x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M
        x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M
        return x ^ (x >> 31)

    nb = [[u for u in g.col[g.rowptr[v]:g.rowptr[v + 1]] if u != v] for v in range(g.n)]
    pr = [(len(nb[v]), h(v ^ seed), v) for v in range(g.n)]
    higher = [[u for u in nb[v] if pr[u] > pr[v]] for v in range(g.n)]
    col = [-1] * g.n

    def mex(v):
        used = {col[u] for u in higher[v]}
        c = 0
        while c in used:
            c += 1
        return c

    core = sorted((v for v in range(g.n) if len(nb[v]) >= T), key=lambda v: pr[v], reverse=True)
    incore = set(core)
    for v in core:
        assert all(u in incore for u in higher[v])  # the core is a prefix of the order
        assert all(col[u] >= 0 for u in higher[v])
        col[v] = mex(v)
    rest = [v for v in range(g.n) if v not in incore]
    rounds = 0
    while rest:
        ready = [v for v in rest if all(col[u] >= 0 for u in higher[v])]
        assert ready
        for v in ready:
            col[v] = mex(v)
        done = set(ready)
        rest = [v for v in rest if v not in done]
        rounds += 1
    return col, rounds


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("T", [2, 8, 32, 1 << 20])
def test_core_first_schedule_gives_the_oracle_colouring(seed, T):
    """Colouring a degree core first (without rounds) and the rest by rounds
    gives the colouring of the priority order: the largest-degree-first
    priority makes the core a prefix of that order."""
    g = gg.rmat(9, 8, seed=40 + seed)
    K, c = oracle.color(g.rowptr, g.col, 91 + seed, 0)
    got, rounds = _core_first_colouring(g, 91 + seed, T)
    assert got == list(c)
    if T == 2:  # nearly everything in the core: few rounds remain
        assert rounds <= 3


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("order", [0, 1])
def test_colouring_matches_independent_greedy(seed, order):
    g = gg.rmat(9, 8, seed=seed)
    K, c = oracle.color(g.rowptr, g.col, 77 + seed, order)
    ref = _independent_greedy_colouring(g, 77 + seed, order)
    assert list(c) == ref and K == max(ref) + 1
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    off = src != g.col
    assert np.all(c[src[off]] != c[g.col[off]])  # proper


@pytest.mark.parametrize("wl", ["planted1k", "rmat_small", "chunglu_small"])
def test_phase_invariants(wl):
    if wl == "planted1k":
        g, prm = gg.workload("planted1k")
    elif wl == "rmat_small":
        g = gg.rmat(12, 8, seed=5)
        prm = dict(vertex_following=1, coloring=1, theta_low=1e-6, theta_high=1e-2,
                   color_cutoff=500)
    else:
        g = gg.chunglu(5000, 2.1, 0.7, 20000, 200.0, seed=6)
        prm = dict(vertex_following=1, coloring=1, theta_low=1e-6, theta_high=1e-2,
                   color_cutoff=1000)
    r = oracle.run(g.rowptr, g.col, g.w, trace=1, **prm)
    assert r.two_m == g.two_m
    prev_end = None
    for pi, p in enumerate(r.phases):
        rp, col, w = p.graph
        assert oracle.validate(rp, col, w) == (0, g.two_m)  # m preserved, CSR valid
        if prev_end is not None:
            assert p.N_start == prev_end  # singleton Q of G_{p+1} == final Q of G_p
        for lab in p.iter_labels:
            assert lab.min() >= 0 and lab.max() < p.n
        # labels of original vertices: valid partition into n_next communities
        assert set(np.unique(p.labels)) == set(range(p.n_next))
        # Q on the phase graph equals Q of the composed labels on the input graph
        N, _ = oracle.modularity_num(g.rowptr, g.col, g.w, p.labels)
        assert N == p.N_end
        assert -0.5 <= p.q < 1
        if p.colored:
            assert list(p.colors) == _independent_greedy_colouring(
                type(g)(p.n, rp, col, w), 0x5EED + pi)
        prev_end = p.N_end
    # recorded per-iteration numerators are the modularity of the labels
    for ph, it, moved, N, _ in r.iters:
        p = r.phases[ph]
        Nchk, _ = oracle.modularity_num(*p.graph, p.iter_labels[it - 1])
        assert Nchk == N


def test_rebuild_matches_definition():
    rng = np.random.default_rng(9)
    g = gg.random_graph(40, 0.15, wmax=6, loops=0.3, seed=9)
    lab = rng.integers(0, 7, size=g.n).astype(np.int32)
    rp, col, w = oracle.rebuild(g.rowptr, g.col, g.w, lab)
    used = sorted(set(lab.tolist()))
    nid = {c: i for i, c in enumerate(used)}
    W = {}
    for u in range(g.n):
        for e in range(g.rowptr[u], g.rowptr[u + 1]):
            key = (nid[int(lab[u])], nid[int(lab[g.col[e]])])
            W[key] = W.get(key, 0) + int(g.w[e])
    got = {}
    for c in range(len(rp) - 1):
        for e in range(rp[c], rp[c + 1]):
            got[(c, int(col[e]))] = int(w[e])
        assert list(col[rp[c]:rp[c + 1]]) == sorted(col[rp[c]:rp[c + 1]])
    assert got == W
    # coarsening keeps Q of the induced partition: singletons of the coarse graph
    N1, _ = oracle.modularity_num(rp, col, w, np.arange(len(rp) - 1))
    N0, _ = oracle.modularity_num(g.rowptr, g.col, g.w, lab)
    assert N0 == N1


# --------------------------------------------------------------- boundary
def test_validation_codes():
    ok = gg.from_edges(3, [(0, 1), (1, 2)])
    assert oracle.validate(ok.rowptr, ok.col, ok.w) == (0, 4)
    rp, col, w = ok.rowptr.copy(), ok.col.copy(), ok.w.copy()
    w2 = w.copy(); w2[0] = 0
    assert oracle.validate(rp, col, w2)[0] == -3  # weight
    w3 = w.copy(); w3[0] = 2
    assert oracle.validate(rp, col, w3)[0] == -2  # asymmetric weight
    col2 = col.copy(); col2[1] = 7
    assert oracle.validate(rp, col2, w)[0] == -1  # column out of range
    g = gg.from_edges(3, [(0, 1), (0, 2)])
    col3 = g.col.copy(); col3[0], col3[1] = col3[1], col3[0]
    assert oracle.validate(g.rowptr, col3, g.w)[0] == -1  # unsorted
    col4 = g.col.copy(); col4[1] = col4[0]
    assert oracle.validate(g.rowptr, col4, g.w)[0] == -4  # duplicate
    e = gg.from_edges(3, [])
    assert oracle.validate(e.rowptr, e.col, e.w)[0] == -6  # empty
    big = gg.from_edges(2, [(0, 1, 2 ** 30)])
    assert oracle.validate(big.rowptr, big.col, big.w)[0] == -5  # 2m >= 2^31
    bad = np.array([0, 2, 1, 2], dtype=np.int64)
    assert oracle.validate(bad, ok.col, ok.w)[0] == -1  # decreasing rowptr
    with pytest.raises(oracle.OracleError):
        oracle.run(e.rowptr, e.col, e.w)


def test_isolated_vertices_stay():
    g = gg.from_edges(8, [(0, 1), (1, 2), (0, 2), (5, 6, 2)])
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0)
    lab = r.final_labels
    assert len({lab[3], lab[4], lab[7]}) == 3
    assert lab[0] == lab[1] == lab[2] and lab[5] == lab[6]


# --------------------------------------------------------------------------
# Heuristic variants of the Sec. 5 experiments and the qualitative comparison
# --------------------------------------------------------------------------
def test_compare_hand_example():
    # pairs of {0,1,2,3} under s = {01|23}, p = {012|3}: TP {01}; FP {02},{12};
    # FN {23}; TN {03},{13}
    c = oracle.compare([0, 0, 1, 1], [5, 5, 5, 7])
    assert (c["tp"], c["fp"], c["fn"], c["tn"]) == (1, 2, 1, 2)
    assert c["sp"] == 1 / 3 and c["se"] == 1 / 2 and c["oq"] == 1 / 4 and c["rand"] == 1 / 2


def test_compare_identical_and_symmetric():
    rng = np.random.default_rng(3)
    s = rng.integers(0, 7, size=60)
    perm = rng.permutation(7)
    c = oracle.compare(s, perm[s])  # same partition under other labels
    assert c["fp"] == c["fn"] == 0 and c["sp"] == c["se"] == c["oq"] == c["rand"] == 1.0
    p = rng.integers(0, 5, size=60)
    a, b = oracle.compare(s, p), oracle.compare(p, s)
    assert (a["tp"], a["fp"], a["fn"], a["tn"]) == (b["tp"], b["fn"], b["fp"], b["tn"])
    assert a["tp"] + a["fp"] + a["fn"] + a["tn"] == 60 * 59 // 2


def test_compare_matches_contingency_counts():
    # independent route: TP = sum over the contingency table of C(n_ij, 2)
    rng = np.random.default_rng(4)
    s = rng.integers(0, 9, size=300)
    p = rng.integers(0, 4, size=300) + 3 * (s % 3)
    c = oracle.compare(s, p)
    pairs = lambda x: int((x * (x - 1) // 2).sum())
    _, nij = np.unique(np.stack([s, p], 1), axis=0, return_counts=True)
    _, ni = np.unique(s, return_counts=True)
    _, nj = np.unique(p, return_counts=True)
    tp = pairs(nij)
    assert c["tp"] == tp and c["fn"] == pairs(ni) - tp and c["fp"] == pairs(nj) - tp
    sk = pytest.importorskip("sklearn.metrics")
    assert abs(c["rand"] - sk.rand_score(s, p)) < 1e-12


def test_absolute_threshold_two_cycles_on_planted1k():
    # R9: with |N_C - N_P| the synchronous uncoloured sweep of the 1,000-vertex
    # planted graph falls into a 2-cycle and only the max_iters guard ends it;
    # the signed test stops it
    g, _ = gg.workload("planted1k")
    signed = oracle.run(g.rowptr, g.col, g.w, coloring=0, max_iters=40)
    absm = oracle.run(g.rowptr, g.col, g.w, coloring=0, max_iters=40, abs_threshold=1)
    assert signed.phases[0].iterations < 40
    assert absm.phases[0].iterations == 40
    # the cycle: labels two iterations apart agree, consecutive ones differ
    tr = oracle.run(g.rowptr, g.col, g.w, coloring=0, max_iters=40, abs_threshold=1, trace=1,
                    max_phases=1)
    it = tr.phases[0].iter_labels
    assert np.array_equal(it[-1], it[-3]) and not np.array_equal(it[-1], it[-2])


def test_colour_first_phase_only():
    g = gg.rmat(12, 12, seed=9)
    full = oracle.run(g.rowptr, g.col, g.w, color_cutoff=0, theta_high=0.0)
    first = oracle.run(g.rowptr, g.col, g.w, color_cutoff=0, theta_high=0.0, color_phases=1)
    assert [p.colored for p in full.phases][:2] == [True, True]
    assert first.phases[0].colored and not any(p.colored for p in first.phases[1:])
    # phase 0 is the same run in both
    assert np.array_equal(full.phases[0].labels, first.phases[0].labels)
    assert full.phases[0].N_end == first.phases[0].N_end


# ------------------------------------------- Sec. 4.3: recursive VF reading
def _lemma3_mergeable(rp, col, w, two_m):
    """Single-neighbour vertices i (one neighbour j != i, optional self-loop)
    whose Lemma 3 lower bound stays positive for any community of j:
    2m * w(i, j) > k_i * (2m - k_i), the largest a_C(j) being 2m - k_i."""
    out = []
    for i in range(len(rp) - 1):
        c, ww = col[rp[i]:rp[i + 1]], w[rp[i]:rp[i + 1]]
        other = c != i
        if other.sum() == 1:
            k = int(ww.sum())
            if two_m * int(ww[other][0]) > k * (two_m - k):
                out.append(i)
    return out


@pytest.mark.parametrize("make", [lambda: gg.rmat(14, 16, seed=2),
                                  lambda: gg.chunglu(4000, 2.1, 0.7, 16000, 300.0, seed=7),
                                  lambda: gg.random_graph(300, 0.01, wmax=5, loops=0.1, seed=3)])
def test_recursive_vf_stops_at_single_degree(make):
    """Extending VF to single-neighbour vertices (Sec. 4.3's recursive idea)
    under Lemma 3's own bound merges nothing more on these graphs: after VF
    every single-neighbour vertex carries a self-loop, and the bound fails
    unless its degree is a large share of 2m."""
    g = make()
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, trace=1, max_phases=1)
    rp, col, w = r.phases[0].graph
    single = sum(1 for i in range(len(rp) - 1) if (col[rp[i]:rp[i + 1]] != i).sum() == 1)
    assert single > 0 or len(rp) < 500
    assert _lemma3_mergeable(rp, col, w, r.two_m) == []
    # the bound holds for every single-degree vertex (plain VF: vertex 2) and
    # for a looped one when its pair dominates the graph (vertex 0)
    h = gg.from_edges(3, [(0, 0, 100), (0, 1, 50), (1, 2, 1)])
    assert _lemma3_mergeable(h.rowptr, h.col, h.w, int(h.w.sum())) == [0, 2]


# ------------------------------------ R3, R12, R14: survivor, thresholds, order
def test_vf_isolated_edge_keeps_the_larger_end():
    """R3: of an isolated edge the smaller id is removed into the larger.
    Triangle 0-2-4 and isolated edge 1-3: vertex 1 goes into 3, the survivors
    0, 2, 3, 4 become 0, 1, 2, 3, and 3 carries the self-loop 2 * w(1, 3)."""
    g = gg.from_edges(5, [(0, 2, 1), (2, 4, 1), (0, 4, 1), (1, 3, 1)])
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, trace=1)
    assert list(r.vf_map) == [0, 2, 1, 2, 3]
    rp, col, w = r.phases[0].graph
    assert list(rp) == [0, 2, 4, 5, 7]
    assert list(col) == [1, 3, 0, 3, 2, 0, 1]
    assert list(w) == [1, 1, 1, 1, 2, 1, 1]


def _coarse_by_definition(rp, col, w, labels):
    """Sec. 4.5: one vertex per non-empty community in ascending label (R14);
    every arc (u, v, w) becomes (c'(u), c'(v), w) and equal pairs are summed."""
    _, inv = np.unique(labels, return_inverse=True)
    u = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    cu, cv = inv[u], inv[col]
    key = cu.astype(np.int64) * (inv.max() + 1) + cv
    order = np.argsort(key, kind="stable")
    k_sorted, w_sorted = key[order], w[order].astype(np.int64)
    uk, start = np.unique(k_sorted, return_index=True)
    ws = np.add.reduceat(w_sorted, start)
    nn = inv.max() + 1
    rows = uk // nn
    rp2 = np.zeros(nn + 1, dtype=np.int64)
    np.add.at(rp2, rows + 1, 1)
    return np.cumsum(rp2), (uk % nn).astype(np.int32), ws.astype(np.int32)


@pytest.mark.parametrize("make", [lambda: gg.planted(1000, 10, 0.1, 0.002, 1, 1, seed=1),
                                  lambda: gg.random_graph(300, 0.02, wmax=5, loops=0.2, seed=4),
                                  lambda: gg.rmat(10, 8, seed=5)])
def test_rebuild_matches_definition(make):
    """Every phase graph equals the coarse graph of the previous phase's last
    labels, built here with numpy straight from the definition."""
    g = make()
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0, trace=1)
    assert len(r.phases) >= 2
    for a, b in zip(r.phases, r.phases[1:]):
        rp, col, w = a.graph
        want = _coarse_by_definition(rp, col, w, a.iter_labels[-1])
        got = b.graph
        for x, y in zip(want, got):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def _stop_rule_holds(r, theta_high, theta_low, cutoff, max_iters=10_000):
    """R9, R10, R12, R13 checked on the recorded numerators: every phase ends
    at the first iteration that moves nothing, gains less than theta times
    |N| of the iteration before (signed, from the second iteration), or hits
    max_iters; a phase colours iff n_p >= cutoff and no earlier coloured
    phase gained less than theta_high relative to its start."""
    colour_stopped = False
    for p, ph in enumerate(r.phases):
        its = [t for t in r.iters if t[0] == p]
        assert ph.colored == (ph.n >= cutoff and not colour_stopped), p
        theta = theta_high if ph.colored else theta_low
        prev = None
        for t, (_, it, moved, N, _) in enumerate(its, start=1):
            stop = moved == 0 or (prev is not None and N - prev < theta * abs(prev)) or t >= max_iters
            assert stop == (t == len(its)), (p, t)
            prev = N
        if ph.colored and ph.N_end - ph.N_start < theta_high * abs(ph.N_start):
            colour_stopped = True


@pytest.mark.parametrize("make", [lambda: gg.rmat(12, 16, seed=6),
                                  lambda: gg.planted(3000, 30, 0.02, 0.001, 1, 4, seed=8)])
def test_stop_rules_on_recorded_numerators(make):
    g = make()
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=1, color_cutoff=500,
                   theta_high=1e-2, theta_low=1e-6)
    assert any(p.colored for p in r.phases)
    _stop_rule_holds(r, 1e-2, 1e-6, 500)


def test_sweep_sample_is_the_first_iteration():
    """The oracle's timing sample over every vertex is the first uncoloured
    iteration of its own run (same moves, every arc scanned once)."""
    g = gg.rmat(12, 16, seed=2)
    mv, vis, sec = oracle.sweep_sample(g.rowptr, g.col, g.w, 0, g.n)
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=0, coloring=0, max_iters=1,
                   max_phases=1)
    assert mv == r.iters[0][2] and vis == g.arcs and sec >= 0.0
    mv2, vis2, _ = oracle.sweep_sample(g.rowptr, g.col, g.w, 100, 50)
    assert vis2 == int(g.rowptr[150] - g.rowptr[100]) and 0 <= mv2 <= 50


# ------------------------- Sec. 4.3 closing paragraph: recursive VF (R23)
def test_recursive_vf_fixtures():
    """Hand-derived merges of the recursive single-neighbour rounds.

    Looped pair: edges (0,0,100), (0,1,50), (1,2,1), 2m = 202.  Plain VF
    removes vertex 2 into 1 (loop 2).  Then vertex 0 (loop 100, w 50, k 150)
    passes k^2 = 22500 > 2m l = 20200, and vertex 1 (loop 2, w 50, k 52)
    passes 2704 > 404: two single-neighbour vertices facing each other, so
    the smaller (0) merges into 1 and one vertex is left.

    Weighted path (0,1,8), (1,2,8), (2,3,1), 2m = 34: plain VF removes 0
    into 1 (loop 16) and 3 into 2 (loop 2); then 1 (k 24: 576 > 544) and 2
    (k 10: 100 > 68) pass towards each other and 1 merges into 2.

    Unweighted path of 6 vertices: after plain VF the ends carry loop 2 with
    w 1 (k 3: 9 > 2m l = 20 fails), so nothing more merges."""
    g = gg.from_edges(3, [(0, 0, 100), (0, 1, 50), (1, 2, 1)])
    a = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0)
    b = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1)
    assert a.vf_n == 2 and list(a.vf_map) == [0, 1, 1]
    assert b.vf_n == 1 and list(b.vf_map) == [0, 0, 0]
    g = gg.from_edges(4, [(0, 1, 8), (1, 2, 8), (2, 3, 1)])
    b = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1,
                   trace=1)
    assert b.vf_n == 1 and list(b.vf_map) == [0, 0, 0, 0]
    rp, col, w = b.phases[0].graph
    assert list(rp) == [0, 1] and list(col) == [0] and list(w) == [34]
    g = gg.from_edges(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)])
    a = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0)
    b = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1)
    assert b.vf_n == a.vf_n == 4 and list(b.vf_map) == list(a.vf_map)
    # a looped pair 1-5 (w 50, loops 3) beside a 0-2-3-4 block, 2m = 116:
    # both pass (53^2 = 2809 > 348), so 1 merges into 5 (R3) and the
    # survivors 0, 2, 3, 4, 5 become 0..4
    g = gg.from_edges(6, [(0, 2), (2, 3), (0, 3), (3, 4), (2, 4), (1, 5, 50), (1, 1, 3),
                          (5, 5, 3)])
    b = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1)
    assert list(b.vf_map) == [0, 4, 1, 2, 3, 4]


def _pendant_graph(seed):
    """A core where every vertex keeps >= 2 core neighbours, plus looped
    pendants (one core neighbour each), so plain VF merges nothing and the
    first recursive round decides every pendant on its own."""
    rng = np.random.default_rng(seed)
    nc, npd = 8, 5
    edges = [(i, (i + 1) % nc, int(rng.integers(1, 6))) for i in range(nc)]
    for i in range(nc):
        for j in range(i + 2, nc):
            if rng.random() < 0.3 and not (i == 0 and j == nc - 1):
                edges.append((i, j, int(rng.integers(1, 6))))
    pend = []
    for t in range(npd):
        p, j = nc + t, int(rng.integers(0, nc))
        edges.append((p, j, int(rng.integers(1, 31))))
        edges.append((p, p, int(rng.integers(1, 7))))
        pend.append((p, j))
    return gg.from_edges(nc + npd, edges), pend


@pytest.mark.parametrize("seed", range(12))
def test_recursive_vf_is_lemma3_guarantee(seed):
    """A pendant merges iff Lemma 3's guarantee holds for it: when merged,
    its exact gain (Eq. 4) towards C(j) is positive for random partitions
    with it alone; when kept, the partition {i} | everything else (where
    a_C(j) = 2m - k_i, the bound's worst case) gives a gain <= 0."""
    g, pend = _pendant_graph(seed)
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1,
                   max_phases=1, max_iters=1)
    rng = np.random.default_rng(100 + seed)
    n = g.n
    for p, j in pend:
        merged = r.vf_map[p] == r.vf_map[j]
        if merged:
            for _ in range(30):
                lab = rng.integers(0, 4, size=n).astype(np.int32)
                lab[p] = 4  # alone
                assert oracle.gain(g.rowptr, g.col, g.w, lab, p, int(lab[j])) > 0
        else:
            lab = np.zeros(n, dtype=np.int32)
            lab[p] = 1
            assert oracle.gain(g.rowptr, g.col, g.w, lab, p, 0) <= 0


def test_recursive_vf_cases_cover_both_outcomes():
    """The seeds above include pendants that merge and pendants that stay."""
    seen = 0
    for seed in range(12):
        g, pend = _pendant_graph(seed)
        r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1,
                       max_phases=1, max_iters=1)
        for p, j in pend:
            seen |= 1 if r.vf_map[p] == r.vf_map[j] else 2
    assert seen == 3


@pytest.mark.parametrize("make", [lambda: _pendant_graph(3)[0],
                                  lambda: gg.random_graph(200, 0.02, wmax=9, loops=0.3, seed=8),
                                  lambda: gg.from_edges(4, [(0, 1, 8), (1, 2, 8), (2, 3, 1)])])
def test_recursive_vf_is_an_exact_coarsening(make):
    """Like plain VF (R1, R2): Q of any partition of the merged graph equals
    Q of the expanded partition on the input graph."""
    g = make()
    r = oracle.run(g.rowptr, g.col, g.w, vertex_following=1, coloring=0, vf_recursive=1,
                   trace=1, max_phases=1, max_iters=1)
    rp, col, w = r.phases[0].graph
    rng = np.random.default_rng(1)
    for _ in range(10):
        lab = rng.integers(0, max(1, (len(rp) - 1) // 2), size=len(rp) - 1).astype(np.int32)
        N1, t1 = oracle.modularity_num(rp, col, w, lab)
        N0, t0 = oracle.modularity_num(g.rowptr, g.col, g.w, lab[r.vf_map])
        assert (N1, t1) == (N0, t0)
