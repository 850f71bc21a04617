"""Seeded synthetic graph generators shared by the tests, the bench and the oracle.

This module only produces inputs: symmetric CSR graphs with integer weights
(rows sorted ascending, duplicates merged, each undirected edge stored in both
rows, a self-loop stored once).  It holds none of the community-detection
arithmetic, so both the CUDA path and the serial oracle may consume what it
makes.

The heavy lifting is in ``graphgen.c`` (built with gcc by :func:`build`).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to the source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        i64, i32, f64, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
        lib.gg_planted.restype = vp
        lib.gg_planted.argtypes = [i64, i32, f64, f64, i32, i32, u64]
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [i32, i64, f64, f64, f64, u64]
        lib.gg_chunglu.restype = vp
        lib.gg_chunglu.argtypes = [i64, f64, f64, i64, f64, u64]
        lib.gg_from_edges.restype = vp
        lib.gg_from_edges.argtypes = [i64, i64, vp, vp, vp]
        lib.gg_size.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.gg_stats.argtypes = [vp] + [ctypes.POINTER(i64)] * 3
        lib.gg_copy.argtypes = [vp, vp, vp, vp]
        lib.gg_free.argtypes = [vp]
        lib.gg_set_threads.argtypes = [i32]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Symmetric CSR: ``rowptr`` int64[n+1], ``col`` int32[arcs], ``w`` int32[arcs]."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""
    stats: dict = field(default_factory=dict)

    @property
    def arcs(self) -> int:
        return int(self.rowptr[-1])

    @property
    def two_m(self) -> int:
        return int(self.w.astype(np.int64).sum())

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _take(h, name: str) -> Graph:
    if not h:
        raise ValueError(f"generator {name}: invalid arguments")
    lib = _load()
    n, a = ctypes.c_int64(), ctypes.c_int64()
    lib.gg_size(h, ctypes.byref(n), ctypes.byref(a))
    rowptr = np.empty(n.value + 1, dtype=np.int64)
    col = np.empty(max(a.value, 0), dtype=np.int32)
    w = np.empty(max(a.value, 0), dtype=np.int32)
    lib.gg_copy(h, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data)
    d, s, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib.gg_stats(h, ctypes.byref(d), ctypes.byref(s), ctypes.byref(m))
    lib.gg_free(h)
    return Graph(int(n.value), rowptr, col, w, name,
                 {"draws": d.value, "self_draws": s.value, "dup_merged": m.value})


def planted(n: int, blocks: int, p_in: float, p_out: float, wmin: int = 1, wmax: int = 1,
            seed: int = 1) -> Graph:
    """Planted partition: ``blocks`` contiguous near-equal blocks, independent
    pairs with probability ``p_in`` inside a block and ``p_out`` across."""
    lib = _load()
    return _take(lib.gg_planted(n, blocks, p_in, p_out, wmin, wmax, seed),
                 f"planted(n={n},B={blocks},seed={seed})")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2) -> Graph:
    """R-MAT with ``edge_factor * 2**scale`` draws; self draws dropped,
    duplicates merged into integer weights (multiplicity)."""
    lib = _load()
    draws = edge_factor * (1 << scale)
    return _take(lib.gg_rmat(scale, draws, a, b, c, seed), f"rmat(scale={scale},seed={seed})")


def chunglu(n: int, gamma: float = 2.1, core_frac: float = 0.7, edges: int = 250_000_000,
            dmax: float = 1.0e5, seed: int = 3) -> Graph:
    """Chung-Lu power-law core plus pendant (degree-1) layer, ids shuffled."""
    lib = _load()
    return _take(lib.gg_chunglu(n, gamma, core_frac, edges, dmax, seed),
                 f"chunglu(n={n},seed={seed})")


def from_edges(n: int, edges, name: str = "") -> Graph:
    """CSR from an undirected edge list of (u, v) or (u, v, w) tuples.
    Duplicate edges are summed; (u, u) is a self-loop stored once."""
    lib = _load()
    rows = [tuple(e) if len(e) == 3 else (e[0], e[1], 1) for e in edges]
    if not rows:
        return _empty(n)
    arr = np.asarray(rows, dtype=np.int64)
    u = np.ascontiguousarray(arr[:, 0], dtype=np.int32)
    v = np.ascontiguousarray(arr[:, 1], dtype=np.int32)
    w = np.ascontiguousarray(arr[:, 2], dtype=np.int32)
    h = lib.gg_from_edges(n, len(u), u.ctypes.data, v.ctypes.data, w.ctypes.data)
    return _take(h, name or f"edges(n={n})")


def random_graph(n: int, p: float, wmax: int = 1, loops: float = 0.0, seed: int = 0) -> Graph:
    """Small Erdos-Renyi-style test graph with weights in [1, wmax] and each
    vertex given a self-loop with probability ``loops`` (numpy generator)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    iu, ju = iu[keep], ju[keep]
    ww = rng.integers(1, wmax + 1, size=iu.shape[0])
    edges = list(zip(iu.tolist(), ju.tolist(), ww.tolist()))
    if loops > 0:
        for v in np.nonzero(rng.random(n) < loops)[0].tolist():
            edges.append((v, v, int(rng.integers(1, wmax + 1))))
    if not edges:
        return _empty(n)
    return from_edges(n, edges, name=f"random(n={n},p={p},seed={seed})")


def _empty(n: int) -> Graph:
    return Graph(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                 np.zeros(0, dtype=np.int32), f"empty(n={n})")


# ----------------------------------------------------------------------------
# Named workloads.  Each entry gives the generator recipe and the heuristic
# switches it is run with (vertex following, colouring, threshold schedule).
# ----------------------------------------------------------------------------
WORKLOADS = {
    # 1,000 vertices in 10 blocks of 100, p_in 0.1, p_out 0.002, weight 1
    "planted1k": dict(gen=lambda: planted(1000, 10, 0.1, 0.002, 1, 1, seed=1),
                      params=dict(vertex_following=1, coloring=0, theta_low=1e-6,
                                  theta_high=0.0, color_cutoff=100_000)),
    # R-MAT scale 20, edge factor 16, (0.57, 0.19, 0.19, 0.05)
    "rmat20": dict(gen=lambda: rmat(20, 16, 0.57, 0.19, 0.19, seed=2),
                   params=dict(vertex_following=1, coloring=1, theta_low=1e-6,
                               theta_high=1e-2, color_cutoff=100_000)),
    # Chung-Lu, 2^24 vertices, exponent 2.1, 30% pendant, ~2.5e8 edges
    "chunglu24": dict(gen=lambda: chunglu(1 << 24, 2.1, 0.7, 250_000_000, 1.0e5, seed=3),
                      params=dict(vertex_following=1, coloring=1, theta_low=1e-6,
                                  theta_high=1e-2, color_cutoff=100_000)),
    # smaller members of the same families, for parity tests and ncu captures
    "rmat16": dict(gen=lambda: rmat(16, 16, 0.57, 0.19, 0.19, seed=2),
                   params=dict(vertex_following=1, coloring=1, theta_low=1e-6,
                               theta_high=1e-2, color_cutoff=10_000)),
    "chunglu20": dict(gen=lambda: chunglu(1 << 20, 2.1, 0.7, 15_000_000, 1.0e4, seed=3),
                      params=dict(vertex_following=1, coloring=1, theta_low=1e-6,
                                  theta_high=1e-2, color_cutoff=100_000)),
}


def workload(name: str):
    """Return (Graph, run-parameter dict) for a named workload."""
    wl = WORKLOADS[name]
    g = wl["gen"]()
    g.name = name
    return g, dict(wl["params"])


# ----------------------------------------------------------------------------
# Batches of graphs: a disjoint union stored as one CSR plus vertex offsets.
# ----------------------------------------------------------------------------
@dataclass
class Batch:
    """``num_graphs`` graphs; graph g owns vertices [gptr[g], gptr[g+1]) of the
    union CSR (rowptr, col, w), and its arcs stay inside that range."""

    gptr: np.ndarray
    rowptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""

    @property
    def num_graphs(self) -> int:
        return len(self.gptr) - 1

    @property
    def n(self) -> int:
        return int(self.gptr[-1])

    @property
    def arcs(self) -> int:
        return int(self.rowptr[-1])

    def graph(self, g: int) -> Graph:
        """Graph g alone, with local vertex ids."""
        lo, hi = int(self.gptr[g]), int(self.gptr[g + 1])
        a0, a1 = int(self.rowptr[lo]), int(self.rowptr[hi])
        return Graph(hi - lo, self.rowptr[lo:hi + 1] - a0, self.col[a0:a1] - lo,
                     self.w[a0:a1].copy(), f"{self.name}[{g}]")


def concat(graphs: list, name: str = "") -> Batch:
    """Disjoint union of graphs (vertex ids shifted by the preceding sizes)."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    gptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=gptr[1:])
    arcs = np.array([g.arcs for g in graphs], dtype=np.int64)
    aoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(arcs, out=aoff[1:])
    rowptr = np.empty(int(gptr[-1]) + 1, dtype=np.int64)
    col = np.empty(int(aoff[-1]), dtype=np.int32)
    w = np.empty(int(aoff[-1]), dtype=np.int32)
    for i, g in enumerate(graphs):
        lo, hi = int(gptr[i]), int(gptr[i + 1])
        rowptr[lo:hi] = g.rowptr[:-1] + aoff[i]
        col[aoff[i]:aoff[i + 1]] = g.col + lo
        w[aoff[i]:aoff[i + 1]] = g.w
    rowptr[-1] = aoff[-1]
    return Batch(gptr, rowptr, col, w, name)


def planted_batch(num_graphs: int = 4096, nmin: int = 100, nmax: int = 50_000, bmin: int = 2,
                  bmax: int = 200, intra_deg: float = 12.0, inter_deg: float = 2.0, wmax: int = 8,
                  seed: int = 4) -> Batch:
    """Batch of planted-partition graphs: n log-uniform in [nmin, nmax], B
    uniform in [bmin, bmax] clipped so blocks have >= 3 vertices, p_in so the
    mean intra-block degree is intra_deg, p_out so the mean inter-block degree
    is inter_deg, weights uniform in [1, wmax].  Graph g uses seed
    (seed << 20) + g."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=num_graphs)).astype(np.int64)
    bs = rng.integers(bmin, bmax + 1, size=num_graphs)
    graphs = []
    for g in range(num_graphs):
        n = int(ns[g])
        b = int(min(bs[g], max(1, n // 3)))
        sz = n / b
        p_in = min(1.0, intra_deg / max(sz - 1.0, 1.0))
        p_out = min(1.0, inter_deg / max(n - sz, 1.0)) if b > 1 else 0.0
        graphs.append(planted(n, b, p_in, p_out, 1, wmax, seed=(seed << 20) + g))
    return concat(graphs, f"planted_batch({num_graphs},seed={seed})")


def _planted_degrees(n: int, b: int, intra_deg: float, inter_deg: float, wmax: int,
                     seed: int) -> Graph:
    """Planted partition with mean intra- and inter-block degrees given."""
    b = int(min(b, max(1, n // 3)))
    sz = n / b
    p_in = min(1.0, intra_deg / max(sz - 1.0, 1.0))
    p_out = min(1.0, inter_deg / max(n - sz, 1.0)) if b > 1 else 0.0
    return planted(n, b, p_in, p_out, 1, wmax, seed=seed)


def served_specs(num_requests: int = 200, rate: float = 200.0, seed: int = 5,
                 rmat_scales=(10, 20), rmat_ef=(8, 16), planted_n=(1_000, 1_000_000)):
    """Recipe of the request stream for serving: Poisson arrivals at ``rate``
    per second; each request is, with equal odds, an R-MAT graph (scale and
    edge factor uniform integers in the given ranges, (a,b,c) = (0.57, 0.19,
    0.19)) or a planted-partition graph (n log-uniform in ``planted_n``,
    2..200 blocks, mean intra-block degree 12, inter-block 2, weights 1..8).
    Returns a list of (arrival seconds, kind, parameters, seed); request i
    uses seed (seed << 20) + i."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=num_requests))
    out = []
    for i in range(num_requests):
        s = (seed << 20) + i
        if rng.random() < 0.5:
            sc = int(rng.integers(rmat_scales[0], rmat_scales[1] + 1))
            ef = int(rng.integers(rmat_ef[0], rmat_ef[1] + 1))
            out.append((float(arrivals[i]), "rmat", (sc, ef), s))
        else:
            n = int(np.exp(rng.uniform(np.log(planted_n[0]), np.log(planted_n[1]))))
            b = int(rng.integers(2, 201))
            out.append((float(arrivals[i]), "planted", (n, b), s))
    return out


def served_request(spec) -> Graph:
    """The graph of one request of :func:`served_specs`."""
    _, kind, prm, s = spec
    if kind == "rmat":
        return rmat(prm[0], prm[1], seed=s)
    return _planted_degrees(prm[0], prm[1], 12.0, 2.0, 8, s)


def served_stream(num_requests: int = 200, rate: float = 200.0, seed: int = 5,
                  rmat_scales=(10, 20), rmat_ef=(8, 16), planted_n=(1_000, 1_000_000),
                  workers: int = 0):
    """The request stream of :func:`served_specs` as a list of (arrival
    seconds, Graph).  ``workers`` > 1 generates that many requests side by
    side (each with a share of the cores); the graphs are the same."""
    specs = served_specs(num_requests, rate, seed, rmat_scales, rmat_ef, planted_n)
    if workers <= 1:
        return [(sp[0], served_request(sp)) for sp in specs]
    import concurrent.futures as cf
    lib = _load()
    share = max(1, (os.cpu_count() or 1) // workers)

    def one(sp):
        lib.gg_set_threads(share)
        return served_request(sp)

    # largest first, so the long R-MAT requests do not end up last
    order = sorted(range(len(specs)), key=lambda i: -_spec_cost(specs[i]))
    graphs = [None] * len(specs)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for i, g in zip(order, ex.map(one, [specs[i] for i in order])):
            graphs[i] = g
    return [(sp[0], g) for sp, g in zip(specs, graphs)]


def _spec_cost(spec) -> float:
    _, kind, prm, _ = spec
    return float(prm[1] << prm[0]) if kind == "rmat" else 14.0 * prm[0]
