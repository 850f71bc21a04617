"""Serial CPU oracle of the parallel Louvain method (arXiv 1410.1237).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline leg may import this package; the library itself never does.  The C
source ``lv_oracle.c`` is a plain, slow, exact restatement of the paper's
method (Eqs. 1-5, Algorithm 1, Secs. 4.1-4.5) and shares no code with the
CUDA path.  This module only marshals arguments (ctypes) and converts the
exact 128-bit numerators to Python integers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lv_oracle.c")
_LIB = os.path.join(_HERE, "liblv_oracle.so")
# tests that plant mistakes in a copy of the oracle point this at their build
_LIB_OVERRIDE = os.environ.get("LV_ORACLE_LIB")
_lib = None

STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_NOT_SYMMETRIC", -3: "ERR_WEIGHT",
          -4: "ERR_DUPLICATE", -5: "ERR_OVERFLOW", -6: "ERR_EMPTY", -8: "ERR_OOM",
          -10: "ERR_STATE"}

DEFAULTS = dict(vertex_following=1, coloring=1, theta_low=1e-6, theta_high=1e-2,
                color_cutoff=100_000, max_iters=10_000, max_phases=64, color_seed=0x5EED,
                trace=0, color_phases=0, abs_threshold=0, vf_recursive=0,
                color_order=0)


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code} ({STATUS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile ``liblv_oracle.so`` (gcc -O2, single-threaded by design)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared",
                               "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("vertex_following", ctypes.c_int32), ("coloring", ctypes.c_int32),
                ("theta_low", ctypes.c_double), ("theta_high", ctypes.c_double),
                ("color_cutoff", ctypes.c_int64), ("max_iters", ctypes.c_int32),
                ("max_phases", ctypes.c_int32), ("color_seed", ctypes.c_uint64),
                ("trace", ctypes.c_int32), ("color_phases", ctypes.c_int32),
                ("abs_threshold", ctypes.c_int32), ("vf_recursive", ctypes.c_int32),
                ("color_order", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        P = ctypes.POINTER
        L.orc_validate.restype = ctypes.c_int
        L.orc_validate.argtypes = [i64, vp, vp, vp, P(i64)]
        L.orc_modularity.restype = ctypes.c_int
        L.orc_modularity.argtypes = [i64, vp, vp, vp, vp, P(i64), P(u64), P(i64)]
        L.orc_gain.restype = ctypes.c_int
        L.orc_gain.argtypes = [i64, vp, vp, vp, vp, i32, i32, P(i64), P(u64)]
        L.orc_color.restype = i32
        L.orc_color.argtypes = [i64, vp, vp, u64, i32, vp]
        L.orc_rebuild.restype = ctypes.c_int
        L.orc_rebuild.argtypes = [i64, vp, vp, vp, vp, P(vp)]
        L.orc_vertex_following.restype = ctypes.c_int
        L.orc_vertex_following.argtypes = [i64, vp, vp, vp, vp, P(vp)]
        L.orc_graph_size.argtypes = [vp, P(i64), P(i64)]
        L.orc_graph_copy.argtypes = [vp, vp, vp, vp]
        L.orc_graph_free.argtypes = [vp]
        L.orc_run.restype = ctypes.c_int
        L.orc_run.argtypes = [i64, vp, vp, vp, P(_Params), P(vp)]
        L.orc_num_phases.restype = i32
        L.orc_num_phases.argtypes = [vp]
        L.orc_two_m.restype = i64
        L.orc_two_m.argtypes = [vp]
        L.orc_vf_n.restype = i64
        L.orc_vf_n.argtypes = [vp]
        L.orc_seconds_total.restype = ctypes.c_double
        L.orc_seconds_total.argtypes = [vp]
        L.orc_vf_map.argtypes = [vp, vp]
        L.orc_phase_info.restype = ctypes.c_int
        L.orc_phase_info.argtypes = [vp, i32, vp, vp, vp, vp]
        L.orc_phase_labels.restype = ctypes.c_int
        L.orc_phase_labels.argtypes = [vp, i32, vp]
        L.orc_phase_graph.restype = vp
        L.orc_phase_graph.argtypes = [vp, i32]
        L.orc_phase_colors.restype = ctypes.c_int
        L.orc_phase_colors.argtypes = [vp, i32, vp]
        L.orc_phase_iter_labels.restype = ctypes.c_int
        L.orc_phase_iter_labels.argtypes = [vp, i32, i32, vp]
        L.orc_num_iters.restype = i64
        L.orc_num_iters.argtypes = [vp]
        L.orc_iters.argtypes = [vp, vp, vp, vp, vp]
        L.orc_free.argtypes = [vp]
        L.orc_sweep_sample.restype = ctypes.c_int
        L.orc_sweep_sample.argtypes = [i64, vp, vp, vp, i64, i64, P(i64), P(i64),
                                       P(ctypes.c_double)]
        L.orc_compare.restype = ctypes.c_int
        L.orc_compare.argtypes = [i64, vp, vp, vp]
        _lib = L
    return _lib


def _csr(rowptr, col, w):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32) if w is not None else None
    return rowptr, col, w


def _i128(hi: int, lo: int) -> int:
    return (int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)


def _graph_out(h):
    L = _load()
    n, a = ctypes.c_int64(), ctypes.c_int64()
    L.orc_graph_size(h, ctypes.byref(n), ctypes.byref(a))
    rowptr = np.empty(n.value + 1, dtype=np.int64)
    col = np.empty(a.value, dtype=np.int32)
    w = np.empty(a.value, dtype=np.int32)
    L.orc_graph_copy(h, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data)
    return rowptr, col, w


# ----------------------------------------------------------------- functions
def validate(rowptr, col, w, n: int | None = None) -> tuple[int, int]:
    """Return (status, 2m) for a CSR per the problem statement of Sec. 2."""
    rowptr, col, w = _csr(rowptr, col, w)
    n = len(rowptr) - 1 if n is None else n
    tm = ctypes.c_int64()
    st = _load().orc_validate(n, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                              ctypes.byref(tm))
    return st, tm.value


def modularity_num(rowptr, col, w, labels) -> tuple[int, int]:
    """Exact (N, 2m) with Q = N / (2m)^2, Eq. 3 evaluated from scratch."""
    rowptr, col, w = _csr(rowptr, col, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    hi, lo, tm = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
    st = _load().orc_modularity(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data,
                                w.ctypes.data, labels.ctypes.data, ctypes.byref(hi),
                                ctypes.byref(lo), ctypes.byref(tm))
    if st:
        raise OracleError(st)
    return _i128(hi.value, lo.value), tm.value


def modularity(rowptr, col, w, labels) -> Fraction:
    N, tm = modularity_num(rowptr, col, w, labels)
    return Fraction(N, tm * tm)


def gain(rowptr, col, w, labels, i: int, c: int) -> int:
    """Exact integer gain G = dQ * (2m)^2 / 2 of moving i alone to c (Eq. 4)."""
    rowptr, col, w = _csr(rowptr, col, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    hi, lo = ctypes.c_int64(), ctypes.c_uint64()
    st = _load().orc_gain(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                          labels.ctypes.data, i, c, ctypes.byref(hi), ctypes.byref(lo))
    if st:
        raise OracleError(st)
    return _i128(hi.value, lo.value)


def color(rowptr, col, seed: int, order: int = 0) -> tuple[int, np.ndarray]:
    """Greedy distance-1 colouring in decreasing priority (R11): (degree,
    hash, id) for order 0, (hash, id) for order 1."""
    rowptr, col, _ = _csr(rowptr, col, None)
    n = len(rowptr) - 1
    out = np.empty(n, dtype=np.int32)
    K = _load().orc_color(n, rowptr.ctypes.data, col.ctypes.data, seed, order,
                          out.ctypes.data)
    return int(K), out


def vertex_following(rowptr, col, w):
    """VF preprocessing (Sec. 4.3): returns ((rowptr, col, w), map)."""
    rowptr, col, w = _csr(rowptr, col, w)
    n = len(rowptr) - 1
    m = np.empty(n, dtype=np.int32)
    h = ctypes.c_void_p()
    L = _load()
    L.orc_vertex_following(n, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                           m.ctypes.data, ctypes.byref(h))
    out = _graph_out(h)
    L.orc_graph_free(h)
    return out, m


def sweep_sample(rowptr, col, w, first: int, count: int) -> tuple[int, int, float]:
    """Timing sample for the host-core baseline: the oracle's sweep of
    vertices [first, first + count) as one class of an uncoloured first
    iteration from the singleton partition.  Returns (moves, arcs scanned,
    seconds of the sweep alone)."""
    rowptr, col, w = _csr(rowptr, col, w)
    mv, vis, sec = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    st = _load().orc_sweep_sample(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data,
                                  w.ctypes.data, first, count, ctypes.byref(mv),
                                  ctypes.byref(vis), ctypes.byref(sec))
    if st:
        raise OracleError(st)
    return mv.value, vis.value, sec.value


def rebuild(rowptr, col, w, labels):
    """Coarse graph of a partition (Sec. 4.5 i-iii); labels renumbered by
    ascending non-empty label."""
    rowptr, col, w = _csr(rowptr, col, w)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    h = ctypes.c_void_p()
    L = _load()
    st = L.orc_rebuild(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                       labels.ctypes.data, ctypes.byref(h))
    if st:
        raise OracleError(st)
    out = _graph_out(h)
    L.orc_graph_free(h)
    return out


@dataclass
class Phase:
    n: int
    arcs: int
    n_next: int
    colored: bool
    num_colors: int
    iterations: int
    two_m: int
    N_start: int
    N_end: int
    theta: float
    seconds: float
    labels: np.ndarray
    graph: tuple | None = None
    colors: np.ndarray | None = None
    iter_labels: list = field(default_factory=list)

    @property
    def q(self) -> float:
        return float(self.N_end) / float(self.two_m * self.two_m)


@dataclass
class Result:
    n: int
    two_m: int
    vf_n: int
    vf_map: np.ndarray
    phases: list
    iters: list  # (phase, iter, moved, N, seconds)
    seconds: float

    @property
    def final_labels(self) -> np.ndarray:
        return self.phases[-1].labels

    @property
    def q(self) -> float:
        return self.phases[-1].q


def compare(labels_s, labels_p) -> dict:
    """Qualitative comparison of two partitions (Sec. 5) by its plain
    definition over all vertex pairs: TP, FP, FN, TN and SP = TP/(TP+FP),
    SE = TP/(TP+FN), OQ = TP/(TP+FP+FN), Rand = (TP+TN)/all pairs (a ratio
    with a zero denominator is reported as 1)."""
    s = np.ascontiguousarray(labels_s, dtype=np.int32)
    p = np.ascontiguousarray(labels_p, dtype=np.int32)
    if s.shape != p.shape:
        raise ValueError("partitions of different sizes")
    out = np.zeros(4, dtype=np.uint64)
    st = _load().orc_compare(len(s), s.ctypes.data, p.ctypes.data, out.ctypes.data)
    if st:
        raise OracleError(st)
    tp, fp, fn, tn = (int(x) for x in out)

    def ratio(a, b):
        return a / b if b else 1.0
    return dict(tp=tp, fp=fp, fn=fn, tn=tn, sp=ratio(tp, tp + fp), se=ratio(tp, tp + fn),
                oq=ratio(tp, tp + fp + fn), rand=ratio(tp + tn, tp + fp + fn + tn))


def run(rowptr, col, w, **params) -> Result:
    """Full multi-phase run (Sec. 4.4 steps 1-4).  Raises OracleError on an
    invalid input."""
    prm = dict(DEFAULTS)
    prm.update(params)
    rowptr, col, w = _csr(rowptr, col, w)
    n = len(rowptr) - 1
    L = _load()
    p = _Params(int(prm["vertex_following"]), int(prm["coloring"]), float(prm["theta_low"]),
                float(prm["theta_high"]), int(prm["color_cutoff"]), int(prm["max_iters"]),
                int(prm["max_phases"]), int(prm["color_seed"]), int(prm["trace"]),
                int(prm["color_phases"]), int(prm["abs_threshold"]), int(prm["vf_recursive"]),
                int(prm["color_order"]))
    h = ctypes.c_void_p()
    st = L.orc_run(n, rowptr.ctypes.data, col.ctypes.data, w.ctypes.data, ctypes.byref(p),
                   ctypes.byref(h))
    if st:
        raise OracleError(st)
    try:
        phases = []
        for ph in range(L.orc_num_phases(h)):
            ints = np.zeros(7, dtype=np.int64)
            hi = np.zeros(2, dtype=np.int64)
            lo = np.zeros(2, dtype=np.uint64)
            dbl = np.zeros(2, dtype=np.float64)
            L.orc_phase_info(h, ph, ints.ctypes.data, hi.ctypes.data, lo.ctypes.data,
                             dbl.ctypes.data)
            lab = np.empty(n, dtype=np.int32)
            L.orc_phase_labels(h, ph, lab.ctypes.data)
            P_ = Phase(int(ints[0]), int(ints[1]), int(ints[2]), bool(ints[3]), int(ints[4]),
                       int(ints[5]), int(ints[6]), _i128(hi[0], lo[0]), _i128(hi[1], lo[1]),
                       float(dbl[0]), float(dbl[1]), lab)
            if prm["trace"]:
                gh = L.orc_phase_graph(h, ph)
                P_.graph = _graph_out(gh)
                if P_.colored:
                    c = np.empty(P_.n, dtype=np.int32)
                    L.orc_phase_colors(h, ph, c.ctypes.data)
                    P_.colors = c
                for t in range(P_.iterations):
                    il = np.empty(P_.n, dtype=np.int32)
                    L.orc_phase_iter_labels(h, ph, t, il.ctypes.data)
                    P_.iter_labels.append(il)
            phases.append(P_)
        ni = L.orc_num_iters(h)
        pim = np.zeros(3 * ni, dtype=np.int64)
        hi = np.zeros(ni, dtype=np.int64)
        lo = np.zeros(ni, dtype=np.uint64)
        secs = np.zeros(ni, dtype=np.float64)
        L.orc_iters(h, pim.ctypes.data, hi.ctypes.data, lo.ctypes.data, secs.ctypes.data)
        iters = [(int(pim[3 * t]), int(pim[3 * t + 1]), int(pim[3 * t + 2]),
                  _i128(hi[t], lo[t]), float(secs[t])) for t in range(ni)]
        vm = np.empty(n, dtype=np.int32)
        L.orc_vf_map(h, vm.ctypes.data)
        return Result(n, int(L.orc_two_m(h)), int(L.orc_vf_n(h)), vm, phases, iters,
                      float(L.orc_seconds_total(h)))
    finally:
        L.orc_free(h)
