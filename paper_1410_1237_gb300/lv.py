"""ctypes binding of ``liblv.so`` (include/lv.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the C names; arrays may be numpy arrays
(host) or CUDA torch tensors (device).  There is no fallback: if the library
is not built or no GPU is present, the calls fail.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

LV_OK = 0
LV_ERR_STATE = -10
STATUS_NAMES = {0: "LV_OK", -1: "LV_ERR_ARG", -2: "LV_ERR_NOT_SYMMETRIC", -3: "LV_ERR_WEIGHT",
                -4: "LV_ERR_DUPLICATE", -5: "LV_ERR_OVERFLOW", -6: "LV_ERR_EMPTY",
                -7: "LV_ERR_CUDA", -8: "LV_ERR_OOM", -9: "LV_ERR_TIMEOUT", -10: "LV_ERR_STATE",
                -11: "LV_ERR_HASH"}


class LVError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {STATUS_NAMES.get(code, code)}"
        if _lib is not None:
            msg += f" ({_lib.lv_status_string(code).decode()})"
            if code == -7:
                msg += f": {_lib.lv_last_error().decode()}"
        super().__init__(msg)


class lv_params(ctypes.Structure):
    _fields_ = [("vertex_following", ctypes.c_int32), ("coloring", ctypes.c_int32),
                ("theta_low", ctypes.c_double), ("theta_high", ctypes.c_double),
                ("color_cutoff", ctypes.c_int64), ("max_iters", ctypes.c_int32),
                ("max_phases", ctypes.c_int32), ("color_seed", ctypes.c_uint64),
                ("collect_timing", ctypes.c_int32), ("keep_graphs", ctypes.c_int32),
                ("bin_lane_arcs", ctypes.c_int32), ("bin_warp_max", ctypes.c_int32),
                ("bin_cta_max", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("graph_capture", ctypes.c_int32), ("color_phases", ctypes.c_int32),
                ("abs_threshold", ctypes.c_int32), ("vf_recursive", ctypes.c_int32),
                ("color_order", ctypes.c_int32), ("sweep_blocks_per_sm", ctypes.c_int32),
                ("hub_slots_per_arc", ctypes.c_int32), ("persistent_sms", ctypes.c_int32)]


class lv_phase_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("arcs", ctypes.c_int64), ("n_next", ctypes.c_int64),
                ("two_m", ctypes.c_int64), ("N_start", ctypes.c_int64), ("N_end", ctypes.c_int64),
                ("q", ctypes.c_double), ("theta", ctypes.c_double), ("colored", ctypes.c_int32),
                ("num_colors", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("color_rounds", ctypes.c_int32), ("ms_color", ctypes.c_double),
                ("ms_iterate", ctypes.c_double), ("ms_rebuild", ctypes.c_double)]


class lv_iter_stat(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int32), ("iter", ctypes.c_int32),
                ("color_steps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("moved", ctypes.c_int64), ("N", ctypes.c_int64), ("arcs", ctypes.c_int64),
                ("ms", ctypes.c_double)]


class lv_stats(ctypes.Structure):
    _fields_ = [("num_phases", ctypes.c_int32), ("total_iterations", ctypes.c_int32),
                ("edge_visits", ctypes.c_int64), ("vf_n", ctypes.c_int64),
                ("sweep_launches", ctypes.c_int64), ("ms_total", ctypes.c_double),
                ("ms_vf", ctypes.c_double), ("ms_color", ctypes.c_double),
                ("ms_iterate", ctypes.c_double), ("ms_rebuild", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("graph_launches", ctypes.c_int64)]


class lv_batch_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("arcs", ctypes.c_int64), ("two_m", ctypes.c_int64),
                ("n_final", ctypes.c_int64), ("N_final", ctypes.c_int64), ("q", ctypes.c_double),
                ("num_phases", ctypes.c_int32), ("iterations", ctypes.c_int32)]


class lv_batch_sweep(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int32), ("sweep", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("vertices", ctypes.c_int64),
                ("arcs", ctypes.c_int64), ("moved", ctypes.c_int64), ("ms", ctypes.c_double)]


class lv_partition_compare(ctypes.Structure):
    _fields_ = [("tp", ctypes.c_uint64), ("fp", ctypes.c_uint64), ("fn", ctypes.c_uint64),
                ("tn", ctypes.c_uint64), ("sp", ctypes.c_double), ("se", ctypes.c_double),
                ("oq", ctypes.c_double), ("rand", ctypes.c_double)]


class lv_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_graphs", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("params", lv_params)]


class lv_server_result_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("num_phases", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_int64), ("arcs", ctypes.c_int64), ("two_m", ctypes.c_int64),
                ("n_final", ctypes.c_int64), ("N_final", ctypes.c_int64), ("q", ctypes.c_double),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


class lv_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("peak_graphs", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ms_admit", ctypes.c_double),
                ("ms_append", ctypes.c_double), ("ms_iterate", ctypes.c_double),
                ("ms_rebuild", ctypes.c_double), ("ms_results", ctypes.c_double)]


_lib = None

# every function declared in include/lv.h, with its ctypes signature
_P = ctypes.POINTER
_vp = ctypes.c_void_p
SIGNATURES = {
    "lv_params_default": (None, [_P(lv_params)]),
    "lv_graph_create": (ctypes.c_int, [_P(_vp), ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "lv_run": (ctypes.c_int, [_vp, _P(lv_params)]),
    "lv_check_bounded_wait": (ctypes.c_int, [ctypes.c_int32]),
    "lv_num_phases": (ctypes.c_int, [_vp, _P(ctypes.c_int32)]),
    "lv_get_labels": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int]),
    "lv_get_modularity": (ctypes.c_int, [_vp, ctypes.c_int32, _P(ctypes.c_double),
                                         _P(ctypes.c_int64), _P(ctypes.c_uint64),
                                         _P(ctypes.c_int64)]),
    "lv_get_phase_info": (ctypes.c_int, [_vp, ctypes.c_int32, _P(lv_phase_info)]),
    "lv_get_num_iterations": (ctypes.c_int, [_vp, _P(ctypes.c_int64)]),
    "lv_get_iteration_stats": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "lv_get_stats": (ctypes.c_int, [_vp, _P(lv_stats)]),
    "lv_get_tuning": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "lv_batch_get_tuning": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "lv_get_vf_map": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lv_get_phase_graph": (ctypes.c_int, [_vp, ctypes.c_int32, _P(ctypes.c_int64),
                                          _P(ctypes.c_int64), _vp, _vp, _vp, ctypes.c_int]),
    "lv_get_phase_colors": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int]),
    "lv_modularity_noalloc": (ctypes.c_int, [ctypes.c_int64, _vp, _vp, _vp, _vp,
                                             _P(ctypes.c_int64), _P(ctypes.c_uint64),
                                             _P(ctypes.c_int64), _vp]),
    "lv_compare_partitions": (ctypes.c_int, [ctypes.c_int64, _vp, _vp, ctypes.c_int,
                                             _P(lv_partition_compare), _vp]),
    "lv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lv_last_error": (ctypes.c_char_p, []),
    "lv_graph_destroy": (None, [_vp]),
    "lv_batch_create": (ctypes.c_int, [_P(_vp), ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_int,
                                       _vp]),
    "lv_batch_run": (ctypes.c_int, [_vp, _P(lv_params)]),
    "lv_batch_num_graphs": (ctypes.c_int, [_vp, _P(ctypes.c_int32)]),
    "lv_batch_get_labels": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int]),
    "lv_batch_get_graph_info": (ctypes.c_int, [_vp, ctypes.c_int32, _P(lv_batch_graph_info)]),
    "lv_batch_get_phase_info": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32,
                                               _P(lv_phase_info)]),
    "lv_batch_get_stats": (ctypes.c_int, [_vp, _P(lv_stats)]),
    "lv_batch_get_num_sweeps": (ctypes.c_int, [_vp, _P(ctypes.c_int64)]),
    "lv_batch_get_sweeps": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "lv_batch_destroy": (None, [_vp]),
    "lv_server_create": (ctypes.c_int, [_P(_vp), _P(lv_server_config), _vp]),
    "lv_server_submit": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp, _vp, _P(ctypes.c_int64)]),
    "lv_server_wait": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, _P(ctypes.c_int32)]),
    "lv_server_result": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, _P(lv_server_result_info)]),
    "lv_server_release": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lv_server_get_stats": (ctypes.c_int, [_vp, _P(lv_server_stats)]),
    "lv_server_destroy": (None, [_vp]),
}


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load liblv.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1410_1237_gb300._build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != LV_OK:
        raise LVError(code, where)


def _ptr(x) -> tuple[int, bool]:
    """(address, on_device) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data, False
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), bool(x.is_cuda)
    raise TypeError(f"unsupported array type {type(x)}")


# ------------------------------------------------------------- C-named API
def lv_params_default() -> lv_params:
    p = lv_params()
    load().lv_params_default(ctypes.byref(p))
    return p


def make_params(**kw) -> lv_params:
    p = lv_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def lv_graph_create(n: int, rowptr, col, w, stream: int = 0) -> int:
    """Return an opaque handle (int).  Arrays: numpy (host) or CUDA tensors."""
    L = load()
    rp, d0 = _ptr(np.ascontiguousarray(rowptr, dtype=np.int64)
                  if isinstance(rowptr, np.ndarray) else rowptr)
    cp, d1 = _ptr(np.ascontiguousarray(col, dtype=np.int32) if isinstance(col, np.ndarray) else col)
    wp, d2 = _ptr(np.ascontiguousarray(w, dtype=np.int32) if isinstance(w, np.ndarray) else w)
    if not (d0 == d1 == d2):
        raise ValueError("rowptr, col and w must all be host or all be device arrays")
    h = ctypes.c_void_p()
    _check(L.lv_graph_create(ctypes.byref(h), int(n), rp, cp, wp, int(d0), stream or None),
           "lv_graph_create")
    return h.value


def lv_run(h: int, params: lv_params | None = None):
    _check(load().lv_run(h, ctypes.byref(params) if params is not None else None), "lv_run")


def lv_num_phases(h: int) -> int:
    out = ctypes.c_int32()
    _check(load().lv_num_phases(h, ctypes.byref(out)), "lv_num_phases")
    return out.value


def lv_get_labels(h: int, phase: int, out) -> None:
    p, dev = _ptr(out)
    _check(load().lv_get_labels(h, phase, p, int(dev)), "lv_get_labels")


def lv_get_modularity(h: int, phase: int = -1) -> tuple[float, int, int]:
    """(q, numerator, denominator) with q = numerator / denominator."""
    q, hi, lo, den = ctypes.c_double(), ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
    _check(load().lv_get_modularity(h, phase, ctypes.byref(q), ctypes.byref(hi), ctypes.byref(lo),
                                    ctypes.byref(den)), "lv_get_modularity")
    num = (hi.value << 64) | lo.value
    return q.value, num, den.value


def lv_get_phase_info(h: int, phase: int) -> lv_phase_info:
    out = lv_phase_info()
    _check(load().lv_get_phase_info(h, phase, ctypes.byref(out)), "lv_get_phase_info")
    return out


def lv_get_iteration_stats(h: int) -> list:
    L = load()
    cnt = ctypes.c_int64()
    _check(L.lv_get_num_iterations(h, ctypes.byref(cnt)), "lv_get_num_iterations")
    arr = (lv_iter_stat * max(cnt.value, 1))()
    _check(L.lv_get_iteration_stats(h, arr, cnt.value), "lv_get_iteration_stats")
    return [arr[i] for i in range(cnt.value)]


def lv_get_stats(h: int) -> lv_stats:
    out = lv_stats()
    _check(load().lv_get_stats(h, ctypes.byref(out)), "lv_get_stats")
    return out


TUNING_FIELDS = ("lane_arcs", "warp_max", "cta_max", "blocks_per_sm", "hub_slots_per_arc")


def _tuning(fn, h: int, index: int):
    out = np.zeros(5, dtype=np.int32)
    code = fn(h, index, out.ctypes.data)
    if code == LV_ERR_STATE:
        return None
    _check(code, fn.__name__)
    return dict(zip(TUNING_FIELDS, (int(x) for x in out)))


def lv_get_tuning(h: int, phase: int):
    """The autotuner's choice for a phase as a dict, or None if not tuned."""
    return _tuning(load().lv_get_tuning, h, phase)


def lv_batch_get_tuning(h: int, rnd: int):
    """The autotuner's choice for a batched phase round, or None."""
    return _tuning(load().lv_batch_get_tuning, h, rnd)


def lv_get_vf_map(h: int, out) -> None:
    p, dev = _ptr(out)
    _check(load().lv_get_vf_map(h, p, int(dev)), "lv_get_vf_map")


def lv_get_phase_graph(h: int, phase: int):
    L = load()
    n, a = ctypes.c_int64(), ctypes.c_int64()
    _check(L.lv_get_phase_graph(h, phase, ctypes.byref(n), ctypes.byref(a), None, None, None, 0),
           "lv_get_phase_graph")
    rp = np.empty(n.value + 1, dtype=np.int64)
    col = np.empty(a.value, dtype=np.int32)
    w = np.empty(a.value, dtype=np.int32)
    _check(L.lv_get_phase_graph(h, phase, None, None, rp.ctypes.data, col.ctypes.data,
                                w.ctypes.data, 0), "lv_get_phase_graph")
    return rp, col, w


def lv_get_phase_colors(h: int, phase: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _check(load().lv_get_phase_colors(h, phase, out.ctypes.data, 0), "lv_get_phase_colors")
    return out


def lv_modularity_noalloc(n: int, rowptr, col, w, labels, stream: int = 0) -> tuple[int, int]:
    """(N, den) of a labelling, with device-resident CSR and labels (CUDA
    tensors), using only the library's fixed scratch array (no allocation)."""
    ptrs = [_ptr(x) for x in (rowptr, col, w, labels)]
    if not all(d for _, d in ptrs):
        raise ValueError("lv_modularity_noalloc takes device arrays only")
    hi, lo, den = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
    _check(load().lv_modularity_noalloc(int(n), *[p for p, _ in ptrs], ctypes.byref(hi),
                                        ctypes.byref(lo), ctypes.byref(den), stream or None),
           "lv_modularity_noalloc")
    return (hi.value << 64) | lo.value, den.value


def lv_check_bounded_wait(polls: int = 10_000) -> int:
    """Status of the bounded-wait check (LV_ERR_TIMEOUT expected)."""
    return int(load().lv_check_bounded_wait(int(polls)))


def lv_compare_partitions(labels_s, labels_p, stream: int = 0) -> dict:
    """SP, SE, OQ, Rand index and the pair counts of two labellings (Sec. 5);
    numpy (host) or CUDA tensors, both alike."""
    ps, d0 = _ptr(_arr(labels_s, np.int32))
    pp, d1 = _ptr(_arr(labels_p, np.int32))
    if d0 != d1:
        raise ValueError("both labellings must be host or both device arrays")
    n = len(labels_s)
    if len(labels_p) != n:
        raise ValueError("labellings of different sizes")
    out = lv_partition_compare()
    _check(load().lv_compare_partitions(n, ps, pp, int(d0), ctypes.byref(out), stream or None),
           "lv_compare_partitions")
    return {f: getattr(out, f) for f, _ in lv_partition_compare._fields_}


def lv_status_string(code: int) -> str:
    return load().lv_status_string(code).decode()


def lv_graph_destroy(h: int) -> None:
    if h:
        load().lv_graph_destroy(h)


def _arr(x, dtype):
    return np.ascontiguousarray(x, dtype=dtype) if isinstance(x, np.ndarray) else x


def lv_batch_create(n_graphs: int, gptr, rowptr, col, w, stream: int = 0) -> int:
    """Handle of a batch: the disjoint union CSR (union vertex ids) and the
    int64 graph starts ``gptr``; numpy (host) or CUDA tensors, all alike."""
    ptrs = [_ptr(_arr(gptr, np.int64)), _ptr(_arr(rowptr, np.int64)), _ptr(_arr(col, np.int32)),
            _ptr(_arr(w, np.int32))]
    if len({d for _, d in ptrs}) != 1:
        raise ValueError("gptr, rowptr, col and w must all be host or all be device arrays")
    h = ctypes.c_void_p()
    _check(load().lv_batch_create(ctypes.byref(h), int(n_graphs), *[p for p, _ in ptrs],
                                  int(ptrs[0][1]), stream or None), "lv_batch_create")
    return h.value


def lv_batch_run(h: int, params: lv_params | None = None):
    _check(load().lv_batch_run(h, ctypes.byref(params) if params is not None else None),
           "lv_batch_run")


def lv_batch_num_graphs(h: int) -> int:
    out = ctypes.c_int32()
    _check(load().lv_batch_num_graphs(h, ctypes.byref(out)), "lv_batch_num_graphs")
    return out.value


def lv_batch_get_labels(h: int, graph: int, phase: int, out) -> None:
    p, dev = _ptr(out)
    _check(load().lv_batch_get_labels(h, graph, phase, p, int(dev)), "lv_batch_get_labels")


def lv_batch_get_graph_info(h: int, graph: int) -> lv_batch_graph_info:
    out = lv_batch_graph_info()
    _check(load().lv_batch_get_graph_info(h, graph, ctypes.byref(out)), "lv_batch_get_graph_info")
    return out


def lv_batch_get_phase_info(h: int, graph: int, phase: int) -> lv_phase_info:
    out = lv_phase_info()
    _check(load().lv_batch_get_phase_info(h, graph, phase, ctypes.byref(out)),
           "lv_batch_get_phase_info")
    return out


def lv_batch_get_stats(h: int) -> lv_stats:
    out = lv_stats()
    _check(load().lv_batch_get_stats(h, ctypes.byref(out)), "lv_batch_get_stats")
    return out


def lv_batch_get_sweeps(h: int) -> list:
    L = load()
    cnt = ctypes.c_int64()
    _check(L.lv_batch_get_num_sweeps(h, ctypes.byref(cnt)), "lv_batch_get_num_sweeps")
    arr = (lv_batch_sweep * max(cnt.value, 1))()
    _check(L.lv_batch_get_sweeps(h, arr, cnt.value), "lv_batch_get_sweeps")
    return list(arr[:cnt.value])


def lv_batch_destroy(h: int) -> None:
    if h:
        load().lv_batch_destroy(h)


def lv_server_create(mem_budget_bytes: int = 0, max_graphs: int = 0, stream: int = 0,
                     **params) -> int:
    """A serving handle; params as make_params (defaults: every heuristic on)."""
    cfg = lv_server_config()
    cfg.mem_budget_bytes = int(mem_budget_bytes)
    cfg.max_graphs = int(max_graphs)
    cfg.params = make_params(**params)
    h = ctypes.c_void_p()
    _check(load().lv_server_create(ctypes.byref(h), ctypes.byref(cfg), stream or None),
           "lv_server_create")
    return h.value


def lv_server_submit(h: int, rowptr, col, w) -> int:
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.int32)
    rid = ctypes.c_int64()
    _check(load().lv_server_submit(h, len(rp) - 1, rp.ctypes.data, cl.ctypes.data, ww.ctypes.data,
                                   ctypes.byref(rid)), "lv_server_submit")
    return rid.value


def lv_server_wait(h: int, request_id: int, timeout_s: float = -1.0) -> bool:
    done = ctypes.c_int32()
    _check(load().lv_server_wait(h, request_id, timeout_s, ctypes.byref(done)), "lv_server_wait")
    return bool(done.value)


def lv_server_result(h: int, request_id: int, n: int | None = None):
    """(labels or None, lv_server_result_info); raises LVError for a failed request."""
    info = lv_server_result_info()
    code = load().lv_server_result(h, request_id, None, ctypes.byref(info))
    if code != LV_OK:
        raise LVError(code, "lv_server_result")
    lab = np.empty(info.n, dtype=np.int32)
    _check(load().lv_server_result(h, request_id, lab.ctypes.data, ctypes.byref(info)),
           "lv_server_result")
    return lab, info


def lv_server_release(h: int, request_id: int) -> None:
    _check(load().lv_server_release(h, request_id), "lv_server_release")


def lv_server_get_stats(h: int) -> lv_server_stats:
    out = lv_server_stats()
    _check(load().lv_server_get_stats(h, ctypes.byref(out)), "lv_server_get_stats")
    return out


def lv_server_destroy(h: int) -> None:
    if h:
        load().lv_server_destroy(h)


# ------------------------------------------------------- convenience layer
@dataclass
class PhaseResult:
    n: int
    arcs: int
    n_next: int
    colored: bool
    num_colors: int
    iterations: int
    two_m: int
    N_start: int
    N_end: int
    q: float
    theta: float
    labels: np.ndarray
    ms_color: float
    ms_iterate: float
    ms_rebuild: float


@dataclass
class Result:
    n: int
    two_m: int
    phases: list
    iters: list      # (phase, iter, color_steps, moved, N, arcs, ms)
    stats: dict
    vf_map: np.ndarray

    @property
    def final_labels(self) -> np.ndarray:
        return self.phases[-1].labels

    @property
    def q(self) -> float:
        return self.phases[-1].q


def collect(h: int, n: int) -> Result:
    phases = []
    for p in range(lv_num_phases(h)):
        info = lv_get_phase_info(h, p)
        lab = np.empty(n, dtype=np.int32)
        lv_get_labels(h, p, lab)
        phases.append(PhaseResult(info.n, info.arcs, info.n_next, bool(info.colored),
                                  info.num_colors, info.iterations, info.two_m, info.N_start,
                                  info.N_end, info.q, info.theta, lab, info.ms_color,
                                  info.ms_iterate, info.ms_rebuild))
    its = [(s.phase, s.iter, s.color_steps, s.moved, s.N, s.arcs, s.ms)
           for s in lv_get_iteration_stats(h)]
    st = lv_get_stats(h)
    stats = {f: getattr(st, f) for f, _ in lv_stats._fields_}
    vm = np.empty(n, dtype=np.int32)
    lv_get_vf_map(h, vm)
    return Result(n, phases[0].two_m if phases else 0, phases, its, stats, vm)


def run(rowptr, col, w, stream: int = 0, **params) -> Result:
    """Create a handle, run the whole method, collect the results, destroy."""
    n = len(rowptr) - 1
    h = lv_graph_create(n, rowptr, col, w, stream)
    try:
        lv_run(h, make_params(**params))
        return collect(h, n)
    finally:
        lv_graph_destroy(h)
