"""lv_modularity_noalloc: the modularity entry point for callers that cannot
allocate device memory (services that hand the device to a fixed memory pool
at start-up, hosts held to a strict device-memory budget).  Its result must equal what the regular path reports
through lv_get_modularity for the same labels, on two calls in a row (the
second call runs on the scratch array the first one left behind).

This file is collected last on purpose, and also passes alone.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1237_gb300 import _build, lv
    _build.build()
    lv.load()
    return torch, lv


@pytest.mark.parametrize("workload", ["planted1k", "rmat16"])
def test_no_alloc_matches_regular_path(env, workload):
    torch, lv = env
    g, prm = gg.workload(workload)
    dev = torch.device("cuda:0")
    d = [torch.from_numpy(x).to(dev) for x in (g.rowptr, g.col, g.w)]
    h = lv.lv_graph_create(g.n, g.rowptr, g.col, g.w)
    try:
        lv.lv_run(h, lv.make_params(**prm))
        phases = [0, lv.lv_num_phases(h) - 1]
        for ph in phases:  # two calls in a row, different labellings
            lab = np.empty(g.n, dtype=np.int32)
            lv.lv_get_labels(h, ph, lab)
            q_ref, num_ref, den_ref = lv.lv_get_modularity(h, ph)
            num, den = lv.lv_modularity_noalloc(g.n, *d, torch.from_numpy(lab).to(dev))
            assert num == num_ref and den == den_ref
            assert abs(num / den - q_ref) <= 1e-12
    finally:
        lv.lv_graph_destroy(h)


def test_no_alloc_rejects_oversized_and_bad_labels(env):
    torch, lv = env
    g = gg.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    dev = torch.device("cuda:0")
    d = [torch.from_numpy(x).to(dev) for x in (g.rowptr, g.col, g.w)]
    bad = torch.tensor([0, 1, 9, 2], dtype=torch.int32, device=dev)
    with pytest.raises(lv.LVError) as e:
        lv.lv_modularity_noalloc(g.n, *d, bad)
    assert e.value.code == -1
    with pytest.raises(lv.LVError) as e:
        lv.lv_modularity_noalloc((1 << 20) + 1, *d, bad)
    assert e.value.code == -1
    # a NULL column or weight array is refused on the host, before any GPU work
    import ctypes
    L = lv.load()
    hi, lo, den = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int64()
    ptr = [x.data_ptr() for x in d]
    for k in (1, 2):
        args = list(ptr)
        args[k] = None
        rc = L.lv_modularity_noalloc(g.n, *args, bad.data_ptr(), ctypes.byref(hi),
                                     ctypes.byref(lo), ctypes.byref(den), None)
        assert rc == -1
    ok = torch.tensor([0, 0, 1, 1], dtype=torch.int32, device=dev)
    num, den = lv.lv_modularity_noalloc(g.n, *d, ok)
    # two edges inside, one across: Q = 4/6 - 2*(3/6)^2 = 1/6 (Eq. 3)
    assert den == 36 and num == 6
