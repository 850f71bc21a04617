"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/lv.h declares (no compute calls here)."""
import ctypes
import os
import re

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lv_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_header():
    from paper_1410_1237_gb300 import _build, lv
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared in lv.h but not exported"
    # the binding marshals every declared function
    assert set(names) == set(lv.SIGNATURES)


def test_status_strings_and_defaults_without_gpu():
    from paper_1410_1237_gb300 import lv
    lv.load()
    assert lv.lv_status_string(0) == "ok"
    assert "symmetric" in lv.lv_status_string(-2)
    p = lv.lv_params_default()
    assert (p.vertex_following, p.coloring, p.theta_low, p.theta_high, p.color_cutoff) == \
        (1, 1, 1e-6, 1e-2, 100_000)


def test_built_for_sm103a_only():
    from paper_1410_1237_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
