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


def test_struct_layouts_match_header(tmp_path):
    """Every struct of lv.h has the size and field offsets the binding uses
    (the C compiler's view of the header against the ctypes declarations)."""
    import shutil
    import subprocess

    from paper_1410_1237_gb300 import lv
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = {"lv_params": lv.lv_params, "lv_phase_info": lv.lv_phase_info,
               "lv_iter_stat": lv.lv_iter_stat, "lv_stats": lv.lv_stats,
               "lv_batch_graph_info": lv.lv_batch_graph_info,
               "lv_batch_sweep": lv.lv_batch_sweep, "lv_server_config": lv.lv_server_config,
               "lv_server_result_info": lv.lv_server_result_info,
               "lv_server_stats": lv.lv_server_stats,
               "lv_partition_compare": lv.lv_partition_compare}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lv.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_server_rejects_bad_config_without_gpu():
    # argument checks come before any device work
    from paper_1410_1237_gb300 import lv
    lv.load()
    h = ctypes.c_void_p()
    assert lv.load().lv_server_create(ctypes.byref(h), None, None) == -1
    for bad in (dict(bin_lane_arcs=9), dict(max_iters=0), dict(bin_cta_max=64, bin_warp_max=128)):
        cfg = lv.lv_server_config()
        cfg.params = lv.make_params(**bad)
        assert lv.load().lv_server_create(ctypes.byref(h), ctypes.byref(cfg), None) == -1, bad
    cfg = lv.lv_server_config()
    cfg.params = lv.make_params()
    cfg.max_graphs = -1
    assert lv.load().lv_server_create(ctypes.byref(h), ctypes.byref(cfg), None) == -1


def test_bounded_wait_check_rejects_bad_polls_without_gpu():
    from paper_1410_1237_gb300 import lv
    lv.load()
    for polls in (0, -1, (1 << 24) + 1):
        assert lv.lv_check_bounded_wait(polls) == -1  # LV_ERR_ARG, before any GPU work
