"""The seeded input generators: same bytes whatever the thread count, valid
CSRs under the problem statement of Sec. 2, and the workload sizes the
measurements quote."""
import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen as gg
import oracle
from conftest import ROOT

CHILD = r"""
import hashlib, sys
sys.path.insert(0, sys.argv[1])
import graphgen as gg
gs = [gg.rmat(14, 16, seed=2), gg.chunglu(200_000, 2.1, 0.7, 1_000_000, 2000.0, seed=3),
      gg.planted(20_000, 40, 0.01, 0.0005, 1, 8, seed=4)]
h = hashlib.sha256()
for g in gs:
    for a in (g.rowptr, g.col, g.w):
        h.update(a.tobytes())
print(h.hexdigest())
"""


def _digest(threads: int) -> str:
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=600, check=True)
    return r.stdout.strip()


def test_same_bytes_for_any_thread_count():
    assert _digest(1) == _digest(4)


@pytest.mark.parametrize("make", [lambda: gg.rmat(12, 16, seed=2),
                                  lambda: gg.chunglu(20_000, 2.1, 0.7, 80_000, 500.0, seed=3),
                                  lambda: gg.planted(5_000, 20, 0.01, 0.0005, 1, 8, seed=4),
                                  lambda: gg.random_graph(300, 0.05, wmax=5, loops=0.1, seed=5)])
def test_generated_csr_is_valid(make):
    g = make()
    st, two_m = oracle.validate(g.rowptr, g.col, g.w)
    assert st == 0 and two_m == int(g.w.astype(np.int64).sum())


def test_rmat20_workload_sizes():
    """R-MAT scale 20, 16 * 2^20 draws, (0.57, 0.19, 0.19, 0.05), seed 2."""
    g, prm = gg.workload("rmat20")
    deg = np.diff(g.rowptr)
    assert (g.n, len(g.col)) == (1_048_576, 31_402_876)
    assert int(deg.max()) == 64_659 and int((deg == 0).sum()) == 402_622
    assert prm["coloring"] == 1 and prm["vertex_following"] == 1


def test_served_stream_same_with_parallel_workers():
    """Generating the request stream side by side gives the same requests."""
    a = gg.served_stream(24, 200.0, 5, rmat_scales=(8, 12), planted_n=(500, 20_000))
    b = gg.served_stream(24, 200.0, 5, rmat_scales=(8, 12), planted_n=(500, 20_000), workers=4)
    assert [x for x, _ in a] == [x for x, _ in b]
    for (_, g), (_, h) in zip(a, b):
        assert np.array_equal(g.rowptr, h.rowptr) and np.array_equal(g.col, h.col)
        assert np.array_equal(g.w, h.w)
