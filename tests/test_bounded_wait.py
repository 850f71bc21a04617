"""Bounded device waits end with an error status instead of a hang: a grid
whose block 0 never arrives at its grid barrier (the barrier of every
persistent kernel here) gives up after the given number of polls and raises
the wait flag, and the device then runs a full solve correctly.  No fault,
trap or endless loop is involved."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

LV_ERR_TIMEOUT = -9


@pytest.fixture(scope="module")
def lv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1237_gb300 import _build, lv as lvmod
    _build.build()
    lvmod.load()
    return lvmod


@pytest.mark.parametrize("polls", [1, 1000, 100_000])
def test_barrier_wait_gives_up_and_device_stays_usable(lv, polls):
    assert lv.lv_check_bounded_wait(polls) == LV_ERR_TIMEOUT
    g = gg.rmat(12, 8, seed=3)
    prm = dict(vertex_following=1, coloring=1, color_cutoff=0)
    res = lv.run(g.rowptr, g.col, g.w, **prm)
    ref = oracle.run(g.rowptr, g.col, g.w, **prm)
    assert np.array_equal(res.final_labels, ref.final_labels)
    assert res.phases[-1].N_end == ref.phases[-1].N_end
