"""The multi-rank harness of bench.py on CPU: two gloo ranks (the launch
torchrun makes, one process per rank), the max-over-ranks job time, the
whole-job rate and rank 0 alone printing the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch
import bench
rank, world, local = bench.dist_env()
pg = bench.init_dist(world, torch.device("cpu"))
slowest = bench.max_over_ranks(1.5 + rank, pg, torch.device("cpu"))
rate = bench.whole_job_rate(100.0, world, slowest)
pg.barrier()
print(json.dumps({"rank": rank, "world": world, "slowest": slowest, "rate": rate}), flush=True)
pg.destroy_process_group()
"""


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(world: int, code: str, extra_env=None, timeout=120):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            out, err = p.communicate()
        outs.append((p.returncode, out, err))
    return outs


def test_two_gloo_ranks_take_the_slowest_time():
    pytest.importorskip("torch.distributed")
    outs = launch(2, CHILD)
    lines = []
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
        lines += [json.loads(x) for x in out.splitlines() if x.startswith("{")]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    for l in lines:
        assert l["world"] == 2 and l["slowest"] == 2.5
        assert l["rate"] == pytest.approx(2 * 100.0 / 2.5)


def test_reference_arm_prints_on_rank0_only():
    # the reference arm at N=2 (replica of the launch torchrun makes): rank 1
    # exits 0 without work, rank 0 prints one JSON line
    code = ("import sys, os; sys.path.insert(0, os.environ['ROOT']); import bench; "
            "sys.argv = ['bench.py', '--impl', 'reference', '--workload', 'planted1k', "
            "'--steps', '1', '--warmup', '0']; sys.exit(bench.main())")
    outs = launch(2, code)
    assert all(rc == 0 for rc, _, _ in outs), [e[-1000:] for _, _, e in outs]
    r0 = [x for x in outs[0][1].splitlines() if x.startswith("{")]
    r1 = [x for x in outs[1][1].splitlines() if x.startswith("{")]
    assert len(r0) == 1 and not r1
    line = json.loads(r0[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
