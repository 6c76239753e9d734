"""The multi-GPU path is replicas only: N independent boxes, no collective
on the data path.  What the benchmark does across ranks -- a barrier, the
slowest rank's time by a MAX all-reduce, the whole-job rate from it, and the
reference arm running on rank 0 alone -- is host logic, checked here with two
gloo ranks on the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
mine = [120.0, 150.0][rank]            # this rank's timed milliseconds
tmax = bench.max_over_ranks(torch, dist, ws, mine, "cpu")
rate = bench.whole_job_mlups(ws, 1000, 10, tmax)
with open(os.path.join(sys.argv[2], "rank%d.json" % rank), "w") as fh:
    json.dump({"rank": rank, "tmax": tmax, "rate": rate}, fh)
dist.destroy_process_group()
'''


def _torchrun(args, timeout=240):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=29517"] + args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT, env=env)


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    w = tmp_path / "worker.py"
    w.write_text(WORKER)
    r = _torchrun([str(w), ROOT, str(tmp_path)])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.load(open(tmp_path / ("rank%d.json" % k))) for k in (0, 1)]
    assert sorted(x["rank"] for x in lines) == [0, 1]
    for x in lines:
        assert x["tmax"] == 150.0                       # the slower rank's time on both ranks
        assert x["rate"] == pytest.approx(2 * 1000 * 10 / 0.150 / 1e6)


def test_single_rank_takes_its_own_time():
    import torch
    import bench
    assert bench.max_over_ranks(torch, None, 1, 42.5, "cpu") == 42.5
    assert bench.whole_job_mlups(1, 4194304, 300, 29.0) == pytest.approx(4194304 * 300 / 0.029 / 1e6)


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the reference arm (the CPU oracle) runs on rank 0 alone;
    the other rank exits 0 without work.  A tiny step count keeps it short."""
    r = _torchrun(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"], timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0
