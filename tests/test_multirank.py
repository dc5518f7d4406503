"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards into independent signals (replicas only: every rank plans its
own sampling pattern and processes its own signals, no collective on the data
path).  What crosses ranks is the timing: the job time is the slowest rank's,
and the whole-job value counts the units of all ranks.  Rank 0 alone runs the
reference arm; the other ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        job_ms = bench.job_time_ms(local_ms, world)
        value = bench.job_throughput(1.0e9, 4, world, job_ms)
        wl = synth.workload("grid1024", batch=2, seed=bench.rank_seed(rank))
        out[rank] = {"job_ms": job_ms, "value": value, "x0": float(wl.x[0, 0]), "t_sum": float(wl.t.sum())}
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_units_add_up():
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0]["job_ms"] == res[1]["job_ms"] == 15.0
    # 2 ranks x 4 steps x 1e9 units over the slowest rank's 15 ms
    assert res[0]["value"] == pytest.approx(2 * 4 * 1.0e9 / 15e-3)
    # each rank draws its own signals (replicas over disjoint data)
    assert res[0]["x0"] != res[1]["x0"] and res[0]["t_sum"] != res[1]["t_sum"]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_single_rank_aggregation_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(3.5, 1) == 3.5
    assert bench.job_throughput(2.0e9, 10, 1, 4.0) == pytest.approx(10 * 2.0e9 / 4e-3)
    assert json.dumps({"v": bench.job_throughput(1.0, 1, 1, 1.0)})
