"""The multi-process benchmark path on the CPU: two ranks over gloo run the same replica logic
the GPU launch uses (barrier, time = maximum over ranks, job rate = all ranks' units over that
time), and the reference arm runs on rank 0 alone.  The method exchanges nothing between grids,
so N GPUs are N independent replicas; no data-path collective exists to test."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch
    import bench
    rk = bench.Replicas("gloo", torch.device("cpu"))
    rk.barrier()
    local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
    ms = rk.max_ms(local_ms)
    rate = rk.job_rate(1e9, ms)
    rk.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"world": rk.world, "rank": rk.rank, "ms": ms, "rate": rate}, f)
    rk.dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["world"] == world and d["rank"] == r
        assert d["ms"] == 15.0                          # the slowest rank's time, on every rank
        assert d["rate"] == pytest.approx(world * 1e9 / 15e-3)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.get(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        for k in env:
            os.environ.pop(k, None)
        rk = bench.Replicas("gloo")
        assert rk.world == 1 and rk.dist is None
        rk.barrier()
        assert rk.max_ms(3.5) == 3.5
        assert rk.job_rate(2e9, 4.0) == pytest.approx(5e11)
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v


@pytest.mark.parametrize("workload", ["thermal2d_16384", "batch64", "adjoint2048"])
def test_reference_arm_other_ranks_exit_at_once(workload):
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--workload", workload],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
