"""The multi-rank logic of bench.py on CPU (world size 2, gloo): each rank gets
an independent replica, the timing is the slowest rank's, the value is the
whole job's throughput, and the reference arm runs and prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_ranks_get_independent_replicas():
    import bench
    wl0, _ = bench.make_workload("c1_methane_1500", 0.05, 0)
    wl1, _ = bench.make_workload("c1_methane_1500", 0.05, 1)
    assert np.array_equal(wl0.sample.x, wl1.sample.x)          # same geometry (weak scaling)
    assert not np.array_equal(wl0.sample.seed, wl1.sample.seed)  # own ionisation stream


def test_timed_calls_cover_every_step_once():
    import bench
    assert bench.step_calls(100, 1) == [1] * 100
    assert bench.step_calls(100, 8) == [8] * 12 + [4]
    assert bench.step_calls(96, 8) == [8] * 12
    assert bench.step_calls(5, 8) == [5]
    assert bench.step_calls(0, 8) == []
    for k in range(0, 40):
        for n in (1, 3, 8):
            assert sum(bench.step_calls(k, n)) == k


def test_job_throughput_counts_every_rank():
    import bench
    assert bench.job_throughput(1, 1000, 10, 2.0) == pytest.approx(5.0e6)
    assert bench.job_throughput(4, 1000, 10, 2.0) == pytest.approx(2.0e7)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 * (rank + 1) + 0.25             # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_throughput(world, 1000, 50, slowest)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "value": value}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == pytest.approx(20.25)
        assert r["value"] == pytest.approx(world * 1000 * 50 / 20.25e-3)


def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "c1_methane_1500", "--scale", "0.05"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0
