"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks, each with
its own timing, agree on the slowest rank's time and the whole-job throughput;
the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 0.010 * (r + 1) s for its steps, and a second figure the other way round
    t, u = bench.max_over_ranks([0.010 * (rank + 1), 0.030 - 0.010 * rank], dist)
    value, fps = bench.job_throughput(world, 1_000_000, 20, t)
    with open(f"{out_path}.{rank}", "w") as fh:
        fh.write(f"{t!r} {u!r} {value!r} {fps!r}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time(tmp_path):
    world, port = 2, _free_port()
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    rows = [open(f"{out}.{r}").read().split() for r in range(world)]
    assert rows[0] == rows[1]  # every rank holds the same figures
    t, u, value, fps = (float(v) for v in rows[0])
    assert t == pytest.approx(0.020) and u == pytest.approx(0.030)
    assert value == pytest.approx(2 * 1_000_000 * 20 / 0.020 / 1e6)
    assert fps == pytest.approx(2 * 20 / 0.020)


def test_one_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks([0.5, 2.0]) == [0.5, 2.0]
    assert bench.job_throughput(1, 1_000_000, 10, 0.01) == pytest.approx((1000.0, 1000.0))


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
