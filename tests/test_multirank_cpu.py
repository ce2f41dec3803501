"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path shards over independent sessions (one per GPU, no data-path collective); the only
cross-rank steps are the barrier around the timed region and the max-over-ranks time. Here
two gloo ranks check that reduction, the whole-job rate (units of all ranks / the slowest
rank's time), that each rank draws its own seeded trials, and that the reference arm does
its work on rank 0 only.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]
        slowest = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.whole_job_rate(1000, world, slowest)
        w = dict(bench.WORKLOADS["profile_stream"], n=40)
        x = bench.make_trials(w, 1, seed=42 + rank)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"slowest": slowest, "rate": rate, "x0": float(x[0, 0, 0])}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate(tmp_path):
    world = 2
    tmp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    assert r[0]["slowest"] == r[1]["slowest"] == 17.25
    assert r[0]["rate"] == pytest.approx(2 * 1000 / 0.01725)
    assert r[0]["x0"] != r[1]["x0"]  # independent seeded trials per rank


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""
