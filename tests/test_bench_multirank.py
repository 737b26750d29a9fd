"""The multi-rank host logic of bench.py, run as two gloo ranks on the CPU.

Images are independent problems, so the benchmark shards them over ranks with
no data-path collective: every rank solves its own batch (disjoint seeds), the
job's time is the slowest rank's (a MAX all-reduce), and the rate counts the
images of all ranks.  The reference arm prints from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 135.5][rank]                     # each rank's own step time
        slowest = bench.max_over_ranks(ms, dist, world, "cpu")
        seeds = bench.rank_seeds(rank, 4)
        everyone = [None] * world
        dist.all_gather_object(everyone, seeds)
        rate = bench.aggregate_rate(world, 4, 100, slowest)
        out.put((rank, slowest, everyone, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_images_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, slowest, everyone, rate in res:
        assert slowest == 135.5                       # both ranks see the slowest rank's time
        assert not set(everyone[0]) & set(everyone[1])  # disjoint images, no shared work
        assert rate == pytest.approx(2 * 4 * 100 / 0.1355)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, None, 1, "cpu") == 12.5
    assert bench.rank_seeds(0, 3) == [0, 1, 2]


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_matches_the_gpu_arm_config():
    import bench
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--batch", "2"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config(2, 500, 375, 100, "f16")
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_all_cores_oracle_timing_spawns_one_process_per_core():
    import bench
    rate, slowest = bench.oracle_rate_all_cores(1, 2)
    assert rate is not None and slowest > 0
    assert rate == pytest.approx(2 / slowest)
