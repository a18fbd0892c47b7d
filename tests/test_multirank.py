"""Host-side logic of bench.py's N > 1 path on CPU: world_size-2 gloo process groups.

bench.py runs one replica of the workload per rank (no data-path collective); what
crosses ranks is the barrier around the timed region, the maximum of the per-rank
times, and the rank filter of the output.  These run here with the gloo backend.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_info() == (world, rank, rank)
        # per-rank timed-region lengths (ms); the job is as slow as its slowest rank
        local_ms = [120.0, 180.0][rank]
        dist.barrier()
        total_ms = bench.max_over_ranks_on(local_ms, world, "cpu")
        value = bench.whole_job_rate(world, 1000, total_ms)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{total_ms} {value}\n")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo_world2(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        total_ms, value = map(float, (tmp_path / f"rank{rank}.txt").read_text().split())
        assert total_ms == 180.0
        # two ranks x 1000 solves in the slowest rank's 180 ms
        assert value == pytest.approx(2 * 1000 / 0.180)


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks_on(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(1, 50, 10.0) == pytest.approx(5000.0)


def test_reference_arm_prints_only_on_rank_0():
    """Under torchrun the reference arm runs on rank 0 alone; other ranks exit 0 silently."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
