"""CPU tests of the benchmark's multi-rank logic with world_size-2 `gloo`
process groups (the GPU path uses the same helpers over NCCL):

  - weak scaling over frames: in every step the ranks cast distinct frames,
    and over the run every frame of the cycle is cast;
  - timing is the maximum over ranks, seen identically by every rank;
  - the whole-job rate counts every rank's rays;
  - the reference arm runs on rank 0 only: other ranks exit 0 without work.
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


def _worker(rank, ws, port, n_frames, steps, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        frames = [bench.frame_of(rank, ws, k, n_frames) for k in range(steps)]
        gathered = [None] * ws
        dist.all_gather_object(gathered, frames)
        slowest = bench.max_over_ranks(10.0 + 3.5 * rank, ws)
        q.put((rank, gathered, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,n_frames", [(2, 8), (2, 5)])
def test_frames_shard_and_max_over_ranks(ws, n_frames):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    steps = 12
    procs = [ctx.Process(target=_worker, args=(r, ws, port, n_frames, steps, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    gathered = res[0][1]
    assert all(r[1] == gathered for r in res)          # every rank sees the same schedule
    for k in range(steps):
        step_frames = [gathered[r][k] for r in range(ws)]
        assert len(set(step_frames)) == ws              # distinct frames within a step
    assert set(f for fr in gathered for f in fr) == set(range(n_frames))
    assert all(r[2] == 10.0 + 3.5 * (ws - 1) for r in res)   # the slowest rank's time, everywhere


def test_whole_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.whole_job_rate(1, 4_194_304, 10, 0.05)
    two = bench.whole_job_rate(2, 4_194_304, 10, 0.05)
    assert two == pytest.approx(2 * one) and one == pytest.approx(838.8608)
    assert bench.max_over_ranks(7.25, 1) == 7.25


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
