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


# ---------------------------------------------------------------------------
# triangle-sharded casts: the exchange over world_size-2 gloo ranks, with the
# FP64 oracle standing in for each rank's cast of its slice
# ---------------------------------------------------------------------------
def _oracle_keys(sensors, tris, base, rays):
    import numpy as np
    import oracle
    from paper_2605_10457_gb300.shard import KEY_MISS
    r = oracle.cast(sensors, tris, rays)
    t32 = r["t"].astype(np.float32).view(np.uint32).astype(np.int64)
    hit = r["id"] != oracle.NO_HIT
    return np.where(hit, (t32 << 32) | (base + r["id"].astype(np.int64)), np.int64(KEY_MISS))


def _band_flags(local, glob, base_beta=1e-5):
    """1 where this rank's winner is another triangle than the global
    winner's but lies within its tie band (the cross-shard part of the
    flags exchange)."""
    import numpy as np
    t = lambda k: (k >> 32).astype(np.uint32).view(np.float32)   # noqa: E731
    hit = (local & 0xFFFFFFFF) != 0xFFFFFFFF
    return (hit & (local != glob) & (t(local) <= t(glob) * np.float32(1 + base_beta))).astype(np.uint8)


def _shard_worker(rank, ws, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2605_10457_gb300.shard import all_reduce_max, all_reduce_min, split_ranges
    from scenes import scene_c1
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        sc = scene_c1()
        tris = sc.tris()
        rays = np.arange(0, sc.n_rays, 3, dtype=np.int64)
        lo, hi = split_ranges(tris.shape[0], ws)[rank]
        local = _oracle_keys(sc.sensors, tris[lo:hi], lo, rays)
        glob = all_reduce_min()(torch.from_numpy(local.copy())).numpy()
        fl = all_reduce_max()(torch.from_numpy(_band_flags(local, glob))).numpy()
        q.put((rank, glob, fl, local))
    finally:
        dist.destroy_process_group()


def test_triangle_shards_min_exchange_equals_the_whole_set():
    """The keys of each rank's slice, combined by the MIN all-reduce, give the
    closest hit over all triangles; the flags exchange (MAX) marks exactly the
    rays where another rank's winner lies within the tie band of the global
    winner; every rank sees the same exchange."""
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2605_10457_gb300.shard import KEY_MISS, split_ranges
    from scenes import scene_c1
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(ws)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    glob, fl = res[0][1], res[0][2]
    assert all(np.array_equal(r[1], glob) and np.array_equal(r[2], fl) for r in res)
    sc = scene_c1()
    tris = sc.tris()
    rays = np.arange(0, sc.n_rays, 3, dtype=np.int64)
    whole = _oracle_keys(sc.sensors, tris, 0, rays)
    # the same FP32 distance everywhere; the same id except where two
    # triangles' distances round to the same FP32 value (then the lower id)
    assert np.array_equal(glob >> 32, whole >> 32)
    diff = (glob & 0xFFFFFFFF) != (whole & 0xFFFFFFFF)
    assert diff.sum() <= 2 and np.all((glob[diff] & 0xFFFFFFFF) < (whole[diff] & 0xFFFFFFFF))
    assert (glob != KEY_MISS).sum() > 1000
    # the flags: the union over the ranks of their own cross-shard flags
    assert np.array_equal(fl, np.maximum.reduce([_band_flags(r[3], glob) for r in res]))
    ranges = split_ranges(tris.shape[0], ws)
    owner = [np.searchsorted([h for _, h in ranges], int(k & 0xFFFFFFFF), side="right") for k in glob[glob != KEY_MISS]]
    assert set(owner) == set(range(ws))   # both ranks hold winners


def test_split_ranges_cover_every_triangle_once():
    sys.path.insert(0, ROOT)
    from paper_2605_10457_gb300.shard import split_ranges
    for n, w in ((10040, 2), (7, 3), (5, 8), (21724415, 8)):
        r = split_ranges(n, w)
        assert r[0][0] == 0 and r[-1][1] == n and all(r[k][1] == r[k + 1][0] for k in range(w - 1))
        assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1
