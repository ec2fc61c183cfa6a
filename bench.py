"""Benchmark of the GRCA hot path on GB300.

Workload (default `c5`): 8 spinning LiDARs 128x4096 (360 deg) on one vehicle
rig, 21.7 M FP32 triangles of which 8.9 M are dynamic (rigid movers and
deforming meshes), the near-tie stress set, an animated frame stream.

One step = one frame: the frame's dynamic vertices are written into the
library's scene buffer (grca_update_vertices from a device-resident frame)
and all 8 sensors are cast in one batched FP32 + FP64-recheck frame, replayed
as a CUDA graph.  The metric is Mrays/s (rays per frame / frame time).

Also reported on the same line: the plain single-sensor FP32 path (8 serial
casts per frame), the end-to-end frame through grca_cast_host (host vertices
in, host results out; each frame's copy-out overlaps the next frame),
per-kernel CUDA-event times and the roofline of the
dominant kernel, the CPU oracle timed on a bounded ray sample, and the SM
clocks sampled during the timed region.

`--impl reference` times the FP64 CPU oracle (the reference arm) on bounded
ray samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s and ms/frame (8x128x4096 LiDARs, 22M tris), batched vs plain, oracle-exact"
F_CULL_A = 100.0  # FP32 flops per (triangle, sensor) pair: transform + elevation range + channel search
F_CULL_B = 100.0  # FP32 flops per surviving pair: emitter frame + azimuth range + ray interval
F_SETUP = 200.0   # FP32 flops per live pair: the test setup (edge normals, error bounds)
F_TEST = 30.0     # FP32 flops per candidate ray-triangle test
F_CULL = 200.0    # whole-frame unit: FP32 flops per (triangle, sensor) pair of the culls (150-250)
TRI_BYTES = 36.0
# the code a committed DRAM capture depends on: the kernels, the launch
# parameters chosen by the runtime, and the compiler flags
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2605_10457_gb300", "csrc", f)
                  for f in ("grca_kernels.cu", "grca_internal.h", "grca_api.cu")] + \
                 [os.path.join(ROOT, "paper_2605_10457_gb300", "build.py")]


def kernels_digest(sources=None) -> str:
    """SHA-256 of the kernel sources' code, with comments and whitespace
    removed: a change of the code invalidates a committed capture, a change
    of its comments does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        src = open(f).read()
        if f.endswith(".py"):
            src = re.sub(r"#[^\n]*", " ", src)
        else:
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def measured_traffic(kernel: str, workload: str = "c5"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of
    this workload (profiles/traffic_<workload>.json), or None when there is
    none or the kernel sources changed since the capture."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", f"traffic_{workload}.json")))
    except (OSError, ValueError):
        return None
    e = d.get("kernels", {}).get(kernel)
    if not e or d.get("kernels_sha256") != kernels_digest():
        return None
    return e.get("dram_bytes_per_launch")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float, n_sm: int) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def frame_roofline(n_tris: int, n_rays: int, pairs: int, candidates: int, frame_ms: float, fp32_tflops: float,
                   hbm_gbs: float) -> dict:
    """Whole-frame roofline in the method's own units: bytes = tau * 36 (the
    vertex stream) + rays * 24 (key init, key read, output); FP32 flops =
    pairs * F_CULL + candidates * F_TEST; T_roof = the larger of the two
    times at peak; frac = T_roof / measured frame time."""
    b = n_tris * TRI_BYTES + n_rays * 24.0
    f = pairs * F_CULL + candidates * F_TEST
    t_mem = b / (hbm_gbs * 1e9)
    t_alu = f / (fp32_tflops * 1e12)
    t_roof = max(t_mem, t_alu)
    s = frame_ms / 1e3
    return {"bytes": b, "flops": f, "f_cull_per_pair": F_CULL, "f_test_per_candidate": F_TEST,
            "achieved_gbs": b / s / 1e9, "achieved_tflops": f / s / 1e12,
            "t_roof_ms": 1e3 * t_roof, "frame_ms": frame_ms, "binding": "alu" if t_alu >= t_mem else "hbm",
            "frac": t_roof / s}


def accuracy_rays(sc, n_per_sensor: int = 48, n_stress: int = 96, seed: int = 11) -> np.ndarray:
    """The benchmark's graded ray sample: stratified rays of every sensor
    (every channel when the budget allows, evenly strided azimuths) plus a
    seeded subset of the stress-aimed rays."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from grading import stratified_rays
    rays = stratified_rays(sc.sensors, n_per_sensor, seed=seed)
    stress = getattr(sc, "stress_rays", None)
    if stress is not None and len(stress) and n_stress:
        rng = np.random.default_rng(seed)
        rays = np.unique(np.concatenate([rays, rng.choice(stress, size=min(n_stress, len(stress)), replace=False)]))
    return rays.astype(np.int64)


def grade_accuracy(sc, tris, rays, results: dict, threads: int) -> tuple:
    """Oracle pass over `rays` (timed: the cpu_baseline figure) and the error
    statement of each GPU result against it.  results: name -> (t, id) over
    `rays`.  Returns (per-result summaries, oracle seconds, tie-pass rays)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from grading import grade, oracle_two_pass, summary
    orc = oracle.Oracle(sc.sensors)
    t0 = time.perf_counter()
    ref0 = oracle.cast(orc, tris, rays, n_threads=threads)
    t_plain = time.perf_counter() - t0
    ref = oracle_two_pass(orc, tris, rays, list(results.values()), n_threads=threads, plain_ref=ref0)
    out = {}
    for name, (gt, gid) in results.items():
        g = grade(orc, tris, ref, gt, gid)
        out[name] = summary(g, ref, gt, gid)
    return out, t_plain, ref["tie_pass_rays"]


class Clocks:
    """nvidia-smi sampling in the background during a timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        # the timed region starts once the sampler runs (its first sample is out)
        t_end = time.time() + 3.0
        while self.p is not None and time.time() < t_end and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        text = self.f.read()
        os.unlink(self.f.name)
        return parse_clock_samples(text)


def parse_clock_samples(text: str) -> dict:
    """Median SM clock, maximum clock and the throttle reasons seen in
    `nvidia-smi --query-gpu=index,clocks.sm,clocks.max.sm,power.draw,
    clocks_event_reasons.active,...hw_slowdown,...hw_thermal_slowdown,
    ...sw_thermal_slowdown,...sw_power_cap --format=csv,noheader,nounits` lines."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
            "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def frame_of(rank: int, ws: int, k: int, n_frames: int) -> int:
    """Weak scaling over frames: step k of rank r casts frame (r + k * ws) mod n_frames,
    so the ranks of one step cast distinct frames (ws <= n_frames)."""
    return (rank + k * ws) % n_frames


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """The slowest rank's time (all ranks get it); identity on one rank."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, rays_per_step: int, steps: int, seconds: float) -> float:
    """Whole-job Mrays/s: every rank casts rays_per_step rays per step."""
    return ws * rays_per_step * steps / seconds / 1e6


def cpu_oracle_rate(scene, tris, budget_s: float, seed: int = 0, max_rays: int = 1 << 20, threads: int = 0):
    """FP64 oracle on growing stratified ray samples until `budget_s` of CPU work
    (all host cores unless `threads` is given)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from grading import stratified_rays
    orc = oracle.Oracle(scene.sensors)
    threads = threads or (os.cpu_count() or 1)
    n_done, t_used, k = 0, 0.0, 0
    n = 16
    while t_used < budget_s and n_done < max_rays:
        rays = stratified_rays(scene.sensors, max(1, n // len(scene.sensors)), seed=seed + k)[:n]
        t0 = time.perf_counter()
        oracle.cast(orc, tris, rays, n_threads=threads)
        dt = time.perf_counter() - t0
        n_done += rays.shape[0]
        t_used += dt
        k += 1
        if dt < budget_s / 8:
            n *= 2
    return n_done, t_used, threads


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from scenes import make_config
    sc = make_config(args.config)
    if args.d_max is not None:
        for s_ in sc.sensors:
            s_.d_min, s_.d_max = 0.05, float(args.d_max)
    tris = sc.tris(0)
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from grading import stratified_rays
    orc = oracle.Oracle(sc.sensors)
    threads = os.cpu_count() or 1
    # about a second of oracle work per step on 16 cores; long runs take fewer
    # rays per step so that the whole run stays within a few minutes
    per_step = args.ref_rays or max(8, min(48, 2400 // max(1, args.steps + args.warmup)))
    times = []
    for step in range(args.warmup + args.steps):
        rays = stratified_rays(sc.sensors, max(1, per_step // len(sc.sensors)), seed=100 + step)[:per_step]
        t0 = time.perf_counter()
        oracle.cast(orc, tris, rays, n_threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append((rays.shape[0], dt))
    n = sum(r for r, _ in times)
    t = sum(d for _, d in times)
    value = n / t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.config}: {len(sc.sensors)} LiDARs, {sc.n_rays} rays/frame, {sc.n_tris} tris; "
                               f"FP64 brute-force oracle on {per_step} stratified rays per step",
                   "rays_per_step": per_step, "triangles": sc.n_tris},
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} stratified rays of frame 0 per step x all {sc.n_tris} triangles"},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_triangle_split(args):
    """One frame per step, its triangles split over the ranks (contiguous
    slices; the dynamic tail goes to the ranks that hold it), every sensor
    cast on every rank, the keys combined by NCCL all-reduces (with the FP64
    re-test: the keys MIN, the per-ray flags MAX, the settled keys MIN).
    Headline leg only."""
    import torch
    from paper_2605_10457_gb300 import grca
    from paper_2605_10457_gb300.shard import all_reduce_max, all_reduce_min, sharded_cast, split_ranges
    from scenes import make_config
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        red, red_max = all_reduce_min(), all_reduce_max()
    else:
        red = red_max = lambda t: t   # noqa: E731  (one shard: the exchanges are the identity)
    sc = make_config(args.config)
    if args.d_max is not None:
        for s_ in sc.sensors:
            s_.d_min, s_.d_max = 0.05, float(args.d_max)
    ns, nd = sc.n_static, sc.n_dynamic
    lo, hi = split_ranges(sc.n_tris, ws)[rank]
    frames_host = [sc.dynamic_tris(f % sc.n_frames) for f in range(args.frames)]
    full0 = np.ascontiguousarray(np.concatenate([sc.static_tris, frames_host[0]], 0)[lo:hi])
    d_lo, d_hi = max(lo, ns), hi   # this slice's dynamic triangles (global ids)
    frames_dev = (torch.from_numpy(np.stack([f[d_lo - ns:d_hi - ns] for f in frames_host], 0)).to(dev)
                  if d_hi > d_lo else None)
    c = grca.Caster(local, big_pair_capacity=48 << 20, chunk_capacity=512 << 20, recheck_capacity=64 << 20)
    ids = [c.add_sensor(s) for s in sc.sensors]
    c.upload(full0)
    out = c.outputs(ids)
    FL = grca.CAST_FP64_RECHECK
    if not args.no_autotune:
        c.autotune(ids, FL, out)

    launches = []

    def step(k):
        if frames_dev is not None:
            c.update(frames_dev[k % args.frames], d_lo - lo)
        sharded_cast(c, ids, lo, FL, red, red_max, out, launches=launches)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(args.warmup + k)
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    value = sc.n_rays * args.steps / (ms / 1e3) / 1e6   # one frame per step for the whole job
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.config}: {len(sc.sensors)} LiDARs, {sc.n_tris} tris ({nd} dynamic), "
                                   f"FP32+FP64-recheck, triangles split over {ws} GPU(s)",
                       "rays_per_frame": sc.n_rays, "triangles": sc.n_tris,
                       "parallelism": f"triangles sharded over {ws} GPU(s): per-ray u64 MIN all-reduce "
                                      f"({'NCCL' if ws > 1 else 'none: one shard'}): keys MIN, flags MAX, "
                                      f"settled keys MIN ({17 * sc.n_rays / 1e6:.1f} MB per frame)",
                       "l2": "inputs larger than L2 (vertex stream)"},
            "gpu_launches": int(sum(launches[-args.steps:])), "clocks": clocks,
            "launch_config": c.launch_config(ids, FL)}), flush=True)
    c.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5")
    ap.add_argument("--frames", type=int, default=8, help="distinct animated frames kept on the device")
    ap.add_argument("--subset", type=int, default=0,
                    help="profiling captures: only the first N triangles of the workload's frame 0, no animation "
                         "(with --lean; inputs still larger than L2 for N above ~4 M)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch-config", default=None,
                    help="inline_max,chunk_rays,cull_block,cull_blocks_per_sm: use this launch configuration instead "
                         "of the autotuner's (profiler captures of the benchmark's own configuration)")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of single-core oracle work for the single-core rate; 0 skips the oracle legs")
    ap.add_argument("--acc-rays", type=int, default=48, help="graded stratified rays per sensor (accuracy leg)")
    ap.add_argument("--acc-stress", type=int, default=96, help="graded stress-aimed rays (accuracy leg)")
    ap.add_argument("--ref-rays", type=int, default=None,
                    help="rays per step of the reference arm (default: 48, fewer for long runs)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="default: steps")
    ap.add_argument("--stats", action="store_true", help="print cast statistics to stderr")
    ap.add_argument("--capacity", default="large", choices=["large", "small"],
                    help="device work-queue capacities (small: ~2 GB, for profiler captures)")
    ap.add_argument("--lean", action="store_true", help="headline leg only (no plain / profile / e2e legs)")
    ap.add_argument("--no-group-cull", action="store_true", help="A/B: turn off the group-level (GACP-T_g) cull")
    ap.add_argument("--no-occlusion", action="store_true",
                    help="A/B: test every live pair, also those whose candidate rays already hold closer hits")
    ap.add_argument("--no-hybrid-leg", action="store_true", help="skip the hybrid leg reported beside the headline")
    ap.add_argument("--no-lossy-leg", action="store_true", help="skip the lossy apparent-area leg")
    ap.add_argument("--no-variants-leg", action="store_true", help="skip the sensor-variants leg")
    ap.add_argument("--area-eps", type=float, default=1e-6,
                    help="eps_A of the lossy apparent-area leg (the paper's value: 1e-6)")
    ap.add_argument("--hybrid", action="store_true",
                    help="hybrid static/dynamic pipeline: static triangles through a hierarchy built once")
    ap.add_argument("--d-max", type=float, default=None,
                    help="range variant: every sensor gets [0.05 m, d_max] (default: the workload's own range)")
    ap.add_argument("--split", default="frames", choices=["frames", "triangles"],
                    help="multi-GPU split: frames (each rank casts its own frames, no exchange; weak scaling) or "
                         "triangles (each rank holds a slice of every frame's triangles, per-ray u64 MIN "
                         "all-reduce; strong scaling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.split == "triangles":
        return run_triangle_split(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2605_10457_gb300 import grca
    from scenes import make_config

    sc = make_config(args.config)
    if args.d_max is not None:
        for s_ in sc.sensors:
            s_.d_min, s_.d_max = 0.05, float(args.d_max)
    ns, nd = sc.n_static, sc.n_dynamic
    frames_host = [sc.dynamic_tris(f % sc.n_frames) for f in range(args.frames)]
    full0 = np.ascontiguousarray(np.concatenate([sc.static_tris, frames_host[0]], 0))
    if args.subset:
        # a static prefix of the scene for profiler captures
        full0 = np.ascontiguousarray(full0[:args.subset])
        ns, nd = full0.shape[0], 0
        frames_host = [full0[:0]]
        args.lean = True
    frames_dev = torch.from_numpy(np.stack(frames_host, 0)).to(dev)       # [F, nd, 3, 3]

    caps = dict(big_pair_capacity=48 << 20, chunk_capacity=512 << 20, recheck_capacity=64 << 20)
    if args.capacity == "small":
        caps = dict(big_pair_capacity=8 << 20, chunk_capacity=48 << 20, recheck_capacity=16 << 20,
                    survivor_capacity=96 << 20)
    if args.launch_config:
        lc = [int(x) for x in args.launch_config.split(",")]
        caps.update(inline_max=lc[0], chunk_rays=lc[1], cull_block=lc[2], cull_blocks_per_sm=lc[3])
        args.no_autotune = True
    c = grca.Caster(local, **caps)
    ids = [c.add_sensor(s) for s in sc.sensors]
    c.upload(full0)
    build_s = None
    if args.hybrid and ns:
        # hybrid static/dynamic pipeline: static hierarchy built once, outside the timed region
        t_b = time.time()
        c.build_static(ns)
        build_s = time.time() - t_b
    n_rays = sc.n_rays
    out = c.outputs(ids)
    stream = torch.cuda.current_stream()
    FL = (grca.CAST_FP64_RECHECK | (grca.CAST_NO_GROUP_CULL if args.no_group_cull else 0)
          | (grca.CAST_NO_OCCLUSION if args.no_occlusion else 0))

    tune_ms = None
    if not args.no_autotune:
        tune_ms = c.autotune(ids, FL, out)
    launch_cfg = c.launch_config(ids, FL)

    def step_batched(k):
        f = frame_of(rank, ws, k, args.frames)
        if nd:
            c.update(frames_dev[f % frames_dev.shape[0]], ns)
        c.cast(ids, FL | grca.CAST_GRAPH, out)

    # plain path: one sensor per cast, FP32 only, each into its slice of the outputs
    offs = np.cumsum([0] + [s.n_total for s in sc.sensors])
    plain_out = [(out[0][offs[i]:offs[i + 1]], out[1][offs[i]:offs[i + 1]]) for i in range(len(ids))]

    def step_plain(k):
        f = frame_of(rank, ws, k, args.frames)
        c.update(frames_dev[f], ns)
        for i, sid in enumerate(ids):
            c.cast([sid], grca.CAST_GRAPH | (FL & grca.CAST_NO_GROUP_CULL), plain_out[i])

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps, warmup, profiler_range=False):
        for k in range(warmup):
            fn(k)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if profiler_range:
            # lets `ncu --profile-from-start off` capture exactly the timed steps
            torch.cuda.profiler.start()
        e0.record(stream)
        for k in range(steps):
            fn(warmup + k)
        e1.record(stream)
        if profiler_range:
            torch.cuda.profiler.stop()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), ws, dev)

    # --- headline: batched FP32 + FP64 recheck, CUDA-graph replay -------------
    clk = Clocks(local)
    ms_b = timed(step_batched, args.steps, args.warmup, profiler_range=True)
    clocks = clk.stop()
    launches_per_frame = c.last_launch_count()
    st = c.stats(check=False)
    if args.lean:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": whole_job_rate(ws, n_rays, args.steps, ms_b / 1e3),
                              "unit": "Mrays/s", "ms_per_step": ms_b / args.steps, "lean": True, "launch_config": launch_cfg,
                              "stats": st, "clocks": clocks}), flush=True)
        c.close()
        return 0

    # --- plain single-sensor FP32 path -----------------------------------------
    ms_p = timed(step_plain, args.steps, max(3, args.warmup // 2))
    plain_launches = c.last_launch_count() * len(ids)

    # --- per-kernel CUDA-event times of the batched frame ----------------------
    c.profile(True)
    for k in range(args.steps):
        step_batched(k)
    torch.cuda.synchronize()
    prof = c.profile_read()
    c.profile(False)
    st_prof = c.stats(check=False)

    # --- end to end: host vertices in, host results out -----------------------
    e2e_steps = args.e2e_steps or args.steps
    pin_frames = [torch.from_numpy(frames_host[f]).pin_memory() for f in range(min(args.frames, 4))]
    # two pairs of pinned result arrays: frame k copies its results out (on
    # the library's own stream) while frame k+1 runs; before frame k+1 is
    # enqueued, frame k-1's results are on the host (one frame in flight)
    h_dist = [torch.empty(n_rays, dtype=torch.float32).pin_memory() for _ in range(2)]
    h_tri = [torch.empty(n_rays, dtype=torch.int32).pin_memory() for _ in range(2)]
    ids_a = np.asarray(ids, dtype=np.int32)
    sp = stream.cuda_stream
    fl_e2e = FL | grca.CAST_GRAPH | grca.CAST_HOST_ASYNC

    def step_e2e(k):
        c.cast_host_ptrs(ids_a, pin_frames[k % len(pin_frames)].data_ptr(), ns, nd, h_dist[k % 2].data_ptr(),
                         h_tri[k % 2].data_ptr(), fl_e2e, sp)
        c.host_wait(1)

    for k in range(max(3, args.warmup)):
        step_e2e(k)
    c.host_wait(0)
    # host-to-device bandwidth of this run (outside the timed region): the
    # end-to-end figure follows it, and it varies between runs
    probe_dst = torch.empty_like(frames_dev[0])
    torch.cuda.synchronize()
    t_p = time.perf_counter()
    for k in range(3):
        probe_dst.copy_(pin_frames[k % len(pin_frames)], non_blocking=True)
    torch.cuda.synchronize()
    h2d_gbs = 3 * nd * 36 / (time.perf_counter() - t_p) / 1e9
    del probe_dst
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        step_e2e(k)
    c.host_wait(0)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)

    value = whole_job_rate(ws, n_rays, args.steps, ms_b / 1e3)
    plain_value = whole_job_rate(ws, n_rays, args.steps, ms_p / 1e3)
    e2e_value = whole_job_rate(ws, n_rays, e2e_steps, e2e_s)

    # --- hybrid static/dynamic pipeline on the same frames (static hierarchy
    # built once, outside the timed region; reported beside the headline) ---
    hybrid = None
    if build_s is None and ns and not args.no_hybrid_leg:
        t_b = time.time()
        c.build_static(ns)
        hb_s = time.time() - t_b
        if not args.no_autotune:
            c.autotune(ids, FL, out)
        ms_h = timed(step_batched, args.steps, args.warmup)
        st_h = c.stats(check=False)
        hybrid = {"value": whole_job_rate(ws, n_rays, args.steps, ms_h / 1e3), "unit": "Mrays/s",
                  "ms_per_step": ms_h / args.steps, "static_build_s": hb_s,
                  "path": f"{ns} static triangles through a hierarchy built once (warp-packet traversal), "
                          f"{nd} dynamic through the culls, FP32 + FP64 recheck, one key minimum",
                  "bvh_node_visits": st_h.get("bvh_node_visits"), "bvh_tests": st_h.get("bvh_tests"),
                  "launch_config": c.launch_config(ids, FL)}
        c.build_static(0)

    # --- lossy apparent-area cull (App. A.4.1 Step 1, Eq. apparent_area) at the
    # paper's eps_A: its frame rate, and the paper's Hit% (a hit within 1 mm of
    # the exact distance, or both miss) on every ray of one frame against the
    # exact cast, which the parity tests hold to the FP64 oracle --------------
    lossy = None
    if not args.no_lossy_leg and build_s is None:
        cl = grca.Caster(local, area_eps=args.area_eps, **caps)
        ids_l = [cl.add_sensor(s) for s in sc.sensors]
        cl.upload(full0)
        out_l = cl.outputs(ids_l)
        fl_l = FL | grca.CAST_LOSSY_AREA
        if not args.no_autotune:
            cl.autotune(ids_l, fl_l, out_l)

        def step_lossy(k):
            f = frame_of(rank, ws, k, args.frames)
            cl.update(frames_dev[f], ns)
            cl.cast(ids_l, fl_l | grca.CAST_GRAPH, out_l)

        ms_l = timed(step_lossy, args.steps, args.warmup)
        st_l = cl.stats(check=False)
        f0 = frame_of(rank, ws, 0, args.frames)
        cl.update(frames_dev[f0], ns)
        cl.cast(ids_l, fl_l, out_l)
        c.update(frames_dev[f0], ns)
        c.cast(ids, FL, out)
        torch.cuda.synchronize()
        de, dl = out[0], out_l[0]
        me, ml = torch.isfinite(de), torch.isfinite(dl)
        close = me & ml & ((dl - de).abs() <= 1e-3)
        hit_pct = 100.0 * float(((~me & ~ml) | close).float().mean())
        lossy = {"value": whole_job_rate(ws, n_rays, args.steps, ms_l / 1e3), "unit": "Mrays/s",
                 "ms_per_step": ms_l / args.steps, "eps_a": args.area_eps, "hit_pct": hit_pct,
                 "hit_pct_rule": "hit within 1 mm of the exact distance, or both miss; every ray of one frame",
                 "pairs_live": st_l["pairs_live"], "pairs_live_exact": st_prof["pairs_live"],
                 "launch_config": cl.launch_config(ids_l, fl_l)}
        cl.close()
        del out_l

    # --- sensor variants (App. A.1, A.3): every LiDAR with per-ray azimuth
    # noise (up to 0.45 of the ray spacing) and perturbed channel elevations, a
    # random ray mask with half the rays firing, and 2 cm range noise; exact
    # (FP32 + FP64 recheck).  Correctness is in the GPU tests. ----------------
    variants = None
    if not args.no_variants_leg and build_s is None:
        from scenes import noisy_sensor, ray_mask
        cv = grca.Caster(local, **caps)
        sens_v = [noisy_sensor(s_, 100 + k) for k, s_ in enumerate(sc.sensors)]
        ids_v = [cv.add_sensor(s_) for s_ in sens_v]
        for k, (sid, s_) in enumerate(zip(ids_v, sens_v)):
            cv.set_ray_mask(sid, ray_mask(s_, 200 + k, 0.5, "random"))
            cv.set_range_noise(sid, 0.02, 300 + k)
        cv.upload(full0)
        out_v = cv.outputs(ids_v)
        if not args.no_autotune:
            cv.autotune(ids_v, FL, out_v)

        def step_variants(k):
            f = frame_of(rank, ws, k, args.frames)
            cv.update(frames_dev[f], ns)
            cv.cast(ids_v, FL | grca.CAST_GRAPH, out_v)

        ms_v = timed(step_variants, args.steps, args.warmup)
        st_v = cv.stats(check=False)
        variants = {"value": whole_job_rate(ws, n_rays, args.steps, ms_v / 1e3), "unit": "Mrays/s",
                    "ms_per_step": ms_v / args.steps,
                    "sensors": "per-ray azimuth noise (0.45 ray spacing), perturbed elevations (0.3 gap), "
                               "random ray mask (half the rays fire), range noise 2 cm",
                    "candidates": st_v["candidates"], "candidates_exact_grid": st_prof["candidates"],
                    "launch_config": cv.launch_config(ids_v, FL)}
        cv.close()
        del out_v

    # --- roofline of the dominant kernel ---------------------------------------
    peaks, src = _peaks()
    # the committed DRAM counters belong to one workload (c5, unlimited range)
    traffic_key = args.config if args.d_max is None else f"{args.config}_dmax{args.d_max:g}"
    dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"])
    dom_name, dom_v = dom
    avg_ms = dom_v["total_ms"] / max(1, dom_v["launches"])
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = fp32_peak_tflops(sm_max, n_sm)
    pairs = st_prof["pairs"]
    if dom_name == "k_cull_a":
        flops = pairs * F_CULL_A
    elif dom_name == "k_cull_b":
        # setups only for the live pairs that get one: not the deferred ones
        # (set up by k_expand) nor those dropped as occluded
        setups = st_prof["pairs_live"] - st_prof["big_pairs"] - st_prof.get("pairs_occluded", 0)
        flops = (st_prof["survivors"] * F_CULL_B + setups * F_SETUP
                 + st_prof["candidates_inline"] * F_TEST)
    elif dom_name == "k_test":
        flops = (st_prof["tests"] - st_prof["candidates_inline"]) * F_TEST
    else:
        flops = 0.0
    achieved = flops / (avg_ms / 1e3) / 1e12 if flops else 0.0
    ka = prof.get("k_cull_a", {"total_ms": 1.0, "launches": 1})
    hbm_achieved = (sc.n_tris * TRI_BYTES) / (ka["total_ms"] / max(1, ka["launches"]) / 1e3) / 1e9
    roofline = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak if fp32_peak else None, "traffic": measured_traffic(dom_name, traffic_key),
                "peak_source": f"FP32 {n_sm} SM x 128 lanes x 2 x {sm_max:.0f} MHz (unit counts and max clock)",
                "algorithmic": {"k_cull_a": f"{F_CULL_A:.0f} flop per (tri, sensor) pair",
                                "k_cull_b": f"{F_CULL_B:.0f} flop per surviving pair + {F_SETUP:.0f} per live pair set "
                                            f"up inline (not deferred, not dropped as occluded) + "
                                            f"{F_TEST:.0f} per inline test",
                                "k_test": f"{F_TEST:.0f} flop per queued test"},
                "avg_launch_ms": avg_ms,
                "hbm_vertex_stream_gbs": hbm_achieved, "hbm_peak_gbs": peaks.get("hbm_gbs"),
                "hbm_peak_source": src,
                "frame": frame_roofline(sc.n_tris, n_rays, st_prof["pairs"], st_prof["candidates"],
                                        ms_b / args.steps, fp32_peak, float(peaks.get("hbm_gbs", 6800.0)))}

    # --- accuracy against the FP64 oracle, and the oracle's own rate -----------
    # Frame 0 is cast again through the same caster (launch configuration of
    # the timed frames) with FP32 + FP64 recheck and with the FP32 test only;
    # both are graded on one ray sample with the stated tolerances (id up to
    # near ties / shared edges, distance 1e-5 relative, hit/miss up to 1e-12
    # rad of a silhouette) and no extra exemption for the FP32-only result.
    # The oracle pass over that sample, on all host cores, is the cpu_baseline.
    cpu = None
    accuracy = None
    if rank == 0 and ws == 1 and args.cpu_budget > 0:
        rays_acc = accuracy_rays(sc, args.acc_rays, args.acc_stress)
        f0 = frame_of(rank, ws, 0, args.frames)
        c.update(frames_dev[f0], ns)
        idx = torch.from_numpy(rays_acc).to(dev)
        res = {}
        st_acc = {}
        for name, fl in (("fp32_recheck", FL), ("fp32_only", FL & ~grca.CAST_FP64_RECHECK)):
            c.cast(ids, fl, out)
            torch.cuda.synchronize()
            st_acc[name] = c.stats(check=False)
            res[name] = (out[0][idx].cpu().numpy(), out[1][idx].cpu().numpy().view(np.uint32))
        cores = os.cpu_count() or 1
        summ, t_cpu, n_tie = grade_accuracy(sc, full0, rays_acc, res, cores)
        n1, t1, _ = cpu_oracle_rate(sc, full0, min(2.0, args.cpu_budget / 4), seed=7, threads=1)
        rate = len(rays_acc) / t_cpu
        n_stress = int(np.isin(rays_acc, getattr(sc, "stress_rays", np.zeros(0, np.int64))).sum())
        cpu = {"value": rate / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
               "sample": f"the accuracy sample: {len(rays_acc)} rays of frame 0 ({len(rays_acc) - n_stress} "
                         f"stratified, {n_stress} stress-aimed) x all {sc.n_tris} triangles, FP64 brute force, "
                         f"{t_cpu:.1f} s",
               "single_core_mrays_per_s": n1 / t1 / 1e6,
               "extrapolated_frame_s": n_rays / rate,
               "extrapolation": "rays per frame / measured rate (every ray against every triangle)"}
        accuracy = {"frame": f0, "rays": int(len(rays_acc)), "stress_rays": n_stress,
                    "rule": "id equal, or in the oracle's near-tie set (1e-6 rel), or within 1e-7 rad of the "
                            "GPU triangle with its plane distance within 1e-6 rel; distance within 1e-5 rel; "
                            "hit/miss equal except within 1e-12 rad of the triangle's boundary; the same rule "
                            "for both paths",
                    "fp32_recheck": summ["fp32_recheck"], "fp32_only": summ["fp32_only"],
                    "flagged_rays": st_acc["fp32_recheck"]["flagged_rays"], "tie_pass_rays": n_tie}

    kernel_ms = {k: v["total_ms"] / max(1, v["launches"]) for k, v in prof.items() if v["launches"]}
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_b / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.config}: {len(sc.sensors)} LiDARs x {sc.sensors[0].n_channels}x"
                               f"{sc.sensors[0].n_rays} 360deg, {sc.n_tris} tris ({nd} dynamic), batched "
                               f"FP32+FP64-recheck, CUDA-graph replay"
                               + (f", range [0.05, {args.d_max:g}] m" if args.d_max is not None else "")
                               + (f", hybrid: {ns} static tris through a hierarchy built once" if build_s is not None
                                  else ""),
                   "rays_per_frame": n_rays, "triangles": sc.n_tris, "dynamic_triangles": nd,
                   "sensors": len(sc.sensors), "frames_cycled": args.frames,
                   "l2": "inputs larger than L2 (vertex stream 0.78 GB per frame)",
                   "parallelism": f"weak: frames sharded over {ws} GPU(s)"},
        "plain": {"value": plain_value, "unit": "Mrays/s", "ms_per_step": ms_p / args.steps,
                  "path": "8 serial single-sensor FP32 casts per frame", "gpu_launches": plain_launches * args.steps},
        "hybrid": hybrid,
        "lossy_area": lossy,
        "sensor_variants": variants,
        "e2e": {"value": e2e_value, "unit": "Mrays/s", "h2d_bytes_per_step": int(nd * 36),
                "d2h_bytes_per_step": int(n_rays * 8), "ms_per_step": 1e3 * e2e_s / e2e_steps,
                "schedule": "grca_cast_host per frame from pinned host vertices into two alternating pairs of "
                            "pinned result arrays; a frame's copy-out overlaps the next frame, at most one "
                            "frame in flight",
                "h2d_gbs_probe": h2d_gbs},
        "gpu_launches": launches_per_frame * args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "accuracy": accuracy,
        "clocks": clocks,
        "kernel_ms": kernel_ms,
        "stats": {k: st_prof[k] for k in ("pairs", "survivors", "pairs_live", "candidates", "candidates_inline",
                                          "big_pairs",
                                          "chunks", "tests", "hits", "uncertain", "ties", "flagged_rays",
                                          "recheck_pairs", "group_culled", "bvh_node_visits", "bvh_tests",
                                          "queued_edge", "queued_t", "queued_range", "queued_orient", "queued_tie",
                                          "kept_edge", "kept_t", "kept_range", "kept_orient", "kept_tie",
                                          "t_refined", "pairs_occluded")},
        "autotune_ms": tune_ms,
        "launch_config": launch_cfg,
        "static_build_s": build_s,
        "device_error": st_prof["device_error"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if args.stats and rank == 0:
        print(json.dumps(st, indent=1), file=sys.stderr)
    c.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
