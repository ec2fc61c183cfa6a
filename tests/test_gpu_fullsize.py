"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times (autotuned launch parameters, FP32 + FP64 recheck, CUDA-graph
replay), checked against the FP64 oracle on stratified ray samples (every
channel of every sensor, evenly strided rays) plus every stress-aimed ray.

Sizes: c2 (1 x 128x4096, 1.0 M triangles), c3 (2 x 128x4096, 5.0 M),
c4 (8 LiDARs of uneven shape, 21.7 M, 50 m max range) and c5
(8 x 128x4096, 21.7 M + the near-tie stress set).
"""
import numpy as np
import pytest

import oracle
from grading import grade, stratified_rays
from scenes import make_config

pytestmark = pytest.mark.gpu


def _run(scene, frame, n_per_sensor, extra_rays=None, seed=0):
    import torch
    from paper_2605_10457_gb300 import grca
    c = grca.Caster(0, big_pair_capacity=16 << 20, chunk_capacity=64 << 20, recheck_capacity=32 << 20)
    ids = [c.add_sensor(s) for s in scene.sensors]
    tris = scene.tris(frame)
    c.upload(tris)
    out = c.outputs(ids)
    fl = grca.CAST_FP64_RECHECK
    c.autotune(ids, fl, out)
    c.cast(ids, fl | grca.CAST_GRAPH, out)
    c.cast(ids, fl | grca.CAST_GRAPH, out)   # replay
    torch.cuda.synchronize()
    st = c.stats()
    assert st["device_error"] == 0 and st["pairs"] == len(ids) * tris.shape[0]
    d = out[0].cpu().numpy()
    t = out[1].cpu().numpy().view(np.uint32)
    c.close()
    rays = stratified_rays(scene.sensors, n_per_sensor, seed=seed)
    if extra_rays is not None:
        rays = np.unique(np.concatenate([rays, extra_rays]))
    orc = oracle.Oracle(scene.sensors)
    ref = oracle.cast(orc, tris, rays, ties=True)
    g = grade(orc, tris, ref, d[rays], t[rays])
    return g, st


def test_c2_full_size():
    sc = make_config("c2")
    g, st = _run(sc, frame=10, n_per_sensor=1024, seed=2)
    assert g["errors"] == 0, g
    assert g["hits"] > 500


def test_c3_full_size():
    sc = make_config("c3")
    g, st = _run(sc, frame=20, n_per_sensor=256, seed=3)
    assert g["errors"] == 0, g


def test_c4_full_size_range_50m():
    sc = make_config("c4", d_max=50.0)
    g, st = _run(sc, frame=30, n_per_sensor=32, seed=4)
    assert g["errors"] == 0, g


def test_c5_full_size_with_stress_rays():
    sc = make_config("c5")
    rng = np.random.default_rng(5)
    stress = rng.choice(sc.stress_rays, size=min(160, sc.stress_rays.size), replace=False)
    g, st = _run(sc, frame=45, n_per_sensor=24, extra_rays=stress, seed=5)
    assert g["errors"] == 0, g
    assert st["flagged_rays"] > 0   # the stress set exercises the FP64 recheck
