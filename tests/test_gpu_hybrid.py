"""GPU parity of the hybrid static/dynamic pipeline (Sec. 7): the static
triangles go through a bounding-volume hierarchy traced per ray, the dynamic
ones through the culls, and both commit into the same closest-hit keys.

The hierarchy is an acceleration, so the bar is the culled path's result:
the same triangle on every ray as with GRCA_CAST_NO_STATIC_BVH (same FP32
test, same FP64 re-test), and zero errors against the FP64 oracle.  The
distance may differ in the last bits on rays where one path sends an extra
candidate to the FP64 re-test: the traversal skips subtrees beyond a ray's
best certain hit, the culls test every candidate, and a re-tested ray
reports the FP64 distance rounded to FP32 instead of the FP32 one (both
within the FP32 bound 4e-6 of each other).
"""
import numpy as np
import pytest

import oracle
from grading import grade, stratified_rays
from scenes import make_config, noisy_sensor, ray_mask, scene_c1

pytestmark = pytest.mark.gpu


def _cast(c, ids, flags):
    import torch
    d, t = c.cast(ids, flags)
    torch.cuda.synchronize()
    return d.cpu().numpy(), t.cpu().numpy().view(np.uint32)


def _both(c, ids, flags):
    from paper_2605_10457_gb300 import grca
    d, t = _cast(c, ids, flags)
    st = c.stats()
    d0, t0 = _cast(c, ids, flags | grca.CAST_NO_STATIC_BVH)
    st0 = c.stats()
    return d, t, st, d0, t0, st0


def _agree(d, t, d0, t0):
    """Same triangle on every ray; distances equal up to the FP32 bound."""
    assert np.array_equal(t, t0), np.count_nonzero(t != t0)
    both = np.isfinite(d0)
    assert np.array_equal(np.isfinite(d), both)
    rel = np.abs(d[both].astype(np.float64) - d0[both]) / d0[both]
    assert rel.max(initial=0.0) <= 5e-6, rel.max()
    assert np.count_nonzero(rel) <= max(10, len(rel) // 1000)


def _grade(sensors, tris, d, t, rays=None, cull=False):
    orc = oracle.Oracle(sensors)
    ref = oracle.cast(orc, tris, rays, cull_backface=cull, ties=True)
    return grade(orc, tris, ref, d[ref["ray_ids"]], t[ref["ray_ids"]])


@pytest.mark.parametrize("flags_name", ["fp32", "fp64", "fp64_backface"])
def test_hybrid_c1_all_static_all_rays(flags_name):
    from paper_2605_10457_gb300 import grca
    fl = {"fp32": 0, "fp64": grca.CAST_FP64_RECHECK,
          "fp64_backface": grca.CAST_FP64_RECHECK | grca.CAST_CULL_BACKFACE}[flags_name]
    sc = scene_c1()
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in sc.sensors]
    tris = sc.tris(0)
    c.upload(tris)
    c.build_static(tris.shape[0])
    d, t, st, d0, t0, st0 = _both(c, ids, fl)
    assert st["bvh_node_visits"] > 0 and st["pairs"] == 0
    assert st0["bvh_node_visits"] == 0
    _agree(d, t, d0, t0)
    if fl & grca.CAST_FP64_RECHECK:
        g = _grade(sc.sensors, tris, d, t, cull=bool(fl & grca.CAST_CULL_BACKFACE))
        assert g["errors"] == 0, g


@pytest.mark.parametrize("cfg,d_max", [("c4m", np.inf), ("c4m", 10.0), ("c3m", np.inf), ("c2m", np.inf)])
def test_hybrid_static_plus_dynamic_frames(cfg, d_max):
    """Static part through the hierarchy, dynamic part updated per frame
    through the culls (graph replay), three frames."""
    from paper_2605_10457_gb300 import grca
    sc = make_config(cfg)
    if np.isfinite(d_max):
        for s in sc.sensors:
            s.d_min, s.d_max = 0.05, d_max
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in sc.sensors]
    ns = sc.n_static
    c.upload(sc.tris(0))
    c.build_static(ns)
    fl = grca.CAST_FP64_RECHECK | grca.CAST_GRAPH
    for frame in (0, 7, 23):
        tris = sc.tris(frame)
        c.update(tris[ns:], ns)
        d, t, st, d0, t0, st0 = _both(c, ids, fl)
        assert st["bvh_node_visits"] > 0
        assert st["pairs"] == (tris.shape[0] - ns) * len(ids)
        _agree(d, t, d0, t0)
    g = _grade(sc.sensors, tris, d, t, rays=stratified_rays(sc.sensors, 300, seed=2))
    assert g["errors"] == 0, g


def test_hybrid_stale_after_static_update_and_rebuild():
    from paper_2605_10457_gb300 import grca
    sc = make_config("c4m")
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in sc.sensors]
    tris = sc.tris(0).copy()
    ns = sc.n_static
    c.upload(tris)
    c.build_static(ns)
    # move a static block in front of sensor 0: the hierarchy is now stale
    s0 = sc.sensors[0]
    blk = tris[100:164].copy()
    blk = (blk - blk.mean((0, 1))) * 0.3 + s0.origin + 3.0 * s0.f
    tris[100:164] = blk
    c.update(blk, 100)
    fl = grca.CAST_FP64_RECHECK
    d, t = _cast(c, ids, fl)
    assert c.stats()["bvh_node_visits"] == 0          # fell back to the culls
    g = _grade(sc.sensors, tris, d, t, rays=stratified_rays(sc.sensors, 200, seed=4))
    assert g["errors"] == 0, g
    c.build_static(ns)
    d2, t2 = _cast(c, ids, fl)
    assert c.stats()["bvh_node_visits"] > 0
    _agree(d2, t2, d, t)
    assert np.count_nonzero((t2 >= 100) & (t2 < 164)) > 0
    c.build_static(0)                                   # drop the hierarchy
    d3, t3 = _cast(c, ids, fl)
    assert c.stats()["bvh_node_visits"] == 0 and np.array_equal(t3, t)


def test_hybrid_with_sensor_variants():
    """Masks, angular noise and range noise compose with the hybrid split."""
    import dataclasses
    from paper_2605_10457_gb300 import grca
    base = make_config("c4m")
    sc = dataclasses.replace(base, sensors=[noisy_sensor(s, 30 + k) for k, s in enumerate(base.sensors)])
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in sc.sensors]
    tris = sc.tris(4)
    c.upload(tris)
    c.build_static(sc.n_static)
    c.set_ray_mask(ids[1], ray_mask(sc.sensors[1], 1, 0.5))
    c.set_range_noise(ids[2], 0.03, 5)
    d, t, st, d0, t0, st0 = _both(c, ids, grca.CAST_FP64_RECHECK)
    assert st["bvh_node_visits"] > 0
    _agree(d, t, d0, t0)


def test_build_static_rejects_bad_count():
    from paper_2605_10457_gb300 import grca
    sc = scene_c1()
    c = grca.Caster(0)
    c.add_sensor(sc.sensors[0])
    c.upload(sc.tris(0))
    with pytest.raises(grca.GrcaError):
        c.build_static(sc.tris(0).shape[0] + 1)
