"""GPU checks of the group-level cull (GACP-T_g, Sec. 10.1.1).

The cull is lossless by construction, so its parity bar is exact equality:
the cast with group culling on, the cast with it off (GRCA_CAST_NO_GROUP_CULL)
and the no-cull brute force must give bit-identical outputs, on scenes where
the group test removes most pairs (short ranges) and where it removes few.
The group boxes follow vertex updates; a stale box would drop hits of moved
geometry, which the update test below would catch against the oracle.
"""
import numpy as np
import pytest

import oracle
from grading import grade, stratified_rays
from scenes import make_config, make_sensor, scene_c1

pytestmark = pytest.mark.gpu


def _cast(c, ids, flags):
    import torch
    d, t = c.cast(ids, flags)
    torch.cuda.synchronize()
    return d.cpu().numpy(), t.cpu().numpy().view(np.uint32)


def _ranged(cfg, d_min, d_max):
    sc = make_config(cfg)
    for s in sc.sensors:
        s.d_min, s.d_max = d_min, d_max
    return sc


@pytest.mark.parametrize("cfg,d_min,d_max", [("c4m", 0.05, 10.0), ("c4m", 0.05, 50.0), ("c4m", 20.0, np.inf),
                                             ("c1", 0.0, np.inf), ("c3m", 0.0, 30.0)])
def test_group_cull_is_lossless(cfg, d_min, d_max):
    from paper_2605_10457_gb300 import grca
    sc = _ranged(cfg, d_min, d_max)
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in sc.sensors]
    tris = sc.tris(2)
    c.upload(tris)
    d_on, t_on = _cast(c, ids, 0)
    st = c.stats()
    d_off, t_off = _cast(c, ids, grca.CAST_NO_GROUP_CULL)
    st_off = c.stats()
    d_b, t_b = _cast(c, ids, grca.CAST_BRUTE)
    assert np.array_equal(t_on, t_off) and np.array_equal(d_on, d_off)
    assert np.array_equal(t_on, t_b) and np.array_equal(d_on, d_b)
    assert st_off["group_culled"] == 0
    assert st["pairs_live"] == st_off["pairs_live"]
    if np.isfinite(d_max) and d_max <= 10.0:
        assert st["group_culled"] > 0.5 * st["pairs"], st
    # FP64 recheck path with groups on, against the oracle
    d, t = _cast(c, ids, grca.CAST_FP64_RECHECK | grca.CAST_GRAPH)
    orc = oracle.Oracle(sc.sensors)
    ref = oracle.cast(orc, tris, stratified_rays(sc.sensors, 200, seed=3), ties=True)
    g = grade(orc, tris, ref, d[ref["ray_ids"]], t[ref["ray_ids"]])
    assert g["errors"] == 0, g


def test_group_boxes_follow_vertex_updates():
    """Cast at frame 0 with a 12 m range, then move every dynamic triangle
    (frames 0 -> 9, with graph replay) and a far static block into range."""
    from paper_2605_10457_gb300 import grca
    sc = _ranged("c4m", 0.05, 12.0)
    c = grca.Caster(0)
    ids = [c.add_sensor(s) for s in sc.sensors]
    t0 = sc.tris(0)
    c.upload(t0)
    fl = grca.CAST_FP64_RECHECK | grca.CAST_GRAPH
    _cast(c, ids, fl)
    t9 = sc.tris(9)
    ns = sc.n_static
    c.update(t9[ns:], ns)
    # bring a far static block of 64 triangles next to sensor 0 (a partial group at both ends)
    s0 = sc.sensors[0]
    far = np.linalg.norm(t9[:ns].mean(1) - s0.origin, axis=1)
    k0 = int(np.argmax(far)) // 32 * 32 + 7
    moved = t9[k0:k0 + 64].copy()
    moved = (moved - moved.mean((0, 1))) * 0.2 + s0.origin + 4.0 * s0.f
    t9 = t9.copy()
    t9[k0:k0 + 64] = moved
    c.update(moved, k0)
    d, t = _cast(c, ids, fl)
    assert c.stats()["group_culled"] > 0
    orc = oracle.Oracle(sc.sensors)
    rays = stratified_rays(sc.sensors, 300, seed=8)
    ref = oracle.cast(orc, t9, rays, ties=True)
    g = grade(orc, t9, ref, d[ref["ray_ids"]], t[ref["ray_ids"]])
    assert g["errors"] == 0, g
    hit_moved = (t >= k0) & (t < k0 + 64)
    assert hit_moved.sum() > 0          # the moved block is seen
    # the same triangles uploaded fresh give the same result
    c2 = grca.Caster(0)
    ids2 = [c2.add_sensor(s) for s in sc.sensors]
    c2.upload(t9)
    d2, t2 = _cast(c2, ids2, fl)
    assert np.array_equal(t, t2) and np.array_equal(d, d2)


def test_group_cull_elevation_and_gating():
    """A narrow-FOV sensor (8 channels within +-2 deg, 120 deg wide, 1 km
    range) and a block of small triangles 45 deg above it: the block's groups
    lie above every channel and are dropped by the elevation part of the
    group test; results stay identical to the brute force.  With unlimited
    range on every sensor of the cast the group test does not run."""
    from paper_2605_10457_gb300 import grca
    sc = scene_c1()
    narrow = make_sensor((0.0, 0.0, 1.8), elev=np.deg2rad(np.linspace(-2.0, 2.0, 8)), n_rays=512, fov_deg=120.0,
                         d_max=1000.0)
    rng = np.random.default_rng(4)
    high = (np.array([30.0, 0.0, 31.8]) + rng.normal(0.0, 0.3, (96, 3, 3))).astype(np.float32)
    tris = np.concatenate([sc.tris(0), high])
    c = grca.Caster(0)
    ids = [c.add_sensor(narrow), c.add_sensor(sc.sensors[0])]
    c.upload(tris)
    d, t = _cast(c, ids, 0)
    st = c.stats()
    db, tb = _cast(c, ids, grca.CAST_BRUTE)
    assert np.array_equal(t, tb) and np.array_equal(d, db)
    assert st["group_culled"] >= 2 * 64      # at least the two whole high groups, for both sensors
    d2, t2 = _cast(c, [ids[1]], 0)           # unlimited range only: no group test
    assert c.stats()["group_culled"] == 0
    assert np.array_equal(t2, t[narrow.n_total:])
