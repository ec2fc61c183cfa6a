"""GPU parity of the sensor variants against the FP64 oracle:

  - ray masks of non-spinning / patterned sensors (App. A.3): rays that do not
    fire are misses, the rest are unchanged; masks from host and device memory,
    animated between CUDA-graph replays;
  - horizontal and vertical angular noise (App. A.1, Eq. noise_search): per-ray
    perturbed azimuths and per-channel perturbed elevations, checked on every
    ray of the small scene and for the culling superset (culled == brute);
  - range noise (App. A.1, post-processing): the added offset equals sigma * z
    with z from the oracle's own counter-based generator.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from grading import grade, stratified_rays
from scenes import make_config, noisy_sensor, ray_mask, scene_c1

pytestmark = pytest.mark.gpu


def _caster(**opts):
    from paper_2605_10457_gb300 import grca
    return grca.Caster(0, **opts)


def _cast(c, ids, flags):
    import torch
    d, t = c.cast(ids, flags)
    torch.cuda.synchronize()
    return d.cpu().numpy(), t.cpu().numpy().view(np.uint32)


def _setup(scene, frame=0):
    c = _caster()
    ids = [c.add_sensor(s) for s in scene.sensors]
    tris = scene.tris(frame)
    c.upload(tris)
    return c, ids, tris


def _grade(sensors, tris, d, t, rays=None, masks=None):
    orc = oracle.Oracle(sensors, masks=masks)
    ref = oracle.cast(orc, tris, rays, ties=True)
    return grade(orc, tris, ref, d[ref["ray_ids"]], t[ref["ray_ids"]])


def _bits(m, n):
    q = np.arange(n)
    return ((m[q >> 5] >> (q & 31).astype(np.uint32)) & 1).astype(bool)


def test_ray_masks_host_device_and_animated():
    import torch
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_GRAPH
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    s = sc.sensors[0]
    d_full, t_full = _cast(c, ids, CAST_FP64_RECHECK)
    for step, kind in enumerate(("random", "sector", "stripes")):
        m = ray_mask(s, step, 0.4, kind)
        if step % 2:
            c.set_ray_mask(ids[0], torch.from_numpy(m.view(np.int32)).cuda())
        else:
            c.set_ray_mask(ids[0], m)
        for flags in (CAST_FP64_RECHECK, CAST_FP64_RECHECK | CAST_GRAPH):
            d, t = _cast(c, ids, flags)
            on = _bits(m, s.n_total)
            assert np.all(t[~on] == oracle.NO_HIT) and np.all(np.isinf(d[~on]))
            assert np.array_equal(t[on], t_full[on]) and np.array_equal(d[on], d_full[on])
            g = _grade(sc.sensors, tris, d, t, masks=[m])
            assert g["errors"] == 0, g
    c.set_ray_mask(ids[0], None)
    d, t = _cast(c, ids, CAST_FP64_RECHECK | CAST_GRAPH)
    assert np.array_equal(t, t_full)


def test_angular_noise_all_rays_c1():
    """Perturbed azimuths (within 0.45 dtheta) and elevations on the 16 x 512
    sensor: every ray against the oracle, FP64 recheck on."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    base = scene_c1()
    sc = dataclasses.replace(base, sensors=[noisy_sensor(s, 21) for s in base.sensors])
    c, ids, tris = _setup(sc)
    d, t = _cast(c, ids, CAST_FP64_RECHECK)
    assert c.stats()["device_error"] == 0
    g = _grade(sc.sensors, tris, d, t)
    assert g["errors"] == 0, g
    d0, t0 = _cast(_setup(base)[0], [0], CAST_FP64_RECHECK)
    assert np.count_nonzero(t0 != t) > 100          # the noise moved the rays


@pytest.mark.parametrize("cfg", ["c1", "c4m"])
def test_angular_noise_culled_equals_brute(cfg):
    """With noise the culling spans widen by the largest perturbation; the
    no-cull brute force runs the same FP32 test on every pair, so a hit lost by
    a too-narrow span shows up as a difference."""
    from paper_2605_10457_gb300.grca import CAST_BRUTE
    base = make_config(cfg)
    sc = dataclasses.replace(base, sensors=[noisy_sensor(s, 7 + k) for k, s in enumerate(base.sensors)])
    c, ids, tris = _setup(sc, frame=2)
    d, t = _cast(c, ids, 0)
    db, tb = _cast(c, ids, CAST_BRUTE)
    assert np.array_equal(t, tb) and np.array_equal(d, db)
    if cfg == "c4m":
        from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
        d, t = _cast(c, ids, CAST_FP64_RECHECK)
        g = _grade(sc.sensors, tris, d, t, rays=stratified_rays(sc.sensors, 300, seed=9))
        assert g["errors"] == 0, g


def test_range_noise_matches_generator():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_GRAPH
    sc = make_config("c4m")
    c, ids, tris = _setup(sc, frame=3)
    d0, t0 = _cast(c, ids, CAST_FP64_RECHECK)
    sig = [0.02 * (k + 1) for k in range(len(ids))]
    seeds = [1000 + 77 * k for k in range(len(ids))]
    for k, sid in enumerate(ids):
        c.set_range_noise(sid, sig[k], seeds[k])
    for flags in (CAST_FP64_RECHECK, CAST_FP64_RECHECK | CAST_GRAPH):
        d1, t1 = _cast(c, ids, flags)
        assert np.array_equal(t0, t1)
        off = 0
        for k, s in enumerate(sc.sensors):
            sl = slice(off, off + s.n_total)
            off += s.n_total
            hit = t0[sl] != oracle.NO_HIT
            q = np.nonzero(hit)[0]
            z = oracle.range_noise(seeds[k], q)
            a, b = d0[sl][hit].astype(np.float64), d1[sl][hit].astype(np.float64)
            tol = np.spacing(np.abs(b).astype(np.float32)).astype(np.float64) + 1e-5 * sig[k] * (1 + np.abs(z))
            assert np.all(np.abs(b - a - sig[k] * z) <= tol), np.max(np.abs(b - a - sig[k] * z) - tol)
            assert np.all(np.isinf(d1[sl][~hit]))
            assert abs(np.std(b - a) / sig[k] - 1.0) < 0.05
    # a new seed gives fresh noise; sigma 0 restores the exact distances
    c.set_range_noise(ids[0], sig[0], seeds[0] + 1)
    d2, _ = _cast(c, ids, CAST_FP64_RECHECK)
    n0 = sc.sensors[0].n_total
    assert np.count_nonzero(d2[:n0] != d1[:n0]) > 0.5 * np.count_nonzero(np.isfinite(d1[:n0]))
    for sid in ids:
        c.set_range_noise(sid, 0.0, 0)
    d3, _ = _cast(c, ids, CAST_FP64_RECHECK | CAST_GRAPH)
    assert np.array_equal(d3, d0)


def test_mask_and_noise_together():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    s = sc.sensors[0]
    m = ray_mask(s, 5, 0.5)
    c.set_ray_mask(ids[0], m)
    c.set_range_noise(ids[0], 0.05, 99)
    d, t = _cast(c, ids, CAST_FP64_RECHECK)
    on = _bits(m, s.n_total)
    assert np.all(np.isinf(d[~on])) and np.all(t[~on] == oracle.NO_HIT)
    assert np.isfinite(d[on]).sum() > 1000


def test_sensor_variant_arguments_rejected():
    from paper_2605_10457_gb300.grca import GrcaError
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    s = sc.sensors[0]
    th = s.theta0 + np.arange(s.n_rays) * s.dtheta
    bad = th.copy()
    bad[3] += 1.01 * s.dtheta
    with pytest.raises(GrcaError):
        c.set_azimuths(ids[0], bad)
    bad = th.copy()
    bad[5] = np.nan
    with pytest.raises(GrcaError):
        c.set_azimuths(ids[0], bad)
    with pytest.raises(GrcaError):
        c.set_range_noise(ids[0], -1.0, 0)
    with pytest.raises(GrcaError):
        c.set_range_noise(99, 0.1, 0)
    with pytest.raises(ValueError):
        c.set_ray_mask(ids[0], np.zeros(3, np.uint32))
    # the uniform grid listed explicitly gives the uniform result
    d0, t0 = _cast(c, ids, 0)
    c.set_azimuths(ids[0], th)
    d1, t1 = _cast(c, ids, 0)
    c.set_azimuths(ids[0], None)
    d2, t2 = _cast(c, ids, 0)
    assert np.array_equal(t0, t2) and np.array_equal(d0, d2)
    assert np.count_nonzero(t0 != t1) <= 4     # listed values round like the grid's, up to silhouettes
