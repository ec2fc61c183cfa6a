"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

All inputs are seeded synthetic scenes from `scenes`.  Small scenes are
checked on every ray; larger ones on stratified ray samples the oracle can
brute-force in seconds.
"""
import math

import numpy as np
import pytest

import oracle
from grading import grade, stratified_rays
from scenes import make_config, make_sensor, scene_c1, tiny_scene, Sensor

pytestmark = pytest.mark.gpu


def _caster(**opts):
    from paper_2605_10457_gb300 import grca
    return grca.Caster(0, **opts)


def _cast(c, ids, flags):
    import torch
    d, t = c.cast(ids, flags)
    torch.cuda.synchronize()
    return d.cpu().numpy(), t.cpu().numpy().view(np.uint32)


def _setup(scene, frame=0, **opts):
    c = _caster(**opts)
    ids = [c.add_sensor(s) for s in scene.sensors]
    tris = scene.tris(frame)
    c.upload(tris)
    return c, ids, tris


def _check(scene, tris, d, t, ray_ids=None, cull=False, fp32=False):
    orc = oracle.Oracle(scene.sensors)
    ref = oracle.cast(orc, tris, ray_ids, cull_backface=cull, ties=True)
    rid = ref["ray_ids"]
    g = grade(orc, tris, ref, d[rid], t[rid], edge_eps=(2e-6 if fp32 else 1e-7),
              silhouette_eps=(2e-6 if fp32 else 1e-12), dist_rel=(1e-4 if fp32 else 1e-5))
    return g


# ---------------------------------------------------------------------------
def test_c1_fp64_recheck_all_rays():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    d, t = _cast(c, ids, CAST_FP64_RECHECK)
    st = c.stats()
    assert st["device_error"] == 0
    assert st["pairs"] == len(ids) * tris.shape[0]
    g = _check(sc, tris, d, t)
    assert g["errors"] == 0, g
    assert g["hits"] > 3000


def test_c1_plain_fp32_all_rays():
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    d, t = _cast(c, ids, 0)
    g = _check(sc, tris, d, t, fp32=True)
    assert g["errors"] <= 2, g   # FP32 only: reported, tolerance of the FP32 path


@pytest.mark.parametrize("cfg", ["c1", "c2m", "c3m", "c4m"])
def test_culling_never_drops_a_hit_brute_equals_culled(cfg):
    """Plain FP32: the culled path and the no-cull brute force run the same
    test on every pair, so any hit lost by a cull shows up as a difference."""
    from paper_2605_10457_gb300.grca import CAST_BRUTE
    sc = make_config(cfg)
    c, ids, tris = _setup(sc)
    if cfg in ("c3m", "c4m"):
        ids = ids[:2]   # brute force is O(rays x tris); two sensors suffice here
    d0, t0 = _cast(c, ids, 0)
    d1, t1 = _cast(c, ids, CAST_BRUTE)
    diff = np.nonzero((t0 != t1) | ~((d0 == d1) | (np.isinf(d0) & np.isinf(d1))))[0]
    assert diff.size == 0, (diff[:10], t0[diff[:10]], t1[diff[:10]], d0[diff[:10]], d1[diff[:10]])


@pytest.mark.parametrize("cfg", ["c4m", "c5m"])
def test_launch_configuration_does_not_change_the_result(cfg):
    """The autotuner's knobs only move work between paths: every pair is
    tested with the same bits whether its span is tested inline (inline_max
    1024) or deferred to the per-channel spans of k_expand/k_test
    (inline_max 4), and the closest-hit key minimum and the re-test filter do
    not depend on the order of the commits.  Outputs are equal bit for bit."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_GRAPH
    sc = make_config(cfg)
    knobs = [dict(),
             dict(inline_max=4, chunk_rays=32, cull_block=128, cull_blocks_per_sm=2),
             dict(inline_max=1024, chunk_rays=256, cull_block=256, cull_blocks_per_sm=16)]
    for fl in (0, CAST_FP64_RECHECK | CAST_GRAPH):
        ref = None
        for k in knobs:
            c, ids, tris = _setup(sc, big_pair_capacity=1 << 20, chunk_capacity=16 << 20, **k)
            d, t = _cast(c, ids, fl)
            st = c.stats()
            if k.get("inline_max") == 4:
                assert st["big_pairs"] > 0     # the deferred path carries part of the work
            if ref is None:
                ref = (d, t)
                continue
            assert np.array_equal(t, ref[1]), (k, fl, np.nonzero(t != ref[1])[0][:8])
            assert np.array_equal(d.view(np.uint32), ref[0].view(np.uint32)), (k, fl)


@pytest.mark.parametrize("cfg", ["c4m", "c5m"])
def test_occlusion_drop_does_not_change_the_result(cfg):
    """An FP32 + re-test cast drops a live pair of at most 4 candidate rays
    before its setup when each of those rays already holds a certain hit
    closer than the pair's distance lower bound by more than the tie band.
    Such a pair could neither win, tie nor be kept for the re-test, so the
    output equals the cast that tests every pair (GRCA_CAST_NO_OCCLUSION),
    bit for bit, over several animated frames and two launch configurations."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_GRAPH, CAST_NO_OCCLUSION
    sc = make_config(cfg)
    for k in (dict(), dict(inline_max=1024, chunk_rays=256, cull_block=256, cull_blocks_per_sm=16)):
        c, ids, tris = _setup(sc, big_pair_capacity=1 << 20, chunk_capacity=16 << 20, **k)
        for frame in (0, 7):
            c.update(sc.tris(frame), 0)
            d0, t0 = _cast(c, ids, CAST_FP64_RECHECK | CAST_GRAPH)
            st0 = c.stats()
            d1, t1 = _cast(c, ids, CAST_FP64_RECHECK | CAST_GRAPH | CAST_NO_OCCLUSION)
            st1 = c.stats()
            assert st0["pairs_occluded"] > 0 and st1["pairs_occluded"] == 0, (st0, st1)
            assert st0["pairs_live"] == st1["pairs_live"] and st0["tests"] < st1["tests"]
            assert np.array_equal(t0, t1), (cfg, k, frame, np.nonzero(t0 != t1)[0][:8])
            assert np.array_equal(d0.view(np.uint32), d1.view(np.uint32)), (cfg, k, frame)
            assert st0["flagged_rays"] == st1["flagged_rays"]
        # the plain FP32 path drops nothing this way
        _cast(c, ids, 0)
        assert c.stats()["pairs_occluded"] == 0
        c.close()


def test_tiny_random_scenes_brute_equals_culled():
    from paper_2605_10457_gb300.grca import CAST_BRUTE, CAST_FP64_RECHECK
    for seed in range(6):
        tris = tiny_scene(seed, n_tris=300, extent=6.0)
        sens = [make_sensor((0.0, 0.0, 0.5), channels="c32", n_rays=720),
                make_sensor((0.3, -0.2, 1.0), yaw=0.4, channels="c64", n_rays=512, fov_deg=180.0),
                make_sensor((-0.5, 0.1, 0.2), yaw=-1.0, channels="uniform16", n_rays=360, pitch=0.3, roll=-0.2)]
        c = _caster()
        ids = [c.add_sensor(s) for s in sens]
        c.upload(tris)
        for fl in (0, CAST_FP64_RECHECK):
            d0, t0 = _cast(c, ids, fl)
            d1, t1 = _cast(c, ids, fl | CAST_BRUTE)
            assert np.array_equal(t0, t1), (seed, fl, np.nonzero(t0 != t1)[0][:8])
        sc = type("S", (), {"sensors": sens})
        g = _check(sc, tris, d0, t0)
        assert g["errors"] == 0, (seed, g)


def test_geometry_at_the_sensor_origin_brute_equals_culled():
    """Triangles at a sensor's origin: a vertex exactly at it (its plane
    passes through the origin: no hit from there), triangles 1e-7 .. 1e-5
    and 1e-16 .. 1e-12 across around it, and microscopic ones 1e-20 across,
    whose |w|^2 and the products of the FP32 bounds are subnormal or zero.
    No hit is lost: culled == brute in both modes, and the FP32 + FP64
    re-test cast grades with zero errors against the oracle (the FP64 re-test
    settles the pairs whose FP32 test underflows).  Each triangle spans a
    small range of magnitudes, so the FP64 oracle stays exact on it."""
    from paper_2605_10457_gb300.grca import CAST_BRUTE, CAST_FP64_RECHECK
    rng = np.random.default_rng(17)
    n1, n2, n3, n4 = 20, 10, 8, 8
    parts = [tiny_scene(4, n_tris=200, extent=6.0)]
    parts.append(np.concatenate([np.zeros((n1, 1, 3)), rng.normal(0.0, 2.0, (n1, 2, 3))], 1))
    c2 = np.stack([rng.normal(0.0, 0.5, n2), rng.uniform(2.0, 5.0, n2), rng.normal(0.0, 0.5, n2)], -1)[:, None, :]
    parts.append((c2 + 0.7 * rng.normal(0.0, 1.0, (n2, 3, 3))) * 10.0 ** rng.uniform(-16, -12, (n2, 1, 1)))
    c3 = np.stack([-rng.uniform(2.0, 5.0, n3), rng.normal(0.0, 0.5, n3), rng.normal(0.0, 0.5, n3)], -1)[:, None, :]
    parts.append((c3 + 0.7 * rng.normal(0.0, 1.0, (n3, 3, 3))) * 1e-20)
    c4 = np.stack([rng.uniform(2.0, 5.0, n4), -rng.uniform(2.0, 5.0, n4), rng.normal(0.0, 0.3, n4)], -1)[:, None, :]
    parts.append((c4 + 0.7 * rng.normal(0.0, 1.0, (n4, 3, 3))) * 10.0 ** rng.uniform(-7, -5, (n4, 1, 1)))
    tris = np.ascontiguousarray(np.concatenate(parts, 0).astype(np.float32))
    sens = [make_sensor((0.0, 0.0, 0.0), channels="c32", n_rays=360),
            make_sensor((0.0, 0.0, 0.0), yaw=0.7, channels="uniform16", n_rays=256, pitch=0.3, roll=-0.2),
            make_sensor((0.4, -0.3, 0.2), channels="c32", n_rays=360)]
    c = _caster()
    ids = [c.add_sensor(s) for s in sens]
    c.upload(tris)
    for fl in (0, CAST_FP64_RECHECK):
        d0, t0 = _cast(c, ids, fl)
        assert c.stats()["device_error"] == 0
        d1, t1 = _cast(c, ids, fl | CAST_BRUTE)
        assert np.array_equal(t0, t1), (fl, np.nonzero(t0 != t1)[0][:8])
    b = 200 + n1
    for lo, hi in ((b, b + n2), (b + n2, b + n2 + n3), (b + n2 + n3, b + n2 + n3 + n4)):
        assert np.isin(t0, np.arange(lo, hi)).sum() > 300   # each kind of small triangle is hit
    sc = type("S", (), {"sensors": sens})
    g = _check(sc, tris, d0, t0)
    assert g["errors"] == 0, g


def test_far_from_the_world_origin_brute_equals_culled():
    """Sensors and scene about 3 km from the world origin, where the FP32
    origin's low part o_lo reaches 1e-4 m: the elevation and range culls
    widen their bounds by |o_lo| instead of subtracting it per vertex, and
    must still keep every hit (culled == no-cull, bit for bit), with and
    without range limits and for tilted sensors."""
    from paper_2605_10457_gb300.grca import CAST_BRUTE, CAST_FP64_RECHECK
    off = np.array([2345.678, -1987.654, 12.345])
    for seed in range(3):
        tris = (tiny_scene(seed, n_tris=300, extent=6.0).astype(np.float64) + off).astype(np.float32)
        sens = [make_sensor(off + (0.0, 0.0, 0.5), channels="c32", n_rays=720),
                make_sensor(off + (0.3, -0.2, 1.0), yaw=0.4, channels="c64", n_rays=512, fov_deg=180.0,
                            d_min=0.3, d_max=4.0),
                make_sensor(off + (-0.5, 0.1, 0.2), yaw=-1.0, channels="uniform16", n_rays=360, pitch=0.3,
                            roll=-0.2, d_max=7.0)]
        c = _caster()
        ids = [c.add_sensor(s) for s in sens]
        c.upload(tris)
        for fl in (0, CAST_FP64_RECHECK):
            d0, t0 = _cast(c, ids, fl)
            d1, t1 = _cast(c, ids, fl | CAST_BRUTE)
            assert np.array_equal(t0, t1), (seed, fl, np.nonzero(t0 != t1)[0][:8])
        assert (t0 != 0xFFFFFFFF).sum() > 1000
        sc = type("S", (), {"sensors": sens})
        g = _check(sc, tris, d0, t0)
        assert g["errors"] == 0, (seed, g)


def _grid_wall(x0, x1, z0, z1, y, nx, nz, yaw):
    """Vertical wall y = const (before a yaw about z), nx x nz quads, shared edges."""
    xs, zs = np.linspace(x0, x1, nx + 1), np.linspace(z0, z1, nz + 1)
    c, s_ = math.cos(yaw), math.sin(yaw)
    P = np.array([[[x * c - y * s_, x * s_ + y * c, z] for x in xs] for z in zs])
    tris = []
    for a in range(nz):
        for b in range(nx):
            p00, p01, p10, p11 = P[a, b], P[a, b + 1], P[a + 1, b], P[a + 1, b + 1]
            tris += [[p00, p01, p11], [p00, p11, p10]]
    return np.asarray(tris, np.float32)


def test_grazing_hits_get_exact_distances_without_the_fp64_queue():
    """Rays that meet long yawed walls and the ground at a few degrees of
    incidence: the FP32 distance bound exceeds the accepted one there, and
    the double-float re-evaluation of t must settle every such hit (no entry
    of cause t kept for the FP64 re-test), with distances within 1e-6
    relative of the FP64 oracle and zero errors under the grading rule."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    walls = np.concatenate([_grid_wall(-40.0, 300.0, 0.0, 4.0, 3.0, 170, 4, 0.013),
                            _grid_wall(-40.0, 300.0, 0.0, 4.0, -5.0, 170, 4, -0.021)])
    xs = np.linspace(-60.0, 320.0, 39)
    ys = np.linspace(-40.0, 40.0, 9)
    ground = []
    for a_ in range(len(xs) - 1):
        for b in range(len(ys) - 1):
            p = [(xs[a_], ys[b], 0.0), (xs[a_ + 1], ys[b], 0.0), (xs[a_ + 1], ys[b + 1], 0.0), (xs[a_], ys[b + 1], 0.0)]
            ground += [[p[0], p[1], p[2]], [p[0], p[2], p[3]]]
    # the whole scene turned by psi about z, the sensors pitched and rolled a
    # little: no axis-aligned direction is left to make the FP32 bound small
    psi = 0.7
    cz, sz = math.cos(psi), math.sin(psi)
    R = np.array([[cz, -sz, 0.0], [sz, cz, 0.0], [0.0, 0.0, 1.0]])
    tris = np.concatenate([walls, np.asarray(ground, np.float32)]).astype(np.float64) @ R.T
    tris = tris.astype(np.float32)
    sens = [make_sensor(R @ (0.0, 0.0, 1.5), yaw=psi + 0.0021, channels="c64", n_rays=2048, fov_deg=30.0,
                        pitch=0.05, roll=-0.03),
            make_sensor(R @ (5.0, -1.0, 2.0), yaw=psi - 0.0137, channels="c32", n_rays=1024, fov_deg=20.0,
                        pitch=0.02, roll=0.04)]
    c = _caster()
    ids = [c.add_sensor(s) for s in sens]
    c.upload(tris)
    d, t = _cast(c, ids, CAST_FP64_RECHECK)
    st = c.stats()
    assert st["device_error"] == 0
    assert st["queued_t"] > 200 and st["t_refined"] == st["queued_t"] and st["kept_t"] == 0, st
    sc = type("S", (), {"sensors": sens})
    orc = oracle.Oracle(sens)
    ref = oracle.cast(orc, tris, None, ties=True)
    g = grade(orc, tris, ref, d, t)
    assert g["errors"] == 0, g
    same = (t.astype(np.int64) == ref["id"].astype(np.int64)) & (t != 0xFFFFFFFF)
    assert same.sum() > 20000
    rel = np.abs(d[same] - ref["t"][same]) / ref["t"][same]
    assert rel.max() <= 1e-6, rel.max()


@pytest.mark.parametrize("cfg", ["c1", "c2m", "c3m", "c4m", "c5m"])
def test_candidate_spans_cover_every_exact_hit(cfg):
    """Every (ray, triangle) pair that the FP64 oracle finds hitting must be
    among the candidates the culling passes emit (debug dump), for every
    sensor of the scene: the culls never drop a true hit, whatever the test
    then decides."""
    import torch
    from paper_2605_10457_gb300.grca import CAST_DUMP_CANDIDATES
    sc = scene_c1() if cfg == "c1" else make_config(cfg)
    c, ids, tris = _setup(sc, frame=0 if cfg == "c1" else 2)
    cap = 24_000_000
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    c.set_debug_dump(pairs, cnt)
    _cast(c, ids, CAST_DUMP_CANDIDATES)
    n = int(cnt.item())
    assert 0 < n <= cap
    got = pairs[:2 * n].view(-1, 2).cpu().numpy().astype(np.int64)
    cand = np.unique((got[:, 1] << 32) | got[:, 0])
    off = 0
    # every sensor on the small scenes; the first two (of eight) on c4m / c5m,
    # whose all-pairs oracle pass takes about 10 s per sensor
    for s in sc.sensors[:2] if cfg in ("c4m", "c5m") else sc.sensors:
        hits = oracle.triangle_hits(s, tris)   # (triangle, local ray id)
        need = (hits[:, 0] << 32) | (hits[:, 1] + off)
        missing = need[~np.isin(need, cand)]
        assert missing.size == 0, (cfg, off, missing[:10])
        off += s.n_channels * s.n_rays
    c.set_debug_dump(None)


@pytest.mark.parametrize("cfg,n_sample", [("c2m", None), ("c3m", 3000), ("c4m", 2500), ("c5m", 2500)])
def test_minis_fp64_recheck(cfg, n_sample):
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = make_config(cfg)
    c, ids, tris = _setup(sc, frame=7)
    d, t = _cast(c, ids, CAST_FP64_RECHECK)
    assert c.stats()["device_error"] == 0
    rays = None
    if n_sample:
        rays = stratified_rays(sc.sensors, n_sample // len(sc.sensors), seed=3)
        if sc.stress_rays is not None:
            rays = np.unique(np.concatenate([rays, sc.stress_rays]))
    g = _check(sc, tris, d, t, rays)
    assert g["errors"] == 0, g


@pytest.mark.parametrize("d_max", [10.0, 50.0])
def test_range_cull_c4m(d_max):
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = make_config("c4m")
    for s in sc.sensors:
        s.d_min, s.d_max = 0.05, d_max
    c, ids, tris = _setup(sc, frame=2)
    d, t = _cast(c, ids, CAST_FP64_RECHECK)
    assert np.all(d[np.isfinite(d)] <= d_max * (1 + 1e-6))
    rays = stratified_rays(sc.sensors, 300, seed=5)
    g = _check(sc, tris, d, t, rays)
    assert g["errors"] == 0, g


def test_lossy_apparent_area_mode():
    """GRCA_CAST_LOSSY_AREA (App. A.4.1 Step 1, Eq. apparent_area): the result
    equals the oracle over the triangles the FP64 filter keeps, except on rays
    whose outcome involves a triangle within 1e-3 of the threshold (there FP32
    and FP64 may decide differently).  Also reports the paper's Hit% floor
    against the exact result (distance within 1 mm)."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_LOSSY_AREA
    eps = 1e-5
    sc = make_config("c4m")
    c, ids, tris = _setup(sc, frame=1, area_eps=eps)
    d, t = _cast(c, ids, CAST_FP64_RECHECK | CAST_LOSSY_AREA)
    st = c.stats()
    d_exact, t_exact = _cast(c, ids, CAST_FP64_RECHECK)
    st_exact = c.stats()
    assert st["pairs_live"] < st_exact["pairs_live"]
    keep = oracle.area_keep(sc.sensors, tris, eps)
    rays = stratified_rays(sc.sensors, 400, seed=11)
    orc = oracle.Oracle(sc.sensors)
    bad = None
    for kmask in ((keep > 0), (keep == 1)):
        ref = oracle.cast(orc, tris, rays, ties=True, keep=kmask.astype(np.uint8))
        g = grade(orc, tris, ref, d[rays], t[rays])
        bad = set(g["bad_ids"]) if bad is None else bad & set(g["bad_ids"])
    assert not bad, sorted(bad)[:10]
    # Hit% (paper: hit distance within 1 mm of the exact one, or both miss)
    m_exact = np.isfinite(d_exact[rays])
    m_lossy = np.isfinite(d[rays])
    close = np.zeros(rays.shape[0], bool)
    both = m_exact & m_lossy
    close[both] = np.abs(d[rays][both] - d_exact[rays][both]) <= 1e-3
    same = (~m_exact & ~m_lossy) | close
    print(f"lossy eps={eps}: Hit% = {100 * same.mean():.2f}, live pairs {st['pairs_live']} vs {st_exact['pairs_live']}")
    assert same.mean() > 0.5


def test_backface_cull_c1():
    from paper_2605_10457_gb300.grca import CAST_CULL_BACKFACE, CAST_FP64_RECHECK
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    d, t = _cast(c, ids, CAST_FP64_RECHECK | CAST_CULL_BACKFACE)
    g = _check(sc, tris, d, t, cull=True)
    assert g["errors"] == 0, g
    d2, t2 = _cast(c, ids, CAST_FP64_RECHECK)
    assert np.array_equal(t, t2)   # closed outward meshes seen from outside


def test_graph_replay_and_vertex_update():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_GRAPH
    import torch
    sc = make_config("c2m")
    c, ids, tris = _setup(sc)
    out = c.outputs(ids)
    fl = CAST_FP64_RECHECK
    c.cast(ids, fl | CAST_GRAPH, out)
    c.cast(ids, fl | CAST_GRAPH, out)
    torch.cuda.synchronize()
    a = out[1].cpu().numpy().view(np.uint32).copy()
    d_ng, t_ng = _cast(c, ids, fl)
    assert np.array_equal(a, t_ng)
    # animate: frame 5 through update_vertices, then replay the same graph
    tr5 = sc.tris(5)
    c.update(tr5[sc.n_static:], sc.n_static)
    c.cast(ids, fl | CAST_GRAPH, out)
    torch.cuda.synchronize()
    d5 = out[0].cpu().numpy()
    t5 = out[1].cpu().numpy().view(np.uint32)
    d5n, t5n = _cast(c, ids, fl)
    assert np.array_equal(t5, t5n)
    rays = stratified_rays(sc.sensors, 2000, seed=9)
    g = _check(sc, tr5, d5, t5, rays)
    assert g["errors"] == 0, g


def test_pose_change_and_partial_fov():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = scene_c1()
    c, ids, tris = _setup(sc)
    s90 = make_sensor((1.0, 2.0, 1.2), yaw=0.9, channels="c32", n_rays=300, fov_deg=90.0)
    s270 = make_sensor((-3.0, 1.0, 2.5), yaw=2.0, channels="c64", n_rays=900, fov_deg=270.0, pitch=0.15, roll=0.1)
    i90, i270 = c.add_sensor(s90), c.add_sensor(s270)
    # move the first sensor
    s0 = sc.sensors[0]
    new = make_sensor((2.5, -1.0, 1.5), yaw=-0.7, channels="uniform16", n_rays=512, pitch=-0.05)
    c.set_pose(ids[0], new.origin, new.f, new.r, new.u)
    allids = [ids[0], i90, i270]
    d, t = _cast(c, allids, CAST_FP64_RECHECK)
    S = type("S", (), {"sensors": [c.sensors[i] for i in allids]})
    g = _check(S, tris, d, t)
    assert g["errors"] == 0, g


def test_edge_cases():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    import torch
    sens = make_sensor((0.0, 0.0, 1.0), channels="uniform16", n_rays=64)
    c = _caster()
    sid = c.add_sensor(sens)
    # no triangles: all misses
    c.upload(np.zeros((0, 3, 3), np.float32))
    d, t = _cast(c, [sid], CAST_FP64_RECHECK)
    assert np.all(np.isinf(d)) and np.all(t == 0xFFFFFFFF)
    # zero-area triangles never hit; one valid triangle in front
    tris = np.array([[[3, 0, 1], [3, 0, 1], [3, 1, 1]],          # repeated vertex
                     [[3, -1, 0], [3, 0, 1], [3, 1, 2]],         # collinear
                     [[3, -1, -1], [3, 1, -1], [3, 0, 3]]], np.float32)
    c.upload(tris)
    d, t = _cast(c, [sid], CAST_FP64_RECHECK)
    assert set(np.unique(t).tolist()) <= {2, 0xFFFFFFFF} and np.any(t == 2)
    # extreme grids: 1024 channels x 64 rays, 4 channels x 32768 rays
    s1 = make_sensor((0.0, 0.0, 0.0), elev=np.linspace(-1.5, 1.5, 1024), n_rays=64)
    s2 = make_sensor((0.0, 0.0, 0.0), elev=np.deg2rad([-3.0, -1.0, 1.0, 3.0]), n_rays=32768)
    tris = tiny_scene(11, n_tris=500, extent=5.0)
    c2 = _caster()
    ids = [c2.add_sensor(s1), c2.add_sensor(s2)]
    c2.upload(tris)
    d, t = _cast(c2, ids, CAST_FP64_RECHECK)
    S = type("S", (), {"sensors": [s1, s2]})
    rays = stratified_rays([s1, s2], 3000, seed=1)
    g = _check(S, tris, d, t, rays)
    assert g["errors"] == 0, g


def test_brute_mode_on_the_largest_grid():
    """The no-cull debug mode tests every pair inline, so one pair's span is
    the whole grid: 1024 x 32768 = 2^25 candidates, beyond the range where
    the expansion's float quotient is exact by itself.  Brute force and the
    culled path agree bit for bit."""
    from paper_2605_10457_gb300.grca import CAST_BRUTE
    s = make_sensor((0.0, 0.0, 0.0), elev=np.linspace(-1.2, 1.2, 1024), n_rays=32768)
    tris = np.array([[[4, -1, -1], [4, 1, -1], [4, 0, 1.5]],
                     [[-3, 2, -2], [-3, -2, -2], [-3, 0, 2]],
                     [[0.5, 5, -0.4], [-0.5, 5, -0.4], [0, 5, 0.6]]], np.float32)
    c = _caster()
    sid = c.add_sensor(s)
    c.upload(tris)
    d0, t0 = _cast(c, [sid], 0)
    d1, t1 = _cast(c, [sid], CAST_BRUTE)
    assert np.count_nonzero(t0 != 0xFFFFFFFF) > 1000
    assert np.array_equal(t0, t1) and np.array_equal(d0.view(np.uint32), d1.view(np.uint32))


def test_sixty_four_sensors_in_one_cast():
    """The largest batch one cast takes (64 sensors), of mixed grids, poses,
    fields of view and ranges, every ray against the oracle."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK, CAST_GRAPH
    rng = np.random.default_rng(64)
    sens = []
    for k in range(64):
        n_ch = int(rng.choice([2, 4, 8]))
        elev = np.sort(rng.uniform(-0.4, 0.3, n_ch))
        fov = float(rng.choice([360.0, 180.0, 90.0]))
        d_max = float(rng.choice([np.inf, 8.0, 3.0]))
        sens.append(make_sensor(rng.uniform(-3, 3, 3) * [1, 1, 0.2] + [0, 0, 1], yaw=float(rng.uniform(-3, 3)),
                                elev=elev, n_rays=int(rng.choice([32, 64, 96])), fov_deg=fov,
                                d_min=float(rng.choice([0.0, 0.5])), d_max=d_max,
                                pitch=float(rng.uniform(-0.2, 0.2))))
    tris = tiny_scene(64, n_tris=600, extent=8.0)
    c = _caster()
    ids = [c.add_sensor(s) for s in sens]
    c.upload(tris)
    d, t = _cast(c, ids, CAST_FP64_RECHECK | CAST_GRAPH)
    assert c.stats()["device_error"] == 0
    S = type("S", (), {"sensors": sens})
    g = _check(S, tris, d, t)
    assert g["errors"] == 0, g
    assert g["hits"] > 1000
    with pytest.raises(Exception):
        c.cast(ids + [ids[0]], CAST_FP64_RECHECK)        # 65 sensors: rejected


def test_non_finite_vertices_never_hit():
    """Triangles with NaN or infinite vertices never hit (the oracle's plane and
    edge tests fail on them) and do not disturb the culls, the spans, the
    group boxes or the hierarchy: every other ray matches the oracle."""
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = scene_c1()
    tris = sc.tris(0).copy()
    rng = np.random.default_rng(9)
    bad = rng.choice(tris.shape[0], 300, replace=False)
    vals = np.array([np.nan, np.inf, -np.inf], np.float32)
    for k, b in enumerate(bad):
        tris[b, k % 3, (k // 3) % 3] = vals[k % 3]

    for d_max, hybrid in ((np.inf, False), (12.0, False), (np.inf, True)):
        sens = [make_sensor((0.0, 0.0, 1.8), channels="uniform16", n_rays=512, d_min=0.0, d_max=d_max)]
        c = _caster()
        ids = [c.add_sensor(s) for s in sens]
        c.upload(tris)
        if hybrid:
            c.build_static(tris.shape[0])
        d, t = _cast(c, ids, CAST_FP64_RECHECK)
        assert c.stats()["device_error"] == 0
        assert not np.isin(t, bad).any()
        S = type("S", (), {"sensors": sens})
        g = _check(S, tris, d, t)
        assert g["errors"] == 0, (d_max, hybrid, g)


def test_capacity_overflow_is_reported():
    from paper_2605_10457_gb300.grca import CAST_FP64_RECHECK
    sc = scene_c1()
    c, ids, tris = _setup(sc, big_pair_capacity=4, chunk_capacity=8, inline_max=4)
    _cast(c, ids, CAST_FP64_RECHECK)
    st = c.stats(check=False)
    assert st["status"] == -4 and st["device_error"] != 0
    # the next cast with room reports no error
    c2, ids2, _ = _setup(sc)
    _cast(c2, ids2, CAST_FP64_RECHECK)
    assert c2.stats(check=False)["status"] == 0


def test_bad_arguments_rejected():
    from paper_2605_10457_gb300 import grca
    c = _caster()
    bad = make_sensor((0, 0, 0), channels="c32", n_rays=64)
    bad.elev = bad.elev[::-1].copy()   # not ascending
    with pytest.raises(grca.GrcaError):
        c.add_sensor(bad)
    ok = c.add_sensor(make_sensor((0, 0, 0), channels="c32", n_rays=64))
    out = c.outputs([ok])
    with pytest.raises(grca.GrcaError):
        c.cast([ok + 5], 0, out)
    with pytest.raises(grca.GrcaError):
        c.set_pose(ok, (0, 0, 0), (1, 0, 0), (1, 0, 0), (0, 0, 1))   # not orthonormal


@pytest.mark.parametrize("mode", ["plain", "graph", "range", "hybrid", "full_update"])
def test_host_cast_matches_device_cast(mode):
    """grca_cast_host (host vertices in, host results out; the dynamic tail's
    copy overlaps the static triangles' elevation cull) gives bit-identical
    results to the device-side update + cast, frame after frame."""
    from paper_2605_10457_gb300 import grca
    sc = make_config("c4m")
    if mode == "range":
        for s in sc.sensors:
            s.d_min, s.d_max = 0.05, 12.0
    c_host, ids_h, _ = _setup(sc, frame=0)
    c_dev, ids_d, _ = _setup(sc, frame=0)
    ns = sc.n_static
    if mode == "hybrid":
        c_host.build_static(ns)
        c_dev.build_static(ns)
    fl = grca.CAST_FP64_RECHECK | (0 if mode == "plain" else grca.CAST_GRAPH)
    n = sum(s.n_total for s in sc.sensors)
    out_d = np.empty(n, np.float32)
    out_t = np.empty(n, np.uint32)
    for frame in (3, 11, 4):
        tris = sc.tris(frame)
        if mode == "full_update":
            c_host.cast_host(ids_h, tris, 0, out_d, out_t, fl)
        else:
            c_host.cast_host(ids_h, np.ascontiguousarray(tris[ns:]), ns, out_d, out_t, fl)
        c_dev.update(tris[ns:], ns)
        d, t = _cast(c_dev, ids_d, fl)
        assert np.array_equal(out_t, t) and np.array_equal(out_d, d), (mode, frame, np.count_nonzero(out_t != t))
    g = _check(sc, tris, out_d, out_t, stratified_rays(sc.sensors, 200, seed=6))
    assert g["errors"] == 0, g


@pytest.mark.parametrize("mode", ["plain", "range"])
def test_async_host_casts_match_sync(mode):
    """GRCA_CAST_HOST_ASYNC: frames enqueued back to back, each copying its
    results out on the context's own stream while the next one runs, give the
    same bits as synchronous host casts.  Eleven frames exceed the eight the
    context keeps in flight, and grca_host_wait bounds them in between."""
    from paper_2605_10457_gb300 import grca
    sc = make_config("c4m")
    if mode == "range":
        for s in sc.sensors:
            s.d_min, s.d_max = 0.05, 12.0
    c_a, ids_a, _ = _setup(sc, frame=0)
    c_s, ids_s, _ = _setup(sc, frame=0)
    ns = sc.n_static
    fl = grca.CAST_FP64_RECHECK | grca.CAST_GRAPH
    n = sum(s.n_total for s in sc.sensors)
    frames = (3, 11, 4, 9, 20, 1, 7, 15, 2, 30, 5)
    dyn = [np.ascontiguousarray(sc.tris(f)[ns:]) for f in frames]
    outs = [(np.empty(n, np.float32), np.empty(n, np.uint32)) for _ in frames]
    for k in range(len(frames)):
        c_a.cast_host(ids_a, dyn[k], ns, outs[k][0], outs[k][1], fl | grca.CAST_HOST_ASYNC)
        if k % 3 == 2:
            c_a.host_wait(2)
    c_a.host_wait(0)
    for k in range(len(frames)):
        d = np.empty(n, np.float32)
        t = np.empty(n, np.uint32)
        c_s.cast_host(ids_s, dyn[k], ns, d, t, fl)
        assert np.array_equal(outs[k][1], t) and np.array_equal(outs[k][0].view(np.uint32), d.view(np.uint32)), (mode, k)
    with pytest.raises(grca.GrcaError):
        c_a.cast(ids_a, fl | grca.CAST_HOST_ASYNC)   # the flag belongs to host casts only

