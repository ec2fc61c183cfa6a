"""Pins of the FP64 oracle against facts fixed by the paper and by geometry.

Each check takes an optional compiled oracle library so the planted-mistake
test can run the same checks on mutated copies of the oracle and show that
each plausible mistake fails at least one of them.  None of these checks
re-types the oracle's own formulas: distances come from closed forms of the
hand-placed geometry, hit sets from an independent linear solve, counts and
grid facts from the paper's printed worked example and statements.
"""
import json
import math
import os

import numpy as np

import oracle
from scenes import make_sensor, ray_mask, scene_c1, Sensor

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sensor(h=1.8, n_rays=64, elev_deg=(-30, -10, -2, 0, 3, 12), **kw):
    return make_sensor((0.0, 0.0, h), elev=np.deg2rad(np.array(elev_deg, float)), n_rays=n_rays, **kw)


def _quad(x0, x1, y0, y1, z):
    """Two triangles covering [x0,x1]x[y0,y1] at height z, normal +z."""
    a, b, c, d = (x0, y0, z), (x1, y0, z), (x1, y1, z), (x0, y1, z)
    return np.array([[a, b, c], [a, c, d]], np.float32)


def _wall(X, half=1000.0):
    """Two triangles in the plane x = X facing -x (toward a sensor near the origin)."""
    a, b, c, d = (X, -half, -half), (X, -half, half), (X, half, half), (X, half, -half)
    return np.array([[a, b, c], [a, c, d]], np.float32)


def check_brute_count(lib=None):
    g = json.load(open(os.path.join(GOLDEN, "brute_count.json")))
    total = g["omega"] * g["gamma"] * g["chi"] * g["tau"]
    digits = g["printed_significant_digits"]
    assert float(f"{total:.{digits}g}") == g["printed_total"]
    s1 = _sensor(n_rays=5, elev_deg=(-10, 0, 10))
    s2 = _sensor(n_rays=7, elev_deg=(-5, 5))
    tris = np.random.default_rng(0).normal(0, 3, (11, 3, 3)).astype(np.float32)
    r = oracle.cast(oracle.Oracle([s1, s2], lib), tris)
    assert r["tests"] == (3 * 5 + 2 * 7) * 11


def check_ray_grid(lib=None):
    g = json.load(open(os.path.join(GOLDEN, "ray_grid.json")))
    for c in g["cases"]:
        for yaw in (0.0, 0.7):
            s = make_sensor((1.0, -2.0, 3.0), yaw=yaw, channels="t128", n_rays=c["n_rays"])
            assert abs(s.theta0 + c["centre_ray"] * s.dtheta - c["centre_theta"]) < 1e-12
            zero = int(np.argmin(np.abs(s.elev)))
            assert s.elev[zero] == 0.0
            o = oracle.Oracle([s], lib)
            d = np.empty(3)
            o.lib.orc_ray_dir(o.ptr(0), zero, c["centre_ray"], d.ctypes.data)
            assert np.array_equal(d, s.f), (d, s.f)        # middle ray of the middle channel = f
            o.lib.orc_ray_dir(o.ptr(0), zero, c["quarter_ray"], d.ctypes.data)
            assert np.allclose(d, s.r, atol=1e-12), (d, s.r)  # +90 deg clockwise = right axis
            for j in (0, 40, 127):
                for i in (0, 17, c["n_rays"] - 1):
                    o.lib.orc_ray_dir(o.ptr(0), j, i, d.ctypes.data)
                    assert abs(np.linalg.norm(d) - 1.0) < 1e-14
                    assert abs(np.dot(d, s.u) - math.sin(s.elev[j])) < 1e-14   # channel = elevation


def check_ground(lib=None):
    h = 1.8
    s = _sensor(h=h)
    tris = _quad(-1e4, 1e4, -1e4, 1e4, 0.0)
    r = oracle.cast(oracle.Oracle([s], lib), tris)
    t = r["t"].reshape(s.n_channels, s.n_rays)
    ids = r["id"].reshape(s.n_channels, s.n_rays)
    for j, ph in enumerate(s.elev):
        if ph < 0:
            assert np.allclose(t[j], h / math.sin(-ph), rtol=1e-12, atol=0), (j, t[j][:3])
            assert np.all(ids[j] <= 1)
        else:
            assert np.all(np.isinf(t[j])) and np.all(ids[j] == oracle.NO_HIT)


def check_wall(lib=None):
    X = 7.25
    s = _sensor(h=0.5)
    tris = _wall(X)
    r = oracle.cast(oracle.Oracle([s], lib), tris)
    t = r["t"].reshape(s.n_channels, s.n_rays)
    for j, ph in enumerate(s.elev):
        for i in range(s.n_rays):
            th = s.theta0 + i * s.dtheta
            dx = math.cos(th) * math.cos(ph)
            if dx > 1e-9:
                assert abs(t[j, i] - X / dx) <= 1e-12 * (X / dx), (j, i, t[j, i], X / dx)
            elif dx < -1e-9:
                assert math.isinf(t[j, i])


def check_straddle(lib=None):
    """A tiny triangle centred on one exact ray is hit by that ray only; turned
    by +-1e-3 rad in azimuth it is missed."""
    s = _sensor(h=0.0, n_rays=256, elev_deg=(-4, 0, 4))
    j, i = 1, 100
    th = s.theta0 + i * s.dtheta
    L = 10.0
    for dturn, expect in ((0.0, True), (1e-3, False), (-1e-3, False)):
        a = th + dturn
        # world direction of azimuth a at 0 elevation: cos(a) f + sin(a) r
        c = L * (math.cos(a) * s.f + math.sin(a) * s.r) + s.origin
        e1 = 2e-3 * np.cross(s.u, (c - s.origin) / L)
        e2 = 2e-3 * s.u
        tri = np.array([[c - e1 - e2, c + e1 - e2, c + 2 * e2]], np.float32)
        r = oracle.cast(oracle.Oracle([s], lib), tri)
        ids = r["id"].reshape(s.n_channels, s.n_rays)
        assert (ids[j, i] == 0) == expect, (dturn, ids[j, i])
        assert int(np.sum(ids == 0)) == (1 if expect else 0)


def check_front(lib=None):
    s = _sensor(h=0.3, n_rays=32)
    tris = _wall(5.0, half=1e5)
    r = oracle.cast(oracle.Oracle([s], lib), tris)
    d = oracle.ray_dirs(oracle.Oracle([s], lib)).reshape(-1, 3)
    fwd = d[:, 0] > 1e-9
    assert np.all(np.isfinite(r["t"][fwd])) and np.all(np.isinf(r["t"][d[:, 0] < -1e-9]))


def check_coplanar_tie(lib=None):
    s = _sensor(h=0.0, n_rays=16, elev_deg=(0,))
    base = _wall(3.0, half=2.0)[0]
    other = np.array([[3.0, 5.0, 5.0], [3.0, 6.0, 5.0], [3.0, 5.0, 6.0]], np.float32)  # never hit
    tris = np.stack([other, base, base.copy(), other])
    r = oracle.cast(oracle.Oracle([s], lib), tris, ties=True)
    hit = np.isfinite(r["t"])
    assert hit.any()
    assert np.all(r["id"][hit] == 1)              # ties go to the lower id
    assert np.all(r["n_ties"][hit] == 2)
    assert np.all(r["second"][hit] == r["t"][hit])


def check_fan(lib=None):
    """Fan of 8 triangles around a hub on the forward axis (plane x=4): each ray
    landing inside the octagon is hit by the wedge that contains it."""
    s = _sensor(h=0.0, n_rays=720, elev_deg=tuple(np.linspace(-6, 6, 13)))
    m = 8
    R = 0.4
    rim = [np.array([4.0, R * math.cos(2 * math.pi * k / m), R * math.sin(2 * math.pi * k / m)]) for k in range(m)]
    hub = np.array([4.0, 0.0, 0.0])
    tris = np.array([[hub, rim[k], rim[(k + 1) % m]] for k in range(m)], np.float32)
    r = oracle.cast(oracle.Oracle([s], lib), tris)
    d = oracle.ray_dirs(oracle.Oracle([s], lib)).reshape(-1, 3)
    n_in = 0
    for q in range(d.shape[0]):
        if d[q, 0] <= 0:
            assert r["id"][q] == oracle.NO_HIT
            continue
        p = d[q] * (4.0 / d[q, 0])
        ang = math.atan2(p[2], p[1]) % (2 * math.pi)
        k = int(ang // (2 * math.pi / m))
        # inside the wedge's outer edge (chord between rim k and k+1)?
        a, b = rim[k][1:], rim[(k + 1) % m][1:]
        side = (b[0] - a[0]) * (p[2] - a[1]) - (b[1] - a[1]) * (p[1] - a[0])
        if side > 1e-9:
            n_in += 1
            assert r["id"][q] in (k, (k + 1) % m, (k - 1) % m), (q, r["id"][q], k)
            assert abs(r["t"][q] - 4.0 / d[q, 0]) < 1e-12 * r["t"][q]
        elif side < -1e-9:
            assert r["id"][q] == oracle.NO_HIT
    assert n_in > 5


def check_backface(lib=None):
    sc = scene_c1()
    o = oracle.Oracle(sc.sensors, lib)
    ids = np.arange(0, sc.n_rays, 7, dtype=np.int64)
    a = oracle.cast(o, sc.tris(), ids)
    b = oracle.cast(o, sc.tris(), ids, cull_backface=True)
    assert np.array_equal(a["id"], b["id"]) and np.array_equal(a["t"], b["t"])
    # a single triangle facing away: hit two-sided, culled one-sided
    s = _sensor(h=0.0, n_rays=8, elev_deg=(0,))
    tri = _wall(3.0)[:1]
    flipped = tri[:, [0, 2, 1]].copy()
    o1 = oracle.Oracle([s], lib)
    assert np.isfinite(oracle.cast(o1, tri, cull_backface=True)["t"]).any()
    assert np.isfinite(oracle.cast(o1, flipped)["t"]).any()
    assert not np.isfinite(oracle.cast(o1, flipped, cull_backface=True)["t"]).any()


def check_range(lib=None):
    h = 2.0
    s = _sensor(h=h, elev_deg=(-60, -30, -10, -5))
    t_true = h / np.sin(-s.elev)
    s.d_max = float(t_true[1] + 1e-6)      # channels 2,3 beyond d_max -> miss
    tris = _quad(-1e4, 1e4, -1e4, 1e4, 0.0)
    r = oracle.cast(oracle.Oracle([s], lib), tris)
    t = r["t"].reshape(s.n_channels, s.n_rays)
    assert np.all(np.isfinite(t[:2])) and np.all(np.isinf(t[2:]))
    # d_min: a near plane below d_min is skipped, the far plane behind it is hit
    s2 = _sensor(h=h, elev_deg=(-30,))
    two = np.concatenate([_quad(-1e4, 1e4, -1e4, 1e4, 1.0), _quad(-1e4, 1e4, -1e4, 1e4, 0.0)])
    s2.d_min = 3.0   # near plane at t=2, far plane at t=4
    r2 = oracle.cast(oracle.Oracle([s2], lib), two)
    assert np.allclose(r2["t"], 4.0, rtol=1e-12) and np.all(r2["id"] >= 2)


def check_linear_solve(lib=None):
    """Random rays x random triangles against an independent formulation:
    solve v0 + a e1 + b e2 = o + t d for (a, b, t); hit iff a,b >= 0, a+b <= 1, t > 0."""
    rng = np.random.default_rng(7)
    n_agree = 0
    for _ in range(3000):
        tri = rng.normal(0, 2, (3, 3)).astype(np.float32)
        o3 = rng.normal(0, 1, 3)
        tgt = tri.astype(np.float64).mean(0) + rng.normal(0, 1.5, 3)
        d3 = (tgt - o3) / np.linalg.norm(tgt - o3)
        v = tri.astype(np.float64)
        M = np.stack([v[1] - v[0], v[2] - v[0], -d3], 1)
        if abs(np.linalg.det(M)) < 1e-6:
            continue
        a, b, t = np.linalg.solve(M, o3 - v[0])
        margin = min(a, b, 1 - a - b)
        if abs(margin) < 1e-7 or abs(t) < 1e-7:
            continue
        expect = margin > 0 and t > 0
        got = oracle.hit(o3, d3, tri, lib=lib)
        assert (got is not None) == expect, (a, b, t, got)
        if expect:
            assert abs(got - t) <= 1e-9 * max(1.0, abs(t))
        n_agree += 1
    assert n_agree > 2000


def check_margin(lib=None):
    s = _sensor(h=0.0, n_rays=4, elev_deg=(0,))      # ray 2: theta = 0 -> d = f = +x
    o = oracle.Oracle([s], lib)
    for eps in (1e-3, 1e-6, -1e-4):
        # edge on the line y = -eps*x... : triangle in plane x=1 with an edge along y = eps
        tri = np.array([[1.0, eps, -1.0], [1.0, eps, 1.0], [1.0, eps + 1.0, 0.0]], np.float32)
        tp, m = oracle.ray_tri_margin(o, 2, tri)
        e32 = float(np.float32(eps))
        assert abs(tp - 1.0) < 1e-12
        assert abs(m - (-math.atan(e32))) < 1e-9, (eps, m)


def check_triangle_hits(lib=None):
    s = _sensor(h=1.0, n_rays=48)
    tris = np.random.default_rng(3).normal(0, 4, (40, 3, 3)).astype(np.float32)
    o = oracle.Oracle([s], lib)
    pairs = oracle.triangle_hits(o, tris)
    got = set(map(tuple, pairs.tolist()))
    d = oracle.ray_dirs(o).reshape(-1, 3)
    expect = set()
    for k in range(tris.shape[0]):
        for q in range(d.shape[0]):
            if oracle.hit(s.origin, d[q], tris[k], lib=lib) is not None:
                expect.add((k, q))
    assert got == expect and len(got) > 10


def check_area_keep(lib=None):
    """Eq. apparent_area: a triangle facing the sensor at distance r with area A
    has apparent area A / r^2 (cos = 1); kept iff A / r^2 >= eps.  Edge-on: dropped."""
    s = _sensor(h=0.0, n_rays=8, elev_deg=(0,))
    eps = 1e-6
    o = oracle.Oracle([s], lib)
    rows = []
    for A, r in ((1e-4, 5.0), (1e-4, 20.0), (1e-2, 50.0), (1e-2, 150.0), (4.0, 1000.0), (4.0, 3000.0)):
        L = math.sqrt(2.0 * A)   # right triangle with legs L: area L^2 / 2
        c = np.array([r, 0.0, 0.0])
        tri = np.array([c + [0, -L / 3, -L / 3], c + [0, 2 * L / 3, -L / 3], c + [0, -L / 3, 2 * L / 3]])
        rows.append((A / r ** 2 >= eps, tri))
    edge_on = np.array([[5.0, 0.0, -0.5], [6.0, 0.0, -0.5], [5.5, 0.0, 0.5]])   # plane y = 0 contains o
    tris = np.array([t for _, t in rows] + [edge_on], np.float32)
    keep = oracle.area_keep(o, tris, eps)[0]
    for k, (expect, _) in enumerate(rows):
        assert bool(keep[k]) == expect, (k, keep[k], expect)
    assert keep[-1] == 0
    # the keep mask hides dropped triangles from the cast
    r = oracle.cast(o, tris[:1], keep=np.zeros((1, 1), np.uint8))
    assert np.all(r["id"] == oracle.NO_HIT)


def check_splitmix64(lib=None):
    """SplitMix64's published output sequence for state 0: output n is sm(n * gamma)."""
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    gamma = 0x9E3779B97F4A7C15
    for n, h in enumerate(g["outputs_hex"]):
        assert oracle.splitmix64((g["seed_state"] + n * gamma) % 2**64, lib=lib) == int(h, 16), n


def _normal_cdf(x):
    return 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def check_range_noise(lib=None):
    """Range noise z must be standard normal (Box-Muller) and uncorrelated across
    neighbouring rays and seeds: moments, a Kolmogorov-Smirnov distance and lag-1
    correlation, at bounds 5+ standard errors wide for n = 200k draws."""
    n = 200_000
    q = np.arange(n, dtype=np.int64)
    z = oracle.range_noise(12345, q, lib=lib)
    assert np.all(np.isfinite(z))
    assert abs(z.mean()) < 5.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    zs = np.sort(z)
    ks = np.max(np.abs(_normal_cdf(zs) - (np.arange(n) + 0.5) / n))
    assert ks < 1.63 / math.sqrt(n) + 1.0 / n      # 1% critical value of the KS statistic
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5.0 / math.sqrt(n)
    z2 = oracle.range_noise(12346, q, lib=lib)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5.0 / math.sqrt(n)
    # deterministic in (seed, q): the same draws for a shuffled query
    perm = np.random.default_rng(0).permutation(n)[:1000]
    assert np.array_equal(oracle.range_noise(12345, q[perm], lib=lib), z[perm])


def check_azimuth_list(lib=None):
    """Per-ray azimuths (horizontal noise): a list equal to a grid shifted by c
    gives exactly the results of the uniform sensor with theta0 + c, and a
    permuted-free random list hits the triangles predicted by an independent
    linear solve along each listed direction."""
    rng = np.random.default_rng(11)
    tris = rng.normal(0, 4, (60, 3, 3)).astype(np.float32)
    tris[:, :, 2] = np.abs(tris[:, :, 2])
    base = _sensor(h=1.0, n_rays=96)
    c = 0.5 * base.dtheta
    shifted = Sensor(**{**base.__dict__, "theta0": base.theta0 + c})
    listed = Sensor(**{**base.__dict__, "azimuths": base.theta0 + c + np.arange(base.n_rays) * base.dtheta})
    r_s = oracle.cast(oracle.Oracle([shifted], lib), tris)
    r_l = oracle.cast(oracle.Oracle([listed], lib), tris)
    r_b = oracle.cast(oracle.Oracle([base], lib), tris)
    assert np.array_equal(r_s["id"], r_l["id"])
    hit = r_s["id"] != oracle.NO_HIT
    assert np.allclose(r_s["t"][hit], r_l["t"][hit], rtol=1e-12)
    assert np.count_nonzero(r_b["id"] != r_s["id"]) > 5       # the shift matters on this scene
    # each listed azimuth is used for its own ray: check a random list ray by ray
    th = base.theta0 + np.arange(base.n_rays) * base.dtheta + rng.uniform(-0.45, 0.45, base.n_rays) * base.dtheta
    noisy = Sensor(**{**base.__dict__, "azimuths": th})
    r_n = oracle.cast(oracle.Oracle([noisy], lib), tris)
    f, rr, u = base.f, base.r, base.u
    for q in range(0, noisy.n_total, 7):
        j, i = divmod(q, noisy.n_rays)
        ph = base.elev[j]
        d = math.cos(ph) * (math.cos(th[i]) * f + math.sin(th[i]) * rr) + math.sin(ph) * u
        best, bid = math.inf, oracle.NO_HIT
        for k in range(tris.shape[0]):
            v = tris[k].astype(np.float64)
            M = np.stack([v[1] - v[0], v[2] - v[0], -d], 1)
            if abs(np.linalg.det(M)) < 1e-12:
                continue
            a, b, t = np.linalg.solve(M, base.origin - v[0])
            if min(a, b, 1 - a - b) > 1e-9 and t > 0 and t < best:
                best, bid = t, k
        assert r_n["id"][q] == bid, (q, r_n["id"][q], bid)


def check_ray_mask(lib=None):
    """A ray that does not fire is a miss; the others are unchanged.  Bit order:
    bit q & 31 of word q >> 5 for q = j*n_rays + i (a single set bit fires exactly
    that ray)."""
    s = _sensor(h=1.8, n_rays=40)
    tris = _quad(-50, 50, -50, 50, 0.0)
    full = oracle.cast(oracle.Oracle([s], lib), tris)
    hits = np.nonzero(full["id"] != oracle.NO_HIT)[0]
    assert hits.size > 40
    for q in (int(hits[0]), int(hits[len(hits) // 2]), int(hits[-1])):
        m = np.zeros((s.n_total + 31) // 32, np.uint32)
        m[q >> 5] = np.uint32(1) << np.uint32(q & 31)
        r = oracle.cast(oracle.Oracle([s], lib, masks=[m]), tris)
        assert np.nonzero(r["id"] != oracle.NO_HIT)[0].tolist() == [q]
        assert r["t"][q] == full["t"][q]
    m = ray_mask(s, 4, 0.5)
    r = oracle.cast(oracle.Oracle([s], lib, masks=[m]), tris)
    on = np.array([(int(m[q >> 5]) >> (q & 31)) & 1 for q in range(s.n_total)], bool)
    assert np.array_equal(r["id"][on], full["id"][on]) and np.all(r["id"][~on] == oracle.NO_HIT)
    assert np.all(np.isinf(r["t"][~on]))


ALL_CHECKS = [check_brute_count, check_ray_grid, check_ground, check_wall, check_straddle, check_front,
              check_coplanar_tie, check_fan, check_backface, check_range, check_linear_solve, check_margin,
              check_triangle_hits, check_area_keep, check_splitmix64, check_range_noise, check_azimuth_list,
              check_ray_mask]
