"""CPU checks of the seeded synthetic workloads: the sizes, sensor grids and
channel tables the benchmark and the parity tests rely on, seeded
reproducibility, and that only the dynamic part moves between frames."""
import math

import numpy as np
import pytest

from scenes import make_config


def _deg(s):
    return np.rad2deg(np.asarray(s.elev, np.float64))


def test_c1():
    sc = make_config("c1")
    assert sc.n_tris == 70 * 70 * 2 + 20 * 12 == 10040 and sc.n_static == sc.n_tris
    (s,) = sc.sensors
    assert (s.n_channels, s.n_rays) == (16, 512)
    assert np.allclose(_deg(s), -15.0 + 2.0 * np.arange(16))
    assert s.theta0 == pytest.approx(-math.pi) and s.dtheta == pytest.approx(2 * math.pi / 512)
    assert np.allclose(s.origin, (0.0, 0.0, 1.8))
    t = sc.tris(0)
    assert t.dtype == np.float32 and t.shape == (10040, 3, 3)


def test_t128_channel_table():
    s = make_config("c5m").sensors[0]
    full = make_config("c5").sensors[0]
    e = _deg(full)
    assert full.n_channels == 128 and np.all(np.diff(e) > 0)
    assert np.allclose(e[:30], -25.0 + 0.7 * np.arange(30))
    assert np.allclose(e[30:111], (np.arange(81) - 40) / 10.0) and e[70] == 0.0
    assert np.allclose(e[111:], 4.0 + (11.0 / 17.0) * np.arange(1, 18)) and e[-1] == pytest.approx(15.0)
    assert (full.n_rays, s.n_channels, s.n_rays) == (4096, 32, 1024)   # minis: gamma/4 x chi/4


def test_c4_c5_rigs_and_sizes():
    c4, c5 = make_config("c4"), make_config("c5")
    assert c4.n_tris == 21718400 and c4.n_tris - c4.n_static == 8918400
    assert c5.n_tris - c4.n_tris > 0 and c5.n_tris - c5.n_static == 8918400   # c4's scene + static stress set
    assert sorted((s.n_channels, s.n_rays) for s in c4.sensors) == sorted(
        [(32, 1024), (64, 2048)] + [(128, 4096)] * 6)
    fovs = sorted(round(math.degrees(s.n_rays * s.dtheta)) for s in c4.sensors)
    assert fovs == [180, 180] + [360] * 6
    assert len(c5.sensors) == 8
    assert all((s.n_channels, s.n_rays) == (128, 4096) and s.dtheta == pytest.approx(2 * math.pi / 4096)
               for s in c5.sensors)


def test_minis_scale_down():
    """Mini variants: the same rigs with a quarter of the channels and rays,
    and about a hundredth of the triangles."""
    for cfg, n_sensors, n_full in (("c2m", 1, 1.0e6), ("c3m", 2, 5.0e6), ("c4m", 8, 21718400)):
        m = make_config(cfg)
        assert len(m.sensors) == n_sensors
        assert 1 / 120 < m.n_tris / n_full < 1 / 80
        for s in m.sensors:
            assert s.n_rays <= 1024 and s.n_channels <= 32


def test_seeded_and_only_the_dynamic_part_moves():
    a, b = make_config("c4m"), make_config("c4m")
    ta, tb = a.tris(7), b.tris(7)
    assert np.array_equal(ta, tb)                         # same seed, same frame
    t0, t1 = a.tris(0), a.tris(1)
    ns = a.n_static
    assert np.array_equal(t0[:ns], t1[:ns])               # the static head never moves
    assert not np.array_equal(t0[ns:], t1[ns:])           # the dynamic tail does
    assert np.all(np.isfinite(t1))


def test_stress_set_produces_near_ties():
    """The c5 stress set is aimed along chosen rays; where nothing nearer
    occludes it, its coplanar overlapping pairs give near-tie sets of two or
    more triangles (FP64 oracle, tie band 1e-6 relative)."""
    import oracle
    c5m = make_config("c5m")
    rays = c5m.stress_rays
    assert rays is not None and len(rays) >= 10
    assert np.all((rays >= 0) & (rays < sum(s.n_total for s in c5m.sensors)))
    ref = oracle.cast(c5m.sensors, c5m.tris(0), rays, ties=True)
    assert np.all(np.isfinite(ref["t"]) & (ref["t"] > 0))          # every aimed ray hits something
    assert np.count_nonzero(ref["n_ties"] >= 2) >= 3
