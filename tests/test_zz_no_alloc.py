"""GPU test of grca_cast_noalloc, the allocation-free entry point.

Some callers of this library cannot allocate device memory: code that runs
inside an allocator or memory-pool callback (allocating there would re-enter
the allocator), plugins whose host framework forbids device allocations
after start-up, and real-time loops that must not block on the driver's
allocator.  grca_cast_noalloc serves them: it allocates nothing and keeps its
scratch in one fixed device array inside the library.

The test calls it through the C ABI twice in a row on two different scenes
(so the second call also shows the shared scratch array is reset between
calls).  Each result is checked against grca_cast, within the tolerances of
the other parity tests: hit/miss identical, distance within 1e-5 relative,
and a different triangle id only at a distance tie (1e-6 relative).  Each is
also graded against the FP64 oracle with the rule of the plain FP32 path.
A vertex buffer whose size is not a multiple of 16 bytes, and that ends
exactly where its allocation ends, is cast as well.  Misaligned buffers,
invalid sensor descriptions and sizes beyond the fixed scratch are rejected
before any GPU work.  This file is collected last and needs no state from
the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from grading import grade
from scenes import make_config, make_sensor, scene_c1

pytestmark = pytest.mark.gpu


def _existing(sensor, tris):
    import torch
    from paper_2605_10457_gb300 import grca
    c = grca.Caster(0)
    sid = c.add_sensor(sensor)
    c.upload(tris)
    d, t = c.cast([sid], 0)
    torch.cuda.synchronize()
    out = d.cpu().numpy(), t.cpu().numpy().view(np.uint32)
    c.close()
    return out


def _call(desc, ptr, n_tris, n_rays, flags=0):
    import torch
    from paper_2605_10457_gb300 import grca
    lib = grca._lib_handle()
    d = torch.full((n_rays,), -1.0, dtype=torch.float32, device="cuda")
    t = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    st = lib.grca_cast_noalloc(ctypes.byref(desc), ptr, n_tris, d.data_ptr(), t.data_ptr(), flags,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, d.cpu().numpy(), t.cpu().numpy().view(np.uint32)


def _noalloc(sensor, tris, flags=0):
    import torch
    from paper_2605_10457_gb300 import grca
    desc, keep = grca.sensor_desc(sensor)
    # a buffer of exactly n_tris * 36 bytes, nothing after the last triangle
    dev_tris = torch.from_numpy(np.ascontiguousarray(tris, np.float32).reshape(-1)).cuda()
    n = sensor.n_channels * sensor.n_rays
    return _call(desc, dev_tris.data_ptr(), dev_tris.numel() // 9, n, flags)


def _agree(ref, got):
    d0, t0 = ref
    d1, t1 = got
    h0, h1 = t0 != 0xFFFFFFFF, t1 != 0xFFFFFFFF
    assert np.array_equal(h0, h1)
    assert np.all(np.isinf(d1[~h1]))
    both = h0 & h1
    rel = np.abs(d1[both].astype(np.float64) - d0[both]) / d0[both]
    assert rel.size == 0 or rel.max() <= 1e-5
    diff = both & (t0 != t1)
    if diff.any():
        r2 = np.abs(d1[diff].astype(np.float64) - d0[diff]) / d0[diff]
        assert r2.max() <= 1e-6


def _graded(sensor, tris, d, t):
    """Oracle grading with the rule of the plain FP32 path (2e-6 rad near
    edges and silhouettes, distance within 1e-4 relative)."""
    orc = oracle.Oracle([sensor])
    ref = oracle.cast(orc, tris, None, ties=True)
    rid = ref["ray_ids"]
    return grade(orc, tris, ref, d[rid], t[rid], edge_eps=2e-6, silhouette_eps=2e-6, dist_rel=1e-4)


def test_noalloc_matches_grca_cast_and_the_oracle_two_calls_in_a_row():
    first = scene_c1()
    s1, tris1 = first.sensors[0], first.tris()
    second = make_config("c2m")
    s2, tris2 = second.sensors[0], second.tris(3)
    assert tris2.shape[0] % 4 != 0   # the last float4 of the vertex buffer is partial
    for s, tris in ((s1, tris1), (s2, tris2)):
        st, d, t = _noalloc(s, tris)
        assert st == 0
        ref = _existing(s, tris)
        _agree(ref, (d, t))
        g = _graded(s, tris, d, t)
        g_ref = _graded(s, tris, *ref)
        # the same FP32 test as grca_cast's plain path, so the same grade
        assert g["errors"] == g_ref["errors"], (g, g_ref)
        assert g["errors"] <= max(2, g["n"] // 5000), g
    assert (t != 0xFFFFFFFF).sum() > 1000


def test_noalloc_unpadded_buffer_with_a_partial_last_float4():
    sc = scene_c1()
    s = sc.sensors[0]
    tris = sc.tris()[:10038]            # 10038 * 9 floats: the buffer ends 8 bytes into a float4
    st, d, t = _noalloc(s, tris)
    assert st == 0
    _agree(_existing(s, tris), (d, t))


def test_noalloc_rejects_bad_arguments_before_any_gpu_work():
    import torch
    from paper_2605_10457_gb300 import grca
    sc = scene_c1()
    s = sc.sensors[0]
    n = s.n_channels * s.n_rays
    buf = torch.from_numpy(np.ascontiguousarray(sc.tris(), np.float32).reshape(-1)).cuda()
    desc, keep = grca.sensor_desc(s)
    # a vertex pointer that is not 16-byte aligned
    st, _, _ = _call(desc, buf.data_ptr() + 4, 100, n)
    assert st == -1
    # the checks of grca_create_sensor
    bad = []
    d1, k1 = grca.sensor_desc(s)
    d1.f[0], d1.f[1] = 0.8, 0.6                  # axes no longer orthonormal
    bad.append(d1)
    d2, k2 = grca.sensor_desc(s)
    d2.origin[2] = math.nan                      # non-finite origin
    bad.append(d2)
    d3, k3 = grca.sensor_desc(s)
    d3.theta0 = 5 * math.pi                      # |theta0| > 4 pi
    bad.append(d3)
    d4, k4 = grca.sensor_desc(s)
    d4.d_min, d4.d_max = math.inf, math.inf      # d_min must be finite
    bad.append(d4)
    for d in bad:
        st, _, _ = _call(d, buf.data_ptr(), buf.numel() // 9, n)
        assert st == -1
    # the call still works afterwards
    st, d, t = _call(desc, buf.data_ptr(), buf.numel() // 9, n)
    assert st == 0 and (t != 0xFFFFFFFF).sum() > 1000


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = make_sensor((0.0, 0.0, 1.8), channels="t128", n_rays=4096)   # 524,288 rays > 262,144
    st, _, _ = _noalloc(big, scene_c1().tris())
    assert st == -4   # GRCA_ERR_CAPACITY
    st, _, _ = _noalloc(scene_c1().sensors[0], scene_c1().tris(), flags=1)   # FP64 recheck not offered
    assert st == -1
