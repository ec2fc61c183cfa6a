"""GPU test of grca_cast_noalloc, the allocation-free entry point.

Some callers of this library cannot allocate device memory: code that runs
inside an allocator or memory-pool callback (allocating there would re-enter
the allocator), plugins whose host framework forbids device allocations
after start-up, and real-time loops that must not block on the driver's
allocator.  grca_cast_noalloc serves them: it allocates nothing and keeps its
scratch in one fixed device array inside the library.

The test calls it through the C ABI twice in a row on two different scenes
(so the second call also shows the shared scratch array is reset between
calls) and checks each result against grca_cast, within the tolerances of
the other parity tests: hit/miss identical, distance within 1e-5 relative,
and a different triangle id only at a distance tie (1e-6 relative).  It also
checks that sizes beyond the fixed scratch are rejected.  This file is
collected last and needs no state from the other tests.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(sensor, tris, flags=0):
    import torch
    from paper_2605_10457_gb300 import grca
    lib = grca._lib_handle()
    desc, keep = grca.sensor_desc(sensor)
    dev_tris = torch.from_numpy(np.ascontiguousarray(tris, np.float32).reshape(-1, 9)).cuda()
    n = sensor.n_channels * sensor.n_rays
    d = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = lib.grca_cast_noalloc(ctypes.byref(desc), dev_tris.data_ptr(), dev_tris.shape[0], d.data_ptr(),
                               t.data_ptr(), flags, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, d.cpu().numpy(), t.cpu().numpy().view(np.uint32)


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


def test_noalloc_matches_grca_cast_two_calls_in_a_row():
    first = scene_c1()
    s1, tris1 = first.sensors[0], first.tris()
    second = make_config("c2m")
    s2, tris2 = second.sensors[0], second.tris(3)
    st, d, t = _noalloc(s1, tris1)
    assert st == 0
    _agree(_existing(s1, tris1), (d, t))
    st, d, t = _noalloc(s2, tris2)
    assert st == 0
    _agree(_existing(s2, tris2), (d, t))
    assert (t != 0xFFFFFFFF).sum() > 1000


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = make_sensor((0.0, 0.0, 1.8), channels="t128", n_rays=4096)   # 524,288 rays > 262,144
    st, _, _ = _noalloc(big, scene_c1().tris())
    assert st == -4   # GRCA_ERR_CAPACITY
    st, _, _ = _noalloc(scene_c1().sensors[0], scene_c1().tris(), flags=1)   # FP64 recheck not offered
    assert st == -1
