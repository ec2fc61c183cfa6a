"""CPU tests of the boundary: libgrca.so builds for sm_103a, loads, and exports
every function include/grca.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2605_10457_gb300 import build as B
from paper_2605_10457_gb300 import grca

HEADER = os.path.join(B.ROOT, "include", "grca.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grca_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("grca_create_sensor", "grca_upload_triangles", "grca_update_vertices", "grca_cast"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    assert sorted(grca.EXPORTS) == declared_functions()


def test_status_strings(lib):
    lib.grca_status_string.restype = ctypes.c_char_p
    lib.grca_status_string.argtypes = [ctypes.c_int32]
    assert lib.grca_status_string(0) == b"ok"
    for code in (-1, -2, -3, -4, -5, -6):
        s = lib.grca_status_string(code)
        assert s and s != b"unknown status"
    assert lib.grca_status_string(-99) == b"unknown status"


def test_null_arguments_rejected_without_a_device(lib):
    # argument checks run before any CUDA call
    lib.grca_create.restype = ctypes.c_int32
    lib.grca_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.grca_create(None, 0, None) == -1
    lib.grca_cast.restype = ctypes.c_int32
    lib.grca_cast.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                                       ctypes.c_void_p]
    assert lib.grca_cast(None, None, 0, None, None, 0, None) == -1
    lib.grca_get_stats.restype = ctypes.c_int32
    assert lib.grca_get_stats(None, None, None) == -1
    P = ctypes.c_void_p
    for name, argtypes, args in (
            ("grca_get_launch_config", [P, P, ctypes.c_uint32, ctypes.c_uint32, P], (None, None, 1, 0, None)),
            ("grca_build_static", [P, ctypes.c_uint32, P], (None, 0, None)),
            ("grca_host_wait", [P, ctypes.c_uint32], (None, 0)),
            ("grca_cast_host", [P, P, ctypes.c_uint32, P, ctypes.c_uint32, ctypes.c_uint32, P, P, ctypes.c_uint32, P],
             (None, None, 1, None, 0, 0, None, None, 0, None)),
            ("grca_set_ray_mask", [P, ctypes.c_int32, P, ctypes.c_int, P], (None, 0, None, 0, None)),
            ("grca_set_sensor_azimuths", [P, ctypes.c_int32, P], (None, 0, None)),
            ("grca_set_range_noise", [P, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64], (None, 0, 0.1, 1)),
            ("grca_upload_triangles", [P, P, ctypes.c_uint32, ctypes.c_int, P], (None, None, 0, 0, None)),
            ("grca_update_vertices", [P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, P],
             (None, None, 0, 0, 0, None))):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int32
        fn.argtypes = argtypes
        assert fn(*args) == -1, name


def test_struct_layouts_match_header():
    # the ctypes mirrors must match the C layout (sizes computed by the C rules)
    assert ctypes.sizeof(grca.grca_sensor_desc) == 12 * 8 + 8 + 4 + 4 + 4 * 8
    assert ctypes.sizeof(grca.grca_options) == 3 * 8 + 4 * 4 + 8 + 8
    assert ctypes.sizeof(grca.grca_stats) == 17 * 8 + 2 * 4 + 12 * 8


def test_build_targets_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_sensor_descriptor_marshalling():
    """The binding's grca_sensor_desc carries a scenes.Sensor field for field
    (FP64 origin and axes, the elevation table by pointer, the azimuth grid
    and the range)."""
    import math
    import numpy as np
    from scenes import make_sensor
    s = make_sensor((1.5, -0.8, 1.9), yaw=0.3, channels="t128", n_rays=2048, fov_deg=180.0, d_min=0.05, d_max=50.0)
    d, elev = grca.sensor_desc(s)
    assert list(d.origin) == [1.5, -0.8, 1.9]
    assert np.allclose(list(d.f), s.f) and np.allclose(list(d.r), s.r) and np.allclose(list(d.u), s.u)
    assert d.n_channels == 128 == elev.shape[0] and d.n_rays == 2048
    assert [d.elev_rad[j] for j in (0, 70, 127)] == [float(s.elev[0]), float(s.elev[70]), float(s.elev[127])]
    assert d.dtheta == s.dtheta and d.theta0 == s.theta0 and d.n_rays * d.dtheta == pytest.approx(math.pi)
    assert (d.d_min, d.d_max) == (0.05, 50.0)
