"""ctypes binding of the FP64 brute-force oracle (TEST INFRASTRUCTURE ONLY).

Argument marshalling only; every computation is in grca_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libgrca_oracle.so")
SRC = os.path.join(HERE, "grca_oracle.c")
MAX_TIES = 16
NO_HIT = 0xFFFFFFFF
_lock = threading.Lock()
_lib = None


def compile_oracle(src: str, out: str, include_dir: str = HERE) -> str:
    """gcc build of an oracle source file (no FMA contraction, so x86 and Arm agree)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-I", include_dir, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_oracle(force: bool = False) -> str:
    """Compile grca_oracle.c into libgrca_oracle.so next to it (if stale)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "grca_oracle.h"))):
        return LIB
    return compile_oracle(SRC, LIB)


class _Sensor(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("f", ctypes.c_double * 3), ("r", ctypes.c_double * 3),
                ("u", ctypes.c_double * 3), ("theta0", ctypes.c_double), ("dtheta", ctypes.c_double),
                ("d_min", ctypes.c_double), ("d_max", ctypes.c_double),
                ("elev", ctypes.POINTER(ctypes.c_double)), ("n_channels", ctypes.c_uint32),
                ("n_rays", ctypes.c_uint32), ("theta", ctypes.POINTER(ctypes.c_double)),
                ("mask", ctypes.POINTER(ctypes.c_uint32))]


def load_library(path: str):
    """Load a compiled oracle library (the default build, or a test's planted-mistake copy)."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.orc_cast.argtypes = [P, ctypes.c_uint32, P, ctypes.c_uint32, P, ctypes.c_int64, ctypes.c_int,
                             ctypes.c_double, ctypes.c_int, P, P, P, P, P, P, P]
    lib.orc_area_keep.argtypes = [P, ctypes.c_uint32, P, ctypes.c_uint32, ctypes.c_double, P]
    lib.orc_area_keep.restype = None
    lib.orc_cast.restype = ctypes.c_int
    lib.orc_ray_dir.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, P]
    lib.orc_ray_dir.restype = None
    lib.orc_ray_tri_margin.argtypes = [P, ctypes.c_uint32, ctypes.c_int64, P, P, P]
    lib.orc_ray_tri_margin.restype = ctypes.c_int
    lib.orc_triangle_hits.argtypes = [P, P, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64]
    lib.orc_triangle_hits.restype = ctypes.c_int64
    lib.orc_range_noise.argtypes = [ctypes.c_uint64, P, ctypes.c_int64, P]
    lib.orc_range_noise.restype = None
    lib.orc_splitmix64.argtypes = [ctypes.c_uint64]
    lib.orc_splitmix64.restype = ctypes.c_uint64
    lib.orc_hit.argtypes = [P, P, P, P]
    lib.orc_hit.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            _lib = load_library(LIB)
    return _lib


class Oracle:
    """Holds ctypes copies of a sensor list (keeps the elevation, azimuth and
    mask arrays alive).  masks: optional per-sensor uint32 on/off words (None
    entries: every ray fires); per-ray azimuths come from `s.azimuths`."""

    def __init__(self, sensors: Sequence, lib=None, masks: Optional[Sequence] = None):
        self.lib = lib if lib is not None else _load()
        self._elev = [np.ascontiguousarray(s.elev, dtype=np.float64) for s in sensors]
        self._theta = [None if getattr(s, "azimuths", None) is None else
                       np.ascontiguousarray(s.azimuths, dtype=np.float64) for s in sensors]
        self._mask = [None if masks is None or masks[k] is None else
                      np.ascontiguousarray(masks[k], dtype=np.uint32) for k in range(len(sensors))]
        arr = (_Sensor * len(sensors))()
        for k, s in enumerate(sensors):
            c = arr[k]
            for a in range(3):
                c.origin[a] = float(s.origin[a])
                c.f[a] = float(s.f[a])
                c.r[a] = float(s.r[a])
                c.u[a] = float(s.u[a])
            c.theta0 = float(s.theta0)
            c.dtheta = float(s.dtheta)
            c.d_min = float(s.d_min)
            c.d_max = float(s.d_max)
            c.elev = self._elev[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            c.n_channels = int(s.elev.shape[0])
            c.n_rays = int(s.n_rays)
            if self._theta[k] is not None:
                assert self._theta[k].shape[0] == c.n_rays
                c.theta = self._theta[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            if self._mask[k] is not None:
                assert self._mask[k].shape[0] * 32 >= c.n_rays * c.n_channels
                c.mask = self._mask[k].ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        self.sensors = arr
        self.n = len(sensors)

    def ptr(self, k: int = 0):
        return ctypes.byref(self.sensors, k * ctypes.sizeof(_Sensor))


def _threads(n: Optional[int]) -> int:
    return int(n) if n else (os.cpu_count() or 1)


def cast(sensors, tris: np.ndarray, ray_ids: Optional[np.ndarray] = None, cull_backface: bool = False,
         ties: bool = False, tie_rel: float = 1e-6, n_threads: Optional[int] = None,
         keep: Optional[np.ndarray] = None) -> dict:
    """Brute-force closest hit of the listed global rays (all rays if None).
    keep: optional [n_sensors, n_tris] mask; 0 hides a triangle from that sensor."""
    o = sensors if isinstance(sensors, Oracle) else Oracle(sensors)
    tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    if ray_ids is None:
        total = sum(int(o.sensors[k].n_channels) * int(o.sensors[k].n_rays) for k in range(o.n))
        ray_ids = np.arange(total, dtype=np.int64)
    ray_ids = np.ascontiguousarray(ray_ids, dtype=np.int64)
    n = ray_ids.shape[0]
    best_t = np.empty(n, np.float64)
    best_id = np.empty(n, np.uint32)
    second = np.empty(n, np.float64) if ties else None
    n_ties = np.empty(n, np.uint32) if ties else None
    tie_ids = np.full((n, MAX_TIES), NO_HIT, np.uint32) if ties else None
    tests = np.zeros(1, np.uint64)
    if keep is not None:
        keep = np.ascontiguousarray(keep, dtype=np.uint8).reshape(o.n, tris.shape[0])
    p = lambda a: None if a is None else a.ctypes.data
    rc = o.lib.orc_cast(ctypes.byref(o.sensors), o.n, tris.ctypes.data, tris.shape[0], ray_ids.ctypes.data, n,
                        int(bool(cull_backface)), float(tie_rel), _threads(n_threads), best_t.ctypes.data,
                        best_id.ctypes.data, p(second), p(n_ties), p(tie_ids), tests.ctypes.data, p(keep))
    if rc != 0:
        raise ValueError("orc_cast failed (bad ray id or argument)")
    out = {"t": best_t, "id": best_id, "tests": int(tests[0]), "ray_ids": ray_ids}
    if ties:
        out.update(second=second, n_ties=n_ties, tie_ids=tie_ids)
    return out


def range_noise(seed: int, q: np.ndarray, lib=None) -> np.ndarray:
    """Standard normal range-noise draws z for sensor-local ray indices q (FP64)."""
    lib = lib if lib is not None else _load()
    q = np.ascontiguousarray(q, dtype=np.int64)
    z = np.empty(q.shape[0], np.float64)
    lib.orc_range_noise(int(seed) & (2**64 - 1), q.ctypes.data, q.shape[0], z.ctypes.data)
    return z


def splitmix64(x: int, lib=None) -> int:
    lib = lib if lib is not None else _load()
    return int(lib.orc_splitmix64(int(x) & (2**64 - 1)))


def area_keep(sensors, tris: np.ndarray, eps: float = 1e-6) -> np.ndarray:
    """[n_sensors, n_tris] uint8: 1 keep, 0 drop, 2 keep within 1e-3 of the threshold
    (the apparent-area filter of App. A.4.1 Step 1)."""
    o = sensors if isinstance(sensors, Oracle) else Oracle(sensors)
    tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    out = np.empty((o.n, tris.shape[0]), np.uint8)
    o.lib.orc_area_keep(ctypes.byref(o.sensors), o.n, tris.ctypes.data, tris.shape[0], float(eps), out.ctypes.data)
    return out


def ray_dirs(sensor) -> np.ndarray:
    """[n_channels, n_rays, 3] float64 directions of one sensor (Eq. ray_dir)."""
    o = sensor if isinstance(sensor, Oracle) else Oracle([sensor])
    nc, nr = int(o.sensors[0].n_channels), int(o.sensors[0].n_rays)
    out = np.empty((nc, nr, 3), np.float64)
    d = np.empty(3, np.float64)
    for j in range(nc):
        for i in range(nr):
            o.lib.orc_ray_dir(o.ptr(0), j, i, d.ctypes.data)
            out[j, i] = d
    return out


def ray_tri_margin(oracle: Oracle, ray_id: int, tri: np.ndarray):
    tri = np.ascontiguousarray(tri, dtype=np.float32).reshape(9)
    tp = ctypes.c_double()
    m = ctypes.c_double()
    rc = oracle.lib.orc_ray_tri_margin(ctypes.byref(oracle.sensors), oracle.n, int(ray_id), tri.ctypes.data,
                                       ctypes.byref(tp), ctypes.byref(m))
    if rc != 0:
        raise ValueError("bad ray id")
    return tp.value, m.value


def triangle_hits(sensor, tris: np.ndarray, cull_backface: bool = False, n_threads: Optional[int] = None):
    """All (triangle, local ray id) pairs where the ray hits the triangle (one sensor)."""
    o = sensor if isinstance(sensor, Oracle) else Oracle([sensor])
    tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    n = o.lib.orc_triangle_hits(o.ptr(0), tris.ctypes.data, tris.shape[0], int(bool(cull_backface)),
                                _threads(n_threads), None, 0)
    out = np.empty((max(n, 1), 2), np.int64)
    n2 = o.lib.orc_triangle_hits(o.ptr(0), tris.ctypes.data, tris.shape[0], int(bool(cull_backface)),
                                 _threads(n_threads), out.ctypes.data, n)
    assert n2 == n
    return out[:n]


def hit(o3, d3, tri, lib=None) -> Optional[float]:
    lib = lib if lib is not None else _load()
    o3 = np.ascontiguousarray(o3, np.float64)
    d3 = np.ascontiguousarray(d3, np.float64)
    tri = np.ascontiguousarray(tri, np.float32).reshape(9)
    t = ctypes.c_double()
    return t.value if lib.orc_hit(o3.ctypes.data, d3.ctypes.data, tri.ctypes.data, ctypes.byref(t)) else None


__all__ = ["MAX_TIES", "NO_HIT", "Oracle", "area_keep", "build_oracle", "cast", "compile_oracle", "hit",
           "range_noise", "splitmix64",
           "load_library", "ray_dirs", "ray_tri_margin", "triangle_hits"]
