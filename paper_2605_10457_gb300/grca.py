"""Python binding of libgrca.so (include/grca.h): argument marshalling only.

Every step of the cast runs in the library's CUDA kernels.  PyTorch is used
for device memory and streams.  Loading fails loudly if the library is not
built or cannot be loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

GRCA_OK = 0
GRCA_MEM_HOST = 0
GRCA_MEM_DEVICE = 1
CAST_FP64_RECHECK = 1 << 0
CAST_CULL_BACKFACE = 1 << 1
CAST_BRUTE = 1 << 2
CAST_GRAPH = 1 << 3
CAST_DUMP_CANDIDATES = 1 << 4
CAST_LOSSY_AREA = 1 << 5
CAST_NO_GROUP_CULL = 1 << 6
CAST_NO_STATIC_BVH = 1 << 7
CAST_HOST_ASYNC = 1 << 8
CAST_NO_OCCLUSION = 1 << 9
NO_HIT = 0xFFFFFFFF


class grca_options(ctypes.Structure):
    _fields_ = [("big_pair_capacity", ctypes.c_uint64), ("chunk_capacity", ctypes.c_uint64),
                ("recheck_capacity", ctypes.c_uint64), ("inline_max", ctypes.c_uint32),
                ("chunk_rays", ctypes.c_uint32), ("cull_block", ctypes.c_uint32),
                ("cull_blocks_per_sm", ctypes.c_uint32), ("survivor_capacity", ctypes.c_uint64),
                ("area_eps", ctypes.c_double)]


class grca_sensor_desc(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("f", ctypes.c_double * 3), ("r", ctypes.c_double * 3),
                ("u", ctypes.c_double * 3), ("elev_rad", ctypes.POINTER(ctypes.c_double)),
                ("n_channels", ctypes.c_uint32), ("n_rays", ctypes.c_uint32), ("theta0", ctypes.c_double),
                ("dtheta", ctypes.c_double), ("d_min", ctypes.c_double), ("d_max", ctypes.c_double)]


class grca_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("pairs", "pairs_live", "survivors", "candidates", "candidates_inline",
                                               "big_pairs",
                                               "chunks", "tests", "hits", "uncertain", "ties", "flagged_rays",
                                               "recheck_pairs", "group_culled", "bvh_node_visits", "bvh_tests",
                                               "n_rays")] + \
               [("device_error", ctypes.c_uint32), ("reserved", ctypes.c_uint32)] + \
               [(f"{w}_{c}", ctypes.c_uint64) for w in ("queued", "kept")
                for c in ("edge", "t", "range", "orient", "tie")] + \
               [("t_refined", ctypes.c_uint64), ("pairs_occluded", ctypes.c_uint64)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


class GrcaError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        super().__init__(f"{where}: {_lib_handle().grca_status_string(status).decode()} ({status}) {detail}".strip())
        self.status = status


_LIB = None
EXPORTS = ["grca_create", "grca_destroy", "grca_create_sensor", "grca_set_sensor_pose", "grca_upload_triangles",
           "grca_update_vertices", "grca_cast", "grca_cast_host", "grca_autotune", "grca_set_debug_dump",
           "grca_get_stats", "grca_last_launch_count", "grca_profile_enable", "grca_profile_read",
           "grca_status_string", "grca_last_cuda_error", "grca_cast_noalloc",
           "grca_set_ray_mask", "grca_set_sensor_azimuths", "grca_set_range_noise", "grca_build_static",
           "grca_get_launch_config", "grca_host_wait", "grca_cast_shard", "grca_flag_shard", "grca_resolve_shard", "grca_decode_keys"]


def library_path() -> str:
    return _build.LIB


def _lib_handle(build_if_missing: bool = True):
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libgrca.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32
    lib.grca_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(grca_options)]
    lib.grca_create.restype = i32
    lib.grca_destroy.argtypes = [P]
    lib.grca_destroy.restype = None
    lib.grca_create_sensor.argtypes = [P, ctypes.POINTER(grca_sensor_desc), ctypes.POINTER(i32)]
    lib.grca_create_sensor.restype = i32
    lib.grca_set_sensor_pose.argtypes = [P, i32, P, P, P, P]
    lib.grca_set_sensor_pose.restype = i32
    lib.grca_upload_triangles.argtypes = [P, P, u32, ctypes.c_int, P]
    lib.grca_upload_triangles.restype = i32
    lib.grca_update_vertices.argtypes = [P, P, u32, u32, ctypes.c_int, P]
    lib.grca_update_vertices.restype = i32
    lib.grca_cast.argtypes = [P, P, u32, P, P, u32, P]
    lib.grca_cast.restype = i32
    lib.grca_cast_host.argtypes = [P, P, u32, P, u32, u32, P, P, u32, P]
    lib.grca_cast_host.restype = i32
    lib.grca_cast_shard.argtypes = [P, P, u32, u32, P, u32, P]
    lib.grca_cast_shard.restype = i32
    lib.grca_flag_shard.argtypes = [P, P, P, P]
    lib.grca_flag_shard.restype = i32
    lib.grca_resolve_shard.argtypes = [P, P, P, P]
    lib.grca_resolve_shard.restype = i32
    lib.grca_decode_keys.argtypes = [P, P, P, P, P]
    lib.grca_decode_keys.restype = i32
    lib.grca_host_wait.argtypes = [P, u32]
    lib.grca_host_wait.restype = i32
    lib.grca_autotune.argtypes = [P, P, u32, P, P, u32, P, ctypes.POINTER(ctypes.c_float)]
    lib.grca_autotune.restype = i32
    lib.grca_set_debug_dump.argtypes = [P, P, ctypes.c_uint64, P]
    lib.grca_set_debug_dump.restype = i32
    lib.grca_get_stats.argtypes = [P, ctypes.POINTER(grca_stats), P]
    lib.grca_get_stats.restype = i32
    lib.grca_last_launch_count.argtypes = [P]
    lib.grca_last_launch_count.restype = u32
    lib.grca_profile_enable.argtypes = [P, ctypes.c_int]
    lib.grca_profile_enable.restype = i32
    lib.grca_profile_read.argtypes = [P, u32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32)]
    lib.grca_profile_read.restype = i32
    lib.grca_get_launch_config.argtypes = [P, P, u32, u32, P]
    lib.grca_get_launch_config.restype = i32
    lib.grca_build_static.argtypes = [P, u32, P]
    lib.grca_build_static.restype = i32
    lib.grca_set_ray_mask.argtypes = [P, i32, P, ctypes.c_int, P]
    lib.grca_set_ray_mask.restype = i32
    lib.grca_set_sensor_azimuths.argtypes = [P, i32, P]
    lib.grca_set_sensor_azimuths.restype = i32
    lib.grca_set_range_noise.argtypes = [P, i32, ctypes.c_double, ctypes.c_uint64]
    lib.grca_set_range_noise.restype = i32
    lib.grca_cast_noalloc.argtypes = [ctypes.POINTER(grca_sensor_desc), P, u32, P, P, u32, P]
    lib.grca_cast_noalloc.restype = i32
    lib.grca_status_string.argtypes = [i32]
    lib.grca_status_string.restype = ctypes.c_char_p
    lib.grca_last_cuda_error.argtypes = [P]
    lib.grca_last_cuda_error.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def sensor_desc(s):
    """grca_sensor_desc for a scenes.Sensor; returns (desc, elevation array kept alive by the caller)."""
    elev = np.ascontiguousarray(s.elev, dtype=np.float64)
    d = grca_sensor_desc()
    for k in range(3):
        d.origin[k] = float(s.origin[k])
        d.f[k] = float(s.f[k])
        d.r[k] = float(s.r[k])
        d.u[k] = float(s.u[k])
    d.elev_rad = elev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_channels = elev.shape[0]
    d.n_rays = int(s.n_rays)
    d.theta0 = float(s.theta0)
    d.dtheta = float(s.dtheta)
    d.d_min = float(s.d_min)
    d.d_max = float(s.d_max)
    return d, elev


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Caster:
    """One grca_ctx bound to a CUDA device."""

    def __init__(self, device: int = 0, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("GRCA needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.lib = _lib_handle()
        self.device = device
        o = grca_options()
        for k, v in opts.items():
            setattr(o, k, float(v) if k == "area_eps" else int(v))
        ctx = ctypes.c_void_p()
        torch.cuda.set_device(device)
        st = self.lib.grca_create(ctypes.byref(ctx), device, ctypes.byref(o))
        self._check(st, "grca_create", ctx=None)
        self.ctx = ctx
        self.sensors = []
        self._elev = []
        self.n_tris = 0
        self._tris_dev = None

    def _check(self, st, where, ctx="self"):
        if st != GRCA_OK:
            detail = ""
            c = self.ctx if ctx == "self" else ctx
            if c is not None:
                detail = self.lib.grca_last_cuda_error(c).decode()
            raise GrcaError(st, where, detail)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            self.lib.grca_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- sensors ---------------------------------------------------------
    def add_sensor(self, s) -> int:
        elev = np.ascontiguousarray(s.elev, dtype=np.float64)
        d = grca_sensor_desc()
        for k in range(3):
            d.origin[k] = float(s.origin[k])
            d.f[k] = float(s.f[k])
            d.r[k] = float(s.r[k])
            d.u[k] = float(s.u[k])
        d.elev_rad = elev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.n_channels = elev.shape[0]
        d.n_rays = int(s.n_rays)
        d.theta0 = float(s.theta0)
        d.dtheta = float(s.dtheta)
        d.d_min = float(s.d_min)
        d.d_max = float(s.d_max)
        sid = ctypes.c_int32()
        self._check(self.lib.grca_create_sensor(self.ctx, ctypes.byref(d), ctypes.byref(sid)), "grca_create_sensor")
        self.sensors.append(s)
        self._elev.append(elev)
        az = getattr(s, "azimuths", None)
        if az is not None:
            self.set_azimuths(sid.value, az)
        return sid.value

    def launch_config(self, ids, flags: int = 0) -> dict:
        """The launch parameters a cast of these sensors with these flags would use."""
        ids_a = np.ascontiguousarray(ids, dtype=np.int32)
        out = np.zeros(4, np.int32)
        self._check(self.lib.grca_get_launch_config(self.ctx, ids_a.ctypes.data, ids_a.shape[0], int(flags),
                                                    out.ctypes.data), "grca_get_launch_config")
        return {"inline_max": int(out[0]), "chunk_rays": int(out[1]), "cull_block": int(out[2]),
                "cull_blocks_per_sm": int(out[3])}

    def build_static(self, n_static: int, stream=None):
        """Hybrid pipeline: static hierarchy over triangles [0, n_static) (0 drops it)."""
        self._check(self.lib.grca_build_static(self.ctx, int(n_static), _stream_ptr(stream)), "grca_build_static")

    def set_azimuths(self, sid: int, theta=None):
        """Per-ray azimuths (radians) replacing the uniform grid; None restores it."""
        if theta is None:
            self._check(self.lib.grca_set_sensor_azimuths(self.ctx, sid, None), "grca_set_sensor_azimuths")
            return
        th = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self.lib.grca_set_sensor_azimuths(self.ctx, sid, th.ctypes.data), "grca_set_sensor_azimuths")

    def set_ray_mask(self, sid: int, bits=None, stream=None):
        """On/off bits over the sensor's channel x ray grid (uint32 words; bit q & 31 of
        word q >> 5 for ray q = j*n_rays + i).  numpy: host copy; CUDA tensor: device copy."""
        torch = self.torch
        if bits is None:
            st = self.lib.grca_set_ray_mask(self.ctx, sid, None, GRCA_MEM_HOST, _stream_ptr(stream))
        elif isinstance(bits, torch.Tensor) and bits.is_cuda:
            b = bits.contiguous()
            st = self.lib.grca_set_ray_mask(self.ctx, sid, b.data_ptr(), GRCA_MEM_DEVICE, _stream_ptr(stream))
        else:
            b = np.ascontiguousarray(bits, dtype=np.uint32)
            s = self.sensors[sid]
            if b.size * 32 < len(s.elev) * int(s.n_rays):
                raise ValueError("ray mask shorter than the sensor's channel x ray grid")
            st = self.lib.grca_set_ray_mask(self.ctx, sid, b.ctypes.data, GRCA_MEM_HOST, _stream_ptr(stream))
        self._check(st, "grca_set_ray_mask")

    def set_range_noise(self, sid: int, sigma: float, seed: int = 0):
        """Post-hoc range noise sigma * N(0, 1) on every hit distance of the sensor."""
        self._check(self.lib.grca_set_range_noise(self.ctx, sid, float(sigma), int(seed) & (2**64 - 1)),
                    "grca_set_range_noise")

    def set_pose(self, sid: int, origin, f, r, u):
        arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (origin, f, r, u)]
        self._check(self.lib.grca_set_sensor_pose(self.ctx, sid, *[a.ctypes.data for a in arrs]),
                    "grca_set_sensor_pose")
        s = self.sensors[sid]
        s.origin, s.f, s.r, s.u = arrs

    # -- triangles -------------------------------------------------------
    def upload(self, tris, stream=None):
        torch = self.torch
        if isinstance(tris, torch.Tensor) and tris.is_cuda:
            t = tris.contiguous().view(-1, 9)
            self._check(self.lib.grca_upload_triangles(self.ctx, t.data_ptr(), t.shape[0], GRCA_MEM_DEVICE,
                                                       _stream_ptr(stream)), "grca_upload_triangles")
            self._keep = t
        else:
            t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
            self._check(self.lib.grca_upload_triangles(self.ctx, t.ctypes.data, t.shape[0], GRCA_MEM_HOST,
                                                       _stream_ptr(stream)), "grca_upload_triangles")
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        self.n_tris = t.shape[0]

    def update(self, tris, first: int, stream=None):
        torch = self.torch
        if isinstance(tris, torch.Tensor) and tris.is_cuda:
            t = tris.contiguous().view(-1, 9)
            self._check(self.lib.grca_update_vertices(self.ctx, t.data_ptr(), first, t.shape[0], GRCA_MEM_DEVICE,
                                                      _stream_ptr(stream)), "grca_update_vertices")
        else:
            t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
            self._check(self.lib.grca_update_vertices(self.ctx, t.ctypes.data, first, t.shape[0], GRCA_MEM_HOST,
                                                      _stream_ptr(stream)), "grca_update_vertices")
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    # -- cast ------------------------------------------------------------
    def n_rays(self, ids: Sequence[int]) -> int:
        return int(sum(self.sensors[i].n_total for i in ids))

    def outputs(self, ids):
        torch = self.torch
        n = self.n_rays(ids)
        dev = torch.device("cuda", self.device)
        return (torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.int32, device=dev))

    def cast(self, ids: Sequence[int], flags: int = 0, out=None, stream=None):
        ids_a = np.ascontiguousarray(ids, dtype=np.int32)
        if out is None:
            out = self.outputs(ids)
        dist, tri = out
        st = self.lib.grca_cast(self.ctx, ids_a.ctypes.data, ids_a.shape[0], dist.data_ptr(), tri.data_ptr(),
                                int(flags), _stream_ptr(stream))
        self._check(st, "grca_cast")
        return dist, tri

    # triangle-sharded casts (include/grca.h): key arrays are int64 tensors on
    # this context's device, one entry per ray
    def cast_shard(self, ids: Sequence[int], tri_base: int, keys, flags: int = 0, stream=None):
        ids_a = np.ascontiguousarray(ids, dtype=np.int32)
        st = self.lib.grca_cast_shard(self.ctx, ids_a.ctypes.data, ids_a.shape[0], int(tri_base), keys.data_ptr(),
                                      int(flags), _stream_ptr(stream))
        self._check(st, "grca_cast_shard")
        return keys

    def flag_shard(self, keys_min, flags_out, stream=None):
        st = self.lib.grca_flag_shard(self.ctx, keys_min.data_ptr(), flags_out.data_ptr(), _stream_ptr(stream))
        self._check(st, "grca_flag_shard")
        return flags_out

    def resolve_shard(self, flags_any, keys_out, stream=None):
        st = self.lib.grca_resolve_shard(self.ctx, flags_any.data_ptr(), keys_out.data_ptr(), _stream_ptr(stream))
        self._check(st, "grca_resolve_shard")
        return keys_out

    def decode_keys(self, keys, out, stream=None):
        dist, tri = out
        st = self.lib.grca_decode_keys(self.ctx, keys.data_ptr(), dist.data_ptr(), tri.data_ptr(), _stream_ptr(stream))
        self._check(st, "grca_decode_keys")
        return dist, tri

    def cast_host(self, ids, dyn_tris: Optional[np.ndarray], first_dyn: int, out_dist: np.ndarray,
                  out_tri: np.ndarray, flags: int = 0, stream=None):
        ids_a = np.ascontiguousarray(ids, dtype=np.int32)
        if dyn_tris is None:
            ptr, n = None, 0
        else:
            ptr, n = dyn_tris.ctypes.data, dyn_tris.reshape(-1, 9).shape[0]
        st = self.lib.grca_cast_host(self.ctx, ids_a.ctypes.data, ids_a.shape[0], ptr, first_dyn, n,
                                     out_dist.ctypes.data, out_tri.ctypes.data, int(flags), _stream_ptr(stream))
        self._check(st, "grca_cast_host")

    def cast_host_ptrs(self, ids_a: np.ndarray, dyn_ptr: int, first_dyn: int, n_dyn: int, dist_ptr: int,
                       tri_ptr: int, flags: int, stream_ptr: int):
        st = self.lib.grca_cast_host(self.ctx, ids_a.ctypes.data, ids_a.shape[0], dyn_ptr, first_dyn, n_dyn,
                                     dist_ptr, tri_ptr, int(flags), stream_ptr)
        self._check(st, "grca_cast_host")

    def host_wait(self, max_pending: int = 0):
        """Block until at most `max_pending` asynchronous host casts
        (CAST_HOST_ASYNC) still have results on their way to the host."""
        self._check(self.lib.grca_host_wait(self.ctx, int(max_pending)), "grca_host_wait")

    def autotune(self, ids, flags: int = 0, out=None, stream=None) -> float:
        ids_a = np.ascontiguousarray(ids, dtype=np.int32)
        if out is None:
            out = self.outputs(ids)
        ms = ctypes.c_float()
        st = self.lib.grca_autotune(self.ctx, ids_a.ctypes.data, ids_a.shape[0], out[0].data_ptr(), out[1].data_ptr(),
                                    int(flags), _stream_ptr(stream), ctypes.byref(ms))
        self._check(st, "grca_autotune")
        return ms.value

    def set_debug_dump(self, pairs=None, counter=None):
        if pairs is None:
            self._check(self.lib.grca_set_debug_dump(self.ctx, None, 0, None), "grca_set_debug_dump")
            return
        self._check(self.lib.grca_set_debug_dump(self.ctx, pairs.data_ptr(), pairs.numel() // 2, counter.data_ptr()),
                    "grca_set_debug_dump")

    def stats(self, stream=None, check: bool = True) -> dict:
        s = grca_stats()
        st = self.lib.grca_get_stats(self.ctx, ctypes.byref(s), _stream_ptr(stream))
        if check:
            self._check(st, "grca_get_stats")
        d = s.as_dict()
        d["status"] = st
        return d

    def last_launch_count(self) -> int:
        return int(self.lib.grca_last_launch_count(self.ctx))

    def profile(self, enable: bool):
        self._check(self.lib.grca_profile_enable(self.ctx, int(bool(enable))), "grca_profile_enable")

    def profile_read(self) -> dict:
        n = 16
        names = (ctypes.c_char_p * n)()
        launches = (ctypes.c_uint64 * n)()
        tot = (ctypes.c_double * n)()
        cnt = ctypes.c_uint32()
        self._check(self.lib.grca_profile_read(self.ctx, n, names, launches, tot, ctypes.byref(cnt)),
                    "grca_profile_read")
        return {names[k].decode(): {"launches": int(launches[k]), "total_ms": float(tot[k])}
                for k in range(min(n, cnt.value))}


__all__ = ["Caster", "GrcaError", "CAST_FP64_RECHECK", "CAST_CULL_BACKFACE", "CAST_BRUTE", "CAST_GRAPH",
           "CAST_DUMP_CANDIDATES", "CAST_LOSSY_AREA", "NO_HIT", "EXPORTS", "library_path", "grca_options", "grca_sensor_desc",
           "grca_stats"]
