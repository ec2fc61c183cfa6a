"""Seeded synthetic scenes and LiDAR rigs for the GRCA workloads.

This module is INPUT DATA ONLY: closed triangle meshes, their per-frame
animation and the sensor descriptors (origin, axes, channel elevation table,
azimuth grid, range).  It contains no intersection, culling or closest-hit
arithmetic; both the CUDA path and the CPU oracle consume its arrays.

World frame: right-handed, z up, x forward.  All triangle vertices are
float32, unindexed, shape [n, 3, 3] (triangle, vertex, xyz).  Meshes are
built indexed and gathered, so triangles that share an edge share the
bit-identical vertex values (closed, watertight meshes with outward winding,
normal = (v1-v0) x (v2-v0)).

The paper's benchmark meshes (Power Plant, sports car, ...) are not
available; the configurations below reproduce their shapes and sizes
(triangle counts, dynamic share, sensor rigs, motion and deformation kinds)
with seeded procedural geometry.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

DT = 0.01  # frame step, seconds (the paper's 100 Hz simulation clock)


# ----------------------------------------------------------------------------
# sensors
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Sensor:
    """One spinning LiDAR: origin, orthonormal axes (forward f, right r, up u),
    ascending channel elevations (radians), a uniform azimuth grid
    theta_i = theta0 + i*dtheta for i in [0, n_rays) (or, with noise, the
    listed per-ray azimuths), and the range [d_min, d_max]."""
    origin: np.ndarray
    f: np.ndarray
    r: np.ndarray
    u: np.ndarray
    elev: np.ndarray
    n_rays: int
    theta0: float
    dtheta: float
    d_min: float = 0.0
    d_max: float = math.inf
    azimuths: Optional[np.ndarray] = None   # per-ray azimuths replacing the uniform grid (noise)

    @property
    def n_channels(self) -> int:
        return int(self.elev.shape[0])

    @property
    def n_total(self) -> int:
        return self.n_channels * self.n_rays


def channel_table(kind: str) -> np.ndarray:
    """Elevation tables in radians, ascending."""
    if kind == "uniform16":          # -15 .. +15 deg, 2 deg steps (16 channels)
        deg = -15.0 + 2.0 * np.arange(16)
    elif kind == "t128":             # 128 channels, denser near 0 deg
        low = -25.0 + 0.7 * np.arange(30)                # -25.0 .. -4.7
        mid = (np.arange(81) - 40) / 10.0                 # -4.0 .. +4.0 (exact 0 at k=40)
        high = 4.0 + (11.0 / 17.0) * np.arange(1, 18)     # 4.647 .. 15.0
        deg = np.concatenate([low, mid, high])
    elif kind == "c32":              # -16 .. +15 deg, 1 deg steps
        deg = np.arange(32) - 16.0
    elif kind == "c64":              # -20 .. +11.5 deg, 0.5 deg steps
        deg = (np.arange(64) - 40) / 2.0
    else:
        raise ValueError(kind)
    rad = np.deg2rad(deg.astype(np.float64))
    assert np.all(np.diff(rad) > 0)
    return rad


def subsample_channels(elev: np.ndarray, step: int) -> np.ndarray:
    return np.ascontiguousarray(elev[::step])


def make_sensor(origin, yaw: float = 0.0, channels: str = "t128", n_rays: int = 4096,
                fov_deg: float = 360.0, d_min: float = 0.0, d_max: float = math.inf,
                elev: Optional[np.ndarray] = None, pitch: float = 0.0, roll: float = 0.0) -> Sensor:
    """Sensor whose forward axis points at world yaw `yaw` (radians from +x toward +y),
    optionally pitched/rolled.  Right = forward rotated by -90 deg about up, so that
    the azimuth increases clockwise seen from above (from f toward r)."""
    cy, sy = math.cos(yaw), math.sin(yaw)
    f = np.array([cy, sy, 0.0])
    r = np.array([sy, -cy, 0.0])
    u = np.array([0.0, 0.0, 1.0])
    if pitch != 0.0 or roll != 0.0:
        # pitch: rotate f and u about r; roll: rotate r and u about f
        cp, sp = math.cos(pitch), math.sin(pitch)
        f, u = cp * f + sp * u, -sp * f + cp * u
        cr, sr = math.cos(roll), math.sin(roll)
        r, u = cr * r + sr * u, -sr * r + cr * u
    if elev is None:
        elev = channel_table(channels)
    if abs(fov_deg - 360.0) < 1e-12:
        dtheta = 2.0 * math.pi / n_rays
        theta0 = -math.pi
    else:
        fov = math.radians(fov_deg)
        dtheta = fov / n_rays
        theta0 = -(n_rays // 2) * dtheta
    return Sensor(origin=np.asarray(origin, dtype=np.float64), f=f, r=r, u=u,
                  elev=np.asarray(elev, dtype=np.float64), n_rays=int(n_rays),
                  theta0=float(theta0), dtheta=float(dtheta), d_min=float(d_min), d_max=float(d_max))


def noisy_sensor(s: Sensor, seed: int, az_frac: float = 0.45, elev_frac: float = 0.3) -> Sensor:
    """Copy of `s` with per-ray azimuths drawn uniformly within +-az_frac*dtheta of the
    grid and channel elevations moved by up to +-elev_frac of the smaller neighbouring
    gap (so they stay ascending): horizontal and vertical angular noise."""
    rng = np.random.default_rng(seed)
    th = s.theta0 + np.arange(s.n_rays) * s.dtheta + rng.uniform(-az_frac, az_frac, s.n_rays) * s.dtheta
    e = np.asarray(s.elev, np.float64)
    gap = np.diff(e)
    lim = np.minimum(np.concatenate([[gap[0]], gap]), np.concatenate([gap, [gap[-1]]])) if e.size > 1 else \
        np.array([1e-3])
    e2 = e + rng.uniform(-elev_frac, elev_frac, e.size) * lim
    return dataclasses.replace(s, elev=e2, azimuths=th)


def ray_mask(s: Sensor, seed: int, density: float = 0.5, kind: str = "random") -> np.ndarray:
    """uint32 on/off words over the channel x ray grid (bit q & 31 of word q >> 5 for
    q = j*n_rays + i): "random" (each ray fires with probability `density`),
    "sector" (a contiguous azimuth window of a non-spinning sensor) or "stripes"
    (every other channel, a scan-pattern image)."""
    n = s.n_channels * s.n_rays
    j, i = np.divmod(np.arange(n), s.n_rays)
    if kind == "random":
        on = np.random.default_rng(seed).random(n) < density
    elif kind == "sector":
        w = max(1, int(density * s.n_rays))
        start = int(np.random.default_rng(seed).integers(s.n_rays))
        on = ((i - start) % s.n_rays) < w
    elif kind == "stripes":
        on = (j + seed) % 2 == 0
    else:
        raise ValueError(kind)
    bits = np.zeros(((n + 31) // 32) * 32, bool)
    bits[:n] = on
    return np.packbits(bits.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).ravel()


def ray_offsets(sensors: List[Sensor]) -> np.ndarray:
    """Global ray offset O_n of each sensor (rays are sensor-major, then channel, then ray)."""
    off = [0]
    for s in sensors:
        off.append(off[-1] + s.n_total)
    return np.array(off, dtype=np.int64)


# ----------------------------------------------------------------------------
# meshes (indexed, then gathered)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Mesh:
    verts: np.ndarray   # float64 [nv, 3], object-local
    faces: np.ndarray   # int64 [nf, 3]


def grid_mesh(x0, x1, y0, y1, nx, ny, z=0.0) -> Mesh:
    xs = x0 + (x1 - x0) * (np.arange(nx + 1) / nx)
    ys = y0 + (y1 - y0) * (np.arange(ny + 1) / ny)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    a = (i * (ny + 1) + j).ravel()
    b = ((i + 1) * (ny + 1) + j).ravel()
    c = ((i + 1) * (ny + 1) + j + 1).ravel()
    d = (i * (ny + 1) + j + 1).ravel()
    faces = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], axis=0)
    return Mesh(verts, faces)


def box_mesh(size, n=1) -> Mesh:
    """Closed box centred at 0 with sides `size`, each face split into n x n quads.
    Lattice points are shared between faces (one vertex per surface lattice point)."""
    n = max(1, int(n))
    sx, sy, sz = (float(s) for s in size)
    L = n + 1
    surf = np.zeros((L, L, L), dtype=bool)
    surf[[0, -1], :, :] = True
    surf[:, [0, -1], :] = True
    surf[:, :, [0, -1]] = True
    pts = np.argwhere(surf)
    idx = -np.ones((L, L, L), dtype=np.int64)
    idx[surf] = np.arange(pts.shape[0])
    verts = np.stack([sx * (pts[:, 0] / n - 0.5), sy * (pts[:, 1] / n - 0.5), sz * (pts[:, 2] / n - 0.5)], 1)
    pg, qg = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pg, qg = pg.ravel(), qg.ravel()
    faces = []
    for axis in range(3):
        ax = [a for a in range(3) if a != axis]
        e = np.zeros(3); e[ax[0]] = 1
        g = np.zeros(3); g[ax[1]] = 1
        sgn = np.cross(e, g)[axis]
        for side, outward in ((0, False), (n, True)):
            def lat(a_, b_):
                c = [None, None, None]
                c[axis] = np.full_like(a_, side)
                c[ax[0]] = a_
                c[ax[1]] = b_
                return idx[c[0], c[1], c[2]]
            v00, v10, v11, v01 = lat(pg, qg), lat(pg + 1, qg), lat(pg + 1, qg + 1), lat(pg, qg + 1)
            if (sgn > 0) == outward:
                faces += [np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)]
            else:
                faces += [np.stack([v00, v11, v10], 1), np.stack([v00, v01, v11], 1)]
    return Mesh(verts.astype(np.float64), np.concatenate(faces, 0).astype(np.int64))


def ellipsoid_mesh(radii, n_slices, n_stacks) -> Mesh:
    """Closed UV ellipsoid centred at 0: shared poles and seam, outward winding."""
    n_slices = max(3, int(n_slices))
    n_stacks = max(2, int(n_stacks))
    rx, ry, rz = (float(v) for v in radii)
    th = 2.0 * np.pi * np.arange(n_slices) / n_slices
    ph = np.pi * np.arange(1, n_stacks) / n_stacks  # polar angle, rings only
    P, T = np.meshgrid(ph, th, indexing="ij")       # [rings, slices]
    ring = np.stack([rx * np.sin(P) * np.cos(T), ry * np.sin(P) * np.sin(T), rz * np.cos(P)], -1).reshape(-1, 3)
    top = np.array([[0.0, 0.0, rz]])
    bot = np.array([[0.0, 0.0, -rz]])
    verts = np.concatenate([top, ring, bot], 0)
    nr = n_stacks - 1
    ib = 1 + nr * n_slices

    def rv(k, s):
        return 1 + k * n_slices + (s % n_slices)

    faces = []
    s = np.arange(n_slices)
    faces.append(np.stack([np.zeros_like(s), rv(0, s), rv(0, s + 1)], 1))
    for k in range(nr - 1):
        a, b, c, d = rv(k, s), rv(k + 1, s), rv(k + 1, s + 1), rv(k, s + 1)
        faces.append(np.stack([a, b, c], 1))
        faces.append(np.stack([a, c, d], 1))
    faces.append(np.stack([rv(nr - 1, s), np.full_like(s, ib), rv(nr - 1, s + 1)], 1))
    return Mesh(verts, np.concatenate(faces, 0).astype(np.int64))


def ellipsoid_for_count(radii, n_tris) -> Mesh:
    # 2*slices*(stacks-1) triangles; slices ~ 2*stacks
    st = max(2, int(round(math.sqrt(max(n_tris, 8) / 4.0))))
    sl = max(3, int(round(n_tris / (2.0 * max(st - 1, 1)))))
    return ellipsoid_mesh(radii, sl, st)


def box_for_count(size, n_tris) -> Mesh:
    return box_mesh(size, max(1, int(round(math.sqrt(max(n_tris, 12) / 12.0)))))


def vertex_normals_ellipsoid(verts: np.ndarray, radii) -> np.ndarray:
    g = verts / np.square(np.asarray(radii, dtype=np.float64))
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    return g / np.maximum(nrm, 1e-30)


def yaw_matrix(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


# ----------------------------------------------------------------------------
# scene with animation
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class RigidGroup:
    mesh: Mesh
    c0: np.ndarray        # [k,3] centre at t=0
    yaw0: np.ndarray      # [k]
    vel: np.ndarray       # [k,3] m/s
    yaw_rate: np.ndarray  # [k] rad/s
    n_inst: int


@dataclasses.dataclass
class DeformObject:
    mesh: Mesh
    normals: np.ndarray   # [nv,3]
    c0: np.ndarray        # [3]
    amp: float
    freq: float
    wave: np.ndarray      # [3] phase gradient (rad/m)


@dataclasses.dataclass
class Scene:
    name: str
    sensors: List[Sensor]
    static_tris: np.ndarray                 # float32 [ns,3,3]
    rigid: List[RigidGroup] = dataclasses.field(default_factory=list)
    deform: List[DeformObject] = dataclasses.field(default_factory=list)
    stress_rays: Optional[np.ndarray] = None  # int64 global ray ids aimed at stress geometry
    n_frames: int = 1
    dynamic_ground: bool = False            # ground rewritten every frame (fully dynamic)

    @property
    def n_static(self) -> int:
        return int(self.static_tris.shape[0])

    @property
    def n_dynamic(self) -> int:
        n = sum(g.mesh.faces.shape[0] * g.n_inst for g in self.rigid)
        n += sum(d.mesh.faces.shape[0] for d in self.deform)
        return int(n)

    @property
    def n_tris(self) -> int:
        return self.n_static + self.n_dynamic

    @property
    def n_rays(self) -> int:
        return int(sum(s.n_total for s in self.sensors))

    def dynamic_tris(self, frame: int) -> np.ndarray:
        """float32 [n_dynamic,3,3] at time frame*DT (rigid movers then deforming meshes)."""
        t = frame * DT
        parts = []
        for g in self.rigid:
            V = g.mesh.verts  # [nv,3]
            yaw = g.yaw0 + g.yaw_rate * t
            c, s = np.cos(yaw), np.sin(yaw)
            cen = g.c0 + g.vel * t
            x = c[:, None] * V[None, :, 0] - s[:, None] * V[None, :, 1] + cen[:, 0:1]
            y = s[:, None] * V[None, :, 0] + c[:, None] * V[None, :, 1] + cen[:, 1:2]
            z = np.broadcast_to(V[None, :, 2], x.shape) + cen[:, 2:3]
            W = np.stack([x, y, z], -1).astype(np.float32)       # [k,nv,3]
            parts.append(W[:, g.mesh.faces].reshape(-1, 3, 3))
        for d in self.deform:
            V = d.mesh.verts
            ph = 2.0 * math.pi * d.freq * t + V @ d.wave
            W = (d.c0 + V + (d.amp * np.sin(ph))[:, None] * d.normals).astype(np.float32)
            parts.append(W[d.mesh.faces])
        if not parts:
            return np.zeros((0, 3, 3), np.float32)
        return np.ascontiguousarray(np.concatenate(parts, 0))

    def tris(self, frame: int = 0) -> np.ndarray:
        """float32 [n_tris,3,3]: static triangles first, then the dynamic ones."""
        dyn = self.dynamic_tris(frame)
        if dyn.shape[0] == 0:
            return self.static_tris
        return np.ascontiguousarray(np.concatenate([self.static_tris, dyn], 0))


def gather(mesh: Mesh, offset=(0.0, 0.0, 0.0), rot: Optional[np.ndarray] = None) -> np.ndarray:
    V = mesh.verts if rot is None else mesh.verts @ rot.T
    V = (V + np.asarray(offset, dtype=np.float64)).astype(np.float32)
    return V[mesh.faces]


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def _place_disk(rng, n, r_min, r_max, keepout_xy, clearance):
    out = []
    while len(out) < n:
        rr = math.sqrt(rng.uniform(r_min * r_min, r_max * r_max))
        a = rng.uniform(-math.pi, math.pi)
        p = (rr * math.cos(a), rr * math.sin(a))
        if all(math.hypot(p[0] - k[0], p[1] - k[1]) > clearance for k in keepout_xy):
            out.append(p)
    return out


def scene_c1(seed: int = 1) -> Scene:
    """1 LiDAR at (0,0,1.8), 16 channels -15..+15 deg x 512 rays, 360 deg.
    40x40 m ground (70x70 quads, 9800 triangles) + 20 closed boxes
    (sides U(0.5,4) m, centres uniform in the r<=30 m disk, resting on z=0,
    none within 1 m of the sensor): 10,040 triangles, static."""
    rng = np.random.default_rng(seed)
    sensor = make_sensor((0.0, 0.0, 1.8), channels="uniform16", n_rays=512)
    parts = [gather(grid_mesh(-20.0, 20.0, -20.0, 20.0, 70, 70))]
    n_box = 0
    while n_box < 20:
        size = rng.uniform(0.5, 4.0, 3)
        rr = 30.0 * math.sqrt(rng.uniform())
        a = rng.uniform(-math.pi, math.pi)
        cx, cy = rr * math.cos(a), rr * math.sin(a)
        # reject a box whose footprint comes within 1 m of the sensor's xy
        dx = max(abs(cx) - size[0] / 2, 0.0)
        dy = max(abs(cy) - size[1] / 2, 0.0)
        if math.hypot(dx, dy) < 1.0:
            continue
        parts.append(gather(box_mesh(size, 1), (cx, cy, size[2] / 2)))
        n_box += 1
    return Scene("c1", [sensor], np.ascontiguousarray(np.concatenate(parts, 0)))


def _object_field(rng, tri_budget, surf_lo, surf_hi, area_lo, area_hi, r_min, r_max, keepout, max_tris=20000):
    """Closed static objects (boxes and ellipsoids) until `tri_budget`
    triangles: surface log-uniform in [surf_lo, surf_hi] m^2, triangle area
    log-uniform in [area_lo, area_hi] m^2 per object (clipped so an object has
    12 .. max_tris triangles), yaw uniform, centres uniform in the annulus."""
    parts = []
    total = 0
    while total < tri_budget:
        surf = math.exp(rng.uniform(math.log(surf_lo), math.log(surf_hi)))
        a_t = math.exp(rng.uniform(math.log(area_lo), math.log(area_hi)))
        a_t = min(max(a_t, surf / max_tris), surf / 12.0)
        n_t = max(12, min(max_tris, tri_budget - total, int(round(surf / a_t))))
        aspect = rng.uniform(0.4, 1.0, 3)
        cx, cy = _place_disk(rng, 1, r_min, r_max, keepout, 4.0)[0]
        if rng.uniform() < 0.5:
            q = 2.0 * (aspect[0] * aspect[1] + aspect[1] * aspect[2] + aspect[2] * aspect[0])
            size = math.sqrt(surf / q) * aspect
            m = box_for_count(size, n_t)
            zc = size[2] / 2
        else:
            radii = math.sqrt(surf / (4.0 * math.pi * float(np.mean(aspect * aspect)))) * aspect
            m = ellipsoid_for_count(radii, n_t)
            zc = radii[2] * rng.uniform(0.3, 1.2)
        parts.append(gather(m, (cx, cy, zc), yaw_matrix(rng.uniform(-math.pi, math.pi))))
        total += m.faces.shape[0]
    return parts


def _rigid_movers(rng, n_inst, tris_per_obj, kind, r_min, r_max, keepout, scale_lo, scale_hi):
    base = np.array([4.57, 2.28, 1.08])  # reference vehicle (the paper's sports car at scale 1)
    groups = []
    centres = _place_disk(rng, n_inst, r_min, r_max, keepout, 6.0)
    for k in range(n_inst):
        sc = rng.uniform(scale_lo, scale_hi, 3)
        dims = base * sc
        if kind == "box" or (kind == "mixed" and k % 2 == 0):
            m = box_for_count(dims, tris_per_obj)
            z = dims[2] / 2
        else:
            m = ellipsoid_for_count(dims / 2, tris_per_obj)
            z = dims[2] / 2
        speed = rng.uniform(0.0, 30.0)
        head = rng.uniform(-math.pi, math.pi)
        vel = np.array([[speed * math.cos(head), speed * math.sin(head), 0.0]])
        rate = rng.uniform(0.0, 1.0) * (1 if rng.uniform() < 0.5 else -1)
        groups.append(RigidGroup(m, np.array([[centres[k][0], centres[k][1], z]]),
                                 np.array([rng.uniform(-math.pi, math.pi)]), vel, np.array([rate]), 1))
    return groups


def _deformers(rng, n_obj, tris_per_obj, r_min, r_max, keepout, radii_range=(0.5, 3.0)):
    out = []
    centres = _place_disk(rng, n_obj, r_min, r_max, keepout, 5.0)
    for k in range(n_obj):
        radii = rng.uniform(radii_range[0], radii_range[1], 3)
        m = ellipsoid_for_count(radii, tris_per_obj)
        nrm = vertex_normals_ellipsoid(m.verts, radii)
        amp = rng.uniform(0.05, 0.5)
        c0 = np.array([centres[k][0], centres[k][1], radii[2] + amp + rng.uniform(0.0, 2.0)])
        out.append(DeformObject(m, nrm, c0, amp, rng.uniform(0.5, 2.0), rng.normal(0.0, 1.0, 3)))
    return out


# C4/C5 static objects: ~10.8 M triangles of closed objects, surface 0.5-100 m^2,
# triangle area log-uniform 1e-4..1 m^2 (mean ~ the paper's Power Plant, 384 cm^2)
C45_STATIC = 10_800_000
C45_SURF = (0.5, 100.0)
C45_AREA = (1e-4, 1.0)


def rig_c4(d_max=math.inf, d_min=0.05):
    t = channel_table("t128")
    s = [make_sensor((0.0, 0.0, 2.2), channels="c32", n_rays=1024, d_min=d_min, d_max=d_max),
         make_sensor((1.0, 0.0, 2.0), channels="c64", n_rays=2048, d_min=d_min, d_max=d_max)]
    for (x, y) in [(1.5, 0.8), (1.5, -0.8), (-1.5, 0.8), (-1.5, -0.8)]:
        s.append(make_sensor((x, y, 1.9), elev=t, n_rays=4096, d_min=d_min, d_max=d_max))
    s.append(make_sensor((2.3, 0.0, 0.6), yaw=0.0, elev=t, n_rays=4096, fov_deg=180.0, d_min=d_min, d_max=d_max))
    s.append(make_sensor((-2.3, 0.0, 0.6), yaw=math.pi, elev=t, n_rays=4096, fov_deg=180.0, d_min=d_min, d_max=d_max))
    return s


def rig_c5(d_min=0.05):
    t = channel_table("t128")
    slots = [(0.0, 0.0, 2.2), (1.0, 0.0, 2.0), (1.5, 0.8, 1.9), (1.5, -0.8, 1.9),
             (-1.5, 0.8, 1.9), (-1.5, -0.8, 1.9), (2.3, 0.0, 0.6), (-2.3, 0.0, 0.6)]
    return [make_sensor(p, elev=t, n_rays=4096, d_min=d_min) for p in slots]


def _big_scene(name, sensors, seed, ground_n, static_budget, surf, area, n_rigid, rigid_tpo, n_deform,
               deform_tpo, extent=100.0, n_frames=50, mover_scale=(0.3, 1.2), deform_radii=(0.3, 1.5)):
    rng = np.random.default_rng(seed)
    keep = [(float(s.origin[0]), float(s.origin[1])) for s in sensors]
    parts = []
    if ground_n > 0:
        parts.append(gather(grid_mesh(-extent, extent, -extent, extent, ground_n, ground_n)))
    if static_budget > 0:
        parts += _object_field(rng, static_budget, surf[0], surf[1], area[0], area[1], 8.0, extent * 0.95, keep)
    static = np.ascontiguousarray(np.concatenate(parts, 0)) if parts else np.zeros((0, 3, 3), np.float32)
    rigid = _rigid_movers(rng, n_rigid, rigid_tpo, "mixed", 10.0, extent * 0.8, keep, *mover_scale) if n_rigid else []
    deform = _deformers(rng, n_deform, deform_tpo, 8.0, extent * 0.8, keep, deform_radii) if n_deform else []
    return Scene(name, sensors, static, rigid, deform, n_frames=n_frames)


def scene_c2(seed: int = 2, mini: bool = False) -> Scene:
    """1 LiDAR 128ch (non-uniform) x 4096, 360 deg; ~1.0 M triangles: a 200x200 m
    ground (1 m cells, 80k triangles, rewritten every frame) plus 2000 closed
    box/ellipsoid movers whose triangle counts are log-distributed between
    12 and ~50k, all rigidly moving (speed U(0,30) m/s, yaw rate U(0,1) rad/s)."""
    rng = np.random.default_rng(seed)
    div = 100 if mini else 1
    sens = make_sensor((0.0, 0.0, 1.8), channels="t128", n_rays=4096)
    if mini:
        sens = make_sensor((0.0, 0.0, 1.8), elev=subsample_channels(channel_table("t128"), 4), n_rays=1024)
    gn = 200 if not mini else 20
    ground = gather(grid_mesh(-100.0, 100.0, -100.0, 100.0, gn, gn))
    n_obj = 2000 // (10 if mini else 1)
    # per-mesh triangle counts c_i = 12 * (50000/12)^(u^a), a solved so the total is ~1M
    u = rng.uniform(0.0, 1.0, n_obj)
    target = (1_000_000 - ground.shape[0]) // div

    def tot(a):
        return float(np.sum(np.round(12.0 * (50000.0 / 12.0) ** (u ** a))))
    lo, hi = 0.01, 200.0
    for _ in range(80):
        mid = math.sqrt(lo * hi)
        if tot(mid) > target:
            lo = mid
        else:
            hi = mid
    counts = np.round(12.0 * (50000.0 / 12.0) ** (u ** hi)).astype(int)
    keep = [(0.0, 0.0)]
    centres = _place_disk(rng, n_obj, 8.0, 95.0, keep, 4.0)
    rigid = []
    for k in range(n_obj):
        size = rng.uniform(0.5, 20.0) * rng.uniform(0.3, 1.0, 3)
        if k % 2 == 0:
            m = box_for_count(size, counts[k])
        else:
            m = ellipsoid_for_count(size / 2, counts[k])
        speed = rng.uniform(0.0, 30.0)
        head = rng.uniform(-math.pi, math.pi)
        rate = rng.uniform(0.0, 1.0) * (1 if rng.uniform() < 0.5 else -1)
        rigid.append(RigidGroup(m, np.array([[centres[k][0], centres[k][1], size[2] / 2 + 0.01]]),
                                np.array([rng.uniform(-math.pi, math.pi)]),
                                np.array([[speed * math.cos(head), speed * math.sin(head), 0.0]]),
                                np.array([rate]), 1))
    sc = Scene("c2m" if mini else "c2", [sens], ground, rigid, [], n_frames=50)
    sc.dynamic_ground = True
    return sc


def scene_c3(seed: int = 3, mini: bool = False) -> Scene:
    """2 LiDARs 128x4096 (360 deg at (0,0,1.8); 180 deg front at (2,0,1.8));
    5 M triangles: 3 M static (ground 180k + closed objects with triangle areas
    log-uniform in [1e-4, 10] m^2) and 2 M dynamic (400 deforming ellipsoids of
    5k triangles, per-vertex sinusoidal displacement of amplitude 0.05-0.5 m)."""
    t = channel_table("t128")
    if mini:
        t = subsample_channels(t, 4)
    nr = 1024 if mini else 4096
    s = [make_sensor((0.0, 0.0, 1.8), elev=t, n_rays=nr),
         make_sensor((2.0, 0.0, 1.8), elev=t, n_rays=nr, fov_deg=180.0)]
    if mini:
        return _big_scene("c3m", s, seed, 30, 28_000, (1.0, 300.0), (1e-4, 10.0), 0, 0, 4, 5000,
                          deform_radii=(0.5, 3.0))
    return _big_scene("c3", s, seed, 300, 2_820_000, (1.0, 300.0), (1e-4, 10.0), 0, 0, 400, 5000,
                      deform_radii=(0.5, 3.0))


def scene_c4(seed: int = 4, d_max=math.inf, mini: bool = False) -> Scene:
    """8 LiDARs {32x1024, 64x2048, 4x 128x4096, 2x 128x4096 180 deg} on one rig;
    ~22 M triangles: ~13 M static (2 M ground + closed objects) and ~9 M dynamic
    (~6 M rigid movers + ~3 M deforming meshes)."""
    sens = rig_c4(d_max=d_max)
    if mini:
        for s in sens:
            s.elev = subsample_channels(s.elev, 4)
            s.n_rays //= 4
            s.dtheta *= 4
            s.theta0 = -math.pi if abs(s.n_rays * s.dtheta - 2 * math.pi) < 1e-9 else -(s.n_rays // 2) * s.dtheta
        return _big_scene("c4m", sens, seed, 140, 108_000, C45_SURF, C45_AREA, 12, 5000, 6, 5000)
    return _big_scene("c4", sens, seed, 1000, C45_STATIC, C45_SURF, C45_AREA, 1200, 5000, 600, 5000)


def stress_set(sensors: List[Sensor], rng, n_items: int):
    """Near-tie stress geometry aimed along chosen rays: coplanar overlapping
    pairs on axis-aligned planes (exact float32 coplanarity), shared-edge fans
    around a hub on the ray, and slivers (aspect up to 1e4) whose long edge
    passes through the ray.  Returns (triangles float32 [n,3,3], aimed ray ids)."""
    offs = ray_offsets(sensors)
    tris = []
    rays = []
    for k in range(n_items):
        n = int(rng.integers(len(sensors)))
        s = sensors[n]
        j = int(rng.integers(s.n_channels))
        i = int(rng.integers(s.n_rays))
        th = s.theta0 + i * s.dtheta
        ph = s.elev[j]
        d = math.cos(th) * math.cos(ph) * s.f + math.sin(th) * math.cos(ph) * s.r + math.sin(ph) * s.u
        L = rng.uniform(5.0, 80.0)
        P = s.origin + L * d
        kind = k % 3
        if kind == 0:
            # coplanar overlapping pair on the axis plane most facing the ray
            ax = int(np.argmax(np.abs(d[:2])))
            o1, o2 = [a for a in range(3) if a != ax]
            c = np.float32(P[ax])
            w = rng.uniform(0.2, 1.0)
            sh = rng.uniform(0.1, 0.5) * w
            def tri(du, dv, rot):
                T = np.zeros((3, 3))
                T[:, ax] = c
                for vi, (a_, b_) in enumerate(rot):
                    T[vi, o1] = P[o1] + du + a_
                    T[vi, o2] = P[o2] + dv + b_
                return T
            base = [(-w, -w), (w, -w), (0.0, w)]
            sg = np.sign(d[ax]) if d[ax] != 0 else 1.0
            T1 = tri(0.0, 0.0, base)
            T2 = tri(sh * rng.uniform(-1, 1), sh * rng.uniform(-1, 1), base)
            for T in (T1, T2):
                nrm = np.cross(T[1] - T[0], T[2] - T[0])
                if np.dot(nrm, s.origin - T[0]) < 0:
                    T[[1, 2]] = T[[2, 1]]
                tris.append(T.astype(np.float32))
        elif kind == 1:
            # fan of m triangles around hub P in the plane facing the sensor
            m = int(rng.integers(6, 13))
            e1 = np.cross(d, s.u); e1 /= np.linalg.norm(e1)
            e2 = np.cross(e1, d)
            hub = P.astype(np.float32).astype(np.float64)
            rad = rng.uniform(0.1, 1.0)
            ang = np.sort(rng.uniform(0, 2 * np.pi, m)) if rng.uniform() < 0.5 else 2 * np.pi * np.arange(m) / m
            rim = [(hub + rad * (math.cos(a) * e1 + math.sin(a) * e2)).astype(np.float32) for a in ang]
            for q in range(m):
                T = np.stack([hub.astype(np.float32), rim[q], rim[(q + 1) % m]]).astype(np.float32)
                nrm = np.cross(T[1].astype(np.float64) - T[0], T[2].astype(np.float64) - T[0])
                if np.dot(nrm, s.origin - T[0]) < 0:
                    T[[1, 2]] = T[[2, 1]]
                tris.append(T)
        else:
            # sliver whose long edge passes through P
            length = rng.uniform(0.5, 5.0)
            aspect = math.exp(rng.uniform(math.log(10.0), math.log(1e4)))
            e1 = np.cross(d, s.u); e1 /= np.linalg.norm(e1)
            e2 = np.cross(e1, d)
            a = rng.uniform(0, 2 * np.pi)
            ax_ = math.cos(a) * e1 + math.sin(a) * e2
            bx_ = -math.sin(a) * e1 + math.cos(a) * e2
            f0 = rng.uniform(0.2, 0.8)
            A = P - f0 * length * ax_
            B = P + (1 - f0) * length * ax_
            C = A + 0.5 * length * ax_ + (length / aspect) * bx_
            T = np.stack([A, B, C]).astype(np.float32)
            nrm = np.cross(T[1].astype(np.float64) - T[0], T[2].astype(np.float64) - T[0])
            if np.dot(nrm, s.origin - T[0]) < 0:
                T[[1, 2]] = T[[2, 1]]
            tris.append(T)
        rays.append(int(offs[n] + j * s.n_rays + i))
    return np.ascontiguousarray(np.stack(tris, 0)), np.array(rays, dtype=np.int64)


def scene_c5(seed: int = 5, mini: bool = False, n_stress: int = 1500) -> Scene:
    """8 LiDARs 128x4096 360 deg at the rig's slots; the 22 M-triangle scene
    plus the near-tie stress set (coplanar pairs, fans, slivers on ray paths);
    60 animated frames."""
    sens = rig_c5()
    if mini:
        for s in sens:
            s.elev = subsample_channels(s.elev, 4)
            s.n_rays //= 4
            s.dtheta *= 4
        sc = _big_scene("c5m", sens, seed, 140, 108_000, C45_SURF, C45_AREA, 12, 5000, 6, 5000, n_frames=60)
    else:
        sc = _big_scene("c5", sens, seed, 1000, C45_STATIC, C45_SURF, C45_AREA, 1200, 5000, 600, 5000, n_frames=60)
    rng = np.random.default_rng(seed + 1000)
    st, rays = stress_set(sens, rng, n_stress if not mini else max(30, n_stress // 50))
    sc.static_tris = np.ascontiguousarray(np.concatenate([sc.static_tris, st], 0))
    sc.stress_rays = rays
    return sc


def make_config(name: str, **kw) -> Scene:
    table = {"c1": scene_c1, "c2": scene_c2, "c3": scene_c3, "c4": scene_c4, "c5": scene_c5}
    if name.endswith("m") and name[:-1] in table:
        return table[name[:-1]](mini=True, **kw)
    return table[name](**kw)


def tiny_scene(seed: int, n_tris: int = 200, extent: float = 10.0):
    """Random small triangles scattered around a sensor (for property tests)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, (n_tris, 1, 3))
    c[:, :, 2] = rng.uniform(-2.0, 4.0, (n_tris, 1))
    sz = np.exp(rng.uniform(math.log(0.05), math.log(3.0), (n_tris, 1, 1)))
    tris = (c + sz * rng.normal(0.0, 1.0, (n_tris, 3, 3))).astype(np.float32)
    return np.ascontiguousarray(tris)
