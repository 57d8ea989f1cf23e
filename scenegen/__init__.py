"""Seeded synthetic inputs: procedural interiors, cameras, probe grids and
synthetic per-pixel buffers.

This module holds only input data.  It builds triangle soups, per-triangle
albedo and emission, camera frames and probe-grid placements from a seed, and
random buffers shaped like the per-pixel G-buffer and reservoirs.  It performs
none of the rendering method's arithmetic (no ray casting, no probe update, no
resampling); both the CPU oracle and the CUDA path consume what it produces.

Workloads (stand-ins for the paper's third-party scenes of Sec. 4, which are
not available):

* ``tiny_room``   -- 2 m closed box, 24 triangles, one emissive ceiling quad
                     (radiance 10), 128x128 camera, 4x4x4 probes, 64 rays.
* ``apartment``   -- 4-room apartment (walls with doors, 400 furniture boxes),
                     about 64k triangles, 1024 emissive ceiling triangles with
                     radiance log-uniform in [1, 100], 1920x1080 camera path
                     translating 5 cm per frame, 16x8x16 probes, 256 rays.
* ``tiny_room_1080p`` -- the tiny room rendered at 1920x1080 (learned-target
                     workload).
* ``apartment_dynamic`` -- the apartment plus 200 boxes in sinusoidal rigid
                     motion, emitter halves swapping every 8 frames, probe
                     relocation on, 64 frames.
* ``tiny_room_dynamic`` -- the box with 3 moving boxes and toggling emitters
                     (small full-image case of the dynamics).
* ``multistorey`` -- 4-storey building, about 1M triangles, 8192 emissive
                     triangles, 500 moving boxes, 3840x2160, 32x16x32 probes,
                     64 candidates, 3 spatial passes, bf16 learned target.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

__all__ = [
    "Scene", "Camera", "ProbeGrid", "Settings", "Motion",
    "tiny_room", "tiny_room_1080p", "apartment", "apartment_dynamic", "tiny_room_dynamic", "multistorey",
    "make_scene", "secondary_ddgi",
    "synthetic_gbuffer", "synthetic_reservoirs", "synthetic_irradiance_interior",
    "synthetic_depth_interior",
]


# ---------------------------------------------------------------------------
# containers
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Camera:
    """Pinhole camera frame.  ``right``/``up``/``fwd`` are orthonormal."""
    pos: np.ndarray
    fwd: np.ndarray
    right: np.ndarray
    up: np.ndarray
    tan_half_fovy: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        """Packed float32[16]: pos, fwd, right, up (xyz each), tan, w, h, pad."""
        a = np.zeros(16, np.float32)
        a[0:3] = self.pos
        a[3:6] = self.fwd
        a[6:9] = self.right
        a[9:12] = self.up
        a[12] = self.tan_half_fovy
        a[13] = self.width
        a[14] = self.height
        return a


@dataclasses.dataclass
class ProbeGrid:
    origin: np.ndarray   # float32[3], position of probe (0,0,0)
    spacing: np.ndarray  # float32[3]
    counts: np.ndarray   # int32[3]

    @property
    def num_probes(self) -> int:
        return int(np.prod(self.counts))


@dataclasses.dataclass
class Settings:
    """Method parameters of one workload (readings listed in the design notes)."""
    rays_per_probe: int = 64
    irr_texels: int = 8
    depth_texels: int = 16
    hysteresis: float = 0.97
    le_attenuation: float = 1.0      # slider s; 0 disables the attenuation
    depth_sharpness: float = 50.0
    num_light_candidates: int = 31
    num_bsdf_candidates: int = 1
    candidate_stride: int = 1       # >= 2: only pixels with (x + y + frame) % stride == 0 generate candidates
    temporal_mcap: float = 20.0
    spatial_passes: int = 1
    spatial_neighbours: int = 5
    spatial_radius: int = 30
    normal_reject_cos: float = 0.9
    depth_reject_frac: float = 0.1
    seed: int = 1
    probe_relocation: int = 0    # 1: relocate probes after each update
    learned_target: int = 0      # 1: the network serves p-hat / termination queries
    train_samples: int = 0       # self-training samples per frame
    train_lr: float = 1e-3
    mlp_seed: int = 1
    train_ema: float = 0.97      # served network: moving average of the trained weights
    mlp_bf16: int = 0            # network in bf16 (1) or fp16 (0), fp32 accumulation
    footprint_c: float = 0.2     # path-footprint threshold c of the shading recursion (glossy scenes)


@dataclasses.dataclass
class Motion:
    """Rigid sinusoidal motion of instances about their identity pose: at
    frame f instance i is turned by spin_i (sin(2 pi f / T_i + phi_i) -
    sin(phi_i)) radians about the vertical axis through its centre and
    shifted by amp_i (same bracket) along its horizontal axis, so that frame
    0 is the identity."""
    center: np.ndarray     # float64[I, 3]
    axis: np.ndarray       # float64[I, 3] unit, horizontal
    amp: np.ndarray        # float64[I] metres
    spin: np.ndarray       # float64[I] radians
    period: np.ndarray     # float64[I] frames
    phase: np.ndarray      # float64[I]

    def transforms(self, frame: int) -> np.ndarray:
        """float32[I, 12]: row-major 3x4 transforms [R | t]."""
        s = np.sin(2 * np.pi * frame / self.period + self.phase) - np.sin(self.phase)
        th = self.spin * s
        c, n = np.cos(th), np.sin(th)
        I = len(self.amp)
        R = np.zeros((I, 3, 3))
        R[:, 0, 0], R[:, 0, 2], R[:, 1, 1], R[:, 2, 0], R[:, 2, 2] = c, n, 1.0, -n, c
        t = self.center - np.einsum("ijk,ik->ij", R, self.center) + self.axis * (self.amp * s)[:, None]
        M = np.concatenate([R, t[:, :, None]], axis=2)
        return M.reshape(I, 12).astype(np.float32)


@dataclasses.dataclass
class Scene:
    name: str
    verts: np.ndarray      # float32[T, 3, 3]
    albedo: np.ndarray     # float32[T, 3]
    emission: np.ndarray   # float32[T, 3]
    grid: ProbeGrid
    cameras: List[Camera]
    settings: Settings
    # dynamics (None: static): rigid instance of each triangle (-1 static),
    # its motion, and the period (frames) after which the two halves of the
    # emitters (even / odd position in the emitter list) swap on and off
    tri_instance: Optional[np.ndarray] = None     # int32[T]
    motion: Optional[Motion] = None
    emitter_toggle: int = 0
    # glossy lobe per triangle (None: a diffuse scene): k_s.rgb and GGX
    # roughness alpha; emitters have none
    glossy: Optional[np.ndarray] = None           # float32[T, 4]

    @property
    def num_tris(self) -> int:
        return int(self.verts.shape[0])

    @property
    def num_instances(self) -> int:
        return 0 if self.tri_instance is None else int(self.tri_instance.max(initial=-1)) + 1

    def instance_transforms(self, frame: int) -> Optional[np.ndarray]:
        return None if self.motion is None else self.motion.transforms(frame)

    def emitter_radiance(self, frame: int) -> Optional[np.ndarray]:
        """float32[E, 3] radiance of the emitters (emissive triangles in
        increasing index) at this frame: the even half is on during the first
        `emitter_toggle` frames of every 2 x `emitter_toggle`, the odd half
        during the others."""
        if not self.emitter_toggle:
            return None
        cached = self.__dict__.get("_emitter_le")
        if cached is None or cached[0] is not self.emission:
            cached = (self.emission, self.emission[self.emission.max(axis=1) > 0])
            self.__dict__["_emitter_le"] = cached   # the scan over every triangle runs once
        le = cached[1]
        on_even = (frame // self.emitter_toggle) % 2 == 0
        odd = (np.arange(len(le)) % 2) == 1
        lit = odd != on_even
        return np.where(lit[:, None], le, 0.0).astype(np.float32)


# ---------------------------------------------------------------------------
# geometry helpers (triangle soups with a winding that fixes the facing side)
# ---------------------------------------------------------------------------

def _quad(c, a, b, facing, nu=1, nv=1):
    """Quad centred at ``c`` with half-extent vectors ``a`` and ``b``, wound so
    that cross(v1 - v0, v2 - v0) points along ``facing``; split into
    ``nu x nv`` sub-quads (2 triangles each)."""
    c = np.asarray(c, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if np.dot(np.cross(a, b), facing) < 0:
        a, b = b, a
        nu, nv = nv, nu
    if nu * nv > 64:   # same triangles in the same order, built with array arithmetic
        i = np.repeat(np.arange(nu), nv)[:, None]
        j = np.tile(np.arange(nv), nu)[:, None]
        s0, s1 = -1 + 2 * i / nu, -1 + 2 * (i + 1) / nu
        t0, t1 = -1 + 2 * j / nv, -1 + 2 * (j + 1) / nv
        p0 = c + s0 * a + t0 * b
        p1 = c + s1 * a + t0 * b
        p2 = c + s1 * a + t1 * b
        p3 = c + s0 * a + t1 * b
        out = np.empty((2 * nu * nv, 3, 3))
        out[0::2] = np.stack([p0, p1, p2], 1)
        out[1::2] = np.stack([p0, p2, p3], 1)
        return out
    tris = []
    for i in range(nu):
        for j in range(nv):
            s0, s1 = -1 + 2 * i / nu, -1 + 2 * (i + 1) / nu
            t0, t1 = -1 + 2 * j / nv, -1 + 2 * (j + 1) / nv
            p0 = c + s0 * a + t0 * b
            p1 = c + s1 * a + t0 * b
            p2 = c + s1 * a + t1 * b
            p3 = c + s0 * a + t1 * b
            tris.append([p0, p1, p2])
            tris.append([p0, p2, p3])
    return tris


_AXES = np.eye(3)


def _box_faces(lo, hi, inward=False, tess=(1, 1, 1)):
    """The 6 faces of an axis-aligned box as lists of triangles.  ``tess[k]``
    is the number of subdivisions along axis k.  Normals point out of the solid
    (``inward=False``) or into the enclosed room (``inward=True``)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    faces = []
    for ax in range(3):
        u, v = [k for k in range(3) if k != ax]
        for sgn in (-1.0, 1.0):
            fc = c.copy()
            fc[ax] += sgn * h[ax]
            facing = _AXES[ax] * (sgn if not inward else -sgn)
            faces.append(_quad(fc, _AXES[u] * h[u], _AXES[v] * h[v], facing,
                               tess[u], tess[v]))
    return faces


def _look_camera(pos, target, width, height, vfov_deg=90.0) -> Camera:
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(pos.astype(np.float32), fwd.astype(np.float32),
                  right.astype(np.float32), up.astype(np.float32),
                  float(math.tan(math.radians(vfov_deg) / 2)), width, height)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def tiny_room(seed: int = 1, width: int = 128, height: int = 128,
              frames: int = 16, name: str = "tiny_room") -> Scene:
    """2 m closed box [-1,1]^3: each of the 6 walls is split into 2 quads
    (12 quads, 24 triangles).  The x<0 half of the ceiling is the emitter
    (radiance 10, albedo 0); every other quad has an albedo uniform in
    [0.2, 0.8]^3.  The camera sits at the room centre looking down -z with a
    90 degree vertical field of view; the probe grid is 4x4x4."""
    rng = np.random.default_rng(seed)
    tris, alb, emi = [], [], []
    c = np.zeros(3)
    for ax in range(3):
        u, v = [k for k in range(3) if k != ax]
        for sgn in (-1.0, 1.0):
            facing = -_AXES[ax] * sgn          # into the room
            for half in (-1.0, 1.0):           # split along axis u
                qc = c.copy()
                qc[ax] = sgn
                qc[u] = 0.5 * half
                q = _quad(qc, _AXES[u] * 0.5, _AXES[v] * 1.0, facing)
                is_emitter = (ax == 1 and sgn > 0 and u == 0 and half < 0)
                a = np.zeros(3) if is_emitter else rng.uniform(0.2, 0.8, 3)
                e = np.full(3, 10.0) if is_emitter else np.zeros(3)
                for t in q:
                    tris.append(t)
                    alb.append(a)
                    emi.append(e)
    verts = np.asarray(tris, np.float32)
    grid = ProbeGrid(np.full(3, -0.75, np.float32), np.full(3, 0.5, np.float32),
                     np.array([4, 4, 4], np.int32))
    cams = [_look_camera([0, 0, 0], [0, 0, -1], width, height) for _ in range(frames)]
    st = Settings(rays_per_probe=64, spatial_passes=1, seed=seed)
    return Scene(name, verts, np.asarray(alb, np.float32), np.asarray(emi, np.float32),
                 grid, cams, st)


def _tri_normals(verts):
    n = np.cross(verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0]).astype(np.float64)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def tiny_room_glossy(seed: int = 1, width: int = 128, height: int = 128, frames: int = 16) -> Scene:
    """The tiny room with microfacet materials: a near-mirror floor (GGX
    roughness 0.05, k_s 0.5, albedo halved) and a rough glossy back wall
    (roughness 0.3, k_s 0.25, albedo x 0.75), the rest Lambertian."""
    sc = tiny_room(seed, width, height, frames, name="tiny_room_glossy")
    n = _tri_normals(sc.verts)
    c = sc.verts.mean(axis=1)
    floor = (n[:, 1] > 0.99) & (c[:, 1] < -0.99)
    back = (n[:, 2] > 0.99) & (c[:, 2] < -0.99)
    gl = np.zeros((sc.num_tris, 4), np.float32)
    alb = sc.albedo.copy()
    gl[floor] = (0.5, 0.5, 0.5, 0.05)
    alb[floor] *= 0.5
    gl[back] = (0.25, 0.25, 0.25, 0.3)
    alb[back] *= 0.75
    return dataclasses.replace(sc, albedo=alb, glossy=gl)


def apartment_glossy(seed: int = 7, width: int = 1920, height: int = 1080, frames: int = 16) -> Scene:
    """The apartment with microfacet materials: a polished floor (GGX
    roughness 0.15, k_s 0.35, albedo x 0.6) and glossy tops on the furniture
    and the wall ends (every other upward-facing surface below the ceiling:
    roughness 0.3, k_s 0.3, albedo x 0.7)."""
    sc = apartment(seed, width, height, frames)
    n = _tri_normals(sc.verts)
    c = sc.verts.mean(axis=1)
    up = n[:, 1] > 0.99
    floor = up & (c[:, 1] < 0.01)
    tops = up & ~floor & (c[:, 1] < 2.95) & (sc.emission.max(axis=1) == 0)
    gl = np.zeros((sc.num_tris, 4), np.float32)
    alb = sc.albedo.copy()
    gl[floor] = (0.35, 0.35, 0.35, 0.15)
    alb[floor] *= 0.6
    gl[tops] = (0.3, 0.3, 0.3, 0.3)
    alb[tops] *= 0.7
    return dataclasses.replace(sc, name="apartment_glossy", albedo=alb, glossy=gl)


def tiny_room_1080p(seed: int = 1, frames: int = 32, learned: bool = True) -> Scene:
    """The tiny room rendered at 1920x1080 with the learned target: 65,536
    self-training samples per frame, Adam lr 1e-3."""
    sc = tiny_room(seed, 1920, 1080, frames, name="tiny_room_1080p")
    sc.settings = dataclasses.replace(sc.settings, learned_target=int(learned), train_samples=65536)
    return sc


def apartment(seed: int = 7, width: int = 1920, height: int = 1080,
              frames: int = 16, target_tris: int = 65536) -> Scene:
    """Procedural 4-room apartment, 16 m x 12 m x 3 m.

    * shell: floor, ceiling and 4 outer walls facing into the apartment,
      tessellated so that the whole scene has about ``target_tris`` triangles;
    * two interior walls (0.2 m thick solids) at x = 8 and z = 6, each with two
      door openings 1 m wide and 2.1 m high;
    * 400 furniture boxes (solids) with random sizes and positions, kept out
      of the camera corridor;
    * 512 ceiling light panels (0.3 m x 0.3 m, 2 cm below the ceiling, facing
      down): 1024 emissive triangles whose radiance is log-uniform in
      [1, 100], albedo 0;
    * camera starting in the first room at (2, 1.6, 3) looking along +x and
      slightly toward +z, translating 5 cm per frame along +x;
    * 16x8x16 probes spanning the apartment.
    """
    rng = np.random.default_rng(seed)
    tris, alb, emi = [], [], []

    def add(tri_list, a, e=(0.0, 0.0, 0.0)):
        for t in tri_list:
            tris.append(t)
            alb.append(np.asarray(a, np.float64))
            emi.append(np.asarray(e, np.float64))

    X, Y, Z = 16.0, 3.0, 12.0
    # interior walls with door gaps: list of solid boxes (lo, hi)
    walls = []
    t = 0.1
    # wall at x = 8 along z, doors at z in [2.5,3.5] and [8.5,9.5]
    for z0, z1 in ((0.0, 2.5), (3.5, 8.5), (9.5, Z)):
        walls.append(((8 - t, 0, z0), (8 + t, Y, z1)))
    for z0, z1 in ((2.5, 3.5), (8.5, 9.5)):
        walls.append(((8 - t, 2.1, z0), (8 + t, Y, z1)))
    # wall at z = 6 along x, doors at x in [3.5,4.5] and [11.5,12.5]
    for x0, x1 in ((0.0, 3.5), (4.5, 8 - t), (8 + t, 11.5), (12.5, X)):
        walls.append(((x0, 0, 6 - t), (x1, Y, 6 + t)))
    for x0, x1 in ((3.5, 4.5), (11.5, 12.5)):
        walls.append(((x0, 2.1, 6 - t), (x1, Y, 6 + t)))
    for lo, hi in walls:
        a = rng.uniform(0.5, 0.8, 3)
        for f in _box_faces(lo, hi):
            add(f, a)

    # furniture: 400 boxes away from the camera corridor (z in [2.2, 3.8])
    nbox = 0
    while nbox < 400:
        sx, sz = rng.uniform(0.3, 1.5, 2)
        sy = rng.uniform(0.3, 2.0)
        cx = rng.uniform(0.3 + sx / 2, X - 0.3 - sx / 2)
        cz = rng.uniform(0.3 + sz / 2, Z - 0.3 - sz / 2)
        if cz + sz / 2 > 2.2 and cz - sz / 2 < 3.8:
            continue
        lo = (cx - sx / 2, 0.0, cz - sz / 2)
        hi = (cx + sx / 2, sy, cz + sz / 2)
        a = rng.uniform(0.2, 0.8, 3)
        for f in _box_faces(lo, hi):
            add(f, a)
        nbox += 1

    # ceiling lights: 32 x 16 panels
    for i in range(32):
        for j in range(16):
            cx = (i + 0.5) * X / 32
            cz = (j + 0.5) * Z / 16
            q = _quad((cx, Y - 0.02, cz), (0.15, 0, 0), (0, 0, 0.15), (0, -1, 0))
            for tri in q:
                le = math.exp(rng.uniform(math.log(1.0), math.log(100.0)))
                add([tri], (0, 0, 0), (le, le, le))

    # shell: tessellate to reach target_tris
    remaining = max(target_tris - len(tris), 12)
    # area-proportional split; faces: floor/ceiling (X*Z each), walls 2*(X*Y) + 2*(Z*Y)
    total_area = 2 * X * Z + 2 * X * Y + 2 * Z * Y
    cell = math.sqrt(total_area * 2 / remaining)
    nx, ny, nz = max(1, int(X / cell)), max(1, int(Y / cell)), max(1, int(Z / cell))
    shell_alb = [rng.uniform(0.3, 0.8, 3) for _ in range(6)]
    for k, f in enumerate(_box_faces((0, 0, 0), (X, Y, Z), inward=True, tess=(nx, ny, nz))):
        add(f, shell_alb[k])

    verts = np.asarray(tris, np.float32)
    counts = np.array([16, 8, 16], np.int32)
    spacing = np.array([X / 16, Y / 8, Z / 16], np.float32)
    grid = ProbeGrid((spacing * 0.5).astype(np.float32), spacing, counts)
    cams = []
    for f in range(frames):
        p = np.array([2.0 + 0.05 * f, 1.6, 3.0])
        cams.append(_look_camera(p, p + np.array([1.0, -0.15, 0.35]), width, height))
    st = Settings(rays_per_probe=256, spatial_passes=2, seed=seed)
    return Scene("apartment", verts, np.asarray(alb, np.float32),
                 np.asarray(emi, np.float32), grid, cams, st)


def _moving_boxes(rng, n, lo, hi, size, keep_out=None):
    """n random solid boxes inside [lo, hi] (a box's triangles, its centre)
    with sinusoidal motion parameters."""
    tris, centers = [], []
    while len(centers) < n:
        s = rng.uniform(size[0], size[1], 3)
        c = np.array([rng.uniform(lo[a] + s[a] / 2, hi[a] - s[a] / 2) for a in range(3)])
        if keep_out is not None and keep_out(c, s):
            continue
        tris.append([t for f in _box_faces(c - s / 2, c + s / 2) for t in f])
        centers.append(c)
    ang = rng.uniform(0, 2 * np.pi, n)
    axis = np.stack([np.cos(ang), np.zeros(n), np.sin(ang)], 1)
    motion = Motion(np.asarray(centers), axis, rng.uniform(0.2, 0.6, n), rng.uniform(0.1, 0.5, n),
                    rng.uniform(32, 128, n), rng.uniform(0, 2 * np.pi, n))
    return tris, motion


def _with_instances(sc: Scene, box_tris, motion, rng, toggle, name) -> Scene:
    """Scene plus moving boxes (instances 0..n-1, appended after the static
    triangles) and emitter toggling."""
    extra = [t for b in box_tris for t in b]
    inst = np.concatenate([np.full(sc.num_tris, -1, np.int32),
                           np.repeat(np.arange(len(box_tris), dtype=np.int32), [len(b) for b in box_tris])])
    alb = np.repeat(rng.uniform(0.2, 0.8, (len(box_tris), 3)), [len(b) for b in box_tris], axis=0)
    return Scene(name, np.concatenate([sc.verts, np.asarray(extra, np.float32)]),
                 np.concatenate([sc.albedo, alb.astype(np.float32)]),
                 np.concatenate([sc.emission, np.zeros((len(extra), 3), np.float32)]),
                 sc.grid, sc.cameras, dataclasses.replace(sc.settings, probe_relocation=1),
                 inst, motion, toggle)


def apartment_dynamic(seed: int = 7, width: int = 1920, height: int = 1080, frames: int = 64,
                      moving_boxes: int = 200) -> Scene:
    """The apartment plus 200 boxes (0.2 to 0.6 m, anywhere in the volume
    outside the camera corridor) moving sinusoidally (shift 0.2 to 0.6 m,
    turn 0.1 to 0.5 rad, periods 32 to 128 frames); the two halves of the
    1024 emitters swap on and off every 8 frames; probe relocation on."""
    sc = apartment(seed, width, height, frames)
    rng = np.random.default_rng([seed, 0x6D6F74])      # the "motion" stream
    boxes, motion = _moving_boxes(rng, moving_boxes, (0.3, 0.1, 0.3), (15.7, 2.8, 11.7), (0.2, 0.6),
                                  keep_out=lambda c, s: c[2] + s[2] / 2 > 2.2 and c[2] - s[2] / 2 < 3.8)
    return _with_instances(sc, boxes, motion, rng, 8, "apartment_dynamic")


def tiny_room_dynamic(seed: int = 1, width: int = 64, height: int = 48, frames: int = 8) -> Scene:
    """The box with 3 floating boxes in motion and its two emitter triangles
    swapping every 2 frames (a small full-image case of the dynamics)."""
    sc = tiny_room(seed, width, height, frames)
    rng = np.random.default_rng([seed, 0x6D6F74])
    boxes, motion = _moving_boxes(rng, 3, (-0.9, -0.9, -0.9), (0.9, 0.6, 0.9), (0.15, 0.4),
                                  keep_out=lambda c, s: np.linalg.norm(c[[0, 2]]) < 0.35)
    motion.period[:] = rng.uniform(4, 8, 3)
    return _with_instances(sc, boxes, motion, rng, 2, "tiny_room_dynamic")


def multistorey(seed: int = 11, width: int = 3840, height: int = 2160, frames: int = 128,
                target_tris: int = 1_000_000, moving_boxes: int = 500) -> Scene:
    """Large workload: a 4-storey building, 16 m x 12 m x 12 m.

    * every storey (3 m) has the apartment's two interior walls with doors,
      200 furniture boxes and 32 x 32 ceiling panels (2048 emissive triangles,
      8192 in the building, radiance log-uniform in [1, 100], albedo 0);
      floors are 0.2 m slabs;
    * the storeys' shells are tessellated so that the building has about
      ``target_tris`` triangles;
    * 500 boxes in sinusoidal rigid motion spread over the storeys (the
      dynamic apartment's motion model), emitter halves swapping every 8
      frames, probe relocation on;
    * camera on the second storey at (2, 4.6, 3), translating 5 cm per frame
      along +x; 3840 x 2160;
    * 32 x 16 x 32 probes, 256 rays; 63 emitter + 1 BSDF candidates, temporal
      + 3 spatial passes; learned target in bf16 with 65,536 samples per
      frame.
    """
    rng = np.random.default_rng(seed)
    X, S, Z, NS = 16.0, 3.0, 12.0, 4
    Y = S * NS
    blocks, albs, emis = [], [], []

    def add(tris, a, e=(0.0, 0.0, 0.0)):
        t = np.asarray(tris, np.float64).reshape(-1, 3, 3)
        blocks.append(t)
        albs.append(np.broadcast_to(np.asarray(a, np.float64), (len(t), 3)))
        emis.append(np.broadcast_to(np.asarray(e, np.float64), (len(t), 3)))

    t = 0.1
    for st in range(NS):
        y0 = S * st
        walls = []
        for z0, z1 in ((0.0, 2.5), (3.5, 8.5), (9.5, Z)):
            walls.append(((8 - t, y0, z0), (8 + t, y0 + S, z1)))
        for z0, z1 in ((2.5, 3.5), (8.5, 9.5)):
            walls.append(((8 - t, y0 + 2.1, z0), (8 + t, y0 + S, z1)))
        for x0, x1 in ((0.0, 3.5), (4.5, 8 - t), (8 + t, 11.5), (12.5, X)):
            walls.append(((x0, y0, 6 - t), (x1, y0 + S, 6 + t)))
        for x0, x1 in ((3.5, 4.5), (11.5, 12.5)):
            walls.append(((x0, y0 + 2.1, 6 - t), (x1, y0 + S, 6 + t)))
        if st > 0:
            walls.append(((0.0, y0 - 0.1, 0.0), (X, y0 + 0.1, Z)))   # floor slab
        for lo, hi in walls:
            a = rng.uniform(0.5, 0.8, 3)
            for f in _box_faces(lo, hi):
                add(f, a)
        nbox = 0
        while nbox < 200:
            sx, sz = rng.uniform(0.3, 1.5, 2)
            sy = rng.uniform(0.3, 2.0)
            cx = rng.uniform(0.3 + sx / 2, X - 0.3 - sx / 2)
            cz = rng.uniform(0.3 + sz / 2, Z - 0.3 - sz / 2)
            if cz + sz / 2 > 2.2 and cz - sz / 2 < 3.8:
                continue
            a = rng.uniform(0.2, 0.8, 3)
            for f in _box_faces((cx - sx / 2, y0 + 0.1, cz - sz / 2), (cx + sx / 2, y0 + 0.1 + sy, cz + sz / 2)):
                add(f, a)
            nbox += 1
        for i in range(32):
            for j in range(32):
                q = _quad(((i + 0.5) * X / 32, y0 + S - 0.12, (j + 0.5) * Z / 32), (0.12, 0, 0), (0, 0, 0.09),
                          (0, -1, 0))
                for tri in q:
                    le = math.exp(rng.uniform(math.log(1.0), math.log(100.0)))
                    add([tri], (0, 0, 0), (le, le, le))
    # storey shells, tessellated to reach target_tris
    n_now = sum(len(b) for b in blocks)
    remaining = max(target_tris - n_now - 12 * moving_boxes, 12 * NS)
    area = NS * (2 * X * Z + 2 * X * S + 2 * Z * S)
    cell = math.sqrt(area * 2 / remaining)
    nx, ny, nz = max(1, int(X / cell)), max(1, int(S / cell)), max(1, int(Z / cell))
    for st in range(NS):
        shell_alb = [rng.uniform(0.3, 0.8, 3) for _ in range(6)]
        for k, f in enumerate(_box_faces((0, S * st, 0), (X, S * st + S, Z), inward=True, tess=(nx, ny, nz))):
            add(f, shell_alb[k])
    verts = np.concatenate(blocks).astype(np.float32)
    counts = np.array([32, 16, 32], np.int32)
    spacing = np.array([X / 32, Y / 16, Z / 32], np.float32)
    grid = ProbeGrid((spacing * 0.5).astype(np.float32), spacing, counts)
    cams = []
    for f in range(frames):
        pos = np.array([2.0 + 0.05 * f, S + 1.6, 3.0])
        cams.append(_look_camera(pos, pos + np.array([1.0, -0.15, 0.35]), width, height))
    st = Settings(rays_per_probe=256, spatial_passes=3, num_light_candidates=63, seed=seed,
                  learned_target=1, train_samples=65536, mlp_bf16=1)
    sc = Scene("multistorey", verts, np.concatenate(albs).astype(np.float32),
               np.concatenate(emis).astype(np.float32), grid, cams, st)
    mrng = np.random.default_rng([seed, 0x6D6F74])
    boxes, motion = _moving_boxes(mrng, moving_boxes, (0.3, 0.2, 0.3), (15.7, Y - 0.2, 11.7), (0.2, 0.6),
                                  keep_out=lambda c, s: (c[2] + s[2] / 2 > 2.2 and c[2] - s[2] / 2 < 3.8
                                                         and S < c[1] < 2 * S))
    return _with_instances(sc, boxes, motion, mrng, 8, "multistorey")


def secondary_ddgi(settings: Settings) -> Settings:
    """The paper's "secondary DDGI" comparison (Sec. 4): one cosine BSDF ray
    per pixel terminated in the probe volume, no emitter candidates, no
    temporal or spatial reuse (the same passes with M = 1 and reuse off)."""
    return dataclasses.replace(settings, num_light_candidates=0, num_bsdf_candidates=1, spatial_passes=0,
                               temporal_mcap=0.0)


def make_scene(name: str, **kw) -> Scene:
    return {"tiny_room": tiny_room, "tiny_room_1080p": tiny_room_1080p,
            "apartment": apartment, "apartment_dynamic": apartment_dynamic,
            "tiny_room_dynamic": tiny_room_dynamic, "multistorey": multistorey}[name](**kw)


# ---------------------------------------------------------------------------
# synthetic per-pixel buffers for pass-isolated tests
# ---------------------------------------------------------------------------

def _random_surface_points(scene: Scene, n: int, rng, emissive_frac=0.02):
    """Random triangles and uniform barycentric coordinates (b1, b2)."""
    emissive = np.flatnonzero(scene.emission.max(axis=1) > 0)
    plain = np.flatnonzero(scene.emission.max(axis=1) <= 0)
    use_e = rng.random(n) < emissive_frac if len(emissive) else np.zeros(n, bool)
    tri = np.where(use_e, rng.choice(emissive, n) if len(emissive) else 0,
                   rng.choice(plain, n)).astype(np.int64)
    b1 = rng.random(n)
    b2 = rng.random(n)
    flip = b1 + b2 > 1
    b1[flip], b2[flip] = 1 - b1[flip], 1 - b2[flip]
    v = scene.verts[tri].astype(np.float64)
    # keep points strictly inside the triangle
    b1 = 0.02 + 0.96 * b1
    b2 = 0.02 + 0.96 * b2
    s = b1 + b2
    over = s > 0.98
    b1[over] *= 0.98 / s[over]
    b2[over] *= 0.98 / s[over]
    p = v[:, 0] + b1[:, None] * (v[:, 1] - v[:, 0]) + b2[:, None] * (v[:, 2] - v[:, 0])
    return tri, p


def synthetic_gbuffer(scene: Scene, width: int, height: int, seed: int,
                      invalid_frac: float = 0.03, motion_frac: float = 0.9):
    """Random G-buffer planes shaped like the primary-visibility output.

    Every valid pixel holds a point on a random triangle, that triangle's
    facing normal (the winding normal, passed in as data) and albedo, a
    camera distance uniform in [0.5, 10] and a previous-frame pixel a few
    pixels away (or -1).  Returns three float32 arrays of shape [H*W, 4]
    (pos+dist, normal+tri bits, albedo+prev-pixel bits)."""
    rng = np.random.default_rng(seed)
    n = width * height
    tri, p = _random_surface_points(scene, n, rng)
    v = scene.verts[tri].astype(np.float64)
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    g0 = np.zeros((n, 4), np.float32)
    g1 = np.zeros((n, 4), np.float32)
    g2 = np.zeros((n, 4), np.float32)
    g0[:, :3] = p
    g0[:, 3] = rng.uniform(0.5, 10.0, n)
    g1[:, :3] = nrm
    tri_u = tri.astype(np.uint32)
    invalid = rng.random(n) < invalid_frac
    tri_u[invalid] = 0xFFFFFFFF
    g1[:, 3] = tri_u.view(np.float32)
    g2[:, :3] = scene.albedo[tri]
    px = np.arange(n) % width
    py = np.arange(n) // width
    qx = px + rng.integers(-2, 3, n)
    qy = py + rng.integers(-2, 3, n)
    ok = (qx >= 0) & (qx < width) & (qy >= 0) & (qy < height) & (rng.random(n) < motion_frac)
    prev = np.where(ok, qy * width + qx, -1).astype(np.int32)
    g2[:, 3] = prev.view(np.float32)
    return g0, g1, g2


def synthetic_reservoirs(scene: Scene, n: int, seed: int, empty_frac: float = 0.05):
    """Random reservoirs: a point y on a random triangle, W log-normal, M in
    [1, 40], a cached radiance uniform in [0, 5]^3 and a random tag.  Returns
    (r0 float32[n,4] = y.xyz,W; r1 float32[n,4] = L.rgb,M; r2 uint32[n,2] =
    y-triangle, tag)."""
    rng = np.random.default_rng(seed)
    tri, p = _random_surface_points(scene, n, rng, emissive_frac=0.3)
    r0 = np.zeros((n, 4), np.float32)
    r1 = np.zeros((n, 4), np.float32)
    r2 = np.zeros((n, 2), np.uint32)
    r0[:, :3] = p
    r0[:, 3] = np.exp(rng.normal(0.0, 1.0, n))
    r1[:, :3] = rng.uniform(0.0, 5.0, (n, 3))
    r1[:, 3] = rng.integers(1, 41, n)
    r2[:, 0] = tri
    r2[:, 1] = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    empty = rng.random(n) < empty_frac
    r0[empty] = 0
    r1[empty] = 0
    r2[empty, 0] = 0xFFFFFFFF
    r2[empty, 1] = 0
    return r0, r1, r2


def synthetic_irradiance_interior(grid: ProbeGrid, n: int, seed: int):
    """Random positive irradiance for the n x n interior texels of every probe:
    float32[P, n, n, 3] (row-major: [probe, row, column, rgb])."""
    rng = np.random.default_rng(seed)
    P = grid.num_probes
    base = rng.uniform(0.2, 3.0, (P, 1, 1, 3))
    var = rng.uniform(0.5, 1.5, (P, n, n, 3))
    return (base * var).astype(np.float32)


def synthetic_depth_interior(grid: ProbeGrid, n: int, seed: int):
    """Random mean / mean-square distances for the n x n interior depth texels
    of every probe: float32[P, n, n, 2] with mean in [0.05, 1.5] x max spacing
    and a non-negative variance."""
    rng = np.random.default_rng(seed)
    P = grid.num_probes
    s = float(np.max(grid.spacing))
    mu = rng.uniform(0.05, 1.5, (P, n, n)) * s
    var = rng.uniform(0.0, 0.1, (P, n, n)) * s * s
    return np.stack([mu, mu * mu + var], axis=-1).astype(np.float32)
