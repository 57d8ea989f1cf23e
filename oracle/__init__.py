"""CPU oracle for DDGI resampling -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It wraps ``ddgi_oracle.c`` (plain C99, fp64,
brute-force intersection, single thread) with ctypes and numpy marshalling,
and adds the error metrics of Sec. 4 (MAPE with epsilon 0.01, and MSE).

The C library is compiled on first use with the system C compiler
(``build()``); nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddgi_oracle.c")
_HDR = os.path.join(_HERE, "ddgi_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PASS_INITIAL = 0
PASS_SPATIAL0 = 1
PASS_TEMPORAL = 5
PASS_PROBE_ROT = 7


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (strict IEEE: no contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


# ---------------------------------------------------------------------------
# ctypes structures (mirror ddgi_oracle.h)
# ---------------------------------------------------------------------------
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint32)
_fp = C.POINTER(C.c_float)


class _Scene(C.Structure):
    _fields_ = [("num_tris", C.c_int32), ("verts", _dp), ("albedo", _dp), ("emission", _dp),
                ("tri_instance", _ip), ("num_instances", C.c_int32), ("object_verts", _dp),
                ("normal", _dp), ("area", _dp), ("num_emitters", C.c_int32),
                ("emitter_tri", _ip), ("emitter_of", _ip), ("emitter_cdf", _fp), ("area_total", C.c_double),
                ("inst_cur", _dp), ("inst_prev", _dp), ("glossy", _dp)]


class _Settings(C.Structure):
    _fields_ = [("rays_per_probe", C.c_int32), ("irr_n", C.c_int32), ("depth_n", C.c_int32),
                ("hysteresis", C.c_double), ("le_attenuation", C.c_double),
                ("depth_sharpness", C.c_double), ("n_light", C.c_int32), ("n_bsdf", C.c_int32),
                ("temporal_mcap", C.c_double), ("spatial_neighbours", C.c_int32),
                ("spatial_radius", C.c_int32), ("normal_reject_cos", C.c_double),
                ("depth_reject_frac", C.c_double), ("seed", C.c_uint32), ("relocate", C.c_int32),
                ("candidate_stride", C.c_int32), ("footprint_c", C.c_double)]


class _Volume(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("spacing", C.c_double * 3), ("counts", C.c_int32 * 3),
                ("irr_n", C.c_int32), ("depth_n", C.c_int32), ("irr", _dp), ("depth", _dp),
                ("offset", _dp), ("updates", C.c_int32), ("mlp", _dp), ("mlp_lo", C.c_double * 3),
                ("mlp_scale", C.c_double), ("use_mlp", C.c_int32)]


class _Camera(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("fwd", C.c_double * 3), ("right", C.c_double * 3),
                ("up", C.c_double * 3), ("tan_half_fovy", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32)]


class _GBuf(C.Structure):
    _fields_ = [("pos", _dp), ("dist", _dp), ("nrm", _dp), ("alb", _dp), ("tri", _ip),
                ("prev", _ip), ("width", C.c_int32), ("height", C.c_int32), ("eye", C.c_double * 3)]


class _Res(C.Structure):
    _fields_ = [("y", _dp), ("W", _dp), ("L", _dp), ("M", _dp), ("tri", _ip), ("tag", _up), ("ny", _dp)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.or_pcg.restype = C.c_uint32
            L.or_pcg.argtypes = [C.c_uint32]
            L.or_rng_u32.restype = C.c_uint32
            L.or_rng_u32.argtypes = [C.c_uint32] * 6
            L.or_rng.restype = C.c_double
            L.or_rng.argtypes = [C.c_uint32] * 6
            L.or_ddgi_query.restype = C.c_double
            L.or_target.restype = C.c_double
            L.or_sample_emitter.restype = C.c_int32
            L.or_sample_emitter.argtypes = [C.POINTER(_Scene), C.c_double]
            L.or_ggx_D.restype = C.c_double
            L.or_ggx_G1.restype = C.c_double
        return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def _v3(a):
    return (C.c_double * 3)(*[float(x) for x in a])


def _pixarg(pix):
    if pix is None:
        return None, None
    pix = np.ascontiguousarray(pix, np.int32)
    return pix, _p(pix, _ip)


# ---------------------------------------------------------------------------
# high-level wrappers
# ---------------------------------------------------------------------------

class Scene:
    """Oracle view of a ``scenegen.Scene`` (fp64 copies of its float32 data)."""

    def __init__(self, sc):
        self.src = sc
        self.verts = np.ascontiguousarray(sc.verts, np.float64).reshape(-1)
        self.albedo = np.ascontiguousarray(sc.albedo, np.float64).reshape(-1)
        self.emission = np.ascontiguousarray(sc.emission, np.float64).reshape(-1)
        self.s = _Scene()
        self.s.num_tris = sc.num_tris
        self.s.verts, self.s.albedo, self.s.emission = _p(self.verts), _p(self.albedo), _p(self.emission)
        inst = getattr(sc, "tri_instance", None)
        if inst is not None:
            self.tri_instance = np.ascontiguousarray(inst, np.int32)
            self.object_verts = self.verts.copy()
            self.s.tri_instance = _p(self.tri_instance, _ip)
            self.s.num_instances = int(self.tri_instance.max(initial=-1)) + 1
            self.s.object_verts = _p(self.object_verts)
        gl = getattr(sc, "glossy", None)
        if gl is not None:
            self.glossy = np.ascontiguousarray(gl, np.float64).reshape(-1)
            self.s.glossy = _p(self.glossy)
        if lib().or_scene_init(C.byref(self.s)) != 0:
            raise MemoryError("or_scene_init")
        self.settings = settings_of(sc.settings)

    def update(self, xf=None, emitter_radiance=None):
        """Move the instances to the poses xf ([I][12] row-major 3x4, relative
        to the identity pose) and / or set the emitters' radiance ([E][3])."""
        a = None if xf is None else np.ascontiguousarray(xf, np.float64).reshape(-1, 12)
        b = None if emitter_radiance is None else np.ascontiguousarray(emitter_radiance, np.float64)
        n = 0 if a is None else a.shape[0]
        rc = lib().or_scene_update(C.byref(self.s), None if a is None else _p(a), C.c_int32(n),
                                   None if b is None else _p(b))
        if rc != 0:
            raise ValueError("or_scene_update: transform count differs from the instance count")

    def __del__(self):
        try:
            lib().or_scene_free(C.byref(self.s))
        except Exception:
            pass

    @property
    def normals(self):
        return np.ctypeslib.as_array(self.s.normal, (self.s.num_tris, 3)).copy()

    @property
    def area_total(self):
        return self.s.area_total

    def area(self):
        return np.ctypeslib.as_array(self.s.area, (self.s.num_tris,)).copy()


def _settings(scene, settings):
    """The scene's settings, or the given ones (ctypes struct or scenegen Settings)."""
    if settings is None:
        return scene.settings
    return settings if isinstance(settings, _Settings) else settings_of(settings)


def settings_of(st) -> _Settings:
    o = _Settings()
    o.rays_per_probe = st.rays_per_probe
    o.irr_n = st.irr_texels
    o.depth_n = st.depth_texels
    o.hysteresis = st.hysteresis
    o.le_attenuation = st.le_attenuation
    o.depth_sharpness = st.depth_sharpness
    o.n_light = st.num_light_candidates
    o.n_bsdf = st.num_bsdf_candidates
    o.temporal_mcap = st.temporal_mcap
    o.spatial_neighbours = st.spatial_neighbours
    o.spatial_radius = st.spatial_radius
    o.normal_reject_cos = st.normal_reject_cos
    o.depth_reject_frac = st.depth_reject_frac
    o.seed = st.seed
    o.relocate = int(getattr(st, "probe_relocation", 0))
    o.candidate_stride = int(getattr(st, "candidate_stride", 1))
    o.footprint_c = float(getattr(st, "footprint_c", 0.2))
    return o


class Volume:
    """Probe volume state: padded irradiance / depth tiles and offsets (fp64)."""

    def __init__(self, grid, irr_n=8, depth_n=16):
        P = int(np.prod(grid.counts))
        self.P, self.irr_n, self.depth_n = P, irr_n, depth_n
        self.irr = np.zeros((P, irr_n + 2, irr_n + 2, 3))
        self.depth = np.zeros((P, depth_n + 2, depth_n + 2, 2))
        self.offset = np.zeros((P, 3))
        self.v = _Volume()
        self.v.origin = _v3(grid.origin)
        self.v.spacing = _v3(grid.spacing)
        self.v.counts = (C.c_int32 * 3)(*[int(c) for c in grid.counts])
        self.v.irr_n, self.v.depth_n = irr_n, depth_n
        self.v.updates = 0
        self._bind()

    def _bind(self):
        self.v.irr, self.v.depth, self.v.offset = _p(self.irr), _p(self.depth), _p(self.offset)

    @property
    def updates(self):
        return self.v.updates

    @updates.setter
    def updates(self, n):
        self.v.updates = n

    def set_mlp(self, flat_params, lo, scale, use=True):
        """Serve (Le + L_DDGI+) from the network (library parameter layout)."""
        self._mlp = np.ascontiguousarray(flat_params, np.float64)
        self.v.mlp = _p(self._mlp)
        self.v.mlp_lo = _v3(lo)
        self.v.mlp_scale = float(scale)
        self.v.use_mlp = 1 if use else 0

    def set_interior(self, irr_int, depth_int):
        """Fill the interior texels and rebuild the borders."""
        n, m = self.irr_n, self.depth_n
        self.irr[:, 1:n + 1, 1:n + 1, :] = irr_int
        self.depth[:, 1:m + 1, 1:m + 1, :] = depth_int
        lib().or_fill_gutters(C.byref(self.v))

    def copy(self):
        o = Volume.__new__(Volume)
        o.P, o.irr_n, o.depth_n = self.P, self.irr_n, self.depth_n
        o.irr, o.depth, o.offset = self.irr.copy(), self.depth.copy(), self.offset.copy()
        o.v = _Volume()
        C.pointer(o.v)[0] = self.v
        o._bind()
        if getattr(self, "_mlp", None) is not None:
            o._mlp = self._mlp
        return o


def camera(cam) -> _Camera:
    c = _Camera()
    c.pos, c.fwd, c.right, c.up = _v3(cam.pos), _v3(cam.fwd), _v3(cam.right), _v3(cam.up)
    c.tan_half_fovy = cam.tan_half_fovy
    c.width, c.height = cam.width, cam.height
    return c


class GBuffer:
    def __init__(self, n, width, height):
        self.pos = np.zeros((n, 3))
        self.dist = np.zeros(n)
        self.nrm = np.zeros((n, 3))
        self.alb = np.zeros((n, 3))
        self.tri = np.full(n, -1, np.int32)
        self.prev = np.full(n, -1, np.int32)
        self.width, self.height = width, height
        self.eye = np.zeros(3)          # camera position the G-buffer was rendered from

    def c(self) -> _GBuf:
        g = _GBuf()
        g.pos, g.dist, g.nrm, g.alb = _p(self.pos), _p(self.dist), _p(self.nrm), _p(self.alb)
        g.tri, g.prev = _p(self.tri, _ip), _p(self.prev, _ip)
        g.width, g.height = self.width, self.height
        g.eye = _v3(self.eye)
        return g

    @staticmethod
    def from_planes(g0, g1, g2, width, height, eye=None):
        """From packed float32 planes (pos+dist, normal+tri bits, albedo+prev
        bits).  The library marks a surface on a moving instance with bit 30
        of the previous-pixel word; the oracle finds that from the triangle's
        instance itself, so the flag is dropped here."""
        n = g0.shape[0]
        o = GBuffer(n, width, height)
        o.pos[:] = g0[:, :3]
        o.dist[:] = g0[:, 3]
        o.nrm[:] = g1[:, :3]
        o.alb[:] = g2[:, :3]
        o.tri[:] = np.ascontiguousarray(g1[:, 3]).view(np.int32)
        prev = np.ascontiguousarray(g2[:, 3]).view(np.int32)
        o.prev[:] = np.where(prev >= 0, prev & ~0x40000000, prev)
        if eye is not None:
            o.eye[:] = eye
        return o

    def planes(self):
        """Packed float32 planes in the CUDA library's layout."""
        n = self.tri.shape[0]
        g0 = np.zeros((n, 4), np.float32)
        g1 = np.zeros((n, 4), np.float32)
        g2 = np.zeros((n, 4), np.float32)
        g0[:, :3], g0[:, 3] = self.pos, self.dist
        g1[:, :3] = self.nrm
        g1[:, 3] = self.tri.view(np.float32)
        g2[:, :3] = self.alb
        g2[:, 3] = self.prev.view(np.float32)
        return g0, g1, g2


class Reservoirs:
    """Per-pixel reservoirs: the kept sample (point y, its triangle, its unit
    normal ny when found, cached radiance L), W, M and the origin tag."""

    FIELDS = ("y", "W", "L", "M", "tri", "tag", "ny")

    def __init__(self, n):
        self.y = np.zeros((n, 3))
        self.W = np.zeros(n)
        self.L = np.zeros((n, 3))
        self.M = np.zeros(n)
        self.tri = np.full(n, -1, np.int32)
        self.tag = np.zeros(n, np.uint32)
        self.ny = np.zeros((n, 3))

    def c(self) -> _Res:
        r = _Res()
        r.y, r.W, r.L, r.M = _p(self.y), _p(self.W), _p(self.L), _p(self.M)
        r.tri, r.tag = _p(self.tri, _ip), _p(self.tag, _up)
        r.ny = _p(self.ny)
        return r

    @staticmethod
    def from_planes(r0, r1, r2, scene=None):
        """From float32 planes (y, W | L, M | triangle, tag); the samples'
        normals are those of their triangles in `scene` (required when any
        reservoir holds a sample)."""
        n = r0.shape[0]
        o = Reservoirs(n)
        o.y[:] = r0[:, :3]
        o.W[:] = r0[:, 3]
        o.L[:] = r1[:, :3]
        o.M[:] = r1[:, 3]
        o.tri[:] = np.ascontiguousarray(r2[:, 0]).view(np.int32)
        o.tag[:] = r2[:, 1]
        has = o.tri >= 0
        if np.any(has):
            if scene is None:
                raise ValueError("Reservoirs.from_planes: the samples' normals need the scene")
            o.ny[has] = scene.normals[o.tri[has]]
        return o

    def planes(self):
        n = self.W.shape[0]
        r0 = np.zeros((n, 4), np.float32)
        r1 = np.zeros((n, 4), np.float32)
        r2 = np.zeros((n, 2), np.uint32)
        r0[:, :3], r0[:, 3] = self.y, self.W
        r1[:, :3], r1[:, 3] = self.L, self.M
        r2[:, 0] = self.tri.view(np.uint32)
        r2[:, 1] = self.tag
        return r0, r1, r2


# --- thin functional wrappers --------------------------------------------------

def rng(seed, pixel, frame, pas, cand, dim) -> float:
    return lib().or_rng(seed, pixel, frame, pas, cand, dim)


def rng_u32(seed, pixel, frame, pas, cand, dim) -> int:
    return lib().or_rng_u32(seed, pixel, frame, pas, cand, dim)


def pcg(v: int) -> int:
    return lib().or_pcg(v)


def intersect(scene: Scene, o, d, tmin=1e-4, tmax=1e30):
    o = np.ascontiguousarray(o, np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
    n = o.shape[0]
    tri = np.zeros(n, np.int32)
    t = np.zeros(n)
    lib().or_trace_batch(C.byref(scene.s), C.c_int32(n), _p(o), _p(d), C.c_double(tmin),
                         C.c_double(tmax), _p(tri, _ip), _p(t))
    return tri, t


def prev_position(scene: Scene, tri: int, x):
    """Position of point x on triangle tri one scene update earlier."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros(3)
    lib().or_prev_position(C.byref(scene.s), C.c_int32(tri), _p(x), _p(out))
    return out


def sample_emitter(scene: Scene, u: float) -> int:
    return lib().or_sample_emitter(C.byref(scene.s), C.c_double(u))


def oct_encode(d):
    uv = np.zeros(2)
    lib().or_oct_encode(_p(np.ascontiguousarray(d, np.float64)), _p(uv))
    return uv


def oct_decode(uv):
    d = np.zeros(3)
    lib().or_oct_decode(_p(np.ascontiguousarray(uv, np.float64)), _p(d))
    return d


def texel_dir(i, j, n):
    d = np.zeros(3)
    lib().or_texel_dir(C.c_int32(i), C.c_int32(j), C.c_int32(n), _p(d))
    return d


def sf_dir(i, n):
    d = np.zeros(3)
    lib().or_sf_dir(C.c_int32(i), C.c_int32(n), _p(d))
    return d


def probe_rotation(seed, frame):
    R = np.zeros(9)
    lib().or_probe_rotation(C.c_uint32(seed), C.c_uint32(frame), _p(R))
    return R.reshape(3, 3)


def probe_ray_dirs(seed, frame, n):
    R = probe_rotation(seed, frame).reshape(-1).copy()
    out = np.zeros((n, 3))
    for r in range(n):
        lib().or_probe_ray_dir(_p(R), C.c_int32(r), C.c_int32(n), _p(out[r]))
    return out


def onb_local_to_world(n, l):
    w = np.zeros(3)
    lib().or_onb_local_to_world(_p(np.ascontiguousarray(n, np.float64)),
                                _p(np.ascontiguousarray(l, np.float64)), _p(w))
    return w


def gutter(tile, n):
    t = np.ascontiguousarray(tile, np.float64).copy()
    lib().or_gutter(_p(t), C.c_int32(n), C.c_int32(t.shape[-1]))
    return t


def bilinear(tile, n, d):
    t = np.ascontiguousarray(tile, np.float64)
    out = np.zeros(t.shape[-1])
    lib().or_bilinear(_p(t), C.c_int32(n), C.c_int32(t.shape[-1]),
                      _p(np.ascontiguousarray(d, np.float64)), _p(out))
    return out


def ddgi_query(vol: Volume, q, n):
    E = np.zeros(3)
    sw = lib().or_ddgi_query(C.byref(vol.v), _p(np.ascontiguousarray(q, np.float64)),
                             _p(np.ascontiguousarray(n, np.float64)), _p(E))
    return E, sw


def biased_query(vol: Volume, y, n, frm):
    """Irradiance E at y (normal n) with the view-path bias of Sec. 3.4: the
    query point moves from y toward the previous path vertex ``frm``."""
    E = np.zeros(3)
    a = [np.ascontiguousarray(v, np.float64) for v in (y, n, frm)]
    lib().or_biased_query(C.byref(vol.v), _p(a[0]), _p(a[1]), _p(a[2]), _p(E))
    return E


def probe_trace(scene: Scene, vol: Volume, frame: int, probes=None, settings=None):
    st = _settings(scene, settings)
    pr, pp = _pixarg(probes)
    n = vol.P if probes is None else len(pr)
    rays = np.zeros((n, st.rays_per_probe, 4))
    lib().or_probe_trace(C.byref(scene.s), C.byref(vol.v), C.byref(st), C.c_uint32(frame),
                         pp, C.c_int32(n), _p(rays))
    return rays


def probe_blend(vol: Volume, rays, frame: int, settings, probes=None):
    pr, pp = _pixarg(probes)
    n = vol.P if probes is None else len(pr)
    rays = np.ascontiguousarray(rays, np.float64)
    lib().or_probe_blend(C.byref(vol.v), C.byref(settings), C.c_uint32(frame), pp,
                         C.c_int32(n), _p(rays))


def probe_relocate(vol: Volume, rays, frame: int, settings, probes=None):
    """Probe relocation from one frame's rays (offsets updated in place)."""
    pr, pp = _pixarg(probes)
    n = vol.P if probes is None else len(pr)
    rays = np.ascontiguousarray(rays, np.float64)
    lib().or_probe_relocate(C.byref(vol.v), C.byref(settings), C.c_uint32(frame), pp,
                            C.c_int32(n), _p(rays))


def probe_update(scene: Scene, vol: Volume, frame: int, settings=None):
    st = _settings(scene, settings)
    rc = lib().or_probe_update(C.byref(scene.s), C.byref(vol.v), C.byref(st), C.c_uint32(frame))
    if rc != 0:
        raise MemoryError("or_probe_update")


def gbuffer(scene: Scene, cam, prev_cam=None, pix=None) -> GBuffer:
    pr, pp = _pixarg(pix)
    n = cam.width * cam.height if pix is None else len(pr)
    g = GBuffer(n, cam.width, cam.height)
    gc = g.c()
    c = camera(cam)
    pc = camera(prev_cam) if prev_cam is not None else None
    lib().or_gbuffer(C.byref(scene.s), C.byref(c), C.byref(pc) if pc is not None else None,
                     pp, C.c_int32(n), C.byref(gc))
    g.eye[:] = cam.pos
    return g


def restir_initial(scene: Scene, vol: Volume, g: GBuffer, frame: int, pix=None, settings=None):
    st = _settings(scene, settings)
    pr, pp = _pixarg(pix)
    n = g.tri.shape[0] if pix is None else len(pr)
    out = Reservoirs(n)
    resid = np.zeros((n, 3))
    gc, oc = g.c(), out.c()
    lib().or_restir_initial(C.byref(scene.s), C.byref(vol.v), C.byref(st), C.byref(gc),
                            C.c_uint32(frame), pp, C.c_int32(n), C.byref(oc), _p(resid))
    return out, resid


def restir_temporal(scene: Scene, g: GBuffer, gp: GBuffer, prev_cam_pos, cur: Reservoirs,
                    prev: Reservoirs, frame: int, pix=None, settings=None, requery: "Volume" = None):
    """Temporal reuse (Sec. 3.1 step 2) with the radiance cached in the
    reservoirs (Sec. 3.6), or, with ``requery`` (a test setting: caching off),
    queried afresh from that volume at the current pixel."""
    _need_full(g, cur)
    _need_full(gp, prev)
    prev_px = g.prev if pix is None else g.prev[np.asarray(pix)]
    if np.any(prev_px >= gp.tri.shape[0]):
        raise ValueError("previous-pixel indices beyond the previous G-buffer")
    st = _settings(scene, settings)
    pr, pp = _pixarg(pix)
    n = g.tri.shape[0] if pix is None else len(pr)
    out = Reservoirs(n)
    gc, gpc, cc, prc, oc = g.c(), gp.c(), cur.c(), prev.c(), out.c()
    cp = np.ascontiguousarray(prev_cam_pos, np.float64)
    rq = C.byref(requery.v) if requery is not None else None
    lib().or_restir_temporal_rq(C.byref(scene.s), C.byref(st), C.byref(gc), C.byref(gpc), _p(cp),
                                C.byref(cc), C.byref(prc), C.c_uint32(frame), pp, C.c_int32(n), rq,
                                C.byref(oc))
    return out


def restir_spatial(scene: Scene, g: GBuffer, res_in: Reservoirs, frame: int, pass_idx: int,
                   pix=None, settings=None, requery: "Volume" = None):
    """Spatial reuse pass (Sec. 3.1 step 2); ``requery`` as in restir_temporal."""
    _need_full(g, res_in)
    st = _settings(scene, settings)
    pr, pp = _pixarg(pix)
    n = g.tri.shape[0] if pix is None else len(pr)
    out = Reservoirs(n)
    gc, ic, oc = g.c(), res_in.c(), out.c()
    rq = C.byref(requery.v) if requery is not None else None
    lib().or_restir_spatial_rq(C.byref(scene.s), C.byref(st), C.byref(gc), C.byref(ic),
                               C.c_uint32(frame), C.c_uint32(pass_idx), pp, C.c_int32(n), rq,
                               C.byref(oc))
    return out


def _need_full(g: GBuffer, *bufs):
    """Inputs indexed by pixel must cover the whole image."""
    for b in bufs:
        m = b.W.shape[0] if isinstance(b, Reservoirs) else np.asarray(b).shape[0]
        if m != g.tri.shape[0]:
            raise ValueError(f"input buffer holds {m} entries, the image {g.tri.shape[0]} pixels")


def shade(scene: Scene, vol: Volume, g: GBuffer, res: Reservoirs, resid, pix=None, frame: int = 0,
          settings=None):
    """Eq. Algorithm's estimate per pixel; ``frame`` keys the random numbers
    of the specular recursion (glossy scenes only)."""
    _need_full(g, res, resid)
    st = _settings(scene, settings)
    pr, pp = _pixarg(pix)
    n = g.tri.shape[0] if pix is None else len(pr)
    rad = np.zeros((n, 3))
    gc, rc = g.c(), res.c()
    resid = np.ascontiguousarray(resid, np.float64)
    lib().or_shade(C.byref(scene.s), C.byref(vol.v), C.byref(st), C.byref(gc), C.byref(rc), _p(resid),
                   C.c_uint32(frame), pp, C.c_int32(n), _p(rad))
    return rad


def shade_radiance(scene: Scene, vol: Volume, eye, x1, n1, y, tri: int, pix: int, frame: int, settings=None):
    """Radiance at y toward x1 with the specular recursion of Sec. 3.3, and
    the number of path vertices it used (x1 counted)."""
    st = _settings(scene, settings)
    a = [np.ascontiguousarray(v, np.float64) for v in (eye, x1, n1, y)]
    L = np.zeros(3)
    verts = C.c_int32(0)
    lib().or_shade_radiance(C.byref(scene.s), C.byref(vol.v), C.byref(st), _p(a[0]), _p(a[1]), _p(a[2]),
                            _p(a[3]), C.c_int32(tri), C.c_uint32(pix), C.c_uint32(frame), _p(L), C.byref(verts))
    return L, verts.value


def ggx_D(nh, alpha) -> float:
    return lib().or_ggx_D(C.c_double(nh), C.c_double(alpha))


def ggx_G1(nw, alpha) -> float:
    return lib().or_ggx_G1(C.c_double(nw), C.c_double(alpha))


def ggx_sample_h(n, alpha, u0, u1):
    h = np.zeros(3)
    lib().or_ggx_sample_h(_p(np.ascontiguousarray(n, np.float64)), C.c_double(alpha), C.c_double(u0),
                          C.c_double(u1), _p(h))
    return h


def glossy_sample(n, wo, ks, alpha, u0, u1):
    """(wi, weight f_g cos / pdf per channel, pdf), or None below the surface."""
    wi, wgt, pdf = np.zeros(3), np.zeros(3), C.c_double(0.0)
    a = [np.ascontiguousarray(v, np.float64) for v in (n, wo, ks)]
    ok = lib().or_glossy_sample(_p(a[0]), _p(a[1]), _p(a[2]), C.c_double(alpha), C.c_double(u0),
                                C.c_double(u1), _p(wi), _p(wgt), C.byref(pdf))
    return (wi, wgt, pdf.value) if ok else None


def radiance(scene: Scene, vol: Volume, y, tri, frm, u=None):
    """Outgoing radiance (Le + L_DDGI+)(y, y -> frm) for batches of points;
    u ([n][2], optional) are the random numbers of the glossy sample."""
    y = np.ascontiguousarray(y, np.float64).reshape(-1, 3)
    frm = np.ascontiguousarray(frm, np.float64).reshape(-1, 3)
    tri = np.ascontiguousarray(tri, np.int32)
    uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1, 2)
    L = np.zeros_like(y)
    lib().or_radiance_batch(C.byref(scene.s), C.byref(vol.v), C.c_int32(y.shape[0]), _p(y),
                            _p(tri, _ip), _p(frm), _p(uu), _p(L))
    return L


def pt_reference(scene: Scene, cam, pix, seed, sample0, spp):
    """Sum of spp path-traced samples for each listed pixel ([n, 3])."""
    pix = np.ascontiguousarray(pix, np.int32)
    out = np.zeros((len(pix), 3))
    c = camera(cam)
    for k, q in enumerate(pix):
        lib().or_pt_pixel(C.byref(scene.s), C.byref(c), C.c_int32(int(q)), C.c_uint32(seed),
                          C.c_uint32(sample0), C.c_uint32(spp), _p(out[k]))
    return out


def mlp_eval(vol: Volume, p, n):
    p = np.ascontiguousarray(p, np.float64).reshape(-1, 3)
    n = np.ascontiguousarray(n, np.float64).reshape(-1, 3)
    out = np.zeros_like(p)
    for k in range(p.shape[0]):
        lib().or_mlp_eval(C.byref(vol.v), _p(p[k]), _p(n[k]), _p(out[k]))
    return out


def target(scene: Scene, x, nx, rho, y, tri, L) -> float:
    a = [np.ascontiguousarray(v, np.float64) for v in (x, nx, rho, y, L)]
    return lib().or_target(C.byref(scene.s), _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]),
                           C.c_int32(tri), _p(a[4]))


# --- frame chain ------------------------------------------------------------------

class Renderer:
    """The whole per-frame path on the CPU, in the order of Sec. 3.1:
    probe update, primary visibility, initial candidates, temporal reuse,
    spatial reuse passes, shading."""

    def __init__(self, sc, settings=None):
        self.sc = sc
        self.scene = Scene(sc)
        if settings is not None:
            self.scene.settings = settings
        st = sc.settings
        self.vol = Volume(sc.grid, st.irr_texels, st.depth_texels)
        self.prev_g: Optional[GBuffer] = None
        self.prev_res: Optional[Reservoirs] = None
        self.prev_cam = None

    def frame(self, f: int, cam=None, probe_update_enabled=True, xf=None, emitter_radiance=None):
        """One frame; xf / emitter_radiance (optional) first move the scene."""
        sc, S = self.sc, self.scene
        cam = cam or sc.cameras[f % len(sc.cameras)]
        out = {}
        if xf is not None or emitter_radiance is not None:
            S.update(xf, emitter_radiance)
        if probe_update_enabled:
            probe_update(S, self.vol, f)
        g = gbuffer(S, cam, self.prev_cam)
        out["gbuffer"] = g
        res, resid = restir_initial(S, self.vol, g, f)
        out["initial"], out["resid"] = res, resid
        if self.prev_res is not None:
            res = restir_temporal(S, g, self.prev_g, self.prev_cam.pos, res, self.prev_res, f)
        out["temporal"] = res
        for i in range(sc.settings.spatial_passes):
            res = restir_spatial(S, g, res, f, i)
            out[f"spatial{i}"] = res
        out["final"] = res
        out["radiance"] = shade(S, self.vol, g, res, resid, frame=f)
        self.prev_g, self.prev_res, self.prev_cam = g, res, cam
        return out


# --- metrics (Sec. 4) ------------------------------------------------------------

def mape(v, ref, eps=0.01) -> float:
    """Mean absolute percentage error of Sec. 4: mean of |v - ref| / (ref + eps)
    over every pixel value (each colour channel counts as one value)."""
    v = np.asarray(v, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    return float(np.mean(np.abs(v - ref) / (ref + eps)))


def mse(v, ref) -> float:
    v = np.asarray(v, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    return float(np.mean((v - ref) ** 2))
