"""ctypes binding of libddgi.so (``include/ddgi.h``): the same entry points,
argument marshalling only.  Every step of the frame runs in the library's
CUDA kernels; there is no CPU path.  Buffers are torch CUDA tensors; streams
are torch CUDA streams (default: the current stream).

Raises ``RuntimeError`` at load time if the library has not been built, and
``DDGIError`` whenever an entry point returns a non-zero status.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

from . import build as _build

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_NOT_READY = -3
ERR_TRAVERSAL_LIMIT = -4
ERR_BOUNDS = -5
ERR_OOM = -6
ERR_DEVICE_WAIT = -7

_f3 = C.c_float * 3
_i3 = C.c_int32 * 3


class Scene(C.Structure):
    _fields_ = [("num_tris", C.c_uint32), ("vertices", C.c_void_p), ("albedo", C.c_void_p),
                ("emission", C.c_void_p), ("tri_instance", C.c_void_p), ("num_instances", C.c_uint32),
                ("glossy", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("origin", _f3), ("spacing", _f3), ("counts", _i3), ("rays_per_probe", C.c_uint32),
                ("irr_texels", C.c_uint32), ("depth_texels", C.c_uint32), ("hysteresis", C.c_float),
                ("le_attenuation", C.c_float), ("depth_sharpness", C.c_float),
                ("num_light_candidates", C.c_uint32), ("num_bsdf_candidates", C.c_uint32),
                ("temporal_mcap", C.c_float), ("spatial_neighbours", C.c_uint32),
                ("spatial_radius", C.c_uint32), ("normal_reject_cos", C.c_float),
                ("depth_reject_frac", C.c_float), ("seed", C.c_uint32),
                ("learned_target", C.c_uint32), ("train_samples", C.c_uint32), ("train_lr", C.c_float),
                ("mlp_seed", C.c_uint32), ("train_ema", C.c_float), ("probe_relocation", C.c_uint32),
                ("mlp_bf16", C.c_uint32), ("candidate_stride", C.c_uint32),
                ("footprint_c", C.c_float), ("mlp_fp32", C.c_uint32), ("traversal_visit_cap", C.c_uint32)]


class Camera(C.Structure):
    _fields_ = [("pos", _f3), ("fwd", _f3), ("right", _f3), ("up", _f3),
                ("tan_half_fovy", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class GBuf(C.Structure):
    _fields_ = [("g0", C.c_void_p), ("g1", C.c_void_p), ("g2", C.c_void_p),
                ("width", C.c_uint32), ("height", C.c_uint32), ("eye", _f3)]


class Res(C.Structure):
    _fields_ = [("rec", C.c_void_p), ("num_pixels", C.c_uint32)]


class Info(C.Structure):
    _fields_ = [("num_tris", C.c_uint32), ("num_emitters", C.c_uint32), ("num_probes", C.c_uint32),
                ("rays_per_probe", C.c_uint32), ("irr_tile", C.c_uint32), ("depth_tile", C.c_uint32),
                ("bvh_nodes", C.c_uint32), ("bvh_depth", C.c_uint32), ("updates", C.c_uint32),
                ("device_bytes", C.c_uint64)]


class DDGIError(RuntimeError):
    def __init__(self, fn, code, msg=""):
        super().__init__(f"{fn} returned {code}: {msg}")
        self.code = code


_lib = None

# entry points declared in include/ddgi.h (all return ddgi_status except the last)
EXPORTS = ["ddgi_create", "ddgi_destroy", "ddgi_get_info", "ddgi_probe_update", "ddgi_probe_trace",
           "ddgi_probe_blend", "ddgi_probe_relocate", "ddgi_scene_update", "ddgi_state_save",
           "ddgi_state_load", "ddgi_probe_state_get", "ddgi_probe_state_set",
           "ddgi_probe_rays_get", "ddgi_probe_rays_set", "ddgi_gbuffer", "restir_initial",
           "restir_temporal", "restir_initial_temporal", "restir_spatial", "ddgi_reservoirs_attach_normals", "ddgi_shade", "ddgi_reference_accumulate", "ddgi_image_metrics",
           "ddgi_image_metrics_static", "ddgi_mlp_train", "ddgi_mlp_infer", "ddgi_mlp_grad",
           "ddgi_mlp_step", "ddgi_mlp_params_get", "ddgi_mlp_params_served_get",
           "ddgi_mlp_params_set", "ddgi_mlp_serve", "ddgi_mlp_samples_get",
           "ddgi_mlp_status", "ddgi_get_status", "ddgi_last_error"]

MLP_NPARAM = 18184


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libddgi.so (fails loudly if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libddgi.so not built ({p}); run paper_2108_05263_gb300.build.build()")
    L = C.CDLL(p)
    vp = C.c_void_p
    st = C.c_int32
    L.ddgi_create.argtypes = [C.POINTER(Scene), C.POINTER(Config), C.POINTER(vp)]
    L.ddgi_destroy.argtypes = [vp]
    L.ddgi_get_info.argtypes = [vp, C.POINTER(Info)]
    for fn in ("ddgi_probe_update", "ddgi_probe_trace", "ddgi_probe_blend", "ddgi_probe_relocate"):
        getattr(L, fn).argtypes = [vp, C.c_uint32, vp]
    L.ddgi_scene_update.argtypes = [vp, vp, C.c_uint32, vp, vp]
    L.ddgi_state_save.argtypes = [vp, vp, C.POINTER(C.c_size_t), vp]
    L.ddgi_state_load.argtypes = [vp, vp, C.c_size_t, vp]
    L.ddgi_probe_state_get.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_uint32), vp]
    L.ddgi_probe_state_set.argtypes = [vp, vp, vp, vp, C.c_uint32, vp]
    L.ddgi_probe_rays_get.argtypes = [vp, vp, vp]
    L.ddgi_probe_rays_set.argtypes = [vp, vp, vp]
    L.ddgi_gbuffer.argtypes = [vp, C.POINTER(Camera), C.POINTER(Camera), C.POINTER(GBuf), vp]
    L.restir_initial.argtypes = [vp, C.POINTER(GBuf), C.POINTER(Res), vp, C.c_uint32, vp]
    L.restir_temporal.argtypes = [vp, C.POINTER(GBuf), C.POINTER(C.c_float), C.POINTER(Res),
                                  C.POINTER(Res), C.POINTER(Res), C.c_uint32, vp]
    L.restir_spatial.argtypes = [vp, C.POINTER(GBuf), C.POINTER(Res), C.POINTER(Res), C.c_uint32,
                                 C.c_uint32, vp]
    L.restir_initial_temporal.argtypes = [vp, C.POINTER(GBuf), C.POINTER(C.c_float), C.POINTER(Res),
                                          C.POINTER(Res), C.POINTER(Res), vp, C.c_uint32, vp]
    L.ddgi_reservoirs_attach_normals.argtypes = [vp, C.POINTER(Res), vp]
    L.ddgi_shade.argtypes = [vp, C.POINTER(GBuf), C.POINTER(Res), vp, vp, C.c_uint32, vp]
    L.ddgi_reference_accumulate.argtypes = [vp, C.POINTER(Camera), C.c_uint32, C.c_uint32, vp, vp, vp]
    L.ddgi_image_metrics.argtypes = [vp, vp, C.c_uint32, vp, C.c_uint32, vp, vp]
    L.ddgi_image_metrics_static.argtypes = [vp, vp, C.c_uint32, vp, vp]
    L.ddgi_mlp_train.argtypes = [vp, C.c_uint32, vp]
    L.ddgi_mlp_infer.argtypes = [vp, vp, vp, C.c_uint32, vp]
    L.ddgi_mlp_grad.argtypes = [vp, vp, C.c_uint32, vp, vp]
    L.ddgi_mlp_step.argtypes = [vp, vp, C.c_uint32, vp]
    L.ddgi_mlp_params_get.argtypes = [vp, vp, vp]
    L.ddgi_mlp_params_served_get.argtypes = [vp, vp, vp]
    L.ddgi_mlp_params_set.argtypes = [vp, vp, vp]
    L.ddgi_mlp_samples_get.argtypes = [vp, vp, vp]
    L.ddgi_mlp_serve.argtypes = [vp, C.c_int32, vp]
    L.ddgi_mlp_status.argtypes = [vp, vp, vp]
    L.ddgi_get_status.argtypes = [vp, vp]
    L.ddgi_last_error.argtypes = [vp]
    L.ddgi_last_error.restype = C.c_char_p
    for fn in EXPORTS[:-1]:
        getattr(L, fn).restype = st
    _lib = L
    return L


# ---------------------------------------------------------------------------
# buffers
# ---------------------------------------------------------------------------

def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class GBuffer:
    """Three [N, 4] float32 planes (see ddgi_gbuf)."""

    def __init__(self, width: int, height: int, device="cuda", planes=None, eye=None):
        self.width, self.height = width, height
        n = width * height
        if planes is None:
            planes = [torch.empty((n, 4), dtype=torch.float32, device=device) for _ in range(3)]
        self.g0, self.g1, self.g2 = planes
        # camera position the planes were rendered from (Context.gbuffer sets it)
        self.eye = np.zeros(3, np.float32) if eye is None else np.asarray(eye, np.float32)

    def c(self) -> GBuf:
        return GBuf(self.g0.data_ptr(), self.g1.data_ptr(), self.g2.data_ptr(), self.width, self.height,
                    _f3(*[float(a) for a in self.eye]))

    def numpy(self):
        return tuple(t.cpu().numpy() for t in (self.g0, self.g1, self.g2))


class Reservoirs:
    """One 64-byte record per pixel: a [N, 16] float32 tensor (see
    ddgi_reservoirs): y.xyz, W | L.rgb, M | owner normal.xyz, owner distance
    (> 0 exactly for a valid owner) | uint32 bits of (triangle of y, tag),
    octahedral map of y's normal (2 floats)."""

    def __init__(self, n: int, device="cuda", rec: Optional[torch.Tensor] = None):
        self.n = n
        self.rec = rec if rec is not None else torch.empty((n, 16), dtype=torch.float32, device=device)

    def c(self) -> Res:
        return Res(self.rec.data_ptr(), self.n)

    def numpy(self) -> np.ndarray:
        return self.rec.cpu().numpy()

    @staticmethod
    def fields(rec: np.ndarray) -> dict:
        """Named views of a [N, 16] record array."""
        bits = np.ascontiguousarray(rec[:, 12:16]).view(np.uint32)
        return {"y": rec[:, 0:3], "W": rec[:, 3], "L": rec[:, 4:7], "M": rec[:, 7],
                "n": rec[:, 8:11], "dist": rec[:, 11], "tri": bits[:, 0].view(np.int32),
                "tag": bits[:, 1], "valid": (rec[:, 11] > 0).astype(np.uint32), "ny_oct": rec[:, 14:16]}


METRIC_SCRATCH_DOUBLES = 2048


def image_metrics(img: torch.Tensor, ref: torch.Tensor, scratch: Optional[torch.Tensor] = None,
                  out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """(MSE, MAPE) of [n, 4] float32 CUDA images as a float64 CUDA tensor [2]."""
    L = load()
    n = img.shape[0]
    if scratch is None:
        scratch = torch.empty(METRIC_SCRATCH_DOUBLES, dtype=torch.float64, device=img.device)
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=img.device)
    rc = L.ddgi_image_metrics(_ptr(img), _ptr(ref), n, _ptr(scratch), scratch.numel(), _ptr(out),
                              _stream(stream))
    if rc != OK:
        raise DDGIError("ddgi_image_metrics", rc)
    return out


def camera(cam) -> Camera:
    """From any object with pos/fwd/right/up/tan_half_fovy/width/height."""
    return Camera(_f3(*map(float, cam.pos)), _f3(*map(float, cam.fwd)), _f3(*map(float, cam.right)),
                  _f3(*map(float, cam.up)), float(cam.tan_half_fovy), int(cam.width), int(cam.height))


def config_from(grid, settings) -> Config:
    """From a probe grid (origin/spacing/counts) and method settings."""
    c = Config()
    c.origin = _f3(*map(float, grid.origin))
    c.spacing = _f3(*map(float, grid.spacing))
    c.counts = _i3(*map(int, grid.counts))
    c.rays_per_probe = settings.rays_per_probe
    c.irr_texels = settings.irr_texels
    c.depth_texels = settings.depth_texels
    c.hysteresis = settings.hysteresis
    c.le_attenuation = settings.le_attenuation
    c.depth_sharpness = settings.depth_sharpness
    c.num_light_candidates = settings.num_light_candidates
    c.num_bsdf_candidates = settings.num_bsdf_candidates
    c.temporal_mcap = settings.temporal_mcap
    c.spatial_neighbours = settings.spatial_neighbours
    c.spatial_radius = settings.spatial_radius
    c.normal_reject_cos = settings.normal_reject_cos
    c.depth_reject_frac = settings.depth_reject_frac
    c.seed = settings.seed
    c.learned_target = int(getattr(settings, "learned_target", 0))
    c.train_samples = int(getattr(settings, "train_samples", 0))
    c.train_lr = float(getattr(settings, "train_lr", 1e-3))
    c.mlp_seed = int(getattr(settings, "mlp_seed", 1))
    c.train_ema = float(getattr(settings, "train_ema", 0.97))
    c.probe_relocation = int(getattr(settings, "probe_relocation", 0))
    c.mlp_bf16 = int(getattr(settings, "mlp_bf16", 0))
    c.candidate_stride = int(getattr(settings, "candidate_stride", 1))
    c.footprint_c = float(getattr(settings, "footprint_c", 0.2))
    c.mlp_fp32 = int(getattr(settings, "mlp_fp32", 0))
    c.traversal_visit_cap = int(getattr(settings, "traversal_visit_cap", 0))
    return c


class Context:
    """Owns a ddgi_ctx (scene BVH, emitter table, probe maps, probe rays)."""

    def __init__(self, verts, albedo, emission, grid, settings, tri_instance=None, glossy=None):
        L = load()
        self.L = L
        self._v = np.ascontiguousarray(verts, np.float32)
        self._a = np.ascontiguousarray(albedo, np.float32)
        self._e = np.ascontiguousarray(emission, np.float32)
        sc = Scene(self._v.shape[0], self._v.ctypes.data, self._a.ctypes.data, self._e.ctypes.data)
        if tri_instance is not None:
            self._ti = np.ascontiguousarray(tri_instance, np.int32)
            sc.tri_instance = self._ti.ctypes.data
            sc.num_instances = int(self._ti.max(initial=-1)) + 1
        if glossy is not None:
            self._gl = np.ascontiguousarray(glossy, np.float32)
            sc.glossy = self._gl.ctypes.data
        self.cfg = config_from(grid, settings)
        self.settings = settings
        h = C.c_void_p()
        rc = L.ddgi_create(C.byref(sc), C.byref(self.cfg), C.byref(h))
        if rc != OK:
            raise DDGIError("ddgi_create", rc)
        self.h = h
        self.info = self.get_info()

    @staticmethod
    def from_scene(sc, settings=None) -> "Context":
        return Context(sc.verts, sc.albedo, sc.emission, sc.grid, settings or sc.settings,
                       getattr(sc, "tri_instance", None), getattr(sc, "glossy", None))

    def close(self):
        if getattr(self, "h", None):
            self.L.ddgi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, fn, rc):
        if rc != OK:
            raise DDGIError(fn, rc, self.L.ddgi_last_error(self.h).decode())

    def get_info(self) -> Info:
        i = Info()
        self._check("ddgi_get_info", self.L.ddgi_get_info(self.h, C.byref(i)))
        return i

    # --- scene dynamics ---
    def scene_update(self, xf=None, emitter_radiance=None, stream=None):
        """Instance transforms ([I][12] row-major 3x4) and / or emitter
        radiance ([E][3]); either may be None."""
        a = None if xf is None else np.ascontiguousarray(xf, np.float32).reshape(-1, 12)
        b = None if emitter_radiance is None else np.ascontiguousarray(emitter_radiance, np.float32)
        self._check("ddgi_scene_update",
                    self.L.ddgi_scene_update(self.h, None if a is None else a.ctypes.data,
                                             0 if a is None else a.shape[0],
                                             None if b is None else b.ctypes.data, _stream(stream)))

    # --- checkpoint / resume ---
    def state_save(self, stream=None) -> bytes:
        n = C.c_size_t(0)
        self._check("ddgi_state_save", self.L.ddgi_state_save(self.h, None, C.byref(n), _stream(stream)))
        buf = C.create_string_buffer(n.value)
        self._check("ddgi_state_save", self.L.ddgi_state_save(self.h, buf, C.byref(n), _stream(stream)))
        return buf.raw[:n.value]

    def state_load(self, blob: bytes, stream=None):
        buf = C.create_string_buffer(blob, len(blob))
        self._check("ddgi_state_load", self.L.ddgi_state_load(self.h, buf, len(blob), _stream(stream)))

    # --- probe update (Sec. 3.2) ---
    def probe_update(self, frame, stream=None):
        self._check("ddgi_probe_update", self.L.ddgi_probe_update(self.h, frame, _stream(stream)))

    def probe_trace(self, frame, stream=None):
        self._check("ddgi_probe_trace", self.L.ddgi_probe_trace(self.h, frame, _stream(stream)))

    def probe_blend(self, frame, stream=None):
        self._check("ddgi_probe_blend", self.L.ddgi_probe_blend(self.h, frame, _stream(stream)))

    def probe_relocate(self, frame, stream=None):
        self._check("ddgi_probe_relocate", self.L.ddgi_probe_relocate(self.h, frame, _stream(stream)))

    def probe_state_get(self, stream=None):
        i = self.info
        P = i.num_probes
        irr = np.zeros((P, i.irr_tile, i.irr_tile, 4), np.float32)
        dep = np.zeros((P, i.depth_tile, i.depth_tile, 2), np.float32)
        off = np.zeros((P, 4), np.float32)
        upd = C.c_uint32()
        self._check("ddgi_probe_state_get",
                    self.L.ddgi_probe_state_get(self.h, irr.ctypes.data, dep.ctypes.data,
                                                off.ctypes.data, C.byref(upd), _stream(stream)))
        return irr, dep, off, upd.value

    def probe_state_set(self, irr=None, depth=None, offsets=None, updates=0, stream=None):
        arrs = [None if a is None else np.ascontiguousarray(a, np.float32) for a in (irr, depth, offsets)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        self._check("ddgi_probe_state_set",
                    self.L.ddgi_probe_state_set(self.h, ptrs[0], ptrs[1], ptrs[2], updates,
                                                _stream(stream)))

    def probe_rays_get(self, stream=None):
        i = self.info
        out = np.zeros((i.num_probes, i.rays_per_probe, 4), np.float32)
        self._check("ddgi_probe_rays_get", self.L.ddgi_probe_rays_get(self.h, out.ctypes.data, _stream(stream)))
        return out

    def probe_rays_set(self, rays, stream=None):
        a = np.ascontiguousarray(rays, np.float32)
        self._check("ddgi_probe_rays_set", self.L.ddgi_probe_rays_set(self.h, a.ctypes.data, _stream(stream)))

    # --- per-frame passes ---
    def gbuffer(self, cam, prev_cam, out: GBuffer, stream=None):
        c = camera(cam)
        pc = camera(prev_cam) if prev_cam is not None else None
        out.eye = np.asarray(cam.pos, np.float32)
        g = out.c()
        self._check("ddgi_gbuffer", self.L.ddgi_gbuffer(self.h, C.byref(c), C.byref(pc) if pc else None,
                                                        C.byref(g), _stream(stream)))

    def restir_initial(self, g: GBuffer, out: Reservoirs, residual: torch.Tensor, frame, stream=None):
        gc, oc = g.c(), out.c()
        self._check("restir_initial", self.L.restir_initial(self.h, C.byref(gc), C.byref(oc),
                                                            _ptr(residual), frame, _stream(stream)))

    def restir_temporal(self, g: GBuffer, prev_cam_pos, cur: Reservoirs, prev: Reservoirs,
                        out: Reservoirs, frame, stream=None):
        gc, cc, pc, oc = g.c(), cur.c(), prev.c(), out.c()
        cp = _f3(*map(float, prev_cam_pos))
        self._check("restir_temporal",
                    self.L.restir_temporal(self.h, C.byref(gc), cp, C.byref(cc), C.byref(pc),
                                           C.byref(oc), frame, _stream(stream)))

    def restir_initial_temporal(self, g: GBuffer, prev_cam_pos, scratch: Reservoirs, prev: Reservoirs,
                                out: Reservoirs, residual: torch.Tensor, frame, stream=None):
        """restir_initial and restir_temporal in one pass; scratch holds no
        reservoirs afterwards."""
        gc, sc_, pc, oc = g.c(), scratch.c(), prev.c(), out.c()
        cp = _f3(*map(float, prev_cam_pos))
        self._check("restir_initial_temporal",
                    self.L.restir_initial_temporal(self.h, C.byref(gc), cp, C.byref(sc_), C.byref(pc),
                                                   C.byref(oc), _ptr(residual), frame, _stream(stream)))

    def restir_spatial(self, g: GBuffer, src: Reservoirs, out: Reservoirs, frame, pass_idx,
                       stream=None):
        gc, ic, oc = g.c(), src.c(), out.c()
        self._check("restir_spatial", self.L.restir_spatial(self.h, C.byref(gc), C.byref(ic),
                                                            C.byref(oc), frame, pass_idx,
                                                            _stream(stream)))

    def reservoirs_attach_normals(self, res: Reservoirs, stream=None):
        """Words 14..15 (normal of y's triangle) of records written by the caller."""
        rc = res.c()
        self._check("ddgi_reservoirs_attach_normals",
                    self.L.ddgi_reservoirs_attach_normals(self.h, C.byref(rc), _stream(stream)))

    def shade(self, g: GBuffer, res: Reservoirs, residual: torch.Tensor, radiance: torch.Tensor,
              stream=None, frame: int = 0):
        gc, rc = g.c(), res.c()
        self._check("ddgi_shade", self.L.ddgi_shade(self.h, C.byref(gc), C.byref(rc), _ptr(residual),
                                                    _ptr(radiance), frame, _stream(stream)))

    def reference_accumulate(self, cam, sample0: int, spp: int, accum: torch.Tensor,
                             mean: Optional[torch.Tensor] = None, stream=None):
        c = camera(cam)
        self._check("ddgi_reference_accumulate",
                    self.L.ddgi_reference_accumulate(self.h, C.byref(c), sample0, spp, _ptr(accum), _ptr(mean),
                                                     _stream(stream)))

    # --- learned target form ---
    def mlp_train(self, frame, stream=None):
        self._check("ddgi_mlp_train", self.L.ddgi_mlp_train(self.h, frame, _stream(stream)))

    def mlp_infer(self, queries: torch.Tensor, out: torch.Tensor, stream=None):
        self._check("ddgi_mlp_infer", self.L.ddgi_mlp_infer(self.h, _ptr(queries), _ptr(out),
                                                            queries.shape[0], _stream(stream)))

    def mlp_grad(self, samples, stream=None) -> np.ndarray:
        a = np.ascontiguousarray(samples, np.float32)
        g = np.zeros(MLP_NPARAM, np.float32)
        self._check("ddgi_mlp_grad", self.L.ddgi_mlp_grad(self.h, a.ctypes.data, a.shape[0], g.ctypes.data,
                                                          _stream(stream)))
        return g

    def mlp_step(self, samples, stream=None):
        a = np.ascontiguousarray(samples, np.float32)
        self._check("ddgi_mlp_step", self.L.ddgi_mlp_step(self.h, a.ctypes.data, a.shape[0], _stream(stream)))
        torch.cuda.current_stream().synchronize()

    def mlp_params(self, stream=None) -> np.ndarray:
        p = np.zeros(MLP_NPARAM, np.float32)
        self._check("ddgi_mlp_params_get", self.L.ddgi_mlp_params_get(self.h, p.ctypes.data, _stream(stream)))
        return p

    def mlp_params_served(self, stream=None) -> np.ndarray:
        """The served network: moving average of the trained weights."""
        p = np.zeros(MLP_NPARAM, np.float32)
        self._check("ddgi_mlp_params_served_get",
                    self.L.ddgi_mlp_params_served_get(self.h, p.ctypes.data, _stream(stream)))
        return p

    def mlp_set_params(self, params, stream=None):
        a = np.ascontiguousarray(params, np.float32)
        self._check("ddgi_mlp_params_set", self.L.ddgi_mlp_params_set(self.h, a.ctypes.data, _stream(stream)))

    def mlp_serve(self, mode: int, stream=None):
        """0: judge decides, 1: always the network, 2: always the probes."""
        self._check("ddgi_mlp_serve", self.L.ddgi_mlp_serve(self.h, mode, _stream(stream)))

    def mlp_samples(self, stream=None) -> np.ndarray:
        n = self.cfg.train_samples
        out = np.zeros((n, 12), np.float32)
        self._check("ddgi_mlp_samples_get", self.L.ddgi_mlp_samples_get(self.h, out.ctypes.data, _stream(stream)))
        return out

    def mlp_status(self, stream=None) -> dict:
        o = np.zeros(8, np.float64)
        self._check("ddgi_mlp_status", self.L.ddgi_mlp_status(self.h, o.ctypes.data, _stream(stream)))
        keys = ["loss_scale", "overflow", "count", "judge_mlp", "judge_probe", "judge_n", "use_mlp", "step"]
        return dict(zip(keys, o.tolist()))

    def get_status(self, stream=None) -> int:
        return self.L.ddgi_get_status(self.h, _stream(stream))

    def last_error(self) -> str:
        return self.L.ddgi_last_error(self.h).decode()


class Frame:
    """Per-frame buffers of one resolution and a driver for the whole path
    (probe update, initial, temporal, spatial passes, shade) on one stream;
    ping-pongs the G-buffer and the final reservoirs between frames.

    With ``pipelined`` renders, a frame's probe trace runs during the frame
    before it: the trace of frame f + 1 -- which reads only frame f's
    blended maps (and relocated probes) and writes only the probe ray
    buffer, which nothing else reads until the next blend -- is issued on a
    side stream before frame f's shading pass and runs beside it (issued
    right after the blend it ran beside the resampling passes, whose
    issue-bound kernels it slowed more: 1.932 against 1.912 ms per frame);
    the next render waits for it and blends.  The results are those of the
    sequential frame.  If the next render moves the scene or renders another
    frame index, it waits for that trace and traces again on its own
    stream."""

    def __init__(self, ctx: Context, width: int, height: int, spatial_passes: int, device="cuda"):
        n = width * height
        self.ctx, self.width, self.height, self.n = ctx, width, height, n
        self.spatial_passes = spatial_passes
        self.g = [GBuffer(width, height, device), GBuffer(width, height, device)]
        self.res = [Reservoirs(n, device) for _ in range(4)]
        self.resid = torch.empty((n, 4), dtype=torch.float32, device=device)
        self.radiance = torch.empty((n, 4), dtype=torch.float32, device=device)
        self.prev_final: Optional[Reservoirs] = None
        self.prev_cam = None
        self.cur = 0
        self.side = torch.cuda.Stream(device)   # the next frame's probe trace
        self.ev_maps = torch.cuda.Event()        # this frame's maps blended (and probes relocated)
        self.ev_trace = torch.cuda.Event()       # the next frame's probe rays traced
        self.pending: Optional[int] = None      # frame whose probe trace is in flight on `side`

    def _probe_update(self, frame: int, stream, moved: bool):
        ctx = self.ctx
        st = stream if stream is not None else torch.cuda.current_stream()
        if self.pending is not None:
            st.wait_event(self.ev_trace)     # done before the ray buffer is read or rewritten
        if self.pending != frame or moved:
            ctx.probe_trace(frame, stream)
        self.pending = None
        ctx.probe_blend(frame, stream)
        if ctx.cfg.probe_relocation:
            ctx.probe_relocate(frame, stream)

    def _trace_next(self, frame: int, stream):
        """Issue frame + 1's probe trace on the side stream, after the work
        enqueued on `stream` so far (this frame's blend among it)."""
        st = stream if stream is not None else torch.cuda.current_stream()
        self.ev_maps.record(st)
        self.side.wait_event(self.ev_maps)
        self.ctx.probe_trace(frame + 1, self.side)
        self.ev_trace.record(self.side)
        self.pending = frame + 1

    def finish(self, stream=None):
        """Make `stream` wait for a probe trace still in flight."""
        if self.pending is not None:
            (stream or torch.cuda.current_stream()).wait_event(self.ev_trace)

    def render(self, frame: int, cam, gbuf: Optional[GBuffer] = None, stream=None,
               probe_update=True, xf=None, emitter_radiance=None, out: Optional[torch.Tensor] = None,
               fused: bool = False, pipelined: bool = False):
        """One frame.  If ``gbuf`` is given it is used as this frame's
        G-buffer (the primary-visibility pass is skipped); xf /
        emitter_radiance (optional) first move the scene; ``out`` (optional,
        [n][4] float32 on the device) receives the radiance instead of the
        frame's own buffer; ``fused`` runs the initial and temporal passes as
        one (restir_initial_temporal; same results); ``pipelined`` issues the
        next frame's probe trace on the side stream (class docstring)."""
        ctx = self.ctx
        moved = xf is not None or emitter_radiance is not None
        if moved:
            if self.pending is not None:   # the scene must not move under a trace in flight
                (stream or torch.cuda.current_stream()).wait_event(self.ev_trace)
            ctx.scene_update(xf, emitter_radiance, stream)
        if probe_update:
            self._probe_update(frame, stream, moved)
        elif self.pending is not None:
            self.finish(stream)
            self.pending = None
        g = gbuf
        if g is None:
            g = self.g[self.cur]
            ctx.gbuffer(cam, self.prev_cam, g, stream)
        init, tmp = self._free_pair()
        if fused and self.prev_final is not None:
            ctx.restir_initial_temporal(g, self.prev_cam.pos, init, self.prev_final, tmp, self.resid, frame,
                                        stream)
            res = tmp
        else:
            ctx.restir_initial(g, init, self.resid, frame, stream)
            res = init
            if self.prev_final is not None:
                ctx.restir_temporal(g, self.prev_cam.pos, init, self.prev_final, tmp, frame, stream)
                res = tmp
        for i in range(self.spatial_passes):
            nxt = self._other(res)
            ctx.restir_spatial(g, res, nxt, frame, i, stream)
            res = nxt
        rad = self.radiance if out is None else out
        if pipelined and probe_update:
            self._trace_next(frame, stream)
        ctx.shade(g, res, self.resid, rad, stream, frame=frame)
        self.prev_final, self.prev_cam = res, cam
        self.cur ^= 1
        return rad

    def _free_pair(self):
        free = [r for r in self.res if r is not self.prev_final]
        self._free = free
        return free[0], free[1]

    def _other(self, r):
        for c in self._free:
            if c is not r:
                return c
        raise AssertionError


class HostFramePipeline:
    """Frames from host G-buffers to host radiance, the copies overlapped
    with the computation: the next frame's G-buffer uploads on one stream
    and the last frame's radiance downloads on another while the current
    frame runs on the caller's stream (double-buffered device G-buffers and
    radiance, ordered by events).  Host buffers should be pinned."""

    def __init__(self, ctx: Context, width: int, height: int, spatial_passes: int, device="cuda",
                 fused: bool = False, pipelined: bool = False):
        n = width * height
        self.fused = fused   # restir_initial_temporal instead of the two passes
        self.pipelined = pipelined   # the next frame's probe trace beside this frame (Frame)
        self.frame = Frame(ctx, width, height, spatial_passes, device)
        self.gbuf = [GBuffer(width, height, device), GBuffer(width, height, device)]
        self.rad = [torch.empty((n, 4), dtype=torch.float32, device=device) for _ in range(2)]
        self.up = torch.cuda.Stream(device)
        self.down = torch.cuda.Stream(device)
        self.ev_in = [torch.cuda.Event() for _ in range(2)]     # upload into slot done
        self.ev_used = [torch.cuda.Event() for _ in range(2)]   # frame on slot done
        self.ev_out = [torch.cuda.Event() for _ in range(2)]    # download from slot done
        self.k = 0       # frames run
        self.n_up = 0    # G-buffers uploaded

    def upload(self, host_planes):
        """Queue the upload of the G-buffer of the next frame to run (at most
        one frame ahead of `run`)."""
        b = self.n_up % 2
        self.n_up += 1
        with torch.cuda.stream(self.up):
            self.up.wait_event(self.ev_used[b])                 # the slot's last frame is done with it
            for d, h in zip((self.gbuf[b].g0, self.gbuf[b].g1, self.gbuf[b].g2), host_planes):
                d.copy_(h, non_blocking=True)
            self.ev_in[b].record(self.up)

    def run(self, frame: int, cam, host_out, stream=None):
        """Render the frame whose G-buffer was queued first and queue the
        download of its radiance into host_out."""
        st = stream or torch.cuda.current_stream()
        b = self.k % 2
        st.wait_event(self.ev_in[b])
        st.wait_event(self.ev_out[b])                           # the slot's radiance was read out
        self.frame.render(frame, cam, gbuf=self.gbuf[b], stream=st, probe_update=True, out=self.rad[b],
                          fused=self.fused, pipelined=self.pipelined)
        self.ev_used[b].record(st)
        with torch.cuda.stream(self.down):
            self.down.wait_event(self.ev_used[b])
            host_out.copy_(self.rad[b], non_blocking=True)
            self.ev_out[b].record(self.down)
        self.k += 1

    def finish(self, stream=None):
        """Make `stream` wait for the last download (and a probe trace still
        in flight)."""
        st = stream or torch.cuda.current_stream()
        st.wait_event(self.ev_out[(self.k - 1) % 2])
        self.frame.finish(st)
