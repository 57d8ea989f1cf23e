"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point that include/ddgi.h declares, and
rejects invalid arguments before touching the device.  Also checks that the
oracle and the CUDA library share no code."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ddgi.h")).read()
    return re.findall(r"^(?:ddgi_status|const char\*)\s+(\w+)\(", src, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_2108_05263_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_the_header():
    from paper_2108_05263_gb300 import ddgi
    assert sorted(ddgi.EXPORTS) == sorted(_declared())


def _config(**kw):
    from paper_2108_05263_gb300 import ddgi
    import scenegen
    sc = scenegen.tiny_room()
    cfg = ddgi.config_from(sc.grid, sc.settings)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return sc, cfg


@pytest.mark.parametrize("field,value", [
    ("rays_per_probe", 0), ("rays_per_probe", 5000), ("irr_texels", 1), ("depth_texels", 64),
    ("hysteresis", 1.0), ("num_bsdf_candidates", 0), ("num_light_candidates", 70),
    ("spatial_radius", 0), ("spatial_neighbours", 99), ("depth_sharpness", -1.0),
])
def test_create_rejects_bad_config_on_the_host(lib, field, value):
    from paper_2108_05263_gb300 import ddgi
    ddgi.load()
    sc, cfg = _config(**{field: value})
    v = np.ascontiguousarray(sc.verts, np.float32)
    a = np.ascontiguousarray(sc.albedo, np.float32)
    e = np.ascontiguousarray(sc.emission, np.float32)
    scene = ddgi.Scene(sc.num_tris, v.ctypes.data, a.ctypes.data, e.ctypes.data)
    h = C.c_void_p()
    rc = ddgi.load().ddgi_create(C.byref(scene), C.byref(cfg), C.byref(h))
    assert rc == ddgi.ERR_INVALID_ARG
    assert not h.value


def test_create_rejects_non_finite_geometry(lib):
    from paper_2108_05263_gb300 import ddgi
    sc, cfg = _config()
    v = np.ascontiguousarray(sc.verts, np.float32).copy()
    v[3, 1, 2] = np.nan
    a = np.ascontiguousarray(sc.albedo, np.float32)
    e = np.ascontiguousarray(sc.emission, np.float32)
    scene = ddgi.Scene(sc.num_tris, v.ctypes.data, a.ctypes.data, e.ctypes.data)
    h = C.c_void_p()
    assert ddgi.load().ddgi_create(C.byref(scene), C.byref(cfg), C.byref(h)) == ddgi.ERR_INVALID_ARG


def test_null_context_is_rejected(lib):
    from paper_2108_05263_gb300 import ddgi
    L = ddgi.load()
    assert L.ddgi_destroy(None) == ddgi.ERR_INVALID_ARG
    assert L.ddgi_probe_update(None, 0, None) == ddgi.ERR_INVALID_ARG
    assert L.ddgi_get_status(None, None) == ddgi.ERR_INVALID_ARG


def test_oracle_and_library_share_no_code():
    pkg = os.path.join(ROOT, "paper_2108_05263_gb300")
    orc = os.path.join(ROOT, "oracle")
    for d, bad in ((pkg, ("oracle", "ddgi_oracle")), (orc, ("paper_2108_05263_gb300", "csrc", "ddgi.h"))):
        for root, _, files in os.walk(d):
            for f in files:
                if not f.endswith((".py", ".c", ".h", ".cu", ".cuh", ".cpp")):
                    continue
                text = open(os.path.join(root, f)).read()
                for b in bad:
                    assert not re.search(rf"(import|include|from)\s+[\"<]?[\w./]*{re.escape(b)}", text), (f, b)
