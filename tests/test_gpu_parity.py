"""GPU <-> oracle parity of every pass, through the C ABI.

Pass-isolated tests feed the CUDA pass exactly the inputs the oracle pass
receives (oracle upstream outputs, or seeded synthetic buffers) and compare
element by element.  Chain tests run the whole frame on both sides.

Tolerances (float32 kernels vs the fp64 oracle):
* hit triangles, reservoir triangles / tags: identical wherever no floating
  point tie decides; >= 99.9 % identical overall;
* radiance, W, cached radiance, residual, probe maps: |gpu - ref| <=
  1e-4 |ref| + ABS per value, on >= 99.9 % of the values (ABS is a small
  absolute floor stated per quantity: values at the float32 resolution of
  their neighbours).
"""
import math

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def dd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_05263_gb300 import build
    build.build()
    from paper_2108_05263_gb300 import ddgi
    ddgi.load()
    return ddgi


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _t(a, dtype=None):
    import torch
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a)
    return t.cuda()


def _gbuf_to_gpu(dd, g):
    g0, g1, g2 = g.planes()
    return dd.GBuffer(g.width, g.height, planes=[_t(g0), _t(g1), _t(g2)])


def _pack(y, W, L, M, tri, tag, nrm, dist, valid):
    """Reservoir records in the library's layout (the owning pixel's normal
    and distance come from its G-buffer; an invalid owner has distance 0).
    Words 14..15, the normal of y's triangle, are left to
    ddgi_reservoirs_attach_normals."""
    n = len(W)
    rec = np.zeros((n, 16), np.float32)
    rec[:, 0:3], rec[:, 3] = y, W
    rec[:, 4:7], rec[:, 7] = L, M
    rec[:, 8:11], rec[:, 11] = nrm, np.where(np.asarray(valid) != 0, dist, 0.0)
    bits = np.zeros((n, 4), np.uint32)
    bits[:, 0] = np.asarray(tri).astype(np.int64).astype(np.uint32)
    bits[:, 1] = tag
    rec[:, 12:14] = bits[:, :2].view(np.float32)
    return rec


def _upload_res(dd, ctx, rec):
    r = dd.Reservoirs(rec.shape[0], rec=_t(rec))
    ctx.reservoirs_attach_normals(r)
    return r


def _res_to_gpu(dd, ctx, r, g):
    rec = _pack(r.y, r.W, r.L, r.M, r.tri, r.tag, g.nrm, g.dist, (g.tri >= 0).astype(np.uint32))
    return _upload_res(dd, ctx, rec)


def _synthetic_res_to_gpu(dd, ctx, res, gplanes):
    r0, r1, r2 = res
    g0, g1, _ = gplanes
    valid = (np.ascontiguousarray(g1[:, 3]).view(np.uint32) != 0xFFFFFFFF).astype(np.uint32)
    rec = _pack(r0[:, :3], r0[:, 3], r1[:, :3], r1[:, 3], r2[:, 0].view(np.int32), r2[:, 1],
                g1[:, :3], g0[:, 3], valid)
    return _upload_res(dd, ctx, rec)


def _vol_to_gpu(ctx, vol):
    P = vol.P
    irr = np.zeros(vol.irr.shape[:-1] + (4,), np.float32)
    irr[..., :3] = vol.irr
    off = np.zeros((P, 4), np.float32)
    off[:, :3] = vol.offset
    ctx.probe_state_set(irr, vol.depth.astype(np.float32), off, vol.updates)


def _close(gpu, ref, abs_floor, rel=REL):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(gpu - ref) <= rel * np.abs(ref) + abs_floor


def _frac(mask):
    return float(np.mean(mask)) if mask.size else 1.0


def _res_compare(rec, orr, w_abs=1e-6, l_abs=1e-5, what=""):
    """GPU reservoir records vs oracle Reservoirs; returns tag agreement."""
    from paper_2108_05263_gb300 import ddgi
    f = ddgi.Reservoirs.fields(rec)
    same = (f["tri"] == orr.tri) & (f["tag"] == orr.tag)
    agree = _frac(same)
    assert agree >= 0.999, f"{what}: selections agree on {agree:.5f}"
    np.testing.assert_array_equal(f["M"], orr.M.astype(np.float32))
    ok = same & (orr.tri >= 0)
    assert _frac(_close(f["W"][ok], orr.W[ok], w_abs)) >= 0.999, what
    assert _frac(_close(f["L"][ok], orr.L[ok], l_abs).all(axis=1)) >= 0.999, what
    assert _frac(_close(f["y"][ok], orr.y[ok], 1e-5).all(axis=1)) >= 0.999, what
    return agree


# ---------------------------------------------------------------------------
# tiny room: every pass in isolation, all pixels
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny(dd, orc):
    """Oracle run of the tiny room for two frames (the GPU inputs)."""
    sc = scenegen.tiny_room()
    R = orc.Renderer(sc)
    frames = [R.frame(f) for f in range(2)]
    vol_after = R.vol.copy()
    return sc, R, frames, vol_after


def test_gbuffer_parity(dd, orc, tiny):
    sc, R, _, _ = tiny
    ctx = dd.Context.from_scene(sc)
    cam, pc = sc.cameras[1], sc.cameras[0]
    g = dd.GBuffer(cam.width, cam.height)
    ctx.gbuffer(cam, pc, g)
    g0, g1, g2 = g.numpy()
    ref = orc.gbuffer(orc.Scene(sc), cam, pc)
    tri = g1[:, 3].view(np.int32)
    assert _frac(tri == ref.tri) >= 0.999
    ok = tri == ref.tri
    assert _frac(_close(g0[ok, :3], ref.pos[ok], 1e-5).all(1)) == 1.0
    assert _frac(_close(g0[ok, 3], ref.dist[ok], 1e-6)) == 1.0
    np.testing.assert_allclose(g1[ok, :3], ref.nrm[ok], atol=1e-6)
    np.testing.assert_array_equal(g2[ok, 3].view(np.int32), ref.prev[ok])
    assert ctx.get_status() == dd.OK


def test_probe_trace_and_blend_parity(dd, orc, tiny):
    sc, _, _, _ = tiny
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid)
    for f in range(3):
        orc.probe_update(S, vol, f)
    ctx = dd.Context.from_scene(sc)
    _vol_to_gpu(ctx, vol)
    # trace, isolated: same maps in, rays out
    ctx.probe_trace(3)
    rays = ctx.probe_rays_get()
    ref = orc.probe_trace(S, vol, 3)
    hit_same = np.sign(rays[..., 3]) == np.sign(ref[..., 3])
    assert _frac(hit_same) >= 0.999
    assert _frac(_close(np.abs(rays[..., 3])[hit_same], np.abs(ref[..., 3])[hit_same], 1e-6)) >= 0.999
    assert _frac(_close(rays[..., :3][hit_same], ref[..., :3][hit_same], 1e-5).all(-1)) >= 0.999
    # blend, isolated: oracle rays in, maps out
    ctx.probe_rays_set(ref.astype(np.float32))
    ctx.probe_blend(3)
    orc.probe_blend(vol, ref, 3, S.settings)
    irr, dep, _, upd = ctx.probe_state_get()
    assert upd == 4
    assert _frac(_close(irr[..., :3], vol.irr, 1e-5)) >= 0.9999
    assert _frac(_close(dep, vol.depth, 1e-5)) >= 0.9999
    assert ctx.get_status() == dd.OK


@pytest.mark.parametrize("irr_n,depth_n,rays", [(8, 16, 256), (5, 7, 37), (2, 3, 1), (32, 32, 64), (16, 32, 1024)])
def test_probe_blend_shapes_parity(dd, orc, irr_n, depth_n, rays):
    """The blend alone on seeded ray data (radiance; front-face, back-face
    and missed distances) for map and ray-set shapes that exercise its
    padding: odd texel counts (texel rows padded to 4), a ray count that
    leaves a ragged last chunk of weights, one ray, 32 x 32 maps, and
    16 x 32 maps with 1024 rays, whose products are split over several CTAs
    (borders then refreshed by a kernel of their own); two updates, the
    second mixing by the hysteresis.  Then a probe trace, whose hits query
    the blended maps through the query's 2x2 tap blocks (written by the
    blend, or rebuilt after the border kernel when the products were
    split)."""
    import dataclasses
    sc = scenegen.tiny_room(width=32, height=24, frames=1)
    sc.settings = dataclasses.replace(sc.settings, rays_per_probe=rays, irr_texels=irr_n, depth_texels=depth_n)
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid, irr_n, depth_n)
    ctx = dd.Context.from_scene(sc)
    P = vol.P
    rng = np.random.default_rng(1000 * irr_n + 10 * depth_n + rays)
    for f in range(2):
        ray = np.zeros((P, rays, 4), np.float32)
        ray[..., :3] = rng.uniform(0.0, 2.0, (P, rays, 3))
        t = rng.uniform(0.05, 4.0, (P, rays))
        kind = rng.random((P, rays))
        ray[..., 3] = np.where(kind < 0.2, -t, np.where(kind < 0.35, 1e30, t))
        ctx.probe_rays_set(ray)
        ctx.probe_blend(f)
        vol.updates = f   # the blend mixes by the hysteresis from the second update on
        orc.probe_blend(vol, ray.astype(np.float64), f, S.settings)
    irr, dep, _, upd = ctx.probe_state_get()
    assert upd == 2
    assert _frac(_close(irr[..., :3], vol.irr, 1e-5)) >= 0.9999
    assert _frac(_close(dep, vol.depth, 1e-5)) >= 0.9999
    assert np.abs(irr[..., 3]).max() == 0.0   # the fourth channel is untouched
    ctx.probe_trace(2)
    rays2 = ctx.probe_rays_get()
    ref2 = orc.probe_trace(S, vol, 2)
    same = np.sign(rays2[..., 3]) == np.sign(ref2[..., 3])
    assert _frac(same) >= 0.999
    assert _frac(_close(rays2[..., :3][same], ref2[..., :3][same], 1e-5).all(-1)) >= 0.999
    assert ctx.get_status() == dd.OK


def test_probe_update_chain_parity(dd, orc, tiny):
    sc, _, _, _ = tiny
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid)
    ctx = dd.Context.from_scene(sc)
    for f in range(6):
        orc.probe_update(S, vol, f)
        ctx.probe_update(f)
    irr, dep, _, _ = ctx.probe_state_get()
    # six free-running updates (each frame's maps feed the next trace):
    # the parity bar of 1e-4 relative with the radiance floor 1e-5
    assert _frac(_close(irr[..., :3], vol.irr, 1e-5)) >= 0.999
    assert _frac(_close(dep, vol.depth, 1e-5)) >= 0.999
    assert np.abs(irr[..., :3] - vol.irr).max() <= 1e-4 * np.abs(vol.irr).max()


def test_initial_parity(dd, orc, tiny):
    import torch
    sc, R, frames, _ = tiny
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid)
    for f in range(3):
        orc.probe_update(S, vol, f)
    g = frames[1]["gbuffer"]
    ref, resid = orc.restir_initial(S, vol, g, 7)
    ctx = dd.Context.from_scene(sc)
    _vol_to_gpu(ctx, vol)
    gg = _gbuf_to_gpu(dd, g)
    out = dd.Reservoirs(g.tri.shape[0])
    rr = torch.empty((g.tri.shape[0], 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(gg, out, rr, 7)
    _res_compare(out.numpy(), ref, what="initial")
    # the record carries its pixel's G-buffer geometry verbatim
    f = dd.Reservoirs.fields(out.numpy())
    g0, g1, _ = g.planes()
    valid = g.tri >= 0
    np.testing.assert_array_equal(f["valid"], valid.astype(np.uint32))
    np.testing.assert_array_equal(f["n"][valid], g1[valid, :3])
    np.testing.assert_array_equal(f["dist"][valid], g0[valid, 3])
    # and the unit normal of its sample's triangle, octahedral map (Meyer et
    # al. 2010): (u, v, 1 - |u| - |v|), the lower half folded, normalised
    has = f["tri"] >= 0
    u, v = f["ny_oct"][has, 0].astype(np.float64), f["ny_oct"][has, 1].astype(np.float64)
    z = 1.0 - np.abs(u) - np.abs(v)
    x = np.where(z < 0, (1.0 - np.abs(v)) * np.where(u >= 0, 1.0, -1.0), u)
    y = np.where(z < 0, (1.0 - np.abs(u)) * np.where(v >= 0, 1.0, -1.0), v)
    d = np.stack([x, y, z], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(d, S.normals[f["tri"][has]], atol=1e-6)
    assert np.all(f["ny_oct"][~has] == 0)
    assert _frac(_close(rr.cpu().numpy()[:, :3], resid, 1e-5).all(1)) >= 0.999
    assert ctx.get_status() == dd.OK


def test_temporal_parity(dd, orc, tiny):
    sc, R, frames, _ = tiny
    S = orc.Scene(sc)
    f0, f1 = frames
    ref = orc.restir_temporal(S, f1["gbuffer"], f0["gbuffer"], sc.cameras[0].pos, f1["initial"], f0["final"], 1)
    ctx = dd.Context.from_scene(sc)
    out = dd.Reservoirs(ref.W.shape[0])
    ctx.restir_temporal(_gbuf_to_gpu(dd, f1["gbuffer"]), sc.cameras[0].pos,
                        _res_to_gpu(dd, ctx, f1["initial"], f1["gbuffer"]),
                        _res_to_gpu(dd, ctx, f0["final"], f0["gbuffer"]), out, 1)
    _res_compare(out.numpy(), ref, what="temporal")


def test_spatial_parity(dd, orc, tiny):
    sc, R, frames, _ = tiny
    S = orc.Scene(sc)
    f1 = frames[1]
    ref = orc.restir_spatial(S, f1["gbuffer"], f1["temporal"], 1, 0)
    ctx = dd.Context.from_scene(sc)
    out = dd.Reservoirs(ref.W.shape[0])
    ctx.restir_spatial(_gbuf_to_gpu(dd, f1["gbuffer"]), _res_to_gpu(dd, ctx, f1["temporal"], f1["gbuffer"]),
                       out, 1, 0)
    _res_compare(out.numpy(), ref, what="spatial")


def test_shade_parity(dd, orc, tiny):
    import torch
    sc, R, frames, vol_after = tiny
    S = orc.Scene(sc)
    f1 = frames[1]
    ref = orc.shade(S, vol_after, f1["gbuffer"], f1["final"], f1["resid"])
    ctx = dd.Context.from_scene(sc)
    _vol_to_gpu(ctx, vol_after)
    n = ref.shape[0]
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    resid = np.zeros((n, 4), np.float32)
    resid[:, :3] = f1["resid"]
    ctx.shade(_gbuf_to_gpu(dd, f1["gbuffer"]), _res_to_gpu(dd, ctx, f1["final"], f1["gbuffer"]), _t(resid), rad)
    out = rad.cpu().numpy()
    assert _frac(_close(out[:, :3], ref, 1e-5).all(1)) >= 0.999
    assert ctx.get_status() == dd.OK


# ---------------------------------------------------------------------------
# whole frames on both sides
# ---------------------------------------------------------------------------

def _chain(dd, orc, sc, nframes, fused=False):
    R = orc.Renderer(sc)
    ctx = dd.Context.from_scene(sc)
    cam0 = sc.cameras[0]
    fr = dd.Frame(ctx, cam0.width, cam0.height, sc.settings.spatial_passes)
    stats = []
    for f in range(nframes):
        cam = sc.cameras[f % len(sc.cameras)]
        xf, le = sc.instance_transforms(f), sc.emitter_radiance(f)
        ref = R.frame(f, cam, xf=xf, emitter_radiance=le)
        rad = fr.render(f, cam, xf=xf, emitter_radiance=le, fused=fused).cpu().numpy()[:, :3]
        fl = dd.Reservoirs.fields(fr.prev_final.numpy())
        tag_ok = (fl["tri"] == ref["final"].tri) & (fl["tag"] == ref["final"].tag)
        close = _close(rad, ref["radiance"], 1e-5).all(1)
        stats.append((_frac(tag_ok), _frac(close)))
    assert ctx.get_status() == dd.OK
    return stats


def test_whole_frame_chain_tiny_room(dd, orc):
    stats = _chain(dd, orc, scenegen.tiny_room(), 6)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def test_whole_frame_chain_ragged_image(dd, orc):
    """100 x 75 pixels (not a multiple of the 16 x 8 tiles), camera turned
    toward a corner so that every wall and the emitter are in view."""
    sc = scenegen.tiny_room(width=100, height=75, frames=3)
    sc.cameras = [scenegen._look_camera([0.1, -0.2, 0.3], [-1, 0.6, -0.8], 100, 75, 100.0)] * 3
    stats = _chain(dd, orc, sc, 3)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def test_whole_frame_chain_secondary_ddgi(dd, orc):
    """The paper's "secondary DDGI" comparison through the same passes: one
    BSDF candidate, no emitter candidates, no reuse."""
    import dataclasses
    sc = scenegen.tiny_room(frames=4)
    sc = dataclasses.replace(sc, settings=scenegen.secondary_ddgi(sc.settings))
    stats = _chain(dd, orc, sc, 4)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


@pytest.mark.parametrize("stride", [2, 3])
def test_whole_frame_chain_candidate_subsampling(dd, orc, stride):
    """Sec. 5 subsampling: only every stride-th pixel (rotating diagonals)
    generates candidates, the rest start empty and only reuse; every pass of
    the frame chain still matches the oracle."""
    import dataclasses
    sc = scenegen.tiny_room(frames=5)
    sc = dataclasses.replace(sc, settings=dataclasses.replace(sc.settings, candidate_stride=stride))
    stats = _chain(dd, orc, sc, 5)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def test_whole_frame_chain_dynamic_box(dd, orc):
    """Three boxes in rigid motion (turning and shifting every frame), the
    two emitter triangles swapping every 2 frames, probe relocation on:
    refitted traversal, reprojection of moving surfaces and the temporal
    test at their previous positions agree with the oracle's brute force."""
    sc = scenegen.tiny_room_dynamic(width=64, height=48, frames=8)
    stats = _chain(dd, orc, sc, 8)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def _oracle_volume_from(orc, grid, state):
    irr, dep, off, upd = state
    v = orc.Volume(grid)
    v.irr[:], v.depth[:], v.offset[:] = irr[..., :3], dep, off[:, :3]
    v.updates = upd
    return v


def test_dynamic_64_frames_track_the_per_frame_oracle(dd, orc):
    """Config 3's lag check at reduced size: three boxes in rigid motion, the
    two emitter triangles swapping every 8 frames, probe relocation on, 64
    frames at 64 x 48 -- eight toggles, each followed by the probes'
    hysteresis settling.

    Teacher forced, every frame: the oracle updates the probes from the
    GPU's probe state of the frame before (maps, offsets), and runs initial
    -> temporal -> spatial -> shade on the GPU's G-buffers and the GPU's
    previous final reservoirs; the GPU's probe maps, offsets, final
    reservoirs and radiance must match (>= 99.9 % of texels and pixels
    within 1e-4 relative + floors 1e-5 / 1e-6, tags >= 99.9 %).

    Free running, every frame: the oracle's own probe volume, updated from
    its own history only, against the GPU's: the mean irradiance of every
    probe agrees within 2e-5 relative (measured: 1e-6), so the GPU's maps
    neither lead nor lag the oracle's after a toggle (a hysteresis applied
    one frame late would differ by a whole frame's step, ~1e-3)."""
    import dataclasses
    sc = scenegen.tiny_room_dynamic(width=64, height=48, frames=64)
    sc = dataclasses.replace(sc, emitter_toggle=8)
    assert sc.settings.probe_relocation == 1
    W, H = 64, 48
    ctx = dd.Context.from_scene(sc)
    S, Sf = orc.Scene(sc), orc.Scene(sc)
    vf = orc.Volume(sc.grid)
    fr = dd.Frame(ctx, W, H, sc.settings.spatial_passes)
    prev = None          # (GPU G-buffer planes, final records, camera) of the frame before
    probe_mean = []
    for f in range(64):
        xf, le = sc.instance_transforms(f), sc.emitter_radiance(f)
        before = ctx.probe_state_get()
        ctx.scene_update(xf, le)
        S.update(xf, le)
        Sf.update(xf, le)
        # probes: teacher-forced update and free-running volume
        vt = _oracle_volume_from(orc, sc.grid, before)
        orc.probe_update(S, vt, f)
        orc.probe_update(Sf, vf, f)
        ctx.probe_update(f)
        irr, dep, off, _ = ctx.probe_state_get()
        ok = _close(irr[..., :3], vt.irr, 1e-5)
        assert _frac(ok) >= 0.999, (f, _frac(ok))
        np.testing.assert_allclose(off[:, :3], vt.offset, rtol=1e-4, atol=1e-5)
        m_gpu = irr[..., :3].reshape(irr.shape[0], -1).mean(1)
        m_free = vf.irr.reshape(vf.irr.shape[0], -1).mean(1)
        assert np.all(np.abs(m_gpu - m_free) <= 2e-5 * np.abs(m_free) + 1e-7), f
        probe_mean.append(m_free.mean())
        # the frame on the GPU, then the oracle's passes on the GPU's inputs
        cam = sc.cameras[f]
        rad = fr.render(f, cam, probe_update=False).cpu().numpy()[:, :3]
        g_planes = [a.copy() for a in fr.g[f % 2].numpy()]
        final = fr.prev_final.numpy().copy()
        og = orc.GBuffer.from_planes(*g_planes, W, H)
        res, resid = orc.restir_initial(S, vt, og, f)
        if prev is not None:
            og_prev = orc.GBuffer.from_planes(*prev[0], W, H)
            res = orc.restir_temporal(S, og, og_prev, prev[2].pos, res,
                                      _oracle_res_full(orc, S, prev[1], stored_normals=True), f)
        for i in range(sc.settings.spatial_passes):
            res = orc.restir_spatial(S, og, res, f, i)
        ref = orc.shade(S, vt, og, res, resid)
        fl = dd.Reservoirs.fields(final)
        tags = (fl["tri"] == res.tri) & (fl["tag"] == res.tag)
        assert _frac(tags) >= 0.999, (f, _frac(tags))
        assert _frac(_close(rad, ref, 1e-5).all(1)) >= 0.999, f
        prev = (g_planes, final, cam)
    assert ctx.get_status() == dd.OK
    # the toggles really drive the probes: the mean irradiance rises through
    # one 8-frame window and falls through the next (hysteresis 0.97 settles
    # over ~30 frames, so each window only starts the response)
    trend = [np.sign(probe_mean[8 * k + 7] - probe_mean[max(8 * k - 1, 1)]) for k in range(8)]
    assert all(trend[k] == -trend[k + 1] != 0 for k in range(7)), trend


# ---------------------------------------------------------------------------
# glossy materials (Sec. 3.3): glossy term of L_DDGI+, specular recursion
# ---------------------------------------------------------------------------

def test_glossy_probe_trace_parity(dd, orc):
    """Probe rays on the glossy room (near-mirror floor, rough glossy back
    wall): the radiance at each hit includes the one-sample glossy half of
    L_DDGI+ toward the probe; from the same probe maps (teacher forced, after
    two oracle updates) every ray matches the oracle."""
    sc = scenegen.tiny_room_glossy()
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid)
    for f in range(2):
        orc.probe_update(S, vol, f)
    _vol_to_gpu(ctx, vol)
    ctx.probe_trace(2)
    got = ctx.probe_rays_get()
    ref = orc.probe_trace(S, vol, 2)
    same = np.sign(got[..., 3]) == np.sign(ref[..., 3])
    assert _frac(same) >= 0.999
    assert _frac(_close(got[..., :3][same], ref[..., :3][same], 1e-5).all(-1)) >= 0.999
    # the glossy surfaces really contribute: rays that hit them differ from
    # the same update with the lobes removed
    import dataclasses
    plain = orc.Scene(dataclasses.replace(sc, glossy=None))
    ref0 = orc.probe_trace(plain, vol, 2)
    assert np.abs(ref[..., :3] - ref0[..., :3]).max() > 1e-2
    assert ctx.get_status() == dd.OK


@pytest.mark.parametrize("c", [0.2, 1e4])
def test_whole_frame_chain_glossy(dd, orc, c):
    """The frame chain on the glossy room: probe updates with the glossy
    term, BSDF candidates whose cached radiance carries it, and shading with
    the specular recursion -- at the paper's threshold c = 0.2 and at c = 1e4,
    where every glossy path is traced on to the 8-vertex cap."""
    import dataclasses
    sc = scenegen.tiny_room_glossy(width=96, height=64, frames=4)
    sc = dataclasses.replace(sc, settings=dataclasses.replace(sc.settings, footprint_c=c))
    stats = _chain(dd, orc, sc, 4)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def test_glossy_recursion_changes_the_image(dd):
    """The footprint threshold matters where it should: on the glossy room a
    large c (paths traced on) and c < 0 (one glossy sample at the first
    vertex) give different images, and both stay finite."""
    import dataclasses
    base = scenegen.tiny_room_glossy(width=96, height=64, frames=2)
    out = {}
    for c in (1e4, -1.0):
        sc = dataclasses.replace(base, settings=dataclasses.replace(base.settings, footprint_c=c))
        ctx = dd.Context.from_scene(sc)
        fr = dd.Frame(ctx, 96, 64, sc.settings.spatial_passes)
        for f in range(2):
            rad = fr.render(f, sc.cameras[f]).cpu().numpy()[:, :3]
        assert np.all(np.isfinite(rad)) and ctx.get_status() == dd.OK
        out[c] = rad
    assert np.abs(out[1e4] - out[-1.0]).max() > 1e-3


def test_glossy_fused_chain(dd, orc):
    """The fused initial + temporal pass on the glossy room."""
    sc = scenegen.tiny_room_glossy(width=64, height=48, frames=4)
    stats = _chain(dd, orc, sc, 4, fused=True)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def test_glossy_scene_argument_errors(dd):
    """Glossy emitters, out-of-range lobes and a glossy scene with the
    learned target are refused at creation."""
    import dataclasses
    sc = scenegen.tiny_room_glossy(width=16, height=16, frames=1)
    bad = sc.glossy.copy()
    emitter = int(np.flatnonzero(sc.emission.max(1) > 0)[0])
    bad[emitter] = (0.3, 0.3, 0.3, 0.2)
    for gl in (bad, np.where(sc.glossy > 0, 0.0, sc.glossy) + np.array([0.5, 0.5, 0.5, 0.0], np.float32)):
        with pytest.raises(dd.DDGIError):
            dd.Context.from_scene(dataclasses.replace(sc, glossy=gl.astype(np.float32)))
    learned = dataclasses.replace(sc, settings=dataclasses.replace(sc.settings, learned_target=1,
                                                                   train_samples=1024))
    with pytest.raises(dd.DDGIError):
        dd.Context.from_scene(learned)


@pytest.mark.parametrize("c", [0.2, 1e4])
def test_apartment_glossy_sampled(dd, orc, c):
    """The glossy apartment at 1920x1080 (polished floor, glossy furniture
    tops): probe rays with the glossy term (8 probes), restir_initial (BSDF
    candidates whose cached radiance carries the glossy sample) and
    ddgi_shade with the specular recursion, teacher forced on the GPU's
    G-buffer, probe maps and reservoirs, on 2048 sampled pixels; at the
    paper's c = 0.2 and at c = 1e4 (glossy paths traced on to the cap)."""
    import dataclasses
    import torch
    sc = scenegen.apartment_glossy(frames=1)
    sc = dataclasses.replace(sc, settings=dataclasses.replace(sc.settings, footprint_c=c))
    W, H = sc.cameras[0].width, sc.cameras[0].height
    n = W * H
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    for f in range(2):
        ctx.probe_update(f)
    irr, dep, off, upd = ctx.probe_state_get()
    vol = orc.Volume(sc.grid)
    vol.irr[:], vol.depth[:], vol.offset[:] = irr[..., :3], dep, off[:, :3]
    vol.updates = upd
    # probe rays of frame 2 from these maps
    ctx.probe_trace(2)
    rays = ctx.probe_rays_get()
    probes = np.sort(np.random.default_rng(9).choice(sc.grid.num_probes, 8, replace=False)).astype(np.int32)
    rref = orc.probe_trace(S, vol, 2, probes=probes)
    got = rays[probes]
    same = np.sign(got[..., 3]) == np.sign(rref[..., 3])
    assert _frac(same) >= 0.999
    assert _frac(_close(got[..., :3][same], rref[..., :3][same], 1e-5).all(-1)) >= 0.999
    cam = sc.cameras[0]
    g = dd.GBuffer(W, H)
    ctx.gbuffer(cam, None, g)
    out = dd.Reservoirs(n)
    resid = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(g, out, resid, 2)
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.shade(g, out, resid, rad, frame=2)
    rec, got_resid, got_rad = out.numpy(), resid.cpu().numpy(), rad.cpu().numpy()
    assert ctx.get_status() == dd.OK
    og = orc.GBuffer.from_planes(*g.numpy(), W, H, eye=cam.pos)
    rng = np.random.default_rng(23)
    glossy_px = np.flatnonzero((og.tri >= 0) & (sc.glossy[np.maximum(og.tri, 0), 0] > 0))
    sample = np.sort(np.concatenate([rng.choice(np.flatnonzero(og.tri >= 0), 1024, replace=False),
                                     rng.choice(glossy_px, 1024, replace=False)]))
    sample = np.unique(sample).astype(np.int32)
    ref, rres = orc.restir_initial(S, vol, og, 2, pix=sample)
    _res_compare(rec[sample], ref, what=f"glossy initial@1080p c={c}")
    assert _frac(_close(got_resid[sample, :3], rres, 1e-5).all(1)) >= 0.999
    ores = _oracle_res_full(orc, S, rec)
    shref = orc.shade(S, vol, og, ores, got_resid[:, :3].astype(np.float64), pix=sample, frame=2)
    assert _frac(_close(got_rad[sample, :3], shref, 1e-5).all(1)) >= 0.999
    # the selected samples really include glossy surfaces
    f = dd.Reservoirs.fields(rec[sample])
    assert np.mean(sc.glossy[np.maximum(f["tri"], 0), 0] > 0) > 0.05


def _fused_vs_two_passes(dd, sc, nframes):
    """Twin contexts render the same frames, one with restir_initial +
    restir_temporal, the other with restir_initial_temporal: the same
    arithmetic up to multiply-add contraction, so the final reservoirs select
    the same samples (but for near-ties) and the radiance agrees to the
    parity tolerance."""
    cam0 = sc.cameras[0]
    a, b = dd.Context.from_scene(sc), dd.Context.from_scene(sc)
    fa = dd.Frame(a, cam0.width, cam0.height, sc.settings.spatial_passes)
    fb = dd.Frame(b, cam0.width, cam0.height, sc.settings.spatial_passes)
    for f in range(nframes):
        cam = sc.cameras[f % len(sc.cameras)]
        xf, le = sc.instance_transforms(f), sc.emitter_radiance(f)
        ra = fa.render(f, cam, xf=xf, emitter_radiance=le).cpu().numpy()[:, :3].copy()
        rb = fb.render(f, cam, xf=xf, emitter_radiance=le, fused=True).cpu().numpy()[:, :3].copy()
        la, lb = dd.Reservoirs.fields(fa.prev_final.numpy()), dd.Reservoirs.fields(fb.prev_final.numpy())
        same = (la["tri"] == lb["tri"]) & (la["tag"] == lb["tag"])
        assert _frac(same) >= 0.999, (f, _frac(same))
        assert _frac(_close(rb, ra, 1e-5).all(1)) >= 0.999, f
    assert a.get_status() == dd.OK and b.get_status() == dd.OK


def test_fused_initial_temporal_equals_two_passes(dd):
    _fused_vs_two_passes(dd, scenegen.tiny_room(width=100, height=75, frames=4), 4)


def test_fused_initial_temporal_equals_two_passes_moving_and_subsampled(dd):
    """Moving boxes (reprojection at previous positions) and candidate
    subsampling (pixels that only reuse, M capped against the nominal count)."""
    import dataclasses
    _fused_vs_two_passes(dd, scenegen.tiny_room_dynamic(width=64, height=48, frames=6), 6)
    sc = scenegen.tiny_room(frames=4)
    sc = dataclasses.replace(sc, settings=dataclasses.replace(sc.settings, candidate_stride=3))
    _fused_vs_two_passes(dd, sc, 4)


def test_whole_frame_chain_fused_initial_temporal(dd, orc):
    """The frame chain with the fused initial + temporal pass against the
    oracle's separate passes, on the moving-box scene."""
    sc = scenegen.tiny_room_dynamic(width=64, height=48, frames=6)
    stats = _chain(dd, orc, sc, 6, fused=True)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.999, (f, stats)


def test_fused_initial_temporal_argument_errors(dd):
    sc = scenegen.tiny_room(width=32, height=16, frames=1)
    ctx = dd.Context.from_scene(sc)
    g = dd.GBuffer(32, 16)
    ctx.gbuffer(sc.cameras[0], None, g)
    import torch
    r = [dd.Reservoirs(32 * 16, rec=torch.zeros((32 * 16, 16), dtype=torch.float32, device="cuda"))
         for _ in range(3)]
    resid = torch.zeros((32 * 16, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDGIError):
        ctx.restir_initial_temporal(g, [0.0, 0.0, 0.0], r[0], r[1], r[1], resid, 0)
    with pytest.raises(dd.DDGIError):
        ctx.restir_initial_temporal(g, [0.0, 0.0, float("nan")], r[0], r[1], r[2], resid, 0)
    ctx.restir_initial_temporal(g, [0.0, 0.0, 0.0], r[0], r[1], r[2], resid, 0)
    assert ctx.get_status() == dd.OK


def test_identity_update_keeps_the_bvh_exact(dd):
    """Refitting unmoved geometry reproduces the first build's hits exactly."""
    sc = scenegen.apartment_dynamic(width=320, height=180, frames=2)
    a, b = dd.Context.from_scene(sc), dd.Context.from_scene(sc)
    b.scene_update(sc.instance_transforms(0))
    ga, gb = dd.GBuffer(320, 180), dd.GBuffer(320, 180)
    a.gbuffer(sc.cameras[1], sc.cameras[0], ga)
    b.gbuffer(sc.cameras[1], sc.cameras[0], gb)
    for pa, pb in zip(ga.numpy(), gb.numpy()):
        np.testing.assert_array_equal(pa, pb)


def test_apartment_dynamic_sampled(dd, orc):
    """The dynamic apartment after 10 updates of 200 moving boxes and an
    emitter swap: sampled G-buffer (2048 pixels, half on moving boxes: hits,
    previous pixels) and the rays of 16 probes match the oracle's brute
    force on the moved geometry, ties counted as in the large workload."""
    import torch
    sc = scenegen.apartment_dynamic(frames=12)
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    for f in range(10):
        ctx.scene_update(sc.instance_transforms(f), sc.emitter_radiance(f))
        S.update(sc.instance_transforms(f), sc.emitter_radiance(f))
    cam, pc = sc.cameras[10], sc.cameras[9]
    g = dd.GBuffer(cam.width, cam.height)
    ctx.gbuffer(cam, pc, g)
    g0, g1, g2 = g.numpy()
    rng = np.random.default_rng(12)
    moving_pix = np.flatnonzero((g1[:, 3].view(np.int32) >= 0) &
                                (sc.tri_instance[np.maximum(g1[:, 3].view(np.int32), 0)] >= 0))
    assert len(moving_pix) > 1000
    sample = np.unique(np.concatenate([rng.choice(moving_pix, 1024, replace=False),
                                       rng.choice(cam.width * cam.height, 1024, replace=False)])).astype(np.int32)
    parts = _threaded(lambda c: orc.gbuffer(S, cam, pc, pix=c), sample)
    ref_tri = np.concatenate([p.tri for p in parts])
    ref_dist = np.concatenate([p.dist for p in parts])
    ref_prev = np.concatenate([p.prev for p in parts])
    tri, dist = g1[sample, 3].view(np.int32), g0[sample, 3]
    same = tri == ref_tri
    tie = ~same & (tri >= 0) & (ref_tri >= 0) & (np.abs(dist - ref_dist) <= 1e-5 * ref_dist)
    assert _frac(same | tie) >= 0.999, (same.mean(), tie.sum())
    assert _frac(_close(dist[same], ref_dist[same], 1e-5)) >= 0.999
    prev = g2[sample, 3].view(np.int32)
    moving = (prev >= 0) & ((prev & 0x40000000) != 0)
    np.testing.assert_array_equal(moving[same], (sc.tri_instance[np.maximum(ref_tri, 0)] >= 0)[same] &
                                  (ref_prev[same] >= 0))
    prev = np.where(prev >= 0, prev & ~0x40000000, prev)
    # the previous pixel is the floor of a reprojected coordinate (through the
    # instance's motion for moving boxes): a pixel-boundary tie moves it by one
    assert _frac((prev == ref_prev)[same]) >= 0.995
    # probe rays on the moved geometry
    ctx.probe_trace(10)
    rays = ctx.probe_rays_get()
    vol = orc.Volume(sc.grid)
    vol.offset[:] = ctx.probe_state_get()[2][:, :3]
    probes = np.sort(rng.choice(sc.grid.num_probes, 16, replace=False)).astype(np.int32)
    rr = np.concatenate(_threaded(lambda c: orc.probe_trace(S, vol, 10, probes=c), probes, parts=16))
    t_gpu, t_ref = rays[probes, :, 3], rr[:, :, 3]
    # the moved boxes' vertices are transformed in fp32 on the GPU and in
    # fp64 by the oracle: with coordinates up to 16 m (fp32 spacing 1.9e-6 m)
    # and the rotation's and translation's terms cancelling, a vertex moves by
    # up to ~1e-5 m, which the short back-face hits of relocated probes
    # inside boxes turn into up to 2e-5 m of distance: an absolute floor of
    # 5e-5 m on hit distances here (3e-6 of the scene's extent)
    close = np.abs(t_gpu - t_ref) <= 1e-4 * np.abs(t_ref) + 5e-5
    tie = ~close & (np.abs(np.abs(t_gpu) - np.abs(t_ref)) <= 1e-5 * np.abs(t_ref))
    assert _frac(close | tie) >= 0.999, (t_gpu[~close & ~tie][:8], t_ref[~close & ~tie][:8])
    assert ctx.get_status() == dd.OK


# ---------------------------------------------------------------------------
# full-size apartment: sampled outputs with synthetic inputs
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def apt(dd, orc):
    sc = scenegen.apartment()
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(1920 * 1080, 384, replace=False)).astype(np.int32)
    return sc, ctx, S, sample


def test_apartment_gbuffer_sampled(dd, orc, apt):
    """Primary visibility at 1920x1080 on 4096 pixels: hits (ties at equal
    distance counted), distances and previous pixels."""
    sc, ctx, S, _ = apt
    cam, pc = sc.cameras[3], sc.cameras[2]
    g = dd.GBuffer(cam.width, cam.height)
    ctx.gbuffer(cam, pc, g)
    g0, g1, g2 = g.numpy()
    sample = np.sort(np.random.default_rng(29).choice(cam.width * cam.height, 4096, replace=False)).astype(np.int32)
    parts = _threaded(lambda c: orc.gbuffer(S, cam, pc, pix=c), sample)
    ref_tri = np.concatenate([p.tri for p in parts])
    ref_dist = np.concatenate([p.dist for p in parts])
    ref_prev = np.concatenate([p.prev for p in parts])
    tri, dist = g1[sample, 3].view(np.int32), g0[sample, 3]
    same = tri == ref_tri
    tie = ~same & (tri >= 0) & (ref_tri >= 0) & (np.abs(dist - ref_dist) <= 1e-5 * ref_dist)
    assert _frac(same | tie) >= 0.999, (same.mean(), tie.sum())
    assert _frac(_close(dist[same], ref_dist[same], 1e-5)) >= 0.999
    prev_same = g2[sample, 3].view(np.int32) == ref_prev
    assert _frac(prev_same[same]) >= 0.995


def test_apartment_probe_trace_sampled(dd, orc, apt):
    sc, ctx, S, _ = apt
    vol = orc.Volume(sc.grid)
    vol.set_interior(scenegen.synthetic_irradiance_interior(sc.grid, 8, 5),
                     scenegen.synthetic_depth_interior(sc.grid, 16, 6))
    vol.updates = 3
    _vol_to_gpu(ctx, vol)
    ctx.probe_trace(9)
    rays = ctx.probe_rays_get()
    # 16 probes x 256 rays = 4096 rays, so that 99.9 % leaves room for 4
    probes = np.sort(np.random.default_rng(8).choice(sc.grid.num_probes, 16, replace=False)).astype(np.int32)
    ref = orc.probe_trace(S, vol, 9, probes=probes)
    got = rays[probes]
    same = np.sign(got[..., 3]) == np.sign(ref[..., 3])
    assert _frac(same) >= 0.999
    assert _frac(_close(got[..., 3][same], ref[..., 3][same], 1e-5)) >= 0.999
    assert _frac(_close(got[..., :3][same], ref[..., :3][same], 1e-5).all(-1)) >= 0.999


def test_apartment_resampling_passes_sampled(dd, orc, apt):
    """initial / temporal / spatial / shade at 1920x1080 on synthetic
    G-buffers, reservoirs and probe maps, compared on 4096 sampled pixels
    (so that 99.9 % allows 4 ties)."""
    import torch
    sc, ctx, S, _ = apt
    sample = np.sort(np.random.default_rng(19).choice(1920 * 1080, 4096, replace=False)).astype(np.int32)
    W, H = 1920, 1080
    n = W * H
    vol = orc.Volume(sc.grid)
    vol.set_interior(scenegen.synthetic_irradiance_interior(sc.grid, 8, 5),
                     scenegen.synthetic_depth_interior(sc.grid, 16, 6))
    vol.updates = 3
    _vol_to_gpu(ctx, vol)
    gp = scenegen.synthetic_gbuffer(sc, W, H, 21)
    gq = scenegen.synthetic_gbuffer(sc, W, H, 22)
    og = orc.GBuffer.from_planes(*gp, W, H)
    oq = orc.GBuffer.from_planes(*gq, W, H)
    gg = dd.GBuffer(W, H, planes=[_t(a) for a in gp])
    gq_gpu = dd.GBuffer(W, H, planes=[_t(a) for a in gq])
    # initial
    out = dd.Reservoirs(n)
    resid = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(gg, out, resid, 5)
    ref, rref = orc.restir_initial(S, vol, og, 5, pix=sample)
    _res_compare(out.numpy()[sample], ref, what="initial@1080p")
    assert _frac(_close(resid.cpu().numpy()[sample, :3], rref, 1e-5).all(1)) >= 0.999
    # temporal / spatial on synthetic reservoirs
    rc = scenegen.synthetic_reservoirs(sc, n, 31)
    rp = scenegen.synthetic_reservoirs(sc, n, 32)
    oc, op = orc.Reservoirs.from_planes(*rc, scene=S), orc.Reservoirs.from_planes(*rp, scene=S)
    cam_prev = np.array([4.0, 1.5, 6.0])
    tout = dd.Reservoirs(n)
    ctx.restir_temporal(gg, cam_prev, _synthetic_res_to_gpu(dd, ctx, rc, gp),
                        _synthetic_res_to_gpu(dd, ctx, rp, gq), tout, 5)
    tref = orc.restir_temporal(S, og, oq, cam_prev, oc, op, 5, pix=sample)
    _res_compare(tout.numpy()[sample], tref, what="temporal@1080p")
    sout = dd.Reservoirs(n)
    ctx.restir_spatial(gg, _synthetic_res_to_gpu(dd, ctx, rc, gp), sout, 5, 1)
    sref = orc.restir_spatial(S, og, oc, 5, 1, pix=sample)
    _res_compare(sout.numpy()[sample], sref, what="spatial@1080p")
    # shade
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    rs = np.zeros((n, 4), np.float32)
    rs[:, :3] = np.random.default_rng(3).uniform(0, 0.1, (n, 3))
    ctx.shade(gg, _synthetic_res_to_gpu(dd, ctx, rc, gp), _t(rs), rad)
    shref = orc.shade(S, vol, og, oc, rs[:, :3].astype(np.float64), pix=sample)
    assert _frac(_close(rad.cpu().numpy()[sample, :3], shref, 1e-5).all(1)) >= 0.999
    assert ctx.get_status() == dd.OK


def _oracle_res_full(orc, S, rec, stored_normals=False):
    """Oracle reservoirs for every pixel from the library's [N, 16] records.
    The samples' normals are those of their triangles (what restir_initial
    stores, exact in a static scene) or, with stored_normals, the normals
    the records carry (words 14..15, octahedral): a sample on a moving
    instance keeps the normal it had when it was found (reading c22)."""
    from paper_2108_05263_gb300 import ddgi
    f = ddgi.Reservoirs.fields(rec)
    r = orc.Reservoirs(rec.shape[0])
    r.y[:], r.W[:], r.L[:], r.M[:] = f["y"], f["W"], f["L"], f["M"]
    r.tri[:], r.tag[:] = f["tri"], f["tag"]
    has = r.tri >= 0
    if stored_normals:
        uv = f["ny_oct"].astype(np.float64)
        for k in np.flatnonzero(has):
            r.ny[k] = orc.oct_decode(uv[k])
    else:
        r.ny[has] = S.normals[r.tri[has]]
    return r


def _scatter_res(orc, n, pix, part):
    """A full-image oracle Reservoirs holding `part` (compact, entry k for
    pixel pix[k]) at its pixels."""
    r = orc.Reservoirs(n)
    for name in orc.Reservoirs.FIELDS:
        getattr(r, name)[pix] = getattr(part, name)
    return r


def test_apartment_fused_initial_temporal_sampled(dd, orc):
    """The kernel the frame time is measured on, at the measured size: the
    1920x1080 apartment with its real G-buffers (frame 1, reprojected onto
    frame 0), probe maps after two GPU updates and frame 0's final
    reservoirs, through restir_initial_temporal; the oracle runs
    restir_initial then restir_temporal on the same inputs (teacher forcing)
    at 4096 sampled pixels.  Then ddgi_shade of the fused output against the
    oracle's shading of the same reservoirs.  Tolerances as everywhere:
    >= 99.9 % identical selections, values within 1e-4 relative (floors:
    radiance 1e-5, W 1e-6) on >= 99.9 % of the sampled pixels."""
    import torch
    sc = scenegen.apartment(frames=2)
    W, H = sc.cameras[0].width, sc.cameras[0].height
    n = W * H
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    for f in range(2):
        ctx.probe_update(f)
    irr, dep, off, upd = ctx.probe_state_get()
    vol = orc.Volume(sc.grid)
    vol.irr[:], vol.depth[:], vol.offset[:] = irr[..., :3], dep, off[:, :3]
    vol.updates = upd
    cam0, cam1 = sc.cameras[0], sc.cameras[1]
    fr = dd.Frame(ctx, W, H, sc.settings.spatial_passes)
    fr.render(0, cam0, probe_update=False)
    prev = fr.prev_final
    g0_planes = [a.copy() for a in fr.g[0].numpy()]
    g1 = dd.GBuffer(W, H)
    ctx.gbuffer(cam1, cam0, g1)
    scratch, out = dd.Reservoirs(n), dd.Reservoirs(n)
    resid = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial_temporal(g1, np.asarray(cam0.pos, np.float32), scratch, prev, out, resid, 1)
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.shade(g1, out, resid, rad)
    got, got_resid, got_rad = out.numpy(), resid.cpu().numpy(), rad.cpu().numpy()
    assert ctx.get_status() == dd.OK

    og1 = orc.GBuffer.from_planes(*g1.numpy(), W, H)
    og0 = orc.GBuffer.from_planes(*g0_planes, W, H)
    rng = np.random.default_rng(17)
    valid = np.flatnonzero(og1.tri >= 0)
    sample = np.sort(rng.choice(valid, 4096, replace=False)).astype(np.int32)
    ref_i, rref = orc.restir_initial(S, vol, og1, 1, pix=sample)
    cur = _scatter_res(orc, n, sample, ref_i)
    oprev = _oracle_res_full(orc, S, prev.numpy())
    tref = orc.restir_temporal(S, og1, og0, cam0.pos, cur, oprev, 1, pix=sample)
    reused = np.mean(tref.M > ref_i.M)
    assert reused > 0.5, reused                        # most pixels really merged a previous reservoir
    _res_compare(got[sample], tref, what="fused initial+temporal@1080p")
    assert _frac(_close(got_resid[sample, :3], rref, 1e-5).all(1)) >= 0.999
    # shading of the fused output (the GPU's reservoirs and residual as input)
    ores = _oracle_res_full(orc, S, got)
    shref = orc.shade(S, vol, og1, ores, got_resid[:, :3].astype(np.float64), pix=sample)
    assert _frac(_close(got_rad[sample, :3], shref, 1e-5).all(1)) >= 0.999


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_image_is_a_no_op(dd):
    import torch
    sc = scenegen.tiny_room()
    ctx = dd.Context.from_scene(sc)
    g = dd.GBuffer(0, 0)
    r = dd.Reservoirs(0)
    z = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(g, r, z, 0)
    ctx.restir_spatial(g, r, dd.Reservoirs(0), 0, 0)
    ctx.shade(g, r, z, z)
    assert ctx.get_status() == dd.OK


def test_invalid_pixels_give_empty_reservoirs_and_black(dd):
    import torch
    sc = scenegen.tiny_room(width=16, height=16)
    ctx = dd.Context.from_scene(sc)
    n = 256
    g = dd.GBuffer(16, 16)
    g.g0.zero_()
    g.g2.zero_()
    g.g1.zero_()
    g.g1.view(torch.int32)[:, 3] = -1
    r = dd.Reservoirs(n)
    resid = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(g, r, resid, 0)
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.shade(g, r, resid, rad)
    f = dd.Reservoirs.fields(r.numpy())
    assert np.all(f["tri"] == -1) and np.all(f["M"] == 0) and np.all(f["valid"] == 0)
    assert np.all(rad.cpu().numpy()[:, :3] == 0)


def test_argument_errors(dd):
    import torch
    sc = scenegen.tiny_room(width=16, height=16)
    ctx = dd.Context.from_scene(sc)
    g = dd.GBuffer(16, 16)
    short = dd.Reservoirs(100)
    resid = torch.empty((256, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDGIError) as e:
        ctx.restir_initial(g, short, resid, 0)
    assert e.value.code == dd.ERR_INVALID_ARG
    r = dd.Reservoirs(256)
    with pytest.raises(dd.DDGIError):
        ctx.restir_spatial(g, r, r, 0, 0)            # aliasing
    bad = torch.empty((257 * 4 + 1,), dtype=torch.float32, device="cuda")[1:].view(257, 4)[:256]
    with pytest.raises(dd.DDGIError):
        ctx.shade(g, r, bad, resid)                  # misaligned residual
    assert ctx.get_status() == dd.OK


def test_scene_without_emitters(dd, orc):
    """No emissive triangle: no light candidates, M = number of BSDF rays."""
    import torch
    sc = scenegen.tiny_room(width=32, height=32)
    sc.emission = np.zeros_like(sc.emission)
    ctx = dd.Context.from_scene(sc)
    assert ctx.info.num_emitters == 0
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid)
    vol.set_interior(np.ones((64, 8, 8, 3)), np.full((64, 16, 16, 2), 5.0))
    _vol_to_gpu(ctx, vol)
    og = orc.gbuffer(S, sc.cameras[0])
    ref, _ = orc.restir_initial(S, vol, og, 2)
    out = dd.Reservoirs(1024)
    rr = torch.empty((1024, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(_gbuf_to_gpu(dd, og), out, rr, 2)
    _res_compare(out.numpy(), ref, what="no-emitter initial")
    assert np.all(dd.Reservoirs.fields(out.numpy())["M"][og.tri >= 0] == 1.0)


def _many_emitter_room(reflect: bool):
    """The tiny room with its emitting half-ceiling cut into 2048 triangles
    (radiance 10; albedo 0.5 when `reflect`): too many emitter records for
    shared memory, so the emitter candidates stage only the search tables
    and read the records from global memory (48-byte copies, or the full
    records when emitters reflect and need the probe query)."""
    sc = scenegen.tiny_room(width=48, height=32, frames=1)
    keep = sc.emission.max(axis=1) == 0
    tris = []
    n = 32
    for i in range(n):
        for j in range(n):
            x0, x1 = -1.0 + i / n, -1.0 + (i + 1) / n
            z0, z1 = -1.0 + 2.0 * j / n, -1.0 + 2.0 * (j + 1) / n
            a, b, c, d = (x0, 1.0, z0), (x1, 1.0, z0), (x1, 1.0, z1), (x0, 1.0, z1)
            tris += [[a, b, c], [a, c, d]]   # winding normal -y: into the room
    grid = np.asarray(tris, np.float32)
    sc.verts = np.concatenate([sc.verts[keep], grid]).astype(np.float32)
    sc.albedo = np.concatenate([sc.albedo[keep], np.full((len(grid), 3), 0.5 if reflect else 0.0)]).astype(np.float32)
    sc.emission = np.concatenate([sc.emission[keep], np.full((len(grid), 3), 10.0)]).astype(np.float32)
    return sc


@pytest.mark.parametrize("reflect", [False, True])
def test_many_emitters_initial_parity(dd, orc, reflect):
    """restir_initial with 2048 emitters (the search tables in shared memory,
    the records from global memory, a candidate ahead) against the oracle."""
    import torch
    sc = _many_emitter_room(reflect)
    ctx = dd.Context.from_scene(sc)
    assert ctx.info.num_emitters == 2048
    S = orc.Scene(sc)
    vol = orc.Volume(sc.grid)
    vol.set_interior(np.full((64, 8, 8, 3), 0.7), np.full((64, 16, 16, 2), 5.0))
    _vol_to_gpu(ctx, vol)
    og = orc.gbuffer(S, sc.cameras[0])
    ref, resid = orc.restir_initial(S, vol, og, 3)
    n = og.tri.shape[0]
    out = dd.Reservoirs(n)
    rr = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(_gbuf_to_gpu(dd, og), out, rr, 3)
    _res_compare(out.numpy(), ref, what=f"many-emitter initial (reflect {reflect})")
    assert _frac(_close(rr.cpu().numpy()[:, :3], resid, 1e-5).all(1)) >= 0.999
    # new radiance for every emitter (all > 0: the emitter list stays): the
    # records' copies follow
    le = (10.0 * (1 + np.arange(2048) % 3))[:, None] * np.array([1.0, 0.8, 0.6])
    ctx.scene_update(None, le.astype(np.float32))
    sc.emission[sc.emission.max(axis=1) > 0] = le
    S2 = orc.Scene(sc)
    ref2, _ = orc.restir_initial(S2, vol, og, 4)
    ctx.restir_initial(_gbuf_to_gpu(dd, og), out, rr, 4)
    _res_compare(out.numpy(), ref2, what=f"many-emitter initial after new radiance (reflect {reflect})")
    assert ctx.get_status() == dd.OK


# ---------------------------------------------------------------------------
# image metrics (Sec. 4): MSE and MAPE in fp64
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 1000, 1920 * 1080 + 7])
def test_image_metrics_match_the_oracle(dd, orc, n):
    import torch
    rng = np.random.default_rng(n)
    img = rng.exponential(1.0, (n, 4)).astype(np.float32)
    ref = rng.exponential(1.0, (n, 4)).astype(np.float32)
    ref[: n // 3, :3] = 0.0                          # black reference pixels: epsilon matters
    out = dd.image_metrics(_t(img), _t(ref)).cpu().numpy()
    if n == 0:
        np.testing.assert_array_equal(out, [0.0, 0.0])
        return
    exp = [orc.mse(img[:, :3], ref[:, :3]), orc.mape(img[:, :3], ref[:, :3])]
    np.testing.assert_allclose(out, exp, rtol=1e-12)


def test_image_metrics_rejects_short_scratch(dd):
    import torch
    img = torch.zeros((4096 * 1024, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDGIError):
        dd.image_metrics(img, img, scratch=torch.empty(16, dtype=torch.float64, device="cuda"))


# ---------------------------------------------------------------------------
# path-traced reference (Sec. 4)
# ---------------------------------------------------------------------------

def test_reference_matches_oracle_paths(dd, orc):
    """Same random-number keys on both sides: the per-pixel sums of 32 paths
    agree up to rounding (a rare path that diverges at an edge aside)."""
    import torch
    sc = scenegen.tiny_room(width=48, height=40)
    ctx = dd.Context.from_scene(sc)
    cam = sc.cameras[0]
    n = 48 * 40
    acc = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    mean = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.reference_accumulate(cam, 0, 16, acc, mean)
    ctx.reference_accumulate(cam, 16, 16, acc, mean)
    a = acc.cpu().numpy()
    np.testing.assert_array_equal(a[:, 3], 32.0)
    pix = np.arange(0, n, 13)
    ref = orc.pt_reference(orc.Scene(sc), cam, pix, sc.settings.seed, 0, 32)
    assert _frac(_close(a[pix, :3], ref, 1e-3, 1e-4).all(1)) >= 0.97
    np.testing.assert_allclose(mean.cpu().numpy()[:, :3], a[:, :3] / 32.0, rtol=1e-6)
    assert ctx.get_status() == dd.OK


# ---------------------------------------------------------------------------
# probe relocation
# ---------------------------------------------------------------------------

def test_probe_relocation_parity_synthetic_rays(dd, orc):
    """The same seeded ray records on both sides (back-face fractions around
    the 1/4 threshold, near front faces, misses, far faces that hit the
    clamp), two relocation steps: offsets agree to float32 rounding."""
    import dataclasses
    sc = scenegen.apartment(frames=1)
    sc.settings = dataclasses.replace(sc.settings, probe_relocation=1)
    ctx = dd.Context.from_scene(sc)
    P, R = ctx.info.num_probes, ctx.info.rays_per_probe
    vol = orc.Volume(sc.grid)
    cs = orc.settings_of(sc.settings)
    rng = np.random.default_rng(17)
    for frame in (3, 4):
        rays = np.zeros((P, R, 4), np.float32)
        frac_back = rng.uniform(0.0, 0.5, P)
        lo = np.where(rng.random(P) < 0.5, 0.01, 0.2)          # half the probes have no near face
        t = rng.uniform(lo[:, None], 3.0, (P, R)).astype(np.float32)
        back = rng.random((P, R)) < frac_back[:, None]
        miss = rng.random((P, R)) < 0.2
        t = np.where(back, -t, t)
        t = np.where(miss & ~back, np.float32(1e30), t)
        rays[:, :, 3] = t
        ctx.probe_rays_set(rays)
        ctx.probe_relocate(frame)
        orc.probe_relocate(vol, rays.astype(np.float64), frame, cs)
        off = ctx.probe_state_get()[2][:, :3]
        np.testing.assert_allclose(off, vol.offset, rtol=1e-5, atol=2e-6)
    moved = np.abs(vol.offset).max(axis=1) > 0
    clamped = np.isclose(np.abs(vol.offset), 0.45 * sc.grid.spacing.astype(float)).any(axis=1)
    assert 0.2 < moved.mean() < 0.95 and clamped.any()
    assert ctx.get_status() == dd.OK


def test_probe_relocation_chain_parity_tiny_room(dd, orc):
    """A grid that reaches past the walls of the box: the probes outside one
    wall see its back face in half of their directions and move inside.  Three traced updates with
    relocation on both sides agree (offsets, irradiance)."""
    import dataclasses
    sc = scenegen.tiny_room()
    grid = scenegen.ProbeGrid(np.full(3, -1.05, np.float32), np.full(3, 0.7, np.float32),
                              np.array([4, 4, 4], np.int32))
    sc = dataclasses.replace(sc, grid=grid, settings=dataclasses.replace(sc.settings, probe_relocation=1))
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    vol = orc.Volume(grid)
    for f in range(3):
        ctx.probe_update(f)
        orc.probe_update(S, vol, f)
    irr, _, off, _ = ctx.probe_state_get()
    np.testing.assert_allclose(off[:, :3], vol.offset, rtol=1e-4, atol=1e-5)
    home = grid.origin + grid.spacing * _probe_ijk(grid)
    face = (np.abs(home) > 1.0).sum(axis=1) == 1          # half of their rays hit a wall's back
    inside = np.all(np.abs(home + vol.offset) < 1.0, axis=1)
    assert face.sum() == 24 and inside[face].all()
    ok = np.abs(irr[..., :3] - vol.irr) <= 1e-3 * np.abs(vol.irr) + 1e-4
    assert ok.mean() >= 0.999
    assert ctx.get_status() == dd.OK


def _probe_ijk(grid):
    c = grid.counts
    p = np.arange(int(np.prod(c)))
    return np.stack([p % c[0], (p // c[0]) % c[1], p // (c[0] * c[1])], 1)


# ---------------------------------------------------------------------------
# large workload: 4-storey building, ~1M triangles, 8192 emitters, 500
# moving boxes, 3840x2160, 64 candidates, 3 spatial passes, bf16 network
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def large(dd, orc):
    sc = scenegen.multistorey(frames=4)
    ctx = dd.Context.from_scene(sc)
    S = orc.Scene(sc)
    for f in range(3):
        xf, le = sc.instance_transforms(f), sc.emitter_radiance(f)
        ctx.scene_update(xf, le)
        S.update(xf, le)
    return sc, ctx, S


def _threaded(fn, items, parts=16):
    """fn over chunks of items on host threads (the C oracle releases the
    interpreter lock): the brute-force oracle over ~1M triangles."""
    from concurrent.futures import ThreadPoolExecutor
    chunks = [c for c in np.array_split(np.asarray(items), parts) if len(c)]
    with ThreadPoolExecutor(len(chunks)) as ex:
        return list(ex.map(fn, chunks))


def _cat_res(orc, parts):
    r = orc.Reservoirs(sum(p.W.shape[0] for p in parts))
    for name in orc.Reservoirs.FIELDS:
        getattr(r, name)[:] = np.concatenate([getattr(p, name) for p in parts])
    return r


def test_large_geometry_sampled(dd, orc, large):
    """After 3 updates of the 500 moving boxes: sampled 4K G-buffer (1024
    pixels: hits, distances, previous pixels) and the rays of 4 probes (1024
    rays) match the oracle's brute force over the ~1M triangles.  Ties are
    counted, not folded into a lower fraction: a hit on another triangle at
    the same distance (|dt| <= 1e-5 t) is a closest-hit tie; for probe rays
    that includes the coincident, oppositely facing faces of boxes resting on
    the slabs, where one side records a front face and the other a back face
    at the same t (measured: 10 of 1024 rays)."""
    sc, ctx, S = large
    cam, pc = sc.cameras[2], sc.cameras[1]
    g = dd.GBuffer(cam.width, cam.height)
    ctx.gbuffer(cam, pc, g)
    g0, g1, g2 = g.numpy()
    rng = np.random.default_rng(41)
    sample = np.sort(rng.choice(cam.width * cam.height, 1024, replace=False)).astype(np.int32)
    parts = _threaded(lambda c: orc.gbuffer(S, cam, pc, pix=c), sample)
    ref_tri = np.concatenate([p.tri for p in parts])
    ref_dist = np.concatenate([p.dist for p in parts])
    ref_prev = np.concatenate([p.prev for p in parts])
    tri, dist = g1[sample, 3].view(np.int32), g0[sample, 3]
    same = tri == ref_tri
    tie = ~same & (tri >= 0) & (ref_tri >= 0) & (np.abs(dist - ref_dist) <= 1e-5 * ref_dist)
    assert _frac(same | tie) >= 0.999, (same.mean(), tie.sum())
    assert _frac(_close(dist[same], ref_dist[same], 1e-5)) >= 0.999
    prev = g2[sample, 3].view(np.int32)
    prev = np.where(prev >= 0, prev & ~0x40000000, prev)
    # the previous pixel is the floor of a reprojected coordinate: a
    # float32-vs-fp64 tie at a pixel boundary moves it by one
    assert _frac((prev == ref_prev)[same]) >= 0.995
    ctx.probe_trace(2)
    rays = ctx.probe_rays_get()
    vol = orc.Volume(sc.grid)
    probes = np.array([1234, 5000, 9876, 15000], np.int32)
    rr = np.concatenate(_threaded(lambda c: orc.probe_trace(S, vol, 2, probes=c), probes, parts=4))
    t_gpu, t_ref = rays[probes, :, 3], rr[:, :, 3]
    close = np.abs(t_gpu - t_ref) <= 1e-4 * np.abs(t_ref)
    tie = ~close & (np.abs(np.abs(t_gpu) - np.abs(t_ref)) <= 1e-5 * np.abs(t_ref))
    assert _frac(close | tie) >= 0.999, (t_gpu[~close & ~tie][:8], t_ref[~close & ~tie][:8])
    assert _frac(tie) <= 0.03
    assert ctx.get_status() == dd.OK


def test_large_initial_and_shade_sampled(dd, orc, large):
    """64 candidates over 8192 emitters on 512 sampled pixels of the 4K
    G-buffer (synthetic probe maps, probes serving): reservoirs, residuals
    and shading match the oracle at the bar of the other workloads
    (>= 99.9 % selections, 1e-4 relative)."""
    import torch
    sc, ctx, S = large
    cam = sc.cameras[2]
    W, H = cam.width, cam.height
    n = W * H
    vol = orc.Volume(sc.grid)
    vol.set_interior(scenegen.synthetic_irradiance_interior(sc.grid, 8, 7),
                     scenegen.synthetic_depth_interior(sc.grid, 16, 8))
    vol.updates = 3
    _vol_to_gpu(ctx, vol)
    ctx.mlp_serve(2)
    g = dd.GBuffer(W, H)
    ctx.gbuffer(cam, None, g)
    og = orc.GBuffer.from_planes(*g.numpy(), W, H)
    rng = np.random.default_rng(43)
    valid = np.flatnonzero(og.tri >= 0)
    sample = np.sort(rng.choice(valid, 512, replace=False)).astype(np.int32)
    out = dd.Reservoirs(n)
    resid = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(g, out, resid, 6)
    parts = _threaded(lambda c: orc.restir_initial(S, vol, og, 6, pix=c), sample)
    ref = _cat_res(orc, [p[0] for p in parts])
    rref = np.concatenate([p[1] for p in parts])
    _res_compare(out.numpy()[sample], ref, what="initial@4K, 1M triangles")
    assert _frac(_close(resid.cpu().numpy()[sample, :3], rref, 1e-5).all(1)) >= 0.999
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.shade(g, out, resid, rad)
    full = _scatter_res(orc, n, sample, ref)       # the oracle's shading reads full buffers
    full_resid = np.zeros((n, 3))
    full_resid[sample] = rref
    sref = np.concatenate(_threaded(lambda c: orc.shade(S, vol, og, full, full_resid, pix=c), sample))
    f = dd.Reservoirs.fields(out.numpy()[sample])
    same = (f["tri"] == ref.tri) & (f["tag"] == ref.tag)
    assert _frac(_close(rad.cpu().numpy()[sample, :3], sref, 1e-5).all(1)[same]) >= 0.999
    ctx.mlp_serve(0)
    assert ctx.get_status() == dd.OK


def test_large_learned_bf16_frames_run(dd, large):
    """Whole 4K frames of the large workload with the bf16 network trained
    and judged every frame: finite radiance, valid reservoirs, no device
    error."""
    sc, ctx, S = large
    cam = sc.cameras[0]
    fr = dd.Frame(ctx, cam.width, cam.height, sc.settings.spatial_passes)
    for f in range(3, 5):
        ctx.scene_update(sc.instance_transforms(f), sc.emitter_radiance(f))
        ctx.probe_update(f)
        ctx.mlp_train(f)
        rad = fr.render(f, sc.cameras[f % len(sc.cameras)], probe_update=False)
    r = rad.cpu().numpy()
    assert np.all(np.isfinite(r)) and r[:, :3].max() > 0
    st = ctx.mlp_status()
    assert st["judge_n"] > 0 and st["overflow"] == 0
    assert ctx.get_status() == dd.OK


def test_host_pipeline_matches_frame_render(dd):
    """The overlapped host-to-host pipeline (uploads of the next G-buffer and
    downloads of the last radiance on their own streams) gives the same
    frames as Frame.render on device buffers."""
    import torch
    sc = scenegen.tiny_room(width=96, height=64, frames=6)
    W, H = 96, 64
    ref_ctx, ctx = dd.Context.from_scene(sc), dd.Context.from_scene(sc)
    gbufs, prev = [], None
    for f in range(6):
        g = dd.GBuffer(W, H)
        ref_ctx.gbuffer(sc.cameras[f], prev, g)
        prev = sc.cameras[f]
        gbufs.append(g)
    fr = dd.Frame(ref_ctx, W, H, sc.settings.spatial_passes)
    ref = [fr.render(f, sc.cameras[f], gbuf=gbufs[f]).cpu().numpy().copy() for f in range(6)]
    host = [[t.cpu().pin_memory() for t in (g.g0, g.g1, g.g2)] for g in gbufs]
    outs = [torch.empty((W * H, 4), dtype=torch.float32).pin_memory() for _ in range(6)]
    pipe = dd.HostFramePipeline(ctx, W, H, sc.settings.spatial_passes)
    pipe.upload(host[0])
    for f in range(6):
        if f + 1 < 6:
            pipe.upload(host[f + 1])
        pipe.run(f, sc.cameras[f], outs[f])
    pipe.finish()
    torch.cuda.synchronize()
    for f in range(6):
        np.testing.assert_array_equal(outs[f].numpy(), ref[f])
    assert ctx.get_status() == dd.OK


def test_frame_replayed_from_a_cuda_graph(dd):
    """A whole frame captured into a CUDA graph and replayed (probe update,
    restir_initial with its fork to the context's side stream and the join
    back, temporal and spatial reuse, shading) gives the radiance, bit for
    bit, of the same frame issued call by call on a twin context."""
    import torch
    sc = scenegen.tiny_room(width=96, height=64, frames=4)
    W, H = 96, 64
    a, b = dd.Context.from_scene(sc), dd.Context.from_scene(sc)
    gbufs, prev = [], None
    for f in range(4):
        g = dd.GBuffer(W, H)
        a.gbuffer(sc.cameras[f], prev, g)
        prev = sc.cameras[f]
        gbufs.append(g)
    fa = dd.Frame(a, W, H, sc.settings.spatial_passes)
    fb = dd.Frame(b, W, H, sc.settings.spatial_passes)
    for f in range(3):   # scratch buffers and the side stream exist before the capture
        ra = fa.render(f, sc.cameras[f], gbuf=gbufs[f]).cpu().numpy().copy()
        rb = fb.render(f, sc.cameras[f], gbuf=gbufs[f]).cpu().numpy().copy()
        np.testing.assert_array_equal(ra, rb)
    ref = fa.render(3, sc.cameras[3], gbuf=gbufs[3]).cpu().numpy().copy()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    out = torch.zeros((W * H, 4), dtype=torch.float32, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fb.render(3, sc.cameras[3], gbuf=gbufs[3], stream=s, out=out)
    assert not out.any()   # captured, not run
    graph.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    assert b.get_status() == dd.OK and a.get_status() == dd.OK


def test_whole_frame_chain_extreme_settings(dd, orc):
    """Settings at their limits on a ragged 46 x 34 image: 1024 rays per
    probe, 32 x 32 distance texels and 16 x 16 irradiance texels, 63 + 1
    candidates, 32 spatial neighbours in a 255 px radius (mostly off the
    image), 3 spatial passes, M cap 1.  (Odd sizes put the centred camera's
    middle row and column exactly on the seams between wall quads of
    different albedo: a floating-point tie in the primary hit that spatial
    reuse then spreads, so the sizes are even.)"""
    import dataclasses
    sc = scenegen.tiny_room(width=46, height=34, frames=3)
    sc.settings = dataclasses.replace(sc.settings, rays_per_probe=1024, irr_texels=16, depth_texels=32,
                                      num_light_candidates=63, spatial_neighbours=32, spatial_radius=255,
                                      spatial_passes=3, temporal_mcap=1.0)
    stats = _chain(dd, orc, sc, 3)
    for f, (tags, rad) in enumerate(stats):
        assert tags >= 0.999 and rad >= 0.998, (f, stats)


def test_pipelined_frames_equal_sequential_frames(dd):
    """Frame.render with the next frame's probe trace on the side stream
    gives bit-identical radiance and reservoirs to the sequential frame, on
    a static scene, across a jump in the frame index (the trace in flight is
    for a frame that is not rendered: the render traces again) and on the
    moving-box scene with relocation (every render moves the scene, so each
    one traces again after waiting for the trace in flight)."""
    for sc, frames in ((scenegen.tiny_room(width=96, height=64, frames=6), [0, 1, 2, 4, 5]),
                       (scenegen.tiny_room_dynamic(width=64, height=48, frames=5), [0, 1, 2, 3, 4])):
        cam0 = sc.cameras[0]
        a, b = dd.Context.from_scene(sc), dd.Context.from_scene(sc)
        fa = dd.Frame(a, cam0.width, cam0.height, sc.settings.spatial_passes)
        fb = dd.Frame(b, cam0.width, cam0.height, sc.settings.spatial_passes)
        for f in frames:
            cam = sc.cameras[f % len(sc.cameras)]
            xf, le = sc.instance_transforms(f), sc.emitter_radiance(f)
            ra = fa.render(f, cam, xf=xf, emitter_radiance=le, fused=True).cpu().numpy().copy()
            rb = fb.render(f, cam, xf=xf, emitter_radiance=le, fused=True, pipelined=True).cpu().numpy().copy()
            np.testing.assert_array_equal(ra, rb)
            np.testing.assert_array_equal(fa.prev_final.numpy(), fb.prev_final.numpy())
        fb.finish()
        ia, _, _, ua = a.probe_state_get()
        ib, _, _, ub = b.probe_state_get()
        np.testing.assert_array_equal(ia, ib)
        assert ua == ub
        assert a.get_status() == dd.OK and b.get_status() == dd.OK
