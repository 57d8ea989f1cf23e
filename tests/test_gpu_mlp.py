"""GPU <-> oracle parity of the learned target form, through the C ABI.

The GPU network computes with fp16 (or bf16) weights and activations and
fp32 accumulation on the tensor cores, or, in its fp32 debug form, in fp32
on the CUDA cores.  The oracle repeats the computation in fp64 on the same
inputs.  Outputs of the 16-bit forms are compared within 1e-2 relative
(+1e-2 of the mean magnitude; 5e-2 for bf16).  Gradients are compared entry
by entry, against an oracle that rounds the product operands (layer inputs
and deltas) to the kernel's 16-bit format and sums in fp64: every entry
within 1e-2 relative plus half a 16-bit ulp of the layer's largest entry
(2^-12 for fp16, 2^-9 for bf16; the floor covers entries that cancel to
near zero, where a rounding that flips between fp32 and fp64 sums shows);
the fp32 form within 1e-3 relative plus 1e-6 of the layer's largest entry.
Both sides encode the same fp32 normalised position (p - lo) * scale: the
top frequency's gain 2^11 pi turns that position's fp32 rounding into
~4e-4 of feature error, a property of the input, not of the arithmetic
under test."""
import dataclasses

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


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
def M():
    import oracle
    oracle.build()
    from oracle import mlp
    return mlp


def _bf16(x):
    """float32 -> nearest bf16 (round half to even), returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def _to_oracle(flat, M, round16=True, bf16=False):
    """GPU parameter layout -> oracle [(W, b)] (weights rounded to fp16 or
    bf16 as the kernels use them; biases stay fp32)."""
    flat = np.asarray(flat, np.float32)
    offs_w = [0, 5120, 9216, 13312, 17408]
    out = []
    for l, (o, i) in enumerate(M.layer_shapes()):
        W = flat[offs_w[l]:offs_w[l] + o * i].reshape(o, i)
        if round16:
            W = _bf16(W) if bf16 else W.astype(np.float16)
        b = flat[17920 + 64 * l:17920 + 64 * l + o]
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


def _flat(grads):
    """oracle gradients -> GPU layout (W5 padded to 8 rows)."""
    flat = np.zeros(18184)
    offs_w = [0, 5120, 9216, 13312, 17408]
    for l, (gW, gb) in enumerate(grads):
        flat[offs_w[l]:offs_w[l] + gW.size] = gW.reshape(-1)
        flat[17920 + 64 * l:17920 + 64 * l + gb.size] = gb
    return flat


LAYER_OFFS = [0, 5120, 9216, 13312, 17408, 17920, 18184]


def _q16(a):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def _qbf(a):
    return _bf16(np.asarray(a, np.float32)).astype(np.float64)


def _encode32(M, p, n, lo, scale):
    """The network input of positions p as the kernels form it: (p - lo) *
    scale rounded to fp32 at each step, then the exact encoding."""
    pq = ((np.asarray(p, np.float32) - np.float32(lo).astype(np.float32)) * np.float32(scale)).astype(np.float32)
    return M.encode(pq.astype(np.float64), np.asarray(n, np.float64), np.zeros(3), 1.0)


def _oracle_grad(M, flat, s, lo, scale, q=None):
    """Gradient of the mean relative-L2 loss over samples s (library layout)
    for the network with parameters flat; q rounds the weights, biases and
    product operands as the 16-bit tensor-core form does."""
    params = _to_oracle(flat, M, round16=False)
    if q is not None:
        params = [(q(W), q(b)) for W, b in params]
    x = _encode32(M, s[:, 0:3], s[:, 4:7], lo, scale)
    out, cache = M.forward(params, x, q=q)
    valid = s[:, 11] > 0
    t = s[:, 8:11].astype(np.float64)
    # the kernels round the unnormalised delta; the mean's 1 / (3 count) comes after
    dout = np.where(valid[:, None], 2.0 * (out - t) / (out ** 2 + 0.01), 0.0)
    return _flat(M.backward(params, cache, dout, q=q)) / (3 * valid.sum()), params


def _assert_grad_elementwise(g, ref, rel, floor):
    for a, b in zip(LAYER_OFFS[:-1], LAYER_OFFS[1:]):
        err = np.abs(g[a:b] - ref[a:b])
        lim = rel * np.abs(ref[a:b]) + floor * np.abs(ref[a:b]).max()
        bad = np.flatnonzero(err > lim)
        assert bad.size == 0, (a, b, bad[:8] + a, g[a + bad[:8]], ref[a + bad[:8]])


def _fp32_ctx(dd, sc):
    import types
    st = types.SimpleNamespace(**dataclasses.asdict(sc.settings), mlp_fp32=1)
    return dd.Context.from_scene(sc, st)


def _samples(sc, n, seed):
    rng = np.random.default_rng(seed)
    y = rng.uniform(-1, 1, (n, 3))
    nn = rng.normal(size=(n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    t = rng.uniform(0, 3, (n, 3))
    w = (rng.random(n) > 0.1).astype(np.float32)
    s = np.zeros((n, 12), np.float32)
    s[:, 0:3], s[:, 3] = y, 1.0
    s[:, 4:7] = nn
    s[:, 8:11], s[:, 11] = t, w
    return s


def _close_frac(a, b, rel, absf):
    return float(np.mean(np.abs(a - b) <= rel * np.abs(b) + absf))


def test_inference_matches_oracle(dd, M):
    import torch
    sc = scenegen.tiny_room()
    ctx = dd.Context.from_scene(sc)
    params = _to_oracle(ctx.mlp_params(), M)
    lo, scale = M.scene_box(sc.verts)
    rng = np.random.default_rng(3)
    n = 5000
    p = rng.uniform(-1, 1, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    q = np.zeros((n, 8), np.float32)
    q[:, 0:3], q[:, 3], q[:, 4:7] = p, 1.0, nrm
    q[::7, 3] = 0.0                                    # invalid queries
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.mlp_infer(torch.from_numpy(q).cuda(), out)
    got = out.cpu().numpy()
    ref, _ = M.forward(params, M.encode(p, nrm, lo, scale))
    np.testing.assert_array_equal(got[:, 3], q[:, 3])
    ok = q[:, 3] > 0
    assert _close_frac(got[ok, :3], ref[ok], 1e-2, 1e-2 * np.abs(ref).mean()) >= 0.99


def test_gradients_match_oracle(dd, M):
    """fp16 tensor-core gradients, entry by entry (module docstring)."""
    sc = scenegen.tiny_room()
    ctx = dd.Context.from_scene(sc)
    lo, scale = M.scene_box(sc.verts)
    s = _samples(sc, 4096, 5)
    g = ctx.mlp_grad(s)
    ref, _ = _oracle_grad(M, ctx.mlp_params(), s, lo, scale, q=_q16)
    _assert_grad_elementwise(g, ref, 1e-2, 2.0 ** -12)


def test_gradients_of_many_samples_match_oracle(dd, M):
    """40,000 samples (313 tiles of 128, the last one ragged), entry by entry
    against the oracle as above; a second call on the same samples agrees
    with the first to float rounding (the tiles' sums meet in atomics, so
    their order, and the last bits, may differ)."""
    sc = scenegen.tiny_room()
    ctx = dd.Context.from_scene(sc)
    lo, scale = M.scene_box(sc.verts)
    s = _samples(sc, 40000, 9)
    g1 = ctx.mlp_grad(s)
    g2 = ctx.mlp_grad(s)
    np.testing.assert_allclose(g1, g2, rtol=1e-5, atol=1e-7 * np.abs(g1).max())
    ref, _ = _oracle_grad(M, ctx.mlp_params(), s, lo, scale, q=_q16)
    _assert_grad_elementwise(g1, ref, 1e-2, 2.0 ** -12)
    assert ctx.get_status() == dd.OK


def test_fp32_gradients_match_oracle_elementwise(dd, M):
    """The fp32 debug form's gradients against the fp64 oracle, every entry
    within 1e-3 relative plus 1e-6 of its layer's largest entry."""
    sc = scenegen.tiny_room()
    ctx = _fp32_ctx(dd, sc)
    lo, scale = M.scene_box(sc.verts)
    for seed in (5, 7):
        s = _samples(sc, 4096, seed)
        g = ctx.mlp_grad(s)
        ref, _ = _oracle_grad(M, ctx.mlp_params(), s, lo, scale)
        _assert_grad_elementwise(g, ref, 1e-3, 1e-6)
    assert ctx.get_status() == dd.OK


def test_fp32_inference_matches_oracle(dd, M):
    import torch
    sc = scenegen.tiny_room()
    ctx = _fp32_ctx(dd, sc)
    params = _to_oracle(ctx.mlp_params(), M, round16=False)
    lo, scale = M.scene_box(sc.verts)
    rng = np.random.default_rng(3)
    n = 5000
    p = rng.uniform(-1, 1, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    q = np.zeros((n, 8), np.float32)
    q[:, 0:3], q[:, 3], q[:, 4:7] = p, 1.0, nrm
    q[::7, 3] = 0.0
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.mlp_infer(torch.from_numpy(q).cuda(), out)
    got = out.cpu().numpy()
    ref, _ = M.forward(params, _encode32(M, q[:, 0:3], q[:, 4:7], lo, scale))
    np.testing.assert_array_equal(got[:, 3], q[:, 3])
    np.testing.assert_allclose(got[:, :3], ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    assert ctx.get_status() == dd.OK


def test_fp32_adam_step_matches_oracle_elementwise(dd, M):
    """One Adam step of the fp32 form: every parameter whose gradient is
    clear of zero (above 1e-5 of its layer's largest) moves as the oracle's
    Adam moves it, to 1e-6 (lr = 1e-3); parameters with a zero gradient do
    not move; the rest move by at most lr."""
    sc = scenegen.tiny_room()
    ctx = _fp32_ctx(dd, sc)
    p0 = ctx.mlp_params()
    lo, scale = M.scene_box(sc.verts)
    s = _samples(sc, 4096, 6)
    ref_g, _ = _oracle_grad(M, p0, s, lo, scale)
    ctx.mlp_step(s)
    d_gpu = ctx.mlp_params() - p0
    master = _to_oracle(p0, M, round16=False)
    offs = [0, 5120, 9216, 13312, 17408]
    grads = []
    for l, (W, b) in enumerate(master):
        gW = ref_g[offs[l]:offs[l] + W.size].reshape(W.shape)
        gb = ref_g[17920 + 64 * l:17920 + 64 * l + b.size]
        grads.append((gW, gb))
    d_ref = _flat(M.Adam(master).step(master, grads)) - p0
    for a, b in zip(LAYER_OFFS[:-1], LAYER_OFFS[1:]):
        g = np.abs(ref_g[a:b])
        clear = g > 1e-5 * g.max()
        np.testing.assert_allclose(d_gpu[a:b][clear], d_ref[a:b][clear], atol=1e-6, rtol=0)
        np.testing.assert_array_equal(d_gpu[a:b][g == 0], 0.0)
        assert np.abs(d_gpu[a:b]).max() <= 1e-3 * (1 + 1e-5)


def test_adam_step_matches_oracle(dd, M):
    sc = scenegen.tiny_room()
    ctx = dd.Context.from_scene(sc)
    p0 = ctx.mlp_params()
    params16 = _to_oracle(p0, M)
    lo, scale = M.scene_box(sc.verts)
    s = _samples(sc, 4096, 6)
    ctx.mlp_step(s)
    p1 = ctx.mlp_params()
    x = M.encode(s[:, 0:3].astype(np.float64), s[:, 4:7].astype(np.float64), lo, scale)
    out, cache = M.forward(params16, x)
    _, dout = M.rel_l2(out, s[:, 8:11].astype(np.float64), s[:, 11] > 0)
    grads = M.backward(params16, cache, dout)
    master = _to_oracle(p0, M, round16=False)
    opt = M.Adam(master)
    ref = _flat(opt.step(master, grads))
    d_gpu, d_ref = p1 - p0, ref - p0
    live = np.abs(_flat(grads)) > 0
    assert _close_frac(d_gpu[live], d_ref[live], 0.0, 1e-4) >= 0.95
    assert np.abs(d_gpu - d_ref).max() <= 2.1e-3          # at most 2 lr apart (sign of a ~0 gradient)
    np.testing.assert_array_equal(p1[17408 + 3 * 64:17920], 0.0)   # padded output rows stay 0


def test_overflowing_step_is_skipped(dd, M):
    """Dynamic loss scaling: a step whose gradient overflows (one sample's
    target 1e38) leaves the parameters as they were, halves the loss scale
    and reports the overflow; the next, clean step is Adam's first (the
    skipped step does not count in the bias correction) and starts from clean
    gradient buffers, so it equals the oracle's first step."""
    sc = scenegen.tiny_room()
    ctx = dd.Context.from_scene(sc)
    p0 = ctx.mlp_params()
    s = _samples(sc, 4096, 6)
    bad = s.copy()
    k = int(np.flatnonzero(s[:, 11] > 0)[0])
    bad[k, 8:11] = 1e38
    scale0 = ctx.mlp_status()["loss_scale"]
    ctx.mlp_step(bad)
    st = ctx.mlp_status()
    assert st["overflow"] == 1 and st["loss_scale"] == max(scale0 * 0.5, 1.0 / 1024.0)
    np.testing.assert_array_equal(ctx.mlp_params(), p0)
    ctx.mlp_step(s)
    st = ctx.mlp_status()
    assert st["overflow"] == 0 and st["step"] == 2
    p1 = ctx.mlp_params()
    assert np.isfinite(p1).all()
    params16 = _to_oracle(p0, M)
    lo, scale = M.scene_box(sc.verts)
    x = M.encode(s[:, 0:3].astype(np.float64), s[:, 4:7].astype(np.float64), lo, scale)
    out, cache = M.forward(params16, x)
    _, dout = M.rel_l2(out, s[:, 8:11].astype(np.float64), s[:, 11] > 0)
    grads = M.backward(params16, cache, dout)
    master = _to_oracle(p0, M, round16=False)
    ref = _flat(M.Adam(master).step(master, grads))
    d_gpu, d_ref = p1 - p0, ref - p0
    live = np.abs(_flat(grads)) > 0
    assert _close_frac(d_gpu[live], d_ref[live], 0.0, 1e-4) >= 0.95
    assert np.abs(d_gpu - d_ref).max() <= 2.1e-3


def test_training_samples_match_oracle(dd, M):
    import oracle
    sc = scenegen.tiny_room()
    sc.settings = dataclasses.replace(sc.settings, train_samples=4096)
    ctx = dd.Context.from_scene(sc)
    S = oracle.Scene(sc)
    for f in range(2):
        ctx.probe_update(f)
    p0 = ctx.mlp_params()
    ctx.mlp_train(7)
    got = ctx.mlp_samples()
    params = _to_oracle(p0, M)
    lo, scale = M.scene_box(sc.verts)
    y, ny, target, valid = M.training_samples(oracle, S, sc, params, 7, 4096, sc.settings.seed, lo, scale)
    gv = got[:, 3] > 0
    assert np.mean(gv == valid) >= 0.999
    both = gv & valid
    assert _close_frac(got[both, 0:3], y[both], 1e-5, 1e-5) >= 0.999
    np.testing.assert_allclose(got[both, 4:7], ny[both], atol=1e-6)
    assert _close_frac(got[both, 8:11], target[both], 1e-2, 1e-2) >= 0.99
    w = both & (np.arange(4096) % 16 != 15)
    np.testing.assert_array_equal(got[:, 11] > 0, w)
    st = ctx.mlp_status()
    assert st["count"] == w.sum() and st["step"] == 1 and st["overflow"] == 0
    assert st["judge_n"] == (valid & (np.arange(4096) % 16 == 15)).sum()
    assert st["use_mlp"] in (0.0, 1.0)


def test_learned_frame_runs_and_trains(dd, M):
    """Learned target on the tiny room: training lowers the held-out error
    of the network, and frames rendered with it stay finite and error-free."""
    sc = scenegen.tiny_room(frames=24)
    sc.settings = dataclasses.replace(sc.settings, learned_target=1, train_samples=8192, train_ema=0.0)
    ctx = dd.Context.from_scene(sc)
    fr = dd.Frame(ctx, 128, 128, sc.settings.spatial_passes)
    errs = []
    for f in range(24):
        ctx.probe_update(f)
        ctx.mlp_train(f)
        st = ctx.mlp_status()
        errs.append(st["judge_mlp"] / max(st["judge_n"], 1))
        rad = fr.render(f, sc.cameras[f], probe_update=False).cpu().numpy()
        assert np.all(np.isfinite(rad))
    assert np.mean(errs[-4:]) < 0.5 * np.mean(errs[:2])
    assert ctx.get_status() == dd.OK


def test_served_network_is_the_moving_average(dd):
    """After each training call the served weights are a * old + (1 - a) *
    trained, the trained ones being those the Adam steps produced."""
    sc = scenegen.tiny_room()
    sc.settings = dataclasses.replace(sc.settings, learned_target=1, train_samples=4096, train_ema=0.9)
    ctx = dd.Context.from_scene(sc)
    ctx.probe_update(0)
    served = ctx.mlp_params_served()
    np.testing.assert_array_equal(served, ctx.mlp_params())
    for f in range(3):
        ctx.mlp_train(f)
        trained = ctx.mlp_params()
        want = np.float32(0.9) * served + np.float32(0.1) * trained
        served = ctx.mlp_params_served()
        np.testing.assert_allclose(served, want, rtol=1e-6, atol=1e-7)
    assert np.abs(served - trained).max() > 1e-4
    assert ctx.get_status() == dd.OK


def _learned_setup(dd, M):
    import oracle
    sc = scenegen.tiny_room()
    sc.settings = dataclasses.replace(sc.settings, learned_target=1, train_samples=4096)
    ctx = dd.Context.from_scene(sc)
    S = oracle.Scene(sc)
    vol = oracle.Volume(sc.grid)
    for f in range(3):
        oracle.probe_update(S, vol, f)
    irr = np.zeros(vol.irr.shape[:-1] + (4,), np.float32)
    irr[..., :3] = vol.irr
    ctx.probe_state_set(irr, vol.depth.astype(np.float32), np.zeros((vol.P, 4), np.float32), vol.updates)
    # a network with visible output: oracle init with positive output biases
    params = M.init_params(31)
    W5, b5 = params[4]
    params[4] = (W5, b5 + 0.5)
    flat = np.zeros(18184, np.float32)
    offs = [0, 5120, 9216, 13312, 17408]
    for l, (W, b) in enumerate(params):
        flat[offs[l]:offs[l] + W.size] = W.reshape(-1)
        flat[17920 + 64 * l:17920 + 64 * l + b.size] = b
    ctx.mlp_set_params(flat)
    ctx.mlp_serve(1)
    f16 = flat.copy()
    f16[:17920] = flat[:17920].astype(np.float16).astype(np.float32)
    lo, scale = M.scene_box(sc.verts)
    vol.set_mlp(f16.astype(np.float64), lo, scale)
    return sc, ctx, S, vol


def _rec_fields(dd, out):
    return dd.Reservoirs.fields(out.numpy())


def test_learned_initial_and_shade_match_oracle(dd, M):
    import oracle
    import torch
    sc, ctx, S, vol = _learned_setup(dd, M)
    cam = sc.cameras[0]
    g = oracle.gbuffer(S, cam)
    ref, resid = oracle.restir_initial(S, vol, g, 4)
    g0, g1, g2 = g.planes()
    gg = dd.GBuffer(g.width, g.height, planes=[torch.from_numpy(a).cuda() for a in (g0, g1, g2)])
    n = g.tri.shape[0]
    out = dd.Reservoirs(n)
    rr = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.restir_initial(gg, out, rr, 4)
    f = _rec_fields(dd, out)
    same = (f["tri"] == ref.tri) & (f["tag"] == ref.tag)
    assert same.mean() >= 0.99
    ok = same & (ref.tri >= 0)
    assert _close_frac(f["L"][ok], ref.L[ok], 2e-2, 1e-3) >= 0.99
    assert _close_frac(f["W"][ok], ref.W[ok], 2e-2, 1e-6) >= 0.99
    # shade the oracle's reservoirs with the network's fresh query
    rad = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    rec = np.zeros((n, 16), np.float32)
    rec[:, 0:3], rec[:, 3], rec[:, 4:7], rec[:, 7] = ref.y, ref.W, ref.L, ref.M
    rec[:, 8:11], rec[:, 11] = g.nrm, np.where(g.tri >= 0, g.dist, 0.0)
    bits = np.zeros((n, 2), np.uint32)
    bits[:, 0] = ref.tri.astype(np.int64).astype(np.uint32)
    bits[:, 1] = ref.tag
    rec[:, 12:14] = bits.view(np.float32)
    res4 = np.zeros((n, 4), np.float32)
    res4[:, :3] = resid
    rs = dd.Reservoirs(n, rec=torch.from_numpy(rec).cuda())
    ctx.reservoirs_attach_normals(rs)
    ctx.shade(gg, rs, torch.from_numpy(res4).cuda(), rad)
    sref = oracle.shade(S, vol, g, ref, resid)
    assert _close_frac(rad.cpu().numpy()[:, :3], sref, 2e-2, 1e-3) >= 0.99
    assert ctx.get_status() == dd.OK


def _form_error(dd, sc, ref, frames, measure, learned):
    import torch
    cam = sc.cameras[0]
    ctx = dd.Context.from_scene(sc)
    fr = dd.Frame(ctx, cam.width, cam.height, sc.settings.spatial_passes)
    mean = torch.zeros_like(ref, dtype=torch.float64)
    served = []
    for f in range(frames):
        ctx.probe_update(f)
        if learned:
            ctx.mlp_train(f)
        rad = fr.render(f, cam, probe_update=False)
        if f >= frames - measure:
            mean += rad.double()
            if learned:
                served.append(ctx.mlp_status()["use_mlp"])
    assert ctx.get_status() == dd.OK
    m = dd.image_metrics((mean / measure).float().contiguous(), ref).cpu().numpy()
    return float(m[0]), float(m[1]), served


def test_learned_form_has_less_bias_than_probes(dd):
    """The gain of the learned form on the box: the mean of 32 frames after
    256 frames of self-training (the judge deciding who serves) is closer to
    the path-traced reference, in MSE and in MAPE, than the mean of the
    probe form's frames.  Per-frame noise averages out of the mean, so the
    comparison weighs the two radiance caches' bias."""
    import torch
    W = H = 192
    base = scenegen.tiny_room(width=W, height=H, frames=1)
    ctx0 = dd.Context.from_scene(base)
    acc = torch.zeros((W * H, 4), dtype=torch.float64, device="cuda")
    ref = torch.empty((W * H, 4), dtype=torch.float32, device="cuda")
    for k in range(0, 8192, 256):
        ctx0.reference_accumulate(base.cameras[0], k, 256, acc, ref)
    learned = dataclasses.replace(base, settings=dataclasses.replace(
        base.settings, learned_target=1, train_samples=65536))
    mse_p, mape_p, _ = _form_error(dd, base, ref, 256, 32, False)
    mse_l, mape_l, served = _form_error(dd, learned, ref, 256, 32, True)
    assert np.mean(served) >= 0.5
    assert mse_l < 0.9 * mse_p
    assert mape_l < 0.75 * mape_p


def _bf16_ctx(dd):
    sc = scenegen.tiny_room()
    sc.settings = dataclasses.replace(sc.settings, mlp_bf16=1)
    return sc, dd.Context.from_scene(sc)


def test_bf16_inference_matches_oracle(dd, M):
    """bf16 weights and activations (8-bit significand), fp32 accumulation:
    outputs within 5e-2 relative (+5e-2 of the mean magnitude) of the fp64
    oracle on the bf16-rounded weights."""
    import torch
    sc, ctx = _bf16_ctx(dd)
    params = _to_oracle(ctx.mlp_params(), M, bf16=True)
    lo, scale = M.scene_box(sc.verts)
    rng = np.random.default_rng(13)
    n = 5000
    p = rng.uniform(-1, 1, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    q = np.zeros((n, 8), np.float32)
    q[:, 0:3], q[:, 3], q[:, 4:7] = p, 1.0, nrm
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ctx.mlp_infer(torch.from_numpy(q).cuda(), out)
    got = out.cpu().numpy()
    ref, _ = M.forward(params, M.encode(p, nrm, lo, scale))
    assert _close_frac(got[:, :3], ref, 5e-2, 5e-2 * np.abs(ref).mean()) >= 0.99
    assert ctx.get_status() == dd.OK


def test_bf16_gradients_match_oracle(dd, M):
    """bf16 tensor-core gradients, entry by entry (module docstring)."""
    sc, ctx = _bf16_ctx(dd)
    lo, scale = M.scene_box(sc.verts)
    s = _samples(sc, 4096, 15)
    g = ctx.mlp_grad(s)
    ref, _ = _oracle_grad(M, ctx.mlp_params(), s, lo, scale, q=_qbf)
    _assert_grad_elementwise(g, ref, 1e-2, 2.0 ** -9)


def test_bf16_learned_frame_trains(dd):
    """A bf16 learned-target context trains (held-out error falls) and renders
    finite frames."""
    sc = scenegen.tiny_room(frames=16)
    sc.settings = dataclasses.replace(sc.settings, learned_target=1, train_samples=8192, train_ema=0.0,
                                      mlp_bf16=1)
    ctx = dd.Context.from_scene(sc)
    fr = dd.Frame(ctx, 128, 128, sc.settings.spatial_passes)
    errs = []
    for f in range(16):
        ctx.probe_update(f)
        ctx.mlp_train(f)
        st = ctx.mlp_status()
        errs.append(st["judge_mlp"] / max(st["judge_n"], 1))
        rad = fr.render(f, sc.cameras[f], probe_update=False).cpu().numpy()
        assert np.all(np.isfinite(rad))
    assert np.mean(errs[-3:]) < 0.5 * np.mean(errs[:2])
    assert ctx.get_status() == dd.OK


def test_judge_matches_the_oracle_judge(dd, M):
    """The fallback judge (reading c16) against the oracle's judge, given the
    same inputs: the frame's held-out samples and targets, the served network
    after its moving-average blend, and the context's probe maps.  The error
    sums must agree to the network's fp16 tolerance (the probe sum, fp32
    against fp64, far tighter), the held-out count exactly, and the verdict
    wherever the two sums are not within that tolerance of each other."""
    import oracle
    sc = scenegen.tiny_room()
    sc.settings = dataclasses.replace(sc.settings, learned_target=1, train_samples=16384)
    ctx = dd.Context.from_scene(sc)
    lo, scale = M.scene_box(sc.verts)
    per = 16384 // int(np.prod(sc.grid.counts))
    decided = 0
    for f in range(8):
        ctx.probe_update(f)
        ctx.mlp_train(f)
        st = ctx.mlp_status()
        smp = ctx.mlp_samples()
        served = ctx.mlp_params_served()
        irr, dep, off, _ = ctx.probe_state_get()
        vol = oracle.Volume(sc.grid)
        vol.irr[:] = irr[..., :3]
        vol.depth[:] = dep
        vol.offset[:] = off[:, :3]
        params = _to_oracle(served, M)
        # inference rounds the biases to fp16 too (they ride in the weight tile)
        params = [(W, b.astype(np.float16).astype(np.float64)) for W, b in params]
        s_net, s_probe, n, use = M.judge(oracle, vol, params, smp[:, 0:3], smp[:, 4:7], smp[:, 8:11],
                                         smp[:, 3] > 0, per, lo, scale)
        assert st["judge_n"] == n > 0
        assert st["judge_mlp"] == pytest.approx(s_net, rel=1e-2), f
        assert st["judge_probe"] == pytest.approx(s_probe, rel=1e-4), f
        if abs(s_net - s_probe) > 2e-2 * max(s_net, s_probe):
            assert st["use_mlp"] == float(use), (f, s_net, s_probe)
            decided += 1
    assert decided >= 4
    assert ctx.get_status() == dd.OK


def test_fp32_learned_frame_trains(dd):
    """The fp32 debug form serves every network query of a frame (BSDF-hit
    radiance, shading, training targets, the judge) and trains: the held-out
    error falls, frames stay finite."""
    import types
    sc = scenegen.tiny_room(frames=12)
    st = types.SimpleNamespace(**dataclasses.asdict(dataclasses.replace(
        sc.settings, learned_target=1, train_samples=8192, train_ema=0.0)), mlp_fp32=1)
    ctx = dd.Context.from_scene(sc, st)
    fr = dd.Frame(ctx, 128, 128, sc.settings.spatial_passes)
    errs = []
    for f in range(12):
        ctx.probe_update(f)
        ctx.mlp_train(f)
        s = ctx.mlp_status()
        errs.append(s["judge_mlp"] / max(s["judge_n"], 1))
        rad = fr.render(f, sc.cameras[f], probe_update=False).cpu().numpy()
        assert np.all(np.isfinite(rad))
    assert np.mean(errs[-3:]) < 0.5 * np.mean(errs[:2])
    assert ctx.get_status() == dd.OK
