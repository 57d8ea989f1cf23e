"""Pins of the learned-form oracle (oracle/mlp.py) to independent
computations: torch's fp64 autograd and Adam, central finite differences,
numpy's sin/cos, and a fit of a known function."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M():
    from oracle import mlp
    return mlp


def _torch_net(M, params):
    layers = []
    for l, (W, b) in enumerate(params):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        layers.append(lin)
        if l < len(params) - 1:
            layers.append(torch.nn.ReLU())
    return torch.nn.Sequential(*layers)


def _batch(M, n=257, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-1, 1, (n, 3))
    nn_ = rng.normal(size=(n, 3))
    nn_ /= np.linalg.norm(nn_, axis=1, keepdims=True)
    x = M.encode(p, nn_, np.full(3, -1.0), 0.5)
    t = rng.uniform(0, 3, (n, 3))
    valid = rng.random(n) > 0.1
    return x, t, valid


def test_encoding_matches_numpy_trig(M):
    p = np.array([[0.0, 0.0, 0.0], [0.25, 0.5, 0.125], [1.0, 0.3, 0.7]])
    n = np.array([[0, 0, 1.0], [0, 1.0, 0], [1.0, 0, 0]])
    x = M.encode(p, n, np.zeros(3), 1.0)
    assert x.shape == (3, 80)
    for a in range(3):
        for k in range(12):
            np.testing.assert_allclose(x[:, 24 * a + 2 * k], np.sin(2 ** k * np.pi * p[:, a]), atol=1e-12)
            np.testing.assert_allclose(x[:, 24 * a + 2 * k + 1], np.cos(2 ** k * np.pi * p[:, a]), atol=1e-12)
    np.testing.assert_array_equal(x[:, 72:75], n)
    np.testing.assert_array_equal(x[:, 75:], 0.0)


def test_forward_matches_torch(M):
    params = M.init_params(3)
    for W, b in params:
        b += np.random.default_rng(1).normal(0, 0.1, b.shape)
    x, _, _ = _batch(M)
    out, _ = M.forward(params, x)
    ref = _torch_net(M, params)(torch.from_numpy(x)).detach().numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_backward_matches_torch_autograd(M):
    params = M.init_params(4)
    x, t, valid = _batch(M)
    out, cache = M.forward(params, x)
    loss, dout = M.rel_l2(out, t, valid)
    grads = M.backward(params, cache, dout)
    net = _torch_net(M, params)
    xt = torch.from_numpy(x)
    pred = net(xt)
    tt, vt = torch.from_numpy(t), torch.from_numpy(valid)
    den = pred.detach() ** 2 + 0.01
    r = torch.where(vt[:, None], (pred - tt) ** 2 / den, torch.zeros_like(pred))
    tl = r.sum() / (vt.sum() * 3)
    tl.backward()
    assert loss == pytest.approx(tl.item(), rel=1e-12)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (gW, gb), lin in zip(grads, lins):
        np.testing.assert_allclose(gW, lin.weight.grad.numpy(), rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(gb, lin.bias.grad.numpy(), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_operand_rounding_matches_torch_autograd_with_rounding_hooks(M, fmt):
    """forward / backward with q (the 16-bit operand precision of the
    tensor-core form) against torch's fp64 autograd where each layer's input
    passes through a rounding function whose backward is the identity and
    each pre-activation's gradient is rounded by a hook: layer inputs and
    deltas rounded, products and sums fp64.  With q = None the rounding must
    vanish (bit-identical to the plain forward / backward)."""
    def q_np(a):
        a = np.asarray(a, np.float64)
        if fmt == "fp16":
            return a.astype(np.float16).astype(np.float64)
        b = a.astype(np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
        return b.astype(np.uint32).view(np.float32).astype(np.float64)

    def q_t(t):
        return torch.from_numpy(q_np(t.detach().numpy()))

    class Round(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            return q_t(a)

        @staticmethod
        def backward(ctx, g):
            return g

    params = M.init_params(6)
    for W, b in params:
        b += np.random.default_rng(2).normal(0, 0.1, b.shape)
    x, t, valid = _batch(M, seed=3)
    out, cache = M.forward(params, x, q=q_np)
    dout = np.where(valid[:, None], 2.0 * (out - t) / (out ** 2 + 0.01), 0.0)
    grads = M.backward(params, cache, dout, q=q_np)
    net = _torch_net(M, params)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    a = torch.from_numpy(x)
    for l, lin in enumerate(lins):
        z = lin(Round.apply(a))
        z.register_hook(lambda g: q_t(g))
        a = torch.relu(z) if l < len(lins) - 1 else z
    np.testing.assert_allclose(out, a.detach().numpy(), rtol=1e-12, atol=1e-12)
    a.backward(torch.from_numpy(dout))
    for (gW, gb), lin in zip(grads, lins):
        np.testing.assert_allclose(gW, lin.weight.grad.numpy(), rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(gb, lin.bias.grad.numpy(), rtol=1e-10, atol=1e-13)
    # rounding really happened, and q = None is the plain fp64 network
    out0, cache0 = M.forward(params, x)
    assert np.abs(out0 - out).max() > 1e-6
    out1, cache1 = M.forward(params, x, q=None)
    np.testing.assert_array_equal(out0, out1)


def test_gradients_match_finite_differences(M):
    params = M.init_params(5)
    x, t, valid = _batch(M, n=64, seed=2)
    out, cache = M.forward(params, x)
    _, dout = M.rel_l2(out, t, valid)
    grads = M.backward(params, cache, dout)
    den = out ** 2 + 0.01          # held constant, as in the loss definition

    def loss_at(ps):
        o, _ = M.forward(ps, x)
        r = np.where(valid[:, None], (o - t) ** 2 / den, 0.0)
        return r.sum() / (valid.sum() * 3)

    rng = np.random.default_rng(7)
    h = 1e-6
    for l in range(5):
        for _ in range(6):
            W, b = params[l]
            i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h
            Wm[i, j] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (loss_at(pp) - loss_at(pm)) / (2 * h)
            assert fd == pytest.approx(grads[l][0][i, j], rel=1e-5, abs=1e-10)


def test_adam_matches_torch(M):
    params = M.init_params(6)
    x, t, valid = _batch(M, n=128, seed=3)
    opt = M.Adam(params)
    net = _torch_net(M, params)
    topt = torch.optim.Adam(net.parameters(), lr=1e-3, betas=(0.9, 0.99), eps=1e-8)
    for _ in range(3):
        out, cache = M.forward(params, x)
        _, dout = M.rel_l2(out, t, valid)
        params = opt.step(params, M.backward(params, cache, dout))
        topt.zero_grad()
        pred = net(torch.from_numpy(x))
        den = pred.detach() ** 2 + 0.01
        vt = torch.from_numpy(valid)
        r = torch.where(vt[:, None], (pred - torch.from_numpy(t)) ** 2 / den, torch.zeros_like(pred))
        (r.sum() / (vt.sum() * 3)).backward()
        topt.step()
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for (W, b), lin in zip(params, lins):
        np.testing.assert_allclose(W, lin.weight.detach().numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(b, lin.bias.detach().numpy(), rtol=1e-9, atol=1e-12)


def test_network_learns_a_smooth_field(M):
    """A known smooth function of position is fitted well below its variance."""
    rng = np.random.default_rng(9)
    p = rng.uniform(0, 1, (2048, 3))
    n = np.tile([0, 0, 1.0], (2048, 1))
    f = np.stack([1 + np.sin(2 * np.pi * p[:, 0]), 1 + p[:, 1] ** 2, 2 - p[:, 2]], 1)
    x = M.encode(p, n, np.zeros(3), 1.0)
    params = M.init_params(11)
    opt = M.Adam(params, lr=3e-3)
    valid = np.ones(len(p), bool)
    first = None
    for it in range(300):
        out, cache = M.forward(params, x)
        loss, dout = M.rel_l2(out, f, valid)
        first = first if first is not None else loss
        params = opt.step(params, M.backward(params, cache, dout))
    assert loss < 0.02 * first


def test_training_targets_without_network_are_emission(M):
    """With a zero network the target is Le(z): 10 toward the emitter, else 0;
    the fraction of emitter targets is the mean cosine-weighted solid angle of
    the emitter seen from the hit points (checked against brute force)."""
    import oracle
    import scenegen
    sc = scenegen.tiny_room()
    S = oracle.Scene(sc)
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in M.init_params(0)]
    lo, scale = M.scene_box(sc.verts)
    y, ny, target, valid = M.training_samples(oracle, S, sc, params, 0, 4096, 1, lo, scale)
    assert valid.mean() > 0.99
    vals = np.unique(np.round(target[valid], 9))
    assert set(vals.tolist()) <= {0.0, 10.0}
    assert 0.0 < (target[valid, 0] > 0).mean() < 0.5


def test_c_network_matches_numpy_network(M):
    """The C oracle's network (used inside its radiance lookup in the learned
    form) agrees with the numpy network pinned to torch above."""
    import oracle
    import scenegen
    sc = scenegen.tiny_room()
    params = M.init_params(21)
    rng = np.random.default_rng(2)
    for W, b in params:
        b += rng.normal(0, 0.2, b.shape)
    flat = np.zeros(18184)
    offs = [0, 5120, 9216, 13312, 17408]
    for l, (W, b) in enumerate(params):
        flat[offs[l]:offs[l] + W.size] = W.reshape(-1)
        flat[17920 + 64 * l:17920 + 64 * l + b.size] = b
    vol = oracle.Volume(sc.grid)
    lo, scale = M.scene_box(sc.verts)
    vol.set_mlp(flat, lo, scale)
    p = rng.uniform(-1, 1, (200, 3))
    n = rng.normal(size=(200, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    ref, _ = M.forward(params, M.encode(p, n, lo, scale))
    np.testing.assert_allclose(oracle.mlp_eval(vol, p, n), ref, rtol=1e-11, atol=1e-12)


def _constant_net(M, c):
    """Zero weights, output bias c: f = c for every input."""
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in M.init_params(0)]
    params[-1][1][:] = c
    return params


def _triangle_of_points(verts, pts):
    """Index of the triangle each point lies on (plane distance and
    barycentric coordinates, computed here in numpy), -1 if none."""
    v0, e1, e2 = verts[:, 0], verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0]
    nrm = np.cross(e1, e2)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    out = np.full(len(pts), -1)
    for k, y in enumerate(pts):
        d = y - v0
        on_plane = np.abs(np.einsum("ij,ij->i", d, nrm)) < 1e-5
        a11, a12, a22 = (e1 * e1).sum(1), (e1 * e2).sum(1), (e2 * e2).sum(1)
        b1, b2 = (d * e1).sum(1), (d * e2).sum(1)
        det = a11 * a22 - a12 * a12
        u, v = (a22 * b1 - a12 * b2) / det, (a11 * b2 - a12 * b1) / det
        inside = on_plane & (u >= -1e-6) & (v >= -1e-6) & (u + v <= 1 + 1e-6)
        if inside.any():
            out[k] = int(np.argmax(inside))
    return out


def test_training_targets_with_a_constant_network(M):
    """A network with zero weights and output bias c predicts f = c at every
    point, so the self-training target of a sample is Le(z) + rho(z) max(c, 0)
    with z the point its cosine bounce hits: 10 where z is on the emitter,
    else the albedo of z's quad times max(c, 0).  With c = (0.3, -0.2, 0.7):
    channel 1 must be exactly 0 (the clamp), and (t_r / 0.3, t_b / 0.7) must
    be the (r, b) albedo of one of the room's quads -- never that of the quad
    y lies on, since a bounce cannot return to its own plane.  Dropping the
    rho(z) factor or the clamp, or using rho(y), fails here."""
    import oracle
    import scenegen
    sc = scenegen.tiny_room()
    S = oracle.Scene(sc)
    c = np.array([0.3, -0.2, 0.7])
    lo, scale = M.scene_box(sc.verts)
    y, ny, target, valid = M.training_samples(oracle, S, sc, _constant_net(M, c), 0, 4096, 1, lo, scale)
    assert valid.mean() > 0.99
    t = target[valid]
    emit = np.all(t == 10.0, axis=1)
    assert 0.0 < emit.mean() < 0.5
    assert np.all(t[~emit, 1] == 0.0)
    alb = sc.albedo.astype(np.float64)
    ytri = _triangle_of_points(sc.verts.astype(np.float64), y[valid])
    assert np.all(ytri >= 0)
    implied = np.stack([t[~emit, 0] / c[0], t[~emit, 2] / c[2]], 1)
    dist = np.abs(implied[:, None, :] - alb[None, :, [0, 2]]).max(2)       # [samples, triangles]
    match = dist < 1e-9
    assert np.all(match.any(1))
    # the matched albedo is never y's own quad's
    own = alb[ytri[~emit]][:, [0, 2]]
    assert np.all(np.abs(implied - own).max(1) > 1e-6)
    # every non-emitting quad seen from the others is hit by some bounce
    assert len(np.unique(np.round(implied, 9), axis=0)) >= 8


def _constant_volume(o, grid, E):
    """Probe maps of constant irradiance E (per channel) with open distance
    maps: the probe query returns E everywhere."""
    v = o.Volume(grid)
    P = int(np.prod(grid.counts))
    depth = np.zeros((P, 16, 16, 2))
    depth[..., 0], depth[..., 1] = 100.0, 1e4
    v.set_interior(np.broadcast_to(np.asarray(E, np.float64), (P, 8, 8, 3)), depth)
    return v


def _judge_inputs(M, sc, n, m, seed):
    """n synthetic samples: points and normals in the room, targets m * X
    with X ~ Exp(1) (positive, heavy-tailed Monte-Carlo noise around m)."""
    rng = np.random.default_rng(seed)
    y = rng.uniform(-0.9, 0.9, (n, 3))
    ny = rng.normal(size=(n, 3))
    ny /= np.linalg.norm(ny, axis=1, keepdims=True)
    target = m * rng.exponential(1.0, (n, 3))
    valid = rng.random(n) > 0.05
    return y, ny, target, valid


def test_judge_counts_only_held_out_samples_and_an_exact_network_wins(M):
    """Samples 16 j + 15 with a valid hit are the held-out set; a network
    that reproduces every target exactly has error 0 and serves."""
    import oracle
    import scenegen
    sc = scenegen.tiny_room()
    lo, scale = M.scene_box(sc.verts)
    y, ny, target, valid = _judge_inputs(M, sc, 4096, 1.0, 1)
    c = np.array([0.4, 0.9, 1.7])
    target[:] = c
    vol = _constant_volume(oracle, sc.grid, math.pi * 2.0)
    s_net, s_probe, cnt, use = M.judge(oracle, vol, _constant_net(M, c), y, ny, target, valid, 64, lo, scale)
    assert cnt == int(valid[15::16].sum())
    assert s_net == 0.0 and s_probe > 0.0 and use


@pytest.mark.parametrize("seed", [2, 3])
def test_judge_weighs_bias_not_the_targets_noise(M, seed):
    """The two errors share a denominator that does not depend on the noisy
    target, so the noise adds the same expected amount to both and the
    verdict follows the bias: against targets m X (X ~ Exp(1), as noisy as
    their mean), an unbiased cache must beat one biased 30 % low, in either
    role.  A denominator built from the target instead (relative error
    against the noisy target) prefers the prediction biased toward zero and
    fails the second case."""
    import oracle
    import scenegen
    sc = scenegen.tiny_room()
    lo, scale = M.scene_box(sc.verts)
    m = np.array([0.8, 0.5, 0.3])
    y, ny, target, valid = _judge_inputs(M, sc, 65536, m, seed)
    # network unbiased, probes 30 % low
    vol = _constant_volume(oracle, sc.grid, math.pi * 0.7 * m)
    s_net, s_probe, _, use = M.judge(oracle, vol, _constant_net(M, m), y, ny, target, valid, 1024, lo, scale)
    assert use and s_net < s_probe
    # network 30 % low, probes unbiased
    vol = _constant_volume(oracle, sc.grid, math.pi * m)
    s_net, s_probe, _, use = M.judge(oracle, vol, _constant_net(M, 0.7 * m), y, ny, target, valid, 1024, lo,
                                     scale)
    assert not use and s_probe < s_net
