"""Oracle of the learned target form -- TEST INFRASTRUCTURE (fp64 numpy).

The network stands in for the probe lookup as the cached radiance of Sec. 3.6
and the end-of-path radiance (the paper names neural radiance caches as an
interchangeable cache, Sec. 2 and Sec. 5): for a surface point y with normal
n it predicts E(y)/pi, so that the reflected indirect radiance is
rho(y) * max(f(y), 0).

* input: frequency encoding of the position normalised to the scene box,
  sin(2^k pi p'_a), cos(2^k pi p'_a) for k = 0..11 and the three axes (72
  values, ordered axis-major, then frequency, then sin / cos), the normal (3)
  and 5 zeros: 80 values;
* 4 hidden layers of 64 ReLU units, a linear 3-channel output (weights and
  biases per layer);
* loss: relative L2, mean over valid samples and channels of
  (f - t)^2 / (sg(f)^2 + 0.01), with the denominator held constant;
* optimiser: Adam (Kingma & Ba 2015) with lr 1e-3, beta (0.9, 0.99), eps 1e-8;
* training samples: rays from the probe centres (spherical Fibonacci set per
  probe under a per-frame rotation) hit y; a cosine-distributed bounce from y
  hits z; the target is Le(z) + rho(z) * max(f(z), 0) when z faces y (0
  otherwise), an unbiased one-bounce estimate of E(y)/pi under the current
  network.
"""
from __future__ import annotations

import math

import numpy as np

N_FREQ = 12
N_IN = 80
N_HIDDEN = 64
N_LAYERS = 5            # 4 hidden + output
N_OUT = 3
PASS_TRAIN_ROT = 9
PASS_TRAIN_BOUNCE = 10
LR, BETA1, BETA2, EPS = 1e-3, 0.9, 0.99, 1e-8
REL_EPS = 0.01


def layer_shapes():
    """(out, in) of every layer."""
    return [(N_HIDDEN, N_IN), (N_HIDDEN, N_HIDDEN), (N_HIDDEN, N_HIDDEN), (N_HIDDEN, N_HIDDEN),
            (N_OUT, N_HIDDEN)]


def scene_box(verts):
    """Normalisation of positions: p' = (p - lo) * scale, scale = 1 / max extent."""
    v = np.asarray(verts, np.float64).reshape(-1, 3)
    lo, hi = v.min(axis=0), v.max(axis=0)
    return lo, 1.0 / float(np.max(hi - lo))


def encode(p, n, lo, scale):
    """[N, 80] inputs for positions p [N, 3] and normals n [N, 3]."""
    p = (np.asarray(p, np.float64) - lo) * scale
    N = p.shape[0]
    x = np.zeros((N, N_IN))
    for a in range(3):
        for k in range(N_FREQ):
            arg = (2.0 ** k) * math.pi * p[:, a]
            x[:, a * 2 * N_FREQ + 2 * k] = np.sin(arg)
            x[:, a * 2 * N_FREQ + 2 * k + 1] = np.cos(arg)
    x[:, 72:75] = n
    return x


def init_params(seed: int):
    """Uniform He-style initialisation, seeded (weights W [out, in], biases b [out])."""
    rng = np.random.default_rng(seed)
    params = []
    for (o, i) in layer_shapes():
        bound = math.sqrt(6.0 / i)
        params.append((rng.uniform(-bound, bound, (o, i)), np.zeros(o)))
    return params


def forward(params, x, q=None):
    """Returns the output [N, 3] and the per-layer inputs / pre-activations.

    q (optional) rounds every product operand the activations supply -- the
    input of each layer -- to the operand precision the tensor-core form
    fixes (fp16 or bf16 operands, Sec. "precision" of the learned form); the
    products and sums stay fp64.  Without q every value is fp64."""
    acts = []
    pre = []
    a = x
    for l, (W, b) in enumerate(params):
        if q is not None:
            a = q(a)
        acts.append(a)
        z = a @ W.T + b
        pre.append(z)
        a = np.maximum(z, 0.0) if l < N_LAYERS - 1 else z
    acts.append(a)
    return a, (acts, pre)


def backward(params, cache, dout, q=None):
    """Gradients (dW, db) of every layer for upstream gradient dout [N, 3].

    q (optional) rounds each layer's delta, the product operand of both of
    its gradient products, as forward's q rounds the layer inputs."""
    acts, pre = cache
    grads = [None] * N_LAYERS
    d = dout if q is None else q(dout)
    for l in range(N_LAYERS - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            # ReLU derivative: 1 where layer l's input (the ReLU output) is > 0
            d = (d @ W) * (acts[l] > 0.0)
            if q is not None:
                d = q(d)
    return grads


def rel_l2(pred, target, valid):
    """Loss and its gradient w.r.t. pred (denominator not differentiated)."""
    valid = np.asarray(valid, bool)
    cnt = max(int(valid.sum()), 1) * N_OUT
    den = pred ** 2 + REL_EPS
    r = np.where(valid[:, None], (pred - target) ** 2 / den, 0.0)
    g = np.where(valid[:, None], 2.0 * (pred - target) / den, 0.0) / cnt
    return float(r.sum() / cnt), g


class Adam:
    def __init__(self, params, lr=LR, b1=BETA1, b2=BETA2, eps=EPS):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[l][j] + (1 - self.b1) * g
                v = self.b2 * self.v[l][j] + (1 - self.b2) * g * g
                self.m[l] = (m, self.m[l][1]) if j == 0 else (self.m[l][0], m)
                self.v[l] = (v, self.v[l][1]) if j == 0 else (self.v[l][0], v)
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
            out.append((new[0], new[1]))
        return out


def predict(params, p, n, lo, scale):
    return forward(params, encode(p, n, lo, scale))[0]


# ---------------------------------------------------------------------------
# training samples (uses the brute-force oracle for ray casting)
# ---------------------------------------------------------------------------

def training_rays(o, scene, grid, frame, samples, seed):
    """Origins and directions of the training rays: samples / P per probe, a
    spherical Fibonacci set rotated by a per-frame random rotation."""
    P = int(np.prod(grid.counts))
    per = samples // P
    R = _rotation(o, seed, frame)
    sf = np.array([o.sf_dir(i, per) for i in range(per)])
    dirs = sf @ R.T
    idx = np.arange(P * per)
    p = idx // per
    i = p % grid.counts[0]
    j = (p // grid.counts[0]) % grid.counts[1]
    k = p // (grid.counts[0] * grid.counts[1])
    org = np.asarray(grid.origin, np.float64) + np.asarray(grid.spacing, np.float64) * np.stack([i, j, k], 1)
    return org, dirs[idx % per]


def _rotation(o, seed, frame):
    u0 = o.rng(seed, 0, frame, PASS_TRAIN_ROT, 0, 0)
    u1 = o.rng(seed, 0, frame, PASS_TRAIN_ROT, 0, 1)
    u2 = o.rng(seed, 0, frame, PASS_TRAIN_ROT, 0, 2)
    a, b = math.sqrt(1 - u0), math.sqrt(u0)
    x, y = a * math.sin(2 * math.pi * u1), a * math.cos(2 * math.pi * u1)
    z, w = b * math.sin(2 * math.pi * u2), b * math.cos(2 * math.pi * u2)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def training_samples(o, S, sc, params, frame, samples, seed, lo, scale):
    """Inputs (y, n_y), targets and validity of the frame's training samples.

    S is an ``oracle.Scene``, sc the ``scenegen.Scene``."""
    org, dirs = training_rays(o, S, sc.grid, frame, samples, seed)
    tri, t = o.intersect(S, org, dirs)
    nrm = S.normals
    N = len(tri)
    valid = tri >= 0
    ny = np.zeros((N, 3))
    ny[valid] = nrm[tri[valid]]
    valid &= np.einsum("ij,ij->i", ny, dirs) < 0.0
    y = org + t[:, None] * dirs
    # cosine bounce at y
    w = np.zeros((N, 3))
    for s in range(N):
        if not valid[s]:
            continue
        u0 = o.rng(seed, s, frame, PASS_TRAIN_BOUNCE, 0, 0)
        u1 = o.rng(seed, s, frame, PASS_TRAIN_BOUNCE, 0, 1)
        r, ph = math.sqrt(u0), 2 * math.pi * u1
        w[s] = o.onb_local_to_world(ny[s], [r * math.cos(ph), r * math.sin(ph), math.sqrt(max(0.0, 1 - u0))])
    tz, t2 = o.intersect(S, y, np.where(valid[:, None], w, [0, 0, 1.0]))
    hitz = valid & (tz >= 0)
    nz = np.zeros((N, 3))
    nz[hitz] = nrm[tz[hitz]]
    face = hitz & (np.einsum("ij,ij->i", nz, w) < 0.0)
    z = y + t2[:, None] * w
    target = np.zeros((N, 3))
    if face.any():
        tzf = tz[face]
        fz = np.maximum(predict(params, z[face], nz[face], lo, scale), 0.0)
        target[face] = sc.emission[tzf] + sc.albedo[tzf] * fz
    return y, ny, target, valid


# ---------------------------------------------------------------------------
# fallback judge (the probes stay the judge of the network's error)
# ---------------------------------------------------------------------------

def judge(o, vol, params, y, ny, target, valid, per, lo, scale):
    """Held-out comparison of the served network with the probe lookup.

    Samples 16 j + 15 are held out of training.  For each held-out sample
    whose ray hit a front face (``valid``), the network predicts
    m = max(f(y), 0) and the probes predict p = E(y) / pi, E the irradiance
    query at y with the view-path bias of Sec. 3.4 taken from the sample's
    probe (the ray's origin, probe index // per).  Per colour channel, both
    squared errors against the one-bounce target t are divided by the same
    denominator 0.5 (m^2 + p^2) + 0.01, which does not depend on t: the
    target's noise then adds the same expected amount to both sums, and their
    difference weighs only the two predictions' biases.  The network serves
    the next queries when its sum is not larger.

    Returns (sum over the network, sum over the probes, count, use network).
    """
    y = np.asarray(y, np.float64)
    ny = np.asarray(ny, np.float64)
    target = np.asarray(target, np.float64)
    held = np.arange(15, len(y), 16)
    held = held[np.asarray(valid)[held]]
    if len(held) == 0:
        return 0.0, 0.0, 0, False
    m = np.maximum(predict(params, y[held], ny[held], lo, scale), 0.0)
    grid_counts = np.asarray(vol.v.counts[:], np.int64)
    origin = np.asarray(vol.v.origin[:], np.float64)
    spacing = np.asarray(vol.v.spacing[:], np.float64)
    pr = np.zeros_like(m)
    for k, i in enumerate(held):
        p = i // per
        ijk = np.array([p % grid_counts[0], (p // grid_counts[0]) % grid_counts[1],
                        p // (grid_counts[0] * grid_counts[1])])
        P = origin + spacing * ijk + vol.offset[p]
        pr[k] = o.biased_query(vol, y[i], ny[i], P) / math.pi
    den = 0.5 * (m * m + pr * pr) + 0.01
    t = target[held]
    s_net = float(np.sum((m - t) ** 2 / den))
    s_probe = float(np.sum((pr - t) ** 2 / den))
    return s_net, s_probe, int(len(held)), bool(s_net <= s_probe)
