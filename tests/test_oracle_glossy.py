"""Pins of the oracle's glossy lobe, glossy L_DDGI+ term and specular shading
recursion (Sec. 3.3, Eq. lddgiplus, the footprint termination) to facts other
than the oracle itself: the normalisation of the GGX distribution, the closed
form of its half-vector CDF, the importance-sampling identity for the density
of reflected directions, the Smith projected-area identity, the mirror limit
of a uniform environment, a hand-computed footprint, and the mirror image of
the emitter that only the recursion can see.  CPU only."""
import dataclasses
import math

import numpy as np
import pytest

import scenegen


@pytest.fixture(scope="module")
def o():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0])
def test_ggx_distribution_is_normalised(o, alpha):
    """The projected distribution of normals integrates to one:
    2 pi int_0^1 D(c) c dc = 1 (trapezoid rule in x = 1 - c on a
    logarithmic grid, which resolves the peak at c = 1)."""
    x = np.concatenate([[0.0], np.geomspace(1e-12, 1.0, 20000)])
    c = 1.0 - x
    f = np.array([o.ggx_D(ci, alpha) * ci for ci in c])
    integral = 2 * math.pi * np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(x))
    assert integral == pytest.approx(1.0, rel=1e-4)


@pytest.mark.parametrize("alpha", [0.05, 0.4])
def test_ggx_half_vectors_follow_the_closed_form_cdf(o, alpha):
    """Half vectors drawn from D(h) (n.h): tan^2 theta has the CDF
    T / (alpha^2 + T), the azimuth is uniform (Kolmogorov-Smirnov)."""
    rng = np.random.default_rng(3)
    nrm = np.array([0.3, 0.8, -0.52])
    nrm /= np.linalg.norm(nrm)
    N = 4000
    t2, ph = np.zeros(N), np.zeros(N)
    ref = np.array([1.0, 0.0, 0.0]) - nrm * nrm[0]
    ref /= np.linalg.norm(ref)
    other = np.cross(nrm, ref)
    for k in range(N):
        h = o.ggx_sample_h(nrm, alpha, rng.random(), rng.random())
        assert abs(np.linalg.norm(h) - 1) < 1e-12
        c = h @ nrm
        t2[k] = (1 - c * c) / (c * c)
        ph[k] = math.atan2(h @ other, h @ ref)
    t2.sort()
    cdf = t2 / (alpha * alpha + t2)
    ks = np.max(np.abs(cdf - (np.arange(N) + 0.5) / N))
    assert ks < 1.63 / math.sqrt(N)                   # 1 % level
    u = np.sort((ph + math.pi) / (2 * math.pi))
    assert np.max(np.abs(u - (np.arange(N) + 0.5) / N)) < 1.63 / math.sqrt(N)


def test_reflected_directions_have_the_stated_density(o):
    """wi is the mirror image of wo about h, and its density is
    D (n.h) / (4 wo.h): importance sampling with that density must
    integrate 1 and cos^2 over the hemisphere to 2 pi and 2 pi / 3."""
    rng = np.random.default_rng(4)
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([math.sin(0.7), 0.0, math.cos(0.7)])
    ks = np.ones(3)
    N = 60000
    s1 = s2 = 0.0
    for _ in range(N):
        r = o.glossy_sample(n, wo, ks, 0.6, rng.random(), rng.random())
        if r is None:
            continue
        wi, wgt, pdf = r
        h = (wi + wo) / np.linalg.norm(wi + wo)
        assert abs(wi @ h - wo @ h) < 1e-12 and abs(np.linalg.norm(wi) - 1) < 1e-12
        s1 += 1.0 / pdf
        s2 += wi[2] ** 2 / pdf
    assert s1 / N == pytest.approx(2 * math.pi, rel=0.02)
    assert s2 / N == pytest.approx(2 * math.pi / 3, rel=0.02)


@pytest.mark.parametrize("theta_o", [0.2, 1.0, 1.4])
def test_smith_masking_projected_area_identity(o, theta_o):
    """For the Smith model the visible microfacet area projected on wo equals
    the macro surface's: G1(wo) int D(h) max(0, wo.h) dh = cos theta_o
    (quadrature over the hemisphere of h)."""
    alpha = 0.5
    wo = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])
    nt, nph = 800, 400
    acc = 0.0
    for i in range(nt):
        t = (i + 0.5) * (math.pi / 2) / nt
        st, ct = math.sin(t), math.cos(t)
        D = o.ggx_D(ct, alpha)
        phis = (np.arange(nph) + 0.5) * 2 * math.pi / nph
        oh = np.maximum(0.0, st * np.cos(phis) * wo[0] + ct * wo[2])
        acc += D * oh.sum() * st * (math.pi / 2 / nt) * (2 * math.pi / nph)
    assert o.ggx_G1(wo[2], alpha) * acc == pytest.approx(wo[2], rel=2e-3)
    assert o.ggx_G1(1.0, alpha) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("theta_o", [0.3, 0.9, 1.3])
def test_sampled_weight_matches_quadrature_of_the_lobe(o, theta_o):
    """The one-sample weight f_g (n.wi) / pdf (an algebraically simplified
    ratio) averages to the lobe's directional albedo, integrated here by
    quadrature over wi from its definition k_s D(h) G1(wo) G1(wi) /
    (4 |n.wo| |n.wi|) times n.wi, h = (wo + wi) / |wo + wi| -- for a rough
    lobe (alpha = 0.4), where neither masking nor the half-vector Jacobian
    is close to 1."""
    alpha = 0.4
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])
    nt, nph = 300, 300
    acc = 0.0
    for i in range(nt):
        t = (i + 0.5) * (math.pi / 2) / nt
        for ph in (np.arange(nph) + 0.5) * 2 * math.pi / nph:
            wi = np.array([math.sin(t) * math.cos(ph), math.sin(t) * math.sin(ph), math.cos(t)])
            h = (wo + wi) / np.linalg.norm(wo + wi)
            f = o.ggx_D(h[2], alpha) * o.ggx_G1(wo[2], alpha) * o.ggx_G1(wi[2], alpha) / (4 * wo[2] * wi[2])
            acc += f * wi[2] * math.sin(t) * (math.pi / 2 / nt) * (2 * math.pi / nph)
    rng = np.random.default_rng(6)
    N = 40000
    w = 0.0
    for _ in range(N):
        r = o.glossy_sample(n, wo, np.ones(3), alpha, rng.random(), rng.random())
        if r is not None:
            w += r[1][0]
    assert w / N == pytest.approx(acc, rel=1.5e-2)


def test_glossy_term_reflects_a_uniform_environment_in_the_mirror_limit(o):
    """Probe maps of constant irradiance E = pi L (open distance maps): the
    one-sample glossy term of Eq. lddgiplus at a near-mirror surface
    (alpha = 0.01, where masking vanishes) must average to k_s L at an
    oblique view, and the diffuse half to rho L -- with the 1/pi reading of
    the normalisation (1/(2 pi) would give half)."""
    sc = scenegen.tiny_room_glossy()
    S = o.Scene(dataclasses.replace(sc, glossy=np.where(sc.glossy[:, 3:] > 0, np.concatenate(
        [sc.glossy[:, :3], np.full((sc.num_tris, 1), 0.01, np.float32)], 1), sc.glossy)))
    Lenv = 2.0
    v = o.Volume(sc.grid)
    depth = np.zeros((64, 16, 16, 2))
    depth[..., 0], depth[..., 1] = 100.0, 1e4
    v.set_interior(np.full((64, 8, 8, 3), math.pi * Lenv), depth)
    floor = int(np.flatnonzero(sc.glossy[:, 3] == 0.05)[0])
    y = sc.verts[floor].astype(np.float64).mean(0)
    frm = y + np.array([0.8, 0.5, 0.0])                # 58 degrees off the normal
    rng = np.random.default_rng(5)
    N = 4000
    u = rng.random((N, 2))
    L = o.radiance(S, v, np.tile(y, (N, 1)), np.full(N, floor, np.int32), np.tile(frm, (N, 1)), u)
    rho, ks = sc.albedo[floor].astype(np.float64), sc.glossy[floor, :3].astype(np.float64)
    np.testing.assert_allclose(L.mean(0), (rho + ks) * Lenv, rtol=2e-3)


def _mirror_setup(o, c):
    """The glossy room with a near-mirror floor (alpha = 0.01), black probe
    maps, x1 on the back wall and y on the floor placed so that the mirror
    direction of y -> x1 points into the emitter (the x < 0 ceiling half)."""
    sc = scenegen.tiny_room_glossy()
    gl = sc.glossy.copy()
    gl[gl[:, 3] == 0.05, 3] = 0.01
    sc = dataclasses.replace(sc, glossy=gl, settings=dataclasses.replace(sc.settings, footprint_c=c))
    S = o.Scene(sc)
    v = o.Volume(sc.grid)                              # black: the probes hold no light
    floor = int(np.flatnonzero(gl[:, 3] == 0.01)[0])
    return sc, S, v, floor


def test_footprint_termination_in_a_hand_case(o):
    """eye (0, 0, 0), x1 = (-0.5, 0, -1) on the back wall (n +z), y =
    (-0.5, -1, -0.5) on the floor: a_0 = |x0 - x1|^2 / (4 pi cos_0) with
    cos_0 = 1 / |x0 - x1|, and a(x1, y) = |x1 - y|^2 / (p_1 cos_2) with
    p_1 = cos_1 / pi the Lambertian density at x1.  The recursion stops at y
    exactly when a(x1, y) > c a_0: two vertices just below that c, three
    (the glossy ray reaches the emitter) just above it."""
    eye, x1, n1, y = np.zeros(3), np.array([-0.5, 0.0, -1.0]), np.array([0, 0, 1.0]), np.array([-0.5, -1.0, -0.5])
    d0 = np.linalg.norm(eye - x1)
    a0 = d0 * d0 / (4 * math.pi * ((eye - x1) @ n1 / d0))
    w1 = (y - x1) / np.linalg.norm(y - x1)
    a1 = np.linalg.norm(y - x1) ** 2 / ((n1 @ w1) / math.pi * abs(w1[1]))
    for c, verts_expected in ((0.999 * a1 / a0, 2), (1.001 * a1 / a0, 3)):
        sc, S, v, floor = _mirror_setup(o, c)
        _, verts = o.shade_radiance(S, v, eye, x1, n1, y, floor, 7, 3)
        assert verts == verts_expected, (c, verts)


def test_recursion_sees_the_mirror_image_of_the_emitter(o):
    """Same scene, black probes: without recursion (c = 0.2, the footprint
    is already large) the mirror floor returns nothing; with it (c large)
    the glossy ray reaches the emitter and the floor returns the emitter's
    mirror image, k_s Le G1 G1 ~ k_s Le = 5 in the mirror limit."""
    eye, x1, n1, y = np.zeros(3), np.array([-0.5, 0.0, -1.0]), np.array([0, 0, 1.0]), np.array([-0.5, -1.0, -0.5])
    sc, S, v, floor = _mirror_setup(o, 0.2)
    L, verts = o.shade_radiance(S, v, eye, x1, n1, y, floor, 7, 3)
    assert verts == 2 and np.all(L == 0.0)
    sc, S, v, floor = _mirror_setup(o, 1e4)
    acc = np.zeros(3)
    for f in range(200):
        L, verts = o.shade_radiance(S, v, eye, x1, n1, y, floor, 7, f)
        assert verts == 3
        acc += L
    np.testing.assert_allclose(acc / 200, 0.5 * 10.0, rtol=0.02)


def test_diffuse_scene_is_unchanged_by_the_glossy_machinery(o):
    """A scene with a glossy table of zeros renders exactly as without one."""
    sc = scenegen.tiny_room(width=24, height=16, frames=2)
    plain = o.Renderer(sc)
    zero = o.Renderer(dataclasses.replace(sc, glossy=np.zeros((sc.num_tris, 4), np.float32)))
    for f in range(2):
        a, b = plain.frame(f)["radiance"], zero.frame(f)["radiance"]
        np.testing.assert_array_equal(a, b)
