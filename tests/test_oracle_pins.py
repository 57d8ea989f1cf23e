"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each test checks the oracle against a closed form, an invariant, a textbook
special case or an independent brute-force computation, so that a plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.
"""
import dataclasses
import math

import numpy as np
import pytest

import scenegen


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def _custom_scene(base, albedo=None, emission=None, settings=None, verts=None, grid=None):
    return scenegen.Scene(base.name,
                          base.verts if verts is None else np.asarray(verts, np.float32),
                          base.albedo if albedo is None else np.asarray(albedo, np.float32),
                          base.emission if emission is None else np.asarray(emission, np.float32),
                          base.grid if grid is None else grid,
                          base.cameras,
                          settings or base.settings)


def _icosphere(r, subdiv=4):
    """Triangulated sphere of radius r with normals pointing inward."""
    t = (1 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, float) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    tris = [[v[a], v[b], v[c]] for a, b, c in f]
    for _ in range(subdiv):
        nt = []
        for a, b, c in tris:
            ab, bc, ca = [(p + q) / np.linalg.norm(p + q) for p, q in ((a, b), (b, c), (c, a))]
            nt += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        tris = nt
    tris = np.asarray(tris) * r
    # icosahedron faces above are outward-wound; flip to face the centre
    return tris[:, [0, 2, 1], :]


def _rect_form_factor(x0, x1, z0, z1, c):
    """Form factor from a differential area to a parallel rectangle
    [x0,x1] x [z0,z1] at height c above it (signed superposition of the
    corner-rectangle formula, Howell's catalogue)."""
    def corner(a, b):
        A, B = a / c, b / c
        sa, sb = math.sqrt(1 + A * A), math.sqrt(1 + B * B)
        return (A / sa * math.atan(B / sa) + B / sb * math.atan(A / sb)) / (2 * math.pi)
    return corner(x1, z1) - corner(x0, z1) - corner(x1, z0) + corner(x0, z0)


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------

def test_pcg_hash_is_a_permutation_and_uniform(oracle_lib):
    o = oracle_lib
    vals = np.array([o.pcg(i) for i in range(1 << 17)], np.uint64)
    assert len(np.unique(vals)) == len(vals)          # bijection on uint32
    # chi-square of the top 8 bits of the chained key over many pixels
    h = np.array([o.rng_u32(1, p, 3, 0, 5, 2) >> 24 for p in range(1 << 16)])
    cnt = np.bincount(h, minlength=256)
    exp = len(h) / 256
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 5 * math.sqrt(2 * 255)
    u = np.array([o.rng(7, p, 0, 1, 2, 3) for p in range(4096)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(np.round(u * 2 ** 24) == u * 2 ** 24)   # 24-bit grid


# ---------------------------------------------------------------------------
# ray casting
# ---------------------------------------------------------------------------

def test_intersection_axis_rays_hit_walls_at_unit_distance(oracle_lib):
    o = oracle_lib
    sc = o.Scene(scenegen.tiny_room())
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1.]])
    dirs = dirs + 1e-3 * np.array([0.3, 0.2, 0.1])   # stay off the quad seams
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    tri, t = o.intersect(sc, np.zeros((6, 3)), dirs)
    assert np.all(tri >= 0)
    ax = np.argmax(np.abs(dirs), axis=1)
    np.testing.assert_allclose(t, 1.0 / np.abs(dirs[np.arange(6), ax]), rtol=1e-12)
    n = sc.normals[tri]
    assert np.all(np.einsum("ij,ij->i", n, dirs) < 0)   # room walls face inward


def _numpy_closest_hit(verts, o, d, tmin=1e-4):
    """Independent closest hit: plane intersection + same-side edge tests."""
    v0, v1, v2 = verts[:, 0], verts[:, 1], verts[:, 2]
    N = np.cross(v1 - v0, v2 - v0)
    best_t = np.full(len(o), np.inf)
    best_i = np.full(len(o), -1)
    margin = np.zeros(len(o))
    for k in range(len(o)):
        dn = N @ d[k]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.einsum("ij,ij->i", v0 - o[k], N) / dn
        p = o[k] + t[:, None] * d[k]
        s0 = np.einsum("ij,ij->i", np.cross(v1 - v0, p - v0), N)
        s1 = np.einsum("ij,ij->i", np.cross(v2 - v1, p - v1), N)
        s2 = np.einsum("ij,ij->i", np.cross(v0 - v2, p - v2), N)
        nn = np.einsum("ij,ij->i", N, N)
        inside = (s0 >= 0) & (s1 >= 0) & (s2 >= 0) & np.isfinite(t) & (t > tmin)
        if inside.any():
            i = np.flatnonzero(inside)[np.argmin(t[inside])]
            best_t[k], best_i[k] = t[i], i
            margin[k] = min(s0[i], s1[i], s2[i]) / nn[i]
    return best_i, best_t, margin


def test_intersection_matches_independent_brute_force(oracle_lib):
    o = oracle_lib
    ap = scenegen.apartment(width=8, height=8, frames=1)
    sc = o.Scene(ap)
    rng = np.random.default_rng(3)
    n = 96
    org = np.column_stack([rng.uniform(0.5, 15.5, n), rng.uniform(0.2, 2.8, n), rng.uniform(0.5, 11.5, n)])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tri, t = o.intersect(sc, org, d)
    bi, bt, margin = _numpy_closest_hit(ap.verts.astype(np.float64), org, d)
    clear = margin > 1e-9
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(tri[clear], bi[clear])
    np.testing.assert_allclose(t[clear], bt[clear], rtol=1e-9)


def test_emitter_sampling_is_area_proportional(oracle_lib):
    o = oracle_lib
    ap = scenegen.apartment(width=8, height=8, frames=1)
    # scale the panel triangles unevenly so the areas differ
    v = ap.verts.astype(np.float64).copy()
    em = np.flatnonzero(ap.emission.max(1) > 0)
    rng = np.random.default_rng(0)
    for i in em:
        c = v[i].mean(0)
        v[i] = c + (v[i] - c) * rng.uniform(0.5, 1.5)
    v = v.astype(np.float32).astype(np.float64)
    sc = o.Scene(_custom_scene(ap, verts=v))
    area = 0.5 * np.linalg.norm(np.cross(v[em, 1] - v[em, 0], v[em, 2] - v[em, 0]), axis=1)
    assert sc.area_total == pytest.approx(area.sum(), rel=1e-12)
    picks = np.array([o.sample_emitter(sc, o.rng(1, k, 0, 0, 0, 0)) for k in range(1 << 18)])
    assert np.all(np.isin(picks, em))
    cnt = np.array([(picks == i).sum() for i in em])
    exp = area / area.sum() * len(picks)
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    dof = len(em) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


# ---------------------------------------------------------------------------
# probe representation
# ---------------------------------------------------------------------------

def test_octahedral_round_trip(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(1)
    d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:4] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0]]
    for k in range(len(d)):
        uv = o.oct_encode(d[k])
        assert abs(uv[0]) <= 1 and abs(uv[1]) <= 1
        assert abs(uv[0]) + abs(uv[1]) <= 1 + 1e-12 or d[k, 2] < 0
        back = o.oct_decode(uv)
        assert np.linalg.norm(back - d[k]) < 1e-12


def test_texel_centres_round_trip(oracle_lib):
    o = oracle_lib
    for n in (8, 16):
        for j in range(n):
            for i in range(n):
                d = o.texel_dir(i, j, n)
                assert abs(np.linalg.norm(d) - 1) < 1e-14
                uv = o.oct_encode(d)
                np.testing.assert_allclose(uv, [2 * (i + .5) / n - 1, 2 * (j + .5) / n - 1], atol=1e-12)


@pytest.mark.parametrize("n", [8, 16])
def test_border_makes_bilinear_lookup_continuous(oracle_lib, n):
    """A map holding its own texel directions must reproduce any direction by
    bilinear lookup within the discretisation error -- also next to the
    octahedral fold, which only works if the border repeats the right texel."""
    o = oracle_lib
    tile = np.zeros((n + 2, n + 2, 3))
    for j in range(n):
        for i in range(n):
            tile[j + 1, i + 1] = o.texel_dir(i, j, n)
    tile = o.gutter(tile, n)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(5000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    err = np.array([np.linalg.norm(o.bilinear(tile, n, x) - x) for x in d])
    near_fold = np.array([max(abs(o.oct_encode(x))) > 1 - 1.0 / n for x in d])
    bound = 0.6 * (2.0 / n) ** 1 * 1.2
    assert err.max() < bound
    assert err[near_fold].max() < 2 * max(err[~near_fold].max(), 1e-3)


def test_spherical_fibonacci_and_rotation(oracle_lib):
    o = oracle_lib
    for n in (64, 256):
        d = np.array([o.sf_dir(i, n) for i in range(n)])
        np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, atol=1e-14)
        np.testing.assert_allclose(d[:, 2], 1 - (2 * np.arange(n) + 1) / n, atol=1e-14)
        assert np.linalg.norm(d.mean(0)) < 2.0 / n
    Rs = np.array([o.probe_rotation(1, f) for f in range(4096)])
    for R in Rs[:64]:
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
    assert np.abs(Rs.mean(0)).max() < 0.04   # uniform rotations average to 0


def test_orthonormal_basis(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(4)
    ns = rng.normal(size=(200, 3))
    ns /= np.linalg.norm(ns, axis=1, keepdims=True)
    ns[:3] = [[0, 0, 1], [0, 0, -1], [0, 1, 0]]
    for n in ns:
        t = o.onb_local_to_world(n, [1, 0, 0])
        b = o.onb_local_to_world(n, [0, 1, 0])
        z = o.onb_local_to_world(n, [0, 0, 1])
        B = np.array([t, b, z])
        np.testing.assert_allclose(B @ B.T, np.eye(3), atol=1e-12)
        np.testing.assert_allclose(z, n, atol=1e-14)
        assert np.linalg.det(B) == pytest.approx(1.0, abs=1e-12)


# ---------------------------------------------------------------------------
# probe update (Sec. 3.2)
# ---------------------------------------------------------------------------

def _enclosure(L, attenuation=0.0, rays=64):
    base = scenegen.tiny_room()
    T = base.num_tris
    st = dataclasses.replace(base.settings, le_attenuation=attenuation, rays_per_probe=rays)
    return _custom_scene(base, albedo=np.zeros((T, 3)), emission=np.tile(L, (T, 1)), settings=st)


def test_uniform_enclosure_gives_pi_L_after_first_update(oracle_lib):
    o = oracle_lib
    L = np.array([1.0, 2.0, 3.0])
    sc = _enclosure(L)
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    o.probe_update(S, vol, 0)
    inner = vol.irr[:, 1:9, 1:9]
    np.testing.assert_allclose(inner, np.broadcast_to(np.pi * L, inner.shape), rtol=1e-12)
    np.testing.assert_allclose(vol.irr, np.broadcast_to(np.pi * L, vol.irr.shape), rtol=1e-12)


def test_hysteresis_step_response_closed_form(oracle_lib):
    o = oracle_lib
    L1, L2 = np.array([1.0, 1.0, 1.0]), np.array([4.0, 0.5, 2.0])
    sc1, sc2 = _enclosure(L1), _enclosure(L2)
    S1, S2 = o.Scene(sc1), o.Scene(sc2)
    vol = o.Volume(sc1.grid)
    a = sc1.settings.hysteresis
    for u in range(10):
        o.probe_update(S1 if u < 3 else S2, vol, u)
        exp = np.pi * L1 if u < 3 else np.pi * L2 + (np.pi * L1 - np.pi * L2) * a ** (u - 2)
        np.testing.assert_allclose(vol.irr[:, 1:9, 1:9], np.broadcast_to(exp, (64, 8, 8, 3)), rtol=1e-12)


def _sphere_scene(r, L, attenuation):
    base = scenegen.tiny_room()
    v = _icosphere(r)
    T = len(v)
    grid = scenegen.ProbeGrid(np.zeros(3, np.float32), np.ones(3, np.float32), np.ones(3, np.int32))
    st = dataclasses.replace(base.settings, le_attenuation=attenuation, rays_per_probe=256)
    return _custom_scene(base, verts=v, albedo=np.zeros((T, 3)), emission=np.tile(L, (T, 1)),
                         settings=st, grid=grid)


def test_depth_moments_at_sphere_centre(oracle_lib):
    o = oracle_lib
    r = 1.2
    sc = _sphere_scene(r, np.ones(3), 0.0)
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    o.probe_update(S, vol, 0)
    mu = vol.depth[0, 1:17, 1:17, 0]
    mu2 = vol.depth[0, 1:17, 1:17, 1]
    v = sc.verts.astype(np.float64)
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    r_in = np.min(np.abs(np.einsum("ij,ij->i", nrm, v[:, 0])) / np.linalg.norm(nrm, axis=1))
    r_out = np.linalg.norm(v, axis=2).max()
    assert r_in > 0.99 * r
    assert mu.min() >= r_in - 1e-12 and mu.max() <= r_out + 1e-12
    assert np.abs(mu2 - mu * mu).max() < 1e-3 * r * r


def test_le_attenuation_closed_form_in_sphere(oracle_lib):
    """Second update inside a sphere of radius 1.2 around a probe of unit
    cell: the backward mean distance (about 1.2) is clipped to the cell
    boundary 0.5 / max|w|, so each ray's Le is scaled by (t / (t + d))^2."""
    o = oracle_lib
    r, L = 1.2, np.array([2.0, 1.0, 0.5])
    sc = _sphere_scene(r, L, 1.0)
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    o.probe_update(S, vol, 0)
    np.testing.assert_allclose(vol.irr[0, 1:9, 1:9], np.broadcast_to(np.pi * L, (8, 8, 3)), rtol=1e-12)
    o.probe_update(S, vol, 1)
    R = 256
    w = o.probe_ray_dirs(sc.settings.seed, 1, R)
    _, t = o.intersect(S, np.zeros((R, 3)), w)
    d = 0.5 / np.abs(w).max(axis=1)
    att = (t / (t + d)) ** 2
    a = sc.settings.hysteresis
    for j in range(8):
        for i in range(8):
            dt = o.texel_dir(i, j, 8)
            c = np.maximum(w @ dt, 0)
            est = np.pi * L * (c * att).sum() / c.sum()
            np.testing.assert_allclose(vol.irr[0, j + 1, i + 1], a * np.pi * L + (1 - a) * est, rtol=1e-12)


# ---------------------------------------------------------------------------
# probe query (DDGI volume + view-path bias)
# ---------------------------------------------------------------------------

def test_query_of_constant_field_is_that_constant(oracle_lib):
    o = oracle_lib
    sc = scenegen.tiny_room()
    vol = o.Volume(sc.grid)
    rng = np.random.default_rng(5)
    E0 = np.array([0.7, 1.3, 2.1])
    irr = np.broadcast_to(E0, (64, 8, 8, 3))
    depth = scenegen.synthetic_depth_interior(sc.grid, 16, 3).astype(np.float64)
    vol.set_interior(irr, depth)
    for _ in range(300):
        q = rng.uniform(-1.2, 1.2, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        E, sw = o.ddgi_query(vol, q, n)
        assert sw > 0
        np.testing.assert_allclose(E, E0, rtol=1e-12)


def test_query_at_a_probe_returns_its_texels(oracle_lib):
    o = oracle_lib
    sc = scenegen.tiny_room()
    vol = o.Volume(sc.grid)
    vol.set_interior(scenegen.synthetic_irradiance_interior(sc.grid, 8, 1),
                     scenegen.synthetic_depth_interior(sc.grid, 16, 2))
    rng = np.random.default_rng(6)
    for p in [0, 21, 42, 63]:
        i, j, k = p % 4, (p // 4) % 4, p // 16
        P = sc.grid.origin.astype(np.float64) + sc.grid.spacing * np.array([i, j, k])
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        E, _ = o.ddgi_query(vol, P, n)
        np.testing.assert_allclose(E, o.bilinear(vol.irr[p], 8, n), rtol=1e-12)


def test_chebyshev_weight_is_one_inside_the_mean_distance(oracle_lib):
    o = oracle_lib
    sc = scenegen.tiny_room()
    irr = scenegen.synthetic_irradiance_interior(sc.grid, 8, 1)
    rng = np.random.default_rng(7)
    big = np.zeros((64, 16, 16, 2))
    big[..., 0] = 10.0
    v1, v2 = o.Volume(sc.grid), o.Volume(sc.grid)
    b2 = big.copy()
    b2[..., 1] = rng.uniform(0, 50, (64, 16, 16))   # any second moment
    v1.set_interior(irr, big)
    v2.set_interior(irr, b2)
    for _ in range(100):
        q = rng.uniform(-0.9, 0.9, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        np.testing.assert_array_equal(o.ddgi_query(v1, q, n)[0], o.ddgi_query(v2, q, n)[0])


def test_probes_on_the_normal_side_dominate(oracle_lib):
    """Probes the surface faces must outweigh probes behind it: with the
    upper probe layer at E = 1 and the lower at E = 100, an upward-facing
    query halfway between them must stay much closer to 1."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    irr = np.ones((64, 8, 8, 3))
    for p in range(64):
        if (p // 4) % 4 == 1:       # layer j = 1 (y = -0.25) is below the query
            irr[p] = 100.0
    depth = np.zeros((64, 16, 16, 2))
    depth[..., 0], depth[..., 1] = 10.0, 100.0
    v = o.Volume(sc.grid)
    v.set_interior(irr, depth)
    up = o.ddgi_query(v, np.array([0.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))[0][0]
    down = o.ddgi_query(v, np.array([0.0, 0.0, 0.0]), np.array([0.0, -1.0, 0.0]))[0][0]
    assert up < 30.0 and down > 70.0


def test_occluded_probe_is_suppressed(oracle_lib):
    """A probe whose distance map says every surface is 1 cm away (zero
    variance) must contribute almost nothing to a query 25 cm away."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    irr = np.ones((64, 8, 8, 3))
    irr[0] = 100.0
    depth = np.zeros((64, 16, 16, 2))
    depth[..., 0], depth[..., 1] = 10.0, 100.0
    depth_occ = depth.copy()
    depth_occ[0, ..., 0], depth_occ[0, ..., 1] = 0.01, 1e-4
    q = np.array([-0.5, -0.5, -0.5])
    n = np.array([0.0, 1.0, 0.0])
    v_open, v_occ = o.Volume(sc.grid), o.Volume(sc.grid)
    v_open.set_interior(irr, depth)
    v_occ.set_interior(irr, depth_occ)
    assert o.ddgi_query(v_open, q, n)[0][0] > 5.0
    assert o.ddgi_query(v_occ, q, n)[0][0] < 1.0 + 1e-6


def _two_probe_volume(o, E0, E1, mean=100.0, var=0.0):
    """Two probes on the x axis (x = 0 and x = 1; spacings 1, 0.5, 0.7, so the
    smallest is 0.5), each with a constant irradiance map (E0, E1) and a
    constant distance map (mean, mean^2 + var)."""
    grid = scenegen.ProbeGrid(np.zeros(3, np.float32), np.array([1.0, 0.5, 0.7], np.float32),
                              np.array([2, 1, 1], np.int32))
    v = o.Volume(grid)
    irr = np.zeros((2, 8, 8, 3))
    irr[0], irr[1] = E0, E1
    depth = np.zeros((2, 16, 16, 2))
    depth[..., 0], depth[..., 1] = mean, mean * mean + var
    v.set_interior(irr, depth)
    return v


def test_view_path_bias_distance_in_a_hand_case(oracle_lib):
    """Sec. 3.4, reading c4: the query point moves from y toward the previous
    path vertex by min(0.2 x smallest spacing, half the segment).  Two probes
    with open distance maps and a normal perpendicular to the axis that joins
    them weigh the two maps linearly in x (wrap-shading and visibility equal
    for both), so the returned irradiance reveals where the query was taken:
    E = (1 - x) E0 + x E1.  A bias away from the vertex, max in place of min,
    or a distance not scaled by the smallest spacing fails here."""
    o = oracle_lib
    E0, E1 = 1.0, 3.0
    v = _two_probe_volume(o, E0, E1)
    n = np.array([0.0, 1.0, 0.0])
    y = np.array([0.3, 0.0, 0.0])

    def x_of(E):
        np.testing.assert_allclose(E, E[0], rtol=1e-13)
        return (E[0] - E0) / (E1 - E0)

    # far previous vertex: d = 0.2 x 0.5 = 0.1, toward it (+x)
    assert x_of(o.biased_query(v, y, n, [0.9, 0.0, 0.0])) == pytest.approx(0.4, abs=1e-12)
    # near previous vertex (segment 0.12): d = half the segment = 0.06
    assert x_of(o.biased_query(v, y, n, [0.42, 0.0, 0.0])) == pytest.approx(0.36, abs=1e-12)
    # the vertex on the other side (-x): the point moves the other way
    assert x_of(o.biased_query(v, y, n, [-0.5, 0.0, 0.0])) == pytest.approx(0.2, abs=1e-12)
    # a vertex off the axis moves the point along the segment (0.3, 0.4):
    # d = 0.1, of which 0.06 along x; the normal is turned to z so that both
    # probes still see the same wrap-shading term
    E = o.biased_query(v, y, [0.0, 0.0, 1.0], [0.6, 0.4, 0.0])
    assert x_of(E) == pytest.approx(0.3 + 0.1 * 0.6, abs=1e-12)
    # no segment (the vertex is y itself): the plain query at y
    assert x_of(o.biased_query(v, y, n, y)) == pytest.approx(0.3, abs=1e-12)


def test_view_path_bias_keeps_a_thin_wall_from_leaking(oracle_lib):
    """A thin wall at x = 0.5 between the two probes: each probe's distance
    map puts a surface 0.5 m away in every direction (zero variance).  Seen
    from the previous vertex on probe 0's side, the wall's face toward it must
    return probe 0's irradiance alone, and from the other side probe 1's;
    the query exactly on the wall (no bias) mixes the two, which is the leak
    the bias exists to prevent.  Biasing away from the previous vertex picks
    the wrong probe and fails."""
    o = oracle_lib
    E0, E1 = np.array([1.0, 2.0, 3.0]), np.array([30.0, 20.0, 10.0])
    v = _two_probe_volume(o, E0, E1, mean=0.5, var=0.0)
    left = o.biased_query(v, [0.5, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.2, 0.1, 0.0])
    right = o.biased_query(v, [0.5, 0.0, 0.0], [1.0, 0.0, 0.0], [0.8, -0.1, 0.05])
    np.testing.assert_allclose(left, E0, rtol=1e-9)
    np.testing.assert_allclose(right, E1, rtol=1e-9)
    on_wall = o.biased_query(v, [0.5, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.5, 0.0, 0.0])
    frac = (on_wall - E0) / (E1 - E0)                 # 1/7 of the way: weights 1.2 : 0.2
    assert np.all(frac > 0.1) and np.all(frac < 0.9), frac


# ---------------------------------------------------------------------------
# primary visibility
# ---------------------------------------------------------------------------

def test_gbuffer_closed_form_in_tiny_room(oracle_lib):
    o = oracle_lib
    sc = scenegen.tiny_room(width=32, height=32)
    S = o.Scene(sc)
    cam = sc.cameras[0]
    g = o.gbuffer(S, cam, cam)
    W = H = 32
    i, j = np.arange(W * H) % W, np.arange(W * H) // W
    sx = 2 * (i + 0.5) / W - 1
    sy = 1 - 2 * (j + 0.5) / H
    assert np.all(g.tri >= 0)
    np.testing.assert_allclose(g.pos[:, 2], -1.0, atol=1e-12)
    np.testing.assert_allclose(g.dist, np.sqrt(1 + sx ** 2 + sy ** 2), rtol=1e-12)
    np.testing.assert_allclose(g.pos[:, 0], sx, atol=1e-12)
    np.testing.assert_allclose(g.nrm, np.broadcast_to([0, 0, 1.0], g.nrm.shape), atol=1e-12)
    np.testing.assert_array_equal(g.prev, np.arange(W * H))


# ---------------------------------------------------------------------------
# resampling estimator (Sec. 3.1, 3.5, 3.6, Eq. Algorithm)
# ---------------------------------------------------------------------------

def _point_gbuffer(o, S, pts, nrm, rho, cam_pos, width=None):
    n = len(pts)
    width = width or n
    g = o.GBuffer(n, width, n // width)
    tri, t = o.intersect(S, pts + 1e-3 * nrm, -nrm)
    assert np.all(tri >= 0)
    g.pos[:] = pts
    g.nrm[:] = nrm
    g.alb[:] = rho
    g.tri[:] = tri
    g.dist[:] = np.linalg.norm(pts - cam_pos, axis=1)
    g.prev[:] = np.arange(n)
    return g


@pytest.mark.slow
def test_direct_light_estimate_matches_form_factor(oracle_lib):
    """With empty probes, the estimator (candidates + selection + shadow ray)
    must average to the reflected direct light rho * Le * F, F the closed-form
    point-to-rectangle form factor of the ceiling emitter."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    pts = np.array([[x, -1.0, z] for x in (-0.8, -0.3, 0.4) for z in (-0.6, 0.1, 0.7)])
    nrm = np.tile([0.0, 1.0, 0.0], (len(pts), 1))
    rho = np.tile([0.5, 0.6, 0.7], (len(pts), 1))
    g = _point_gbuffer(o, S, pts, nrm, rho, np.zeros(3))
    F = np.array([_rect_form_factor(-1 - p[0], -p[0], -1 - p[2], 1 - p[2], 2.0) for p in pts])
    exp = rho * 10.0 * F[:, None]
    N = 3000
    acc = np.zeros((N, len(pts), 3))
    for f in range(N):
        res, resid = o.restir_initial(S, vol, g, f)
        acc[f] = o.shade(S, vol, g, res, resid)
    mean, sd = acc.mean(0), acc.std(0) / math.sqrt(N)
    assert np.all(np.abs(mean - exp) <= 4 * sd + 1e-9), (mean, exp, sd)


def test_form_factor_formula_against_quadrature():
    """The textbook formula used above, checked by midpoint quadrature."""
    x0, x1, z0, z1, c = -0.7, 0.3, -1.4, 0.6, 2.0
    n = 1500
    xs = x0 + (np.arange(n) + 0.5) * (x1 - x0) / n
    zs = z0 + (np.arange(n) + 0.5) * (z1 - z0) / n
    X, Z = np.meshgrid(xs, zs)
    r2 = X ** 2 + Z ** 2 + c * c
    F = (c * c / (np.pi * r2 ** 2)).sum() * (x1 - x0) * (z1 - z0) / n / n
    assert _rect_form_factor(x0, x1, z0, z1, c) == pytest.approx(F, rel=1e-5)


@pytest.mark.slow
def test_bounded_plus_residual_matches_bsdf_sampling_near_emitter(oracle_lib):
    """Points on a side wall just under the emitter see it at G >> 1: the
    bounded resampled term plus the residual must average to the plain
    cosine-sampled estimate of the same (probe-augmented) transport."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    for f in range(4):
        o.probe_update(S, vol, f)
    pts = np.array([[-1.0, 0.97, -0.5], [-1.0, 0.9, 0.2], [-1.0, 0.8, 0.6]])
    nrm = np.tile([1.0, 0.0, 0.0], (3, 1))
    rho = np.tile([0.6, 0.5, 0.4], (3, 1))
    g = _point_gbuffer(o, S, pts, nrm, rho, np.zeros(3))
    # brute force: cosine-distributed directions, rho * L(y) per sample
    rng = np.random.default_rng(9)
    K = 1 << 17
    ref = []
    for p in range(3):
        u0, u1 = rng.random(K), rng.random(K)
        r, ph = np.sqrt(u0), 2 * np.pi * u1
        loc = np.column_stack([r * np.cos(ph), r * np.sin(ph), np.sqrt(1 - u0)])
        w = np.array([o.onb_local_to_world(nrm[p], l) for l in loc])
        tri, t = o.intersect(S, np.tile(pts[p], (K, 1)), w)
        y = pts[p] + t[:, None] * w
        L = o.radiance(S, vol, y, tri, np.tile(pts[p], (K, 1)))
        L[tri < 0] = 0
        v = rho[p] * L
        ref.append((v.mean(0), v.std(0) / math.sqrt(K)))
    N = 3000
    acc = np.zeros((N, 3, 3))
    for f in range(N):
        res, resid = o.restir_initial(S, vol, g, 100 + f)
        acc[f] = o.shade(S, vol, g, res, resid)
    mean, sd = acc.mean(0), acc.std(0) / math.sqrt(N)
    for p in range(3):
        tol = 4 * np.sqrt(sd[p] ** 2 + ref[p][1] ** 2)
        assert np.all(np.abs(mean[p] - ref[p][0]) <= tol), (p, mean[p], ref[p])


@pytest.mark.slow
def test_temporal_and_spatial_reuse_keep_the_estimate_unbiased(oracle_lib):
    """An 8x8 image whose pixels all see the same floor point: with equal
    target functions, merging reservoirs across pixels and frames must not
    change the expectation (still rho * Le * F)."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    p = np.array([-0.3, -1.0, 0.2])
    n = 64
    cam = np.array([-0.3, 1.0, 0.2])
    g = _point_gbuffer(o, S, np.tile(p, (n, 1)), np.tile([0, 1.0, 0], (n, 1)),
                       np.tile([0.5, 0.5, 0.5], (n, 1)), cam, width=8)
    F = _rect_form_factor(-1 - p[0], -p[0], -1 - p[2], 1 - p[2], 2.0)
    exp = 0.5 * 10.0 * F
    T = 700
    acc = np.zeros((T, 3))
    for k in range(T):
        f0, f1 = 2 * k, 2 * k + 1
        prev, _ = o.restir_initial(S, vol, g, f0)
        prev.M[:] = 5000.0                         # exercises the M cap
        cur, resid = o.restir_initial(S, vol, g, f1)
        tmp = o.restir_temporal(S, g, g, cam, cur, prev, f1)
        assert np.all(tmp.M <= cur.M * (1 + sc.settings.temporal_mcap) + 1e-9)
        res = o.restir_spatial(S, g, tmp, f1, 0)
        acc[k] = o.shade(S, vol, g, res, resid).mean(0)
    mean, sd = acc.mean(0), acc.std(0) / math.sqrt(T)
    assert np.all(np.abs(mean - exp) <= 4 * sd), (mean, exp, sd)


def _constant_volume(o, grid, E):
    """Probe maps of constant irradiance E with open distance maps (the query
    returns E everywhere: pinned by test_query_of_constant_field_is_that_constant)."""
    v = o.Volume(grid)
    P = int(np.prod(grid.counts))
    depth = np.zeros((P, 16, 16, 2))
    depth[..., 0], depth[..., 1] = 100.0, 1e4
    v.set_interior(np.full((P, 8, 8, 3), E, np.float64), depth)
    return v


@pytest.mark.slow
def test_query_caching_adds_no_bias(oracle_lib):
    """Sec. 3.6: reusing a sample with the radiance cached when it was found
    adds noise but no bias.  The 8x8 one-point image of the reuse test above,
    with indirect light: the previous frame's reservoirs were made under a
    probe field of E0 = 1.5 and the current frame's under E1 = 6, so every
    cached wall radiance in a temporally reused sample is stale by a factor
    of 4.  The chain initial -> temporal (M cap active) -> spatial -> shade
    is run with caching on (the library's reading) and off (the target of a
    reused sample re-queried from the current probes); both must average to
    the brute-force one-bounce integral rho_x E[L(y)] under E1 (cosine-
    sampled, 2^17 directions).  Shading with the cached radiance instead of
    a fresh query, or a contribution weight whose target is not the selected
    sample's own, fails here."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    S = o.Scene(sc)
    vol0 = _constant_volume(o, sc.grid, 1.5)
    vol1 = _constant_volume(o, sc.grid, 6.0)
    p = np.array([-0.3, -1.0, 0.2])
    nrm = np.array([0.0, 1.0, 0.0])
    rho = 0.5
    n = 64
    cam = np.array([-0.3, 1.0, 0.2])
    g = _point_gbuffer(o, S, np.tile(p, (n, 1)), np.tile(nrm, (n, 1)),
                       np.tile([rho, rho, rho], (n, 1)), cam, width=8)
    # brute force under the current field
    rng = np.random.default_rng(11)
    K = 1 << 17
    u0, u1 = rng.random(K), rng.random(K)
    r, ph = np.sqrt(u0), 2 * np.pi * u1
    loc = np.column_stack([r * np.cos(ph), r * np.sin(ph), np.sqrt(1 - u0)])
    w = np.array([o.onb_local_to_world(nrm, l) for l in loc])
    tri, t = o.intersect(S, np.tile(p, (K, 1)), w)
    L = o.radiance(S, vol1, p + t[:, None] * w, tri, np.tile(p, (K, 1)))
    L[tri < 0] = 0
    ref, ref_sd = rho * L.mean(0), rho * L.std(0) / math.sqrt(K)
    T = 600
    acc = {"cached": np.zeros((T, 3)), "fresh": np.zeros((T, 3))}
    differ = 0
    for k in range(T):
        f0, f1 = 2 * k, 2 * k + 1
        prev, _ = o.restir_initial(S, vol0, g, f0)
        prev.M[:] = 5000.0
        cur, resid = o.restir_initial(S, vol1, g, f1)
        out = {}
        for mode, rq in (("cached", None), ("fresh", vol1)):
            tmp = o.restir_temporal(S, g, g, cam, cur, prev, f1, requery=rq)
            res = o.restir_spatial(S, g, tmp, f1, 0, requery=rq)
            out[mode] = o.shade(S, vol1, g, res, resid)
            acc[mode][k] = out[mode].mean(0)
        differ += int(not np.array_equal(out["cached"], out["fresh"]))
    assert differ > T // 2                     # the two settings really select differently
    for mode in acc:
        mean, sd = acc[mode].mean(0), acc[mode].std(0) / math.sqrt(T)
        assert np.all(np.abs(mean - ref) <= 4 * np.sqrt(sd ** 2 + ref_sd ** 2)), (mode, mean, ref, sd)


def test_candidate_subsampling_pattern_and_cap(oracle_lib):
    """Sec. 5 subsampling, stride 3: only pixels with (x + y + f) % 3 == 0
    generate candidates (M = 32), the others start empty with M = 0; a
    pixel that generated none merges the previous reservoir capped at
    20 x the nominal 32 candidates, and its W is then the previous W."""
    import dataclasses
    o = oracle_lib
    sc = scenegen.tiny_room()
    st = dataclasses.replace(sc.settings, candidate_stride=3)
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    p = np.array([-0.3, -1.0, 0.2])
    W_, H_ = 6, 4
    cam = np.array([-0.3, 1.0, 0.2])
    g = _point_gbuffer(o, S, np.tile(p, (W_ * H_, 1)), np.tile([0, 1.0, 0], (W_ * H_, 1)),
                       np.tile([0.5, 0.5, 0.5], (W_ * H_, 1)), cam, width=W_)
    x, y = np.arange(W_ * H_) % W_, np.arange(W_ * H_) // W_
    for f in (4, 5):
        res, resid = o.restir_initial(S, vol, g, f, settings=st)
        gen = (x + y + f) % 3 == 0
        np.testing.assert_array_equal(res.M, np.where(gen, 32.0, 0.0))
        assert np.all(res.tri[~gen] == -1) and np.all(res.W[~gen] == 0) and np.all(resid[~gen] == 0)
        assert np.all(res.tri[gen] >= 0)
    # stride 1 is the plain method
    a, _ = o.restir_initial(S, vol, g, 7, settings=dataclasses.replace(st, candidate_stride=1))
    b, _ = o.restir_initial(S, vol, g, 7)
    np.testing.assert_array_equal(a.W, b.W)
    np.testing.assert_array_equal(a.tag, b.tag)
    # temporal merge onto a pixel without candidates
    prev, _ = o.restir_initial(S, vol, g, 4)             # every pixel generated
    prev.M[:] = 5000.0
    cur, _ = o.restir_initial(S, vol, g, 5, settings=st)
    out = o.restir_temporal(S, g, g, cam, cur, prev, 5, settings=st)
    empty = cur.M == 0
    np.testing.assert_array_equal(out.M[empty], 20.0 * 32.0)
    has = empty & (prev.tri >= 0)
    np.testing.assert_allclose(out.W[has], prev.W[has], rtol=1e-12)
    np.testing.assert_array_equal(out.tag[has], prev.tag[has])


@pytest.mark.slow
def test_subsampled_reuse_keeps_the_estimate_unbiased(oracle_lib):
    """The equal-target 8x8 image of the previous test with candidate stride
    2: half the pixels generate candidates each frame (alternating), the rest
    only reuse through temporal and spatial merges; the mean still converges
    to rho * Le * F (with empty probes there is no residual term to lose)."""
    import dataclasses
    o = oracle_lib
    sc = scenegen.tiny_room()
    st = dataclasses.replace(sc.settings, candidate_stride=2)
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    p = np.array([-0.3, -1.0, 0.2])
    n = 64
    cam = np.array([-0.3, 1.0, 0.2])
    g = _point_gbuffer(o, S, np.tile(p, (n, 1)), np.tile([0, 1.0, 0], (n, 1)),
                       np.tile([0.5, 0.5, 0.5], (n, 1)), cam, width=8)
    F = _rect_form_factor(-1 - p[0], -p[0], -1 - p[2], 1 - p[2], 2.0)
    exp = 0.5 * 10.0 * F
    T = 700
    acc = np.zeros((T, 3))
    for k in range(T):
        f0, f1 = 2 * k, 2 * k + 1
        prev, _ = o.restir_initial(S, vol, g, f0, settings=st)
        cur, resid = o.restir_initial(S, vol, g, f1, settings=st)
        tmp = o.restir_temporal(S, g, g, cam, cur, prev, f1, settings=st)
        res = o.restir_spatial(S, g, tmp, f1, 0, settings=st)
        acc[k] = o.shade(S, vol, g, res, resid).mean(0)
    mean, sd = acc.mean(0), acc.std(0) / math.sqrt(T)
    assert np.all(np.abs(mean - exp) <= 4 * sd), (mean, exp, sd)


def test_reservoir_merge_special_case(oracle_lib):
    """Two reservoirs with equal target: the merged W equals the M-weighted
    mean of the input W (target cancels), and M adds up (no cap hit)."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    S = o.Scene(sc)
    pts = np.array([[0.0, -1.0, 0.0]] * 2)
    g = _point_gbuffer(o, S, pts, np.tile([0, 1.0, 0], (2, 1)), np.tile([0.5] * 3, (2, 1)),
                       np.array([0.0, 1.0, 0.0]), width=2)
    cur = o.Reservoirs(2)
    prev = o.Reservoirs(2)
    ytri, _ = o.intersect(S, np.array([[-0.5, 0.5, 0.0]]), np.array([[0, 1.0, 0]]))
    for r, W, M in ((cur, 0.8, 32.0), (prev, 2.0, 100.0)):
        r.y[:] = [-0.5, 1.0, 0.0]
        r.L[:] = 10.0
        r.tri[:] = ytri[0]
        r.ny[:] = S.normals[ytri[0]]
        r.W[:] = W
        r.M[:] = M
        r.tag[:] = 7 if r is cur else 9
    out = o.restir_temporal(S, g, g, np.array([0.0, 1.0, 0.0]), cur, prev, 3)
    np.testing.assert_allclose(out.M, 132.0)
    np.testing.assert_allclose(out.W, (0.8 * 32 + 2.0 * 100) / 132.0, rtol=1e-12)


def test_reused_sample_keeps_its_normal(oracle_lib):
    """A reused sample is evaluated with the normal it was found with (cached
    with its point and radiance), not its triangle's current one: with the
    previous sample's normal turned from (0,-1,0) to (1,0,0), |cos| at y drops
    from 2 / sqrt(4.25) to 0.5 / sqrt(4.25), so its target is a quarter of the
    current sample's and the merged W follows in closed form."""
    o = oracle_lib
    sc = scenegen.tiny_room()
    S = o.Scene(sc)
    pts = np.array([[0.0, -1.0, 0.0]] * 2)
    g = _point_gbuffer(o, S, pts, np.tile([0, 1.0, 0], (2, 1)), np.tile([0.5] * 3, (2, 1)),
                       np.array([0.0, 1.0, 0.0]), width=2)
    ytri, _ = o.intersect(S, np.array([[-0.5, 0.5, 0.0]]), np.array([[0, 1.0, 0]]))
    np.testing.assert_allclose(S.normals[ytri[0]], [0.0, -1.0, 0.0], atol=1e-12)
    cur, prev = o.Reservoirs(2), o.Reservoirs(2)
    for r, W, M, n in ((cur, 0.8, 32.0, [0.0, -1.0, 0.0]), (prev, 2.0, 100.0, [1.0, 0.0, 0.0])):
        r.y[:] = [-0.5, 1.0, 0.0]
        r.L[:] = 10.0
        r.tri[:] = ytri[0]
        r.ny[:] = n
        r.W[:] = W
        r.M[:] = M
        r.tag[:] = 7 if r is cur else 9
    out = o.restir_temporal(S, g, g, np.array([0.0, 1.0, 0.0]), cur, prev, 3)
    np.testing.assert_allclose(out.M, 132.0)
    for k in range(2):
        exp = (0.8 * 32 + 0.25 * 2.0 * 100) / 132.0 if out.tag[k] == 7 else (4 * 0.8 * 32 + 2.0 * 100) / 132.0
        assert out.tag[k] in (7, 9)
        np.testing.assert_allclose(out.W[k], exp, rtol=1e-12)
        np.testing.assert_array_equal(out.ny[k], [0.0, -1.0, 0.0] if out.tag[k] == 7 else [1.0, 0.0, 0.0])


def test_mape_definition():
    import oracle
    ref = np.array([0.0, 1.0, 2.0])
    v = np.array([0.01, 1.5, 1.0])
    assert oracle.mape(v, ref) == pytest.approx((0.01 / 0.01 + 0.5 / 1.01 + 1.0 / 2.01) / 3)
    assert oracle.mse(v, ref) == pytest.approx((1e-4 + 0.25 + 1.0) / 3)


# ---------------------------------------------------------------------------
# path-traced reference (Sec. 4)
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_reference_furnace(oracle_lib):
    """Closed box where every surface emits Le = 1 and has albedo 0.5: the
    radiance is Le / (1 - rho) = 2 everywhere."""
    o = oracle_lib
    base = scenegen.tiny_room(width=8, height=8)
    T = base.num_tris
    sc = _custom_scene(base, albedo=np.full((T, 3), 0.5), emission=np.ones((T, 3)))
    S = o.Scene(sc)
    spp = 20000
    # pixels in the middle of the back wall (next-event estimation from points
    # near the box's creases has a heavy tail)
    est = o.pt_reference(S, sc.cameras[0], [18, 21, 27, 36, 42, 45], 3, 0, spp) / spp
    np.testing.assert_allclose(est, 2.0, rtol=0.02)


@pytest.mark.slow
def test_reference_direct_light_form_factor(oracle_lib):
    """Only the floor reflects (albedo 0.5): a floor pixel's reference is
    rho * Le * F with F the point-to-rectangle form factor of the emitter."""
    o = oracle_lib
    base = scenegen.tiny_room(width=16, height=16)
    alb = np.zeros_like(base.albedo)
    S0 = o.Scene(base)
    floor = np.flatnonzero(S0.normals[:, 1] > 0.9)
    alb[floor] = 0.5
    sc = _custom_scene(base, albedo=alb)
    cam = scenegen._look_camera([0.05, 0.5, 0.02], [0.05, -1.0, 0.0], 16, 16, 60.0)
    S = o.Scene(sc)
    g = o.gbuffer(S, cam)
    pix = np.flatnonzero(g.tri >= 0)[::9]
    spp = 1500
    est = o.pt_reference(S, cam, pix, 5, 0, spp) / spp
    for k, q in enumerate(pix):
        px = g.pos[q]
        F = _rect_form_factor(-1 - px[0], -px[0], -1 - px[2], 1 - px[2], 2.0)
        assert est[k, 0] == pytest.approx(0.5 * 10.0 * F, rel=0.06), (q, est[k], F)


# ---------------------------------------------------------------------------
# probe relocation (cited probe volume, Sec. 2; Majercik et al. 2021)
# ---------------------------------------------------------------------------

def _cube(c, h, outward=True):
    """12 triangles of an axis-aligned cube of half-size h around c, with
    normals pointing out of (or into) the cube."""
    c = np.asarray(c, float)
    tris = []
    for ax in range(3):
        u, v = [k for k in range(3) if k != ax]
        for sgn in (-1.0, 1.0):
            qc = c.copy()
            qc[ax] += sgn * h
            a, b = np.zeros(3), np.zeros(3)
            a[u], b[v] = h, h
            facing = np.zeros(3)
            facing[ax] = sgn if outward else -sgn
            tris += scenegen._quad(qc, a, b, facing)
    return np.asarray(tris)


def _reloc_setup(tris, grid):
    import oracle
    base = scenegen.tiny_room()
    T = len(tris)
    sc = _custom_scene(base, albedo=np.full((T, 3), 0.5), emission=np.zeros((T, 3)), verts=tris, grid=grid)
    st = dataclasses.replace(base.settings, rays_per_probe=256, probe_relocation=1)
    S = oracle.Scene(dataclasses.replace(sc, settings=st))
    return oracle, S, st, oracle.settings_of(st)


def test_relocation_moves_a_probe_out_of_a_box_it_sits_in(oracle_lib):
    """A probe 0.03 m off the centre of a closed, outward-facing cube of
    half-size 0.1 sees only back faces: it moves along its ray closest to the
    near (-x) face, by that ray's exit distance + delta/2, and lands outside
    the cube within delta/2 of the face plane.  The exit distances are
    recomputed here from the slab formula, not with the oracle's intersector."""
    grid = scenegen.ProbeGrid(np.zeros(3, np.float32), np.full(3, 1.0, np.float32), np.array([1, 1, 1], np.int32))
    c, h = np.array([0.03, 0.0, 0.0]), 0.1
    oracle, S, st, cs = _reloc_setup(_cube(c, h), grid)
    vol = oracle.Volume(grid)
    rays = oracle.probe_trace(S, vol, 3, settings=cs)
    assert np.all(rays[0, :, 3] < 0)                       # every hit is a back face
    dirs = oracle.probe_ray_dirs(st.seed, 3, st.rays_per_probe)
    hi = (c + h).astype(np.float32).astype(float)         # the scene stores float32 vertices
    lo = (c - h).astype(np.float32).astype(float)
    with np.errstate(divide="ignore"):
        slab = np.where(dirs > 0, hi / dirs, np.where(dirs < 0, lo / dirs, np.inf))
    t_exit = slab.min(axis=1)
    np.testing.assert_allclose(-rays[0, :, 3], t_exit, rtol=1e-9)
    rb = int(np.argmin(t_exit))
    delta = 0.1
    oracle.probe_relocate(vol, rays, 3, cs)
    want = dirs[rb] * (t_exit[rb] + 0.5 * delta)
    np.testing.assert_allclose(vol.offset[0], want, rtol=1e-12, atol=1e-15)
    P = vol.offset[0]
    assert P[0] < lo[0] and P[0] > lo[0] - 0.5 * delta - 1e-12
    assert np.all(np.abs(P[1:] - c[1:]) < h)


def test_relocation_pushes_a_probe_off_a_near_front_face(oracle_lib):
    """0.3 delta above an upward-facing floor (no back faces): the probe moves
    against its closest front hit by delta - t_f; a probe 0.2 m above the
    floor (> delta) and one in empty space stay put."""
    grid = scenegen.ProbeGrid(np.zeros(3, np.float32), np.full(3, 1.0, np.float32), np.array([1, 1, 1], np.int32))
    delta = 0.1
    for height, moves in ((0.3 * delta, True), (0.2, False)):
        floor = np.asarray(scenegen._quad([0, -height, 0], [5, 0, 0], [0, 0, 5], [0, 1, 0]))
        oracle, S, st, cs = _reloc_setup(floor, grid)
        vol = oracle.Volume(grid)
        rays = oracle.probe_trace(S, vol, 0, settings=cs)
        dirs = oracle.probe_ray_dirs(st.seed, 0, st.rays_per_probe)
        down = dirs[:, 1] < 0
        hf = float(np.float32(height))
        t_plane = np.where(down, hf / np.where(down, -dirs[:, 1], 1.0), np.inf)
        steep = dirs[:, 1] < -0.1                          # hit points well inside the 10 m floor
        np.testing.assert_allclose(rays[0, steep, 3], t_plane[steep], rtol=1e-9)
        assert np.all((rays[0, :, 3] > 0) | (rays[0, :, 3] >= 1e30))
        oracle.probe_relocate(vol, rays, 0, cs)
        if moves:
            rf = int(np.argmin(t_plane))
            np.testing.assert_allclose(vol.offset[0], -dirs[rf] * (delta - t_plane[rf]), rtol=1e-12)
            assert vol.offset[0][1] > 0
        else:
            np.testing.assert_array_equal(vol.offset[0], 0.0)


def test_relocation_threshold_and_clamp(oracle_lib):
    """Synthetic ray records: 16 of 64 back faces (exactly a quarter) do not
    move a probe, 17 do; a far back face moves it only to the 0.45 x spacing
    clamp on each axis."""
    import oracle
    grid = scenegen.ProbeGrid(np.zeros(3, np.float32), np.array([1.0, 0.5, 2.0], np.float32),
                              np.array([1, 1, 1], np.int32))
    st = dataclasses.replace(scenegen.tiny_room().settings, rays_per_probe=64, probe_relocation=1)
    cs = oracle.settings_of(st)
    dirs = oracle.probe_ray_dirs(st.seed, 2, 64)
    for nback, moved in ((16, False), (17, True)):
        vol = oracle.Volume(grid)
        rays = np.zeros((1, 64, 4))
        rays[0, :, 3] = 1e30
        rays[0, :nback, 3] = -np.linspace(5.0, 6.0, nback)   # closest back face: ray 0 at 5 m
        oracle.probe_relocate(vol, rays, 2, cs)
        if moved:
            lim = 0.45 * grid.spacing.astype(float)
            want = np.clip(dirs[0] * (5.0 + 0.5 * 0.05), -lim, lim)
            np.testing.assert_allclose(vol.offset[0], want, rtol=1e-12)
            np.testing.assert_array_equal(np.abs(vol.offset[0]), lim)
        else:
            np.testing.assert_array_equal(vol.offset[0], 0.0)


# ---------------------------------------------------------------------------
# scene dynamics: rigid instances, emitter toggling, reprojection
# ---------------------------------------------------------------------------

def _translation(I, t):
    M = np.tile(np.eye(3, 4), (I, 1, 1))
    M[:, :, 3] = t
    return M.reshape(I, 12)


def test_moved_instance_is_hit_where_it_moved(oracle_lib):
    """A ray toward a box translated by d along its axis hits it d closer
    (the static walls do not move); areas are unchanged by a rotation."""
    O = oracle_lib
    sc = scenegen.tiny_room_dynamic()
    S = O.Scene(sc)
    c = sc.motion.center[0]
    o = np.array([c[0], c[1], -0.999])
    d = np.array([0.0, 0.0, 1.0])
    tri0, t0 = O.intersect(S, o, d)
    assert sc.tri_instance[tri0] == 0
    shift = np.zeros((3, 3))
    shift[0, 2] = -0.05
    S.update(_translation(3, shift))
    tri1, t1 = O.intersect(S, o, d)
    assert sc.tri_instance[tri1] == 0
    assert t1 == pytest.approx(t0 - 0.05, abs=1e-9)
    area0 = S.area().copy()
    S.update(sc.instance_transforms(3))
    np.testing.assert_allclose(S.area(), area0, rtol=1e-6)
    moved = sc.tri_instance >= 0
    assert np.abs(S.verts.reshape(-1, 3, 3)[moved] - sc.verts[moved]).max() > 1e-3
    np.testing.assert_array_equal(S.verts.reshape(-1, 3, 3)[~moved], sc.verts[~moved].astype(float))


def test_previous_position_follows_the_instance(oracle_lib):
    """x_prev of a point on a moved triangle has the same barycentric
    coordinates on the triangle's previous pose; static points stay."""
    O = oracle_lib
    sc = scenegen.tiny_room_dynamic()
    S = O.Scene(sc)
    S.update(sc.instance_transforms(1))
    before = S.verts.reshape(-1, 3, 3).copy()
    S.update(sc.instance_transforms(2))
    after = S.verts.reshape(-1, 3, 3)
    rng = np.random.default_rng(4)
    for tri in list(np.flatnonzero(sc.tri_instance >= 0)[::5]) + [0, 7]:
        b = rng.dirichlet([1, 1, 1])
        x = b @ after[tri]
        xp = O.prev_position(S, int(tri), x)
        np.testing.assert_allclose(xp, b @ before[tri], atol=1e-12)


def test_emitter_toggle_keeps_the_emitter_list(oracle_lib):
    """Switching emitters off changes their radiance only: the emitter list
    and its area distribution, and so the choice of emitter for a given u,
    stay the same."""
    O = oracle_lib
    sc = scenegen.apartment_dynamic(frames=1)
    S = O.Scene(sc)
    us = np.random.default_rng(3).random(200)
    before = [O.sample_emitter(S, u) for u in us]
    le = sc.emitter_radiance(8)
    S.update(emitter_radiance=le)
    assert [O.sample_emitter(S, u) for u in us] == before
    em = np.flatnonzero(sc.emission.max(axis=1) > 0)
    np.testing.assert_array_equal(S.emission.reshape(-1, 3)[em], le.astype(float))
    assert (le.max(axis=1) > 0).sum() == len(em) // 2


def test_gbuffer_reprojects_a_moving_box(oracle_lib):
    """Static camera, box translated along the camera's right axis by d at
    depth z: its pixels' previous pixel is d / (z tan(fov/2) aspect) x W/2
    columns to the left (exact up to the pixel grid)."""
    O = oracle_lib
    sc = scenegen.tiny_room_dynamic(width=96, height=72)
    S = O.Scene(sc)
    cam = sc.cameras[0]
    S.update(_translation(3, np.zeros((3, 3))))
    shift = np.zeros((3, 3))
    shift[:, 0] = 0.06                                    # camera right is +x (looking down -z)
    S.update(_translation(3, shift))
    g = O.gbuffer(S, cam, cam)
    W, H = cam.width, cam.height
    on_box = np.flatnonzero((g.tri >= 0) & (sc.tri_instance[np.maximum(g.tri, 0)] >= 0))
    assert len(on_box) > 50
    z = -g.pos[on_box, 2]                                 # depth along the view axis (camera at the origin)
    dcol = 0.06 / (z * cam.tan_half_fovy * W / H) * W / 2
    i = on_box % W
    pq = g.prev[on_box]
    ok = pq >= 0
    pcol = pq[ok] % W
    exp = np.floor((i[ok] + 0.5) - dcol[ok])
    assert np.mean(np.abs(pcol - exp) <= 1) == 1.0
    assert np.mean(pcol == exp) > 0.95
    static = np.flatnonzero((g.tri >= 0) & (sc.tri_instance[np.maximum(g.tri, 0)] < 0))
    np.testing.assert_array_equal(g.prev[static], static)


def test_secondary_ddgi_collapses_to_the_one_bounce_estimator(oracle_lib):
    """With one BSDF candidate, no emitter candidates and no reuse (the
    paper's "secondary DDGI" comparison), the resampled term f W (W = 1/p_B)
    plus the residual of Sec. 3.5 collapse to rho_x L(y_B) for every pixel
    and frame: Le(x) + rho_x times the radiance cached at the BSDF hit."""
    o = oracle_lib
    base = scenegen.tiny_room(width=32, height=32)
    st = scenegen.secondary_ddgi(base.settings)
    sc = dataclasses.replace(base, settings=st)
    S = o.Scene(sc)
    vol = o.Volume(sc.grid)
    for f in range(3):
        o.probe_update(S, vol, f)
    g = o.gbuffer(S, sc.cameras[0])
    le_x = S.emission.reshape(-1, 3)[np.maximum(g.tri, 0)] * (g.tri >= 0)[:, None]
    for f in (4, 5):
        res, resid = o.restir_initial(S, vol, g, f)
        assert np.all(res.M[g.tri >= 0] == 1.0)
        out = o.shade(S, vol, g, res, resid)
        exp = le_x + g.alb * res.L * (res.tri >= 0)[:, None]
        np.testing.assert_allclose(out, exp, rtol=1e-9, atol=1e-12)
        assert (res.L.max(axis=1) > 0).mean() > 0.5
