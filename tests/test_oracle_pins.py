"""Pins of the CPU checker against things other than itself.

Each test below ties a part of the checker to a closed form, a textbook
special case, brute force on small inputs or an invariant of the method, so
that a dropped term, a wrong sign or index, or a transposed operand in the
checker fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _quad_x(x, half=1.0):
    """Two triangles spanning the plane x = const, |y|,|z| <= half."""
    V = np.array([[x, -half, -half], [x, half, -half], [x, half, half], [x, -half, half]], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return V, F


def _ray(o, d, tmin=0.0, tmax=1e30):
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.array([[*o, tmin, *d, tmax]], dtype=np.float32)


# --------------------------------------------------------------------------
# watertight ray/triangle test
# --------------------------------------------------------------------------
def test_watertight_golden_cases():
    cases = json.load(open(os.path.join(GOLDEN, "watertight_cases.json")))["cases"]
    for c in cases:
        hit, out = O.watertight(c["o"], c["d"], c["a"], c["b"], c["c"])
        assert hit == c["hit"], c["name"]
        if hit:
            assert out[0] == pytest.approx(c["t"], rel=1e-12, abs=1e-12), c["name"]
            assert out[1] == pytest.approx(c["u"], abs=1e-12), c["name"]
            assert out[2] == pytest.approx(c["v"], abs=1e-12), c["name"]


def test_watertight_random_points_reconstruct():
    """A hit reproduces its own point: o + t d == (1-u-v) a + u b + v c."""
    g = np.random.default_rng(1)
    for _ in range(2000):
        a, b, c = g.normal(size=(3, 3))
        w = g.dirichlet([1, 1, 1])
        p = w[0] * a + w[1] * b + w[2] * c
        o = p + g.normal(size=3) * 3
        d = (p - o) / np.linalg.norm(p - o)
        hit, (t, u, v) = O.watertight(o, d, a, b, c)
        assert hit
        assert np.allclose(o + t * d, (1 - u - v) * a + u * b + v * c, atol=1e-9)
        assert u == pytest.approx(w[1], abs=1e-7) and v == pytest.approx(w[2], abs=1e-7)


def test_watertight_no_leak_through_shared_edges_and_vertices():
    """Rays aimed exactly at mesh vertices and edge midpoints of a closed mesh
    seen from inside must always hit (no cracks between triangles)."""
    V, F = S.icosphere(2)
    V = V * 2.0
    E = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    targets = np.concatenate([V, 0.5 * (V[E[:, 0]] + V[E[:, 1]])])
    g = np.random.default_rng(2)
    origins = g.uniform(-0.5, 0.5, size=(targets.shape[0], 3))
    d = targets - origins
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([origins, np.zeros((len(d), 1)), d, np.full((len(d), 1), 1e30)], axis=1).astype(np.float32)
    hits = O.trace_brute(V, F, rays)
    assert np.all(hits["tracer"] == 1)


# --------------------------------------------------------------------------
# closest hit: brute force, BVH, closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_bvh_equals_brute_force(name):
    s = S.make_scene(name)
    bvh = O.BVH(s.verts, s.tris)
    rays = np.concatenate([R.primary_rays(s, 48, 32), R.gi_rays(s, 1500, 3, s.diagonal)])
    hb = O.trace_brute(s.verts, s.tris, rays)
    hv = bvh.trace(rays)
    assert np.array_equal(hb["prim"], hv["prim"])
    assert np.array_equal(hb["t"], hv["t"])
    assert np.array_equal(hb["tracer"], hv["tracer"])
    # any-hit agrees on whether something is hit
    ha = bvh.trace(rays, any_hit=True)
    assert np.array_equal(ha["tracer"] > 0, hb["tracer"] > 0)


def test_room_walls_closed_form():
    """Inside an empty room the first hit is the nearest wall along the ray:
    t = min over axes of (wall - o_a) / d_a."""
    V, F = S.room_mesh(4.0, 3.0, 5.0)
    g = np.random.default_rng(3)
    n = 4000
    o = g.uniform([0.1, 0.1, 0.1], [3.9, 2.9, 4.9], size=(n, 3))
    d = g.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((n, 1)), d, np.full((n, 1), 100.0)], axis=1).astype(np.float32)
    o32 = rays[:, 0:3].astype(np.float64)
    d32 = rays[:, 4:7].astype(np.float64)
    room = np.array([4.0, 3.0, 5.0])
    tw = np.where(d32 > 0, (room - o32) / d32, np.where(d32 < 0, -o32 / d32, np.inf)).min(axis=1)
    hits = O.BVH(V, F).trace(rays)
    assert np.all(hits["tracer"] == 1)
    np.testing.assert_allclose(hits["t"], tw, rtol=1e-12)
    # the wall that is hit is one of the two triangles on the plane the ray exits through
    axis = np.argmin(np.where(d32 > 0, (room - o32) / d32, np.where(d32 < 0, -o32 / d32, np.inf)), axis=1)
    n_f = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    hit_axis = np.argmax(np.abs(n_f[hits["prim"]]), axis=1)
    assert np.array_equal(hit_axis, axis)


def test_tiny_box_closed_form():
    """Rays at the axis-aligned box of the tiny scene: t = slab entry distance."""
    s = S.make_scene("tiny")
    box = [o for o in s.objects if o.kind == "box"][0]
    V = s.verts[box.first_tri * 0:]  # verts are shared; use the triangles of the box only
    F = s.tris[box.first_tri:box.first_tri + box.n_tris]
    lo = s.verts.astype(np.float64)[np.unique(F)].min(axis=0)
    hi = s.verts.astype(np.float64)[np.unique(F)].max(axis=0)
    g = np.random.default_rng(4)
    n = 2000
    tgt = g.uniform(lo + 0.05 * (hi - lo), hi - 0.05 * (hi - lo), size=(n, 3))
    o = tgt + g.normal(size=(n, 3)) * 3
    o = np.where(np.all((o > lo) & (o < hi), axis=1)[:, None], o + 5, o)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((n, 1)), d, np.full((n, 1), 100.0)], axis=1).astype(np.float32)
    o32, d32 = rays[:, 0:3].astype(np.float64), rays[:, 4:7].astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - o32) / d32
        t1 = (hi - o32) / d32
    tent = np.minimum(t0, t1).max(axis=1)
    hits = O.trace_brute(V, F, rays)
    assert np.all(hits["tracer"] == 1)
    np.testing.assert_allclose(hits["t"], tent, rtol=1e-9)


def test_icosphere_hit_between_inscribed_and_circumscribed_spheres():
    """An icosphere with vertices on a sphere of radius r contains the ball of its
    inradius r_in; a ray aimed at the centre hits at t in [|c-o|-r, |c-o|-r_in]."""
    V0, F = S.icosphere(3)
    r = 0.8
    c = np.array([0.3, -0.2, 0.5])
    V = V0 * r + c
    n_f = np.cross(V0[F[:, 1]] - V0[F[:, 0]], V0[F[:, 2]] - V0[F[:, 0]])
    r_in = r * np.min(np.abs(np.einsum("ij,ij->i", n_f / np.linalg.norm(n_f, axis=1, keepdims=True), V0[F[:, 0]])))
    g = np.random.default_rng(5)
    n = 1500
    dirs = g.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    o = c + dirs * g.uniform(1.5, 4, size=(n, 1))
    d = c - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((n, 1)), d, np.full((n, 1), 100.0)], axis=1).astype(np.float32)
    dist = np.linalg.norm(c - rays[:, 0:3].astype(np.float64), axis=1)
    hits = O.BVH(V, F).trace(rays)
    assert np.all(hits["tracer"] == 1)
    assert np.all(hits["t"] >= dist - r - 1e-6)
    assert np.all(hits["t"] <= dist - r_in + 1e-6)


def test_interval_is_closed_and_respected():
    V, F = _quad_x(2.0)
    bvh = O.BVH(V, F)
    # hit exactly at t_max and t_min counts, just outside does not
    rs = np.concatenate([_ray([0, 0.1, 0.2], [1, 0, 0], 0.0, 2.0), _ray([0, 0.1, 0.2], [1, 0, 0], 2.0, 5.0),
                         _ray([0, 0.1, 0.2], [1, 0, 0], 0.0, 1.999), _ray([0, 0.1, 0.2], [1, 0, 0], 2.001, 5.0),
                         _ray([3, 0.1, 0.2], [1, 0, 0], -5.0, 5.0)])
    h = bvh.trace(rs)
    assert list(h["tracer"]) == [1, 1, 0, 0, 1]
    assert h["t"][4] == pytest.approx(-1.0)


# --------------------------------------------------------------------------
# signed distance
# --------------------------------------------------------------------------
def test_box_sdf_closed_form():
    """The distance to a box made of exactly 12 triangles is the box SDF:
    outside |max(q,0)|, inside max(q) with q = |p - c| - half extent."""
    V0, F = S.box_mesh()
    ext = np.array([0.7, 0.4, 1.1])
    c = np.array([0.2, -0.1, 0.3])
    V = V0 * ext + c
    g = np.random.default_rng(6)
    P = g.uniform(-1.5, 1.5, size=(4000, 3))
    q = np.abs(P - c) - ext / 2
    exact = np.linalg.norm(np.maximum(q, 0), axis=1) + np.minimum(q.max(axis=1), 0)
    got = O.sdf_points_brute(V, F, P)
    np.testing.assert_allclose(got, exact, atol=1e-12)
    got_b = O.BVH(V, F).sdf_points(P)
    np.testing.assert_array_equal(got_b, got)


def test_rotated_box_sdf_closed_form():
    V0, F = S.box_mesh()
    ext = np.array([0.9, 0.5, 0.3])
    Rm = S.quat_to_matrix(0.3, 0.6, 0.1)
    c = np.array([1.0, 2.0, -1.0])
    V = (V0 * ext) @ Rm.T + c
    g = np.random.default_rng(7)
    P = c + g.uniform(-1.2, 1.2, size=(3000, 3))
    L = (P - c) @ Rm  # into the box frame
    q = np.abs(L) - ext / 2
    exact = np.linalg.norm(np.maximum(q, 0), axis=1) + np.minimum(q.max(axis=1), 0)
    np.testing.assert_allclose(O.sdf_points_brute(V, F, P), exact, atol=1e-12)


def test_room_interior_sdf_is_distance_to_nearest_wall():
    V, F = S.room_mesh(4.0, 3.0, 5.0)
    g = np.random.default_rng(8)
    P = g.uniform([0, 0, 0], [4, 3, 5], size=(3000, 3))
    exact = np.minimum(P, np.array([4.0, 3.0, 5.0]) - P).min(axis=1)
    np.testing.assert_allclose(O.sdf_points_brute(V, F, P), exact, atol=1e-12)
    # outside the room the field is negative
    Pout = np.array([[-0.5, 1, 1], [2, 3.5, 2], [2, 1, 6.0]])
    assert np.all(O.sdf_points_brute(V, F, Pout) < 0)


def test_icosphere_sdf_between_sphere_bounds():
    """rho - r <= phi <= rho - r_in for the distance rho to the centre (outside and inside)."""
    V0, F = S.icosphere(2)
    r = 0.6
    c = np.array([2.0, 1.5, 2.0])
    V = V0 * r + c
    n_f = np.cross(V0[F[:, 1]] - V0[F[:, 0]], V0[F[:, 2]] - V0[F[:, 0]])
    r_in = r * np.min(np.abs(np.einsum("ij,ij->i", n_f / np.linalg.norm(n_f, axis=1, keepdims=True), V0[F[:, 0]])))
    g = np.random.default_rng(9)
    dirs = g.normal(size=(3000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rho = g.uniform(0.0, 2.0, size=3000)
    P = c + dirs * rho[:, None]
    phi = O.sdf_points_brute(V, F, P)
    assert np.all(phi >= rho - r - 1e-12)
    assert np.all(phi <= rho - r_in + 1e-12)
    assert np.all(phi[rho < r_in - 1e-9] < 0)
    assert np.all(phi[rho > r + 1e-9] > 0)


def test_bake_bvh_equals_brute_and_features():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    P = O.grid_points(s.lo, s.hi, [12, 10, 12])
    a, fa = O.sdf_points_brute(s.verts, s.tris, P, feature=True)
    b, fb = bvh.sdf_points(P, feature=True)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(fa, fb)
    # lazily evaluated grid returns the same numbers
    grid = O.Grid(s.lo, s.hi, [12, 10, 12], src=bvh)
    idx = np.arange(P.shape[0])[::7]
    np.testing.assert_array_equal(grid.values(idx), a[idx])


# --------------------------------------------------------------------------
# trilinear interpolant and the march
# --------------------------------------------------------------------------
def _affine_grid(lo, hi, n, coef, const):
    P = O.grid_points(lo, hi, n)
    return P @ np.asarray(coef, dtype=np.float64) + const


def test_trilinear_exact_on_affine_fields():
    lo, hi, n = [-1.0, 0.5, 2.0], [3.0, 2.5, 5.0], [9, 5, 13]
    coef, const = [0.3, -1.7, 0.9], 0.25
    g = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, coef, const))
    rng = np.random.default_rng(10)
    P = rng.uniform(lo, hi, size=(2000, 3))
    phi, grad = g.sample(P)
    np.testing.assert_allclose(phi, P @ coef + const, atol=1e-12)
    np.testing.assert_allclose(grad, np.broadcast_to(coef, grad.shape), atol=1e-11)


def test_trilinear_matches_manual_interpolation_on_random_grid():
    """Random (non-affine) values: the checker's sample equals a direct
    evaluation of sum_k w_k v_k with the trilinear weights (x fastest)."""
    lo, hi, n = np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 3.0]), np.array([4, 6, 5])
    vals = np.random.default_rng(11).normal(size=n[::-1])
    g = O.Grid(lo, hi, n, values=vals)
    P = np.random.default_rng(12).uniform(lo, hi, size=(500, 3))
    h = (hi - lo) / (n - 1)
    u = (P - lo) / h
    i0 = np.minimum(np.floor(u).astype(int), n - 2)
    f = u - i0
    ref = np.zeros(len(P))
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                w = (f[:, 0] if bx else 1 - f[:, 0]) * (f[:, 1] if by else 1 - f[:, 1]) * (f[:, 2] if bz else 1 - f[:, 2])
                ref += w * vals[i0[:, 2] + bz, i0[:, 1] + by, i0[:, 0] + bx]
    np.testing.assert_allclose(g.sample(P)[0], ref, atol=1e-12)


def _plane_case(n_hat, c0, o, d, eps):
    """Sphere tracing on phi(p) = n.p - c0 (unit n): phi_k = phi_0 q^k, q = 1 + n.d;
    the march stops at the first k with phi_k < eps, at t = sum_{j<k} phi_j."""
    phi0 = float(np.dot(n_hat, o) - c0)
    q = 1.0 + float(np.dot(n_hat, d))
    t, phi, k = 0.0, phi0, 0
    while phi >= eps:
        t += phi
        phi = phi0 * q ** (k + 1)
        k += 1
    return t, k + 1


def test_march_on_plane_matches_geometric_series():
    lo, hi, n = [0.0, 0.0, 0.0], [8.0, 8.0, 8.0], [17, 17, 17]
    n_hat = np.array([0.2, 0.9, -0.1])
    n_hat /= np.linalg.norm(n_hat)
    c0 = float(np.dot(n_hat, [4, 1, 4]))
    g = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, n_hat, -c0))
    rng = np.random.default_rng(13)
    eps_vox = 0.01
    eps = eps_vox * 0.5
    checked = 0
    for _ in range(1000):
        o = rng.uniform([1, 4, 1], [7, 7.5, 7])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if np.dot(n_hat, d) > -0.3:
            continue
        ray = np.array([[*o, 0.0, *d, 100.0]], dtype=np.float32)
        o32, d32 = ray[0, 0:3].astype(np.float64), ray[0, 4:7].astype(np.float64)
        t_ref, steps = _plane_case(n_hat, c0, o32, d32, eps)
        p_hit = o32 + t_ref * d32
        if np.any(p_hit < 0) or np.any(p_hit > 8):
            continue
        prm = O.make_params(mode=3, max_steps=1000, hit_eps_vox=eps_vox, min_step_vox=eps_vox)
        h = O.trace_sdf(g, ray, prm, precision=64)[0]
        assert h["tracer"] == 2
        assert h["t"] == pytest.approx(t_ref, rel=1e-10)
        assert h["steps"] == steps
        checked += 1
    assert checked > 50


def test_march_margin_on_plane_is_the_closest_gap_of_the_series():
    """The decision margin is min_j |phi_j - eps| over the march's steps; on a
    plane phi_j = phi_0 q^j (closed form), ending at the first phi_k < eps."""
    lo, hi, n = [0.0, 0.0, 0.0], [8.0, 8.0, 8.0], [17, 17, 17]
    n_hat = np.array([-0.3, 0.8, 0.2])
    n_hat /= np.linalg.norm(n_hat)
    c0 = float(np.dot(n_hat, [4, 1, 4]))
    g = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, n_hat, -c0))
    rng = np.random.default_rng(21)
    eps_vox = 0.01
    eps = eps_vox * 0.5
    checked = 0
    for _ in range(600):
        o = rng.uniform([1, 4, 1], [7, 7.5, 7])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if np.dot(n_hat, d) > -0.3:
            continue
        ray = np.array([[*o, 0.0, *d, 100.0]], dtype=np.float32)
        o32, d32 = ray[0, 0:3].astype(np.float64), ray[0, 4:7].astype(np.float64)
        t_ref, steps = _plane_case(n_hat, c0, o32, d32, eps)
        if np.any(o32 + t_ref * d32 < 0) or np.any(o32 + t_ref * d32 > 8):
            continue
        phi0 = float(np.dot(n_hat, o32) - c0)
        q = 1.0 + float(np.dot(n_hat, d32))
        want = min(abs(phi0 * q ** j - eps) for j in range(steps))
        prm = O.make_params(mode=3, max_steps=1000, hit_eps_vox=eps_vox, min_step_vox=eps_vox)
        h = O.trace_sdf(g, ray, prm, precision=64)[0]
        assert h["margin"] == pytest.approx(want, rel=1e-9, abs=1e-12)
        checked += 1
    assert checked > 50
    # a query that never marches has no margin
    miss = np.array([[-5, -5, -5, 0.0, -1, 0, 0, 1.0]], dtype=np.float32)
    assert np.isinf(O.trace_sdf(g, miss, O.make_params(mode=3), precision=64)[0]["margin"])


def test_tri_check_closed_form():
    """Ray aimed at the point of barycentric weights (u, v) of a triangle from
    distance dist, at a chosen angle to its normal: hit exactly when the point
    is inside, t = dist, the same (u, v) inside or out, |n . d| = cos(angle)."""
    rng = np.random.default_rng(22)
    V = rng.normal(size=(60, 3))
    F = np.arange(60, dtype=np.int32).reshape(20, 3)
    rays, prims, want = [], [], []
    for k in range(20):
        a, b, c = V[F[k]]
        nrm = np.cross(b - a, c - a)
        nrm /= np.linalg.norm(nrm)
        tang = np.cross(nrm, b - a)
        tang /= np.linalg.norm(tang)
        for u, v in ((0.2, 0.3), (0.6, 0.35), (-0.25, 0.5), (0.7, 0.6), (0.5, -1e-3)):
            p = (1 - u - v) * a + u * b + v * c
            ang = rng.uniform(0.1, 1.2)
            d = -(np.cos(ang) * nrm + np.sin(ang) * tang) * rng.choice([-1, 1])
            dist = rng.uniform(0.5, 3.0)
            o = p - dist * d
            rays.append([*o, 0.0, *d, 100.0])
            prims.append(k)
            want.append((u >= 0 and v >= 0 and u + v <= 1, dist, u, v, np.cos(ang)))
    rays = np.array(rays, dtype=np.float64)
    # the float32 ray the checker sees
    r32 = rays.astype(np.float32)
    got = O.tri_check(V, F, r32, np.array(prims))
    for i, (inside, dist, u, v, cs) in enumerate(want):
        assert got["hit"][i] == inside, i
        # the float32 rounding of o and d moves the point by ~1e-7 relative
        assert got["t"][i] == pytest.approx(dist, rel=1e-5, abs=1e-5)
        assert got["u"][i] == pytest.approx(u, abs=1e-4) and got["v"][i] == pytest.approx(v, abs=1e-4)
        assert got["ndotd"][i] == pytest.approx(cs, abs=1e-5)
    # no triangle: no test
    none = O.tri_check(V, F, r32[:2], np.array([-1, 20]))
    assert not none["hit"].any() and np.isinf(none["t"]).all()


def test_grid_export_knows_exactly_what_was_evaluated():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = [9, 7, 8]
    g = O.Grid(s.lo, s.hi, n, src=bvh)
    vals, known = g.export()
    assert not known.any() and not vals.any()
    idx = np.array([0, 5, 17, 100, 503])
    got = g.values(idx)
    vals, known = g.export()
    assert np.array_equal(np.nonzero(known)[0], idx)
    np.testing.assert_array_equal(vals[idx], got)
    np.testing.assert_allclose(got, O.sdf_points_brute(s.verts, s.tris, O.grid_points(s.lo, s.hi, n)[idx]),
                               rtol=0, atol=1e-12)
    dense = O.Grid(s.lo, s.hi, n, values=np.arange(9 * 7 * 8, dtype=np.float64))
    vals, known = dense.export()
    assert known.all() and np.array_equal(vals, np.arange(9 * 7 * 8))


def test_march_start_inside_hits_at_t_min_and_step_limit_flags():
    lo, hi, n = [0.0, 0.0, 0.0], [4.0, 4.0, 4.0], [9, 9, 9]
    g = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, [1, 0, 0], -1.0))  # phi = x - 1
    inside = np.array([[0.5, 2, 2, 0.25, 1, 0, 0, 10]], dtype=np.float32)
    h = O.trace_sdf(g, inside, O.make_params(mode=3), 64)[0]
    assert h["tracer"] == 2 and h["t"] == 0.25 and h["steps"] == 1
    # parallel to the surface, far from it: marches until the grid box ends -> miss
    par = np.array([[3.0, 2, 0.1, 0, 0, 0, 1, 100]], dtype=np.float32)
    h = O.trace_sdf(g, par, O.make_params(mode=3), 64)[0]
    assert h["tracer"] == 0 and h["flags"] == 0
    # grazing approach with a tiny step budget -> miss with the step-limit flag
    d = np.array([-0.02, 0, 1.0])
    d /= np.linalg.norm(d)
    gr = np.array([[3.0, 2, 0.1, 0, *d, 100]], dtype=np.float32)
    h = O.trace_sdf(g, gr, O.make_params(mode=3, max_steps=1), 64)[0]
    assert h["tracer"] == 0 and h["flags"] & O.FLAG_STEP_LIMIT and h["steps"] == 1


def test_march_outside_grid_is_clipped():
    lo, hi, n = [0.0, 0.0, 0.0], [4.0, 4.0, 4.0], [9, 9, 9]
    g = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, [-1, 0, 0], 3.0))  # phi = 3 - x
    miss = np.array([[-1.0, 5.0, 2, 0, 1, 0, 0, 100]], dtype=np.float32)  # passes above the box
    assert O.trace_sdf(g, miss, O.make_params(mode=3), 64)[0]["tracer"] == 0
    enter = np.array([[-2.0, 2.0, 2, 0, 1, 0, 0, 100]], dtype=np.float32)  # enters at t=2, plane x=3 at t=5
    h = O.trace_sdf(g, enter, O.make_params(mode=3), 64)[0]
    assert h["tracer"] == 2 and h["t"] == pytest.approx(5.0, abs=1e-12)


def test_nan_query_is_a_miss():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    grid = O.Grid(s.lo, s.hi, [8, 8, 8], src=bvh)
    base = np.array([2.0, 1.5, 2.0, 0.0, 1.0, 0.0, 0.0, 10.0], dtype=np.float32)
    rays = np.tile(base, (9, 1))
    for k in range(8):
        rays[k + 1, k] = np.nan
    for mode in range(4):
        for prec in (64, 32):
            h = O.trace_combined(bvh, grid, rays, O.make_params(mode=mode), prec)
            assert h["tracer"][0] > 0 and np.all(h["tracer"][1:] == 0)
    assert np.all(bvh.trace(rays)["tracer"][1:] == 0)
    # t_min > t_max is empty even where a wall sits exactly at t_max
    rev = np.array([[2.0, 1.5, 2.0, 2.5, 1.0, 0.0, 0.0, 2.0]], dtype=np.float32)
    for mode in range(4):
        assert O.trace_combined(bvh, grid, rev, O.make_params(mode=mode), 32)["tracer"][0] == 0


def test_fp32_march_close_to_fp64():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = [32, 32, 32]
    grid = O.Grid(s.lo, s.hi, n, values=O.bake_brute(s.verts, s.tris, s.lo, s.hi, n))
    rays = R.gi_rays(s, 3000, 21, s.diagonal)
    p = O.make_params(mode=3)
    a = O.trace_sdf(grid, rays, p, 64)
    b = O.trace_sdf(grid, rays, p, 32)
    assert np.array_equal(a["tracer"], b["tracer"])
    both = (a["tracer"] == 2)
    assert np.max(np.abs(a["t"][both] - b["t"][both]) / np.maximum(1, a["t"][both])) < 1e-3


# --------------------------------------------------------------------------
# the combined query: split rule, ordering and the pure endpoints
# --------------------------------------------------------------------------
def test_split_rule_golden_cases():
    spec = json.load(open(os.path.join(GOLDEN, "split_rule_cases.json")))
    lo, hi, n = [-1.0, -2.0, -2.0], [11.0, 2.0, 2.0], [25, 9, 9]
    for c in spec["cases"]:
        V, F = _quad_x(c["wall"])
        bvh = O.BVH(V, F)
        grid = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, [-1, 0, 0], c["field"]))
        m_near = math.inf if c["m_near"] == "inf" else c["m_near"]
        p = O.make_params(mode=c["mode"], any_hit=c["any_hit"], m_near=m_near, m_far=c["m_far"])
        ray = np.array([[0, 0.1, -0.3, 0, 1, 0, 0, 10]], dtype=np.float32)
        for prec in (64, 32):
            h = O.trace_combined(bvh, grid, ray, p, prec)[0]
            assert h["tracer"] == c["tracer"], (c, prec)
            if c["tracer"]:
                assert h["t"] == pytest.approx(c["t"], abs=1e-6), (c, prec)


@pytest.mark.parametrize("any_hit", [0, 1])
def test_endpoints_equal_pure_techniques(any_hit):
    """Section 3 compares against the pure techniques: a multiplier of 0 is the
    distance field alone and an infinite one is triangles alone, hit for hit."""
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = [32, 32, 32]
    grid = O.Grid(s.lo, s.hi, n, values=O.bake_brute(s.verts, s.tris, s.lo, s.hi, n))
    rays = R.gi_rays(s, 2000, 5, s.diagonal)
    for prec in (64, 32):
        for mode in (1, 2):
            p0 = O.make_params(mode=mode, any_hit=any_hit, m_near=0.0, m_far=0.0)
            pinf = O.make_params(mode=mode, any_hit=any_hit, m_near=math.inf, m_far=math.inf)
            np.testing.assert_array_equal(O.trace_combined(bvh, grid, rays, p0, prec),
                                          O.trace_sdf(grid, rays, p0, prec))
            hb = bvh.trace(rays, any_hit=bool(any_hit))
            hc = O.trace_combined(bvh, grid, rays, pinf, prec)
            np.testing.assert_array_equal(hc["tracer"], hb["tracer"])
            np.testing.assert_array_equal(hc["t"], hb["t"])
            np.testing.assert_array_equal(hc["prim"], hb["prim"])


def test_combined_middle_ground_between_pure_techniques():
    """The combined result lies between the pure techniques: its hit-t
    disagreement with triangles-only is below distance-field-only's (Section 3)."""
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = [32, 32, 32]
    grid = O.Grid(s.lo, s.hi, n, values=O.bake_brute(s.verts, s.tris, s.lo, s.hi, n))
    rays = R.gi_rays(s, 4000, 6, s.diagonal)
    ref = bvh.trace(rays)["t"]
    err = {}
    for m in (0.0, 2.0, 8.0):
        t = O.trace_combined(bvh, grid, rays, O.make_params(mode=1, m_near=m), 64)["t"]
        ok = np.isfinite(t) & np.isfinite(ref)
        err[m] = np.mean(np.abs(t[ok] - ref[ok]))
    assert err[8.0] < err[2.0] < err[0.0]


def test_sdf_sign_negative_inside_objects_positive_in_free_space():
    s = S.make_scene("medium")
    bvh = O.BVH(s.verts, s.tris)
    sph = [o for o in s.objects if o.kind == "sphere"]
    g = np.random.default_rng(14)
    inside = np.concatenate([o.center + 0.5 * o.radius * g.uniform(-0.5, 0.5, size=(20, 3)) for o in sph])
    assert np.all(bvh.sdf_points(inside) < 0)
    free = R.free_space_rays(s, 500, 3, margin=0.05)[:, 0:3]
    assert np.all(bvh.sdf_points(free) > 0)


# --------------------------------------------------------------------------
# adjoint of the distance-field hit distance
# --------------------------------------------------------------------------
def test_adjoint_closed_form_on_plane():
    """phi = n.p - c0: the root of phi = eps is t* = (eps - phi(o)) / (n.d), and
    dt*/dtheta_k = -w_k(p*) / (n.d) with the trilinear weights w_k."""
    lo, hi, n = [0.0, 0.0, 0.0], [4.0, 4.0, 4.0], [9, 9, 9]
    n_hat = np.array([0.3, 0.8, 0.2])
    n_hat /= np.linalg.norm(n_hat)
    g = O.Grid(lo, hi, n, values=_affine_grid(lo, hi, n, n_hat, -2.0))
    rng = np.random.default_rng(15)
    p = O.make_params(mode=3, max_steps=1000)
    eps = 0.01 * 0.5
    for _ in range(50):
        o = rng.uniform(1.5, 3.5, size=3)
        o = o + n_hat * (3.5 - np.dot(n_hat, o))  # start above the plane
        d = -n_hat + 0.4 * rng.normal(size=3)
        d /= np.linalg.norm(d)
        ray = np.array([[*o, 0, *d, 50]], dtype=np.float32)
        o32, d32 = ray[0, :3].astype(np.float64), ray[0, 4:7].astype(np.float64)
        t, idx, w = O.sdf_root_adjoint(g, ray, p)
        p_root = o32 + t[0] * d32
        if not np.all((p_root > 0) & (p_root < 4)):
            continue
        nd = float(np.dot(n_hat, d32))
        assert t[0] == pytest.approx((eps - (np.dot(n_hat, o32) - 2.0)) / nd, rel=1e-9)
        assert np.all(idx[0] >= 0)
        # weights of the corners sum to 1 -> sum of dt/dtheta = -1/(n.d)
        assert w[0].sum() == pytest.approx(-1.0 / nd, rel=1e-9)


def test_adjoint_matches_central_differences():
    s = S.make_scene("tiny")
    n = [32, 32, 32]
    vals = O.bake_brute(s.verts, s.tris, s.lo, s.hi, n).reshape(-1)
    vals = vals + np.random.default_rng(16).normal(scale=0.01, size=vals.size)
    rays = R.gi_rays(s, 64, 17, s.diagonal)
    p = O.make_params(mode=3)
    g = O.Grid(s.lo, s.hi, n, values=vals)
    t0, idx, w = O.sdf_root_adjoint(g, rays, p)
    checked = 0
    for i in range(len(rays)):
        if idx[i, 0] < 0:
            continue
        k = int(np.argmax(np.abs(w[i])))
        vi = idx[i, k]
        delta = 1e-6
        vp = vals.copy(); vp[vi] += delta
        vm = vals.copy(); vm[vi] -= delta
        tp = O.sdf_root_adjoint(O.Grid(s.lo, s.hi, n, values=vp), rays[i:i + 1], p)[0][0]
        tm = O.sdf_root_adjoint(O.Grid(s.lo, s.hi, n, values=vm), rays[i:i + 1], p)[0][0]
        fd = (tp - tm) / (2 * delta)
        if not (np.isfinite(tp) and np.isfinite(tm)):
            continue
        assert fd == pytest.approx(w[i, k], rel=1e-2, abs=1e-6)
        checked += 1
    assert checked >= 20


# --------------------------------------------------------------------------
# the seeded workloads
# --------------------------------------------------------------------------
def test_cosine_hemisphere_moments():
    n = np.tile(np.array([[0.0, 0.0, 1.0]]), (200000, 1))
    from synth import rng
    u = rng.uniform(1, 2, 400000).reshape(-1, 2)
    d = R.cosine_hemisphere(n, u[:, 0], u[:, 1])
    cos = d[:, 2]
    assert np.all(cos >= 0)
    assert cos.mean() == pytest.approx(2 / 3, abs=3e-3)  # E[cos] for p ~ cos / pi
    assert (cos ** 2).mean() == pytest.approx(0.5, abs=3e-3)


def test_scene_triangle_counts_and_seed_determinism():
    assert S.make_scene("tiny").n_tris == 344
    a = S.make_scene("medium", seed=9)
    b = S.make_scene("medium", seed=9)
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
    assert S.make_scene("medium", seed=10).verts.tobytes() != a.verts.tobytes()


def test_icosphere_is_closed_and_outward():
    V, F = S.icosphere(3)
    assert F.shape[0] == 20 * 4 ** 3
    E = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    _, counts = np.unique(E, axis=0, return_counts=True)
    assert np.all(counts == 2)  # every edge shared by exactly two faces
    vol = np.einsum("ij,ij->i", V[F[:, 0]], np.cross(V[F[:, 1]], V[F[:, 2]])).sum() / 6
    assert 0 < vol < 4 / 3 * math.pi
