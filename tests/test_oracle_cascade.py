"""Pins of the checker's camera-centred cascade (Section 3, "Distance Field
Generation"; split points from the voxel size at the ray's start and end,
Section 3, "GI & Shadow Rays").

Each test ties the cascade part of the checker to something other than
itself: hand-derived split points, brute-force level lookup, the single-grid
path it reduces to with one level, the geometric series of a march on a plane
inside one level, and the exact distance at the lattice points.
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
H0 = float(np.float32(0.1))


def _affine_cascade(center, h0, n, levels, coef, const):
    """Cascade whose every level holds phi(p) = coef . p + const at its lattice points."""
    shell = O.Cascade(center, h0, n, levels, values=np.zeros((levels, n, n, n)))
    vals = np.stack([shell.points(k) @ np.asarray(coef, dtype=np.float64) + const for k in range(levels)])
    return O.Cascade(center, h0, n, levels, values=vals)


def test_split_points_golden_cases():
    spec = json.load(open(os.path.join(GOLDEN, "cascade_split_cases.json")))
    n, L = spec["n"], spec["levels"]
    cas = O.Cascade(spec["center"], float(np.float32(spec["h0"])), n, L, values=np.ones((L, n, n, n)))
    far = O.BVH(np.array([[900.0, 900, 900], [901, 900, 900], [900, 901, 900]]), np.array([[0, 1, 2]], dtype=np.int32))
    for c in spec["cases"]:
        tmax = math.inf if c["tmax"] == "inf" else c["tmax"]
        ray = np.array([[*c["o"], c["tmin"], *c["d"], tmax]], dtype=np.float32)
        p = O.make_params(mode=c["mode"], m_near=c["m_near"], m_far=c["m_far"])
        for prec in (64, 32):
            _, t12 = O.trace_combined(far, cas, ray, p, prec, split_points=True)
            for got, want in ((t12[0, 0], c["t1"]), (t12[0, 1], c["t2"])):
                if want == "inf":
                    assert got == math.inf, (c, prec)
                else:
                    assert got == pytest.approx(want, abs=2e-6 * max(1.0, want)), (c, prec, got)


def test_geometry_is_camera_centred_nested_and_moves_by_whole_samples():
    rng = np.random.default_rng(40)
    n, L = 64, 5
    for _ in range(50):
        c = rng.uniform(-30, 30, size=3)
        cas = O.Cascade(c, H0, n, L, values=np.zeros((L, n, n, n)))
        prev = None
        for k in range(L):
            ilo, h = cas.level(k)
            assert h == H0 * 2 ** k
            lo, hi = cas.box(k)
            # the centre sits in the middle cell of every level
            cell = np.floor((c - lo) / h)
            assert np.all(cell == (n - 1) // 2)
            assert np.all(lo <= c) and np.all(c <= hi)
            if prev is not None:
                assert np.all(prev[0] >= lo) and np.all(prev[1] <= hi), "levels must nest"
            prev = (lo, hi)
        # moving the centre by m whole voxels of level k moves that lattice by m samples
        k = int(rng.integers(0, L))
        ilo0, h = cas.level(k)
        step = rng.integers(-5, 6, size=3)
        moved = O.Cascade(c + step * h, H0, n, L, values=np.zeros((L, n, n, n)))
        ilo1, _ = moved.level(k)
        # floor((c + m h) / h) = floor(c / h) + m unless c / h rounds across an integer
        frac = c / h - np.floor(c / h)
        ok = (frac > 1e-9) & (frac < 1 - 1e-9)
        assert np.all((ilo1 - ilo0)[ok] == step[ok])


@pytest.mark.parametrize("precision", [64, 32])
def test_level_lookup_equals_brute_force(precision):
    n, L = 16, 4
    cas = O.Cascade([0.3, -0.2, 0.7], 0.0625, n, L, values=np.zeros((L, n, n, n)))
    rng = np.random.default_rng(41)
    P = rng.uniform(-5, 5, size=(20000, 3))
    # points on the faces of every box (closed boxes)
    faces = []
    for k in range(L):
        lo, hi = cas.box(k)
        for a in range(3):
            for v in (lo[a], hi[a]):
                q = rng.uniform(lo, hi, size=(50, 3))
                q[:, a] = v
                faces.append(q)
    P = np.concatenate([P] + faces)
    dt = np.float64 if precision == 64 else np.float32
    Pq = P.astype(dt)
    want = np.full(P.shape[0], L - 1)
    for k in reversed(range(L - 1)):
        lo, hi = (b.astype(dt) for b in cas.box(k))
        inside = np.all((Pq >= lo) & (Pq <= hi), axis=1)
        want[inside] = k
    got = cas.level_of(Pq.astype(np.float64), precision)
    np.testing.assert_array_equal(got, want)
    assert len(set(got.tolist())) == L


@pytest.mark.parametrize("mode,any_hit", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0)])
def test_one_level_cascade_equals_single_grid(mode, any_hit):
    """With one level, a cascade is a single grid: same samples, same voxel,
    same split points, so every hit record equals the single-grid checker's."""
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n, h0 = 33, 0.125
    center = np.array([2.03, 1.51, 1.97])
    cas_shell = O.Cascade(center, h0, n, 1, values=np.zeros((1, n, n, n)))
    lo, hi = cas_shell.box(0)
    vals = bvh.sdf_points(cas_shell.points(0))
    cas = O.Cascade(center, h0, n, 1, values=vals)
    grid = O.Grid(lo, hi, [n, n, n], values=vals)
    rays = R.gi_rays(s, 1500, 42, s.diagonal)
    p = O.make_params(mode=mode, any_hit=any_hit, m_near=3.0, m_far=1.5)
    for prec in (64, 32):
        a = O.trace_combined(bvh, cas, rays, p, prec)
        b = O.trace_combined(bvh, grid, rays, p, prec)
        np.testing.assert_array_equal(a, b)
    assert np.any(a["tracer"] == 2)


def _plane_case(n_hat, c0, o, d, eps):
    """Sphere tracing on phi(p) = n.p - c0 (unit n): phi_k = phi_0 q^k, q = 1 + n.d;
    stops at the first k with phi_k < eps, at t = sum_{j<k} phi_j."""
    phi0 = float(np.dot(n_hat, o) - c0)
    q = 1.0 + float(np.dot(n_hat, d))
    t, phi, k = 0.0, phi0, 0
    while phi >= eps:
        t += phi
        phi = phi0 * q ** (k + 1)
        k += 1
    return t, k + 1


def test_march_inside_one_level_uses_that_levels_voxel():
    """A march that stays inside level 3 (outside level 2) follows the plane's
    geometric series with eps = 0.01 h_3: a checker that used the finest voxel,
    or the wrong level's samples, takes a different number of steps."""
    n, L = 64, 5
    n_hat = np.array([-1.0, 0.15, 0.05])
    n_hat /= np.linalg.norm(n_hat)
    c0 = float(np.dot(n_hat, [23.0, 0.0, 0.0]))  # the plane crosses the x axis at 23 m
    cas = _affine_cascade([0, 0, 0], H0, n, L, n_hat, -c0)  # phi = n.p - c0, positive for x < 23
    lo2, hi2 = cas.box(2)
    lo3, hi3 = cas.box(3)
    h3 = cas.level(3)[1]
    eps_vox = 0.01
    rng = np.random.default_rng(43)
    checked = 0
    for _ in range(400):
        o = np.array([rng.uniform(14, 18), rng.uniform(-5, 5), rng.uniform(-5, 5)])
        d = rng.normal(size=3)
        d[1:] /= np.linalg.norm(d[1:])
        d[0] = rng.uniform(0.25, 0.6)
        d[1:] *= math.sqrt(1 - d[0] ** 2)
        ray = np.array([[*o, 0.0, *d, 60.0]], dtype=np.float32)
        o32, d32 = ray[0, 0:3].astype(np.float64), ray[0, 4:7].astype(np.float64)
        t_ref, steps = _plane_case(n_hat, c0, o32, d32, eps_vox * h3)
        p_hit = o32 + t_ref * d32
        if not (np.all(p_hit >= lo3) and np.all(p_hit <= hi3)) or p_hit[0] <= hi2[0] + 0.1 or steps < 6:
            continue
        prm = O.make_params(mode=3, max_steps=1000, hit_eps_vox=eps_vox, min_step_vox=eps_vox)
        h = O.trace_combined(None, cas, ray, prm, 64)[0]
        assert h["tracer"] == 2
        assert h["steps"] == steps
        assert h["t"] == pytest.approx(t_ref, rel=1e-10)
        checked += 1
    assert checked > 100


def test_lazy_level_values_are_the_exact_distance_at_the_lattice_points():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n, L = 16, 3
    cas = O.Cascade([1.7, 1.2, 2.2], 0.0625, n, L, src=bvh)
    rng = np.random.default_rng(44)
    for k in range(L):
        idx = rng.choice(n ** 3, size=300, replace=False)
        got = cas.values(k, idx)
        want = O.sdf_points_brute(s.verts, s.tris, cas.points(k)[idx])
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("any_hit", [0, 1])
def test_cascade_endpoints_equal_pure_techniques(any_hit):
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n, L = 16, 4
    shell = O.Cascade(s.camera.eye, 0.0625, n, L, values=np.zeros((L, n, n, n)))
    vals = np.stack([bvh.sdf_points(shell.points(k)) for k in range(L)])
    cas = O.Cascade(s.camera.eye, 0.0625, n, L, values=vals)
    rays = R.gi_rays(s, 1500, 45, s.diagonal)
    for prec in (64, 32):
        for mode in (1, 2):
            p0 = O.make_params(mode=mode, any_hit=any_hit, m_near=0.0, m_far=0.0)
            pinf = O.make_params(mode=mode, any_hit=any_hit, m_near=math.inf, m_far=math.inf)
            psdf = O.make_params(mode=3, any_hit=any_hit)
            np.testing.assert_array_equal(O.trace_combined(bvh, cas, rays, p0, prec),
                                          O.trace_combined(bvh, cas, rays, psdf, prec))
            hb = bvh.trace(rays, any_hit=bool(any_hit))
            hc = O.trace_combined(bvh, cas, rays, pinf, prec)
            np.testing.assert_array_equal(hc["tracer"], hb["tracer"])
            np.testing.assert_array_equal(hc["t"], hb["t"])
            np.testing.assert_array_equal(hc["prim"], hb["prim"])
    # the field-only cascade query does hit, at several levels
    h = O.trace_combined(None, cas, rays, O.make_params(mode=3), 64)
    hit = h["tracer"] == 2
    assert hit.mean() > 0.9
    lv = cas.level_of(rays[hit, 0:3].astype(np.float64) + h["t"][hit, None] * rays[hit, 4:7].astype(np.float64))
    assert len(set(lv.tolist())) >= 2


@pytest.mark.parametrize("mode", [1, 2])
def test_near_hits_over_the_field_from_t1_equal_the_in_order_query(mode):
    """The sub-intervals of Eq. 2 are ordered: a hit in [t_min, t_1] lies before
    any point of [t_1, t_max].  So a closest-hit query can trace its field (and
    far) sub-intervals from t_1 without waiting for its near result, and put the
    near hit, where there is one, over their record (Section 2; the concurrent
    program of the stage kernels relies on it).  Checked on the checker alone:
    the near sub-interval as a triangles-only query on [t_min, t_1], the rest
    as a query starting at t_1 with m_near = 0, merged, against the in-order
    query, with the t_1 of every query taken from the checker (float mode, so t_1
    is a float and the rays can carry it)."""
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n, L = 16, 4
    shell = O.Cascade(s.camera.eye, 0.0625, n, L, values=np.zeros((L, n, n, n)))
    vals = np.stack([bvh.sdf_points(shell.points(k)) for k in range(L)])
    cas = O.Cascade(s.camera.eye, 0.0625, n, L, values=vals)
    rays = R.gi_rays(s, 3000, 46, s.diagonal)
    for m in (0.5, 2.0, 8.0):
        p = O.make_params(mode=mode, m_near=m, m_far=2.0)
        ref, t12 = O.trace_combined(bvh, cas, rays, p, 32, split_points=True)
        t1 = t12[:, 0]
        assert np.all(np.isfinite(t1)) and np.array_equal(t1.astype(np.float32).astype(np.float64), t1)
        near_rays = rays.copy()
        near_rays[:, 7] = t1
        near = O.trace_combined(bvh, cas, near_rays, O.make_params(mode=0), 32)
        rest_rays = rays.copy()
        rest_rays[:, 3] = t1
        rest = O.trace_combined(bvh, cas, rest_rays, O.make_params(mode=mode, m_near=0.0, m_far=2.0), 32)
        if mode == 1:
            # with m_near > 0 the field sub-interval [t_1, t_max] is empty when t_1 = t_max
            # (with m_near = 0 it would be the closed point t_max): a miss there
            empty = t1 >= rays[:, 7]
            rest["tracer"][empty] = 0
            rest["t"][empty] = np.inf
            rest["prim"][empty] = -1
        got = rest.copy()
        hit = near["tracer"] == 1
        got[hit] = near[hit]
        assert 0 < hit.sum() < rays.shape[0], (mode, m)
        for f in ("tracer", "prim"):
            np.testing.assert_array_equal(got[f], ref[f], err_msg=f"{f} mode={mode} m={m}")
        fin = np.isfinite(ref["t"])
        np.testing.assert_array_equal(np.isfinite(got["t"]), fin)
        np.testing.assert_array_equal(got["t"][fin], ref["t"][fin])
        np.testing.assert_array_equal(got["u"][hit], ref["u"][hit])
        np.testing.assert_array_equal(got["v"][hit], ref["v"][hit])
