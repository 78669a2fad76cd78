"""Pins of the checker's field build (Section 3, "Distance Field Generation":
voxelisation, jump flooding, fast sweeping).

The triangle/box test is checked against polygon clipping (an independent
algorithm), the single precision point/triangle distance against the fp64 one,
the voxelisation against brute force, and the flooded field against closed
forms and against the exact distance it approximates (it can never be
smaller: every site is a real triangle).
"""
import numpy as np
import pytest

import oracle as O
from synth import scene as S


def _clip_nonempty(tri, lo, hi, eps=0.0):
    """Sutherland-Hodgman clip of a triangle by the box [lo, hi] (fp64): True
    when anything is left (within eps of the box)."""
    poly = [np.asarray(v, dtype=np.float64) for v in tri]
    for a in range(3):
        for side, bound in ((1, hi[a] + eps), (-1, lo[a] - eps)):
            out = []
            m = len(poly)
            for i in range(m):
                cur, nxt = poly[i], poly[(i + 1) % m]
                fc, fn = side * (cur[a] - bound), side * (nxt[a] - bound)
                if fc <= 0:
                    out.append(cur)
                if (fc < 0 < fn) or (fn < 0 < fc):
                    t = fc / (fc - fn)
                    out.append(cur + t * (nxt - cur))
            poly = out
            if not poly:
                return False
    return True


def _box_tri_gap(tri, lo, hi):
    """Smallest eps for which the eps-grown box meets the triangle, by bisection
    on the clipping test (for excluding near-touching cases)."""
    if _clip_nonempty(tri, lo, hi):
        return 0.0
    a, b = 0.0, 10.0
    for _ in range(40):
        m = 0.5 * (a + b)
        if _clip_nonempty(tri, lo, hi, m):
            b = m
        else:
            a = m
    return b


def test_triangle_box_test_agrees_with_polygon_clipping():
    rng = np.random.default_rng(60)
    checked = overlaps = 0
    for _ in range(4000):
        c = rng.uniform(-1, 1, 3).astype(np.float32)
        hs = rng.uniform(0.05, 0.5, 3).astype(np.float32)
        tri = rng.uniform(-1.5, 1.5, (3, 3)).astype(np.float32)
        if rng.random() < 0.3:  # small triangles near the box too
            tri = (c + rng.uniform(-0.6, 0.6, 3) + 0.2 * rng.normal(size=(3, 3))).astype(np.float32)
        lo, hi = c.astype(np.float64) - hs, c.astype(np.float64) + hs
        gap = _box_tri_gap(tri.astype(np.float64), lo, hi)
        if 0.0 < gap < 1e-4:
            continue  # touching within float rounding: either answer is right
        got = O.tri_box_overlap(c, hs, tri[0], tri[1], tri[2])
        assert got == (gap == 0.0), (c, hs, tri, gap)
        checked += 1
        overlaps += got
    assert checked > 3500 and 0.1 < overlaps / checked < 0.9


def test_single_precision_triangle_distance_matches_fp64():
    rng = np.random.default_rng(61)
    for _ in range(3000):
        tri = rng.normal(size=(3, 3))
        if rng.random() < 0.2:
            tri[2] = tri[0] + 1e-3 * rng.normal(size=3)  # slivers
        p = rng.normal(size=3) * rng.choice([0.01, 1.0, 10.0])
        tri32, p32 = tri.astype(np.float32), p.astype(np.float32)
        d2f = O.tri_dist2_f(p32, tri32[0], tri32[1], tri32[2])
        ref = O.sdf_points_brute(tri32.astype(np.float64), np.array([[0, 1, 2]], dtype=np.int32),
                                 p32.astype(np.float64)[None])[0] ** 2
        assert d2f == pytest.approx(ref, rel=2e-4, abs=1e-9)


def _grid(s, n):
    return O.Grid(s.lo, s.hi, [n, n, n], values=np.zeros(n ** 3))


def _points_f32_as_f64(s, n):
    """Sample positions as the build computes them (float fma of i, h, lo)."""
    lo = np.asarray(s.lo, dtype=np.float32)
    hi = np.asarray(s.hi, dtype=np.float32)
    h = (hi - lo) / np.float32(n - 1)
    i = np.arange(n, dtype=np.float32)
    k, j, ii = np.meshgrid(i, i, i, indexing="ij")
    P = np.stack([ii * h[0] + lo[0], j * h[1] + lo[1], k * h[2] + lo[2]], axis=-1).reshape(-1, 3)
    return P.astype(np.float64), h.astype(np.float64)


def test_voxelisation_marks_exactly_the_overlapped_voxels():
    """Stage 1 against brute force: a sample has a site iff some triangle meets
    its voxel box (side h (1 + 2^-8)), and the site is the nearest of the
    triangles that do."""
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = 12
    sites = O.df_sites(bvh, _grid(s, n), stage=1)
    P, h = _points_f32_as_f64(s, n)
    V = s.verts.astype(np.float32).astype(np.float64)
    F = s.tris
    rng = np.random.default_rng(62)
    sel = rng.choice(P.shape[0], 400, replace=False)
    checked = surface = 0
    hs = (0.5 * h.astype(np.float32) + h.astype(np.float32) / np.float32(512)).astype(np.float64)
    for idx in sel:
        lo, hi = P[idx] - hs, P[idx] + hs
        best, best_d2, ambiguous = -1, np.inf, False
        for t in range(F.shape[0]):
            tri = V[F[t]]
            if np.any(tri.max(axis=0) < lo - 1e-3) or np.any(tri.min(axis=0) > hi + 1e-3):
                continue
            gap = _box_tri_gap(tri, lo, hi)
            if 0.0 < gap < 1e-5:
                ambiguous = True
                continue
            if gap == 0.0:
                d2 = O.sdf_points_brute(V, F[t:t + 1], P[idx][None])[0] ** 2
                if d2 < best_d2 - 1e-12:
                    best, best_d2 = t, d2
                elif abs(d2 - best_d2) <= 1e-12:
                    ambiguous = True
        if ambiguous:
            continue
        assert sites[idx] == best, (idx, sites[idx], best)
        checked += 1
        surface += best >= 0
    assert checked > 300 and surface > 30


@pytest.mark.parametrize("where", ["middle", "end"])
def test_one_triangle_floods_everywhere_with_the_exact_distance(where):
    """Jump flooding alone (stage 2) carries a single site to every sample: from
    one end of a 64-sample line it needs every step 32, 16, ..., 1."""
    V = np.array([[0.3, 0.2, 0.4], [0.9, 0.35, 0.5], [0.5, 0.8, 0.6]])
    if where == "end":
        V = V * [0.02, 1, 1]  # within the first voxels along x
    F = np.array([[0, 1, 2]], dtype=np.int32)
    bvh = O.BVH(V, F)
    lo, hi, n = ([0.0, 0.0, 0.0], [2.0, 1.5, 1.0], [17, 13, 9]) if where == "middle" else \
        ([0.0, 0.0, 0.0], [6.3, 1.0, 1.0], [64, 5, 5])
    g = O.Grid(lo, hi, n, values=np.zeros(int(np.prod(n))))
    for stage in (2, 3):
        sites = O.df_sites(bvh, g, stage=stage)
        assert np.all(sites == 0)
    phi = O.df_field(bvh, g, sites)
    exact = O.sdf_points_brute(V, F, O.grid_points(lo, hi, n))
    np.testing.assert_allclose(np.abs(phi), np.abs(exact), atol=1e-12)


def test_empty_room_field_is_the_distance_to_the_nearest_wall():
    V, F = S.room_mesh(4.0, 3.0, 5.0)
    bvh = O.BVH(V, F)
    lo, hi, n = np.array([0.0, 0.0, 0.0]), np.array([4.0, 3.0, 5.0]), [21, 16, 26]
    g = O.Grid(lo, hi, n, values=np.zeros(int(np.prod(n))))
    phi = O.df_field(bvh, g, O.df_sites(bvh, g, stage=3))
    P = O.grid_points(lo, hi, n)
    wall = np.minimum(P - lo, hi - P).min(axis=1)
    np.testing.assert_allclose(phi, wall, atol=1e-9)


@pytest.fixture(scope="module")
def tiny_build():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = 24
    g = _grid(s, n)
    stages = {st: O.df_sites(bvh, g, stage=st) for st in (1, 2, 3)}
    P = O.grid_points(s.lo, s.hi, [n] * 3)
    exact, feat = bvh.sdf_points(P, feature=True)
    return dict(s=s, bvh=bvh, g=g, n=n, stages=stages, exact=exact, tri=feat // 8, P=P)


def test_flooded_field_never_undershoots_and_is_mostly_exact(tiny_build):
    b = tiny_build
    phi = O.df_field(b["bvh"], b["g"], b["stages"][3])
    h = (np.asarray(b["s"].hi) - np.asarray(b["s"].lo)) / (b["n"] - 1)
    excess = np.abs(phi) - np.abs(b["exact"])
    assert excess.min() > -1e-6                      # a site is a real triangle
    assert np.mean(excess < 1e-9) > 0.97             # and nearly always the nearest one
    assert excess.max() < 0.5 * h.min()              # the rest are near-ties
    near = np.abs(b["exact"]) > 1e-6                 # off the surface the sign is the exact one
    assert np.mean(np.sign(phi[near]) == np.sign(b["exact"][near])) > 0.9999


def test_each_step_only_improves_the_sites(tiny_build):
    """Jump flooding and the sweeps replace a site only by a nearer one."""
    b = tiny_build
    d = {st: np.abs(O.df_field(b["bvh"], b["g"], b["stages"][st])) for st in (1, 2, 3)}
    has1 = b["stages"][1] >= 0
    assert np.all(b["stages"][2] >= 0) and np.all(b["stages"][3] >= 0)
    assert np.all(d[2][has1] <= d[1][has1] + 1e-12)
    assert np.all(d[3] <= d[2] + 1e-12)
    assert np.mean(d[3] < d[2] - 1e-12) > 0  # the sweeps do fix something here


def test_cascade_levels_are_seeded_from_the_coarser_level():
    """A cascade level whose box holds no surface still gets sites, through the
    next coarser level (the coarsest level spans the whole room)."""
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    free = np.array([2.0, 2.2, 2.0])  # 0.8 m from the nearest surface
    n, L, h0 = 16, 4, 0.05            # level 0 spans 0.75 m around it; level 3 holds the room
    cas = O.Cascade(free, h0, n, L, values=np.zeros((L, n, n, n)))
    lo3, hi3 = cas.box(L - 1)
    assert np.all(lo3 <= 0) and np.all(hi3 >= np.asarray(s.room))
    # level 0 holds no surface of its own: every sample is further from the
    # surface than its voxel's half diagonal
    assert np.min(np.abs(bvh.sdf_points(cas.points(0)))) > np.sqrt(3) * 0.51 * h0
    sites = O.df_sites(bvh, cas, stage=3)
    assert np.all(sites >= 0)
    phi = O.df_field(bvh, cas, sites)
    for k in range(L):
        exact = bvh.sdf_points(cas.points(k))
        excess = np.abs(phi[k]) - np.abs(exact)
        assert excess.min() > -1e-6
        assert np.mean(excess < 1e-9) > 0.9, k
        assert excess.max() < 2 * cas.level(k)[1], (k, excess.max())
