"""The parity classifier (tests/parity.py) itself: it must pass records equal
to the checker's, explain a real rounding-boundary case, and fail a planted
mistake of each kind (a wrong triangle, a lost triangle hit away from every
edge, a wrong field t, a false any-hit record).  Mistakes are planted in a
copy of the checker's own records, on the CPU."""
import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import compare, segment_ends, tri_spans


@pytest.fixture(scope="module")
def world():
    s = S.make_scene("tiny")
    bvh = O.BVH(s.verts, s.tris)
    n = [32, 32, 32]
    grid = O.Grid(s.lo, s.hi, n, values=O.bake_brute(s.verts, s.tris, s.lo, s.hi, n).reshape(-1))
    rays = np.concatenate([R.primary_rays(s, 32, 24), R.gi_rays(s, 768, 9, s.diagonal)])
    h = float(np.max((s.hi - s.lo) / (n[0] - 1)))
    hmin = np.float32(np.min((np.float32(s.hi) - np.float32(s.lo)) / np.float32(n[0] - 1)))
    return dict(s=s, bvh=bvh, grid=grid, rays=rays, h=h, eps=np.float32(0.01) * hmin)


def _as_device(o):
    """The checker's records in the layout of gpu_hits_to_numpy (t rounded to float)."""
    return {"t": o["t"].astype(np.float32).astype(np.float64), "prim": o["prim"].astype(np.int64),
            "u": o["u"].astype(np.float32).astype(np.float64), "v": o["v"].astype(np.float32).astype(np.float64),
            "tracer": o["tracer"].astype(np.int64), "flags": o["flags"].astype(np.int64)}


def _cmp(w, g, o, mode, any_hit=False, check=True):
    ends = segment_ends(w["rays"], mode, 2.0, 2.0, w["h"])
    return compare(g, o, w["rays"], w["s"].verts, w["s"].tris, any_hit=any_hit, ends=ends, spans=tri_spans(mode),
                   eps_hit=w["eps"], check=check)


def test_equal_records_pass(world):
    w = world
    o = O.trace_combined(w["bvh"], w["grid"], w["rays"], O.make_params(mode=1, m_near=2.0), precision=32)
    rep = _cmp(w, _as_device(o), o, 1)
    assert rep["equal"] == 1.0 and rep["unexplained"] == 0
    assert np.any(o["tracer"] == 1) and np.any(o["tracer"] == 2)


def test_planted_mistakes_are_caught(world):
    w = world
    o = O.trace_combined(w["bvh"], w["grid"], w["rays"], O.make_params(mode=0), precision=32)
    tri = np.nonzero(o["tracer"] == 1)[0]
    # a triangle hit far from every edge, not grazing
    inner = [i for i in tri if min(o["u"][i], o["v"][i], 1 - o["u"][i] - o["v"][i]) > 0.05]
    i = inner[0]
    # 1. a wrong triangle id (one the ray does not hit)
    g = _as_device(o)
    others = [k for k in range(w["s"].tris.shape[0]) if not O.tri_check(w["s"].verts, w["s"].tris, w["rays"][i:i + 1],
                                                                         np.array([k]))["hit"][0]]
    g["prim"][i] = others[0]
    assert _cmp(w, g, o, 0, check=False)["unexplained"] == 1
    # 2. a lost triangle hit
    g = _as_device(o)
    g["tracer"][i], g["prim"][i], g["t"][i] = 0, -1, np.inf
    assert _cmp(w, g, o, 0, check=False)["unexplained"] == 1
    # 3. a triangle t off by 1e-3 relative
    g = _as_device(o)
    g["t"][i] *= 1.001
    assert _cmp(w, g, o, 0, check=False)["unexplained"] == 1
    with pytest.raises(AssertionError):
        _cmp(w, g, o, 0)


def test_wrong_field_t_is_caught(world):
    w = world
    o = O.trace_combined(w["bvh"], w["grid"], w["rays"], O.make_params(mode=3), precision=32)
    i = np.nonzero(o["tracer"] == 2)[0][0]
    g = _as_device(o)
    g["t"][i] *= 1.01
    rep = _cmp(w, g, o, 3, check=False)
    assert rep["unexplained"] == 1 and rep["sdf_bit_equal"] < 1.0


def test_edge_ray_difference_is_explained(world):
    """A ray aimed exactly at the middle of a shared edge may go to either
    triangle (or, in float, to neither): the classifier explains the
    difference as an edge case confirmed in fp64."""
    w = world
    s = w["s"]
    V = s.verts.astype(np.float64)
    a, b = s.tris[0][0], s.tris[0][1]
    mid = 0.5 * (V[a] + V[b])
    nrm = np.cross(V[s.tris[0][1]] - V[s.tris[0][0]], V[s.tris[0][2]] - V[s.tris[0][0]])
    nrm /= np.linalg.norm(nrm)
    o_pt = mid + 0.5 * nrm
    ray = R.pack(o_pt[None], -nrm[None], 0.0, 2.0)
    rays = np.repeat(ray, 2, axis=0)
    o = O.trace_combined(w["bvh"], None, rays, O.make_params(mode=0))
    assert o["tracer"][0] == 1
    g = _as_device(o)
    g["tracer"][0], g["prim"][0], g["t"][0] = 0, -1, np.inf   # the float test lost it on the edge
    rep = compare(g, o, rays, s.verts, s.tris, eps_hit=w["eps"], min_equal=0.5)
    assert rep["edge"] == 1 and rep["unexplained"] == 0


def test_any_hit_records_are_validated(world):
    w = world
    o = O.trace_combined(w["bvh"], w["grid"], w["rays"], O.make_params(mode=0, any_hit=True), precision=32)
    i = np.nonzero(o["tracer"] == 1)[0][0]
    g = _as_device(o)
    rep = _cmp(w, g, o, 0, any_hit=True)
    assert rep["unexplained"] == 0
    # a reported triangle that the ray does not hit
    others = [k for k in range(w["s"].tris.shape[0]) if not O.tri_check(w["s"].verts, w["s"].tris, w["rays"][i:i + 1],
                                                                         np.array([k]))["hit"][0]]
    g["prim"][i] = others[0]
    assert _cmp(w, g, o, 0, any_hit=True, check=False)["unexplained"] == 1
