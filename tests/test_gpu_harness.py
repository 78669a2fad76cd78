"""The AO / direct-light harness (paper_2305_07253_gb300.harness; the estimates
of Section 3, "Occlusion Queries" and "GI & Shadow Rays", whose images are
Fig. 2 and Fig. 3) against the same estimates formed here from the CPU
checker's query records, pixel by pixel.

Inputs: the medium scene (25,732 triangles) and its 64^3 grid baked by the
checker in fp64 and rounded to float32 on both sides; a 64 x 48 image whose
visible points come from the checker's fp64 primary hits; 4 AO rays per pixel
(t_ao 0.5 m and 2 m) and shadow rays to 4 point lights.  Forms: triangles
only, combined (m = 2: one split for AO, two splits with any hit for shadows)
and field only.  A pixel's AO and direct light must equal the checker's
wherever its queries are equal (tests/parity.py); the queries that differ must
be explained there, and move the pixel by at most their own share."""
import math

import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import compare, gpu_hits_to_numpy, segment_ends, tri_spans

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W, H, SPP, POWER = 64, 48, 4, 25.0


@pytest.fixture(scope="module")
def world():
    import paper_2305_07253_gb300 as rq
    from paper_2305_07253_gb300 import harness as HN
    s = S.make_scene("medium")
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    bvh = O.BVH(s.verts, s.tris)
    vals64 = O.Grid(s.lo, s.hi, [n, n, n], src=bvh).values(np.arange(n ** 3))
    sdf = rq.rt_sdf_create(torch.from_numpy(vals64.astype(np.float32).reshape(n, n, n)).cuda(), s.lo, s.hi)
    rq.rt_sdf_prepare(sdf)
    ogrid = O.Grid(s.lo, s.hi, [n, n, n], values=vals64)
    prim_rays = R.primary_rays(s, W, H)
    ph = bvh.trace(prim_rays)
    x, nx, seen = HN.visible_points(prim_rays, ph["t"], ph["prim"], s.verts, s.tris)
    h = float(np.max((s.hi - s.lo) / (n - 1)))
    hmin = np.float32(np.min((np.float32(s.hi) - np.float32(s.lo)) / np.float32(n - 1)))
    return dict(rq=rq, HN=HN, s=s, scene=scene, sdf=sdf, bvh=bvh, ogrid=ogrid, x=x[seen], nx=nx[seen],
                h=h, eps=np.float32(0.01) * hmin, bias=1e-3 * s.diagonal, lights=S.free_lights(s))


FORMS = {"triangles": (0, math.inf), "combined": (1, 2.0), "field": (3, 0.0)}


def _check_queries(w, g_hits, rays, mode, m, any_hit):
    o = O.trace_combined(w["bvh"], w["ogrid"], rays, O.make_params(mode=mode, any_hit=any_hit, m_near=m, m_far=m),
                         precision=32)
    rep = compare(gpu_hits_to_numpy(g_hits), o, rays, w["s"].verts, w["s"].tris, any_hit=any_hit,
                  ends=segment_ends(rays, mode, m, m, w["h"]), spans=tri_spans(mode), eps_hit=w["eps"])
    return o, rep["mask_equal"]


@pytest.mark.parametrize("t_ao", [0.5, 2.0])
@pytest.mark.parametrize("form", list(FORMS))
def test_ao_per_pixel_matches_checker_records(world, form, t_ao):
    w = world
    rq, HN = w["rq"], w["HN"]
    mode, m = FORMS[form]
    p = rq.split_params(mode=mode, m_near=m)
    ao, rays_d, hits = HN.ambient_occlusion(w["scene"], w["sdf"] if mode else None, p, w["x"], w["nx"], SPP, t_ao,
                                            seed=51, bias=w["bias"])
    rays = R.ao_rays(w["x"], w["nx"], np.full(w["x"].shape[0], SPP, dtype=np.int64), 51, t_ao, w["bias"])
    assert np.array_equal(rays, rays_d.cpu().numpy())
    o, eq = _check_queries(w, hits, rays, mode, m, False)
    # the checker's estimate: share of each point's rays without a hit
    ao_ref = (o["tracer"] == 0).reshape(-1, SPP).mean(axis=1)
    got = ao.cpu().numpy()
    all_eq = eq.reshape(-1, SPP).all(axis=1)
    assert np.array_equal(got[all_eq], ao_ref[all_eq])
    n_diff = (~eq).reshape(-1, SPP).sum(axis=1)
    assert np.all(np.abs(got - ao_ref) <= n_diff / SPP + 1e-15)
    assert 0.05 < got.mean() < 0.999  # the test sees occlusion


@pytest.mark.parametrize("form", list(FORMS))
def test_direct_light_per_pixel_matches_checker_records(world, form):
    w = world
    rq, HN = w["rq"], w["HN"]
    mode, m = FORMS[form]
    smode = 2 if mode == 1 else mode  # shadow rays: two splits in the combined form
    p = rq.split_params(mode=smode, any_hit=True, m_near=m, m_far=m)
    E, rays_d, hits = HN.direct_light(w["scene"], w["sdf"] if mode else None, p, w["x"], w["nx"], w["lights"],
                                      POWER, w["bias"])
    rays, cos, inv_d2 = R.light_rays(w["x"], w["nx"], w["lights"], w["bias"])
    assert np.array_equal(rays, rays_d.cpu().numpy())
    o, eq = _check_queries(w, hits, rays, smode, m, True)
    L = w["lights"].shape[0]
    vis = (o["tracer"] == 0).reshape(-1, L)
    E_ref = (POWER * vis * cos * inv_d2).sum(axis=1)
    got = E.cpu().numpy()
    all_eq = eq.reshape(-1, L).all(axis=1)
    np.testing.assert_allclose(got[all_eq], E_ref[all_eq], rtol=1e-12, atol=0)
    # a differing shadow query moves the point by at most that light's term
    bound = (POWER * cos * inv_d2 * (~eq).reshape(-1, L)).sum(axis=1)
    assert np.all(np.abs(got - E_ref) <= bound * (1 + 1e-12) + 1e-12 * np.abs(E_ref))
    assert 0.05 < np.mean(vis) < 0.999


def test_one_bounce_combines_direct_and_bounced_light(world):
    """The GI estimate's direct part equals direct_light's; the bounce adds
    non-negative light; every radiance is finite."""
    w = world
    rq, HN = w["rq"], w["HN"]
    s = w["s"]
    V, F = s.verts.astype(np.float64), s.tris
    fn = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    fn = torch.from_numpy(fn / np.linalg.norm(fn, axis=1, keepdims=True)).cuda()
    grid = w["sdf"].grid
    levels = [(grid, tuple(s.lo), tuple(s.hi))]
    gi_p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    sh_p = rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0, any_hit=True)
    out = HN.one_bounce(w["scene"], w["sdf"], gi_p, sh_p, w["x"], w["nx"], fn, levels, w["lights"], POWER, 0.7, 4,
                        seed=52, bias=w["bias"])
    E, _, _ = HN.direct_light(w["scene"], w["sdf"], sh_p, w["x"], w["nx"], w["lights"], POWER, w["bias"])
    assert torch.equal(out["direct"], (0.7 / math.pi) * E)
    rad = out["radiance"]
    assert bool(torch.isfinite(rad).all())
    assert bool((rad >= out["direct"]).all())
    assert float((rad - out["direct"]).sum()) > 0
