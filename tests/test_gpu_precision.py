"""Full-size parity of the precision configuration: the 8,201,612-triangle scene
(40 x 8 x 40 m room), a 512^3 grid baked in float32 and stored again in float16,
1080p GI rays traced in one call as the precision workload runs them, checked on
a seeded sample of rays that the CPU checker computes one by one (its own BVH
and its own exact bake of the voxels each sampled ray touches).

float32 grid: against the checker's float march, at the bar of the frame scene.
float16 grid: against the checker's fp64 query.  Storing the field in float16
moves its values by up to 2^-11 relative, so a field march may take a different
last step; the bar is the stated 1e-3 relative on field-resolved t (99 % of the
rays both resolve with the field), and triangle-resolved hits are held to the
usual bar."""
import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import check_bvh_resolved, check_sdf_resolved, gpu_hits_to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SAMPLE = 512


@pytest.fixture(scope="module")
def precision():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("precision")
    assert s.n_tris == 8201612
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    g32 = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    sdf32 = rq.rt_sdf_create(g32, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf32, rq.BAKE_BVH)
    g16 = g32.half()
    sdf16 = rq.rt_sdf_create(g16, s.lo, s.hi)
    rq.rt_sdf_prepare(sdf16)
    rays = R.gi_rays(s, 1920 * 1080, 7, 30.0)
    rays_d = torch.from_numpy(rays).cuda()
    bvh = O.BVH(s.verts, s.tris)
    ogrid = O.Grid(s.lo, s.hi, [n, n, n], src=bvh)
    sample = np.sort(np.random.default_rng(13).choice(rays.shape[0], N_SAMPLE, replace=False))
    return dict(rq=rq, s=s, scene=scene, sdf32=sdf32, sdf16=sdf16, rays=rays, rays_d=rays_d, bvh=bvh,
                ogrid=ogrid, sample=sample)


def _device(w, sdf, m):
    rq = w["rq"]
    hits = rq.rt_trace_combined(w["scene"], sdf, w["rays_d"], rq.split_params(mode=rq.MODE_SPLIT1, m_near=m))
    g_all = gpu_hits_to_numpy(hits)
    assert not np.any(g_all["flags"] & rq.FLAG_STACK_OVERFLOW)
    return {k: v[w["sample"]] for k, v in g_all.items()}


def test_precision_f32_matches_the_float_checker(precision):
    w = precision
    g = _device(w, w["sdf32"], 2.0)
    rays = w["rays"][w["sample"]]
    o = O.trace_combined(w["bvh"], w["ogrid"], rays, O.make_params(mode=1, m_near=2.0), precision=32)
    same = g["tracer"] == o["tracer"]
    assert same.mean() >= 0.995
    check_bvh_resolved(g, o, rays, w["s"].verts, w["s"].tris, sel=same & (o["tracer"] == 1))
    check_sdf_resolved(g, o, sel=same & (o["tracer"] == 2), max_flip_frac=0.005)


@pytest.mark.parametrize("m", [0.0, 2.0])
def test_precision_f16_within_tolerance_of_fp64(precision, m):
    w = precision
    g = _device(w, w["sdf16"], m)
    rays = w["rays"][w["sample"]]
    o = O.trace_combined(w["bvh"], w["ogrid"], rays, O.make_params(mode=1, m_near=m), precision=64)
    same = g["tracer"] == o["tracer"]
    assert same.mean() >= 0.99
    check_bvh_resolved(g, o, rays, w["s"].verts, w["s"].tris, sel=same & (o["tracer"] == 1))
    both = same & (o["tracer"] == 2)
    assert both.sum() >= 0.5 * N_SAMPLE
    rel = np.abs(g["t"][both] - o["t"][both]) / np.maximum(1.0, np.abs(o["t"][both]))
    assert np.quantile(rel, 0.99) <= 1e-3
    assert np.mean(rel) <= 1e-4
