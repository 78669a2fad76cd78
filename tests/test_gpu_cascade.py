"""Camera-centred cascade (Section 3, "Distance Field Generation"; split points
from the voxel at the ray's start and end, Section 3, "GI & Shadow Rays"):
device path against the CPU checker on seeded inputs.

Sizes: the tiny scene (344 triangles) with 4 levels of 16^3 centred on its
sphere (voxels 0.0625 to 0.5 m, so that the rays' hits fall in every level; a
centre at the camera, which sits near a wall, leaves the finest levels almost
unused), 64x64 primary rays
plus GI rays with a ragged tail; the full-size frame workload with the paper's
5 x 64^3 cascade (0.1 m smallest voxel) and its field-only variant
(5 x 128^3, 0.05 m) is sampled at the end.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import compare, ends_from_split_points, gpu_hits_to_numpy, tri_spans

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, L, H0 = 16, 4, 0.0625


def _eps_top(h0, levels):
    """The largest float hit threshold of a cascade (its coarsest level's)."""
    return np.float32(0.01) * np.float32(np.float32(h0) * 2.0 ** (levels - 1))


def _cmp(g, o, t12, rays, s, mode, any_hit=False, eps=None):
    return compare(g, o, rays, s.verts, s.tris, any_hit=any_hit, ends=ends_from_split_points(rays, t12),
                   spans=tri_spans(mode), eps_hit=eps if eps is not None else _eps_top(H0, L))


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _level_values(bvh, center, h0, n, levels):
    shell = O.Cascade(center, h0, n, levels, values=np.zeros((levels, n, n, n)))
    return np.stack([bvh.sdf_points(shell.points(k)) for k in range(levels)]).reshape(levels, n, n, n)


class CascWorld:
    def __init__(self):
        import paper_2305_07253_gb300 as rq
        self.rq = rq
        s = self.s = S.make_scene("tiny")
        self.scene = rq.rt_scene_build(_cuda(s.verts), _cuda(s.tris))
        self.bvh = O.BVH(s.verts, s.tris)
        self.center = np.asarray(s.objects[0].center, dtype=np.float32)
        c64 = self.center.astype(np.float64)
        self.vals64 = _level_values(self.bvh, c64, H0, N, L)
        v32 = self.vals64.astype(np.float32)
        self.cas32 = O.Cascade(c64, H0, N, L, values=v32.astype(np.float64))
        self.gridt = _cuda(v32)
        self.sdf = rq.rt_cascade_create(self.gridt, H0, self.center)
        rq.rt_sdf_prepare(self.sdf)
        self.rays = np.concatenate([R.primary_rays(s), R.gi_rays(s, 4096 + 77, 5, s.diagonal)])
        self.rays_d = _cuda(self.rays)


TUNINGS = {
    "wavefront": dict(kernel=0),
    "simple": dict(kernel=1),
    "wavefront-refill1-b64": dict(kernel=0, refill_min=1, refill_min_field=1, block=64),
    "wavefront-bvh8": dict(kernel=0, bvh_width=8),
    "simple-plain-layout": dict(kernel=1, grid_layout=1),
    "wavefront-input-order": dict(kernel=0, order_bits=0),
    "simple-order2": dict(kernel=1, order_bits=2),
}


@pytest.fixture(params=list(TUNINGS))
def tuning(request):
    import paper_2305_07253_gb300 as rq
    prev = rq.rt_set_tuning(**TUNINGS[request.param])
    yield request.param
    rq.rt_set_tuning(prev)


@pytest.fixture(scope="module")
def cw():
    return CascWorld()


def _shadow_rays(s, n, seed):
    src = R.gi_rays(s, n, seed, 1.0)
    g = np.random.default_rng(seed)
    lights = g.uniform([0.3, 0.3, 0.3], np.array(s.room) - 0.3, size=(n, 3))
    o = src[:, :3].astype(np.float64)
    d = lights - o
    dist = np.linalg.norm(d, axis=1)
    d /= dist[:, None]
    return R.pack(o, d, 0.0, dist - 1e-3 * s.diagonal)


def test_rays_cross_several_levels(cw):
    o = O.trace_combined(None, cw.cas32, cw.rays, O.make_params(mode=3), precision=64)
    hit = o["tracer"] == 2
    p = cw.rays[hit, 0:3].astype(np.float64) + o["t"][hit, None] * cw.rays[hit, 4:7].astype(np.float64)
    lv = cw.cas32.level_of(p)
    counts = np.bincount(lv, minlength=L)
    assert np.all(counts > 100), counts


def test_cascade_field_trace_matches_float_march(cw, tuning):
    rq = cw.rq
    g = gpu_hits_to_numpy(rq.rt_trace_sdf(cw.sdf, cw.rays_d, rq.split_params(mode=rq.MODE_SDF)))
    o = O.trace_combined(None, cw.cas32, cw.rays, O.make_params(mode=3), precision=32)
    assert np.array_equal(g["tracer"], o["tracer"])
    rep = compare(g, o, cw.rays, cw.s.verts, cw.s.tris, eps_hit=_eps_top(H0, L), min_equal=1.0)
    assert rep["sdf_bit_equal"] == 1.0, rep


@pytest.mark.parametrize("m", [1.0, 2.0, 4.0])
def test_cascade_combined_one_split(cw, m, tuning):
    rq = cw.rq
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
    g = gpu_hits_to_numpy(rq.rt_trace_combined(cw.scene, cw.sdf, cw.rays_d, p))
    o, t12 = O.trace_combined(cw.bvh, cw.cas32, cw.rays, O.make_params(mode=1, m_near=m), precision=32,
                              split_points=True)
    assert np.any(o["tracer"] == 1) and np.any(o["tracer"] == 2)
    rep = _cmp(g, o, t12, cw.rays, cw.s, 1)
    assert rep["sdf_bit_equal"] == 1.0, rep


@pytest.mark.parametrize("any_hit", [True, False])
def test_cascade_two_split_shadow(cw, any_hit, tuning):
    rq = cw.rq
    rays = _shadow_rays(cw.s, 3000, 8)
    p = rq.split_params(mode=rq.MODE_SPLIT2, any_hit=any_hit, m_near=2.0, m_far=2.0)
    g = gpu_hits_to_numpy(rq.rt_trace_combined(cw.scene, cw.sdf, _cuda(rays), p))
    o, t12 = O.trace_combined(cw.bvh, cw.cas32, rays, O.make_params(mode=2, any_hit=any_hit, m_near=2.0, m_far=2.0),
                              precision=32, split_points=True)
    rep = _cmp(g, o, t12, rays, cw.s, 2, any_hit=any_hit)
    assert rep["sdf_bit_equal"] == 1.0, rep


def test_cascade_endpoint_identities(cw, tuning):
    rq = cw.rq
    for mode in (rq.MODE_SPLIT1, rq.MODE_SPLIT2):
        for any_hit in (False, True):
            p0 = rq.split_params(mode=mode, any_hit=any_hit, m_near=0.0, m_far=0.0)
            a = rq.rt_trace_combined(cw.scene, cw.sdf, cw.rays_d, p0)
            b = rq.rt_trace_sdf(cw.sdf, cw.rays_d, p0)
            assert torch.equal(a, b)
            pi = rq.split_params(mode=mode, any_hit=any_hit, m_near=math.inf, m_far=math.inf)
            a = rq.rt_trace_combined(cw.scene, cw.sdf, cw.rays_d, pi)
            b = rq.rt_trace_bvh(cw.scene, cw.rays_d, any_hit=any_hit)
            if not any_hit:
                assert torch.equal(a, b)
            else:
                ga, gb = gpu_hits_to_numpy(a), gpu_hits_to_numpy(b)
                assert np.array_equal(ga["tracer"] > 0, gb["tracer"] > 0)


def test_cascade_f16_matches_float_march_on_rounded_values(cw, tuning):
    rq = cw.rq
    v16 = cw.vals64.astype(np.float16)
    gt = _cuda(v16)
    sdf16 = rq.rt_cascade_create(gt, H0, cw.center)
    rq.rt_sdf_prepare(sdf16)
    cas = O.Cascade(cw.center.astype(np.float64), H0, N, L, values=v16.astype(np.float64))
    for mode, m in ((rq.MODE_SDF, 0.0), (rq.MODE_SPLIT1, 2.0)):
        p = rq.split_params(mode=mode, m_near=m)
        g = gpu_hits_to_numpy(rq.rt_trace_combined(cw.scene, sdf16, cw.rays_d, p))
        o, t12 = O.trace_combined(cw.bvh, cas, cw.rays, O.make_params(mode=mode, m_near=m), precision=32,
                                  split_points=True)
        rep = _cmp(g, o, t12, cw.rays, cw.s, mode)
        assert rep["sdf_bit_equal"] == 1.0, rep


@pytest.mark.parametrize("method", ["brute", "bvh"])
def test_cascade_bake_matches_exact_distance(cw, method):
    rq = cw.rq
    g = torch.empty((L, N, N, N), dtype=torch.float32, device="cuda")
    sdf = rq.rt_cascade_create(g, H0, cw.center)
    rq.rt_sdf_bake(cw.scene, sdf, rq.BAKE_BRUTE if method == "brute" else rq.BAKE_BVH)
    got = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - cw.vals64)) < 2e-6
    # the bake also built the cell copy: tracing it equals tracing a fresh
    # cascade of the same values prepared explicitly
    p = rq.split_params(mode=rq.MODE_SDF)
    g2 = g.clone()
    sdf2 = rq.rt_cascade_create(g2, H0, cw.center)
    rq.rt_sdf_prepare(sdf2)
    assert torch.equal(rq.rt_trace_sdf(sdf, cw.rays_d, p), rq.rt_trace_sdf(sdf2, cw.rays_d, p))


def test_cascade_level_geometry_matches_checker(cw):
    rq = cw.rq
    for k in range(L):
        ilo, h = rq.rt_cascade_level(cw.sdf, k)
        want_ilo, want_h = cw.cas32.level(k)
        assert list(ilo) == want_ilo.tolist()
        assert h == np.float32(want_h)


@pytest.mark.parametrize("offset", [(0.2, -0.13, 0.07), (0.7, 0.0, -0.4), (3.0, 0.1, 0.0)])
def test_rolling_recenter_equals_fresh_bake(cw, offset):
    """Section 3: a moving camera updates only the cascade slices that changed.
    The rolled cascade holds exactly the values of a full bake at the new
    centre, and traces identically."""
    rq = cw.rq
    g = torch.empty((L, N, N, N), dtype=torch.float32, device="cuda")
    sdf = rq.rt_cascade_create(g, H0, cw.center)
    rq.rt_sdf_bake(cw.scene, sdf, rq.BAKE_BVH)
    c1 = (cw.center.astype(np.float64) + np.asarray(offset)).astype(np.float32)
    before = [rq.rt_cascade_level(sdf, k)[0] for k in range(L)]
    moved = rq.rt_cascade_recenter(cw.scene, sdf, c1)
    ref = O.Cascade(c1.astype(np.float64), H0, N, L, values=np.zeros((L, N, N, N)))
    after = [rq.rt_cascade_level(sdf, k)[0] for k in range(L)]
    assert [list(a) for a in after] == [ref.level(k)[0].tolist() for k in range(L)]
    assert moved == sum(1 for a, b in zip(after, before) if a != b)
    assert moved >= 1
    g2 = torch.empty_like(g)
    fresh = rq.rt_cascade_create(g2, H0, c1)
    rq.rt_sdf_bake(cw.scene, fresh, rq.BAKE_BVH)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    assert torch.equal(rq.rt_trace_combined(cw.scene, sdf, cw.rays_d, p),
                       rq.rt_trace_combined(cw.scene, fresh, cw.rays_d, p))
    # recentring to the same place changes nothing
    assert rq.rt_cascade_recenter(cw.scene, sdf, c1) == 0
    assert torch.equal(g, g2)


def test_cascade_batches_equal_one_call_per_batch(cw):
    rq = cw.rq
    shadow = _cuda(_shadow_rays(cw.s, 1500, 9))
    gi = cw.rays_d
    specs = [(gi, rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)),
             (shadow, rq.split_params(mode=rq.MODE_SPLIT2, any_hit=True, m_near=2.0, m_far=2.0)),
             (gi, rq.split_params(mode=rq.MODE_SDF)),
             (shadow, rq.split_params(mode=rq.MODE_SPLIT2, m_near=1.0, m_far=4.0))]
    outs = rq.rt_trace_batches(cw.scene, cw.sdf, specs)
    for (r, p), h in zip(specs, outs):
        assert torch.equal(h, rq.rt_trace_combined(cw.scene, cw.sdf, r, p))


def test_cascade_noalloc_and_counted_give_the_same_hits(cw):
    rq = cw.rq
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    ref = rq.rt_trace_combined(cw.scene, cw.sdf, cw.rays_d, p)
    assert torch.equal(rq.rt_trace_combined_noalloc(cw.scene, cw.sdf, cw.rays_d, p, torch.empty_like(ref)), ref)
    hits, counts = rq.rt_trace_combined_counted(cw.scene, cw.sdf, cw.rays_d, p)
    assert torch.equal(hits, ref)
    assert counts[2] > 0 and counts[0] > 0


def test_cascade_backward_is_refused(cw):
    rq = cw.rq
    p = rq.split_params(mode=rq.MODE_SDF, refine_root=True)
    hits = rq.rt_trace_sdf(cw.sdf, cw.rays_d, p)
    grad_t = torch.ones(cw.rays_d.shape[0], device="cuda")
    with pytest.raises(rq.RtError, match="cascade"):
        rq.rt_trace_combined_backward(cw.scene, cw.sdf, cw.rays_d, p, hits, grad_t,
                                      torch.zeros_like(cw.gridt))


# --------------------------------------------------------------------------
# full size: the paper's cascades on the frame scene, 1080p GI rays in one call,
# every query; both sides read the checker's fp64 bake of every level sample
# rounded to float32
# --------------------------------------------------------------------------
FRAME_CASCADES = (("combined", 64, 0.1), ("field_only", 128, 0.05))


@pytest.fixture(scope="module")
def frame_cascade():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    center = np.asarray(s.camera.eye, dtype=np.float32)
    bvh = O.BVH(s.verts, s.tris)
    out = dict(rq=rq, s=s, scene=scene, bvh=bvh, center=center)
    for name, n, h0 in FRAME_CASCADES:
        h0f = float(np.float32(h0))
        vals64 = _level_values(bvh, center.astype(np.float64), h0f, n, 5)
        v32 = vals64.astype(np.float32)
        g = _cuda(v32)
        sdf = rq.rt_cascade_create(g, h0, center)
        rq.rt_sdf_prepare(sdf)
        cas = O.Cascade(center.astype(np.float64), h0f, n, 5, values=v32.astype(np.float64))
        out[name] = (g, sdf, cas, vals64, h0f)
    rays = R.gi_rays(s, 1920 * 1080, 7, 30.0)
    out["rays"] = rays
    out["rays_d"] = torch.from_numpy(rays).cuda()
    return out


def test_fullsize_cascade_device_bake_every_sample(frame_cascade):
    rq = frame_cascade["rq"]
    for name, n, h0 in FRAME_CASCADES:
        _, _, _, vals64, _ = frame_cascade[name]
        g = torch.empty((5, n, n, n), dtype=torch.float32, device="cuda")
        rq.rt_sdf_bake(frame_cascade["scene"], rq.rt_cascade_create(g, h0, frame_cascade["center"]), rq.BAKE_BVH)
        got = g.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - vals64)) < 1e-4, name


@pytest.mark.parametrize("name,m", [("combined", 2.0), ("combined", 0.0), ("field_only", 0.0)])
def test_fullsize_cascade_every_ray(frame_cascade, name, m):
    rq = frame_cascade["rq"]
    _, sdf, cas, _, h0 = frame_cascade[name]
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
    g = gpu_hits_to_numpy(rq.rt_trace_combined(frame_cascade["scene"], sdf, frame_cascade["rays_d"], p))
    assert not np.any(g["flags"] & (rq.FLAG_STACK_OVERFLOW | rq.FLAG_ITER_LIMIT))
    rays = frame_cascade["rays"]
    o, t12 = O.trace_combined(frame_cascade["bvh"], cas, rays, O.make_params(mode=1, m_near=m), precision=32,
                              split_points=True)
    rep = _cmp(g, o, t12, rays, frame_cascade["s"], 1, eps=_eps_top(h0, 5))
    print(f"{name} m={m}: {rep}")
    assert rep["sdf_bit_equal"] == 1.0, rep
