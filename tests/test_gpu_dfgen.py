"""The paper's field build (Section 3, "Distance Field Generation":
voxelisation, jump flooding, fast sweeping) on the device against the CPU
checker.

The sites (the triangle each sample takes its distance from) are decisions
made in single precision on both sides with the same rounding, so they must be
equal after every step; the field values then agree to rounding.  Sizes: the
tiny scene on a 24^3 grid and on a 4-level cascade, the medium scene (25,732
triangles) on 64^3, and the frame scene (2,050,412 triangles) on the paper's
5 x 64^3 cascade.
"""
import numpy as np
import pytest

import oracle as O
from synth import scene as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def tiny():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("tiny")
    return dict(rq=rq, s=s, scene=rq.rt_scene_build(_cuda(s.verts), _cuda(s.tris)), bvh=O.BVH(s.verts, s.tris))


def _check_field(phi_gpu, phi_ref):
    fin = np.isfinite(phi_ref)
    assert np.array_equal(np.isfinite(phi_gpu), fin)
    a, b = phi_gpu[fin], phi_ref[fin]
    near_surface = np.abs(b) < 1e-5
    assert np.all(np.abs(np.abs(a) - np.abs(b)) <= 1e-5 * (1 + np.abs(b)))
    assert np.mean(np.sign(a[~near_surface]) == np.sign(b[~near_surface])) > 0.9999


@pytest.mark.parametrize("stage", [1, 2, 3])
def test_grid_sites_equal_the_checker(tiny, stage):
    rq, s = tiny["rq"], tiny["s"]
    n = 24
    g = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    sdf = rq.rt_sdf_create(g, s.lo, s.hi)
    got = rq.rt_sdf_sites(tiny["scene"], sdf, stage).cpu().numpy().reshape(-1)
    want = O.df_sites(tiny["bvh"], O.Grid(s.lo, s.hi, [n] * 3, values=np.zeros(n ** 3)), stage=stage)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_grid_field_equals_the_checker(tiny, dtype):
    rq, s = tiny["rq"], tiny["s"]
    n = 24
    g = torch.empty((n, n, n), dtype=dtype, device="cuda")
    sdf = rq.rt_sdf_create(g, s.lo, s.hi)
    rq.rt_sdf_bake(tiny["scene"], sdf, rq.BAKE_JFA)
    grid = O.Grid(s.lo, s.hi, [n] * 3, values=np.zeros(n ** 3))
    ref = O.df_field(tiny["bvh"], grid, O.df_sites(tiny["bvh"], grid, stage=3))
    got = g.float().cpu().numpy().reshape(-1).astype(np.float64)
    if dtype == torch.float16:
        ref = ref.astype(np.float16).astype(np.float64)
        fin = np.isfinite(ref)
        assert np.max(np.abs(got[fin] - ref[fin]) / (1 + np.abs(ref[fin]))) < 2e-3
    else:
        _check_field(got, ref)
    # and the cell copy was rebuilt: rays aimed at the sphere hit it
    c = np.asarray(s.objects[0].center)
    o = np.array([[2.0, 1.5, 2.0], [2.5, 2.5, 3.5], [1.0, 0.5, 1.0]])
    d = (c - o) / np.linalg.norm(c - o, axis=1, keepdims=True)
    rays = torch.tensor(np.concatenate([o, np.zeros((3, 1)), d, np.full((3, 1), 10.0)], axis=1),
                        dtype=torch.float32, device="cuda")
    h = rq.hit_fields(rq.rt_trace_sdf(sdf, rays, rq.split_params(mode=rq.MODE_SDF)))
    t_sphere = np.linalg.norm(c - o, axis=1) - s.objects[0].radius
    assert torch.all(h["tracer"] == rq.TRACER_SDF)
    assert np.all(np.abs(h["t"].cpu().numpy() - t_sphere) < 0.1)


def _tiny_cascade(rq, s, dtype=torch.float32):
    center = np.asarray(s.objects[0].center, dtype=np.float32)
    g = torch.empty((4, 16, 16, 16), dtype=dtype, device="cuda")
    return g, rq.rt_cascade_create(g, 0.0625, center), O.Cascade(center.astype(np.float64), 0.0625, 16, 4,
                                                                    values=np.zeros((4, 16, 16, 16)))


@pytest.mark.parametrize("stage", [1, 2, 3])
def test_cascade_sites_equal_the_checker(tiny, stage):
    rq, s = tiny["rq"], tiny["s"]
    g, sdf, cas = _tiny_cascade(rq, s)
    got = rq.rt_sdf_sites(tiny["scene"], sdf, stage).cpu().numpy().reshape(4, -1)
    want = O.df_sites(tiny["bvh"], cas, stage=stage)
    assert np.array_equal(got, want)


def test_cascade_field_equals_the_checker(tiny):
    rq, s = tiny["rq"], tiny["s"]
    g, sdf, cas = _tiny_cascade(rq, s)
    rq.rt_sdf_bake(tiny["scene"], sdf, rq.BAKE_JFA)
    ref = O.df_field(tiny["bvh"], cas, O.df_sites(tiny["bvh"], cas, stage=3))
    _check_field(g.cpu().numpy().reshape(4, -1).astype(np.float64).reshape(-1), ref.reshape(-1))


@pytest.mark.parametrize("offset", [(0.07, 0.0, 0.0), (0.2, -0.13, 0.07), (2.5, 0.3, -0.4)])
def test_rolling_recenter_rebuilds_like_a_fresh_build(tiny, offset):
    rq, s = tiny["rq"], tiny["s"]
    g, sdf, _ = _tiny_cascade(rq, s)
    rq.rt_sdf_bake(tiny["scene"], sdf, rq.BAKE_JFA)
    c1 = (np.asarray(s.objects[0].center, dtype=np.float64) + np.asarray(offset)).astype(np.float32)
    moved = rq.rt_cascade_recenter(tiny["scene"], sdf, c1)
    assert moved >= 1
    g2 = torch.empty_like(g)
    fresh = rq.rt_cascade_create(g2, 0.0625, c1)
    rq.rt_sdf_bake(tiny["scene"], fresh, rq.BAKE_JFA)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)
    cas = O.Cascade(c1.astype(np.float64), 0.0625, 16, 4, values=np.zeros((4, 16, 16, 16)))
    want = O.df_sites(tiny["bvh"], cas, stage=3)
    assert np.array_equal(rq.rt_sdf_sites(tiny["scene"], sdf, 3).cpu().numpy().reshape(4, -1), want)


def test_medium_scene_sites_equal_the_checker():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("medium")
    scene = rq.rt_scene_build(_cuda(s.verts), _cuda(s.tris))
    bvh = O.BVH(s.verts, s.tris)
    n = 64
    g = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    sdf = rq.rt_sdf_create(g, s.lo, s.hi)
    got = rq.rt_sdf_sites(scene, sdf, 3).cpu().numpy().reshape(-1)
    grid = O.Grid(s.lo, s.hi, [n] * 3, values=np.zeros(n ** 3))
    want = O.df_sites(bvh, grid, stage=3)
    assert np.array_equal(got, want)
    rq.rt_sdf_bake(scene, sdf, rq.BAKE_JFA)
    _check_field(g.cpu().numpy().reshape(-1).astype(np.float64), O.df_field(bvh, grid, want))


def test_frame_scene_cascade_sites_equal_the_checker():
    """The paper's combined-mode cascade (5 x 64^3, 0.1 m) on 2,050,412 triangles,
    in the launch configuration the benchmark times."""
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("frame")
    scene = rq.rt_scene_build(_cuda(s.verts), _cuda(s.tris))
    bvh = O.BVH(s.verts, s.tris)
    eye = np.asarray(s.camera.eye, dtype=np.float32)
    g = torch.empty((5, 64, 64, 64), dtype=torch.float32, device="cuda")
    sdf = rq.rt_cascade_create(g, 0.1, eye)
    rq.rt_sdf_bake(scene, sdf, rq.BAKE_JFA)
    got = rq.rt_sdf_sites(scene, sdf, 3).cpu().numpy().reshape(5, -1)
    cas = O.Cascade(eye.astype(np.float64), float(np.float32(0.1)), 64, 5, values=np.zeros((5, 64, 64, 64)))
    want = O.df_sites(bvh, cas, stage=3)
    assert np.array_equal(got, want)
    ref = O.df_field(bvh, cas, want)
    _check_field(g.cpu().numpy().reshape(-1).astype(np.float64), ref.reshape(-1))
