"""Device path against the CPU checker, element by element, on seeded inputs.

Sizes: the tiny scene (344 triangles, 32^3 grid, 64x64 rays plus a ragged
tail) and the medium scene (25,732 triangles, 64^3 grid) span many thread
blocks and a partial last block; the full-size frame workload is sampled in
test_gpu_fullsize.py.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import compare, gpu_hits_to_numpy, segment_ends, tri_spans

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _eps_hit(w):
    s = w.s
    hmin = np.min((np.float32(s.hi) - np.float32(s.lo)) / np.float32(w.n[0] - 1))
    return np.float32(0.01) * np.float32(hmin)


def _cmp(w, g, o, rays, mode, m_near=2.0, m_far=2.0, any_hit=False, **kw):
    h = float(np.max((w.s.hi - w.s.lo) / (w.n[0] - 1)))
    return compare(g, o, rays, w.s.verts, w.s.tris, any_hit=any_hit, ends=segment_ends(rays, mode, m_near, m_far, h),
                   spans=tri_spans(mode), eps_hit=_eps_hit(w), **kw)


class World:
    def __init__(self, name, n_grid, gi_count, ragged=77, bake_oracle=True):
        import paper_2305_07253_gb300 as rq
        self.rq = rq
        self.s = S.make_scene(name)
        s = self.s
        self.n = [n_grid] * 3
        self.scene = rq.rt_scene_build(_cuda(s.verts), _cuda(s.tris))
        self.bvh = O.BVH(s.verts, s.tris)
        self.rays = np.concatenate([R.primary_rays(s), R.gi_rays(s, gi_count + ragged, 5, s.diagonal)])
        self.rays_d = _cuda(self.rays)
        if bake_oracle:
            vals = O.bake_brute(s.verts, s.tris, s.lo, s.hi, self.n).reshape(-1)
        else:
            vals = None
        self.vals64 = vals
        # the checker's grid rounded to float: the same numbers on both sides
        if vals is not None:
            v32 = vals.astype(np.float32)
            self.grid32 = O.Grid(s.lo, s.hi, self.n, values=v32.astype(np.float64))
            self.grid64 = O.Grid(s.lo, s.hi, self.n, values=vals)
            self.gridt = _cuda(v32.reshape(self.n[2], self.n[1], self.n[0]))
            self.sdf = rq.rt_sdf_create(self.gridt, s.lo, s.hi)


TUNINGS = {
    "wavefront-cells": dict(kernel=0, grid_layout=0),
    "wavefront-plain": dict(kernel=0, grid_layout=1),
    "simple-cells": dict(kernel=1, grid_layout=0),
    "simple-plain": dict(kernel=1, grid_layout=1),
    "wavefront-refill1-b64": dict(kernel=0, grid_layout=0, refill_min=1, block=64),
    "wavefront-refill32-b256": dict(kernel=0, grid_layout=0, refill_min=32, block=256, blocks_per_sm=2),
    "wavefront-bvh8": dict(kernel=0, bvh_width=8),
    "wavefront-pairs": dict(kernel=0, grid_layout=2),
    "simple-pairs": dict(kernel=1, grid_layout=2),
    "simple-bvh8": dict(kernel=1, bvh_width=8),
    "wavefront-input-order": dict(kernel=0, order_bits=0),
    "simple-input-order": dict(kernel=1, order_bits=0),
    "wavefront-order1": dict(kernel=0, order_bits=1),
    "simple-order5": dict(kernel=1, order_bits=5),
}


@pytest.fixture(params=list(TUNINGS))
def tuning(request):
    import paper_2305_07253_gb300 as rq
    prev = rq.rt_set_tuning(**TUNINGS[request.param])
    yield request.param
    rq.rt_set_tuning(prev)


@pytest.fixture(scope="module")
def tiny():
    w = World("tiny", 32, 4096)
    w.rq.rt_sdf_prepare(w.sdf)
    return w


@pytest.fixture(scope="module")
def medium():
    return World("medium", 64, 8192, bake_oracle=False)


def test_scene_build_info(tiny, medium):
    for w in (tiny, medium):
        inf = w.scene.info()
        assert inf.n_tris == w.s.n_tris and inf.n_nodes == w.s.n_tris - 1
        assert 1 <= inf.max_depth <= inf.stack_depth
        # the 8-wide tree: fewer levels, at most one node per binary internal node
        assert 1 <= inf.n_wide_nodes <= inf.n_nodes and 1 <= inf.wide_depth < inf.max_depth
        np.testing.assert_allclose(np.array(inf.lo), w.s.verts.min(axis=0), rtol=0, atol=0)
        np.testing.assert_allclose(np.array(inf.hi), w.s.verts.max(axis=0), rtol=0, atol=0)


@pytest.mark.parametrize("which", ["tiny", "medium"])
@pytest.mark.parametrize("any_hit", [False, True])
def test_bvh_parity(which, any_hit, tiny, medium, tuning):
    w = tiny if which == "tiny" else medium
    g = gpu_hits_to_numpy(w.rq.rt_trace_bvh(w.scene, w.rays_d, any_hit=any_hit))
    o = w.bvh.trace(w.rays, any_hit=any_hit)
    # any hit: every reported hit is checked as a real fp64 intersection in [t_min, t_max]
    compare(g, o, w.rays, w.s.verts, w.s.tris, any_hit=any_hit)


def test_bake_parity_tiny(tiny):
    rq = tiny.rq
    s = tiny.s
    for method in (rq.BAKE_BRUTE, rq.BAKE_BVH):
        gt = torch.empty((32, 32, 32), dtype=torch.float32, device="cuda")
        sdf = rq.rt_sdf_create(gt, s.lo, s.hi)
        rq.rt_sdf_bake(tiny.scene, sdf, method)
        torch.cuda.synchronize()
        got = gt.cpu().numpy().reshape(-1).astype(np.float64)
        err = np.abs(got - tiny.vals64)
        assert err.max() < 2e-5, err.max()
    # both methods give the same numbers
    a = torch.empty((32, 32, 32), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    rq.rt_sdf_bake(tiny.scene, rq.rt_sdf_create(a, s.lo, s.hi), rq.BAKE_BRUTE)
    rq.rt_sdf_bake(tiny.scene, rq.rt_sdf_create(b, s.lo, s.hi), rq.BAKE_BVH)
    assert torch.max(torch.abs(a - b)).item() <= 1e-6
    far = torch.abs(a) > 1e-5
    assert torch.equal(torch.sign(a[far]), torch.sign(b[far]))


def test_bake_parity_medium_sampled(medium):
    rq = medium.rq
    s = medium.s
    gt = torch.empty((64, 64, 64), dtype=torch.float32, device="cuda")
    rq.rt_sdf_bake(medium.scene, rq.rt_sdf_create(gt, s.lo, s.hi), rq.BAKE_BVH)
    got = gt.cpu().numpy().reshape(-1).astype(np.float64)
    idx = np.random.default_rng(0).choice(got.size, 4096, replace=False)
    grid = O.Grid(s.lo, s.hi, [64, 64, 64], src=medium.bvh)
    ref = grid.values(idx)
    assert np.max(np.abs(got[idx] - ref)) < 5e-5
    # fp16 storage: the float result rounded once
    gh = torch.empty((64, 64, 64), dtype=torch.float16, device="cuda")
    rq.rt_sdf_bake(medium.scene, rq.rt_sdf_create(gh, s.lo, s.hi), rq.BAKE_BVH)
    assert torch.equal(gh, gt.half())


def test_sdf_trace_matches_float_march(tiny, tuning):
    rq = tiny.rq
    p = rq.split_params(mode=rq.MODE_SDF)
    g = gpu_hits_to_numpy(rq.rt_trace_sdf(tiny.sdf, tiny.rays_d, p))
    o = O.trace_sdf(tiny.grid32, tiny.rays, O.make_params(mode=3), precision=32)
    assert np.array_equal(g["tracer"], o["tracer"])
    rep = _cmp(tiny, g, o, tiny.rays, 3, min_equal=1.0)
    assert rep["sdf_bit_equal"] == 1.0, rep


@pytest.mark.parametrize("m", [0.0, 1.0, 2.0, 4.0, math.inf])
def test_combined_one_split(tiny, m, tuning):
    rq = tiny.rq
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
    g = gpu_hits_to_numpy(rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, p))
    o = O.trace_combined(tiny.bvh, tiny.grid32, tiny.rays, O.make_params(mode=1, m_near=m), precision=32)
    rep = _cmp(tiny, g, o, tiny.rays, 1, m_near=m)
    assert rep["sdf_bit_equal"] == 1.0, rep


def test_endpoint_identities(tiny, tuning):
    """A multiplier of 0 is the pure field trace and +inf the pure triangle trace, bit for bit."""
    rq = tiny.rq
    for mode in (rq.MODE_SPLIT1, rq.MODE_SPLIT2):
        for any_hit in (False, True):
            p0 = rq.split_params(mode=mode, any_hit=any_hit, m_near=0.0, m_far=0.0)
            a = rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, p0)
            b = rq.rt_trace_sdf(tiny.sdf, tiny.rays_d, p0)
            assert torch.equal(a, b)
            pi = rq.split_params(mode=mode, any_hit=any_hit, m_near=math.inf, m_far=math.inf)
            a = rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, pi)
            b = rq.rt_trace_bvh(tiny.scene, tiny.rays_d, any_hit=any_hit)
            if not any_hit:
                assert torch.equal(a, b)
            else:
                ga, gb = gpu_hits_to_numpy(a), gpu_hits_to_numpy(b)
                assert np.array_equal(ga["tracer"] > 0, gb["tracer"] > 0)


def _shadow_rays(s, n, seed):
    src = R.gi_rays(s, n, seed, 1.0)
    g = np.random.default_rng(seed)
    lights = g.uniform([0.3, 0.3, 0.3], np.array(s.room) - 0.3, size=(n, 3))
    o = src[:, :3].astype(np.float64)
    d = lights - o
    dist = np.linalg.norm(d, axis=1)
    d /= dist[:, None]
    return R.pack(o, d, 0.0, dist - 1e-3 * s.diagonal)


@pytest.mark.parametrize("any_hit", [True, False])
def test_combined_two_split_shadow(tiny, any_hit, tuning):
    rq = tiny.rq
    rays = _shadow_rays(tiny.s, 3000, 8)
    p = rq.split_params(mode=rq.MODE_SPLIT2, any_hit=any_hit, m_near=2.0, m_far=2.0)
    g = gpu_hits_to_numpy(rq.rt_trace_combined(tiny.scene, tiny.sdf, _cuda(rays), p))
    o = O.trace_combined(tiny.bvh, tiny.grid32, rays, O.make_params(mode=2, any_hit=any_hit, m_near=2.0, m_far=2.0),
                         precision=32)
    rep = _cmp(tiny, g, o, rays, 2, any_hit=any_hit)
    assert rep["sdf_bit_equal"] == 1.0, rep


def test_fp16_grid_matches_float_march_on_rounded_values(tiny, tuning):
    rq = tiny.rq
    s = tiny.s
    v16 = tiny.vals64.astype(np.float16)
    gt = _cuda(v16.reshape(32, 32, 32))
    sdf16 = rq.rt_sdf_create(gt, s.lo, s.hi)
    rq.rt_sdf_prepare(sdf16)
    grid = O.Grid(s.lo, s.hi, tiny.n, values=v16.astype(np.float64))
    for mode, m in ((rq.MODE_SDF, 0.0), (rq.MODE_SPLIT1, 2.0)):
        p = rq.split_params(mode=mode, m_near=m)
        g = gpu_hits_to_numpy(rq.rt_trace_combined(tiny.scene, sdf16, tiny.rays_d, p))
        o = O.trace_combined(tiny.bvh, grid, tiny.rays, O.make_params(mode=mode, m_near=m), precision=32)
        rep = _cmp(tiny, g, o, tiny.rays, mode, m_near=m)
        assert rep["sdf_bit_equal"] == 1.0, rep


def test_edge_cases(tiny, tuning):
    rq = tiny.rq
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    # empty batch
    empty = torch.empty((0, 8), dtype=torch.float32, device="cuda")
    assert rq.rt_trace_combined(tiny.scene, tiny.sdf, empty, p).shape == (0, 6)
    c = np.array(tiny.s.room) / 2
    rays = np.array([
        [*c, 1.0, 1, 0, 0, 1.0],            # zero-length interval t_min == t_max
        [np.nan, 1, 1, 0, 1, 0, 0, 10],      # NaN origin -> miss
        [-5, -5, -5, 0, 0, 0, 1, 100],       # outside the room, misses everything
        [*c, 0.0, 0, 1, 0, 100],             # axis-aligned direction (zero components)
        [*c, 0.0, 0, 0, -1, 100],
        [*c, 3.0, 1, 0, 0, 2.0],             # t_min > t_max -> miss
    ], dtype=np.float32)
    for mode in range(4):
        pm = rq.split_params(mode=mode, m_near=2.0, m_far=2.0)
        g = gpu_hits_to_numpy(rq.rt_trace_combined(tiny.scene, tiny.sdf, _cuda(rays), pm))
        o = O.trace_combined(tiny.bvh, tiny.grid32, rays, O.make_params(mode=mode, m_near=2.0, m_far=2.0), 32)
        assert g["tracer"][1] == 0 and g["tracer"][2] == 0 and g["tracer"][5] == 0
        assert np.array_equal(g["tracer"], o["tracer"]), (mode, g["tracer"], o["tracer"])
        hit = g["tracer"] > 0
        np.testing.assert_allclose(g["t"][hit], o["t"][hit], rtol=1e-4)


def test_counted_variant_same_hits(tiny, tuning):
    rq = tiny.rq
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    a = rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, p)
    b, cnt = rq.rt_trace_combined_counted(tiny.scene, tiny.sdf, tiny.rays_d, p)
    assert torch.equal(a, b)
    c = cnt.cpu().numpy()
    assert c[0] > 0 and c[1] > 0 and c[2] > 0 and 0 < c[3] <= tiny.rays.shape[0]


def test_invalid_arguments_raise(tiny):
    rq = tiny.rq
    with pytest.raises(rq.RtError):
        rq.rt_trace_combined(None, tiny.sdf, tiny.rays_d, rq.split_params(mode=rq.MODE_SPLIT1))
    with pytest.raises(rq.RtError):
        rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, rq.split_params(m_near=-1.0))


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def noisy(tiny):
    s = tiny.s
    vals = tiny.vals64 + np.random.default_rng(3).normal(scale=0.01, size=tiny.vals64.size)
    v32 = vals.astype(np.float32)
    gt = _cuda(v32.reshape(32, 32, 32))
    sdf = tiny.rq.rt_sdf_create(gt, s.lo, s.hi)
    tiny.rq.rt_sdf_prepare(sdf)
    grid = O.Grid(s.lo, s.hi, tiny.n, values=v32.astype(np.float64))
    rays = R.gi_rays(s, 1024, 31, s.diagonal)
    return gt, sdf, grid, rays, v32.astype(np.float64)


def test_backward_matches_oracle_adjoint(tiny, noisy, tuning):
    rq = tiny.rq
    gt, sdf, grid, rays, _ = noisy
    p = rq.split_params(mode=rq.MODE_SDF, refine_root=True)
    rd = _cuda(rays)
    hits = rq.rt_trace_combined(None, sdf, rd, p)
    g = gpu_hits_to_numpy(hits)
    t_o, idx, w = O.sdf_root_adjoint(grid, rays, O.make_params(mode=3))
    # refined roots agree
    both = (g["tracer"] == 2) & (idx[:, 0] >= 0)
    np.testing.assert_allclose(g["t"][both], t_o[both], rtol=1e-4, atol=1e-5)
    # keep rays that are far from tangent on both sides, weight them randomly
    _, grad = grid.sample(rays[:, :3].astype(np.float64) + t_o[:, None] * rays[:, 4:7].astype(np.float64))
    gd = np.einsum("ij,ij->i", grad, rays[:, 4:7].astype(np.float64))
    keep = both & (gd < -0.1)
    wt = np.random.default_rng(4).normal(size=len(rays)) * keep
    gg = torch.zeros_like(gt)
    rq.rt_trace_combined_backward(None, sdf, rd, p, hits, _cuda(wt.astype(np.float32)), gg)
    ref = np.zeros(gt.numel())
    np.add.at(ref, idx[keep].reshape(-1), (w[keep] * wt[keep, None]).reshape(-1))
    got = gg.cpu().numpy().reshape(-1).astype(np.float64)
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-2 * scale


def test_autograd_function_matches_central_differences(tiny, noisy):
    rq = tiny.rq
    gt, sdf, grid, rays, host_vals = noisy
    p = rq.split_params(mode=rq.MODE_SDF)
    rd = _cuda(rays[:256])
    gparam = gt.clone().requires_grad_(False)
    sdf2 = rq.rt_sdf_create(gparam, sdf.lo, sdf.hi)
    x = gparam.requires_grad_(True)
    t, hits = rq.SdfHitDistance.apply(x, rd, None, sdf2, p)
    ok = torch.isfinite(t)
    loss = (t[ok] ** 2).sum()
    loss.backward()
    assert x.grad is not None and torch.isfinite(x.grad).all()
    # central differences of the checker's fp64 refined root on the voxels with the largest gradient
    vals = host_vals.copy()  # the grid's values as made on the host
    grad = x.grad.cpu().numpy().reshape(-1)
    top = np.argsort(-np.abs(grad))[:16]
    t0, _, _ = O.sdf_root_adjoint(O.Grid(sdf.lo, sdf.hi, tiny.n, values=vals), rays[:256], O.make_params(mode=3))
    fin = np.isfinite(t0)
    for vi in top:
        d = 1e-4
        vp = vals.copy(); vp[vi] += d
        vm = vals.copy(); vm[vi] -= d
        tp, _, _ = O.sdf_root_adjoint(O.Grid(sdf.lo, sdf.hi, tiny.n, values=vp), rays[:256], O.make_params(mode=3))
        tm, _, _ = O.sdf_root_adjoint(O.Grid(sdf.lo, sdf.hi, tiny.n, values=vm), rays[:256], O.make_params(mode=3))
        m = fin & np.isfinite(tp) & np.isfinite(tm) & ok.cpu().numpy()
        fd = np.sum((tp[m] ** 2 - tm[m] ** 2)) / (2 * d)
        assert grad[vi] == pytest.approx(fd, rel=1e-2, abs=1e-3 * np.abs(grad).max())


def test_tunings_give_identical_hits(tiny, medium):
    """Results do not depend on the launch tuning: every kernel/layout/refill setting
    returns the same hit records, bit for bit."""
    rq = tiny.rq
    for w in (tiny,):
        for mode, m in ((rq.MODE_SPLIT1, 2.0), (rq.MODE_SPLIT2, 2.0), (rq.MODE_BVH, 0.0), (rq.MODE_SDF, 0.0)):
            for any_hit in (False, True):
                p = rq.split_params(mode=mode, m_near=m, m_far=m, any_hit=any_hit)
                ref = None
                for name, kw in TUNINGS.items():
                    prev = rq.rt_set_tuning(**kw)
                    try:
                        h = rq.rt_trace_combined(w.scene, w.sdf, w.rays_d, p)
                    finally:
                        rq.rt_set_tuning(prev)
                    if any_hit:
                        h = h[:, 4] > 0  # which valid hit is reported may differ; hit/miss may not
                    if ref is None:
                        ref = h
                    else:
                        assert torch.equal(h, ref), (name, mode, any_hit)


def test_sdf_prepare_tracks_grid_updates(tiny):
    """The cell copy is what the traces read: after writing the grid, prepare refreshes it."""
    rq = tiny.rq
    s = tiny.s
    g = tiny.gridt.clone()
    sdf = rq.rt_sdf_create(g, s.lo, s.hi)
    rq.rt_sdf_prepare(sdf)
    p = rq.split_params(mode=rq.MODE_SDF)
    a = rq.rt_trace_sdf(sdf, tiny.rays_d, p)
    g.add_(0.05)
    rq.rt_sdf_prepare(sdf)
    b = rq.rt_trace_sdf(sdf, tiny.rays_d, p)
    prev = rq.rt_set_tuning(grid_layout=rq.LAYOUT_PLAIN)
    try:
        c = rq.rt_trace_sdf(sdf, tiny.rays_d, p)
    finally:
        rq.rt_set_tuning(prev)
    assert not torch.equal(a, b)
    assert torch.equal(b, c)


def test_timed_variant_reports_each_launch(tiny):
    rq = tiny.rq
    p = rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0)
    a = rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, p)
    b, st = rq.rt_trace_combined_timed(tiny.scene, tiny.sdf, tiny.rays_d, p)
    assert torch.equal(a, b)
    # the query order, then the near stage beside the field and far stages, the near
    # stage's second launch after them, then the merge of the near hits
    assert [x[0] for x in st] == ["order", "bvh_near", "field_split", "bvh_far", "bvh_near_rest", "merge"]
    assert all(ms > 0 for _, ms in st)
    prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE)
    try:
        c, st = rq.rt_trace_combined_timed(tiny.scene, tiny.sdf, tiny.rays_d, p)
    finally:
        rq.rt_set_tuning(prev)
    assert torch.equal(a, c) and [x[0] for x in st] == ["order", "all"]
    prev = rq.rt_set_tuning(order_bits=0)
    try:
        c, st = rq.rt_trace_combined_timed(tiny.scene, tiny.sdf, tiny.rays_d, p)
    finally:
        rq.rt_set_tuning(prev)
    assert torch.equal(a, c) and [x[0] for x in st] == ["bvh_near", "field_split", "bvh_far", "bvh_near_rest", "merge"]


@pytest.mark.parametrize("any_hit", [False, True])
def test_zero_multipliers_launch_no_triangle_stage(tiny, any_hit):
    """m = 0 makes a triangle sub-interval empty for every query, so its stage is
    not launched; the records equal the one-thread-per-query kernel's, which
    evaluates every sub-interval."""
    rq = tiny.rq
    cases = [(dict(mode=rq.MODE_SPLIT1, m_near=0.0), ["field_split"]),
             (dict(mode=rq.MODE_SPLIT2, m_near=0.0, m_far=2.0), ["field_split", "bvh_far"]),
             (dict(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=0.0),
              ["field_split", "bvh_near"] if any_hit else ["bvh_near", "field_split"]),
             (dict(mode=rq.MODE_SPLIT2, m_near=0.0, m_far=0.0), ["field_split"])]
    for kw, stages in cases:
        p = rq.split_params(any_hit=any_hit, **kw)
        a, st = rq.rt_trace_combined_timed(tiny.scene, tiny.sdf, tiny.rays_d, p)
        # with a near sub-interval, a closest-hit call takes the query order, runs the
        # near stage beside the field stage (and again after it), then merges the near hits
        conc = kw["m_near"] > 0 and not any_hit
        assert [x[0] for x in st] == (["order"] + stages + ["bvh_near_rest", "merge"] if conc else stages), kw
        prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE)
        try:
            b = rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, p)
        finally:
            rq.rt_set_tuning(prev)
        assert torch.equal(a, b), kw


def _mixed_batches(w, rq):
    s = w.s
    prim = R.primary_rays(s)
    p, nn = R.surface_points(s, 3000, 61)
    bias = 1e-3 * s.diagonal
    gi = R.gi_rays(s, 2500, 62, s.diagonal)
    ao = R.ao_rays(p, nn, np.random.default_rng(1).integers(1, 5, size=p.shape[0]), 63, 0.5, bias)
    lights = np.random.default_rng(2).uniform(0.3, np.array(s.room) - 0.3, size=(4, 3))
    sh = R.shadow_rays(p, nn, lights, 64, bias)
    mk = lambda **kw: rq.split_params(**kw)  # noqa: E731
    c = np.array(s.room) / 2
    odd = np.array([
        [*c, 1.0, 1, 0, 0, 1.0],            # zero-length interval
        [np.nan, 1, 1, 0, 1, 0, 0, 10],      # NaN origin
        [-5, -5, -5, 0, 0, 0, 1, 100],       # outside the room
        [*c, 0.0, 0, 1, 0, 100],             # axis-aligned direction
        [*c, 3.0, 1, 0, 0, 2.0],             # t_min > t_max
    ], dtype=np.float32)
    odd = np.concatenate([odd, gi[:59]])
    # closest-hit split batches with 0 < m_near < inf make the first two launches
    # run side by side; the m_near = inf and m_near = 0 batches then go through
    # that program too, as do the odd (invalid) queries
    return [
        (prim, mk(mode=rq.MODE_BVH)),
        (gi, mk(mode=rq.MODE_SPLIT1, m_near=2.0)),
        (ao, mk(mode=rq.MODE_SPLIT1, m_near=2.0)),
        (sh, mk(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0, any_hit=True)),
        (gi[:1000], mk(mode=rq.MODE_SPLIT2, m_near=1.0, m_far=3.0)),
        (gi[:777], mk(mode=rq.MODE_SPLIT1, m_near=2.0, any_hit=True)),
        (gi[:0], mk(mode=rq.MODE_SDF)),
        (gi[:555], mk(mode=rq.MODE_SDF)),
        (gi[:600], mk(mode=rq.MODE_SPLIT1, m_near=float("inf"))),
        (gi[:300], mk(mode=rq.MODE_SPLIT2, m_near=0.0, m_far=2.0)),
        (odd, mk(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0)),
        (odd, mk(mode=rq.MODE_BVH)),
        (odd, mk(mode=rq.MODE_SPLIT1, m_near=2.0, any_hit=True)),
    ]


def test_batches_equal_one_call_per_batch(tiny, tuning):
    rq = tiny.rq
    batches = [(_cuda(r), p) for r, p in _mixed_batches(tiny, rq)]
    outs = rq.rt_trace_batches(tiny.scene, tiny.sdf, batches)
    for (rays, p), got in zip(batches, outs):
        ref = rq.rt_trace_combined(tiny.scene, tiny.sdf, rays, p)
        if p.any_hit:
            assert torch.equal(got[:, 4] > 0, ref[:, 4] > 0)
            assert torch.equal(got[:, 4] == rq.TRACER_SDF, ref[:, 4] == rq.TRACER_SDF)
        else:
            assert torch.equal(got, ref), (p.mode, p.m_near)


def test_batches_without_near_split_equal_one_call_per_batch(tiny):
    """Without a closest-hit batch with 0 < m_near < inf the four launches run
    in sequence; the records are the same as one call per batch."""
    rq = tiny.rq
    keep = [(r, p) for r, p in _mixed_batches(tiny, rq)
            if p.any_hit or p.mode in (rq.MODE_BVH, rq.MODE_SDF) or not 0 < p.m_near < float("inf")]
    assert len(keep) >= 6
    batches = [(_cuda(r), p) for r, p in keep]
    outs = rq.rt_trace_batches(tiny.scene, tiny.sdf, batches)
    for (rays, p), got in zip(batches, outs):
        ref = rq.rt_trace_combined(tiny.scene, tiny.sdf, rays, p)
        if p.any_hit:
            assert torch.equal(got[:, 4] > 0, ref[:, 4] > 0)
        else:
            assert torch.equal(got, ref), (p.mode, p.m_near)


def test_batches_replay_in_a_cuda_graph(tiny):
    rq = tiny.rq
    batches = [(_cuda(r), p) for r, p in _mixed_batches(tiny, rq)]
    hits = [torch.empty((r.shape[0], 6), dtype=torch.int32, device="cuda") for r, _ in batches]
    with_hits = [(r, p, h) for (r, p), h in zip(batches, hits)]
    rq.rt_trace_batches(tiny.scene, tiny.sdf, with_hits)  # first call sets up pools outside the capture
    ref = [h.clone() for h in hits]
    for h in hits:
        h.fill_(-1)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            rq.rt_trace_batches(tiny.scene, tiny.sdf, with_hits, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        for h in hits:
            h.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(hits, ref):
            assert torch.equal(a, b)


def test_batches_reject_mixed_march_parameters(tiny):
    rq = tiny.rq
    r = tiny.rays_d[:10]
    with pytest.raises(rq.RtError):
        rq.rt_trace_batches(tiny.scene, tiny.sdf, [(r, rq.split_params(max_steps=100)),
                                                   (r, rq.split_params(max_steps=200))])


def test_autotuner_picks_a_valid_tuning(tiny):
    from paper_2305_07253_gb300 import autotune
    rq = tiny.rq
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    space = autotune.default_space()[::7]
    prev = rq.rt_get_tuning()
    try:
        best, results = autotune.autotune(lambda: rq.rt_trace_combined(tiny.scene, tiny.sdf, tiny.rays_d, p),
                                          space=space, reps=2, warmup=1)
        assert len(results) == len(space) and all(ms > 0 for _, ms in results)
        now = rq.rt_get_tuning().as_dict()
        assert all(now[k] == v for k, v in best.items())
    finally:
        rq.rt_set_tuning(prev)


def _check_tree(nodes, tris, n_tris, max_depth, verts, F):
    """Invariants of the exported binary BVH: every triangle is one leaf, every
    child box holds all triangles below it, and no path is deeper than reported."""
    n_nodes = nodes.shape[0]
    child = nodes[:, 12:14].view(np.int32)
    prim = tris[:, 3].view(np.int32)
    assert sorted(prim.tolist()) == list(range(n_tris))
    # triangle vertices in leaf order match the input mesh
    V = verts.astype(np.float32)
    np.testing.assert_array_equal(tris[:, 0:3], V[F[prim, 0]])
    np.testing.assert_array_equal(tris[:, 4:7], V[F[prim, 1]])
    np.testing.assert_array_equal(tris[:, 8:11], V[F[prim, 2]])
    lo_t = np.minimum(np.minimum(tris[:, 0:3], tris[:, 4:7]), tris[:, 8:11])
    hi_t = np.maximum(np.maximum(tris[:, 0:3], tris[:, 4:7]), tris[:, 8:11])
    # bounds of every subtree, bottom-up over an explicit order (children first)
    order, parent_seen = [], np.zeros(n_nodes, dtype=np.int64)
    stack, depth = [(0, 1)], np.zeros(n_nodes, dtype=np.int64)
    leaves_seen = 0
    while stack:
        nd, dpt = stack.pop()
        order.append(nd)
        depth[nd] = dpt
        for c in child[nd]:
            if c >= 0:
                parent_seen[c] += 1
                stack.append((int(c), dpt + 1))
            else:
                leaves_seen += 1
                assert dpt <= max_depth  # internal nodes on the path, root included
    assert leaves_seen == n_tris and len(order) == n_nodes
    assert np.all(parent_seen[1:] == 1) and parent_seen[0] == 0
    box_lo = np.full((n_nodes, 3), np.inf, dtype=np.float32)
    box_hi = np.full((n_nodes, 3), -np.inf, dtype=np.float32)
    for nd in reversed(order):
        for side in (0, 1):
            c = child[nd, side]
            lo = lo_t[~c] if c < 0 else box_lo[c]
            hi = hi_t[~c] if c < 0 else box_hi[c]
            # the box stored for this child in the parent
            sl = np.array([nodes[nd, 0 + 4 * side], nodes[nd, 2 + 4 * side], nodes[nd, 8 + 2 * side]])
            sh = np.array([nodes[nd, 1 + 4 * side], nodes[nd, 3 + 4 * side], nodes[nd, 9 + 2 * side]])
            assert np.all(sl <= lo) and np.all(sh >= hi), (nd, side)
            box_lo[nd] = np.minimum(box_lo[nd], lo)
            box_hi[nd] = np.maximum(box_hi[nd], hi)


@pytest.mark.parametrize("which", ["tiny", "medium"])
def test_exported_tree_is_a_valid_bvh(which, tiny, medium):
    w = tiny if which == "tiny" else medium
    rq = w.rq
    nodes, tris = rq.rt_scene_export(w.scene)
    inf = w.scene.info()
    _check_tree(nodes.cpu().numpy(), tris.cpu().numpy(), inf.n_tris, inf.max_depth, w.s.verts, w.s.tris)


@pytest.mark.parametrize("bvh_width", [2, 8])
def test_no_ray_leaks_through_shared_edges_or_vertices(bvh_width):
    """Watertightness on the device: 100,000-odd rays from inside a closed
    icosphere, each aimed exactly at one of its vertices or edge midpoints, all
    hit (closest and any hit), as the checker's fp64 test does."""
    import paper_2305_07253_gb300 as rq
    V, F = S.icosphere(3)
    V = (V * 2.0).astype(np.float32)
    E = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    targets = np.concatenate([V, 0.5 * (V[E[:, 0]] + V[E[:, 1]])]).astype(np.float64)
    reps = 100_000 // targets.shape[0] + 1
    tg = np.repeat(targets, reps, axis=0)
    origins = np.random.default_rng(21).uniform(-0.5, 0.5, size=tg.shape)
    d = tg - origins
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([origins, np.zeros((len(d), 1)), d, np.full((len(d), 1), 1e30)], axis=1).astype(np.float32)
    assert rays.shape[0] >= 100_000
    scene = rq.rt_scene_build(_cuda(V), _cuda(F.astype(np.int32)))
    prev = rq.rt_set_tuning(bvh_width=bvh_width)
    try:
        for any_hit in (False, True):
            g = gpu_hits_to_numpy(rq.rt_trace_bvh(scene, _cuda(rays), any_hit=any_hit))
            assert np.all(g["tracer"] == rq.TRACER_BVH), int(np.sum(g["tracer"] != rq.TRACER_BVH))
    finally:
        rq.rt_set_tuning(prev)
