"""Full-size parity on every query: the 1080p GI workload on the 2,050,412-
triangle frame scene with a 256^3 grid, in the launch configuration the
benchmark times (all 2,073,600 rays in one call), and one frame of the batching
configuration (primary, AO, GI and shadow batches).

Both sides march the same float grid: the CPU checker bakes the exact field in
fp64 on the host (every sample), the device traces that bake rounded to
float32, and the checker's float march reads the same rounded values.  So
field-resolved records must agree bit for bit, and every other difference must
be a triangle test on a rounding boundary that the fp64 checker confirms
(tests/parity.py states the rules).  The device's own bake is checked against
the same host bake on every sample."""
import math

import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import compare, gpu_hits_to_numpy, segment_ends, tri_spans

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frame():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("frame")
    n = s.spec.grid_n
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    bvh = O.BVH(s.verts, s.tris)
    # the checker's exact bake of every sample, then the same numbers on both sides
    vals64 = O.Grid(s.lo, s.hi, [n, n, n], src=bvh).values(np.arange(n ** 3))
    ogrid = O.Grid(s.lo, s.hi, [n, n, n], values=vals64)
    grid = torch.from_numpy(vals64.astype(np.float32).reshape(n, n, n)).cuda()
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_prepare(sdf)
    rays = R.gi_rays(s, 1920 * 1080, 7, 30.0)
    h = float(np.max((s.hi - s.lo) / (n - 1)))
    hmin = np.float32(np.min((np.float32(s.hi) - np.float32(s.lo)) / np.float32(n - 1)))
    return dict(rq=rq, s=s, scene=scene, grid=grid, sdf=sdf, rays=rays, rays_d=torch.from_numpy(rays).cuda(),
                bvh=bvh, ogrid=ogrid, vals64=vals64, n=n, h=h, eps_hit=np.float32(0.01) * hmin)


def test_fullsize_device_bake_every_sample(frame):
    """The device's exact bake (BVH-pruned, float) against the checker's fp64
    bake on all 16,777,216 samples."""
    rq, s, n = frame["rq"], frame["s"], frame["n"]
    g = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    rq.rt_sdf_bake(frame["scene"], rq.rt_sdf_create(g, s.lo, s.hi), rq.BAKE_BVH)
    got = g.cpu().numpy().reshape(-1).astype(np.float64)
    ref = frame["vals64"]
    err = np.abs(got - ref)
    assert err.max() < 1e-4, err.max()
    far = np.abs(ref) > 1e-4
    assert np.array_equal(np.sign(got[far]), np.sign(ref[far]))


def _check(frame, p_kw, rays, rays_d, hits=None, sdf=None, ogrid=None, precision=32):
    rq = frame["rq"]
    p = rq.split_params(**p_kw)
    if hits is None:
        hits = rq.rt_trace_combined(frame["scene"], sdf or frame["sdf"], rays_d, p)
    g = gpu_hits_to_numpy(hits)
    assert not np.any(g["flags"] & (rq.FLAG_STACK_OVERFLOW | rq.FLAG_ITER_LIMIT))
    mode = p_kw.get("mode", 1)
    kw = dict(mode=mode, any_hit=p_kw.get("any_hit", False), m_near=p_kw.get("m_near", 2.0),
              m_far=p_kw.get("m_far", 2.0))
    o = O.trace_combined(frame["bvh"], ogrid or frame["ogrid"], rays, O.make_params(**kw), precision=precision)
    ends = segment_ends(rays, mode, kw["m_near"], kw["m_far"], frame["h"])
    return compare(g, o, rays, frame["s"].verts, frame["s"].tris, any_hit=kw["any_hit"], ends=ends,
                   spans=tri_spans(mode), eps_hit=frame["eps_hit"])


@pytest.mark.parametrize("m", [0.0, 2.0, math.inf])
def test_fullsize_combined_every_ray(frame, m):
    rep = _check(frame, dict(mode=1, m_near=m), frame["rays"], frame["rays_d"])
    print(f"m={m}: {rep}")
    # the same grid on both sides: field-resolved records are bit-identical
    assert rep["sdf_bit_equal"] == 1.0, rep


@pytest.mark.parametrize("t_ao", [0.5, 10.0])
def test_fullsize_ao_rays_both_programs_same_records(frame, t_ao):
    """4,194,304 AO rays (262,144 surface points, 16 cosine rays each, Section 3
    occlusion queries, closest hit) at m = 2 and m = 1.  The default path runs
    the near triangle stage beside the field stage and then a second near launch
    that takes what the first left: at t_ao = 0.5 m the near sub-intervals are
    most of the work and that second launch traces a large share of them; at
    10 m the field stage dominates.  The records must equal those of the
    one-thread-per-query kernel, which traces each query's sub-intervals in
    order, and every 16th query is checked against the checker."""
    rq, s = frame["rq"], frame["s"]
    pts, nn = R.surface_points(s, 1 << 18, 31)
    rays = R.ao_rays(pts, nn, np.full(1 << 18, 16, dtype=np.int64), 32, t_ao, 1e-3 * s.diagonal)
    rays_d = torch.from_numpy(rays).cuda()
    for m in (2.0, 1.0):
        p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
        a = rq.rt_trace_combined(frame["scene"], frame["sdf"], rays_d, p)
        prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE)
        try:
            b = rq.rt_trace_combined(frame["scene"], frame["sdf"], rays_d, p)
        finally:
            rq.rt_set_tuning(prev)
        assert torch.equal(a, b), (t_ao, m)
        idx = np.arange(0, rays.shape[0], 16)
        ti = torch.from_numpy(idx).cuda()
        rep = _check(frame, dict(mode=1, m_near=m), rays[idx], rays_d[ti], hits=a[ti])
        print(f"t_ao={t_ao} m={m}: {rep}")
        assert rep["sdf_bit_equal"] == 1.0, rep


def test_fullsize_one_thread_per_query_same_records(frame):
    """The benchmark also times the one-thread-per-query kernel: same records."""
    rq = frame["rq"]
    for m in (0.0, 2.0, math.inf):
        p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=m)
        a = rq.rt_trace_combined(frame["scene"], frame["sdf"], frame["rays_d"], p)
        prev = rq.rt_set_tuning(kernel=rq.KERNEL_SIMPLE)
        try:
            b = rq.rt_trace_combined(frame["scene"], frame["sdf"], frame["rays_d"], p)
        finally:
            rq.rt_set_tuning(prev)
        assert torch.equal(a, b), m


def test_fullsize_mixed_batches_every_ray(frame):
    """One frame of the batching configuration (primary rays, 1-4 AO rays per
    pixel, one GI ray per pixel, shadow rays to 4 point lights) through
    rt_trace_batches: the same records as one call per batch (closest hit) or
    the same outcome (any hit), and every query of every batch checked against
    the checker."""
    rq = frame["rq"]
    batches = R.mixed_frame(frame["s"], 0, 2.0)
    dev = [(torch.from_numpy(r).cuda(), rq.split_params(**kw)) for _, r, kw in batches]
    outs = rq.rt_trace_batches(frame["scene"], frame["sdf"], dev)
    for (name, rays, kw), (rd, p), got in zip(batches, dev, outs):
        ref = rq.rt_trace_combined(frame["scene"], frame["sdf"], rd, p)
        if p.any_hit:  # any valid intersection may be reported
            assert torch.equal(got[:, 4], ref[:, 4]), name
        else:
            assert torch.equal(got, ref), name
        rep = _check(frame, kw, rays, rd, hits=got)
        print(f"{name} ({rays.shape[0]} rays): {rep}")
        assert rep["sdf_bit_equal"] == 1.0, (name, rep)
