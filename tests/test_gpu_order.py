"""The query order (rt_tuning.order_bits): where a call's first kernel
traces near triangle sub-intervals, it takes each window of 1024 consecutive
queries grouped by the cell of a coarse lattice over the scene's box that
holds the query's origin, instead of in input order.

A query's record does not depend on which queries run beside it or when, so
every record must equal the one traced in input order, bit for bit, any-hit
records included.  Hit buffers start filled with a pattern no record has, so
a query that the order dropped or traced twice (leaving another one out)
shows.  Inputs include ragged sizes (1 to 63 queries: below the 64 the order
skips; 64; within one window of 1024; exactly one; one past; several windows
with a ragged last one), invalid queries (NaN or
infinite origins, zero directions, t_min > t_max), origins far outside the
scene's box, and mixed batches with empty ones among them, whose windows
straddle batches.  Calls the order does not apply to (triangles only, field
only, any hit, m_near of 0 or +inf) must run without it."""
import math

import numpy as np
import pytest

from synth import rays as R
from synth import scene as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BITS = [1, 2, 3, 4, 5]
SENTINEL = -0x2a2a2a2b


@pytest.fixture(scope="module")
def world():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("medium")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    grid = torch.empty((64, 64, 64), dtype=torch.float32, device="cuda")
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf)
    return rq, s, scene, sdf


def _rays(s, n, seed):
    r = np.concatenate([R.gi_rays(s, max(n - 8, 1), seed, s.diagonal), R.primary_rays(s, 4, 2)])[:n].copy()
    if n >= 16:
        r[0, 0] = np.nan                       # invalid: NaN origin
        r[1, 1] = np.inf                       # invalid: infinite origin
        r[2, 4:7] = 0.0                        # invalid: zero direction
        r[3, 3], r[3, 7] = 5.0, 1.0            # invalid: t_min > t_max
        r[4, 0:3] = s.hi + 50.0 * s.diagonal   # far outside the box, pointing back in
        r[4, 4:7] = -(s.hi - s.lo) / np.linalg.norm(s.hi - s.lo)
        r[5, 0:3] = s.lo - 3.0 * s.diagonal    # outside, pointing away
    if n >= 64:
        r[32, 0:3] = s.lo - 7.0 * s.diagonal   # another origin outside the box
        r[32, 4:7] = (s.hi - s.lo) / np.linalg.norm(s.hi - s.lo)
    return r


def _trace(rq, scene, sdf, rd, p, **tuning):
    prev = rq.rt_set_tuning(**tuning)
    try:
        h = torch.full((rd.shape[0], 6), SENTINEL, dtype=torch.int32, device="cuda")
        rq.rt_trace_combined(scene if p.mode != rq.MODE_SDF else None, sdf if p.mode != rq.MODE_BVH else None, rd, p, h)
        torch.cuda.synchronize()
        return h
    finally:
        rq.rt_set_tuning(prev)


PARAMS = {
    "one-split": dict(mode=1, m_near=2.0),
    "two-splits": dict(mode=2, m_near=2.0, m_far=3.0),
    "two-splits-any": dict(mode=2, m_near=2.0, m_far=2.0, any_hit=True),
    "triangles": dict(mode=0),
    "triangles-any": dict(mode=0, any_hit=True),
    "field": dict(mode=3),
    "no-near": dict(mode=1, m_near=0.0),
}


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 63, 64, 257, 1024, 1025, 2049, 4173])
@pytest.mark.parametrize("pname", list(PARAMS))
def test_order_changes_no_record(world, kernel, n, pname):
    rq, s, scene, sdf = world
    rd = torch.from_numpy(_rays(s, n, 60 + n)).cuda()
    p = rq.split_params(**PARAMS[pname])
    ref = _trace(rq, scene, sdf, rd, p, kernel=kernel, order_bits=0)
    assert not bool((ref == SENTINEL).all(dim=1).any())
    for bits in BITS:
        got = _trace(rq, scene, sdf, rd, p, kernel=kernel, order_bits=bits)
        assert torch.equal(got, ref), bits


def test_order_of_a_gi_batch_changes_no_record(world):
    """A batch of the GI shape (one query per pixel in screen-tile order),
    over many windows, with a ragged last one."""
    rq, s, scene, sdf = world
    rd = torch.from_numpy(R.gi_rays(s, 640 * 360 + 17, 71, s.diagonal)).cuda()
    for pname in ("one-split", "two-splits-any", "triangles", "field"):
        p = rq.split_params(**PARAMS[pname])
        ref = _trace(rq, scene, sdf, rd, p, order_bits=0)
        for bits in (3, 4, 5):
            assert torch.equal(_trace(rq, scene, sdf, rd, p, order_bits=bits), ref), (pname, bits)


def test_order_of_mixed_batches_changes_no_record(world):
    """rt_trace_batches orders the queries of all its batches together (as one
    index space, so a window may straddle two batches); empty batches at the
    start, middle and end take no query."""
    rq, s, scene, sdf = world
    specs = [(0, dict(mode=1, m_near=2.0)), (1500, dict(mode=1, m_near=2.0)),
             (0, dict(mode=2, m_near=2.0, m_far=2.0, any_hit=True)),
             (333, dict(mode=2, m_near=2.0, m_far=2.0, any_hit=True)), (97, dict(mode=0)), (1024, dict(mode=3)),
             (0, dict(mode=0))]
    batches = []
    for k, (n, kw) in enumerate(specs):
        rd = torch.from_numpy(_rays(s, n, 80 + k)).cuda() if n else torch.empty((0, 8), device="cuda")
        batches.append((rd, rq.split_params(**kw)))

    def run(**tuning):
        prev = rq.rt_set_tuning(**tuning)
        try:
            outs = [torch.full((rd.shape[0], 6), SENTINEL, dtype=torch.int32, device="cuda") for rd, _ in batches]
            rq.rt_trace_batches(scene, sdf, [(rd, p, h) for (rd, p), h in zip(batches, outs)])
            torch.cuda.synchronize()
            return outs
        finally:
            rq.rt_set_tuning(prev)

    ref = run(order_bits=0)
    for bits in BITS:
        got = run(order_bits=bits)
        for k, (g, r) in enumerate(zip(got, ref)):
            assert torch.equal(g, r), (bits, k)


@pytest.mark.parametrize("pname,applies", [("one-split", True), ("two-splits", True), ("two-splits-any", False),
                                           ("triangles", False), ("triangles-any", False), ("field", False),
                                           ("no-near", False), ("near-inf", False)])
def test_order_runs_only_where_it_applies(world, pname, applies):
    rq, s, scene, sdf = world
    rd = torch.from_numpy(_rays(s, 4173, 92)).cuda()
    kw = PARAMS.get(pname, dict(mode=1, m_near=math.inf))
    p = rq.split_params(**kw)
    prev = rq.rt_set_tuning(order_bits=4, kernel=rq.KERNEL_WAVEFRONT)
    try:
        _, st = rq.rt_trace_combined_timed(scene if p.mode != rq.MODE_SDF else None,
                                           sdf if p.mode != rq.MODE_BVH else None, rd, p)
    finally:
        rq.rt_set_tuning(prev)
    assert (st[0][0] == "order") == applies, st


def test_timed_call_reports_the_order(world):
    rq, s, scene, sdf = world
    rd = torch.from_numpy(_rays(s, 4173, 91)).cuda()
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    prev = rq.rt_set_tuning(order_bits=3, kernel=rq.KERNEL_WAVEFRONT)
    try:
        h, st = rq.rt_trace_combined_timed(scene, sdf, rd, p)
        h31, st31 = rq.rt_trace_combined_timed(scene, sdf, rd[:31], p)  # below 64 queries: not ordered
    finally:
        rq.rt_set_tuning(prev)
    assert [x[0] for x in st] == ["order", "bvh_near", "field_split", "bvh_near_rest", "merge"]
    assert [x[0] for x in st31] == ["bvh_near", "field_split", "bvh_near_rest", "merge"]
    assert all(ms > 0 and math.isfinite(ms) for _, ms in st)
    assert torch.equal(h, _trace(rq, scene, sdf, rd, p, order_bits=0))
    assert torch.equal(h31, h[:31])
