"""rt_trace_combined_noalloc: the combined query for callers that cannot
allocate device memory during a call (a frame loop that forbids allocation, a
fixed device-memory budget).  It keeps its scratch in one array compiled into
the library and runs the same stage kernels as rt_trace_combined, so its
records must equal rt_trace_combined's bit for bit (closest hit), call after
call, even though every call reuses that array -- also at its 1,048,576-query
limit with the three-stage program of two splits.

This file is collected last on purpose and builds its own inputs, so it passes
alone in a fresh process as well as after the rest of the suite.
"""
import ctypes
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle as O
from synth import rays as R
from synth import scene as S
from tests.parity import T_REL_BVH, gpu_hits_to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def world():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("medium")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    grid = torch.empty((64, 64, 64), dtype=torch.float32, device="cuda")
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf)
    return rq, s, scene, sdf


def _noalloc_via_abi(rq, scene, sdf, rays_d, params, hits):
    """Call the C entry point directly (argument marshalling only)."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return rq.lib().rt_trace_combined_noalloc(scene.handle if scene else None, sdf.handle if sdf else None,
                                              ctypes.c_void_p(rays_d.data_ptr()), rays_d.shape[0],
                                              ctypes.byref(params), ctypes.c_void_p(hits.data_ptr()), stream)


def _same(rq, s, rays, p, got, ref):
    if not p.any_hit:
        assert torch.equal(got, ref)
        return
    # any hit: the same outcome; every triangle record a real fp64 intersection
    assert torch.equal(got[:, 4], ref[:, 4])
    g = gpu_hits_to_numpy(got)
    tri = np.nonzero(g["tracer"] == 1)[0]
    chk = O.tri_check(s.verts, s.tris, rays[tri], g["prim"][tri])
    assert np.all(chk["hit"])
    assert np.all(np.abs(g["t"][tri] - chk["t"]) <= T_REL_BVH * np.maximum(1.0, chk["t"]))


def _run(rq, s, scene, sdf, rays, p):
    rd = torch.from_numpy(rays).cuda()
    ref = rq.rt_trace_combined(scene, sdf, rd, p)
    got = torch.full_like(ref, -7)
    assert _noalloc_via_abi(rq, scene, sdf, rd, p, got) == rq.RT_OK, rq.lib().rt_last_error()
    torch.cuda.synchronize()
    _same(rq, s, rays, p, got, ref)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(world):
    rq, s, scene, sdf = world
    calls = [
        (R.gi_rays(s, 60000, 41, s.diagonal), rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)),
        (R.gi_rays(s, 23456, 42, 0.5 * s.diagonal),
         rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=3.0, any_hit=False)),
        (R.gi_rays(s, 777, 43, s.diagonal), rq.split_params(mode=rq.MODE_BVH, m_near=math.inf)),
        # zero multipliers: no triangle stage before the field (one launch), or field then far triangles
        (R.gi_rays(s, 5001, 44, s.diagonal), rq.split_params(mode=rq.MODE_SPLIT1, m_near=0.0)),
        (R.gi_rays(s, 4099, 45, s.diagonal),
         rq.split_params(mode=rq.MODE_SPLIT2, m_near=0.0, m_far=2.0, any_hit=True)),
        (R.gi_rays(s, 3000, 46, s.diagonal),
         rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0, any_hit=True)),
    ]
    for rays, p in calls:
        _run(rq, s, scene, sdf, rays, p)


def test_noalloc_at_its_limit_then_again(world):
    """Exactly the maximum number of queries with the three-stage program (two
    splits, both multipliers > 0: triangles, field, triangles, two queues in
    use), then a smaller three-stage call that must not see the first call's
    leftovers in the shared array."""
    rq, s, scene, sdf = world
    p = rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0)
    big = R.gi_rays(s, rq.NOALLOC_MAX_RAYS, 47, s.diagonal)
    assert big.shape[0] == rq.NOALLOC_MAX_RAYS
    _run(rq, s, scene, sdf, big, p)
    _run(rq, s, scene, sdf, R.gi_rays(s, 12345, 48, s.diagonal), rq.split_params(mode=rq.MODE_SPLIT2, m_near=1.0,
                                                                                   m_far=4.0))


def test_noalloc_rejects_batches_above_its_limit(world):
    rq, s, scene, sdf = world
    rays = torch.from_numpy(R.gi_rays(s, 64, 44, s.diagonal)).cuda()
    hits = torch.empty((64, 6), dtype=torch.int32, device="cuda")
    p = rq.split_params()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the size check happens before anything touches the buffers
    st = rq.lib().rt_trace_combined_noalloc(scene.handle, sdf.handle, ctypes.c_void_p(rays.data_ptr()),
                                            rq.NOALLOC_MAX_RAYS + 1, ctypes.byref(p),
                                            ctypes.c_void_p(hits.data_ptr()), stream)
    assert st == rq.RT_ERR_INVALID_ARG
    assert b"at most" in rq.lib().rt_last_error()


def test_noalloc_rejects_a_cascade_without_cells_after_a_good_call(world):
    """A refused call after a successful one on the same device leaves the
    entry point usable: the next call still equals rt_trace_combined."""
    rq, s, scene, sdf = world
    rays = R.gi_rays(s, 2048, 49, s.diagonal)
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    _run(rq, s, scene, sdf, rays, p)
    cg = torch.zeros((2, 8, 8, 8), dtype=torch.float32, device="cuda")
    cas = rq.rt_cascade_create(cg, 0.5, s.lo + 0.5 * (s.hi - s.lo))
    rd = torch.from_numpy(rays).cuda()
    hits = torch.empty((rays.shape[0], 6), dtype=torch.int32, device="cuda")
    assert _noalloc_via_abi(rq, scene, cas, rd, p, hits) == rq.RT_ERR_INVALID_ARG
    assert b"cell copy" in rq.lib().rt_last_error()
    _run(rq, s, scene, sdf, rays, p)


_NO_GROWTH = textwrap.dedent("""
    import ctypes, sys
    sys.path.insert(0, {root!r})
    import torch
    import paper_2305_07253_gb300 as rq
    from synth import rays as R, scene as S
    s = S.make_scene("medium")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    grid = torch.empty((64, 64, 64), dtype=torch.float32, device="cuda")
    sdf = rq.rt_sdf_create(grid, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf)
    rays = torch.from_numpy(R.gi_rays(s, 200000, 50, s.diagonal)).cuda()
    hits = torch.empty((rays.shape[0], 6), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    params = [rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0), rq.split_params(mode=rq.MODE_SDF),
              rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0, any_hit=True),
              rq.split_params(mode=rq.MODE_BVH)]
    def rnd():
        for p in params:
            for n in (rays.shape[0], 777):
                st = rq.lib().rt_trace_combined_noalloc(scene.handle, sdf.handle, ctypes.c_void_p(rays.data_ptr()),
                                                        n, ctypes.byref(p), ctypes.c_void_p(hits.data_ptr()), stream)
                assert st == 0, rq.lib().rt_last_error()
    rnd()  # first calls: address look-up and the kernels' first launches
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rnd()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print("free bytes", free0, free1)
    assert free1 == free0, (free0, free1)
""")


def test_noalloc_calls_take_no_device_memory():
    """In a fresh process: after the first calls, further calls leave the
    device's free memory unchanged to the byte."""
    r = subprocess.run([sys.executable, "-c", _NO_GROWTH.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("bits", [5, 1])
def test_noalloc_query_order_changes_no_record(world, bits):
    """With a query order the no-allocation entry point keeps the order in
    its fixed array too; at the array's limit its records equal those of the
    allocating entry point traced in input order, any-hit records included
    (a query's traversal does not depend on which other queries run beside
    it)."""
    rq, s, scene, sdf = world
    rays = R.gi_rays(s, rq.NOALLOC_MAX_RAYS, 49, s.diagonal)
    rd = torch.from_numpy(rays).cuda()
    for p in (rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0),
              rq.split_params(mode=rq.MODE_SPLIT2, m_near=2.0, m_far=2.0, any_hit=True)):
        prev = rq.rt_set_tuning(order_bits=0)
        try:
            ref = rq.rt_trace_combined(scene, sdf, rd, p)
        finally:
            rq.rt_set_tuning(prev)
        prev = rq.rt_set_tuning(order_bits=bits)
        try:
            got = torch.full_like(ref, -7)
            assert _noalloc_via_abi(rq, scene, sdf, rd, p, got) == rq.RT_OK, rq.lib().rt_last_error()
            torch.cuda.synchronize()
        finally:
            rq.rt_set_tuning(prev)
        assert torch.equal(got, ref)
