"""rt_trace_combined_noalloc: the combined query for callers that cannot
allocate device memory during a call (a frame loop that forbids allocation, a
fixed device-memory budget).  It keeps its scratch in one array compiled into
the library, so its results must match rt_trace_combined's, call after call,
even though every call reuses that array.

This file is collected last on purpose and builds its own inputs, so it passes
alone in a fresh process as well as after the rest of the suite.
"""
import ctypes
import math

import numpy as np
import pytest

from synth import rays as R
from synth import scene as S
from tests.parity import T_REL_BVH, T_REL_SDF, gpu_hits_to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return rq.lib().rt_trace_combined_noalloc(scene.handle, sdf.handle, ctypes.c_void_p(rays_d.data_ptr()),
                                              rays_d.shape[0], ctypes.byref(params),
                                              ctypes.c_void_p(hits.data_ptr()), stream)


def _agree(a, b):
    ga, gb = gpu_hits_to_numpy(a), gpu_hits_to_numpy(b)
    assert np.array_equal(ga["tracer"], gb["tracer"])
    bvh = ga["tracer"] == 1
    sdf = ga["tracer"] == 2
    assert np.array_equal(ga["prim"][bvh], gb["prim"][bvh])
    rel = lambda x, y: np.abs(x - y) / np.maximum(1.0, np.abs(y))  # noqa: E731
    assert np.all(rel(ga["t"][bvh], gb["t"][bvh]) <= T_REL_BVH)
    assert np.all(rel(ga["t"][sdf], gb["t"][sdf]) <= T_REL_SDF)


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
    ]
    for rays, p in calls:
        rd = torch.from_numpy(rays).cuda()
        ref = rq.rt_trace_combined(scene, sdf, rd, p)
        got = torch.full_like(ref, -7)
        assert _noalloc_via_abi(rq, scene, sdf, rd, p, got) == rq.RT_OK, rq.lib().rt_last_error()
        torch.cuda.synchronize()
        _agree(got, ref)


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
