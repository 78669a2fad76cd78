"""rt_trace_combined_host: rays in host memory, pieces pipelined over copy
streams.  The records must equal those of the device-memory call, whatever the
number of pieces, for pinned and for pageable host memory."""
import numpy as np
import pytest

from synth import rays as R
from synth import scene as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world():
    import paper_2305_07253_gb300 as rq
    s = S.make_scene("tiny")
    scene = rq.rt_scene_build(torch.from_numpy(s.verts).cuda(), torch.from_numpy(s.tris).cuda())
    g = torch.empty((32, 32, 32), dtype=torch.float32, device="cuda")
    sdf = rq.rt_sdf_create(g, s.lo, s.hi)
    rq.rt_sdf_bake(scene, sdf, rq.BAKE_BVH)
    rays = R.gi_rays(s, 10000 + 37, 9, s.diagonal)
    return rq, scene, sdf, rays


@pytest.mark.parametrize("chunks", [0, 1, 3, 7, 64])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_equals_device_call(world, chunks, pinned):
    rq, scene, sdf, rays = world
    n = rays.shape[0]
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    ref = rq.rt_trace_combined(scene, sdf, torch.from_numpy(rays).cuda(), p)
    rays_h = torch.from_numpy(rays)
    hits_h = torch.zeros((n, 6), dtype=torch.int32)
    if pinned:
        rays_h, hits_h = rays_h.pin_memory(), hits_h.pin_memory()
    rays_d = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    hits_d = torch.empty((n, 6), dtype=torch.int32, device="cuda")
    rq.trace_combined_from_host(scene, sdf, rays_h, p, hits_h, rays_d, hits_d, chunks=chunks)
    torch.cuda.synchronize()
    assert torch.equal(hits_h, ref.cpu())


def test_host_pipeline_small_and_invalid(world):
    rq, scene, sdf, rays = world
    p = rq.split_params(mode=rq.MODE_SPLIT1, m_near=2.0)
    few = torch.from_numpy(rays[:3]).pin_memory()
    hits_h = torch.zeros((3, 6), dtype=torch.int32).pin_memory()
    rays_d = torch.empty((3, 8), dtype=torch.float32, device="cuda")
    hits_d = torch.empty((3, 6), dtype=torch.int32, device="cuda")
    rq.trace_combined_from_host(scene, sdf, few, p, hits_h, rays_d, hits_d, chunks=8)  # more pieces than rays
    torch.cuda.synchronize()
    assert torch.equal(hits_h, rq.rt_trace_combined(scene, sdf, few.cuda(), p).cpu())
    with pytest.raises(rq.RtError):
        rq.trace_combined_from_host(scene, sdf, few, p, hits_h, rays_d, hits_d, chunks=65)
