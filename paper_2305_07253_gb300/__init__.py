"""GB300 (sm_103a) combined ray query: Python binding of the C library.

The binding only marshals arguments: every step of every query runs in the
CUDA kernels of `csrc/`, reached through the C entry points declared in
`include/rt_api.h` (same names here).  PyTorch provides device memory and
streams.  There is no CPU path: if the compiled library is missing the first
call raises.

Buffers
  rays  : float32 CUDA tensor (n, 8) = ox oy oz t_min dx dy dz t_max (Eq. 1)
  hits  : int32 CUDA tensor (n, 6) = t | prim | u | v | tracer | flags
          (float fields stored bit-for-bit; see `hit_fields`)
  grid  : float32 or float16 CUDA tensor (nz, ny, nx), samples at lo + (i,j,k) h
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librt_gb300.so")

RT_OK, RT_ERR_INVALID_ARG, RT_ERR_CUDA, RT_ERR_OOM, RT_ERR_DEVICE_LIMIT, RT_ERR_NOT_IMPLEMENTED = range(6)
MODE_BVH, MODE_SPLIT1, MODE_SPLIT2, MODE_SDF = range(4)
TRACER_MISS, TRACER_BVH, TRACER_SDF = range(3)
FLAG_STACK_OVERFLOW, FLAG_STEP_LIMIT, FLAG_ITER_LIMIT = 1, 2, 4
GRID_F32, GRID_F16 = 0, 1
BAKE_AUTO, BAKE_BRUTE, BAKE_BVH, BAKE_JFA = 0, 1, 2, 3

KERNEL_WAVEFRONT, KERNEL_SIMPLE, KERNEL_AUTO = 0, 1, 2
LAYOUT_CELLS, LAYOUT_PLAIN, LAYOUT_PAIRS = 0, 1, 2

EXPORTS = ("rt_scene_build", "rt_scene_info_get", "rt_scene_destroy", "rt_sdf_create", "rt_sdf_destroy",
           "rt_sdf_prepare", "rt_sdf_bake", "rt_trace_bvh", "rt_trace_sdf", "rt_trace_combined",
           "rt_trace_combined_counted", "rt_trace_combined_timed", "rt_trace_combined_noalloc",
           "rt_trace_combined_backward", "rt_trace_batches", "rt_set_tuning", "rt_get_tuning",
           "rt_cascade_create", "rt_cascade_recenter", "rt_cascade_level", "rt_sdf_sites", "rt_trace_combined_host", "rt_scene_export", "rt_last_error",
           "rt_version")


class RtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rt status {status}: {msg}")
        self.status = status


class rt_split_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("any_hit", ctypes.c_int32), ("m_near", ctypes.c_float),
                ("m_far", ctypes.c_float), ("max_steps", ctypes.c_int32), ("hit_eps_vox", ctypes.c_float),
                ("min_step_vox", ctypes.c_float), ("refine_root", ctypes.c_int32)]


class rt_tuning(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("refill_min", ctypes.c_int32), ("grid_layout", ctypes.c_int32), ("refill_min_field", ctypes.c_int32),
                ("bvh_width", ctypes.c_int32), ("order_bits", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class rt_batch(ctypes.Structure):
    _fields_ = [("d_rays", ctypes.c_void_p), ("d_hits", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("params", rt_split_params)]


MAX_BATCHES = 16


class rt_scene_info(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_int64), ("n_verts", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("max_depth", ctypes.c_int32), ("stack_depth", ctypes.c_int32), ("n_wide_nodes", ctypes.c_int64),
                ("wide_depth", ctypes.c_int32), ("pad_", ctypes.c_int32), ("lo", ctypes.c_float * 3),
                ("hi", ctypes.c_float * 3), ("device_bytes", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2305_07253_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        st = ctypes.c_int
        sig = {
            "rt_scene_build": [P, i64, P, i64, P, P],
            "rt_scene_info_get": [P, P],
            "rt_scene_destroy": [P],
            "rt_sdf_create": [P, i32, P, P, P, P],
            "rt_sdf_destroy": [P],
            "rt_sdf_prepare": [P, P],
            "rt_set_tuning": [P],
            "rt_get_tuning": [P],
            "rt_sdf_bake": [P, P, i32, P],
            "rt_trace_bvh": [P, P, i64, i32, P, P],
            "rt_trace_sdf": [P, P, i64, P, P, P],
            "rt_trace_combined": [P, P, P, i64, P, P, P],
            "rt_trace_combined_counted": [P, P, P, i64, P, P, P, P],
            "rt_trace_combined_timed": [P, P, P, i64, P, P, P, P, P, P],
            "rt_trace_combined_noalloc": [P, P, P, i64, P, P, P],
            "rt_trace_batches": [P, P, P, i32, P],
            "rt_trace_combined_backward": [P, P, P, i64, P, P, P, P, P],
            "rt_cascade_create": [P, i32, i32, i32, ctypes.c_float, P, P],
            "rt_cascade_recenter": [P, P, P, P, P],
            "rt_cascade_level": [P, i32, P, P],
            "rt_sdf_sites": [P, P, i32, P, P],
            "rt_trace_combined_host": [P, P, P, i64, P, P, P, P, i32, P],
            "rt_scene_export": [P, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = st
        L.rt_last_error.restype = ctypes.c_char_p
        L.rt_version.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(status: int) -> None:
    if status != RT_OK:
        raise RtError(status, lib().rt_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor | None) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f3(x) -> ctypes.Array:
    return (ctypes.c_float * 3)(*[float(v) for v in x])


def split_params(mode: int = MODE_SPLIT1, any_hit: bool = False, m_near: float = 2.0, m_far: float = 2.0,
                 max_steps: int = 256, hit_eps_vox: float = 0.01, min_step_vox: float = 0.01,
                 refine_root: bool = False) -> rt_split_params:
    return rt_split_params(int(mode), int(any_hit), float(m_near), float(m_far), int(max_steps), float(hit_eps_vox),
                           float(min_step_vox), int(refine_root))


class Scene:
    """rt_scene handle: LBVH over a triangle mesh, on the current CUDA device."""

    def __init__(self, handle: int, n_tris: int):
        self.handle = ctypes.c_void_p(handle)
        self.n_tris = n_tris

    def info(self) -> rt_scene_info:
        inf = rt_scene_info()
        _check(lib().rt_scene_info_get(self.handle, ctypes.byref(inf)))
        return inf

    def close(self) -> None:
        if self.handle and _lib is not None:
            _lib.rt_scene_destroy(self.handle)
        self.handle = None

    def __del__(self):
        self.close()


class Sdf:
    """rt_sdf handle describing a dense grid tensor (nz, ny, nx), or a cascade
    tensor (levels, n, n, n); keeps the tensor alive."""

    def __init__(self, handle: int, grid: torch.Tensor, lo, hi, levels: int = 0, h0: float = 0.0):
        self.handle = ctypes.c_void_p(handle)
        self.grid = grid
        self.lo = tuple(float(v) for v in lo)
        self.hi = tuple(float(v) for v in hi)
        self.levels = levels
        self.h0 = h0

    def close(self) -> None:
        if self.handle and _lib is not None:
            _lib.rt_sdf_destroy(self.handle)
        self.handle = None

    def __del__(self):
        self.close()


def rt_scene_export(scene: Scene, stream=None):
    """(nodes float32 (n_nodes, 16), tris float32 (n_tris, 12)) copies of the
    binary BVH; the int32 fields (children, input indices) are their bit patterns."""
    inf = scene.info()
    nodes = torch.empty((max(inf.n_nodes, 0), 16), dtype=torch.float32, device="cuda")
    tris = torch.empty((inf.n_tris, 12), dtype=torch.float32, device="cuda")
    _check(lib().rt_scene_export(scene.handle, _dptr(nodes) if nodes.numel() else None, _dptr(tris),
                                 _stream(stream)))
    return nodes, tris


def rt_scene_build(verts: torch.Tensor, tris: torch.Tensor, stream=None) -> Scene:
    """verts (nv,3) float32, tris (nt,3) int32, both CUDA.  Synchronises the stream."""
    assert verts.dtype == torch.float32 and tris.dtype == torch.int32
    out = ctypes.c_void_p()
    _check(lib().rt_scene_build(_dptr(verts), verts.shape[0], _dptr(tris), tris.shape[0], _stream(stream),
                                ctypes.byref(out)))
    return Scene(out.value, tris.shape[0])


def rt_sdf_create(grid: torch.Tensor, lo, hi) -> Sdf:
    """Wrap a (nz, ny, nx) float32/float16 CUDA grid spanning the box [lo, hi]."""
    if grid.dim() != 3:
        raise ValueError("grid must be (nz, ny, nx)")
    dtype = {torch.float32: GRID_F32, torch.float16: GRID_F16}[grid.dtype]
    n = (ctypes.c_int32 * 3)(grid.shape[2], grid.shape[1], grid.shape[0])
    out = ctypes.c_void_p()
    _check(lib().rt_sdf_create(_dptr(grid), dtype, _f3(lo), _f3(hi), n, ctypes.byref(out)))
    return Sdf(out.value, grid, lo, hi)


MAX_LEVELS = 8


def rt_cascade_create(grid: torch.Tensor, h0: float, center) -> Sdf:
    """Wrap a (levels, n, n, n) float32/float16 CUDA tensor as a camera-centred
    cascade: level k has voxel h0 * 2^k and lattice origin
    floor(center / h_k) - (n-1)//2 per axis."""
    if grid.dim() != 4 or not (grid.shape[1] == grid.shape[2] == grid.shape[3]):
        raise ValueError("cascade grid must be (levels, n, n, n)")
    dtype = {torch.float32: GRID_F32, torch.float16: GRID_F16}[grid.dtype]
    out = ctypes.c_void_p()
    _check(lib().rt_cascade_create(_dptr(grid), dtype, grid.shape[0], grid.shape[1], float(h0), _f3(center),
                                   ctypes.byref(out)))
    sdf = Sdf(out.value, grid, (0, 0, 0), (0, 0, 0), levels=grid.shape[0], h0=float(h0))
    lo, hi = rt_cascade_box(sdf, sdf.levels - 1)
    sdf.lo, sdf.hi = tuple(lo), tuple(hi)
    return sdf


def rt_cascade_level(sdf: Sdf, k: int):
    """(ilo (3 ints), h) of level k."""
    ilo = (ctypes.c_int32 * 3)()
    h = ctypes.c_float()
    _check(lib().rt_cascade_level(sdf.handle, int(k), ilo, ctypes.byref(h)))
    return tuple(ilo), h.value


def rt_cascade_box(sdf: Sdf, k: int):
    """Box [lo, hi] of level k (float64 of the lattice corners)."""
    ilo, h = rt_cascade_level(sdf, k)
    n = sdf.grid.shape[1]
    return [i * h for i in ilo], [(i + n - 1) * h for i in ilo]


def rt_cascade_recenter(scene: Scene, sdf: Sdf, center, stream=None) -> int:
    """Rolling update to a new centre; returns the number of levels that moved."""
    moved = ctypes.c_int32(0)
    _check(lib().rt_cascade_recenter(scene.handle, sdf.handle, _f3(center), _stream(stream), ctypes.byref(moved)))
    lo, hi = rt_cascade_box(sdf, sdf.levels - 1)
    sdf.lo, sdf.hi = tuple(lo), tuple(hi)
    return moved.value


def rt_sdf_sites(scene: Scene, sdf: Sdf, stage: int = 3, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Site triangle (input index, -1 none) of every sample after step `stage` of
    the paper's field build (1 voxelisation, 2 jump flooding, 3 sweeps): int32,
    shaped like the grid tensor."""
    if out is None:
        out = torch.empty(sdf.grid.shape, dtype=torch.int32, device=sdf.grid.device)
    assert out.dtype == torch.int32 and out.numel() == sdf.grid.numel()
    _check(lib().rt_sdf_sites(scene.handle, sdf.handle, int(stage), _dptr(out), _stream(stream)))
    return out


def rt_sdf_bake(scene: Scene, sdf: Sdf, method: int = BAKE_AUTO, stream=None) -> None:
    """Fill the grid of `sdf` (a dense grid or a cascade): the exact signed distance
    (BAKE_AUTO, BAKE_BVH, BAKE_BRUTE) or the paper's build, voxelisation + jump
    flooding + sweeps (BAKE_JFA).  Also refreshes its cell copy."""
    _check(lib().rt_sdf_bake(scene.handle, sdf.handle, int(method), _stream(stream)))


def rt_sdf_prepare(sdf: Sdf, stream=None) -> None:
    """(Re)build the cell-corner copy of the grid; call after writing the grid tensor."""
    _check(lib().rt_sdf_prepare(sdf.handle, _stream(stream)))


def rt_get_tuning() -> rt_tuning:
    t = rt_tuning()
    _check(lib().rt_get_tuning(ctypes.byref(t)))
    return t


def rt_set_tuning(t: rt_tuning | None = None, **kw) -> rt_tuning:
    """Set launch tuning (process-wide); keyword arguments override fields of `t`
    (default: the current tuning).  Returns the previous tuning."""
    prev = rt_get_tuning()
    new = rt_tuning.from_buffer_copy(t if t is not None else prev)
    for k, v in kw.items():
        setattr(new, k, int(v))
    _check(lib().rt_set_tuning(ctypes.byref(new)))
    return prev


def _rays_hits(rays: torch.Tensor, hits: torch.Tensor | None) -> torch.Tensor:
    if rays.dtype != torch.float32 or rays.dim() != 2 or rays.shape[1] != 8:
        raise ValueError("rays must be a float32 (n, 8) tensor")
    if hits is None:
        hits = torch.empty((rays.shape[0], 6), dtype=torch.int32, device=rays.device)
    elif hits.shape != (rays.shape[0], 6) or hits.dtype != torch.int32:
        raise ValueError("hits must be an int32 (n, 6) tensor")
    return hits


def rt_trace_bvh(scene: Scene, rays: torch.Tensor, any_hit: bool = False, hits: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    hits = _rays_hits(rays, hits)
    _check(lib().rt_trace_bvh(scene.handle, _dptr(rays), rays.shape[0], int(any_hit), _dptr(hits), _stream(stream)))
    return hits


def rt_trace_sdf(sdf: Sdf, rays: torch.Tensor, params: rt_split_params, hits: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    hits = _rays_hits(rays, hits)
    _check(lib().rt_trace_sdf(sdf.handle, _dptr(rays), rays.shape[0], ctypes.byref(params), _dptr(hits),
                              _stream(stream)))
    return hits


def rt_trace_combined(scene: Scene | None, sdf: Sdf | None, rays: torch.Tensor, params: rt_split_params,
                      hits: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    hits = _rays_hits(rays, hits)
    _check(lib().rt_trace_combined(scene.handle if scene else None, sdf.handle if sdf else None, _dptr(rays),
                                   rays.shape[0], ctypes.byref(params), _dptr(hits), _stream(stream)))
    return hits


def rt_trace_combined_counted(scene: Scene | None, sdf: Sdf | None, rays: torch.Tensor, params: rt_split_params,
                              hits: torch.Tensor | None = None, stream=None):
    """Returns (hits, counters) with counters = [nodes, triangles, march steps, field queries] (int64)."""
    hits = _rays_hits(rays, hits)
    counters = torch.zeros(4, dtype=torch.int64, device=rays.device)
    _check(lib().rt_trace_combined_counted(scene.handle if scene else None, sdf.handle if sdf else None,
                                           _dptr(rays), rays.shape[0], ctypes.byref(params), _dptr(hits),
                                           _dptr(counters), _stream(stream)))
    return hits, counters


NOALLOC_MAX_RAYS = 1 << 20


def rt_trace_combined_noalloc(scene: Scene | None, sdf: Sdf | None, rays: torch.Tensor, params: rt_split_params,
                              hits: torch.Tensor, stream=None) -> torch.Tensor:
    """rt_trace_combined without any device allocation (fixed in-library scratch,
    at most NOALLOC_MAX_RAYS queries per call; concurrent calls race).  `hits`
    must be preallocated by the caller."""
    if hits is None:
        raise ValueError("the caller provides the hit buffer")
    hits = _rays_hits(rays, hits)
    _check(lib().rt_trace_combined_noalloc(scene.handle if scene else None, sdf.handle if sdf else None,
                                           _dptr(rays), rays.shape[0], ctypes.byref(params), _dptr(hits),
                                           _stream(stream)))
    return hits


def rt_trace_batches(scene: Scene | None, sdf: Sdf | None, batches, stream=None) -> list:
    """batches: sequence of (rays, params) or (rays, params, hits); returns the hit tensors.
    One pipeline of persistent stage launches serves all batches (graph-capturable)."""
    if len(batches) > MAX_BATCHES:
        raise ValueError(f"at most {MAX_BATCHES} batches")
    arr = (rt_batch * max(1, len(batches)))()
    outs = []
    for k, bt in enumerate(batches):
        rays, params = bt[0], bt[1]
        hits = _rays_hits(rays, bt[2] if len(bt) > 2 else None)
        outs.append(hits)
        arr[k].d_rays = rays.data_ptr() if rays.numel() else None
        arr[k].d_hits = hits.data_ptr() if hits.numel() else None
        arr[k].n = rays.shape[0]
        arr[k].params = params
    _check(lib().rt_trace_batches(scene.handle if scene else None, sdf.handle if sdf else None, arr, len(batches),
                                  _stream(stream)))
    return outs


STAGE_NAMES = {0: "all", 1: "bvh_full", 2: "bvh_near", 3: "bvh_far", 4: "field_full", 5: "field_split", 6: "order",
               7: "merge", 8: "bvh_near_rest"}


def rt_trace_combined_timed(scene: Scene | None, sdf: Sdf | None, rays: torch.Tensor, params: rt_split_params,
                            hits: torch.Tensor | None = None, stream=None):
    """Returns (hits, [(stage name, ms), ...]) with the device time of each kernel launch."""
    hits = _rays_hits(rays, hits)
    ms = (ctypes.c_float * 6)()
    kinds = (ctypes.c_int32 * 6)()
    n = ctypes.c_int32()
    _check(lib().rt_trace_combined_timed(scene.handle if scene else None, sdf.handle if sdf else None, _dptr(rays),
                                         rays.shape[0], ctypes.byref(params), _dptr(hits), ms, kinds,
                                         ctypes.byref(n), _stream(stream)))
    return hits, [(STAGE_NAMES[kinds[k]], float(ms[k])) for k in range(n.value)]


def rt_trace_combined_backward(scene: Scene | None, sdf: Sdf, rays: torch.Tensor, params: rt_split_params,
                               hits: torch.Tensor, grad_t: torch.Tensor, grad_grid: torch.Tensor,
                               stream=None) -> torch.Tensor:
    """Adds grad_t * dt/dgrid into grad_grid (float32, grid shape) and returns it."""
    assert grad_t.dtype == torch.float32 and grad_grid.dtype == torch.float32
    _check(lib().rt_trace_combined_backward(scene.handle if scene else None, sdf.handle, _dptr(rays), rays.shape[0],
                                            ctypes.byref(params), _dptr(hits), _dptr(grad_t), _dptr(grad_grid),
                                            _stream(stream)))
    return grad_grid


def hit_fields(hits: torch.Tensor) -> dict:
    """Split an (n, 6) int32 hit tensor into named columns (floats reinterpreted)."""
    return {
        "t": hits[:, 0].view(torch.float32),
        "prim": hits[:, 1],
        "u": hits[:, 2].view(torch.float32),
        "v": hits[:, 3].view(torch.float32),
        "tracer": hits[:, 4],
        "flags": hits[:, 5],
    }


def trace_combined_from_host(scene: Scene | None, sdf: Sdf | None, rays_host: torch.Tensor, params: rt_split_params,
                             hits_host: torch.Tensor, rays_dev: torch.Tensor, hits_dev: torch.Tensor,
                             chunks: int = 0, stream=None) -> torch.Tensor:
    """Host-to-host query (rt_trace_combined_host): pinned host rays in, hit records
    out into pinned host memory, the copies of one chunk overlapping the trace of
    the next.  rays_dev / hits_dev are the device staging buffers.  The caller
    synchronises the stream before reading hits_host."""
    assert not rays_host.is_cuda and not hits_host.is_cuda
    assert rays_host.is_contiguous() and hits_host.is_contiguous()
    n = rays_host.shape[0]
    _check(lib().rt_trace_combined_host(scene.handle if scene else None, sdf.handle if sdf else None,
                                        ctypes.c_void_p(rays_host.data_ptr()), n, ctypes.byref(params),
                                        ctypes.c_void_p(hits_host.data_ptr()), _dptr(rays_dev), _dptr(hits_dev),
                                        int(chunks), _stream(stream)))
    return hits_host


class SdfHitDistance(torch.autograd.Function):
    """t of the field-resolved hits as a function of the grid values.

    forward(grid, rays, scene, sdf, params) -> (t, hits): runs rt_trace_combined
    with refine_root=1 (the grid tensor must be the one `sdf` wraps); backward
    runs rt_trace_combined_backward, the adjoint kernel, for dL/dgrid.
    Rays not resolved by the field get t = +inf and zero gradient."""

    @staticmethod
    def forward(ctx, grid, rays, scene, sdf, params):
        if sdf.grid.data_ptr() != grid.data_ptr():
            raise ValueError("grid must be the tensor wrapped by sdf")
        rt_sdf_prepare(sdf)  # the grid may have changed since the last call
        p = rt_split_params.from_buffer_copy(params)
        p.refine_root = 1
        hits = rt_trace_combined(scene, sdf, rays, p)
        t = hit_fields(hits)["t"].clone()
        ctx.save_for_backward(rays, hits)
        ctx.scene, ctx.sdf, ctx.params = scene, sdf, p
        ctx.mark_non_differentiable(hits)
        return t, hits

    @staticmethod
    def backward(ctx, grad_t, _grad_hits):
        rays, hits = ctx.saved_tensors
        g = torch.zeros_like(ctx.sdf.grid, dtype=torch.float32)
        if grad_t is None:
            return g, None, None, None, None
        gt = torch.nan_to_num(grad_t.contiguous().float(), nan=0.0, posinf=0.0, neginf=0.0)
        rt_trace_combined_backward(ctx.scene, ctx.sdf, rays, ctx.params, hits, gt, g)
        return g, None, None, None, None


INF = math.inf
