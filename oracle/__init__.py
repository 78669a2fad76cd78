"""CPU checker for the combined ray query -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  It wraps `oracle.c` (plain C, fp64 ground truth plus a
single-precision mode of the distance-field step rule) through ctypes and
shares no code with the device library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("oracle.c", "march.inc", "dfgen.inc", "oracle.h")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

HIT_DTYPE = np.dtype([("t", "f8"), ("u", "f8"), ("v", "f8"), ("prim", "i4"), ("tracer", "i4"),
                      ("flags", "u4"), ("steps", "i4"), ("margin", "f8")])
FLAG_STEP_LIMIT = 2


class Params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("any_hit", ctypes.c_int32), ("m_near", ctypes.c_double),
                ("m_far", ctypes.c_double), ("max_steps", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("hit_eps_vox", ctypes.c_double), ("min_step_vox", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no fused multiply-add unless written as fma)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB):
        if os.path.getmtime(_LIB) >= max(os.path.getmtime(s) for s in _SRC):
            return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", os.path.join(_HERE, "oracle.c"), "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            L.or_watertight.argtypes = [P] * 6
            L.or_watertight.restype = ctypes.c_int
            L.or_trace_brute.argtypes = [P, P, i64, P, i64, i32, P]
            L.or_bvh_build.argtypes = [P, i64, P, i64]
            L.or_bvh_build.restype = P
            L.or_bvh_free.argtypes = [P]
            L.or_bvh_node_count.argtypes = [P]
            L.or_bvh_node_count.restype = i64
            L.or_trace_bvh.argtypes = [P, P, i64, i32, i32, P]
            L.or_sdf_points_brute.argtypes = [P, i64, P, i64, P, i64, i32, P, P]
            L.or_sdf_points_bvh.argtypes = [P, P, i64, i32, P, P]
            L.or_grid_new.argtypes = [P, P, P, P, P]
            L.or_grid_new.restype = P
            L.or_grid_free.argtypes = [P]
            L.or_grid_values.argtypes = [P, P, i64, i32, P]
            L.or_grid_export.argtypes = [P, P, P]
            L.or_tri_check.argtypes = [P, P, i64, P, P, i64, i32, P]
            L.or_trace_sdf.argtypes = [P, P, i64, P, i32, i32, P]
            L.or_trace_combined.argtypes = [P, P, P, i64, P, i32, i32, P]
            L.or_grid_sample.argtypes = [P, P, i64, P, P]
            L.or_sdf_root_adjoint.argtypes = [P, P, i64, P, P, P, P]
            L.or_grid_new_lattice.argtypes = [P, ctypes.c_double, P, P, P]
            L.or_grid_new_lattice.restype = P
            L.or_cascade_new.argtypes = [P, ctypes.c_double, i32, i32, P, P]
            L.or_cascade_new.restype = P
            L.or_cascade_free.argtypes = [P]
            L.or_cascade_level_grid.argtypes = [P, i32, P, P, P]
            L.or_cascade_level_grid.restype = i32
            L.or_cascade_level_of.argtypes = [P, P, i64, i32, P]
            L.or_trace_combined_cascade.argtypes = [P, P, P, i64, P, i32, i32, P, P]
            L.or_df_sites.argtypes = [P, P, P, P, i32, i32, P]
            L.or_df_field.argtypes = [P, P, P, P]
            L.or_df_sweep.argtypes = [P, P, P]
            L.or_tri_box_overlap.argtypes = [P, P, P, P, P]
            L.or_tri_box_overlap.restype = ctypes.c_int
            L.or_tri_dist2_f.argtypes = [P, P, P, P]
            L.or_tri_dist2_f.restype = ctypes.c_float
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _rays(r):
    r = np.ascontiguousarray(r, dtype=np.float32)
    assert r.ndim == 2 and r.shape[1] == 8
    return r


def watertight(o, d, a, b, c):
    out = np.zeros(3)
    args = [_f64(x) for x in (o, d, a, b, c)]
    hit = lib().or_watertight(*[_ptr(x) for x in args], _ptr(out))
    return bool(hit), out


def tri_check(verts, tris, rays, prims, nthreads: int | None = None) -> np.ndarray:
    """fp64 watertight test of each ray against the one triangle prims[i]:
    a record array with hit (bool), t, u, v and ndotd = |n . d| (n the unit
    normal).  A prim outside the mesh gives hit = False."""
    V = _f64(verts)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    R = _rays(rays)
    pr = np.ascontiguousarray(prims, dtype=np.int32).reshape(-1)
    assert pr.size == R.shape[0]
    out = np.zeros((R.shape[0], 5))
    lib().or_tri_check(_ptr(V), _ptr(F), F.shape[0], _ptr(R), _ptr(pr), R.shape[0], nthreads or default_threads(),
                       _ptr(out))
    rec = np.zeros(R.shape[0], dtype=[("hit", "?"), ("t", "f8"), ("u", "f8"), ("v", "f8"), ("ndotd", "f8")])
    rec["hit"] = out[:, 0] != 0
    rec["t"], rec["u"], rec["v"], rec["ndotd"] = out[:, 1], out[:, 2], out[:, 3], out[:, 4]
    return rec


def trace_brute(verts, tris, rays, nthreads: int | None = None) -> np.ndarray:
    V = _f64(verts)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    R = _rays(rays)
    hits = np.zeros(R.shape[0], dtype=HIT_DTYPE)
    lib().or_trace_brute(_ptr(V), _ptr(F), F.shape[0], _ptr(R), R.shape[0], nthreads or default_threads(), _ptr(hits))
    return hits


class BVH:
    """Plain median-split BVH over the mesh (fp64), with the mesh pseudonormals."""

    def __init__(self, verts, tris):
        self.V = _f64(verts)
        self.F = np.ascontiguousarray(tris, dtype=np.int32)
        self.h = lib().or_bvh_build(_ptr(self.V), self.V.shape[0], _ptr(self.F), self.F.shape[0])

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_bvh_free(self.h)
            self.h = None

    @property
    def node_count(self) -> int:
        return lib().or_bvh_node_count(self.h)

    def trace(self, rays, any_hit: bool = False, nthreads: int | None = None) -> np.ndarray:
        R = _rays(rays)
        hits = np.zeros(R.shape[0], dtype=HIT_DTYPE)
        lib().or_trace_bvh(self.h, _ptr(R), R.shape[0], int(any_hit), nthreads or default_threads(), _ptr(hits))
        return hits

    def sdf_points(self, P, nthreads: int | None = None, feature: bool = False):
        P = _f64(P).reshape(-1, 3)
        out = np.zeros(P.shape[0])
        feat = np.zeros(P.shape[0], dtype=np.int64) if feature else None
        lib().or_sdf_points_bvh(self.h, _ptr(P), P.shape[0], nthreads or default_threads(), _ptr(out),
                                _ptr(feat) if feature else None)
        return (out, feat) if feature else out


def sdf_points_brute(verts, tris, P, nthreads: int | None = None, feature: bool = False):
    V = _f64(verts)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    P = _f64(P).reshape(-1, 3)
    out = np.zeros(P.shape[0])
    feat = np.zeros(P.shape[0], dtype=np.int64) if feature else None
    lib().or_sdf_points_brute(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(P), P.shape[0],
                              nthreads or default_threads(), _ptr(out), _ptr(feat) if feature else None)
    return (out, feat) if feature else out


def grid_points(lo, hi, n) -> np.ndarray:
    """Sample positions lo + (i,j,k) h, h = (hi-lo)/(n-1), x fastest (fp64)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = np.asarray(n, dtype=np.int64)
    h = (hi - lo) / (n - 1)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return np.stack([lo[0] + i * h[0], lo[1] + j * h[1], lo[2] + k * h[2]], axis=-1).reshape(-1, 3)


def bake_brute(verts, tris, lo, hi, n, nthreads: int | None = None) -> np.ndarray:
    """Full grid by the definition (every triangle for every sample); shape (nz, ny, nx)."""
    P = grid_points(lo, hi, n)
    return sdf_points_brute(verts, tris, P, nthreads).reshape(n[2], n[1], n[0])


class Grid:
    """Grid values at lo + (i,j,k) h; dense (given values) or computed on first use from a BVH."""

    def __init__(self, lo, hi, n, values=None, src: BVH | None = None):
        self.lo = _f64(lo)
        self.hi = _f64(hi)
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.src = src
        self._vals = None if values is None else _f64(values).reshape(-1)
        if self._vals is not None:
            assert self._vals.size == int(np.prod(self.n.astype(np.int64)))
        self.h = lib().or_grid_new(_ptr(self.lo), _ptr(self.hi), _ptr(self.n),
                                   _ptr(self._vals) if self._vals is not None else None,
                                   src.h if src is not None else None)
        if not self.h:
            raise ValueError("grid needs n >= 2 per axis and values or a source BVH")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_grid_free(self.h)
            self.h = None

    def values(self, idx, nthreads: int | None = None) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1)
        out = np.zeros(idx.size)
        lib().or_grid_values(self.h, _ptr(idx), idx.size, nthreads or default_threads(), _ptr(out))
        return out

    def export(self):
        """(values fp64, known bool) of every sample, x fastest; a grid computed
        on first use knows the samples evaluated so far (others read 0)."""
        count = int(np.prod(self.n.astype(np.int64)))
        vals = np.zeros(count)
        known = np.zeros(count, dtype=np.uint8)
        lib().or_grid_export(self.h, _ptr(vals), _ptr(known))
        return vals, known.astype(bool)

    def sample(self, P):
        P = _f64(P).reshape(-1, 3)
        phi = np.zeros(P.shape[0])
        grad = np.zeros((P.shape[0], 3))
        lib().or_grid_sample(self.h, _ptr(P), P.shape[0], _ptr(phi), _ptr(grad))
        return phi, grad


class Cascade:
    """Camera-centred cascade of `levels` grids of n^3 samples (Section 3, "Distance
    Field Generation").  Level k: voxel h0 * 2^k, samples at (ilo_k + i) * h_k with
    ilo_k = floor(center / h_k) - (n-1)//2.  values: (levels, n, n, n) or None to
    evaluate samples on first use from `src`."""

    def __init__(self, center, h0: float, n: int, levels: int, values=None, src: BVH | None = None):
        self.center = _f64(center)
        self.h0 = float(h0)
        self.n = int(n)
        self.levels = int(levels)
        self.src = src
        self._vals = None if values is None else _f64(values).reshape(-1)
        if self._vals is not None:
            assert self._vals.size == self.levels * self.n ** 3
        self.h = lib().or_cascade_new(_ptr(self.center), self.h0, self.n, self.levels,
                                      _ptr(self._vals) if self._vals is not None else None,
                                      src.h if src is not None else None)
        if not self.h:
            raise ValueError("cascade needs 1..16 levels, n >= 2, h0 > 0 and values or a source BVH")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_cascade_free(self.h)
            self.h = None

    def level(self, k: int):
        """(ilo (3,) int64, h) of level k."""
        ilo = np.zeros(3, dtype=np.int64)
        h = ctypes.c_double(0.0)
        if not lib().or_cascade_level_grid(self.h, int(k), _ptr(ilo), ctypes.byref(h), None):
            raise IndexError(k)
        return ilo, h.value

    def box(self, k: int):
        ilo, h = self.level(k)
        return ilo * h, (ilo + self.n - 1) * h

    def points(self, k: int) -> np.ndarray:
        """Sample positions of level k, x fastest (fp64)."""
        ilo, h = self.level(k)
        r = np.arange(self.n)
        kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
        return np.stack([(ilo[0] + ii) * h, (ilo[1] + jj) * h, (ilo[2] + kk) * h], axis=-1).reshape(-1, 3)

    def values(self, k: int, idx, nthreads: int | None = None) -> np.ndarray:
        g = ctypes.c_void_p()
        ilo = np.zeros(3, dtype=np.int64)
        h = ctypes.c_double(0.0)
        if not lib().or_cascade_level_grid(self.h, int(k), _ptr(ilo), ctypes.byref(h), ctypes.byref(g)):
            raise IndexError(k)
        idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1)
        out = np.zeros(idx.size)
        lib().or_grid_values(g, _ptr(idx), idx.size, nthreads or default_threads(), _ptr(out))
        return out

    def level_of(self, P, precision: int = 64) -> np.ndarray:
        P = _f64(P).reshape(-1, 3)
        out = np.zeros(P.shape[0], dtype=np.int32)
        lib().or_cascade_level_of(self.h, _ptr(P), P.shape[0], int(precision), _ptr(out))
        return out


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def tri_box_overlap(c, hs, a, b, cc) -> bool:
    """Single precision separating-axis test of triangle (a, b, cc) against the
    box of centre c and half sizes hs (touching counts)."""
    args = [_f32(x) for x in (c, hs, a, b, cc)]
    return bool(lib().or_tri_box_overlap(*[_ptr(x) for x in args]))


def tri_dist2_f(p, a, b, c) -> float:
    args = [_f32(x) for x in (p, a, b, c)]
    return float(lib().or_tri_dist2_f(*[_ptr(x) for x in args]))


def _level_grid(grid, k=None):
    """(or_grid pointer, number of samples, n) of a Grid, or of level k of a Cascade."""
    if isinstance(grid, Cascade):
        g = ctypes.c_void_p()
        ilo = np.zeros(3, dtype=np.int64)
        h = ctypes.c_double(0.0)
        if not lib().or_cascade_level_grid(grid.h, int(k), _ptr(ilo), ctypes.byref(h), ctypes.byref(g)):
            raise IndexError(k)
        return g, grid.n ** 3, (grid.n, grid.n, grid.n)
    n = tuple(int(v) for v in grid.n)
    return ctypes.c_void_p(grid.h), int(np.prod(n)), n


def df_sites(bvh: BVH, grid, stage: int = 3, nthreads: int | None = None):
    """Sites (triangle index per sample, -1 for none) of the paper's field build
    after `stage` (1 voxelisation, 2 jump flooding, 3 sweeps).  One grid: an
    array of n0*n1*n2; a cascade: (levels, n^3), built one level at a time,
    coarsest first: each level runs steps 1..stage, seeded also from the next
    coarser level's sites as they stand after that level's own steps 1..stage."""
    if isinstance(grid, Cascade):
        out = np.zeros((grid.levels, grid.n ** 3), dtype=np.int32)
        for k in reversed(range(grid.levels)):
            g, _, _ = _level_grid(grid, k)
            coarse, gc = (None, None)
            if k + 1 < grid.levels:
                coarse = _ptr(out[k + 1])
                gc, _, _ = _level_grid(grid, k + 1)
            lib().or_df_sites(bvh.h, g, coarse, gc, int(stage), nthreads or default_threads(), _ptr(out[k]))
        return out
    g, count, _ = _level_grid(grid)
    out = np.zeros(count, dtype=np.int32)
    lib().or_df_sites(bvh.h, g, None, None, int(stage), nthreads or default_threads(), _ptr(out))
    return out


def df_field(bvh: BVH, grid, sites) -> np.ndarray:
    """Signed distance from each sample to its site triangle (fp64)."""
    if isinstance(grid, Cascade):
        out = np.zeros((grid.levels, grid.n ** 3))
        for k in range(grid.levels):
            g, _, _ = _level_grid(grid, k)
            s = np.ascontiguousarray(sites[k], dtype=np.int32)
            lib().or_df_field(bvh.h, g, _ptr(s), _ptr(out[k]))
        return out
    g, count, _ = _level_grid(grid)
    s = np.ascontiguousarray(sites, dtype=np.int32).reshape(-1)
    out = np.zeros(count)
    lib().or_df_field(bvh.h, g, _ptr(s), _ptr(out))
    return out


def make_params(mode=1, any_hit=False, m_near=2.0, m_far=2.0, max_steps=256, hit_eps_vox=0.01,
                min_step_vox=0.01) -> Params:
    return Params(int(mode), int(any_hit), float(m_near), float(m_far), int(max_steps), 0, float(hit_eps_vox),
                  float(min_step_vox))


def trace_sdf(grid: Grid, rays, params: Params, precision: int = 64, nthreads: int | None = None):
    R = _rays(rays)
    hits = np.zeros(R.shape[0], dtype=HIT_DTYPE)
    lib().or_trace_sdf(grid.h, _ptr(R), R.shape[0], ctypes.byref(params), precision, nthreads or default_threads(),
                       _ptr(hits))
    return hits


def trace_combined(bvh: BVH | None, grid: Grid | Cascade | None, rays, params: Params, precision: int = 64,
                   nthreads: int | None = None, split_points: bool = False):
    """Combined query on one grid or on a cascade.  split_points=True also returns
    (n, 2) t_1, t_2 of each split query (NaN where the query has no split; cascade only)."""
    R = _rays(rays)
    hits = np.zeros(R.shape[0], dtype=HIT_DTYPE)
    if isinstance(grid, Cascade):
        t12 = np.full((R.shape[0], 2), np.nan)
        lib().or_trace_combined_cascade(bvh.h if bvh else None, grid.h, _ptr(R), R.shape[0], ctypes.byref(params),
                                        precision, nthreads or default_threads(), _ptr(hits), _ptr(t12))
        return (hits, t12) if split_points else hits
    assert not split_points, "split points are reported for cascades"
    lib().or_trace_combined(bvh.h if bvh else None, grid.h if grid else None, _ptr(R), R.shape[0],
                            ctypes.byref(params), precision, nthreads or default_threads(), _ptr(hits))
    return hits


def sdf_root_adjoint(grid: Grid, rays, params: Params):
    R = _rays(rays)
    n = R.shape[0]
    t = np.zeros(n)
    idx = np.zeros((n, 8), dtype=np.int64)
    w = np.zeros((n, 8))
    lib().or_sdf_root_adjoint(grid.h, _ptr(R), n, ctypes.byref(params), _ptr(t), _ptr(idx), _ptr(w))
    return t, idx, w
