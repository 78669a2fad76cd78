"""Seeded ray batches shaped like the paper's workloads.

The paper's queries (Section 3) start at the surface point each pixel sees,
run in tiles across the viewport, and have randomised, divergent directions
within a tile.  Here:

* primary rays: a pinhole camera, one ray through each pixel centre, emitted
  in 8x8 pixel tiles;
* GI rays: one cosine-weighted hemisphere ray per pixel from a point on a
  camera-facing surface inside the view frustum.  Origins are sampled on the
  triangles by area (not found by tracing primary rays, so that producing the
  input never runs any part of the query), projected to their pixel and sorted
  into the same 8x8 tile order, which keeps the per-tile spatial coherence of
  the paper's set-up while the directions stay random;
* free-space rays: uniform origins away from every object, uniform directions.

Ray layout (float32, 8 per ray): ox, oy, oz, t_min, dx, dy, dz, t_max, the
query (o, d, t_min, t_max) of Eq. 1 with d normalised.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng
from .scene import Scene

_S_GI_POS = 11
_S_GI_DIR = 12
_S_FREE = 13
_S_AO = 14
_S_SHADOW = 15
TILE = 8


def _tile_order(px: np.ndarray, py: np.ndarray, width: int) -> np.ndarray:
    ntx = (width + TILE - 1) // TILE
    key = ((py // TILE) * ntx + (px // TILE)) * (TILE * TILE) + (py % TILE) * TILE + (px % TILE)
    return np.argsort(key, kind="stable")


def pack(o: np.ndarray, d: np.ndarray, tmin, tmax) -> np.ndarray:
    n = o.shape[0]
    r = np.empty((n, 8), dtype=np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


def primary_rays(scene: Scene, width: int | None = None, height: int | None = None,
                 t_max: float | None = None) -> np.ndarray:
    cam = scene.camera
    W = width or cam.width
    H = height or cam.height
    py, px = np.mgrid[0:H, 0:W]
    px = px.ravel()
    py = py.ravel()
    order = _tile_order(px, py, W)
    px, py = px[order], py[order]
    aspect = W / H
    x = (2 * (px + 0.5) / W - 1) * cam.tan_half_fov * aspect
    y = (1 - 2 * (py + 0.5) / H) * cam.tan_half_fov
    d = cam.forward[None, :] + x[:, None] * cam.right[None, :] + y[:, None] * cam.up[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(cam.eye, d.shape)
    tm = 1.01 * scene.diagonal if t_max is None else t_max
    return _renorm(pack(o, d, 0.0, tm))


def _renorm(r: np.ndarray) -> np.ndarray:
    """Make the float32 direction unit length in float64 and round once."""
    d = r[:, 4:7].astype(np.float64)
    r[:, 4:7] = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return r


def onb(n: np.ndarray):
    """Orthonormal basis around unit vectors n (Duff et al., JCGT 2017)."""
    sign = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    b1 = np.stack([1 + sign * n[:, 0] ** 2 * a, sign * b, -sign * n[:, 0]], axis=1)
    b2 = np.stack([b, sign + n[:, 1] ** 2 * a, -n[:, 1]], axis=1)
    return b1, b2


def cosine_hemisphere(n: np.ndarray, u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """Cosine-weighted directions around unit normals n (Malley's method)."""
    r = np.sqrt(u1)
    phi = 2 * math.pi * u2
    lx, ly, lz = r * np.cos(phi), r * np.sin(phi), np.sqrt(np.maximum(0.0, 1 - u1))
    b1, b2 = onb(n)
    d = lx[:, None] * b1 + ly[:, None] * b2 + lz[:, None] * n
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _surface_frame(scene: Scene):
    """Per-triangle corner, edges, unit normal and area CDF (cached on the scene)."""
    cached = getattr(scene, "_surface_frame_cache", None)
    if cached is not None:
        return cached
    V = scene.verts.astype(np.float64)
    F = scene.tris
    A = V[F[:, 0]]
    E1 = V[F[:, 1]] - A
    E2 = V[F[:, 2]] - A
    cr = np.cross(E1, E2)
    area2 = np.linalg.norm(cr, axis=1)
    nrm = cr / np.maximum(area2, 1e-300)[:, None]
    cdf = np.cumsum(area2)
    cdf /= cdf[-1]
    out = (A, E1, E2, nrm, cdf)
    scene._surface_frame_cache = out
    return out


def surface_points(scene: Scene, n: int, seed: int, stream: int = _S_GI_POS, width: int | None = None,
                   height: int | None = None):
    """n points on camera-facing triangle surfaces inside the view frustum, chosen
    uniformly by area, returned in 8x8 screen-tile order: (points, unit normals)."""
    cam = scene.camera
    W = width or cam.width
    H = height or cam.height
    A, E1, E2, nrm, cdf = _surface_frame(scene)
    aspect = W / H
    got = []
    have = 0
    offset = 0
    while have < n:
        m = max(4 * (n - have), 4096)
        u = rng.uniform(seed, stream, 4 * m, offset).reshape(m, 4)
        offset += 4 * m
        # candidates in triangle order: sorted lookups into the area CDF
        tri = np.minimum(np.searchsorted(cdf, np.sort(u[:, 0]), side="right"), cdf.size - 1)
        s1 = np.sqrt(u[:, 1])
        b1, b2 = s1 * (1 - u[:, 2]), s1 * u[:, 2]
        p = A[tri] + b1[:, None] * E1[tri] + b2[:, None] * E2[tri]
        nn = nrm[tri]
        q = p - cam.eye
        z = q @ cam.forward
        zs = np.maximum(z, 1e-9)
        x = (q @ cam.right) / (zs * cam.tan_half_fov * aspect)
        y = (q @ cam.up) / (zs * cam.tan_half_fov)
        keep = (np.einsum("ij,ij->i", nn, q) < 0) & (z > 0.05) & (np.abs(x) < 1) & (np.abs(y) < 1)
        idx = np.nonzero(keep)[0]
        # an unbiased subset of the accepted candidates, chosen by their own random key
        if idx.size > n - have:
            idx = idx[np.argpartition(u[idx, 3], n - have - 1)[: n - have]]
        px = np.minimum(((x[idx] + 1) * 0.5 * W).astype(np.int64), W - 1)
        py = np.minimum(((1 - y[idx]) * 0.5 * H).astype(np.int64), H - 1)
        got.append((p[idx], nn[idx], px, py))
        have += idx.size
    p = np.concatenate([g[0] for g in got])
    nn = np.concatenate([g[1] for g in got])
    order = _tile_order(np.concatenate([g[2] for g in got]), np.concatenate([g[3] for g in got]), W)
    return p[order], nn[order]


def gi_rays(scene: Scene, n: int, seed: int, t_max: float, bias_frac: float = 1e-3,
            width: int | None = None, height: int | None = None) -> np.ndarray:
    """n GI rays from camera-facing, in-frustum surface points, tile-ordered."""
    p, nn = surface_points(scene, n, seed, _S_GI_POS, width, height)
    u = rng.uniform(seed, _S_GI_DIR, 2 * n).reshape(n, 2)
    d = cosine_hemisphere(nn, u[:, 0], u[:, 1])
    o = p + (bias_frac * scene.diagonal) * nn
    return _renorm(pack(o, d, 0.0, t_max))


def ao_rays(p: np.ndarray, nn: np.ndarray, per_point: np.ndarray, seed: int, t_ao: float,
            bias: float) -> np.ndarray:
    """AO rays (Section 3, occlusion queries): per_point[i] cosine-weighted rays
    from surface point i, t in [0, t_ao]."""
    rep = np.repeat(np.arange(p.shape[0]), per_point)
    m = rep.size
    u = rng.uniform(seed, _S_AO, 2 * m).reshape(m, 2)
    d = cosine_hemisphere(nn[rep], u[:, 0], u[:, 1])
    o = p[rep] + bias * nn[rep]
    return _renorm(pack(o, d, 0.0, t_ao))


def shadow_rays(p: np.ndarray, nn: np.ndarray, lights: np.ndarray, seed: int, bias: float) -> np.ndarray:
    """Shadow rays (Section 3, GI & shadow rays): from each surface point toward one
    of the point lights picked at random, t in [0, distance - bias]."""
    m = p.shape[0]
    pick = (rng.uniform(seed, _S_SHADOW, m) * lights.shape[0]).astype(np.int64)
    o = p + bias * nn
    d = lights[pick] - o
    dist = np.linalg.norm(d, axis=1)
    d /= np.maximum(dist, 1e-12)[:, None]
    return _renorm(pack(o, d, 0.0, np.maximum(dist - bias, 0.0)))


def light_rays(p: np.ndarray, nn: np.ndarray, lights: np.ndarray, bias: float):
    """Shadow rays from every surface point to every point light (Section 3,
    GI & shadow rays): origin p + bias n, t in [0, distance - bias], point-major
    (ray i * L + l goes from point i to light l).  Also returns the geometry of
    each pair at the point: cos of the angle between n and the light direction
    (clamped at 0) and 1 / distance^2, both (m, L) float64."""
    m, L = p.shape[0], lights.shape[0]
    o = p + bias * nn
    v = lights[None, :, :] - o[:, None, :]
    dist = np.linalg.norm(v, axis=2)
    d = v / np.maximum(dist, 1e-12)[..., None]
    cos = np.maximum(np.einsum("mlk,mk->ml", d, nn), 0.0)
    rays = pack(np.repeat(o, L, axis=0), d.reshape(-1, 3), 0.0, np.maximum(dist - bias, 0.0).reshape(-1))
    return _renorm(rays), cos, 1.0 / np.maximum(dist, 1e-12) ** 2


def free_space_rays(scene: Scene, n: int, seed: int, margin: float, t_max: float | None = None) -> np.ndarray:
    """Origins uniform in the room, at least `margin` outside every object's bounding
    sphere and away from the walls; directions uniform on the sphere."""
    room = np.array(scene.room, dtype=np.float64)
    cs = np.array([o.center for o in scene.objects]).reshape(-1, 3)
    rs = np.array([o.radius for o in scene.objects]).reshape(-1)
    out = []
    have = 0
    offset = 0
    while have < n:
        m = max(2 * (n - have), 1024)
        u = rng.uniform(seed, _S_FREE, 3 * m, offset).reshape(m, 3)
        offset += 3 * m
        o = margin + u * (room - 2 * margin)
        ok = np.ones(m, dtype=bool)
        for c0 in range(0, cs.shape[0], 256):
            dd = np.linalg.norm(o[:, None, :] - cs[None, c0:c0 + 256, :], axis=2)
            ok &= np.all(dd > rs[None, c0:c0 + 256] + margin, axis=1)
        o = o[ok][: n - have]
        out.append(o)
        have += o.shape[0]
    o = np.concatenate(out)
    u = rng.uniform(seed, _S_FREE + 100, 2 * n).reshape(n, 2)
    z = 1 - 2 * u[:, 0]
    r = np.sqrt(np.maximum(0.0, 1 - z * z))
    phi = 2 * math.pi * u[:, 1]
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    tm = scene.diagonal if t_max is None else t_max
    return _renorm(pack(o, d, 0.0, tm))


def mixed_frame(scene: Scene, frame: int, m: float, seed: int = 2305):
    """One frame of the mixed workload (the query kinds of Section 3): primary rays
    (triangles only), 1-4 AO rays per pixel (t_max 0.5 m, one split), one GI ray
    per pixel (t_max 30 m, one split) and shadow rays to 4 random point lights (two
    splits, any hit), their count drawn from [0.5 M, 2.07 M].  Returns
    [(name, rays, split parameters as keywords)] with multiplier m."""
    n_px = 1920 * 1080
    fs = seed * 1000 + frame
    prim = primary_rays(scene)
    p, nn = surface_points(scene, n_px, fs)
    bias = 1e-3 * scene.diagonal
    u = rng.uniform(fs, 901, n_px + 2)
    per_pt = 1 + (u[:n_px] * 4).astype(np.int64)
    ao = ao_rays(p, nn, per_pt, fs, 0.5, bias)
    gi = ao_rays(p, nn, np.ones(n_px, dtype=np.int64), fs + 7, 30.0, bias)
    n_sh = int(500_000 + u[n_px] * (n_px - 500_000))
    lights = 0.5 + rng.uniform(fs, 902, 12).reshape(4, 3) * (np.array(scene.room) - 1.0)
    sh = shadow_rays(p[:n_sh], nn[:n_sh], lights, fs, bias)
    return [("primary", prim, dict(mode=0)), ("ao", ao, dict(mode=1, m_near=m)),
            ("gi", gi, dict(mode=1, m_near=m)),
            ("shadow", sh, dict(mode=2, m_near=m, m_far=m, any_hit=True))]
