"""Renderer-side estimators built on the combined query: the numeric form of the
paper's experiments (Section 3, "Occlusion Queries" and "GI & Shadow Rays";
their images are Fig. 2 and Fig. 3).

  ambient occlusion  AO(x) = share of the spp cosine-weighted rays from x that
                     travel [0, t_ao] without a hit;
  direct light       E(x) = sum over point lights l of
                     power * V(x, l) * cos(theta_l) / |l - x|^2,
                     V = 1 when the shadow ray to l has no hit (any hit, two
                     splits in the combined form, Section 3);
  one-bounce GI      L(x) = albedo / pi * (E(x) + albedo * mean over the spp GI
                     rays of E(y)), y the hit point of a GI ray, constant albedo
                     (the paper's assumption); at a field-resolved y the normal
                     is the gradient of the field itself.

Every query goes through the C-ABI (rt_trace_combined); this module only forms
the query batches from surface points (with the seeded generators of `synth`)
and reduces the hit records.  Surface points are inputs: the benchmark takes
them from the device's primary hits, the tests from the CPU checker's.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from synth import rays as R

from . import TRACER_BVH, TRACER_MISS, TRACER_SDF, hit_fields, rt_trace_combined
from .fit import interpolate


def visible_points(prim_rays: np.ndarray, t: np.ndarray, prim: np.ndarray, verts: np.ndarray, tris: np.ndarray):
    """The surface point each primary ray sees and its unit geometric normal
    turned toward the camera: (points (n, 3) float64, normals (n, 3), seen (n,)
    bool).  Points of rays that see nothing are the ray origins."""
    seen = np.isfinite(t) & (prim >= 0)
    o = prim_rays[:, 0:3].astype(np.float64)
    d = prim_rays[:, 4:7].astype(np.float64)
    x = o + np.where(seen, t, 0.0)[:, None] * d
    V = verts.astype(np.float64)
    tri = np.where(seen, prim, 0)
    nrm = np.cross(V[tris[tri, 1]] - V[tris[tri, 0]], V[tris[tri, 2]] - V[tris[tri, 0]])
    nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-30)
    nrm *= np.where(np.einsum("ij,ij->i", nrm, d) > 0, -1.0, 1.0)[:, None]
    return x, nrm, seen


def ao_from_records(tracer: torch.Tensor, spp: int) -> torch.Tensor:
    """AO per point from the records of its spp consecutive AO queries."""
    return (tracer == TRACER_MISS).double().reshape(-1, spp).mean(dim=1)


def ambient_occlusion(scene, sdf, params, points: np.ndarray, normals: np.ndarray, spp: int, t_ao: float,
                      seed: int, bias: float):
    """AO of every point through spp cosine rays of length t_ao: (AO (m,) float64
    on the device, the rays, the hit records)."""
    rays = torch.from_numpy(R.ao_rays(points, normals, np.full(points.shape[0], spp, dtype=np.int64), seed, t_ao,
                                      bias)).cuda()
    hits = rt_trace_combined(scene, sdf, rays, params)
    return ao_from_records(hits[:, 4], spp), rays, hits


def irradiance_from_records(tracer: torch.Tensor, cos: torch.Tensor, inv_d2: torch.Tensor, power: float):
    """E per point from the shadow-ray records (point-major, L lights per point)
    and the pair geometry of light_rays."""
    vis = (tracer == TRACER_MISS).double().reshape(cos.shape)
    return (power * vis * cos * inv_d2).sum(dim=1)


def direct_light(scene, sdf, params, points: np.ndarray, normals: np.ndarray, lights: np.ndarray, power: float,
                 bias: float):
    """Direct irradiance of every point from the point lights through shadow
    rays: (E (m,) float64 on the device, the rays, the hit records)."""
    rays_h, cos, inv_d2 = R.light_rays(points, normals, lights, bias)
    rays = torch.from_numpy(rays_h).cuda()
    hits = rt_trace_combined(scene, sdf, rays, params)
    E = irradiance_from_records(hits[:, 4], torch.from_numpy(cos).cuda(), torch.from_numpy(inv_d2).cuda(), power)
    return E, rays, hits


def field_normals(levels, y: torch.Tensor, d: torch.Tensor) -> torch.Tensor:
    """Unit gradient of a field at points y (m, 3), turned against the ray
    directions d: central differences of the trilinear interpolant over half a
    voxel.  levels: [(grid (n, n, n) x fastest, lo (3), hi (3))], finest first; a
    point takes the finest level whose box holds it (the coarsest otherwise)."""
    k_of = torch.full((y.shape[0],), len(levels) - 1, dtype=torch.long, device=y.device)
    for k in range(len(levels) - 2, -1, -1):
        lo = torch.tensor(levels[k][1], dtype=y.dtype, device=y.device)
        hi = torch.tensor(levels[k][2], dtype=y.dtype, device=y.device)
        k_of = torch.where(((y >= lo) & (y <= hi)).all(dim=1), torch.full_like(k_of, k), k_of)
    g = torch.zeros_like(y)
    for k, (grid, lo, hi) in enumerate(levels):
        sel = k_of == k
        if not bool(sel.any()):
            continue
        yk = y[sel]
        h = (torch.tensor(hi, dtype=y.dtype, device=y.device) - torch.tensor(lo, dtype=y.dtype, device=y.device)) \
            / (grid.shape[0] - 1)
        gk = torch.empty_like(yk)
        for a in range(3):
            e = torch.zeros(3, dtype=y.dtype, device=y.device)
            e[a] = 0.5 * h[a]
            gk[:, a] = (interpolate(grid, lo, hi, yk + e) - interpolate(grid, lo, hi, yk - e)) / (2 * e[a])
        g[sel] = gk
    g = g / g.norm(dim=1, keepdim=True).clamp(min=1e-30)
    return torch.where(((g * d).sum(dim=1) > 0)[:, None], -g, g)


def one_bounce(scene, sdf, gi_params, shadow_params, points: np.ndarray, normals: np.ndarray, face_normals,
               levels, lights: np.ndarray, power: float, albedo: float, spp: int, seed: int, bias: float):
    """One-bounce GI radiance of every point (see the module docstring):
    returns dict with radiance, direct (E(x)), and the query batches it ran."""
    E_x, r_x, _ = direct_light(scene, sdf, shadow_params, points, normals, lights, power, bias)
    n = points.shape[0]
    gi = torch.from_numpy(R.ao_rays(points, normals, np.full(n, spp, dtype=np.int64), seed, 30.0, bias)).cuda()
    f = hit_fields(rt_trace_combined(scene, sdf, gi, gi_params))
    tg = f["t"].double()
    hit = torch.isfinite(tg)
    y = gi[:, 0:3].double() + torch.where(hit, tg, torch.zeros_like(tg))[:, None] * gi[:, 4:7].double()
    ny = torch.zeros_like(y)
    bvh = f["tracer"] == TRACER_BVH
    if bool(bvh.any()):
        fn = face_normals[f["prim"][bvh].long()]
        db = gi[bvh, 4:7].double()
        ny[bvh] = torch.where(((fn * db).sum(dim=1) > 0)[:, None], -fn, fn)
    fld = f["tracer"] == TRACER_SDF
    if bool(fld.any()):
        ny[fld] = field_normals(levels, y[fld], gi[fld, 4:7].double())
    E_y, r_y, _ = direct_light(scene, sdf, shadow_params, y.cpu().numpy(), ny.cpu().numpy(), lights, power, bias)
    E_y = torch.where(hit, E_y, torch.zeros_like(E_y))
    E_ind = albedo * E_y.reshape(n, spp).mean(dim=1)
    radiance = (albedo / math.pi) * (E_x + E_ind)
    return {"radiance": radiance, "direct": (albedo / math.pi) * E_x, "batches": (r_x, gi, r_y)}
