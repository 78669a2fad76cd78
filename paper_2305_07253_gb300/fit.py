"""Fitting the distance-field grid to the triangle scene through the adjoint kernel.

The paper attributes the visible corner and shadow artefacts of distance-field
tracing to inaccuracies of the field (Fig. 1 and Fig. 3 captions).  Here the
grid values are fitted so that field-only hit distances agree with the exact
triangle hit distances:

  loss = mean over rays hit by both tracers of (t_field - t_triangles)^2
       + surface_weight * mean over rays hit by the triangles of phi(p*)^2

t_field comes from SdfHitDistance (forward: rt_trace_combined in field-only
mode with the root refined inside the last march step; backward: the adjoint
kernel rt_trace_combined_backward), t_triangles from rt_trace_bvh.  The second
term asks the field to vanish at the exact hit points p* = o + t_triangles d:
without it, rays the field misses carry no gradient and the fit can trade hits
for misses.  phi(p*) is the trilinear interpolant of the grid (vertex-centred
samples), written out with tensor gathers.  The optimiser is Adam on the grid.
"""
from __future__ import annotations

import dataclasses
import math

import torch

from . import (MODE_SDF, Scene, Sdf, SdfHitDistance, hit_fields, rt_sdf_prepare, rt_trace_bvh,
               rt_trace_combined, split_params)


@dataclasses.dataclass
class FitStep:
    step: int
    loss: float
    rays_used: int


def disagreement(scene: Scene, sdf: Sdf, rays: torch.Tensor, t_ref: torch.Tensor | None = None,
                 m_near: float | None = None) -> dict:
    """Hit distances of the field-only query (or of the combined query with one
    split at m_near voxels) against the triangles on `rays`: mean |dt|, RMS dt
    over rays both hit, and how often exactly one of the two hits."""
    rt_sdf_prepare(sdf)
    if t_ref is None:
        t_ref = hit_fields(rt_trace_bvh(scene, rays))["t"]
    if m_near is None:
        t = hit_fields(rt_trace_combined(None, sdf, rays, split_params(mode=MODE_SDF)))["t"]
    else:
        t = hit_fields(rt_trace_combined(scene, sdf, rays, split_params(mode=1, m_near=m_near)))["t"]
    both = torch.isfinite(t) & torch.isfinite(t_ref)
    dt = (t - t_ref)[both]
    return {"mean_abs": float(dt.abs().mean()) if dt.numel() else 0.0,
            "rms": float(dt.pow(2).mean().sqrt()) if dt.numel() else 0.0,
            "only_one_hits": float((torch.isfinite(t) ^ torch.isfinite(t_ref)).float().mean()),
            "rays": int(rays.shape[0])}


def interpolate(grid: torch.Tensor, lo, hi, p: torch.Tensor) -> torch.Tensor:
    """Trilinear value of a (nz, ny, nx) grid with samples at lo + (i,j,k) h,
    h = (hi - lo) / (n - 1), at points p (m, 3); clamped to the grid box.
    Differentiable in the grid values."""
    n = torch.tensor([grid.shape[2], grid.shape[1], grid.shape[0]], device=p.device)
    lo_t = torch.tensor(lo, dtype=p.dtype, device=p.device)
    h = (torch.tensor(hi, dtype=p.dtype, device=p.device) - lo_t) / (n - 1)
    u = torch.minimum(torch.clamp((p - lo_t) / h, min=0.0), (n - 1).to(p.dtype))
    i0 = torch.minimum(u.floor().long(), n - 2)
    f = u - i0
    g = grid.reshape(-1)
    val = torch.zeros(p.shape[0], dtype=grid.dtype, device=p.device)
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                idx = (i0[:, 0] + bx) + n[0] * ((i0[:, 1] + by) + n[1] * (i0[:, 2] + bz))
                w = (f[:, 0] if bx else 1 - f[:, 0]) * (f[:, 1] if by else 1 - f[:, 1]) * \
                    (f[:, 2] if bz else 1 - f[:, 2])
                val = val + w * g[idx]
    return val


def fit_grid(scene: Scene, sdf: Sdf, ray_batches, steps: int, lr: float, log_every: int = 0,
             surface_weight: float = 1.0, surface: str = "square") -> list[FitStep]:
    """Adam on sdf.grid (a float32 CUDA tensor, updated in place).

    ray_batches: callable step -> (rays, t_triangles) with t_triangles the exact
    triangle hit distances of those rays (inf on a miss).
    surface: "square" penalises phi(p*)^2; "hinge" penalises max(phi(p*), 0)^2,
    only the values that let a ray pass the surface (a march registers a hit
    once phi drops below its small threshold)."""
    if surface not in ("square", "hinge"):
        raise ValueError(f"surface must be 'square' or 'hinge', not {surface!r}")
    grid = sdf.grid
    if grid.dtype != torch.float32:
        raise ValueError("fitting needs a float32 grid")
    grid.requires_grad_(True)
    opt = torch.optim.Adam([grid], lr=lr)
    params = split_params(mode=MODE_SDF)
    history = []
    for step in range(steps):
        rays, t_ref = ray_batches(step)
        opt.zero_grad(set_to_none=True)
        t, _ = SdfHitDistance.apply(grid, rays, None, sdf, params)
        both = torch.isfinite(t) & torch.isfinite(t_ref)
        n = int(both.sum())
        diff = torch.where(both, t - t_ref, torch.zeros_like(t))
        loss = diff.pow(2).sum() / max(n, 1)
        if surface_weight > 0:
            hit = torch.isfinite(t_ref)
            p_star = rays[hit, 0:3] + t_ref[hit, None] * rays[hit, 4:7]
            phi = interpolate(grid, sdf.lo, sdf.hi, p_star)
            if surface == "hinge":
                phi = torch.clamp(phi, min=0.0)
            loss = loss + surface_weight * phi.pow(2).mean()
        loss.backward()
        opt.step()
        if log_every and (step % log_every == 0 or step == steps - 1):
            history.append(FitStep(step, float(loss.detach()), n))
        elif not log_every:
            history.append(FitStep(step, math.nan, n))
    grid.requires_grad_(False)
    rt_sdf_prepare(sdf)
    return history
