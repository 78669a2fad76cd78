"""Fitting the distance-field grid to the triangle scene through the adjoint kernel.

The paper attributes the visible corner and shadow artefacts of distance-field
tracing to inaccuracies of the field (Fig. 1 and Fig. 3 captions).  Here the
grid values are fitted so that field-only hit distances agree with the exact
triangle hit distances:

  loss = mean over rays hit by both tracers of (t_field - t_triangles)^2

t_field comes from SdfHitDistance (forward: rt_trace_combined in field-only
mode with the root refined inside the last march step; backward: the adjoint
kernel rt_trace_combined_backward), t_triangles from rt_trace_bvh.  The
optimiser is Adam on the grid tensor.
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


def disagreement(scene: Scene, sdf: Sdf, rays: torch.Tensor, t_ref: torch.Tensor | None = None) -> dict:
    """Field-only vs triangle hit distances on `rays`: mean |dt|, RMS dt, and how
    often exactly one of the two tracers hits."""
    rt_sdf_prepare(sdf)
    if t_ref is None:
        t_ref = hit_fields(rt_trace_bvh(scene, rays))["t"]
    t = hit_fields(rt_trace_combined(None, sdf, rays, split_params(mode=MODE_SDF)))["t"]
    both = torch.isfinite(t) & torch.isfinite(t_ref)
    dt = (t - t_ref)[both]
    return {"mean_abs": float(dt.abs().mean()) if dt.numel() else 0.0,
            "rms": float(dt.pow(2).mean().sqrt()) if dt.numel() else 0.0,
            "only_one_hits": float((torch.isfinite(t) ^ torch.isfinite(t_ref)).float().mean()),
            "rays": int(rays.shape[0])}


def fit_grid(scene: Scene, sdf: Sdf, ray_batches, steps: int, lr: float, log_every: int = 0) -> list[FitStep]:
    """Adam on sdf.grid (a float32 CUDA tensor, updated in place).

    ray_batches: callable step -> (rays, t_triangles) with t_triangles the exact
    triangle hit distances of those rays (inf on a miss)."""
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
        loss.backward()
        opt.step()
        if log_every and (step % log_every == 0 or step == steps - 1):
            history.append(FitStep(step, float(loss.detach()), n))
        elif not log_every:
            history.append(FitStep(step, math.nan, n))
    grid.requires_grad_(False)
    rt_sdf_prepare(sdf)
    return history
