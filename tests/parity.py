"""Comparison helpers for device results against the CPU checker.

Tolerances (the bar the tests hold the device path to):
  * triangle-resolved queries: primitive ids equal on >= 99.99% of rays; every
    mismatch must be a tie or an edge/grazing hit that the fp64 checker
    confirms; t within 1e-4 relative.
  * field-resolved queries: same tracer, t within 1e-3 relative of the
    checker's float march (identical step rule).
"""
from __future__ import annotations

import numpy as np

import oracle as O

T_REL_BVH = 1e-4
T_REL_SDF = 1e-3
EDGE_EPS = 1e-4
GRAZE = 1e-3


def gpu_hits_to_numpy(hits) -> dict:
    h = hits.cpu().numpy()
    return {
        "t": h[:, 0].view(np.float32).astype(np.float64),
        "prim": h[:, 1].astype(np.int64),
        "u": h[:, 2].view(np.float32).astype(np.float64),
        "v": h[:, 3].view(np.float32).astype(np.float64),
        "tracer": h[:, 4].astype(np.int64),
        "flags": h[:, 5].astype(np.int64),
    }


def _tri_t64(verts, tris, ray, prim):
    f = tris[prim]
    V = verts.astype(np.float64)
    hit, out = O.watertight(ray[0:3].astype(np.float64), ray[4:7].astype(np.float64), V[f[0]], V[f[1]], V[f[2]])
    return hit, out


def _grazing(verts, tris, ray, prim):
    f = tris[prim]
    V = verts.astype(np.float64)
    n = np.cross(V[f[1]] - V[f[0]], V[f[2]] - V[f[0]])
    n /= np.linalg.norm(n) + 1e-300
    return abs(float(np.dot(n, ray[4:7].astype(np.float64)))) < GRAZE


def _edge(u, v):
    return min(u, v, 1.0 - u - v) < EDGE_EPS


def check_bvh_resolved(g: dict, o: np.ndarray, rays: np.ndarray, verts, tris, sel=None, min_equal=0.9999):
    """Compare triangle-resolved results; returns a summary dict. Asserts the bar."""
    idx = np.arange(len(rays)) if sel is None else np.nonzero(sel)[0]
    g_hit = g["tracer"][idx] == 1
    o_hit = o["tracer"][idx] == 1
    both = g_hit & o_hit
    same_prim = both & (g["prim"][idx] == o["prim"][idx])
    bad = []
    for j in np.nonzero(both & ~same_prim)[0]:
        i = idx[j]
        hit, (t64, u64, v64) = _tri_t64(verts, tris, rays[i], g["prim"][i])
        tie = hit and abs(t64 - o["t"][i]) <= T_REL_BVH * max(1.0, abs(o["t"][i]))
        if not (tie or _edge(g["u"][i], g["v"][i]) or _grazing(verts, tris, rays[i], g["prim"][i])):
            bad.append(("id", int(i)))
    for j in np.nonzero(g_hit & ~o_hit)[0]:
        i = idx[j]
        if not (_edge(g["u"][i], g["v"][i]) or _grazing(verts, tris, rays[i], g["prim"][i])):
            bad.append(("gpu-only hit", int(i)))
    for j in np.nonzero(~g_hit & o_hit)[0]:
        i = idx[j]
        if not (_edge(o["u"][i], o["v"][i]) or _grazing(verts, tris, rays[i], o["prim"][i])):
            bad.append(("gpu miss", int(i)))
    frac_equal = float(same_prim.sum()) / int(both.sum()) if both.any() else 1.0
    terr = np.abs(g["t"][idx][same_prim] - o["t"][idx][same_prim]) / np.maximum(1.0, np.abs(o["t"][idx][same_prim]))
    assert not bad, f"unconfirmed mismatches: {bad[:10]} (of {len(bad)})"
    assert frac_equal >= min_equal, f"prim ids equal on {frac_equal:.6f}"
    if terr.size:
        assert terr.max() <= T_REL_BVH, f"t rel err {terr.max():.3e}"
    return {"n": int(len(idx)), "equal": frac_equal, "t_err_max": float(terr.max()) if terr.size else 0.0,
            "confirmed_mismatch": int((both & ~same_prim).sum() + (g_hit ^ o_hit).sum())}


def check_sdf_resolved(g: dict, o: np.ndarray, sel=None, rel=T_REL_SDF, max_flip_frac=0.0):
    idx = np.arange(len(g["t"])) if sel is None else np.nonzero(sel)[0]
    gs = g["tracer"][idx] == 2
    os_ = o["tracer"][idx] == 2
    flips = gs ^ os_
    both = gs & os_
    err = np.abs(g["t"][idx][both] - o["t"][idx][both]) / np.maximum(1.0, np.abs(o["t"][idx][both]))
    over = err > rel
    frac = (flips.sum() + over.sum()) / max(1, len(idx))
    assert frac <= max_flip_frac, (
        f"field-resolved disagreement on {int(flips.sum())} tracer flips and {int(over.sum())} t errors > {rel} "
        f"of {len(idx)} (max err {err.max() if err.size else 0:.3e})")
    return {"n": int(len(idx)), "flips": int(flips.sum()), "over": int(over.sum()),
            "t_err_max": float(err.max()) if err.size else 0.0,
            "exact": float(np.mean(g["t"][idx][both] == o["t"][idx][both])) if both.any() else 1.0}
