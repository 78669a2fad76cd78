"""Query-by-query comparison of device records with the CPU checker's.

The bar every parity test holds the device path to (the query of Eq. 1, its
sub-intervals of Eq. 2 and the ordering rules after Eq. 2; triangle segments
exact, field segments by the checker's float march on the same grid):

  EQUAL      same tracer, and
               triangle-resolved, closest hit: same primitive, t within 1e-4
                 relative;
               triangle-resolved, any hit: the device's primitive is a real
                 fp64 intersection inside a triangle sub-interval, t within 1e-4
                 relative of the fp64 t (any intersection may be reported);
               field-resolved: t within 1e-3 relative of the checker's float
                 march (the tests also count bit-equal t);
               miss: both miss;
             and the same STEP_LIMIT flag.
  EXPLAINED  a query that is not EQUAL only because one triangle test sits on a
             rounding boundary, confirmed in fp64 on the triangle in question
             (the device's hit, or the checker's when the device has none):
               tie       two different triangles, and the fp64 t of the device's
                         one lies within 1e-4 relative of the checker's t;
               edge      the ray's line meets that triangle within 1e-5 of an
                         edge (fp64 barycentrics: |min(u, v, 1-u-v)| < 1e-5);
               graze     |n . d| < 1e-3 for that triangle;
               boundary  that triangle's fp64 t lies within 1e-4 relative of an
                         end of the query's sub-intervals (t_min, t_1, t_2,
                         t_max), so float and fp64 may place it on either side;
             or a field decision on a rounding boundary:
               field_ulp the checker's float march came within one float ulp of
                         eps_hit at some step (its decision margin).
  Anything else fails the test, and EQUAL must hold on >= 99.99 % of queries.
"""
from __future__ import annotations

import numpy as np

import oracle as O

T_REL_BVH = 1e-4
T_REL_SDF = 1e-3
EDGE_EPS = 1e-5
GRAZE = 1e-3
MIN_EQUAL = 0.9999
FLAG_STEP_LIMIT = 2


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


def segment_ends(rays, mode: int, m_near: float, m_far: float, h: float) -> np.ndarray:
    """(n, 4) t_min, t_1, t_2, t_max of Eq. 2 in fp64 for one dense grid of
    largest voxel edge h (t_1 = t_2 = t_max where a split does not apply)."""
    r = np.asarray(rays, dtype=np.float64)
    tmin, tmax = r[:, 3], r[:, 7]
    with np.errstate(invalid="ignore"):
        t1 = np.minimum(np.maximum(tmin + m_near * h, tmin), tmax) if mode in (1, 2) else tmax
        t2 = np.minimum(np.maximum(tmax - m_far * h, t1), tmax) if mode == 2 else tmax
    return np.stack([tmin, np.broadcast_to(t1, tmin.shape), np.broadcast_to(t2, tmin.shape), tmax], axis=1)


def ends_from_split_points(rays, t12) -> np.ndarray:
    """(n, 4) t_min, t_1, t_2, t_max from the checker's split points (cascades;
    NaN where a query has no split)."""
    r = np.asarray(rays, dtype=np.float64)
    tmin, tmax = r[:, 3], r[:, 7]
    t1 = np.where(np.isnan(t12[:, 0]), tmax, t12[:, 0])
    t2 = np.where(np.isnan(t12[:, 1]), tmax, t12[:, 1])
    return np.stack([tmin, t1, t2, tmax], axis=1)


def _rel(a, b):
    with np.errstate(invalid="ignore"):
        return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def _edge_dist(u, v):
    return np.abs(np.minimum(np.minimum(u, v), 1.0 - u - v))


class Report(dict):
    def __str__(self):
        keys = ("n", "equal", "sdf_bit_equal", "tie", "edge", "graze", "boundary", "field_ulp", "unexplained")
        return ", ".join(f"{k}={self[k]}" for k in keys if k in self)


def tri_spans(mode: int):
    """Column pairs of segment_ends() that bound the triangle sub-intervals."""
    return {0: [(0, 3)], 1: [(0, 1)], 2: [(0, 1), (2, 3)], 3: []}[int(mode)]


def compare(g: dict, o: np.ndarray, rays, verts, tris, *, any_hit: bool = False, ends=None, spans=None,
            eps_hit=None, min_equal: float = MIN_EQUAL, t_rel_sdf: float = T_REL_SDF, check: bool = True) -> Report:
    """Classify every query (see the module docstring) and assert the bar.

    g: device records (gpu_hits_to_numpy); o: the checker's records for the
    same rays; ends: (n, k) sub-interval ends for the boundary rule (default
    t_min and t_max only); spans: column pairs of `ends` bounding the triangle
    sub-intervals, where an any-hit record must lie (default the first to the
    last column); eps_hit: the float hit threshold (the largest one for a
    cascade) for the field_ulp rule (None: no field flip is explained)."""
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    n = rays.shape[0]
    assert len(g["t"]) == n and len(o) == n
    r64 = rays.astype(np.float64)
    if ends is None:
        ends = np.stack([r64[:, 3], r64[:, 7]], axis=1)
    gt, ot = g["tracer"], o["tracer"]
    otp = o["prim"].astype(np.int64)
    step_same = (g["flags"] & FLAG_STEP_LIMIT) == (o["flags"] & FLAG_STEP_LIMIT)
    rel = _rel(g["t"], o["t"])

    # fp64 view of every device triangle hit (all of them for any hit, else where they matter)
    g_tri = gt == 1
    need_g = g_tri & ((ot != 1) | (g["prim"] != otp) | (rel > T_REL_BVH) | bool(any_hit))
    gidx = np.nonzero(need_g)[0]
    gc = O.tri_check(verts, tris, rays[gidx], g["prim"][gidx]) if gidx.size else None
    g64 = {k: np.full(n, np.nan) for k in ("t", "u", "v", "ndotd")}
    g64_hit = np.zeros(n, dtype=bool)
    if gidx.size:
        for k in ("t", "u", "v", "ndotd"):
            g64[k][gidx] = gc[k]
        g64_hit[gidx] = gc["hit"]
    # fp64 view of the checker's own triangle hits that the device lacks
    need_o = (ot == 1) & ~((gt == 1) & (g["prim"] == otp))
    oidx = np.nonzero(need_o)[0]
    o_nd = np.full(n, np.nan)
    if oidx.size:
        o_nd[oidx] = O.tri_check(verts, tris, rays[oidx], otp[oidx])["ndotd"]

    if spans is None:
        spans = [(0, ends.shape[1] - 1)]

    def in_interval(t):
        tol = T_REL_BVH * np.maximum(1.0, np.abs(t))
        ok = np.zeros(n, dtype=bool)
        with np.errstate(invalid="ignore"):
            for a, b in spans:
                ok |= (t >= ends[:, a] - tol) & (t <= ends[:, b] + tol)
        return ok

    def near_end(t):
        tol = T_REL_BVH * np.maximum(1.0, np.abs(ends))
        return np.any(np.abs(ends - t[:, None]) <= tol, axis=1)

    miss_eq = (gt == 0) & (ot == 0)
    if any_hit:
        g_valid = g64_hit & (_rel(g["t"], g64["t"]) <= T_REL_BVH) & in_interval(g64["t"])
        tri_eq = (gt == 1) & (ot == 1) & g_valid
    else:
        tri_eq = (gt == 1) & (ot == 1) & (g["prim"] == otp) & (rel <= T_REL_BVH)
    sdf_eq = (gt == 2) & (ot == 2) & (rel <= t_rel_sdf)
    equal = (miss_eq | tri_eq | sdf_eq) & step_same

    cats = {k: np.zeros(n, dtype=bool) for k in ("tie", "edge", "graze", "boundary", "field_ulp")}
    bad = ~equal
    # the device's triangle hit is the one in question
    gq = bad & (gt == 1)
    with np.errstate(invalid="ignore"):
        cats["tie"] |= gq & (ot == 1) & (g["prim"] != otp) & (_rel(g64["t"], o["t"]) <= T_REL_BVH) & \
            (rel <= T_REL_BVH)
        cats["edge"] |= gq & (_edge_dist(g64["u"], g64["v"]) < EDGE_EPS)
        cats["graze"] |= gq & (g64["ndotd"] < GRAZE)
        cats["boundary"] |= gq & near_end(g64["t"])
    # the device has no (matching) triangle hit: the checker's hit is in question
    oq = bad & (ot == 1) & ((gt != 1) | (g["prim"] != otp))
    with np.errstate(invalid="ignore"):
        cats["edge"] |= oq & (_edge_dist(o["u"], o["v"]) < EDGE_EPS)
        cats["graze"] |= oq & (o_nd < GRAZE)
        cats["boundary"] |= oq & near_end(o["t"])
    # a field decision: neither side's record is a triangle hit
    fq = bad & (gt != 1) & (ot != 1)
    if eps_hit is not None:
        ulp = float(np.spacing(np.float32(eps_hit)))
        cats["field_ulp"] |= fq & (o["margin"] <= ulp)
    explained = np.zeros(n, dtype=bool)
    for v in cats.values():
        explained |= v
    unexplained = np.nonzero(bad & ~explained)[0]
    both_sdf = (gt == 2) & (ot == 2)
    rep = Report(n=int(n), equal=float(equal.mean()) if n else 1.0,
                 sdf_bit_equal=float(np.mean(g["t"][both_sdf] == o["t"][both_sdf])) if both_sdf.any() else 1.0,
                 unexplained=int(unexplained.size), **{k: int((v & bad).sum()) for k, v in cats.items()})
    rep["t_err_max_bvh"] = float(rel[tri_eq].max()) if tri_eq.any() and not any_hit else 0.0
    rep["t_err_max_sdf"] = float(rel[both_sdf].max()) if both_sdf.any() else 0.0
    rep["examples"] = [(int(i), int(gt[i]), int(ot[i]), float(g["t"][i]), float(o["t"][i]), int(g["prim"][i]),
                        int(otp[i])) for i in unexplained[:8]]
    rep["mask_equal"] = equal
    if check:
        assert unexplained.size == 0, f"unexplained mismatches: {rep}; (i, tracer dev/chk, t dev/chk, prim dev/chk): " \
                                      f"{rep['examples']}"
        assert rep["equal"] >= min_equal, f"equal on {rep['equal']:.6f} < {min_equal}: {rep}"
    return rep
