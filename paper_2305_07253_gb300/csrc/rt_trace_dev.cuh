// Device code shared by the trace and adjoint kernels: the two tracing
// techniques of the combined query and the split of Eq. 2.
#pragma once

#include <math.h>

#include "rt_internal.cuh"

namespace rtdev {

struct Hit {
    float t;
    int32_t prim;
    float u, v;
};

struct Counts {
    uint32_t nodes, tris, steps, field;
};

__device__ __forceinline__ float sel3(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Triangle segment: closest (or any) hit on [ta, tb] through the BVH, with
// the watertight ray/triangle test of Woop, Benthin & Wald (JCGT 2013) in
// float.  The edge functions are products and a difference rounded
// separately (no fused multiply-add), so two triangles sharing an edge
// evaluate that edge to exactly opposite values and no ray slips between
// them.  Ties in t go to the smaller triangle index.
// ---------------------------------------------------------------------------
template <bool COUNT>
__device__ __forceinline__ bool bvh_segment(const TraceArgs& a, float3 o, float3 d, float ta, float tb, bool any_hit,
                                            Hit& best, uint32_t& flags, Counts& cnt)
{
    if (a.root == INT32_MIN || !(ta <= tb)) return false;
    // safe reciprocal: components below 2^-80 behave like 2^-80 (slabs stay finite)
    const float eps = 8.27180613e-25f;
    float3 idir = make_float3(1.0f / (fabsf(d.x) > eps ? d.x : copysignf(eps, d.x)),
                              1.0f / (fabsf(d.y) > eps ? d.y : copysignf(eps, d.y)),
                              1.0f / (fabsf(d.z) > eps ? d.z : copysignf(eps, d.z)));
    float3 ood = make_float3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
    // watertight set-up: dominant axis kz, shear constants
    int kz = 0;
    float az = fabsf(d.x);
    if (fabsf(d.y) > az) { kz = 1; az = fabsf(d.y); }
    if (fabsf(d.z) > az) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dkz = sel3(d.x, d.y, d.z, kz);
    if (dkz < 0.f) { int s = kx; kx = ky; ky = s; }
    const float Sx = __fdiv_rn(sel3(d.x, d.y, d.z, kx), dkz);
    const float Sy = __fdiv_rn(sel3(d.x, d.y, d.z, ky), dkz);
    const float Sz = __frcp_rn(dkz);

    int stack[RT_STACK_DEPTH];
    int sp = 0;
    int node = a.root;
    float tbest = tb;
    bool found = false;
    // a tree visit never exceeds 2n-1 nodes; the guard only stops a corrupt structure
    for (uint32_t guard = 0;; ++guard) {
        if (guard > (1u << 26)) {
            flags |= RT_FLAG_ITER_LIMIT;
            break;
        }
        if (node >= 0) {
            const float4* np = reinterpret_cast<const float4*>(a.nodes + node);
            float4 na = ldg4(np), nb = ldg4(np + 1), nc = ldg4(np + 2);
            int4 nd = __ldg(reinterpret_cast<const int4*>(np + 3));
            if (COUNT) ++cnt.nodes;
            float x0 = fmaf(na.x, idir.x, -ood.x), x1 = fmaf(na.y, idir.x, -ood.x);
            float y0 = fmaf(na.z, idir.y, -ood.y), y1 = fmaf(na.w, idir.y, -ood.y);
            float z0 = fmaf(nc.x, idir.z, -ood.z), z1 = fmaf(nc.y, idir.z, -ood.z);
            float tn0 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), ta));
            float tf0 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tbest));
            x0 = fmaf(nb.x, idir.x, -ood.x); x1 = fmaf(nb.y, idir.x, -ood.x);
            y0 = fmaf(nb.z, idir.y, -ood.y); y1 = fmaf(nb.w, idir.y, -ood.y);
            z0 = fmaf(nc.z, idir.z, -ood.z); z1 = fmaf(nc.w, idir.z, -ood.z);
            float tn1 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), ta));
            float tf1 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tbest));
            bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
            if (h0 && h1) {
                int nearc = nd.x, farc = nd.y;
                if (tn1 < tn0) { nearc = nd.y; farc = nd.x; }
                if (sp < RT_STACK_DEPTH) stack[sp++] = farc;
                else flags |= RT_FLAG_STACK_OVERFLOW;
                node = nearc;
                continue;
            }
            if (h0) { node = nd.x; continue; }
            if (h1) { node = nd.y; continue; }
        } else {
            const int tri = ~node;
            if (COUNT) ++cnt.tris;
            const float4* tp = a.tris + 3 * (int64_t)tri;
            float4 v0 = ldg4(tp), v1 = ldg4(tp + 1), v2 = ldg4(tp + 2);
            float A0 = v0.x - o.x, A1 = v0.y - o.y, A2 = v0.z - o.z;
            float B0 = v1.x - o.x, B1 = v1.y - o.y, B2 = v1.z - o.z;
            float C0 = v2.x - o.x, C1 = v2.y - o.y, C2 = v2.z - o.z;
            float Akz = sel3(A0, A1, A2, kz), Bkz = sel3(B0, B1, B2, kz), Ckz = sel3(C0, C1, C2, kz);
            float Ax = __fmaf_rn(-Sx, Akz, sel3(A0, A1, A2, kx)), Ay = __fmaf_rn(-Sy, Akz, sel3(A0, A1, A2, ky));
            float Bx = __fmaf_rn(-Sx, Bkz, sel3(B0, B1, B2, kx)), By = __fmaf_rn(-Sy, Bkz, sel3(B0, B1, B2, ky));
            float Cx = __fmaf_rn(-Sx, Ckz, sel3(C0, C1, C2, kx)), Cy = __fmaf_rn(-Sy, Ckz, sel3(C0, C1, C2, ky));
            float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
            float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
            float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
            bool inside = !((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f));
            float det = U + V + W;
            if (inside && det != 0.f) {
                float T = fmaf(U, Sz * Akz, fmaf(V, Sz * Bkz, W * (Sz * Ckz)));
                float t = __fdiv_rn(T, det);
                int prim = __float_as_int(v0.w);
                if (t >= ta && t <= tbest && (!found || t < tbest || prim < best.prim)) {
                    float rd = __frcp_rn(det);
                    tbest = t;
                    best.t = t;
                    best.prim = prim;
                    best.u = V * rd;
                    best.v = W * rd;
                    found = true;
                    if (any_hit) break;
                }
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return found;
}

// ---------------------------------------------------------------------------
// Distance-field segment.  Section 1 names distance-field tracing as the fast
// technique but the paper gives no step rule; this is plain sphere tracing on
// the trilinear interpolant, with every rounding written out:
//   clip [ta, tb] to the grid box; t = ta; up to max_steps times:
//     p = fma(t, d, o); phi = trilinear(p); phi < eps_hit -> hit at t;
//     t = t + max(phi, eps_min); t > tb -> miss
// trilinear: u = (p - lo) * (1/h), clamped to [0, n-1]; i0 = min(floor(u), n-2);
// f = u - i0; lerp(a, b, f) = fma(f, b - a, a) along x, then y, then z.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float grid_at(const TraceArgs& a, int64_t i)
{
    if (a.grid_f16) return __half2float(__ldg(reinterpret_cast<const __half*>(a.grid) + i));
    return __ldg(reinterpret_cast<const float*>(a.grid) + i);
}

struct Cell {
    int64_t base;
    float f[3];
    bool clamped[3];
};

__device__ __forceinline__ Cell locate(const TraceArgs& a, float px, float py, float pz)
{
    Cell c;
    const float p[3] = {px, py, pz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float u = __fmul_rn(__fsub_rn(p[k], a.glo[k]), a.gih[k]);
        float top = (float)(a.gn[k] - 1);
        c.clamped[k] = (u < 0.f) || (u > top);
        u = fminf(fmaxf(u, 0.f), top);
        int ii = (int)floorf(u);
        if (ii > a.gn[k] - 2) ii = a.gn[k] - 2;
        c.f[k] = __fsub_rn(u, (float)ii);
        if (k == 0) c.base = ii;
        else if (k == 1) c.base += (int64_t)a.gn[0] * ii;
        else c.base += (int64_t)a.gn[0] * a.gn[1] * ii;
    }
    return c;
}

__device__ __forceinline__ float lerp_rn(float f, float x, float y) { return __fmaf_rn(f, __fsub_rn(y, x), x); }

__device__ __forceinline__ float trilinear(const TraceArgs& a, float px, float py, float pz)
{
    Cell c = locate(a, px, py, pz);
    const int64_t sy = a.gn[0], sz = (int64_t)a.gn[0] * a.gn[1];
    float v000 = grid_at(a, c.base), v100 = grid_at(a, c.base + 1);
    float v010 = grid_at(a, c.base + sy), v110 = grid_at(a, c.base + sy + 1);
    float v001 = grid_at(a, c.base + sz), v101 = grid_at(a, c.base + sz + 1);
    float v011 = grid_at(a, c.base + sz + sy), v111 = grid_at(a, c.base + sz + sy + 1);
    float c00 = lerp_rn(c.f[0], v000, v100);
    float c10 = lerp_rn(c.f[0], v010, v110);
    float c01 = lerp_rn(c.f[0], v001, v101);
    float c11 = lerp_rn(c.f[0], v011, v111);
    float c0 = lerp_rn(c.f[1], c00, c10);
    float c1 = lerp_rn(c.f[1], c01, c11);
    return lerp_rn(c.f[2], c0, c1);
}

__device__ __forceinline__ bool clip_grid(const TraceArgs& a, float3 o, float3 d, float& ta, float& tb)
{
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (fabsf(dd[k]) < 1e-30f) {
            if (oo[k] < a.glo[k] || oo[k] > a.ghi[k]) return false;
        } else {
            float inv = __frcp_rn(dd[k]);
            float t0 = __fmul_rn(__fsub_rn(a.glo[k], oo[k]), inv);
            float t1 = __fmul_rn(__fsub_rn(a.ghi[k], oo[k]), inv);
            if (t0 > t1) { float s = t0; t0 = t1; t1 = s; }
            ta = fmaxf(ta, t0);
            tb = fminf(tb, t1);
        }
    }
    return ta <= tb;
}

// March result: hit flag, hit t, the last t before it (NaN if the first sample hit)
struct March {
    bool hit;
    float t, t_prev;
};

template <bool COUNT>
__device__ __forceinline__ March sdf_march(const TraceArgs& a, float3 o, float3 d, float ta, float tb,
                                           uint32_t& flags, Counts& cnt)
{
    March m = {false, ta, __int_as_float(0x7fc00000)};
    if (!clip_grid(a, o, d, ta, tb)) return m;
    if (COUNT) ++cnt.field;
    float t = ta;
    for (int k = 0; k < a.max_steps; ++k) {
        float px = __fmaf_rn(t, d.x, o.x), py = __fmaf_rn(t, d.y, o.y), pz = __fmaf_rn(t, d.z, o.z);
        float phi = trilinear(a, px, py, pz);
        if (COUNT) ++cnt.steps;
        if (phi < a.eps_hit) {
            m.hit = true;
            m.t = t;
            return m;
        }
        m.t_prev = t;
        t = __fadd_rn(t, fmaxf(phi, a.eps_min));
        if (t > tb) return m;
    }
    flags |= RT_FLAG_STEP_LIMIT;
    return m;
}

// root of phi(o + s d) = eps_hit inside the last step [t_prev, t] (24 halvings)
__device__ __forceinline__ float refine(const TraceArgs& a, float3 o, float3 d, float t_prev, float t)
{
    float lo = t_prev, hi = t;
    for (int it = 0; it < 24; ++it) {
        float mid = 0.5f * (lo + hi);
        float phi = trilinear(a, __fmaf_rn(mid, d.x, o.x), __fmaf_rn(mid, d.y, o.y), __fmaf_rn(mid, d.z, o.z));
        if (phi < a.eps_hit) hi = mid; else lo = mid;
    }
    return 0.5f * (lo + hi);
}

// Split points of Eq. 2 (Section 3): t_1 = clamp(t_min + m_near h, t_min, t_max),
// t_2 = clamp(t_max - m_far h, t_1, t_max).
struct Split {
    float t1, t2;
    bool near_bvh, field, far_bvh;
};

__device__ __forceinline__ Split make_split(const TraceArgs& a, float tmin, float tmax)
{
    Split s;
    s.t1 = fminf(fmaxf(__fmaf_rn(a.m_near, a.hsplit, tmin), tmin), tmax);
    s.t2 = fminf(fmaxf(__fmaf_rn(-a.m_far, a.hsplit, tmax), s.t1), tmax);
    s.near_bvh = a.m_near > 0.f;
    if (a.mode == RT_MODE_SPLIT1) {
        s.field = (a.m_near == 0.f) || (s.t1 < tmax);
        s.far_bvh = false;
        s.t2 = tmax;
    } else {
        s.field = (s.t1 < s.t2) || (a.m_near == 0.f && a.m_far == 0.f);
        s.far_bvh = a.m_far > 0.f;
    }
    return s;
}

}  // namespace rtdev
