// Device helpers of the exact distance to triangles, shared by the exact bake
// (rt_bake.cu) and the paper's field build (rt_dfgen.cu): the closest point on
// a triangle from the Voronoi regions of the triangle (Ericson, Real-Time
// Collision Detection, 5.1.5) and the sign from the angle-weighted
// pseudonormal of the closest feature (Baerentzen & Aanaes, IEEE TVCG 2005).
#pragma once

#include "rt_internal.cuh"

namespace rtbake {

__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }

// Closest point q on triangle abc to p; returns the region
// (0 face, 1/2/3 vertex a/b/c, 4 edge ab, 5 edge bc, 6 edge ca).
__device__ __forceinline__ int closest_point(float3 p, float3 a, float3 b, float3 c, float3& q)
{
    float3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
    float d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) { q = a; return 1; }
    float3 bp = sub(p, b);
    float d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.f && d4 <= d3) { q = b; return 2; }
    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        float s = d1 / (d1 - d3);
        q = make_float3(a.x + s * ab.x, a.y + s * ab.y, a.z + s * ab.z);
        return 4;
    }
    float3 cp = sub(p, c);
    float d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.f && d5 <= d6) { q = c; return 3; }
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        float s = d2 / (d2 - d6);
        q = make_float3(a.x + s * ac.x, a.y + s * ac.y, a.z + s * ac.z);
        return 6;
    }
    float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        float s = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        q = make_float3(b.x + s * (c.x - b.x), b.y + s * (c.y - b.y), b.z + s * (c.z - b.z));
        return 5;
    }
    float den = 1.f / (va + vb + vc);
    float v = vb * den, w = vc * den;
    q = make_float3(a.x + ab.x * v + ac.x * w, a.y + ab.y * v + ac.y * w, a.z + ab.z * v + ac.z * w);
    return 0;
}

struct Nearest {
    float d2;
    int32_t k;     // triangle in leaf order
    int32_t prim;  // triangle in input order (tie-break)
};

__device__ __forceinline__ void consider(Nearest& nb, float3 p, const float4* tris, int32_t k)
{
    float4 v0 = __ldg(tris + 3 * (int64_t)k), v1 = __ldg(tris + 3 * (int64_t)k + 1), v2 = __ldg(tris + 3 * (int64_t)k + 2);
    float3 q;
    closest_point(p, xyz(v0), xyz(v1), xyz(v2), q);
    float3 pq = sub(p, q);
    float d2 = dot(pq, pq);
    int32_t prim = __float_as_int(v0.w);
    if (d2 < nb.d2 || (d2 == nb.d2 && prim < nb.prim)) {
        nb.d2 = d2;
        nb.k = k;
        nb.prim = prim;
    }
}

// sign from the pseudonormal of the nearest feature; pn holds per triangle:
// face, edge ab, edge bc, edge ca, vertex a, vertex b, vertex c
__device__ __forceinline__ float signed_distance(float3 p, const Nearest& nb, const float4* tris, const float4* pn)
{
    if (nb.k < 0) return __int_as_float(0x7f800000);
    float4 v0 = __ldg(tris + 3 * (int64_t)nb.k), v1 = __ldg(tris + 3 * (int64_t)nb.k + 1),
           v2 = __ldg(tris + 3 * (int64_t)nb.k + 2);
    float3 q;
    int region = closest_point(p, xyz(v0), xyz(v1), xyz(v2), q);
    const int slot[7] = {0, 4, 5, 6, 1, 2, 3};
    float3 n = xyz(__ldg(pn + 7 * (int64_t)nb.k + slot[region]));
    float dist = sqrtf(nb.d2);
    return dot(sub(p, q), n) >= 0.f ? dist : -dist;
}

}  // namespace rtbake
