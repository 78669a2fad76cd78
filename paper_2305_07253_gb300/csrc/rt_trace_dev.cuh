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

// 32-byte read-only vector load (sm_100 family); p must be 32-byte aligned.
// Not volatile: the load has no side effect, so the compiler may schedule it.
__device__ __forceinline__ void ldg8(const void* p, float v[8])
{
#ifdef RT_LDG8_VOLATILE
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
#else
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
#endif
}

// a 64-byte node as two 32-byte vectors (default) or four 16-byte ones
__device__ __forceinline__ void load_node(const BNode* nodes, int node, float v[8], float w[8])
{
    const float* np = reinterpret_cast<const float*>(nodes + node);
#ifdef RT_NODE_LOAD128
    const float4* q = reinterpret_cast<const float4*>(np);
    float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    w[0] = c.x; w[1] = c.y; w[2] = c.z; w[3] = c.w; w[4] = d.x; w[5] = d.y; w[6] = d.z; w[7] = d.w;
#else
    ldg8(np, v);
    ldg8(np + 8, w);
#endif
}

// ---------------------------------------------------------------------------
// Triangle segment: closest (or any) hit on [ta, tb] through the BVH, with
// the watertight ray/triangle test of Woop, Benthin & Wald (JCGT 2013) in
// float.  The edge functions are products and a difference rounded
// separately (no fused multiply-add), so two triangles sharing an edge
// evaluate that edge to exactly opposite values and no ray slips between
// them.  Ties in t go to the smaller triangle index.
// ---------------------------------------------------------------------------
struct BvhRay {
    float3 o, idir, ood;
    float Sx, Sy, Sz;
    int kx, ky, kz;
};

__device__ __forceinline__ BvhRay bvh_ray(float3 o, float3 d)
{
    BvhRay r;
    r.o = o;
    // safe reciprocal: components below 2^-80 behave like 2^-80 (slabs stay finite)
    const float eps = 8.27180613e-25f;
    r.idir = make_float3(1.0f / (fabsf(d.x) > eps ? d.x : copysignf(eps, d.x)),
                         1.0f / (fabsf(d.y) > eps ? d.y : copysignf(eps, d.y)),
                         1.0f / (fabsf(d.z) > eps ? d.z : copysignf(eps, d.z)));
    r.ood = make_float3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
    // watertight set-up: dominant axis kz, shear constants
    int kz = 0;
    float az = fabsf(d.x);
    if (fabsf(d.y) > az) { kz = 1; az = fabsf(d.y); }
    if (fabsf(d.z) > az) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dkz = sel3(d.x, d.y, d.z, kz);
    if (dkz < 0.f) { int s = kx; kx = ky; ky = s; }
    r.Sx = __fdiv_rn(sel3(d.x, d.y, d.z, kx), dkz);
    r.Sy = __fdiv_rn(sel3(d.x, d.y, d.z, ky), dkz);
    r.Sz = __frcp_rn(dkz);
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    return r;
}

// three-input maximum / minimum (one instruction on sm_100 and later; exact, as a
// chain of two-input ones is, for the finite slab distances they take)
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Slab tests of both children of one node against [ta, tf]; 64-byte node read
// as two 32-byte vectors.
struct NodeHit {
    int nearc, farc;
    bool h0, h1;
};

__device__ __forceinline__ NodeHit visit_node(const BNode* nodes, int node, const BvhRay& r, float ta, float tf)
{
    float v[8], w[8];
    load_node(nodes, node, v, w);
    // v = a (c0 x/y), b (c1 x/y); w = c (z of both), d (children)
    float x0 = fmaf(v[0], r.idir.x, -r.ood.x), x1 = fmaf(v[1], r.idir.x, -r.ood.x);
    float y0 = fmaf(v[2], r.idir.y, -r.ood.y), y1 = fmaf(v[3], r.idir.y, -r.ood.y);
    float z0 = fmaf(w[0], r.idir.z, -r.ood.z), z1 = fmaf(w[1], r.idir.z, -r.ood.z);
    float tn0 = fmaxf(max3f(fminf(x0, x1), fminf(y0, y1), fminf(z0, z1)), ta);
    float tf0 = fminf(min3f(fmaxf(x0, x1), fmaxf(y0, y1), fmaxf(z0, z1)), tf);
    x0 = fmaf(v[4], r.idir.x, -r.ood.x); x1 = fmaf(v[5], r.idir.x, -r.ood.x);
    y0 = fmaf(v[6], r.idir.y, -r.ood.y); y1 = fmaf(v[7], r.idir.y, -r.ood.y);
    z0 = fmaf(w[2], r.idir.z, -r.ood.z); z1 = fmaf(w[3], r.idir.z, -r.ood.z);
    float tn1 = fmaxf(max3f(fminf(x0, x1), fminf(y0, y1), fminf(z0, z1)), ta);
    float tf1 = fminf(min3f(fmaxf(x0, x1), fmaxf(y0, y1), fmaxf(z0, z1)), tf);
    NodeHit h;
    h.h0 = tn0 <= tf0;
    h.h1 = tn1 <= tf1;
    int c0 = __float_as_int(w[4]), c1 = __float_as_int(w[5]);
    bool swap = h.h0 && h.h1 && tn1 < tn0;
    h.nearc = swap ? c1 : c0;
    h.farc = swap ? c0 : c1;
    return h;
}

// Watertight test of triangle `tri` (leaf order); on acceptance updates best/tbest.
__device__ __forceinline__ bool test_triangle(const float4* tris, int tri, const BvhRay& r, float ta, float& tbest,
                                              bool found, Hit& best)
{
    const float4* tp = tris + 3 * (int64_t)tri;
    float4 v0 = ldg4(tp), v1 = ldg4(tp + 1), v2 = ldg4(tp + 2);
    const float3 o = r.o;
    float A0 = v0.x - o.x, A1 = v0.y - o.y, A2 = v0.z - o.z;
    float B0 = v1.x - o.x, B1 = v1.y - o.y, B2 = v1.z - o.z;
    float C0 = v2.x - o.x, C1 = v2.y - o.y, C2 = v2.z - o.z;
    const int kx = r.kx, ky = r.ky, kz = r.kz;
    float Akz = sel3(A0, A1, A2, kz), Bkz = sel3(B0, B1, B2, kz), Ckz = sel3(C0, C1, C2, kz);
    float Ax = __fmaf_rn(-r.Sx, Akz, sel3(A0, A1, A2, kx)), Ay = __fmaf_rn(-r.Sy, Akz, sel3(A0, A1, A2, ky));
    float Bx = __fmaf_rn(-r.Sx, Bkz, sel3(B0, B1, B2, kx)), By = __fmaf_rn(-r.Sy, Bkz, sel3(B0, B1, B2, ky));
    float Cx = __fmaf_rn(-r.Sx, Ckz, sel3(C0, C1, C2, kx)), Cy = __fmaf_rn(-r.Sy, Ckz, sel3(C0, C1, C2, ky));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    bool inside = !((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f));
    float det = U + V + W;
    if (!inside || det == 0.f) return false;
    float T = fmaf(U, r.Sz * Akz, fmaf(V, r.Sz * Bkz, W * (r.Sz * Ckz)));
    float t = __fdiv_rn(T, det);
    int prim = __float_as_int(v0.w);
    if (t >= ta && t <= tbest && (!found || t < tbest || prim < best.prim)) {
        float rd = __frcp_rn(det);
        tbest = t;
        best.t = t;
        best.prim = prim;
        best.u = V * rd;
        best.v = W * rd;
        return true;
    }
    return false;
}

// Traversal iterations a lane runs between two refill checks of its warp.  With
// warp-wide refills (refill_min 32) a warp takes new queries only once every
// lane is idle, so checks in between are pure overhead: the trip runs until the
// lane's segment ends (up to 256 iterations).  Measured on the 1080p GI
// workload, near-triangle stage: 0.256 ms with 8, 0.232 ms with 32 to 4096.
// With partial refills the check comes every 8 iterations.
__host__ __device__ __forceinline__ int trip_budget(int refill_min) { return refill_min >= 32 ? 256 : 8; }

// Resumable traversal state of one segment.
struct Trav {
    int node;
    int sp;
    float ta, tbest;
    bool found;
    uint32_t guard;
};

__device__ __forceinline__ Trav trav_begin(int root, float ta, float tb)
{
    Trav s;
    s.node = root;
    s.sp = 0;
    s.ta = ta;
    s.tbest = tb;
    s.found = false;
    s.guard = 0;
    return s;
}

// Up to `budget` traversal iterations; each iteration visits one internal node
// or tests one leaf (lanes at leaves and lanes at inner nodes share every
// iteration, so none waits for the others to reach a leaf).  Returns true when
// the segment is done.  (Keeping the far child's entry distance on the stack
// to skip stale entries saved 3% of the node visits on the 1080p GI workload
// but cost more in local-memory traffic than it saved.)
template <bool COUNT>
__device__ __forceinline__ bool trav_trip(const TraceArgs& a, const BvhRay& r, Trav& s, int* stack, bool any_hit,
                                          Hit& best, uint32_t& flags, Counts& cnt, int budget)
{
    for (int it = 0; it < budget; ++it) {
        if (s.node >= 0) {
            if (COUNT) ++cnt.nodes;
            NodeHit h = visit_node(a.nodes, s.node, r, s.ta, s.tbest);
            if (h.h0 && h.h1) {
                if (s.sp < RT_STACK_DEPTH) stack[s.sp++] = h.farc;
                else flags |= RT_FLAG_STACK_OVERFLOW;
                s.node = h.nearc;
                continue;
            }
            if (h.h0 || h.h1) {
                s.node = h.h0 ? h.nearc : h.farc;
                continue;
            }
        } else {
            if (COUNT) ++cnt.tris;
            if (test_triangle(a.tris, ~s.node, r, s.ta, s.tbest, s.found, best)) {
                s.found = true;
                if (any_hit) return true;
            }
        }
        if (s.sp == 0) return true;
        s.node = stack[--s.sp];
    }
    // a tree visit is bounded by 2n-1 nodes: the guard, charged a trip at a time
    // (checking it every iteration cost 2 % of the triangles-only time), stops
    // only a corrupt structure
    s.guard += (uint32_t)budget;
    if (s.guard >= (1u << 26)) {
        flags |= RT_FLAG_ITER_LIMIT;
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// 8-wide compressed tree (layout in rt_internal.cuh).  Each iteration tests one
// triangle or visits one node: the 8 child boxes are decoded from their 8-bit
// bounds and slab-tested, inner children that are hit go into a group mask in
// rank order (rank = slot xor ray octant, roughly near to far), leaf triangles
// that are hit into a triangle mask.  Groups wait on a stack of 64-bit entries
// (first child, inner mask, remaining ranks).
// ---------------------------------------------------------------------------
struct WTrav {
    uint32_t base;    // first child of the node whose children form the group
    uint32_t masks;   // inner mask (bits 0-7) | remaining ranks (bits 8-15)
    uint32_t tbase;   // first triangle of the node whose leaves are pending
    uint32_t tmask;   // pending triangles (bit = offset from tbase)
    int sp;
    float ta, tbest;
    bool found;
    uint32_t guard;
    int oct;
};

__device__ __forceinline__ WTrav wtrav_begin(const BvhRay& r, float ta, float tb)
{
    WTrav s;
    s.oct = (r.idir.x < 0.f ? 1 : 0) | (r.idir.y < 0.f ? 2 : 0) | (r.idir.z < 0.f ? 4 : 0);
    s.base = 0;                           // the root: a group of one inner child in slot 0
    s.masks = 1u | ((1u << (0 ^ s.oct)) << 8);
    s.tbase = 0;
    s.tmask = 0;
    s.sp = 0;
    s.ta = ta;
    s.tbest = tb;
    s.found = false;
    s.guard = 0;
    return s;
}

__device__ __forceinline__ float byte_to_float(uint32_t w, int k)
{
    return __uint_as_float(0x4B000000u | ((w >> (8 * k)) & 0xffu)) - 8388608.0f;
}

// slab tests of the 8 children of wide node w; returns the new group and leaf masks.
// The ray's octant picks, per axis, which of the two quantized planes is the
// entry plane, so each child costs 6 FMAs and two 4-way min/max.
__device__ __forceinline__ void visit_wide(const WNode* nodes, uint32_t w, const BvhRay& r, WTrav& s)
{
    const uint4* np = reinterpret_cast<const uint4*>(nodes + w);
    const float4 na = __ldg(reinterpret_cast<const float4*>(np));
    const uint4 nb = __ldg(np + 1), q0 = __ldg(np + 2), q1 = __ldg(np + 3), q2 = __ldg(np + 4);
    const uint32_t bits = __float_as_uint(na.w);
    const float sx = __uint_as_float((bits & 0xffu) << 23) * r.idir.x;
    const float sy = __uint_as_float(((bits >> 8) & 0xffu) << 23) * r.idir.y;
    const float sz = __uint_as_float(((bits >> 16) & 0xffu) << 23) * r.idir.z;
    const float bx = (na.x - r.o.x) * r.idir.x;
    const float by = (na.y - r.o.y) * r.idir.y;
    const float bz = (na.z - r.o.z) * r.idir.z;
    const uint32_t imask = bits >> 24;
    // entry/exit plane words per axis (lo planes for a positive direction)
    const bool fx = s.oct & 1, fy = s.oct & 2, fz = s.oct & 4;
    const uint32_t nx0 = fx ? q1.z : q0.x, nx1 = fx ? q1.w : q0.y, xx0 = fx ? q0.x : q1.z, xx1 = fx ? q0.y : q1.w;
    const uint32_t ny0 = fy ? q2.x : q0.z, ny1 = fy ? q2.y : q0.w, xy0 = fy ? q0.z : q2.x, xy1 = fy ? q0.w : q2.y;
    const uint32_t nz0 = fz ? q2.z : q1.x, nz1 = fz ? q2.w : q1.y, xz0 = fz ? q1.x : q2.z, xz1 = fz ? q1.y : q2.w;
    uint32_t rmask = 0, tmask = 0;
#pragma unroll
    for (int slot = 0; slot < 8; ++slot) {
        const int k = slot & 3;
        const bool hi = slot >= 4;
        const float tnx = fmaf(byte_to_float(hi ? nx1 : nx0, k), sx, bx);
        const float tny = fmaf(byte_to_float(hi ? ny1 : ny0, k), sy, by);
        const float tnz = fmaf(byte_to_float(hi ? nz1 : nz0, k), sz, bz);
        const float tfx = fmaf(byte_to_float(hi ? xx1 : xx0, k), sx, bx);
        const float tfy = fmaf(byte_to_float(hi ? xy1 : xy0, k), sy, by);
        const float tfz = fmaf(byte_to_float(hi ? xz1 : xz0, k), sz, bz);
        const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, s.ta));
        const float tf = fminf(fminf(tfx, tfy), fminf(tfz, s.tbest));
        if (tn <= tf) {
            if (imask & (1u << slot)) {
                rmask |= 1u << (slot ^ s.oct);
            } else {
                const uint32_t meta = ((hi ? nb.w : nb.z) >> (8 * k)) & 0xffu;
                if (meta) tmask |= ((1u << (meta >> 5)) - 1u) << (meta & 31u);
            }
        }
    }
    s.base = nb.x;
    s.masks = imask | (rmask << 8);
    s.tbase = nb.y;
    s.tmask = tmask;
}

// One iteration: test all triangles of the last visited node that were hit,
// then visit the next node (so the lanes visit nodes together), or pop a group.
template <bool COUNT>
__device__ __forceinline__ bool wtrav_trip(const TraceArgs& a, const BvhRay& r, WTrav& s, uint64_t* stack,
                                           bool any_hit, Hit& best, uint32_t& flags, Counts& cnt, int budget)
{
    for (int it = 0; it < budget; ++it) {
        if (++s.guard > (1u << 26)) {  // bounded by the tree size; stops only a corrupt structure
            flags |= RT_FLAG_ITER_LIMIT;
            return true;
        }
        while (s.tmask) {
            const int bit = __ffs(s.tmask) - 1;
            s.tmask &= s.tmask - 1u;
            if (COUNT) ++cnt.tris;
            if (test_triangle(a.wtris, (int)(s.tbase + bit), r, s.ta, s.tbest, s.found, best)) {
                s.found = true;
                if (any_hit) return true;
            }
        }
        uint32_t rm = s.masks >> 8;
        if (rm == 0) {
            if (s.sp == 0) return true;
            const uint64_t e = stack[--s.sp];
            s.base = (uint32_t)(e >> 32);
            s.masks = (uint32_t)e;
            rm = s.masks >> 8;
        }
        const int rank = __ffs(rm) - 1;
        rm &= rm - 1u;
        const uint32_t imask = s.masks & 0xffu;
        const int slot = rank ^ s.oct;
        const uint32_t w = s.base + __popc(imask & ((1u << slot) - 1u));
        if (rm) {
            if (s.sp < RT_WSTACK_DEPTH) stack[s.sp++] = ((uint64_t)s.base << 32) | imask | (rm << 8);
            else flags |= RT_FLAG_STACK_OVERFLOW;
        }
        if (COUNT) ++cnt.nodes;
        visit_wide(a.wnodes, w, r, s);
    }
    return false;
}

// The traversal of either tree behind one interface for the kernels.
template <bool WIDE> struct TravOf;
template <> struct TravOf<false> {
    using state = Trav;
    using entry = int;
    static constexpr int depth = RT_STACK_DEPTH;
};
template <> struct TravOf<true> {
    using state = WTrav;
    using entry = uint64_t;
    static constexpr int depth = RT_WSTACK_DEPTH;
};

template <bool WIDE>
__device__ __forceinline__ typename TravOf<WIDE>::state tbegin(const TraceArgs& a, const BvhRay& r, float ta, float tb)
{
    if constexpr (WIDE) return wtrav_begin(r, ta, tb);
    else return trav_begin(a.root, ta, tb);
}

template <bool COUNT, bool WIDE>
__device__ __forceinline__ bool ttrip(const TraceArgs& a, const BvhRay& r, typename TravOf<WIDE>::state& s,
                                      typename TravOf<WIDE>::entry* stack, bool any_hit, Hit& best, uint32_t& flags,
                                      Counts& cnt, int budget)
{
    if constexpr (WIDE) return wtrav_trip<COUNT>(a, r, s, stack, any_hit, best, flags, cnt, budget);
    else return trav_trip<COUNT>(a, r, s, stack, any_hit, best, flags, cnt, budget);
}

// Whole triangle segment in one call (used by the one-thread-per-query kernel).
template <bool COUNT, bool WIDE = false>
__device__ __forceinline__ bool bvh_segment(const TraceArgs& a, float3 o, float3 d, float ta, float tb, bool any_hit,
                                            Hit& best, uint32_t& flags, Counts& cnt)
{
    if (a.root == INT32_MIN || !(ta <= tb)) return false;
    const BvhRay r = bvh_ray(o, d);
    typename TravOf<WIDE>::entry stack[TravOf<WIDE>::depth];
    typename TravOf<WIDE>::state s = tbegin<WIDE>(a, r, ta, tb);
    while (!ttrip<COUNT, WIDE>(a, r, s, stack, any_hit, best, flags, cnt, 1 << 26)) {
    }
    return s.found;
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
// Grid storage seen by the march, fixed at compile time so that a step has no
// layout or type branches: the caller's plain grid (float32 / float16) or the
// library's cell-corner copy (float32 / float16).
enum GridLayout { GL_PLAIN_F32 = 0, GL_PLAIN_F16 = 1, GL_CELLS_F32 = 2, GL_CELLS_F16 = 3, GL_PAIRS_F32 = 4,
                  GL_PAIRS_F16 = 5, GL_CASC_F32 = 6, GL_CASC_F16 = 7 };

__host__ __device__ constexpr bool is_cascade(int L) { return L == GL_CASC_F32 || L == GL_CASC_F16; }

__host__ __device__ __forceinline__ int grid_layout_of(const TraceArgs& a)
{
    if (a.levels > 0) return GL_CASC_F32 + (a.grid_f16 ? 1 : 0);
    return (a.cells ? 2 : (a.pairs ? 4 : 0)) + (a.grid_f16 ? 1 : 0);
}

template <int L>
__device__ __forceinline__ float grid_at(const TraceArgs& a, int64_t i)
{
    if (L == GL_PLAIN_F16 || L == GL_CELLS_F16) return __half2float(__ldg(reinterpret_cast<const __half*>(a.grid) + i));
    return __ldg(reinterpret_cast<const float*>(a.grid) + i);
}

struct Cell {
    int i0[3];
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
        c.i0[k] = ii;
    }
    return c;
}

__device__ __forceinline__ int64_t grid_base(const TraceArgs& a, const Cell& c)
{
    return c.i0[0] + (int64_t)a.gn[0] * (c.i0[1] + (int64_t)a.gn[1] * c.i0[2]);
}

// Position of cell (i, j, k) in the cell copy, x fastest.  Orders that keep
// 3-d neighbours in one 128-byte line were measured on the 1080p GI workload,
// records unchanged: 2x2 blocks in x-y 0.743 ms, 2x2x2 blocks 0.750 ms,
// against 0.739 ms; a 4x4x4 brick order 0.855 against 0.837 ms (earlier kernel).
__host__ __device__ __forceinline__ int64_t cell_slot(int i, int j, int k, int nx, int ny)
{
    return i + (int64_t)(nx - 1) * (j + (int64_t)(ny - 1) * k);
}

// cells the copy of an nx x ny x nz grid holds
__host__ __device__ __forceinline__ int64_t cell_count(int nx, int ny, int nz)
{
    return (int64_t)(nx - 1) * (ny - 1) * (nz - 1);
}

__device__ __forceinline__ int64_t cell_index(const TraceArgs& a, const Cell& c)
{
    return cell_slot(c.i0[0], c.i0[1], c.i0[2], a.gn[0], a.gn[1]);
}

// the 8 corner values of the cell, order v000 v100 v010 v110 v001 v101 v011 v111
template <int L>
__device__ __forceinline__ void corners(const TraceArgs& a, const Cell& c, float v[8])
{
    if (L == GL_CELLS_F16) {
        uint4 q = __ldg(reinterpret_cast<const uint4*>(a.cells) + cell_index(a, c));
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __half2 h2 = *reinterpret_cast<const __half2*>(&w[k]);
            v[2 * k] = __low2float(h2);
            v[2 * k + 1] = __high2float(h2);
        }
        return;
    }
    if (L == GL_CELLS_F32) {
        ldg8(reinterpret_cast<const float*>(a.cells) + 8 * cell_index(a, c), v);
        return;
    }
    if (L == GL_PAIRS_F32 || L == GL_PAIRS_F16) {
        const int64_t px = a.gn[0] - 1;
        const int64_t p00 = c.i0[0] + px * (c.i0[1] + (int64_t)a.gn[1] * c.i0[2]);
        const int64_t sy = px, sz = px * a.gn[1];
        const int64_t idx[4] = {p00, p00 + sy, p00 + sz, p00 + sz + sy};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (L == GL_PAIRS_F32) {
                const float2 e = __ldg(reinterpret_cast<const float2*>(a.pairs) + idx[q]);
                v[2 * q] = e.x;
                v[2 * q + 1] = e.y;
            } else {
                const __half2 e = __ldg(reinterpret_cast<const __half2*>(a.pairs) + idx[q]);
                v[2 * q] = __low2float(e);
                v[2 * q + 1] = __high2float(e);
            }
        }
        return;
    }
    const int64_t b = grid_base(a, c);
    const int64_t sy = a.gn[0], sz = (int64_t)a.gn[0] * a.gn[1];
    v[0] = grid_at<L>(a, b);
    v[1] = grid_at<L>(a, b + 1);
    v[2] = grid_at<L>(a, b + sy);
    v[3] = grid_at<L>(a, b + sy + 1);
    v[4] = grid_at<L>(a, b + sz);
    v[5] = grid_at<L>(a, b + sz + 1);
    v[6] = grid_at<L>(a, b + sz + sy);
    v[7] = grid_at<L>(a, b + sz + sy + 1);
}

__device__ __forceinline__ float lerp_rn(float f, float x, float y) { return __fmaf_rn(f, __fsub_rn(y, x), x); }

// trilinear interpolation of the 8 corners (order as in corners()) at the cell fractions f
__device__ __forceinline__ float interp8(const float f[3], const float v[8])
{
    float c00 = lerp_rn(f[0], v[0], v[1]);
    float c10 = lerp_rn(f[0], v[2], v[3]);
    float c01 = lerp_rn(f[0], v[4], v[5]);
    float c11 = lerp_rn(f[0], v[6], v[7]);
    float c0 = lerp_rn(f[1], c00, c10);
    float c1 = lerp_rn(f[1], c01, c11);
    return lerp_rn(f[2], c0, c1);
}

// the 8 corners of a 16-byte half-precision cell, held as 4 words in v[0..3], widened in place
__device__ __forceinline__ void widen_f16_cell(float v[8])
{
    const uint32_t w[4] = {__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3])};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h2 = *reinterpret_cast<const __half2*>(&w[k]);
        v[2 * k] = __low2float(h2);
        v[2 * k + 1] = __high2float(h2);
    }
}

template <int L>
__device__ __forceinline__ float trilinear(const TraceArgs& a, float px, float py, float pz)
{
    Cell c = locate(a, px, py, pz);
    float v[8];
    corners<L>(a, c, v);
    return interp8(c.f, v);
}

// ---------------------------------------------------------------------------
// cascade (Section 3, "Distance Field Generation"): the finest level whose
// closed box holds p (the coarsest outside all boxes; a NaN point is outside
// every box); trilinear sample of that level from its cells
// ---------------------------------------------------------------------------
__device__ __forceinline__ int casc_level(const TraceArgs& a, float px, float py, float pz)
{
    int k = 0;
    for (; k < a.levels - 1; ++k) {
        const CascLevel& v = a.lv[k];
        if (px >= v.lo[0] && px <= v.hi[0] && py >= v.lo[1] && py <= v.hi[1] && pz >= v.lo[2] && pz <= v.hi[2])
            break;
    }
    return k;
}

// the cell of level k that holds p (its index in the cell copy) and p's fractions in it
__device__ __forceinline__ int64_t casc_locate(const TraceArgs& a, int k, float px, float py, float pz, float f[3])
{
    const CascLevel& lv = a.lv[k];
    const float p[3] = {px, py, pz};
    const float top = (float)(a.gn[0] - 1);
    int i0[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float u = __fmul_rn(__fsub_rn(p[ax], lv.lo[ax]), lv.ih);
        u = fminf(fmaxf(u, 0.f), top);
        int ii = (int)floorf(u);
        if (ii > a.gn[0] - 2) ii = a.gn[0] - 2;
        f[ax] = __fsub_rn(u, (float)ii);
        i0[ax] = ii;
    }
    return k * a.level_cells + cell_slot(i0[0], i0[1], i0[2], a.gn[0], a.gn[0]);
}

template <int L>
__device__ __forceinline__ float casc_trilinear(const TraceArgs& a, int k, float px, float py, float pz)
{
    float f[3];
    const int64_t idx = casc_locate(a, k, px, py, pz, f);
    float v[8];
    if (L == GL_CASC_F16) {
        uint4 q = __ldg(reinterpret_cast<const uint4*>(a.cells) + idx);
        v[0] = __uint_as_float(q.x);
        v[1] = __uint_as_float(q.y);
        v[2] = __uint_as_float(q.z);
        v[3] = __uint_as_float(q.w);
        widen_f16_cell(v);
    } else {
        ldg8(reinterpret_cast<const float*>(a.cells) + 8 * idx, v);
    }
    return interp8(f, v);
}

// field value and the hit / minimum-step thresholds at p: one grid, or the
// level of a cascade that holds p (thresholds scale with its voxel)
template <int L>
__device__ __forceinline__ float field_at(const TraceArgs& a, float px, float py, float pz, float& eps_hit,
                                          float& eps_min)
{
    if constexpr (is_cascade(L)) {
        const int k = casc_level(a, px, py, pz);
        eps_hit = a.lv[k].eps_hit;
        eps_min = a.lv[k].eps_min;
        return casc_trilinear<L>(a, k, px, py, pz);
    } else {
        eps_hit = a.eps_hit;
        eps_min = a.eps_min;
        return trilinear<L>(a, px, py, pz);
    }
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

// One march step at t; returns 0 to continue, 1 on a hit, 2 on leaving [.., tb].
template <int L>
__device__ __forceinline__ int march_step(const TraceArgs& a, float3 o, float3 d, float& t, float tb, float& t_prev)
{
    float px = __fmaf_rn(t, d.x, o.x), py = __fmaf_rn(t, d.y, o.y), pz = __fmaf_rn(t, d.z, o.z);
    float eps_hit, eps_min;
    float phi = field_at<L>(a, px, py, pz, eps_hit, eps_min);
    if (phi < eps_hit) return 1;
    t_prev = t;
    t = __fadd_rn(t, fmaxf(phi, eps_min));
    return t > tb ? 2 : 0;
}

template <bool COUNT, int L>
__device__ __forceinline__ March sdf_march(const TraceArgs& a, float3 o, float3 d, float ta, float tb,
                                           uint32_t& flags, Counts& cnt)
{
    March m = {false, ta, __int_as_float(0x7fc00000)};
    if (!clip_grid(a, o, d, ta, tb)) return m;
    if (COUNT) ++cnt.field;
    float t = ta;
    for (int k = 0; k < a.max_steps; ++k) {
        if (COUNT) ++cnt.steps;
        int r = march_step<L>(a, o, d, t, tb, m.t_prev);
        if (r == 1) {
            m.hit = true;
            m.t = t;
            return m;
        }
        if (r == 2) return m;
    }
    flags |= RT_FLAG_STEP_LIMIT;
    return m;
}

// root of phi(o + s d) = eps_hit inside the last step [t_prev, t] (24 halvings)
template <int L>
__device__ __forceinline__ float refine(const TraceArgs& a, float3 o, float3 d, float t_prev, float t)
{
    float lo = t_prev, hi = t;
    for (int it = 0; it < 24; ++it) {
        float mid = 0.5f * (lo + hi);
        float eps_hit, eps_min;
        float phi = field_at<L>(a, __fmaf_rn(mid, d.x, o.x), __fmaf_rn(mid, d.y, o.y), __fmaf_rn(mid, d.z, o.z),
                                eps_hit, eps_min);
        if (phi < eps_hit) hi = mid; else lo = mid;
    }
    return 0.5f * (lo + hi);
}

// Split points of Eq. 2 (Section 3): t_1 = clamp(t_min + m_near h_1, t_min, t_max),
// t_2 = clamp(t_max - m_far h_2, t_1, t_max).  One grid: h_1 = h_2 = its
// largest voxel edge.  Cascade: the voxel at the start point o + t_min d and at
// the end point o + t_max d (Section 3, "GI & Shadow Rays").
struct Split {
    float t1, t2;
    bool near_bvh, field, far_bvh;
};

__device__ __forceinline__ Split make_split(int mode, float m_near, float m_far, float h_near, float h_far,
                                            float tmin, float tmax)
{
    Split s;
    s.t1 = fminf(fmaxf(__fmaf_rn(m_near, h_near, tmin), tmin), tmax);
    s.t2 = fminf(fmaxf(__fmaf_rn(-m_far, h_far, tmax), s.t1), tmax);
    s.near_bvh = m_near > 0.f;
    if (mode == RT_MODE_SPLIT1) {
        s.field = (m_near == 0.f) || (s.t1 < tmax);
        s.far_bvh = false;
        s.t2 = tmax;
    } else {
        s.field = (s.t1 < s.t2) || (m_near == 0.f && m_far == 0.f);
        s.far_bvh = m_far > 0.f;
    }
    return s;
}

// voxel edges that set t_1 and t_2 for the query (o, d, t_min, t_max)
__device__ __forceinline__ void split_voxels(const TraceArgs& a, float3 o, float3 d, float tmin, float tmax,
                                             float& h_near, float& h_far)
{
    if (a.levels > 0) {
        h_near = a.lv[casc_level(a, __fmaf_rn(tmin, d.x, o.x), __fmaf_rn(tmin, d.y, o.y), __fmaf_rn(tmin, d.z, o.z))].h;
        h_far = a.lv[casc_level(a, __fmaf_rn(tmax, d.x, o.x), __fmaf_rn(tmax, d.y, o.y), __fmaf_rn(tmax, d.z, o.z))].h;
    } else {
        h_near = h_far = a.hsplit;
    }
}

__device__ __forceinline__ Split make_split(const TraceArgs& a, float3 o, float3 d, float tmin, float tmax)
{
    float hn, hf;
    split_voxels(a, o, d, tmin, tmax, hn, hf);
    return make_split(a.mode, a.m_near, a.m_far, hn, hf, tmin, tmax);
}

// Eq. 1 is defined for real o, d and t_min <= t_max; anything else has no intersection
__device__ __forceinline__ bool valid_query(float3 o, float3 d, float tmin, float tmax)
{
    return !(isnan(o.x) || isnan(o.y) || isnan(o.z) || isnan(d.x) || isnan(d.y) || isnan(d.z)) && (tmin <= tmax);
}

// The query that slot `slot` of a call's first kernel traces (the query
// order, or input order)
__device__ __forceinline__ int64_t first_query(const TraceArgs& a, int64_t slot)
{
    return a.qorder ? (int64_t)__ldg(a.qorder + slot) : slot;
}

__device__ __forceinline__ void store_hit(rt_hit* out, float t, int32_t prim, float u, float v, int32_t tracer,
                                          uint32_t flags)
{
    float2* p = reinterpret_cast<float2*>(out);
    p[0] = make_float2(t, __int_as_float(prim));
    p[1] = make_float2(u, v);
    p[2] = make_float2(__int_as_float(tracer), __uint_as_float(flags));
}

// Append the lanes with `hit` set to a near-hit list (one atomic per warp):
// the record dst, and the hit found (prim kFlagsOnly: none, flags only).
__device__ __forceinline__ void append_hit_entry(HitEntry* list, unsigned* count, bool hit, rt_hit* dst,
                                                 const Hit& best, uint32_t flags)
{
    const unsigned full = 0xffffffffu, lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(full, hit);
    if (m == 0) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == (unsigned)leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(full, base, leader);
    if (hit) {
        HitEntry e;
        e.dst = dst;
        e.flags = flags;
        e.t = best.t;
        e.u = best.u;
        e.v = best.v;
        e.prim = best.prim;
        e.pad = 0;
        list[base + __popc(m & ((1u << lane) - 1u))] = e;
    }
}

}  // namespace rtdev
