// Trace kernel: one query (Eq. 1) per thread, split into the sub-intervals of
// Eq. 2 and processed by the ordering rule of Section 2 (closest hit: in
// order, stop at the first sub-interval that hits; any hit: the distance
// field sub-interval first).  Modes 0 and 3 are the pure techniques.
#include "rt_trace_dev.cuh"

using namespace rtdev;

namespace {

constexpr int kTraceBlock = 128;

__device__ __forceinline__ void store_hit(rt_hit* out, float t, int32_t prim, float u, float v, int32_t tracer,
                                          uint32_t flags)
{
    float2* p = reinterpret_cast<float2*>(out);
    p[0] = make_float2(t, __int_as_float(prim));
    p[1] = make_float2(u, v);
    p[2] = make_float2(__int_as_float(tracer), __uint_as_float(flags));
}

template <bool COUNT>
__device__ __forceinline__ void trace_one(const TraceArgs& a, int64_t i, Counts& cnt)
{
    const float4 r0 = __ldg(a.rays + 2 * i), r1 = __ldg(a.rays + 2 * i + 1);
    const float3 o = make_float3(r0.x, r0.y, r0.z), d = make_float3(r1.x, r1.y, r1.z);
    const float tmin = r0.w, tmax = r1.w;
    Hit h = {__int_as_float(0x7f800000), -1, 0.f, 0.f};
    uint32_t flags = 0;
    int32_t tracer = RT_TRACER_MISS;
    // Eq. 1 is defined for real o, d and t_min <= t_max; anything else has no intersection
    const bool valid = !(isnan(o.x) || isnan(o.y) || isnan(o.z) || isnan(d.x) || isnan(d.y) || isnan(d.z)) &&
                       (tmin <= tmax);

    if (!valid) {
    } else if (a.mode == RT_MODE_BVH) {
        if (bvh_segment<COUNT>(a, o, d, tmin, tmax, a.any_hit, h, flags, cnt)) tracer = RT_TRACER_BVH;
    } else if (a.mode == RT_MODE_SDF) {
        March m = sdf_march<COUNT>(a, o, d, tmin, tmax, flags, cnt);
        if (m.hit) {
            tracer = RT_TRACER_SDF;
            h.t = (a.refine_root && !isnan(m.t_prev)) ? refine(a, o, d, m.t_prev, m.t) : m.t;
        }
    } else {
        const Split s = make_split(a, tmin, tmax);
        if (a.any_hit) {
            // distance field first, then the triangle sub-intervals (Section 2)
            if (s.field) {
                March m = sdf_march<COUNT>(a, o, d, s.t1, s.t2, flags, cnt);
                if (m.hit) {
                    tracer = RT_TRACER_SDF;
                    h.t = (a.refine_root && !isnan(m.t_prev)) ? refine(a, o, d, m.t_prev, m.t) : m.t;
                }
            }
            if (tracer == RT_TRACER_MISS && s.near_bvh && bvh_segment<COUNT>(a, o, d, tmin, s.t1, true, h, flags, cnt))
                tracer = RT_TRACER_BVH;
            if (tracer == RT_TRACER_MISS && s.far_bvh && bvh_segment<COUNT>(a, o, d, s.t2, tmax, true, h, flags, cnt))
                tracer = RT_TRACER_BVH;
        } else {
            // closest hit: in order, early exit (Section 2)
            if (s.near_bvh && bvh_segment<COUNT>(a, o, d, tmin, s.t1, false, h, flags, cnt)) tracer = RT_TRACER_BVH;
            if (tracer == RT_TRACER_MISS && s.field) {
                March m = sdf_march<COUNT>(a, o, d, s.t1, s.t2, flags, cnt);
                if (m.hit) {
                    tracer = RT_TRACER_SDF;
                    h.t = (a.refine_root && !isnan(m.t_prev)) ? refine(a, o, d, m.t_prev, m.t) : m.t;
                }
            }
            if (tracer == RT_TRACER_MISS && s.far_bvh && bvh_segment<COUNT>(a, o, d, s.t2, tmax, false, h, flags, cnt))
                tracer = RT_TRACER_BVH;
        }
    }
    if (tracer != RT_TRACER_BVH) {
        h.prim = -1;
        h.u = h.v = 0.f;
    }
    store_hit(a.hits + i, h.t, h.prim, h.u, h.v, tracer, flags);
}

template <bool COUNT>
__global__ void __launch_bounds__(kTraceBlock) k_trace(const TraceArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Counts cnt = {0, 0, 0, 0};
    if (i < a.n) trace_one<COUNT>(a, i, cnt);
    if (COUNT) {
        if (cnt.nodes) atomicAdd(&a.counters[0], (unsigned long long)cnt.nodes);
        if (cnt.tris) atomicAdd(&a.counters[1], (unsigned long long)cnt.tris);
        if (cnt.steps) atomicAdd(&a.counters[2], (unsigned long long)cnt.steps);
        if (cnt.field) atomicAdd(&a.counters[3], (unsigned long long)cnt.field);
    }
}

}  // namespace

rt_status rt_launch_trace(const TraceArgs& a, bool counted, cudaStream_t s)
{
    const int64_t blocks = (a.n + kTraceBlock - 1) / kTraceBlock;
    if (blocks > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "too many rays");
    if (counted) k_trace<true><<<(unsigned)blocks, kTraceBlock, 0, s>>>(a);
    else k_trace<false><<<(unsigned)blocks, kTraceBlock, 0, s>>>(a);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}
