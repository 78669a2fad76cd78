// Adjoint of the distance-field hit distance with respect to the grid values.
//
// At a field hit the root p* = o + t d of phi = eps_hit satisfies
// phi_theta(p*) = eps_hit.  phi is linear in the grid values theta
// (phi = sum_k w_k(p) theta_k with the trilinear weights w_k), so implicit
// differentiation gives dt/dtheta_k = -w_k(p*) / (grad phi(p*) . d).  The
// kernel does not read a stored forward pass: it re-marches each ray with the
// forward code (same roundings, same steps), refines the root in the last
// step and scatters grad_t * dt/dtheta_k into the gradient grid.
#include "rt_trace_dev.cuh"

using namespace rtdev;

namespace {

constexpr int kBwdBlock = 128;

template <int L>
__global__ void __launch_bounds__(kBwdBlock) k_backward(const TraceArgs a, const float* __restrict__ grad_t,
                                                        float* __restrict__ grad_grid)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int32_t tracer = a.hits[i].tracer;
    if (tracer != RT_TRACER_SDF) return;
    const float g = __ldg(grad_t + i);
    if (g == 0.f) return;
    const float4 r0 = __ldg(a.rays + 2 * i), r1 = __ldg(a.rays + 2 * i + 1);
    const float3 o = make_float3(r0.x, r0.y, r0.z), d = make_float3(r1.x, r1.y, r1.z);
    float ts = r0.w, te = r1.w;
    if (a.mode == RT_MODE_SPLIT1 || a.mode == RT_MODE_SPLIT2) {
        Split s = make_split(a, o, d, r0.w, r1.w);
        ts = s.t1;
        te = s.t2;
    }
    uint32_t flags = 0;
    Counts cnt = {0, 0, 0, 0};
    March m = sdf_march<false, L>(a, o, d, ts, te, flags, cnt);
    if (!m.hit || isnan(m.t_prev)) return;  // a hit at the first sample has no bracket
    const float t = refine<L>(a, o, d, m.t_prev, m.t);
    const float px = __fmaf_rn(t, d.x, o.x), py = __fmaf_rn(t, d.y, o.y), pz = __fmaf_rn(t, d.z, o.z);
    Cell c = locate(a, px, py, pz);
    const int64_t base = grid_base(a, c);
    const int64_t sy = a.gn[0], sz = (int64_t)a.gn[0] * a.gn[1];
    const int64_t off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = grid_at<GL_PLAIN_F32>(a, base + off[k]);
    const float fx = c.f[0], fy = c.f[1], fz = c.f[2];
    const float gx = c.clamped[0] ? 0.f
        : ((v[1] - v[0]) * (1 - fy) * (1 - fz) + (v[3] - v[2]) * fy * (1 - fz) + (v[5] - v[4]) * (1 - fy) * fz +
           (v[7] - v[6]) * fy * fz) * a.gih[0];
    const float gy = c.clamped[1] ? 0.f
        : ((v[2] - v[0]) * (1 - fx) * (1 - fz) + (v[3] - v[1]) * fx * (1 - fz) + (v[6] - v[4]) * (1 - fx) * fz +
           (v[7] - v[5]) * fx * fz) * a.gih[1];
    const float gz = c.clamped[2] ? 0.f
        : ((v[4] - v[0]) * (1 - fx) * (1 - fy) + (v[5] - v[1]) * fx * (1 - fy) + (v[6] - v[2]) * (1 - fx) * fy +
           (v[7] - v[3]) * fx * fy) * a.gih[2];
    const float gd = gx * d.x + gy * d.y + gz * d.z;
    if (gd > -1e-6f) return;  // tangent: the root does not move smoothly
    const float s = -g / gd;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float w = ((k & 1) ? fx : 1 - fx) * ((k & 2) ? fy : 1 - fy) * ((k & 4) ? fz : 1 - fz);
        atomicAdd(grad_grid + base + off[k], s * w);
    }
}

}  // namespace

rt_status rt_launch_backward(const TraceArgs& a, const float* grad_t, float* grad_grid, cudaStream_t s)
{
    const int64_t blocks = (a.n + kBwdBlock - 1) / kBwdBlock;
    if (blocks > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "too many rays");
    // float32 grids only (checked by the caller); the march reads the cell copy when present
    TraceArgs b = a;
    b.pairs = nullptr;
    if (b.cells) k_backward<GL_CELLS_F32><<<(unsigned)blocks, kBwdBlock, 0, s>>>(b, grad_t, grad_grid);
    else k_backward<GL_PLAIN_F32><<<(unsigned)blocks, kBwdBlock, 0, s>>>(b, grad_t, grad_grid);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}
