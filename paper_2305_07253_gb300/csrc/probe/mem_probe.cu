// Memory-system probes for the roofline of the query kernels (mem_probe.h).
//
// - Random gather: a march step of the field stage (Section 3, sphere tracing
//   on the trilinear interpolant) reads one 32-byte cell whose address is
//   known only once the previous step's value is -- a chain of dependent
//   32-byte gathers.  This kernel makes the same chains with addresses drawn
//   uniformly over a buffer larger than the L2, so that no locality helps: its
//   rate is the device's practical ceiling for that access.
// - L2 and L1 reads: coalesced 16-byte loads over a buffer that fits in L2
//   (ld.global.cg) or per-block windows that fit in L1 (ld.global.ca), read
//   over and over: the ceilings of the triangle stages, whose node and
//   triangle reads are mostly served from L1 and L2.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "mem_probe.h"

namespace {

thread_local char g_err[256] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_check(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(2, "%s: %s", what, cudaGetErrorString(e));
    return 0;
}

// the 32-bit finaliser of MurmurHash3 (Appleby, public domain)
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void __launch_bounds__(128) k_gather_probe(const float* __restrict__ cells, uint32_t mask, int32_t steps,
                                                      float* __restrict__ out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t idx = fmix32(tid + 1u) & mask;
    float acc = 0.f;
    for (int32_t s = 0; s < steps; ++s) {
        float v[8];
        asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                     : "l"(cells + 8ull * idx));
        acc += v[0] + v[7];
        idx = fmix32(idx ^ __float_as_uint(v[3]) ^ (uint32_t)s) & mask;
    }
    out[tid] = acc;
}

constexpr int kReadBlock = 256;

__device__ __forceinline__ float4 ld_cg(const float4* p)
{
    float4 v;
    asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ float4 ld_ca(const float4* p)
{
    float4 v;
    asm volatile("ld.global.ca.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

__global__ void __launch_bounds__(kReadBlock) k_l2_read(const float4* __restrict__ buf, int64_t n16, int32_t reps,
                                                       float* __restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * kReadBlock + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * kReadBlock;
    float acc = 0.f;
    for (int32_t r = 0; r < reps; ++r) {
        // four independent loads in flight per thread
        int64_t i = t;
        for (; i + 3 * T < n16; i += 4 * T) {
            const float4 a = ld_cg(buf + i), b = ld_cg(buf + i + T), c = ld_cg(buf + i + 2 * T),
                         d = ld_cg(buf + i + 3 * T);
            acc += (a.x + b.x) + (c.x + d.x);
        }
        for (; i < n16; i += T) acc += ld_cg(buf + i).x;
    }
    out[t] = acc;
}

__global__ void __launch_bounds__(kReadBlock) k_l1_read(const float4* __restrict__ buf, int32_t window16, int32_t reps,
                                                       float* __restrict__ out)
{
    const float4* w = buf + (int64_t)blockIdx.x * window16;
    float acc = 0.f;
    for (int32_t r = 0; r < reps; ++r) {
        int32_t i = threadIdx.x;
        for (; i + 3 * kReadBlock < window16; i += 4 * kReadBlock) {
            const float4 a = ld_ca(w + i), b = ld_ca(w + i + kReadBlock), c = ld_ca(w + i + 2 * kReadBlock),
                         d = ld_ca(w + i + 3 * kReadBlock);
            acc += (a.x + b.x) + (c.x + d.x);
        }
        for (; i < window16; i += kReadBlock) acc += ld_ca(w + i).x;
    }
    out[(int64_t)blockIdx.x * kReadBlock + threadIdx.x] = acc;
}

}  // namespace

extern "C" int mp_random_gather(const void* d_cells, int64_t n_cells, int32_t steps, int32_t blocks, float* d_out,
                                void* stream)
{
    if (!d_cells || !d_out) return fail(1, "null buffer");
    if (((uintptr_t)d_cells & 31u) != 0) return fail(1, "cell buffer not 32-byte aligned");
    if (((uintptr_t)d_out & 3u) != 0) return fail(1, "output not 4-byte aligned");
    if (n_cells < 1 || n_cells > (int64_t(1) << 31) || (n_cells & (n_cells - 1)) != 0)
        return fail(1, "n_cells must be a power of two in [1, 2^31] (got %lld)", (long long)n_cells);
    if (steps < 1) return fail(1, "steps must be >= 1");
    if (blocks < 1 || blocks > (1 << 20)) return fail(1, "blocks must be in [1, 2^20]");
    k_gather_probe<<<blocks, 128, 0, (cudaStream_t)stream>>>(static_cast<const float*>(d_cells),
                                                              (uint32_t)(n_cells - 1), steps, d_out);
    return cuda_check("k_gather_probe");
}

extern "C" int mp_l2_read(const void* d_buf, int64_t n_bytes, int32_t reps, int32_t blocks, float* d_out,
                          void* stream)
{
    if (!d_buf || !d_out) return fail(1, "null buffer");
    if (((uintptr_t)d_buf & 15u) != 0) return fail(1, "buffer not 16-byte aligned");
    if (((uintptr_t)d_out & 3u) != 0) return fail(1, "output not 4-byte aligned");
    if (n_bytes < 16 || n_bytes > (int64_t(1) << 40) || (n_bytes & 15) != 0)
        return fail(1, "n_bytes must be a multiple of 16 in [16, 2^40] (got %lld)", (long long)n_bytes);
    if (reps < 1) return fail(1, "reps must be >= 1");
    if (blocks < 1 || blocks > (1 << 20)) return fail(1, "blocks must be in [1, 2^20]");
    k_l2_read<<<blocks, kReadBlock, 0, (cudaStream_t)stream>>>(static_cast<const float4*>(d_buf), n_bytes / 16, reps,
                                                                d_out);
    return cuda_check("k_l2_read");
}

extern "C" int mp_l1_read(const void* d_buf, int32_t window, int32_t reps, int32_t blocks, float* d_out, void* stream)
{
    if (!d_buf || !d_out) return fail(1, "null buffer");
    if (((uintptr_t)d_buf & 15u) != 0) return fail(1, "buffer not 16-byte aligned");
    if (((uintptr_t)d_out & 3u) != 0) return fail(1, "output not 4-byte aligned");
    if (window < 4096 || window > 131072 || (window & 4095) != 0)
        return fail(1, "window must be a multiple of 4096 in [4096, 131072] (got %d)", window);
    if (reps < 1) return fail(1, "reps must be >= 1");
    if (blocks < 1 || blocks > (1 << 20)) return fail(1, "blocks must be in [1, 2^20]");
    k_l1_read<<<blocks, kReadBlock, 0, (cudaStream_t)stream>>>(static_cast<const float4*>(d_buf), window / 16, reps,
                                                                d_out);
    return cuda_check("k_l1_read");
}

extern "C" const char* mp_last_error(void) { return g_err; }
