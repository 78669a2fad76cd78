// Memory-system probe for the roofline of the field stage.  A march step
// (Section 3, sphere tracing on the trilinear interpolant) reads one 32-byte
// cell whose address is known only once the previous step's value is: a chain
// of dependent 32-byte gathers.  This kernel makes the same chains with
// addresses drawn uniformly over a buffer larger than the L2, so that no
// locality helps: its rate is the device's practical ceiling for that access,
// reported beside the copy bandwidth.
#include "rt_internal.cuh"

namespace {

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

}  // namespace

extern "C" rt_status rt_gather_probe(const void* d_cells, int64_t n_cells, int32_t steps, int32_t blocks,
                                     float* d_out, void* stream)
{
    if (!d_cells || !d_out) return rt_fail(RT_ERR_INVALID_ARG, "null buffer");
    if (((uintptr_t)d_cells & 31u) != 0) return rt_fail(RT_ERR_INVALID_ARG, "cell buffer not 32-byte aligned");
    if (((uintptr_t)d_out & 3u) != 0) return rt_fail(RT_ERR_INVALID_ARG, "output not 4-byte aligned");
    if (n_cells < 1 || n_cells > (int64_t(1) << 31) || (n_cells & (n_cells - 1)) != 0)
        return rt_fail(RT_ERR_INVALID_ARG, "n_cells must be a power of two in [1, 2^31] (got %lld)", (long long)n_cells);
    if (steps < 1) return rt_fail(RT_ERR_INVALID_ARG, "steps must be >= 1");
    if (blocks < 1 || blocks > (1 << 20)) return rt_fail(RT_ERR_INVALID_ARG, "blocks must be in [1, 2^20]");
    k_gather_probe<<<blocks, 128, 0, (cudaStream_t)stream>>>(static_cast<const float*>(d_cells),
                                                              (uint32_t)(n_cells - 1), steps, d_out);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}
