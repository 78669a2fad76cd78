// Distance-field bake: at every grid sample, the distance to the nearest
// triangle with the sign of the angle-weighted pseudonormal of the nearest
// feature (Baerentzen & Aanaes, IEEE TVCG 2005).  Positive on the side the
// triangle normals face.  The closest point on a triangle is found from the
// Voronoi regions of the triangle (Ericson, Real-Time Collision Detection,
// 5.1.5).  The paper builds its field by rasterised voxelisation, jump
// flooding and fast sweeping (Section 3, "Distance Field Generation"); this is
// the exact definition that those steps approximate.
//
// Two kernels with the same result: brute force (every triangle, staged through
// shared memory in tiles) and a BVH-pruned nearest query.
#include <math.h>
#include <string.h>

#include "rt_bake_dev.cuh"
#include "rt_trace_dev.cuh"

namespace {

using namespace rtbake;

constexpr int kBakeBlock = 128;
constexpr int kTile = 128;

struct BakeArgs {
    const BNode* nodes;
    const float4* tris;
    const float4* pn;
    int64_t n_tris;
    void* grid;
    int32_t f16;
    float lo[3], h[3];
    int32_t n[3];
    int64_t count;
    // cascade level: samples at (ilo + i) * h[0], one rounding per coordinate,
    // so a sample's position depends only on its absolute lattice index
    int32_t lattice;
    int32_t ilo[3];
    // rolling update: when set, sample i takes the value of sample i + shift of
    // `keep` (the level before the move) wherever that lies inside the level
    const void* keep;
    int32_t shift[3];
    // Sub-lattice pass: when sub > 0 the threads enumerate only the samples
    // whose indices are multiples of `sub` (a first pass that seeds the bounds).
    int32_t sub;
    // Bound source: a lattice of samples whose exact values are already known.
    // A sample at absolute lattice index a (a = ilo + i on a cascade level,
    // a = i otherwise) takes the source sample j = clamp(round(a / bratio) -
    // bilo, 0, bjmax), stored at element j * bstride of bsrc (per axis), and
    // searches only within |phi(source)| + |p - source|, since the distance
    // function is 1-Lipschitz.  The nearest triangle found is the same as
    // without the bound.  bsrc null: no bound.
    const void* bsrc;
    int32_t bratio, bstride;
    int32_t bilo[3], bjmax[3];
    int32_t bself;  // 1: the source is this grid's own sub-lattice: relative indices
                    // (a = i), and its samples are skipped (baked by the first pass)
};

__device__ __forceinline__ float3 sample_pos(const BakeArgs& b, int64_t i)
{
    int64_t ix = i % b.n[0], iy = (i / b.n[0]) % b.n[1], iz = i / ((int64_t)b.n[0] * b.n[1]);
    if (b.lattice)
        return make_float3(__fmul_rn((float)(b.ilo[0] + ix), b.h[0]), __fmul_rn((float)(b.ilo[1] + iy), b.h[0]),
                           __fmul_rn((float)(b.ilo[2] + iz), b.h[0]));
    return make_float3(fmaf((float)ix, b.h[0], b.lo[0]), fmaf((float)iy, b.h[1], b.lo[1]),
                       fmaf((float)iz, b.h[2], b.lo[2]));
}

// rolling update: copy the kept value of sample i; false when i must be baked
__device__ __forceinline__ bool take_kept(const BakeArgs& b, int64_t i)
{
    if (!b.keep) return false;
    const int64_t nx = b.n[0], ny = b.n[1];
    const int64_t ix = i % nx + b.shift[0], iy = (i / nx) % ny + b.shift[1], iz = i / (nx * ny) + b.shift[2];
    if (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= b.n[2]) return false;
    const int64_t src = ix + nx * (iy + ny * iz);
    if (b.f16) reinterpret_cast<__half*>(b.grid)[i] = reinterpret_cast<const __half*>(b.keep)[src];
    else reinterpret_cast<float*>(b.grid)[i] = reinterpret_cast<const float*>(b.keep)[src];
    return true;
}

__device__ __forceinline__ void store(const BakeArgs& b, int64_t i, float v)
{
    if (b.f16) reinterpret_cast<__half*>(b.grid)[i] = __float2half_rn(v);
    else reinterpret_cast<float*>(b.grid)[i] = v;
}

__global__ void __launch_bounds__(kBakeBlock) k_bake_brute(const BakeArgs b)
{
    __shared__ float4 tile[3 * kTile];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < b.count && !take_kept(b, i);  // every thread stays for the barriers
    const float3 p = sample_pos(b, live ? i : 0);
    Nearest nb = {__int_as_float(0x7f800000), -1, 0x7fffffff};
    for (int64_t t0 = 0; t0 < b.n_tris; t0 += kTile) {
        const int m = (int)min((int64_t)kTile, b.n_tris - t0);
        __syncthreads();
        for (int j = threadIdx.x; j < 3 * m; j += blockDim.x) tile[j] = __ldg(b.tris + 3 * t0 + j);
        __syncthreads();
        if (live) {
            for (int j = 0; j < m; ++j) {
                float3 q;
                closest_point(p, xyz(tile[3 * j]), xyz(tile[3 * j + 1]), xyz(tile[3 * j + 2]), q);
                float3 pq = sub(p, q);
                float d2 = dot(pq, pq);
                int32_t prim = __float_as_int(tile[3 * j].w);
                if (d2 < nb.d2 || (d2 == nb.d2 && prim < nb.prim)) {
                    nb.d2 = d2;
                    nb.k = (int32_t)(t0 + j);
                    nb.prim = prim;
                }
            }
        }
    }
    if (live) store(b, i, signed_distance(p, nb, b.tris, b.pn));
}

__device__ __forceinline__ float box_d2(float lx, float hx, float ly, float hy, float lz, float hz, float3 p)
{
    float dx = fmaxf(fmaxf(lx - p.x, p.x - hx), 0.f);
    float dy = fmaxf(fmaxf(ly - p.y, p.y - hy), 0.f);
    float dz = fmaxf(fmaxf(lz - p.z, p.z - hz), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ float load_value(const void* g, int32_t f16, int64_t i)
{
    return f16 ? __half2float(reinterpret_cast<const __half*>(g)[i]) : reinterpret_cast<const float*>(g)[i];
}

__device__ __forceinline__ int64_t floordiv(int64_t x, int64_t y)  // y > 0
{
    return x >= 0 ? x / y : -((-x + y - 1) / y);
}

// upper bound on the distance at sample (ix, iy, iz) from the bound source
__device__ __forceinline__ float distance_bound(const BakeArgs& b, int64_t ix, int64_t iy, int64_t iz)
{
    if (!b.bsrc) return __int_as_float(0x7f800000);
    const int64_t ii[3] = {ix, iy, iz};
    int64_t el = 0, stride = 1;
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t abs_i = (b.lattice && !b.bself ? b.ilo[a] : 0) + ii[a];
        int64_t j = floordiv(2 * abs_i + b.bratio, 2 * (int64_t)b.bratio) - b.bilo[a];  // round(abs_i / bratio)
        j = j < 0 ? 0 : (j > b.bjmax[a] ? b.bjmax[a] : j);
        const float gap = (float)(abs_i - (j + b.bilo[a]) * b.bratio) * b.h[a];
        d2 += gap * gap;
        el += j * b.bstride * stride;
        stride *= b.n[a];
    }
    const float phi = fabsf(load_value(b.bsrc, b.f16, el));
    // generous margin for the rounding of the stored value (float16 included)
    return (phi + sqrtf(d2)) * 1.002f + 1e-6f;
}

__device__ __forceinline__ bool on_sublattice(const BakeArgs& b, int64_t ix, int64_t iy, int64_t iz)
{
    return ix % b.bstride == 0 && iy % b.bstride == 0 && iz % b.bstride == 0 && ix / b.bstride <= b.bjmax[0] &&
           iy / b.bstride <= b.bjmax[1] && iz / b.bstride <= b.bjmax[2];
}

// nearest triangle to p among those closer than sqrt(d2_start) (BVH-pruned);
// k = -1 when there is none
__device__ __forceinline__ Nearest nearest_bvh(const BakeArgs& b, float3 p, float d2_start)
{
    Nearest nb = {d2_start, -1, 0x7fffffff};
    int stack[RT_STACK_DEPTH];
    float sd[RT_STACK_DEPTH];
    int sp = 0;
    int node = b.n_tris > 1 ? 0 : ~0;
    for (uint32_t guard = 0; guard <= (1u << 26); ++guard) {
        if (node >= 0) {
            const float4* np = reinterpret_cast<const float4*>(b.nodes + node);
            float4 na = __ldg(np), nbx = __ldg(np + 1), nc = __ldg(np + 2);
            int4 nd = __ldg(reinterpret_cast<const int4*>(np + 3));
            float d0 = box_d2(na.x, na.y, na.z, na.w, nc.x, nc.y, p);
            float d1 = box_d2(nbx.x, nbx.y, nbx.z, nbx.w, nc.z, nc.w, p);
            bool v0 = d0 <= nb.d2, v1 = d1 <= nb.d2;
            if (v0 && v1) {
                int nearc = nd.x, farc = nd.y;
                float fd = d1;
                if (d1 < d0) { nearc = nd.y; farc = nd.x; fd = d0; }
                if (sp < RT_STACK_DEPTH) { stack[sp] = farc; sd[sp] = fd; ++sp; }
                node = nearc;
                continue;
            }
            if (v0) { node = nd.x; continue; }
            if (v1) { node = nd.y; continue; }
        } else {
            consider(nb, p, b.tris, ~node);
        }
        bool more = false;
        while (sp > 0) {
            --sp;
            if (sd[sp] <= nb.d2) { node = stack[sp]; more = true; break; }
        }
        if (!more) break;
    }
    return nb;
}

__global__ void __launch_bounds__(kBakeBlock) k_bake_bvh(const BakeArgs b)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = t;
    if (b.sub > 0) {  // enumerate the sub-lattice only
        const int64_t mx = (b.n[0] - 1) / b.sub + 1, my = (b.n[1] - 1) / b.sub + 1, mz = (b.n[2] - 1) / b.sub + 1;
        if (t >= mx * my * mz) return;
        const int64_t jx = t % mx, jy = (t / mx) % my, jz = t / (mx * my);
        i = jx * b.sub + (int64_t)b.n[0] * (jy * b.sub + (int64_t)b.n[1] * (jz * b.sub));
    }
    if (i >= b.count || take_kept(b, i)) return;
    const int64_t ix = i % b.n[0], iy = (i / b.n[0]) % b.n[1], iz = i / ((int64_t)b.n[0] * b.n[1]);
    if (b.bself && on_sublattice(b, ix, iy, iz)) return;
    const float3 p = sample_pos(b, i);
    const float bound = distance_bound(b, ix, iy, iz);
    Nearest nb = nearest_bvh(b, p, bound * bound);
    if (nb.k < 0 && bound < __int_as_float(0x7f800000)) nb = nearest_bvh(b, p, __int_as_float(0x7f800000));
    store(b, i, signed_distance(p, nb, b.tris, b.pn));
}

// cell-corner copy: the 8 corners of cell (i,j,k) stored together, order
// v000 v100 v010 v110 v001 v101 v011 v111 (x fastest), cells x fastest
__global__ void k_cells(const void* grid, int32_t f16, int32_t nx, int32_t ny, int32_t nz, void* cells_out)
{
    const int64_t cx = nx - 1, cy = ny - 1;
    const int64_t count = cx * cy * (int64_t)(nz - 1);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t i = t % cx, j = (t / cx) % cy, k = t / (cx * cy);
    const int64_t c = rtdev::cell_slot((int)i, (int)j, (int)k, nx, ny);
    const int64_t b = i + (int64_t)nx * (j + (int64_t)ny * k);
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t idx[8] = {b, b + 1, b + sy, b + sy + 1, b + sz, b + sz + 1, b + sz + sy, b + sz + sy + 1};
    if (f16) {
        const __half* g = reinterpret_cast<const __half*>(grid);
        __half2 h[4];
        for (int q = 0; q < 4; ++q) h[q] = __halves2half2(g[idx[2 * q]], g[idx[2 * q + 1]]);
        reinterpret_cast<uint4*>(cells_out)[c] = *reinterpret_cast<const uint4*>(h);
    } else {
        const float* g = reinterpret_cast<const float*>(grid);
        float4* out = reinterpret_cast<float4*>(cells_out) + 2 * c;
        out[0] = make_float4(g[idx[0]], g[idx[1]], g[idx[2]], g[idx[3]]);
        out[1] = make_float4(g[idx[4]], g[idx[5]], g[idx[6]], g[idx[7]]);
    }
}

// x-pair copy: entry (i,j,k) = (g[i,j,k], g[i+1,j,k]), i < nx-1, x fastest
__global__ void k_pairs(const void* grid, int32_t f16, int32_t nx, int32_t ny, int32_t nz, void* pairs)
{
    const int64_t px = nx - 1;
    const int64_t count = px * ny * (int64_t)nz;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    const int64_t i = c % px, jk = c / px;
    const int64_t b = i + (int64_t)nx * jk;
    if (f16) {
        const __half* g = reinterpret_cast<const __half*>(grid);
        reinterpret_cast<__half2*>(pairs)[c] = __halves2half2(g[b], g[b + 1]);
    } else {
        const float* g = reinterpret_cast<const float*>(grid);
        reinterpret_cast<float2*>(pairs)[c] = make_float2(g[b], g[b + 1]);
    }
}

}  // namespace

rt_status rt_launch_cascade_cells(const rt_sdf* sdf, int k, cudaStream_t s)
{
    const int64_t n = sdf->n[0];
    const int64_t count = (n - 1) * (n - 1) * (n - 1);
    const int64_t esz = sdf->dtype == RT_GRID_F16 ? 2 : 4;
    const void* grid = static_cast<const char*>(sdf->grid) + k * n * n * n * esz;
    void* cells = static_cast<char*>(sdf->cells) + k * rtdev::cell_count((int)n, (int)n, (int)n) * 8 * esz;
    const int64_t blocks = (count + 255) / 256;
    k_cells<<<(unsigned)blocks, 256, 0, s>>>(grid, sdf->dtype == RT_GRID_F16, (int32_t)n, (int32_t)n, (int32_t)n,
                                             cells);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

rt_status rt_launch_prepare(rt_sdf* sdf, cudaStream_t s)
{
    if (sdf->levels > 0) {
        const int64_t n = sdf->n[0];
        const int64_t bytes =
            sdf->levels * rtdev::cell_count((int)n, (int)n, (int)n) * (sdf->dtype == RT_GRID_F16 ? 16 : 32);
        if (!sdf->cells || sdf->cells_bytes != bytes) {
            if (sdf->cells) cudaFree(sdf->cells);
            sdf->cells = nullptr;
            sdf->cells_bytes = 0;
            RT_CUDA_TRY(cudaMalloc(&sdf->cells, (size_t)bytes));
            sdf->cells_bytes = bytes;
        }
        for (int k = 0; k < sdf->levels; ++k) {
            rt_status st = rt_launch_cascade_cells(sdf, k, s);
            if (st != RT_OK) return st;
        }
        return RT_OK;
    }
    {
        const int64_t pc = (int64_t)(sdf->n[0] - 1) * sdf->n[1] * sdf->n[2];
        const int64_t pb = pc * (sdf->dtype == RT_GRID_F16 ? 4 : 8);
        if (!sdf->pairs || sdf->pairs_bytes != pb) {
            if (sdf->pairs) cudaFree(sdf->pairs);
            sdf->pairs = nullptr;
            sdf->pairs_bytes = 0;
            RT_CUDA_TRY(cudaMalloc(&sdf->pairs, (size_t)pb));
            sdf->pairs_bytes = pb;
        }
        const int64_t blocks = (pc + 255) / 256;
        if (blocks > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "grid too large");
        k_pairs<<<(unsigned)blocks, 256, 0, s>>>(sdf->grid, sdf->dtype == RT_GRID_F16, sdf->n[0], sdf->n[1],
                                                 sdf->n[2], sdf->pairs);
        RT_CUDA_TRY(cudaGetLastError());
    }
    const int64_t count = (int64_t)(sdf->n[0] - 1) * (sdf->n[1] - 1) * (sdf->n[2] - 1);
    const int64_t bytes = rtdev::cell_count(sdf->n[0], sdf->n[1], sdf->n[2]) * (sdf->dtype == RT_GRID_F16 ? 16 : 32);
    if (!sdf->cells || sdf->cells_bytes != bytes) {
        if (sdf->cells) cudaFree(sdf->cells);
        sdf->cells = nullptr;
        sdf->cells_bytes = 0;
        RT_CUDA_TRY(cudaMalloc(&sdf->cells, (size_t)bytes));
        sdf->cells_bytes = bytes;
    }
    const int64_t blocks = (count + 255) / 256;
    if (blocks > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "grid too large");
    k_cells<<<(unsigned)blocks, 256, 0, s>>>(sdf->grid, sdf->dtype == RT_GRID_F16, sdf->n[0], sdf->n[1], sdf->n[2],
                                             sdf->cells);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

constexpr int kSubStride = 4;  // first-pass sub-lattice of a bounded bake

static rt_status launch_one(const BakeArgs& b, int32_t method, cudaStream_t s)
{
    int64_t threads = b.count;
    if (b.sub > 0)
        threads = (int64_t)((b.n[0] - 1) / b.sub + 1) * ((b.n[1] - 1) / b.sub + 1) * ((b.n[2] - 1) / b.sub + 1);
    const int64_t blocks = (threads + kBakeBlock - 1) / kBakeBlock;
    if (blocks > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "grid too large for one launch");
    if (method == RT_BAKE_BRUTE) k_bake_brute<<<(unsigned)blocks, kBakeBlock, 0, s>>>(b);
    else k_bake_bvh<<<(unsigned)blocks, kBakeBlock, 0, s>>>(b);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// BVH bake in two passes over the same grid: the stride-4 sub-lattice first,
// then every other sample bounded by its nearest sub-lattice sample
static rt_status launch_two_pass(BakeArgs b, cudaStream_t s)
{
    b.sub = kSubStride;
    b.bsrc = nullptr;
    rt_status st = launch_one(b, RT_BAKE_BVH, s);
    if (st != RT_OK) return st;
    b.sub = 0;
    b.bsrc = b.grid;
    b.bratio = b.bstride = kSubStride;
    for (int a = 0; a < 3; ++a) {
        b.bilo[a] = 0;
        b.bjmax[a] = (b.n[a] - 1) / kSubStride;
    }
    b.bself = 1;
    return launch_one(b, RT_BAKE_BVH, s);
}

static int32_t pick_method(const BakeArgs& b, int32_t method)
{
    if (method == RT_BAKE_AUTO) method = (double)b.count * (double)b.n_tris <= 17179869184.0 ? RT_BAKE_BRUTE : RT_BAKE_BVH;
    return method;
}

rt_status rt_launch_cascade_bake(const rt_scene* sc, const rt_sdf* sdf, int k, int32_t method, const void* keep,
                                 const int32_t shift[3], cudaStream_t s)
{
    BakeArgs b;
    memset(&b, 0, sizeof(b));
    b.nodes = sc->nodes;
    b.tris = sc->tris;
    b.pn = sc->pn;
    b.n_tris = sc->n_tris;
    const int64_t n = sdf->n[0];
    const int64_t esz = sdf->dtype == RT_GRID_F16 ? 2 : 4;
    b.grid = static_cast<char*>(const_cast<void*>(sdf->grid)) + k * n * n * n * esz;
    b.f16 = sdf->dtype == RT_GRID_F16;
    b.count = n * n * n;
    b.lattice = 1;
    b.h[0] = b.h[1] = b.h[2] = ldexpf(sdf->h0, k);
    for (int a = 0; a < 3; ++a) {
        b.n[a] = (int32_t)n;
        b.ilo[a] = sdf->ilo[k][a];
        b.shift[a] = shift ? shift[a] : 0;
    }
    b.keep = keep;
    method = pick_method(b, method);
    if (method == RT_BAKE_BRUTE) return launch_one(b, method, s);
    b.bratio = 1;
    b.bstride = 1;
    for (int a = 0; a < 3; ++a) b.bjmax[a] = (int32_t)n - 1;
    if (keep) {
        // rolling update: new samples are bounded by the nearest kept sample
        b.bsrc = keep;
        for (int a = 0; a < 3; ++a) b.bilo[a] = sdf->ilo[k][a] - b.shift[a];
        return launch_one(b, method, s);
    }
    if (k + 1 < sdf->levels) {
        // bounded by the next coarser level (baked or moved before this one)
        b.bsrc = static_cast<const char*>(sdf->grid) + (k + 1) * n * n * n * esz;
        b.bratio = 2;
        for (int a = 0; a < 3; ++a) b.bilo[a] = sdf->ilo[k + 1][a];
        return launch_one(b, method, s);
    }
    return launch_two_pass(b, s);
}

rt_status rt_launch_bake(const rt_scene* sc, const rt_sdf* sdf, int32_t method, cudaStream_t s)
{
    if (sdf->levels > 0) {
        for (int k = sdf->levels - 1; k >= 0; --k) {  // coarsest first: each level bounds the next finer one
            rt_status st = rt_launch_cascade_bake(sc, sdf, k, method, nullptr, nullptr, s);
            if (st != RT_OK) return st;
        }
        return RT_OK;
    }
    BakeArgs b;
    memset(&b, 0, sizeof(b));
    b.nodes = sc->nodes;
    b.tris = sc->tris;
    b.pn = sc->pn;
    b.n_tris = sc->n_tris;
    b.grid = const_cast<void*>(sdf->grid);
    b.f16 = sdf->dtype == RT_GRID_F16;
    b.count = 1;
    for (int k = 0; k < 3; ++k) {
        b.lo[k] = sdf->lo[k];
        b.h[k] = sdf->h[k];
        b.n[k] = sdf->n[k];
        b.count *= sdf->n[k];
    }
    method = pick_method(b, method);
    if (method == RT_BAKE_BRUTE) return launch_one(b, method, s);
    return launch_two_pass(b, s);
}
