// Triangle acceleration structure: a linear BVH (LBVH).
//
//   1. per-triangle bounds and centroids, scene bounds by atomic min/max
//   2. 63-bit Morton code of each centroid (21 bits per axis); bit 63 marks a
//      large triangle (box wider than a quarter of the scene), so that the
//      root splits the large triangles (room walls, floors) from the rest and
//      their wide boxes do not enlarge the nodes of the compact geometry
//   3. sort (code, triangle) pairs (CUB radix sort, a library sort primitive)
//   4. internal nodes by the split search of Karras, "Maximizing Parallelism
//      in the Construction of BVHs, Octrees, and k-d Trees" (HPG 2012):
//      node i covers a range of sorted keys found from the longest common
//      prefix; duplicate codes are ordered by their position
//   5. bottom-up bounds: every leaf walks to the root, the second thread to
//      reach a node (atomic counter) merges its two children
//   5b. treelet restructuring for surface-area cost (rt_treelet.cu), leaves
//      renumbered depth-first
//   6. pack 64-byte nodes (child boxes inline), 48-byte triangles in leaf
//      order, and per-triangle pseudonormals for the distance bake
//      (Baerentzen & Aanaes, "Signed distance computation using the angle
//      weighted pseudonormal", IEEE TVCG 2005)
//
// The paper traces this part of each ray with hardware ray tracing on a
// driver-built structure (Section 3); here it is an explicit CUDA structure.
#include <math.h>
#include <stdio.h>

#include <cub/device/device_radix_sort.cuh>

#include "rt_internal.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxWalk = 256;  // bound on any leaf-to-root walk (the stack holds 64)
constexpr float kLargeFrac = 0.25f;  // a triangle wider than this share of the scene is "large"
#ifndef RT_TREELET_PASSES
#define RT_TREELET_PASSES 3
#endif
constexpr int kTreeletPasses = RT_TREELET_PASSES;  // treelet restructuring passes over the Morton hierarchy

__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ __forceinline__ float ord2f(int i)
{
    int b = i >= 0 ? i : i ^ 0x7FFFFFFF;
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

__device__ __forceinline__ float3 load_vert(const float* V, int32_t i)
{
    return make_float3(V[3 * (int64_t)i], V[3 * (int64_t)i + 1], V[3 * (int64_t)i + 2]);
}

// smallest and largest vertex index used by the triangles
__global__ void k_index_range(const int32_t* F, int64_t m, int* range)
{
    int lo = INT32_MAX, hi = INT32_MIN;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        lo = min(lo, F[k]);
        hi = max(hi, F[k]);
    }
    atomicMin(&range[0], lo);
    atomicMax(&range[1], hi);
}

// bounds[0..2] scene lo, [3..5] scene hi, [6..8] centroid lo, [9..11] centroid hi (ordered ints)
__global__ void k_tri_bounds(const float* V, const int32_t* F, int64_t nt, float4* cen, int* bounds)
{
    __shared__ int s[12];
    if (threadIdx.x < 12) s[threadIdx.x] = (threadIdx.x % 6) < 3 ? INT32_MAX : INT32_MIN;
    __syncthreads();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) {
        float3 a = load_vert(V, F[3 * t]), b = load_vert(V, F[3 * t + 1]), c = load_vert(V, F[3 * t + 2]);
        float lo[3] = {fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z)};
        float hi[3] = {fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z)};
        float cc[3] = {0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2])};
        const float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
        cen[t] = make_float4(cc[0], cc[1], cc[2], ext);
        for (int k = 0; k < 3; ++k) {
            atomicMin(&s[k], f2ord(lo[k]));
            atomicMax(&s[3 + k], f2ord(hi[k]));
            atomicMin(&s[6 + k], f2ord(cc[k]));
            atomicMax(&s[9 + k], f2ord(cc[k]));
        }
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        if ((threadIdx.x % 6) < 3) atomicMin(&bounds[threadIdx.x], s[threadIdx.x]);
        else atomicMax(&bounds[threadIdx.x], s[threadIdx.x]);
    }
}

__device__ __forceinline__ uint64_t spread21(uint64_t x)
{
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float4* cen, int64_t nt, const int* bounds, uint64_t* keys, int32_t* vals)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float4 c = cen[t];
    float cc[3] = {c.x, c.y, c.z};
    uint64_t q[3];
    for (int k = 0; k < 3; ++k) {
        float lo = ord2f(bounds[6 + k]), hi = ord2f(bounds[9 + k]);
        float ext = hi - lo;
        float u = ext > 0.f ? (cc[k] - lo) / ext : 0.5f;
        u = fminf(fmaxf(u, 0.f), 1.f);
        q[k] = (uint64_t)fminf(u * 2097152.0f, 2097151.0f);
    }
    float scene_ext = 0.f;
    for (int k = 0; k < 3; ++k) scene_ext = fmaxf(scene_ext, ord2f(bounds[3 + k]) - ord2f(bounds[k]));
    const uint64_t large = c.w > kLargeFrac * scene_ext ? (1ull << 63) : 0ull;
    keys[t] = large | (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    vals[t] = (int32_t)t;
}

// longest common prefix of sorted keys i and j; equal keys compare positions
__device__ __forceinline__ int delta(const uint64_t* keys, int64_t n, int64_t i, int64_t j)
{
    if (j < 0 || j >= n) return -1;
    uint64_t a = keys[i], b = keys[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

// children: >= 0 internal node, < 0 leaf ~k (sorted position k)
__global__ void k_hierarchy(const uint64_t* keys, int64_t n, int2* child, int2* range, int32_t* parent_int,
                            int32_t* parent_leaf)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int64_t lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int64_t s = 0;
    int64_t t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int left = (lo == gamma) ? ~(int)gamma : (int)gamma;
    int right = (hi == gamma + 1) ? ~(int)(gamma + 1) : (int)(gamma + 1);
    child[i] = make_int2(left, right);
    range[i] = make_int2((int)lo, (int)hi);  // sorted triangles lo..hi under node i
    if (left < 0) parent_leaf[~left] = (int32_t)i; else parent_int[left] = (int32_t)i;
    if (right < 0) parent_leaf[~right] = (int32_t)i; else parent_int[right] = (int32_t)i;
    if (i == 0) parent_int[0] = -1;
}

struct Box {
    float lo[3], hi[3];
};

__device__ __forceinline__ void tri_box(const float* V, const int32_t* F, int32_t t, float4& lo, float4& hi)
{
    float3 a = load_vert(V, F[3 * (int64_t)t]), b = load_vert(V, F[3 * (int64_t)t + 1]),
           c = load_vert(V, F[3 * (int64_t)t + 2]);
    lo = make_float4(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z), 0.f);
    hi = make_float4(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z), 0.f);
}

// leaf boxes (sorted order), then walk up; the second arrival at a node merges
__global__ void k_refit(const float* V, const int32_t* F, const int32_t* order, int64_t n, const int2* child,
                        const int32_t* parent_int, const int32_t* parent_leaf, float4* leaf_lo, float4* leaf_hi,
                        float4* node_lo, float4* node_hi, int* visit)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4 lo, hi;
    tri_box(V, F, order[k], lo, hi);
    leaf_lo[k] = lo;
    leaf_hi[k] = hi;
    __threadfence();
    int32_t node = parent_leaf[k];
    for (int guard = 0; node >= 0 && guard < kMaxWalk; ++guard) {
        if (atomicAdd(&visit[node], 1) == 0) return;  // the sibling subtree is not finished yet
        __threadfence();
        int2 c = child[node];
        float4 l0 = c.x < 0 ? __ldcg(&leaf_lo[~c.x]) : __ldcg(&node_lo[c.x]);
        float4 h0 = c.x < 0 ? __ldcg(&leaf_hi[~c.x]) : __ldcg(&node_hi[c.x]);
        float4 l1 = c.y < 0 ? __ldcg(&leaf_lo[~c.y]) : __ldcg(&node_lo[c.y]);
        float4 h1 = c.y < 0 ? __ldcg(&leaf_hi[~c.y]) : __ldcg(&node_hi[c.y]);
        node_lo[node] = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
        node_hi[node] = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
        __threadfence();
        node = parent_int[node];
    }
}

// depth of each leaf; a walk longer than kMaxWalk (a malformed tree) reports kMaxWalk
__global__ void k_depth(const int32_t* parent_int, const int32_t* parent_leaf, int64_t n, int* max_depth)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int depth = 1;
    for (int32_t node = parent_leaf[k]; node > 0 && depth < kMaxWalk; node = parent_int[node]) ++depth;
    atomicMax(max_depth, depth);
}

__global__ void k_pack_nodes(const int2* child, int64_t n_int, const float4* leaf_lo, const float4* leaf_hi,
                             const float4* node_lo, const float4* node_hi, float pad, BNode* out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int2 c = child[i];
    float4 l0 = c.x < 0 ? leaf_lo[~c.x] : node_lo[c.x], h0 = c.x < 0 ? leaf_hi[~c.x] : node_hi[c.x];
    float4 l1 = c.y < 0 ? leaf_lo[~c.y] : node_lo[c.y], h1 = c.y < 0 ? leaf_hi[~c.y] : node_hi[c.y];
    // widen by a margin well above the float rounding of the slab test so that
    // a triangle lying on a box face is never culled
    BNode b;
    b.a = make_float4(l0.x - pad, h0.x + pad, l0.y - pad, h0.y + pad);
    b.b = make_float4(l1.x - pad, h1.x + pad, l1.y - pad, h1.y + pad);
    b.c = make_float4(l0.z - pad, h0.z + pad, l1.z - pad, h1.z + pad);
    b.d = make_int4(c.x, c.y, 0, 0);
    out[i] = b;
}

__global__ void k_pack_tris(const float* V, const int32_t* F, const int32_t* order, int64_t n, float4* out,
                            int32_t* slot)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int32_t t = order[k];
    slot[t] = (int32_t)k;
    float3 a = load_vert(V, F[3 * (int64_t)t]), b = load_vert(V, F[3 * (int64_t)t + 1]),
           c = load_vert(V, F[3 * (int64_t)t + 2]);
    out[3 * k] = make_float4(a.x, a.y, a.z, __int_as_float(t));
    out[3 * k + 1] = make_float4(b.x, b.y, b.z, 0.f);
    out[3 * k + 2] = make_float4(c.x, c.y, c.z, 0.f);
}

// --- pseudonormals ---------------------------------------------------------
__global__ void k_face_normals(const float* V, const int32_t* F, int64_t nt, float4* fn, float* vpn,
                               uint64_t* ekeys, int32_t* evals)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int32_t vi[3] = {F[3 * t], F[3 * t + 1], F[3 * t + 2]};
    float3 p[3] = {load_vert(V, vi[0]), load_vert(V, vi[1]), load_vert(V, vi[2])};
    float3 e1 = make_float3(p[1].x - p[0].x, p[1].y - p[0].y, p[1].z - p[0].z);
    float3 e2 = make_float3(p[2].x - p[0].x, p[2].y - p[0].y, p[2].z - p[0].z);
    float3 n = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
    float len = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
    if (len > 0.f) n = make_float3(n.x / len, n.y / len, n.z / len);
    else n = make_float3(0.f, 0.f, 0.f);
    fn[t] = make_float4(n.x, n.y, n.z, 0.f);
    for (int c = 0; c < 3; ++c) {
        float3 q = p[(c + 1) % 3], r = p[(c + 2) % 3];
        float3 x = make_float3(q.x - p[c].x, q.y - p[c].y, q.z - p[c].z);
        float3 y = make_float3(r.x - p[c].x, r.y - p[c].y, r.z - p[c].z);
        float3 cr = make_float3(x.y * y.z - x.z * y.y, x.z * y.x - x.x * y.z, x.x * y.y - x.y * y.x);
        float ang = atan2f(sqrtf(cr.x * cr.x + cr.y * cr.y + cr.z * cr.z), x.x * y.x + x.y * y.y + x.z * y.z);
        atomicAdd(&vpn[3 * (int64_t)vi[c]], ang * n.x);
        atomicAdd(&vpn[3 * (int64_t)vi[c] + 1], ang * n.y);
        atomicAdd(&vpn[3 * (int64_t)vi[c] + 2], ang * n.z);
        int32_t a = vi[c], b = vi[(c + 1) % 3];
        uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
        ekeys[3 * t + c] = ((uint64_t)lo << 32) | hi;
        evals[3 * t + c] = (int32_t)(3 * t + c);
    }
}

// edge pseudonormal = sum of the unit normals of all faces on the edge
__global__ void k_edge_normals(const uint64_t* keys, const int32_t* vals, int64_t m, const float4* fn, float4* en)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    uint64_t key = keys[k];
    int64_t s = k;
    while (s > 0 && keys[s - 1] == key) --s;
    float3 sum = make_float3(0.f, 0.f, 0.f);
    for (int64_t e = s; e < m && keys[e] == key; ++e) {
        float4 f = fn[vals[e] / 3];
        sum.x += f.x;
        sum.y += f.y;
        sum.z += f.z;
    }
    en[vals[k]] = make_float4(sum.x, sum.y, sum.z, 0.f);
}

__global__ void k_pack_pn(const int32_t* F, const int32_t* order, int64_t n, const float4* fn, const float4* en,
                          const float* vpn, float4* out)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int32_t t = order[k];
    float4* o = out + 7 * k;
    o[0] = fn[t];
    o[1] = en[3 * (int64_t)t];
    o[2] = en[3 * (int64_t)t + 1];
    o[3] = en[3 * (int64_t)t + 2];
    for (int c = 0; c < 3; ++c) {
        int64_t v = F[3 * (int64_t)t + c];
        o[4 + c] = make_float4(vpn[3 * v], vpn[3 * v + 1], vpn[3 * v + 2], 0.f);
    }
}

// scoped device allocation released when the build returns
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    template <class T>
    T* as() { return static_cast<T*>(p); }
};

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace

#define ALLOC(buf, bytes) RT_CUDA_TRY(cudaMalloc(&(buf).p, (size_t)(bytes) > 0 ? (size_t)(bytes) : 16))

rt_status rt_build_scene(const float* V, int64_t nv, const int32_t* F, int64_t nt, cudaStream_t s, rt_scene* sc)
{
    sc->n_tris = nt;
    sc->n_verts = nv;
    sc->n_nodes = nt - 1;
    DevBuf cen, bounds, keys, keys2, vals, vals2, child, par_i, par_l, llo, lhi, nlo, nhi, visit, depth, tmp;
    DevBuf fn, vpn, ek, ek2, ev, ev2, en;
    ALLOC(cen, nt * sizeof(float4));
    ALLOC(bounds, 12 * sizeof(int));
    ALLOC(keys, nt * sizeof(uint64_t));
    ALLOC(keys2, nt * sizeof(uint64_t));
    ALLOC(vals, nt * sizeof(int32_t));
    ALLOC(vals2, nt * sizeof(int32_t));
    ALLOC(child, (nt - 1) * sizeof(int2));
    DevBuf nrange;
    ALLOC(nrange, (nt - 1) * sizeof(int2));
    ALLOC(par_i, (nt - 1) * sizeof(int32_t));
    ALLOC(par_l, nt * sizeof(int32_t));
    ALLOC(llo, nt * sizeof(float4));
    ALLOC(lhi, nt * sizeof(float4));
    ALLOC(nlo, (nt - 1) * sizeof(float4));
    ALLOC(nhi, (nt - 1) * sizeof(float4));
    ALLOC(visit, (nt - 1) * sizeof(int));
    ALLOC(depth, sizeof(int));

    {
        DevBuf range;
        ALLOC(range, 2 * sizeof(int));
        int r0[2] = {INT32_MAX, INT32_MIN}, r1[2];
        RT_CUDA_TRY(cudaMemcpyAsync(range.p, r0, sizeof(r0), cudaMemcpyHostToDevice, s));
        k_index_range<<<1024, kBlock, 0, s>>>(F, 3 * nt, range.as<int>());
        RT_CUDA_TRY(cudaGetLastError());
        RT_CUDA_TRY(cudaMemcpyAsync(r1, range.p, sizeof(r1), cudaMemcpyDeviceToHost, s));
        RT_CUDA_TRY(cudaStreamSynchronize(s));
        if (r1[0] < 0 || (int64_t)r1[1] >= nv)
            return rt_fail(RT_ERR_INVALID_ARG, "triangle vertex indices span [%d, %d], need [0, %lld)", r1[0], r1[1],
                           (long long)nv);
    }
    int init[12];
    for (int k = 0; k < 12; ++k) init[k] = (k % 6) < 3 ? INT32_MAX : INT32_MIN;
    RT_CUDA_TRY(cudaMemcpyAsync(bounds.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_tri_bounds<<<grid_for(nt), kBlock, 0, s>>>(V, F, nt, cen.as<float4>(), bounds.as<int>());
    RT_CUDA_TRY(cudaGetLastError());
    k_morton<<<grid_for(nt), kBlock, 0, s>>>(cen.as<float4>(), nt, bounds.as<int>(), keys.as<uint64_t>(),
                                             vals.as<int32_t>());
    RT_CUDA_TRY(cudaGetLastError());

    size_t tmp_bytes = 0;
    RT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys.as<uint64_t>(), keys2.as<uint64_t>(),
                                                vals.as<int32_t>(), vals2.as<int32_t>(), (int)nt, 0, 64, s));
    ALLOC(tmp, tmp_bytes);
    RT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, keys.as<uint64_t>(), keys2.as<uint64_t>(),
                                                vals.as<int32_t>(), vals2.as<int32_t>(), (int)nt, 0, 64, s));
    const uint64_t* skeys = keys2.as<uint64_t>();
    int32_t* order = vals2.as<int32_t>();

    RT_CUDA_TRY(cudaMemsetAsync(visit.p, 0, (nt > 1 ? nt - 1 : 1) * sizeof(int), s));
    RT_CUDA_TRY(cudaMemsetAsync(depth.p, 0, sizeof(int), s));
    if (nt > 1) {
        k_hierarchy<<<grid_for(nt - 1), kBlock, 0, s>>>(skeys, nt, child.as<int2>(), nrange.as<int2>(), par_i.as<int32_t>(),
                                                        par_l.as<int32_t>());
        RT_CUDA_TRY(cudaGetLastError());
    } else {
        int m1 = -1;
        RT_CUDA_TRY(cudaMemcpyAsync(par_l.p, &m1, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    k_refit<<<grid_for(nt), kBlock, 0, s>>>(V, F, order, nt, child.as<int2>(), par_i.as<int32_t>(),
                                            par_l.as<int32_t>(), llo.as<float4>(), lhi.as<float4>(),
                                            nlo.as<float4>(), nhi.as<float4>(), visit.as<int>());
    RT_CUDA_TRY(cudaGetLastError());
    if (nt > 2) {
        rt_status ts = rt_treelet_optimise(nt, kTreeletPasses, child.as<int2>(), nrange.as<int2>(), par_i.as<int32_t>(),
                                           par_l.as<int32_t>(), order, llo.as<float4>(), lhi.as<float4>(),
                                           nlo.as<float4>(), nhi.as<float4>(), s);
        if (ts != RT_OK) return ts;
    }
    k_depth<<<grid_for(nt), kBlock, 0, s>>>(par_i.as<int32_t>(), par_l.as<int32_t>(), nt, depth.as<int>());
    RT_CUDA_TRY(cudaGetLastError());

    int hb[12];
    int hdepth = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(hb, bounds.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
    RT_CUDA_TRY(cudaMemcpyAsync(&hdepth, depth.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    float mag = 0.f;
    for (int k = 0; k < 6; ++k) {
        float v = ord2f(hb[k]);
        if (k < 3) sc->lo[k] = v; else sc->hi[k - 3] = v;
        mag = fmaxf(mag, fabsf(v));
    }
    for (int k = 0; k < 3; ++k) mag = fmaxf(mag, sc->hi[k] - sc->lo[k]);
    sc->max_depth = hdepth;
    if (!isfinite(mag)) return rt_fail(RT_ERR_INVALID_ARG, "vertex coordinates are not finite");
    if (hdepth > RT_STACK_DEPTH)
        return rt_fail(RT_ERR_DEVICE_LIMIT, "BVH depth %d exceeds the traversal stack (%d)", hdepth, RT_STACK_DEPTH);
    const float pad = ldexpf(mag, -18);

    RT_CUDA_TRY(cudaMalloc(&sc->nodes, (size_t)(nt > 1 ? nt - 1 : 1) * sizeof(BNode)));
    RT_CUDA_TRY(cudaMalloc(&sc->tris, (size_t)nt * 3 * sizeof(float4)));
    RT_CUDA_TRY(cudaMalloc(&sc->pn, (size_t)nt * 7 * sizeof(float4)));
    RT_CUDA_TRY(cudaMalloc(&sc->slot, (size_t)nt * sizeof(int32_t)));
    sc->bytes = (int64_t)((nt > 1 ? nt - 1 : 1) * sizeof(BNode) + nt * 3 * sizeof(float4) + nt * 7 * sizeof(float4) +
                          nt * sizeof(int32_t));
    if (nt > 1) {
        k_pack_nodes<<<grid_for(nt - 1), kBlock, 0, s>>>(child.as<int2>(), nt - 1, llo.as<float4>(), lhi.as<float4>(),
                                                          nlo.as<float4>(), nhi.as<float4>(), pad, sc->nodes);
        RT_CUDA_TRY(cudaGetLastError());
    }
    k_pack_tris<<<grid_for(nt), kBlock, 0, s>>>(V, F, order, nt, sc->tris, sc->slot);
    RT_CUDA_TRY(cudaGetLastError());
    {
        rt_status ws = rt_build_wide(sc, child.as<int2>(), nrange.as<int2>(), nlo.as<float4>(), nhi.as<float4>(),
                                     llo.as<float4>(), lhi.as<float4>(), pad, s);
        if (ws != RT_OK) return ws;
    }

    // pseudonormals
    ALLOC(fn, nt * sizeof(float4));
    ALLOC(vpn, nv * 3 * sizeof(float));
    ALLOC(ek, 3 * nt * sizeof(uint64_t));
    ALLOC(ek2, 3 * nt * sizeof(uint64_t));
    ALLOC(ev, 3 * nt * sizeof(int32_t));
    ALLOC(ev2, 3 * nt * sizeof(int32_t));
    ALLOC(en, 3 * nt * sizeof(float4));
    RT_CUDA_TRY(cudaMemsetAsync(vpn.p, 0, nv * 3 * sizeof(float), s));
    k_face_normals<<<grid_for(nt), kBlock, 0, s>>>(V, F, nt, fn.as<float4>(), vpn.as<float>(), ek.as<uint64_t>(),
                                                   ev.as<int32_t>());
    RT_CUDA_TRY(cudaGetLastError());
    size_t tmp2 = 0;
    RT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp2, ek.as<uint64_t>(), ek2.as<uint64_t>(), ev.as<int32_t>(),
                                                ev2.as<int32_t>(), (int)(3 * nt), 0, 64, s));
    DevBuf tmpb;
    ALLOC(tmpb, tmp2);
    RT_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmpb.p, tmp2, ek.as<uint64_t>(), ek2.as<uint64_t>(), ev.as<int32_t>(),
                                                ev2.as<int32_t>(), (int)(3 * nt), 0, 64, s));
    k_edge_normals<<<grid_for(3 * nt), kBlock, 0, s>>>(ek2.as<uint64_t>(), ev2.as<int32_t>(), 3 * nt, fn.as<float4>(),
                                                       en.as<float4>());
    RT_CUDA_TRY(cudaGetLastError());
    k_pack_pn<<<grid_for(nt), kBlock, 0, s>>>(F, order, nt, fn.as<float4>(), en.as<float4>(), vpn.as<float>(), sc->pn);
    RT_CUDA_TRY(cudaGetLastError());
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    return RT_OK;
}
