// The paper's distance-field build (Section 3, "Distance Field Generation"):
// the triangles are voxelised, the voxelisation is turned into a distance
// field by jump flooding, and fast sweeping refines it.  The paper names the
// three steps only; the steps taken here:
//
//   1. Conservative voxelisation.  Sample s owns the voxel box of side
//      h (1 + 2^-8) centred on it.  Every triangle is tested (separating axes,
//      Akenine-Moller, JGT 2001) against the voxels its bounds can reach: one
//      thread per triangle when they are few, one block per triangle when they
//      are many; an overlapping triangle is a candidate site of the sample.
//      The best candidate wins through a 64-bit atomicMin on (squared
//      distance bits, triangle index).  On a cascade level below the
//      coarsest, the site of the nearest sample of the next coarser level is a
//      candidate too.
//   2. Jump flooding (Rong & Tan, I3D 2006): steps k = 2^(ceil(log2 n)-1) ...
//      1; each sample takes the best of the sites of itself and its 26
//      neighbours at offsets in {-k, 0, k}^3, from the previous step.
//   3. Fast sweeping as axis sweeps, +x, -x, +y, -y, +z, -z: one thread per
//      grid line carries the best site along the line.
//   4. The field value is the signed distance to the site triangle (the
//      exact bake's closest point and pseudonormal sign).
//
// "Best" is the smallest (squared distance from the sample to the site's
// triangle, triangle index).  Every operation of steps 1-3 is rounded once
// (explicit intrinsics), so the sites are those of the CPU checker's single
// precision build, bit for bit.
#include "rt_bake_dev.cuh"
#include "rt_trace_dev.cuh"

namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// single precision geometry, each operation rounded once
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot3r(const float* a, const float* b)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
}

// squared distance from p to triangle abc (Ericson's Voronoi regions)
__device__ float tri_d2_rn(const float* p, const float* a, const float* b, const float* c)
{
    float ab[3], ac[3], ap[3], q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ab[k] = __fsub_rn(b[k], a[k]);
        ac[k] = __fsub_rn(c[k], a[k]);
        ap[k] = __fsub_rn(p[k], a[k]);
    }
    const float d1 = dot3r(ab, ap), d2 = dot3r(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) {
#pragma unroll
        for (int k = 0; k < 3; ++k) q[k] = a[k];
    } else {
        float bp[3], cp[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            bp[k] = __fsub_rn(p[k], b[k]);
            cp[k] = __fsub_rn(p[k], c[k]);
        }
        const float d3 = dot3r(ab, bp), d4 = dot3r(ac, bp);
        const float vc = __fsub_rn(__fmul_rn(d1, d4), __fmul_rn(d3, d2));
        const float d5 = dot3r(ab, cp), d6 = dot3r(ac, cp);
        const float vb = __fsub_rn(__fmul_rn(d5, d2), __fmul_rn(d1, d6));
        const float va = __fsub_rn(__fmul_rn(d3, d6), __fmul_rn(d5, d4));
        if (d3 >= 0.f && d4 <= d3) {
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = b[k];
        } else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
            const float s = __fdiv_rn(d1, __fsub_rn(d1, d3));
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = __fadd_rn(a[k], __fmul_rn(s, ab[k]));
        } else if (d6 >= 0.f && d5 <= d6) {
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = c[k];
        } else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
            const float s = __fdiv_rn(d2, __fsub_rn(d2, d6));
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = __fadd_rn(a[k], __fmul_rn(s, ac[k]));
        } else if (va <= 0.f && __fsub_rn(d4, d3) >= 0.f && __fsub_rn(d5, d6) >= 0.f) {
            const float s = __fdiv_rn(__fsub_rn(d4, d3), __fadd_rn(__fsub_rn(d4, d3), __fsub_rn(d5, d6)));
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = __fadd_rn(b[k], __fmul_rn(s, __fsub_rn(c[k], b[k])));
        } else {
            const float den = __fdiv_rn(1.f, __fadd_rn(__fadd_rn(va, vb), vc));
            const float v = __fmul_rn(vb, den), w = __fmul_rn(vc, den);
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = __fadd_rn(__fadd_rn(a[k], __fmul_rn(ab[k], v)), __fmul_rn(ac[k], w));
        }
    }
    const float pq[3] = {__fsub_rn(p[0], q[0]), __fsub_rn(p[1], q[1]), __fsub_rn(p[2], q[2])};
    return dot3r(pq, pq);
}

__device__ __forceinline__ bool axis_separates(const float* ax, const float* v0, const float* v1, const float* v2,
                                               const float* hs)
{
    const float p0 = dot3r(ax, v0), p1 = dot3r(ax, v1), p2 = dot3r(ax, v2);
    const float lo = fminf(fminf(p0, p1), p2), hi = fmaxf(fmaxf(p0, p1), p2);
    const float r = __fadd_rn(__fadd_rn(__fmul_rn(hs[0], fabsf(ax[0])), __fmul_rn(hs[1], fabsf(ax[1]))),
                              __fmul_rn(hs[2], fabsf(ax[2])));
    return lo > r || hi < -r;
}

// triangle / box overlap by separating axes (touching counts)
__device__ bool tri_box(const float* c, const float* hs, const float* A, const float* B, const float* C)
{
    float v0[3], v1[3], v2[3], e[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v0[k] = __fsub_rn(A[k], c[k]);
        v1[k] = __fsub_rn(B[k], c[k]);
        v2[k] = __fsub_rn(C[k], c[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e[0][k] = __fsub_rn(v1[k], v0[k]);
        e[1][k] = __fsub_rn(v2[k], v1[k]);
        e[2][k] = __fsub_rn(v0[k], v2[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ax[3] = {0.f, 0.f, 0.f};
        ax[k] = 1.f;
        if (axis_separates(ax, v0, v1, v2, hs)) return false;
    }
    const float n[3] = {__fsub_rn(__fmul_rn(e[0][1], e[1][2]), __fmul_rn(e[0][2], e[1][1])),
                        __fsub_rn(__fmul_rn(e[0][2], e[1][0]), __fmul_rn(e[0][0], e[1][2])),
                        __fsub_rn(__fmul_rn(e[0][0], e[1][1]), __fmul_rn(e[0][1], e[1][0]))};
    if (axis_separates(n, v0, v1, v2, hs)) return false;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float ax0[3] = {0.f, -e[j][2], e[j][1]};
        const float ax1[3] = {e[j][2], 0.f, -e[j][0]};
        const float ax2[3] = {-e[j][1], e[j][0], 0.f};
        if (axis_separates(ax0, v0, v1, v2, hs) || axis_separates(ax1, v0, v1, v2, hs) ||
            axis_separates(ax2, v0, v1, v2, hs))
            return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// grid geometry (one grid, or one cascade level)
// ---------------------------------------------------------------------------
struct DfGrid {
    int32_t n[3];
    int32_t lattice;
    int32_t ilo[3];
    float lo[3], h[3], hs[3];
    // conservative sample range of a triangle: origin, 1/h and a margin of a
    // small fraction of a voxel (much more than the rounding of the positions)
    float origin_f[3], ih_f[3], margin[3];
    int64_t count;
};

__device__ __forceinline__ void df_pos(const DfGrid& g, int64_t i, int64_t j, int64_t k, float* p)
{
    const int64_t ii[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        p[a] = g.lattice ? __fmul_rn((float)(g.ilo[a] + ii[a]), g.h[a]) : __fmaf_rn((float)ii[a], g.h[a], g.lo[a]);
}

struct Tris {
    const float4* tris;   // leaf order, 3 per triangle
    const int32_t* slot;  // input index -> leaf position
    int64_t n;
};

__device__ __forceinline__ void tri_verts(const Tris& T, int32_t t, float* A, float* B, float* C)
{
    const int64_t k = 3 * (int64_t)__ldg(T.slot + t);
    const float4 a = __ldg(T.tris + k), b = __ldg(T.tris + k + 1), c = __ldg(T.tris + k + 2);
    A[0] = a.x; A[1] = a.y; A[2] = a.z;
    B[0] = b.x; B[1] = b.y; B[2] = b.z;
    C[0] = c.x; C[1] = c.y; C[2] = c.z;
}

__device__ __forceinline__ float site_d2(const Tris& T, const float* p, int32_t t)
{
    float A[3], B[3], C[3];
    tri_verts(T, t, A, B, C);
    return tri_d2_rn(p, A, B, C);
}

// keep the better of (cur, cur_d2) and candidate t
__device__ __forceinline__ void site_consider(const Tris& T, const float* p, int32_t t, int32_t& cur, float& cur_d2)
{
    if (t < 0 || t == cur) return;
    const float d2 = site_d2(T, p, t);
    if (cur < 0 || d2 < cur_d2 || (d2 == cur_d2 && t < cur)) {
        cur = t;
        cur_d2 = d2;
    }
}

// samples whose voxels the triangle's bounds may reach: the range is widened by
// a small fraction of a voxel, far more than the rounding of the sample
// positions, and the separating-axis test decides
__device__ __forceinline__ bool tri_range(const DfGrid& g, const float* A, const float* B, const float* C,
                                          int64_t r0[3], int64_t r1[3])
{
    bool empty = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo_t = fminf(fminf(A[a], B[a]), C[a]) - g.hs[a];
        const float hi_t = fmaxf(fmaxf(A[a], B[a]), C[a]) + g.hs[a];
        const float x0f = ceilf((lo_t - g.origin_f[a] - g.margin[a]) * g.ih_f[a]);
        const float x1f = floorf((hi_t - g.origin_f[a] + g.margin[a]) * g.ih_f[a]);
        // clamp in float first: far-away triangles give values beyond the int range
        const int64_t x0 = (int64_t)fmaxf(x0f, 0.f);
        const int64_t x1 = (int64_t)fminf(x1f, (float)(g.n[a] - 1));
        r0[a] = x0;
        r1[a] = x1;
        empty = empty || x0 > x1 || x1f < 0.f || x0f > (float)(g.n[a] - 1);
    }
    return !empty;
}

// test one (triangle, sample) pair and keep the better site of the sample
__device__ __forceinline__ void vox_pair(const DfGrid& g, int32_t t, const float* A, const float* B, const float* C,
                                         int64_t i, int64_t j, int64_t k, unsigned long long* keys)
{
    float p[3];
    df_pos(g, i, j, k, p);
    if (!tri_box(p, g.hs, A, B, C)) return;
    const float d2 = tri_d2_rn(p, A, B, C);
    const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (uint32_t)t;
    atomicMin(keys + i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k), key);
}

constexpr int64_t kSmallPairs = 64;  // a thread tests a triangle's voxels itself up to this many

// the grids voxelised by one pass over the triangles (all levels of a cascade at once)
struct VoxPass {
    DfGrid g[RT_MAX_LEVELS];
    unsigned long long* keys[RT_MAX_LEVELS];
    int32_t count;
};

// one thread per triangle and level: small ranges are tested here, large ones
// listed (triangle, level) for k_df_vox_big
__global__ void k_df_vox_small(const VoxPass vp, const Tris T, int2* big, unsigned* n_big)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T.n) return;
    float A[3], B[3], C[3];
    tri_verts(T, (int32_t)t, A, B, C);
    for (int l = 0; l < vp.count; ++l) {
        const DfGrid& g = vp.g[l];
        int64_t r0[3], r1[3];
        if (!tri_range(g, A, B, C, r0, r1)) continue;
        const int64_t count = (r1[0] - r0[0] + 1) * (r1[1] - r0[1] + 1) * (r1[2] - r0[2] + 1);
        if (count > kSmallPairs) {
            big[atomicAdd(n_big, 1u)] = make_int2((int)t, l);
            continue;
        }
        for (int64_t k = r0[2]; k <= r1[2]; ++k)
            for (int64_t j = r0[1]; j <= r1[1]; ++j)
                for (int64_t i = r0[0]; i <= r1[0]; ++i) vox_pair(g, (int32_t)t, A, B, C, i, j, k, vp.keys[l]);
    }
}

// one block per listed (triangle, level), threads over its voxels
__global__ void k_df_vox_big(const VoxPass vp, const Tris T, const int2* big, const unsigned* n_big)
{
    const unsigned nb = *n_big;
    for (unsigned b = blockIdx.x; b < nb; b += gridDim.x) {
        const int2 e = big[b];
        const DfGrid& g = vp.g[e.y];
        float A[3], B[3], C[3];
        tri_verts(T, e.x, A, B, C);
        int64_t r0[3], r1[3];
        tri_range(g, A, B, C, r0, r1);
        const int64_t sx = r1[0] - r0[0] + 1, sy = r1[1] - r0[1] + 1;
        const int64_t count = sx * sy * (r1[2] - r0[2] + 1);
        for (int64_t w = threadIdx.x; w < count; w += blockDim.x)
            vox_pair(g, e.x, A, B, C, r0[0] + w % sx, r0[1] + (w / sx) % sy, r0[2] + w / (sx * sy), vp.keys[e.y]);
    }
}

__device__ __forceinline__ int64_t floordiv(int64_t x, int64_t y)  // y > 0
{
    return x >= 0 ? x / y : -((-x + y - 1) / y);
}

// sites from the voxelisation; on a cascade level also the coarser level's site
__global__ void k_df_seed(const DfGrid g, const Tris T, const unsigned long long* keys, const int32_t* coarse,
                          const DfGrid gc, int32_t* sites)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.count) return;
    const unsigned long long key = keys[s];
    int32_t cur = key == ~0ull ? -1 : (int32_t)(key & 0xffffffffull);
    float cd2 = __uint_as_float((uint32_t)(key >> 32));
    if (coarse) {
        const int64_t ii[3] = {s % g.n[0], (s / g.n[0]) % g.n[1], s / ((int64_t)g.n[0] * g.n[1])};
        int64_t jc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int64_t j = floordiv(g.ilo[a] + ii[a] + 1, 2) - gc.ilo[a];
            jc[a] = j < 0 ? 0 : (j > gc.n[a] - 1 ? gc.n[a] - 1 : j);
        }
        float p[3];
        df_pos(g, ii[0], ii[1], ii[2], p);
        site_consider(T, p, coarse[jc[0] + (int64_t)gc.n[0] * (jc[1] + (int64_t)gc.n[1] * jc[2])], cur, cd2);
    }
    sites[s] = cur;
}

// Neighbours mostly carry the same few sites: the distances of the last few
// distinct candidates are kept, so each is evaluated once per sample.  The
// result is the same minimum.
constexpr int kSiteCache = 4;

__global__ void k_df_jfa(const DfGrid g, const Tris T, const int32_t* in, int32_t* out, int32_t step)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.count) return;
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t i = s % nx, j = (s / nx) % ny, k = s / (nx * ny);
    float p[3];
    df_pos(g, i, j, k, p);
    int32_t best = -1;
    float bd2 = 0.f;
    int32_t seen[kSiteCache];
#pragma unroll
    for (int c = 0; c < kSiteCache; ++c) seen[c] = -1;
    for (int dz = -1; dz <= 1; ++dz) {
        const int64_t z = k + dz * step;
        if (z < 0 || z >= nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int64_t y = j + dy * step;
            if (y < 0 || y >= ny) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int64_t x = i + dx * step;
                if (x < 0 || x >= nx) continue;
                const int32_t t = __ldg(in + x + nx * (y + ny * z));
                if (t < 0) continue;
                bool hit = false;
#pragma unroll
                for (int c = 0; c < kSiteCache; ++c) hit = hit || seen[c] == t;
                if (hit) continue;  // already evaluated at this sample
#pragma unroll
                for (int c = kSiteCache - 1; c > 0; --c) seen[c] = seen[c - 1];
                seen[0] = t;
                site_consider(T, p, t, best, bd2);
            }
        }
    }
    out[s] = best;
}

// one thread per grid line along `axis`, walking in direction dir (+1 / -1).
// The line's sites are read eight at a time (independent loads in flight
// together); each is the value before this sweep reaches it, as in the
// sequential sweep, since the sweep only writes samples it has passed.
constexpr int kSweepChunk = 8;

// the grids swept by one launch (all levels of a cascade at once)
struct SweepPass {
    DfGrid g[RT_MAX_LEVELS];
    int32_t* sites[RT_MAX_LEVELS];
    int64_t first_line[RT_MAX_LEVELS + 1];  // prefix sums of the levels' line counts
    int32_t count;
};

__global__ void k_df_sweep(const SweepPass sp, const Tris T, int axis, int dir)
{
    const int oa = axis == 0 ? 1 : 0, ob = axis == 2 ? 1 : 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= sp.first_line[sp.count]) return;
    int l = 0;
    while (l + 1 < sp.count && t >= sp.first_line[l + 1]) ++l;
    const DfGrid& g = sp.g[l];
    int32_t* sites = sp.sites[l];
    const int64_t line = t - sp.first_line[l];
    const int64_t n[3] = {g.n[0], g.n[1], g.n[2]};
    const int64_t stride[3] = {1, n[0], n[0] * n[1]};
    const int64_t ua = line % n[oa], ub = line / n[oa];
    const int64_t base = ua * stride[oa] + ub * stride[ob];
    const int64_t len = n[axis];
    int32_t prev = sites[base + (dir > 0 ? 0 : len - 1) * stride[axis]];
    for (int64_t c0 = 1; c0 < len; c0 += kSweepChunk) {
        int32_t buf[kSweepChunk];
#pragma unroll
        for (int u = 0; u < kSweepChunk; ++u) {
            const int64_t step = c0 + u;
            const int64_t q = dir > 0 ? step : len - 1 - step;
            buf[u] = step < len ? sites[base + q * stride[axis]] : -1;
        }
#pragma unroll
        for (int u = 0; u < kSweepChunk; ++u) {
            const int64_t step = c0 + u;
            if (step >= len) break;
            int32_t cur = buf[u];
            if (prev >= 0 && prev != cur) {  // otherwise nothing can change
                const int64_t q = dir > 0 ? step : len - 1 - step;
                int64_t ii[3];
                ii[axis] = q;
                ii[oa] = ua;
                ii[ob] = ub;
                float p[3];
                df_pos(g, ii[0], ii[1], ii[2], p);
                float cd2 = cur >= 0 ? site_d2(T, p, cur) : 0.f;
                site_consider(T, p, prev, cur, cd2);
                sites[base + q * stride[axis]] = cur;
            }
            prev = cur;
        }
    }
}

// Both sweeps of one axis for one level: a thread takes one grid line, loads it
// into shared memory, sweeps it in the + direction and then in the - direction
// (lines of one axis are independent, so this equals all + sweeps followed by
// all - sweeps), and writes it back.  The line is stored interleaved
// (sample q of thread t at q * blockDim + t), so a warp's accesses to one q
// fall in different banks.  The site carried along the line keeps its triangle
// in registers: a step loads only the triangle of its own sample's site, and
// only when the two sites differ.  Same operations, same order, same sites as
// k_df_sweep.
constexpr int kLineMax = 1024;  // longest line swept in shared memory

// One step of a sweep at sample q.  CA/CB/CC hold the triangle of the sample's
// own site `cur` (loaded one step ahead by the caller); PA/PB/PC the carried
// site's, valid when prev_loaded.
__device__ __forceinline__ void sweep_step(const DfGrid& g, const Tris& T, int64_t ii[3], int axis, int64_t q,
                                           int32_t cur, const float CA[3], const float CB[3], const float CC[3],
                                           int32_t& prev, float PA[3], float PB[3], float PC[3], bool& prev_loaded,
                                           int32_t* slot)
{
    if (prev >= 0 && prev != cur) {
        ii[axis] = q;
        float p[3];
        df_pos(g, ii[0], ii[1], ii[2], p);
        const float cd2 = cur >= 0 ? tri_d2_rn(p, CA, CB, CC) : 0.f;
        if (!prev_loaded) {
            tri_verts(T, prev, PA, PB, PC);
            prev_loaded = true;
        }
        const float d2 = tri_d2_rn(p, PA, PB, PC);
        if (cur < 0 || d2 < cd2 || (d2 == cd2 && prev < cur)) {
            cur = prev;  // the carried site wins and stays carried
            *slot = cur;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {  // the sample's own site is carried on
                PA[k] = CA[k];
                PB[k] = CB[k];
                PC[k] = CC[k];
            }
        }
    } else if (cur != prev) {
        prev_loaded = false;  // a new carried site whose triangle is not loaded yet
    }
    prev = cur;
}

// the triangle of site t (nothing for t < 0)
__device__ __forceinline__ void site_verts(const Tris& T, int32_t t, float A[3], float B[3], float C[3])
{
    if (t >= 0) tri_verts(T, t, A, B, C);
}

// one direction of a line's sweep: samples q0, q0 + dq, ... (len - 1 of them),
// carrying from q0 - dq; the next sample's triangle is loaded a step ahead
__device__ __forceinline__ void sweep_dir(const DfGrid& g, const Tris& T, int64_t ii[3], int axis, int32_t* L,
                                          int64_t B, int64_t q0, int64_t dq, int64_t count)
{
    float PA[3], PB[3], PC[3], CA[3], CB[3], CC[3];
    bool prev_loaded = false;
    int32_t prev = L[(q0 - dq) * B];
    int32_t cur = L[q0 * B];
    site_verts(T, cur, CA, CB, CC);
    for (int64_t k = 0; k < count; ++k) {
        const int64_t q = q0 + k * dq;
        int32_t nxt = -1;
        float NA[3], NB[3], NC[3];
        if (k + 1 < count) {
            nxt = L[(q + dq) * B];
            site_verts(T, nxt, NA, NB, NC);
        }
        sweep_step(g, T, ii, axis, q, cur, CA, CB, CC, prev, PA, PB, PC, prev_loaded, L + q * B);
        cur = nxt;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            CA[c] = NA[c];
            CB[c] = NB[c];
            CC[c] = NC[c];
        }
    }
}

__global__ void k_df_sweep_line(const DfGrid g, const Tris T, int32_t* sites, int axis)
{
    extern __shared__ int32_t s_line[];
    const int oa = axis == 0 ? 1 : 0, ob = axis == 2 ? 1 : 2;
    const int64_t n[3] = {g.n[0], g.n[1], g.n[2]};
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= n[oa] * n[ob]) return;
    const int64_t stride[3] = {1, n[0], n[0] * n[1]};
    int64_t ii[3];
    ii[oa] = line % n[oa];
    ii[ob] = line / n[oa];
    ii[axis] = 0;
    const int64_t base = ii[oa] * stride[oa] + ii[ob] * stride[ob];
    const int64_t len = n[axis];
    const int64_t B = blockDim.x;
    int32_t* L = s_line + threadIdx.x;
    for (int64_t q = 0; q < len; ++q) L[q * B] = sites[base + q * stride[axis]];
    sweep_dir(g, T, ii, axis, L, B, 1, 1, len - 1);         // + direction: samples 1 .. len-1
    sweep_dir(g, T, ii, axis, L, B, len - 2, -1, len - 1);  // - direction: samples len-2 .. 0
    for (int64_t q = 0; q < len; ++q) sites[base + q * stride[axis]] = L[q * B];
}

// signed distance to the site triangle (the exact bake's closest point and sign)
__global__ void k_df_field(const DfGrid g, const Tris T, const float4* pn, const int32_t* sites, void* grid,
                           int32_t f16)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.count) return;
    const int32_t t = sites[s];
    float v = __int_as_float(0x7f800000);
    if (t >= 0) {
        float pp[3];
        df_pos(g, s % g.n[0], (s / g.n[0]) % g.n[1], s / ((int64_t)g.n[0] * g.n[1]), pp);
        const float3 p = make_float3(pp[0], pp[1], pp[2]);
        const int32_t k = __ldg(T.slot + t);
        rtbake::Nearest nb = {__int_as_float(0x7f800000), -1, 0x7fffffff};
        rtbake::consider(nb, p, T.tris, k);
        v = rtbake::signed_distance(p, nb, T.tris, pn);
    }
    if (f16) reinterpret_cast<__half*>(grid)[s] = __float2half_rn(v);
    else reinterpret_cast<float*>(grid)[s] = v;
}

// geometry of the single grid, or of cascade level k
DfGrid df_grid(const rt_sdf* sdf, int k)
{
    DfGrid g;
    memset(&g, 0, sizeof(g));
    g.count = 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = sdf->n[a];
        g.count *= sdf->n[a];
    }
    double origin[3];
    if (sdf->levels > 0) {
        const float hk = ldexpf(sdf->h0, k);
        g.lattice = 1;
        for (int a = 0; a < 3; ++a) {
            g.ilo[a] = sdf->ilo[k][a];
            g.h[a] = hk;
            origin[a] = (double)sdf->ilo[k][a] * (double)hk;
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            g.lo[a] = sdf->lo[a];
            g.h[a] = sdf->h[a];
            origin[a] = sdf->lo[a];
        }
    }
    for (int a = 0; a < 3; ++a) {
        volatile float half = 0.5f * g.h[a];
        volatile float grow = g.h[a] * (1.f / 512.f);
        g.hs[a] = half + grow;
        g.ih_f[a] = 1.0f / g.h[a];
        g.margin[a] = (float)(1e-2 * g.h[a] + 1e-5 * (fabs(origin[a]) + g.n[a] * (double)g.h[a]));
        g.origin_f[a] = (float)origin[a];
    }
    return g;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Steps 1..stage for the levels `lv[0..nl)` (0 for a single grid), given in
// the order they are built (coarsest first).  All levels are voxelised in one
// pass over the triangles (a level's voxel candidates do not depend on the
// other levels); then each level in turn is seeded (on a cascade also from the
// next coarser level's finished sites in `jfa`), flooded and swept, leaving its
// sites in `jfa` before the next finer level reads them.  The sites of every
// listed level also go to `out`.  jfa, out: one int32 per sample of every
// level (indexed by level), device.
rt_status df_build(const rt_scene* sc, const rt_sdf* sdf, const int* lv, int nl, int32_t stage, int32_t* jfa,
                   int32_t* out, cudaStream_t s)
{
    const Tris T = {sc->tris, sc->slot, sc->n_tris};
    const int64_t per = (int64_t)sdf->n[0] * sdf->n[1] * sdf->n[2];
    if (per > 0x7fffffffLL * (int64_t)kBlock) return rt_fail(RT_ERR_INVALID_ARG, "grid too large");
    const int cascade_levels = sdf->levels;

    // scratch: keys of every listed level, one spare site buffer, the large-triangle list
    const size_t keys_bytes = (size_t)per * 8 * nl, tmp_bytes = (size_t)per * 4, big_bytes = (size_t)T.n * 8 * nl;
    const size_t total = keys_bytes + tmp_bytes + big_bytes + 4 * 256;
    char* base = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&base, total, s));
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + off);
    off = align(off + keys_bytes);
    int32_t* tmp = reinterpret_cast<int32_t*>(base + off);
    off = align(off + tmp_bytes);
    int2* big = reinterpret_cast<int2*>(base + off);
    off = align(off + big_bytes);
    unsigned* n_big = reinterpret_cast<unsigned*>(base + off);

    rt_status st = RT_OK;
    cudaError_t e = cudaMemsetAsync(keys, 0xff, keys_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_big, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) st = rt_cuda_fail(e, "cudaMemsetAsync");

    // 1. voxelisation of all listed levels
    if (st == RT_OK && T.n > 0) {
        VoxPass vp;
        memset(&vp, 0, sizeof(vp));
        vp.count = nl;
        for (int l = 0; l < nl; ++l) {
            vp.g[l] = df_grid(sdf, lv[l]);
            vp.keys[l] = keys + (size_t)l * per;
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        k_df_vox_small<<<blocks_for(T.n), kBlock, 0, s>>>(vp, T, big, n_big);
        k_df_vox_big<<<(unsigned)(sms > 0 ? sms * 4 : 512), kBlock, 0, s>>>(vp, T, big, n_big);
    }
    // 2.-3. per level, coarsest first: seeding, jump flooding, the six sweeps
    for (int l = 0; l < nl && st == RT_OK; ++l) {
        const int k = lv[l];
        int32_t* sites = jfa + (int64_t)k * per;
        const DfGrid g = df_grid(sdf, k);
        DfGrid gc;
        memset(&gc, 0, sizeof(gc));
        const int32_t* coarse = nullptr;
        if (cascade_levels > 0 && k + 1 < cascade_levels) {
            gc = df_grid(sdf, k + 1);
            coarse = jfa + (int64_t)(k + 1) * per;
        }
        k_df_seed<<<blocks_for(g.count), kBlock, 0, s>>>(g, T, keys + (size_t)l * per, coarse, gc, sites);
        if (stage >= 2) {
            int64_t nmax = g.n[0] > g.n[1] ? g.n[0] : g.n[1];
            if (g.n[2] > nmax) nmax = g.n[2];
            int64_t step = 1;
            while (2 * step < nmax) step *= 2;
            int32_t* a = sites;
            int32_t* b = tmp;
            for (; step >= 1; step /= 2) {
                k_df_jfa<<<blocks_for(g.count), kBlock, 0, s>>>(g, T, a, b, (int32_t)step);
                int32_t* t = a;
                a = b;
                b = t;
            }
            if (a != sites) {
                e = cudaMemcpyAsync(sites, a, (size_t)g.count * 4, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) st = rt_cuda_fail(e, "cudaMemcpyAsync");
            }
        }
        if (st == RT_OK && stage >= 3) {
            for (int axis = 0; axis < 3; ++axis) {
                const int oa = axis == 0 ? 1 : 0, ob = axis == 2 ? 1 : 2;
                const int64_t lines = (int64_t)g.n[oa] * g.n[ob];
                if (g.n[axis] <= kLineMax) {
                    const int threads = g.n[axis] <= 512 ? 64 : 32;
                    const size_t smem = (size_t)threads * g.n[axis] * sizeof(int32_t);
                    if (smem > 48 * 1024) {
                        e = cudaFuncSetAttribute(k_df_sweep_line, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
                        if (e != cudaSuccess) {
                            st = rt_cuda_fail(e, "cudaFuncSetAttribute");
                            break;
                        }
                    }
                    k_df_sweep_line<<<(unsigned)((lines + threads - 1) / threads), threads, smem, s>>>(g, T, sites,
                                                                                                      axis);
                } else {
                    SweepPass sp;
                    memset(&sp, 0, sizeof(sp));
                    sp.count = 1;
                    sp.g[0] = g;
                    sp.sites[0] = sites;
                    sp.first_line[1] = lines;
                    for (int dir = 1; dir >= -1; dir -= 2)
                        k_df_sweep<<<(unsigned)((lines + 63) / 64), 64, 0, s>>>(sp, T, axis, dir);
                }
            }
        }
        if (st == RT_OK && out != jfa) {
            e = cudaMemcpyAsync(out + (int64_t)k * per, sites, (size_t)g.count * 4, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = rt_cuda_fail(e, "cudaMemcpyAsync");
        }
    }
    if (st == RT_OK) {
        e = cudaGetLastError();
        if (e != cudaSuccess) st = rt_cuda_fail(e, "field build launch");
    }
    e = cudaFreeAsync(base, s);
    if (st == RT_OK && e != cudaSuccess) st = rt_cuda_fail(e, "cudaFreeAsync");
    return st;
}

rt_status field_values(const rt_scene* sc, const rt_sdf* sdf, const int* lv, int nl, const int32_t* sites,
                       cudaStream_t s)
{
    const Tris T = {sc->tris, sc->slot, sc->n_tris};
    const int64_t per = (int64_t)sdf->n[0] * sdf->n[1] * sdf->n[2];
    const int64_t esz = sdf->dtype == RT_GRID_F16 ? 2 : 4;
    for (int l = 0; l < nl; ++l) {
        const int k = lv[l];
        const DfGrid g = df_grid(sdf, k);
        char* grid = static_cast<char*>(const_cast<void*>(sdf->grid)) + k * per * esz;
        k_df_field<<<blocks_for(g.count), kBlock, 0, s>>>(g, T, sc->pn, sites + k * per, grid,
                                                        sdf->dtype == RT_GRID_F16);
    }
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

}  // namespace

// Sites of every sample after step `stage` (1..3), cascade levels one at a
// time, coarsest first (each seeded also from the next coarser level's sites
// after its steps 1..stage).
// d_sites holds levels * n^3 (or n0 n1 n2) entries.
rt_status rt_launch_df_sites(const rt_scene* sc, const rt_sdf* sdf, int32_t stage, int32_t* d_sites, cudaStream_t s)
{
    int lv[RT_MAX_LEVELS];
    const int nl = sdf->levels > 0 ? sdf->levels : 1;
    for (int l = 0; l < nl; ++l) lv[l] = nl - 1 - l;  // coarsest first
    const int64_t count = (int64_t)nl * sdf->n[0] * sdf->n[1] * sdf->n[2];
    int32_t* jfa = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&jfa, (size_t)count * 4, s));
    rt_status st = df_build(sc, sdf, lv, nl, stage, jfa, d_sites, s);
    cudaError_t e = cudaFreeAsync(jfa, s);
    if (st == RT_OK && e != cudaSuccess) st = rt_cuda_fail(e, "cudaFreeAsync");
    return st;
}

// The listed levels (all of them for a full build; the moved ones of a rolling
// update), coarsest first: finished sites into `jfa_store` (kept by the
// handle: the seeds of finer levels later), field values from them.
rt_status rt_launch_df_levels(const rt_scene* sc, const rt_sdf* sdf, const int* lv, int nl, int32_t* jfa_store,
                              cudaStream_t s)
{
    if (nl <= 0) return RT_OK;
    const int levels = sdf->levels > 0 ? sdf->levels : 1;
    const int64_t count = (int64_t)levels * sdf->n[0] * sdf->n[1] * sdf->n[2];
    int32_t* out = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&out, (size_t)count * 4, s));
    rt_status st = df_build(sc, sdf, lv, nl, 3, jfa_store, out, s);
    if (st == RT_OK) st = field_values(sc, sdf, lv, nl, out, s);
    cudaError_t e = cudaFreeAsync(out, s);
    if (st == RT_OK && e != cudaSuccess) st = rt_cuda_fail(e, "cudaFreeAsync");
    return st;
}
