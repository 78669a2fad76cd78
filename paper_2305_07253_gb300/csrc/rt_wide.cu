// 8-wide compressed BVH, collapsed from the binary LBVH on the device.
//
// The node format and the ray-octant child order follow the compressed wide
// BVH of Ylitie, Karras & Laine, "Efficient Incoherent Ray Traversal on GPUs
// Through Compressed Wide BVHs" (HPG 2017), in this library's own layout (see
// rt_internal.cuh): up to 8 children per 80-byte node, child boxes quantized to
// 8 bits against a power-of-two scale per axis, leaves of up to 3 triangles
// stored contiguously per node.
//
// Collapse, one thread per wide node, level by level: start from the two
// children of the binary node and keep replacing the child with the largest
// surface area by its two children until there are 8 or none can be opened
// (a binary subtree of at most 3 triangles becomes a leaf; the LBVH keeps the
// triangles of any subtree contiguous in leaf order).  Children are placed in
// the slots of the octant their centre lies in (greedy), so a traversal that
// visits slots in order "slot xor ray octant" goes roughly near to far.
#include <math.h>

#include "rt_internal.cuh"

namespace {

constexpr int kLeafMax = 3;
constexpr int kBlock = 128;

struct Entry {
    int ref;           // >= 0: binary internal node; < 0: sorted triangle ~ref
    int first, count;  // sorted triangles first .. first+count-1
    float lo[3], hi[3];
};

struct Item {
    int bin;   // binary internal node, or ~triangle for a one-triangle scene
    int slot;  // wide node index to write
};

__device__ __forceinline__ void entry_of(int c, const int2* range, const float4* nlo, const float4* nhi,
                                         const float4* llo, const float4* lhi, Entry& e)
{
    float4 a, b;
    e.ref = c;
    if (c < 0) {
        e.first = ~c;
        e.count = 1;
        a = llo[~c];
        b = lhi[~c];
    } else {
        int2 r = range[c];
        e.first = r.x;
        e.count = r.y - r.x + 1;
        a = nlo[c];
        b = nhi[c];
    }
    e.lo[0] = a.x; e.lo[1] = a.y; e.lo[2] = a.z;
    e.hi[0] = b.x; e.hi[1] = b.y; e.hi[2] = b.z;
}

__device__ __forceinline__ bool is_inner(const Entry& e) { return e.ref >= 0 && e.count > kLeafMax; }

__device__ __forceinline__ float half_area(const Entry& e)
{
    float dx = e.hi[0] - e.lo[0], dy = e.hi[1] - e.lo[1], dz = e.hi[2] - e.lo[2];
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_collapse(const Item* items, unsigned n_items, const int2* child, const int2* range,
                           const float4* nlo, const float4* nhi, const float4* llo, const float4* lhi,
                           const float4* tris, float pad, Item* next, unsigned* next_count, unsigned* node_counter,
                           unsigned* tri_counter, WNode* wn, float4* wtris, unsigned max_nodes, unsigned n_tris,
                           int* error)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const Item it = items[i];
    Entry E[8];
    int ne = 0;
    if (it.bin >= 0) {
        const int2 c = child[it.bin];
        entry_of(c.x, range, nlo, nhi, llo, lhi, E[0]);
        entry_of(c.y, range, nlo, nhi, llo, lhi, E[1]);
        ne = 2;
    } else {
        entry_of(it.bin, range, nlo, nhi, llo, lhi, E[0]);
        ne = 1;
    }
    // open the largest inner child until 8 children
    while (ne < 8) {
        int best = -1;
        float best_a = -1.f;
        for (int j = 0; j < ne; ++j)
            if (is_inner(E[j])) {
                float a = half_area(E[j]);
                if (a > best_a) { best_a = a; best = j; }
            }
        if (best < 0) break;
        const int2 c = child[E[best].ref];
        Entry a, b;
        entry_of(c.x, range, nlo, nhi, llo, lhi, a);
        entry_of(c.y, range, nlo, nhi, llo, lhi, b);
        E[best] = a;
        E[ne++] = b;
    }
    // padded child boxes, node box
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < ne; ++j)
        for (int k = 0; k < 3; ++k) {
            E[j].lo[k] -= pad;
            E[j].hi[k] += pad;
            lo[k] = fminf(lo[k], E[j].lo[k]);
            hi[k] = fmaxf(hi[k], E[j].hi[k]);
        }
    // octant slots: children far from the centre choose first
    int slot_of[8];
    unsigned used = 0;
    float m[3] = {0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2])};
    float dist[8];
    for (int j = 0; j < ne; ++j) {
        float d = 0.f;
        for (int k = 0; k < 3; ++k) {
            float c = 0.5f * (E[j].lo[k] + E[j].hi[k]) - m[k];
            d += c * c;
        }
        dist[j] = d;
    }
    bool placed[8] = {false, false, false, false, false, false, false, false};
    for (int round = 0; round < ne; ++round) {
        int j = -1;
        for (int q = 0; q < ne; ++q)
            if (!placed[q] && (j < 0 || dist[q] > dist[j])) j = q;
        placed[j] = true;
        float c[3];
        for (int k = 0; k < 3; ++k) c[k] = 0.5f * (E[j].lo[k] + E[j].hi[k]) - m[k];
        int bs = -1;
        float bv = -INFINITY;
        for (int s = 0; s < 8; ++s) {
            if (used & (1u << s)) continue;
            float v = ((s & 1) ? c[0] : -c[0]) + ((s & 2) ? c[1] : -c[1]) + ((s & 4) ? c[2] : -c[2]);
            if (v > bv) { bv = v; bs = s; }
        }
        used |= 1u << bs;
        slot_of[j] = bs;
    }
    // storage
    int n_inner = 0, n_leaf_tris = 0;
    for (int j = 0; j < ne; ++j) {
        if (is_inner(E[j])) ++n_inner;
        else n_leaf_tris += E[j].count;
    }
    const unsigned cb = n_inner ? atomicAdd(node_counter, (unsigned)n_inner) : 0u;
    const unsigned tb = n_leaf_tris ? atomicAdd(tri_counter, (unsigned)n_leaf_tris) : 0u;
    if (cb + n_inner > max_nodes || tb + n_leaf_tris > n_tris) {
        atomicExch(error, 1);
        return;
    }
    // per-axis power-of-two scale with (hi - lo) / scale <= 255
    unsigned ebits[3];
    float scale[3];
    for (int k = 0; k < 3; ++k) {
        float sc = (hi[k] - lo[k]) / 255.f;
        int e = -126;
        if (sc > 0.f) {
            int ee;
            frexpf(sc, &ee);  // sc = f * 2^ee, f in [0.5, 1): 2^ee >= sc
            e = ee;
        }
        e = max(-126, min(e, 127));
        ebits[k] = (unsigned)(e + 127);
        scale[k] = __int_as_float((int)(ebits[k] << 23));
    }
    unsigned char qlo[3][8], qhi[3][8], meta[8];
    for (int s = 0; s < 8; ++s) {
        meta[s] = 0;
        for (int k = 0; k < 3; ++k) { qlo[k][s] = 255; qhi[k][s] = 0; }  // empty slot: inverted box
    }
    unsigned imask = 0;
    int toff = 0;
    for (int j = 0; j < ne; ++j) {
        const int s = slot_of[j];
        for (int k = 0; k < 3; ++k) {
            float a = floorf((E[j].lo[k] - lo[k]) / scale[k]);
            float b = ceilf((E[j].hi[k] - lo[k]) / scale[k]);
            qlo[k][s] = (unsigned char)fminf(fmaxf(a, 0.f), 255.f);
            qhi[k][s] = (unsigned char)fminf(fmaxf(b, 0.f), 255.f);
        }
        if (is_inner(E[j])) {
            imask |= 1u << s;
        } else {
            meta[s] = (unsigned char)((E[j].count << 5) | toff);
            for (int q = 0; q < E[j].count; ++q)
                for (int v = 0; v < 3; ++v)
                    wtris[3 * (size_t)(tb + toff + q) + v] = tris[3 * (size_t)(E[j].first + q) + v];
            toff += E[j].count;
        }
    }
    // inner children: wide index = first child + number of inner children in lower slots
    for (int j = 0; j < ne; ++j)
        if (is_inner(E[j])) {
            const int s = slot_of[j];
            const unsigned w = cb + __popc(imask & ((1u << s) - 1u));
            const unsigned k = atomicAdd(next_count, 1u);
            next[k].bin = E[j].ref;
            next[k].slot = (int)w;
        }
    auto pack4 = [](const unsigned char* b) {
        return (unsigned)b[0] | ((unsigned)b[1] << 8) | ((unsigned)b[2] << 16) | ((unsigned)b[3] << 24);
    };
    WNode n;
    n.a = make_float4(lo[0], lo[1], lo[2], __uint_as_float(ebits[0] | (ebits[1] << 8) | (ebits[2] << 16) | (imask << 24)));
    n.b = make_uint4(cb, tb, pack4(meta), pack4(meta + 4));
    n.q0 = make_uint4(pack4(qlo[0]), pack4(qlo[0] + 4), pack4(qlo[1]), pack4(qlo[1] + 4));
    n.q1 = make_uint4(pack4(qlo[2]), pack4(qlo[2] + 4), pack4(qhi[0]), pack4(qhi[0] + 4));
    n.q2 = make_uint4(pack4(qhi[1]), pack4(qhi[1] + 4), pack4(qhi[2]), pack4(qhi[2] + 4));
    wn[it.slot] = n;
}

struct Buf {
    void* p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
};

}  // namespace

rt_status rt_build_wide(rt_scene* sc, const int2* child, const int2* range, const float4* node_lo,
                        const float4* node_hi, const float4* leaf_lo, const float4* leaf_hi, float pad,
                        cudaStream_t s)
{
    const int64_t nt = sc->n_tris;
    const unsigned max_nodes = (unsigned)(nt > 1 ? nt : 1);
    RT_CUDA_TRY(cudaMalloc(&sc->wnodes, (size_t)max_nodes * sizeof(WNode)));
    RT_CUDA_TRY(cudaMalloc(&sc->wtris, (size_t)nt * 3 * sizeof(float4)));
    Buf items[2], ctr;
    RT_CUDA_TRY(cudaMalloc(&items[0].p, (size_t)max_nodes * sizeof(Item)));
    RT_CUDA_TRY(cudaMalloc(&items[1].p, (size_t)max_nodes * sizeof(Item)));
    RT_CUDA_TRY(cudaMalloc(&ctr.p, 4 * sizeof(unsigned)));
    unsigned* c = static_cast<unsigned*>(ctr.p);  // [0] nodes, [1] triangles, [2] next count, [3] error
    const unsigned init[4] = {1u, 0u, 0u, 0u};
    RT_CUDA_TRY(cudaMemcpyAsync(c, init, sizeof(init), cudaMemcpyHostToDevice, s));
    Item root = {nt > 1 ? 0 : ~0, 0};
    RT_CUDA_TRY(cudaMemcpyAsync(items[0].p, &root, sizeof(Item), cudaMemcpyHostToDevice, s));
    unsigned n_items = 1;
    int level = 0;
    for (; n_items > 0; ++level) {
        if (level > 256) return rt_fail(RT_ERR_DEVICE_LIMIT, "wide BVH collapse did not terminate");
        RT_CUDA_TRY(cudaMemsetAsync(c + 2, 0, sizeof(unsigned), s));
        k_collapse<<<(n_items + kBlock - 1) / kBlock, kBlock, 0, s>>>(
            static_cast<const Item*>(items[level & 1].p), n_items, child, range, node_lo, node_hi, leaf_lo, leaf_hi,
            sc->tris, pad, static_cast<Item*>(items[(level + 1) & 1].p), c + 2, c, c + 1, sc->wnodes, sc->wtris,
            max_nodes, (unsigned)nt, reinterpret_cast<int*>(c + 3));
        RT_CUDA_TRY(cudaGetLastError());
        unsigned h[4];
        RT_CUDA_TRY(cudaMemcpyAsync(h, c, sizeof(h), cudaMemcpyDeviceToHost, s));
        RT_CUDA_TRY(cudaStreamSynchronize(s));
        if (h[3]) return rt_fail(RT_ERR_DEVICE_LIMIT, "wide BVH collapse ran out of node or triangle slots");
        n_items = h[2];
        sc->n_wnodes = h[0];
        if (n_items == 0 && h[1] != (unsigned)nt)
            return rt_fail(RT_ERR_DEVICE_LIMIT, "wide BVH holds %u of %lld triangles", h[1], (long long)nt);
    }
    sc->wide_depth = level;
    sc->bytes += (int64_t)sc->n_wnodes * (int64_t)sizeof(WNode) + nt * 3 * (int64_t)sizeof(float4);
    if (level > RT_WSTACK_DEPTH) {  // deeper than the traversal stack: keep the binary tree only
        cudaFree(sc->wnodes);
        cudaFree(sc->wtris);
        sc->wnodes = nullptr;
        sc->wtris = nullptr;
    }
    return RT_OK;
}
