// Treelet restructuring of the LBVH (Karras & Aila, "Fast Parallel
// Construction of High-Quality Bounding Volume Hierarchies", HPG 2013).
//
// The Morton-code hierarchy is fast to build but its splits ignore the
// surface-area cost that decides how many nodes a ray visits.  Each pass walks
// the tree bottom-up (one thread per leaf, a counter per node: the second
// thread to arrive continues), and every node reached this way becomes the
// root of a treelet: its leaves are found by repeatedly expanding the treelet
// leaf of largest surface area, up to 7 of them, and the binary topology over
// those leaves of least surface-area cost,
//     c(S) = C_node A(S) + min over splits S = P + (S \ P) of c(P) + c(S \ P),
// is found by dynamic programming over the 127 subsets, one warp per treelet.
// When it is cheaper the treelet is rewired with its own internal nodes.  The
// leaves are finally renumbered in depth-first order so that every subtree's
// triangles are contiguous again (the 8-wide collapse relies on that).
#include "rt_internal.cuh"

namespace {

constexpr int kBlock = 128;             // 4 warps, each with its own shared treelet workspace
constexpr int kWarps = kBlock / 32;
constexpr int kTreelet = 7;             // treelet leaves
constexpr int kSubsets = 1 << kTreelet;
constexpr float kCostNode = 1.2f;       // surface-area cost of visiting a node ...
constexpr float kCostTri = 1.0f;        // ... and of testing a triangle
constexpr int kMaxWalk = 256;

__device__ __forceinline__ float half_area(float4 lo, float4 hi)
{
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

struct Tree {
    int2* child;
    int32_t* par_i;     // parent of an internal node (-1 for the root)
    int32_t* par_l;     // parent of a leaf
    const float4* llo;
    const float4* lhi;
    float4* nlo;
    float4* nhi;
    float* cost;        // surface-area cost of every internal node's subtree
    int* visit;
    int64_t n_leaves;
};

__device__ __forceinline__ float4 ref_lo(const Tree& T, int r) { return r < 0 ? __ldcg(T.llo + ~r) : __ldcg(T.nlo + r); }
__device__ __forceinline__ float4 ref_hi(const Tree& T, int r) { return r < 0 ? __ldcg(T.lhi + ~r) : __ldcg(T.nhi + r); }
__device__ __forceinline__ float ref_cost(const Tree& T, int r)
{
    return r < 0 ? kCostTri * half_area(ref_lo(T, r), ref_hi(T, r)) : __ldcg(T.cost + r);
}

// initial subtree costs, bottom-up
__global__ void k_cost(Tree T)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T.n_leaves) return;
    int32_t node = T.par_l[k];
    for (int guard = 0; node >= 0 && guard < kMaxWalk; ++guard) {
        if (atomicAdd(&T.visit[node], 1) == 0) return;
        __threadfence();
        const int2 c = __ldcg(T.child + node);
        T.cost[node] = kCostNode * half_area(__ldcg(T.nlo + node), __ldcg(T.nhi + node)) + ref_cost(T, c.x) +
                       ref_cost(T, c.y);
        __threadfence();
        node = T.par_i[node];
    }
}

struct Workspace {
    int leaf[kTreelet];          // treelet leaves (node or ~leaf references)
    int inner[kTreelet - 1];     // the treelet's internal nodes, root first
    float4 lo[kTreelet], hi[kTreelet];
    float area[kSubsets];
    float copt[kSubsets];
    unsigned char part[kSubsets];
    int n;
};

// the whole warp optimises the treelet rooted at `root`
__device__ void optimise_treelet(const Tree& T, int root, Workspace& w)
{
    const unsigned lane = threadIdx.x & 31u;
    if (lane == 0) {
        // grow the treelet: expand the leaf of largest area that is an internal node
        const int2 c = __ldcg(T.child + root);
        w.leaf[0] = c.x;
        w.leaf[1] = c.y;
        w.inner[0] = root;
        int n = 2;
        while (n < kTreelet) {
            int best = -1;
            float ba = -1.f;
            for (int i = 0; i < n; ++i) {
                if (w.leaf[i] < 0) continue;
                const float a = half_area(ref_lo(T, w.leaf[i]), ref_hi(T, w.leaf[i]));
                if (a > ba) { ba = a; best = i; }
            }
            if (best < 0) break;
            const int node = w.leaf[best];
            const int2 cc = __ldcg(T.child + node);
            w.inner[n - 1] = node;
            w.leaf[best] = cc.x;
            w.leaf[n] = cc.y;
            ++n;
        }
        w.n = n;
        for (int i = 0; i < n; ++i) {
            w.lo[i] = ref_lo(T, w.leaf[i]);
            w.hi[i] = ref_hi(T, w.leaf[i]);
        }
    }
    __syncwarp();
    const int n = w.n;
    const int full = (1 << n) - 1;
    // areas of all subsets, leaf costs
    for (int S = 1 + (int)lane; S <= full; S += 32) {
        float4 lo = make_float4(3.4e38f, 3.4e38f, 3.4e38f, 0.f), hi = make_float4(-3.4e38f, -3.4e38f, -3.4e38f, 0.f);
        for (int i = 0; i < n; ++i) {
            if (!(S & (1 << i))) continue;
            lo = make_float4(fminf(lo.x, w.lo[i].x), fminf(lo.y, w.lo[i].y), fminf(lo.z, w.lo[i].z), 0.f);
            hi = make_float4(fmaxf(hi.x, w.hi[i].x), fmaxf(hi.y, w.hi[i].y), fmaxf(hi.z, w.hi[i].z), 0.f);
        }
        w.area[S] = half_area(lo, hi);
        if (__popc(S) == 1) w.copt[S] = ref_cost(T, w.leaf[__ffs(S) - 1]);
    }
    __syncwarp();
    // subsets by size: the best split of each
    for (int size = 2; size <= n; ++size) {
        for (int S = 1 + (int)lane; S <= full; S += 32) {
            if (__popc(S) != size) continue;
            const int low = S & -S, rest = S ^ low;
            float best = 3.4e38f;
            int bp = low;
            // P holds the lowest leaf of S, so every split is seen once
            for (int sub = rest;; sub = (sub - 1) & rest) {
                const int P = low | sub;
                if (P != S) {
                    const float c = w.copt[P] + w.copt[S ^ P];
                    if (c < best) { best = c; bp = P; }
                }
                if (sub == 0) break;
            }
            w.copt[S] = kCostNode * w.area[S] + best;
            w.part[S] = (unsigned char)bp;
        }
        __syncwarp();
    }
    if (lane == 0 && n >= 3 && w.copt[full] < __ldcg(T.cost + root) * (1.f - 1e-6f)) {
        // rewire: internal nodes in the order they are assigned (parents first)
        int stack_set[kTreelet], stack_node[kTreelet], order[kTreelet - 1];
        int sp = 0, next = 1, m = 0;
        stack_set[sp] = full;
        stack_node[sp++] = root;
        while (sp > 0) {
            --sp;
            const int S = stack_set[sp], node = stack_node[sp];
            order[m++] = node;
            const int P = w.part[S], Q = S ^ P;
            int ref[2];
            const int sets[2] = {P, Q};
            for (int side = 0; side < 2; ++side) {
                const int X = sets[side];
                if (__popc(X) == 1) {
                    ref[side] = w.leaf[__ffs(X) - 1];
                } else {
                    ref[side] = w.inner[next++];
                    stack_set[sp] = X;
                    stack_node[sp++] = ref[side];
                }
                if (ref[side] < 0) T.par_l[~ref[side]] = node;
                else T.par_i[ref[side]] = node;
            }
            T.child[node] = make_int2(ref[0], ref[1]);
        }
        // boxes and costs, children before parents
        for (int i = m - 1; i >= 0; --i) {
            const int node = order[i];
            const int2 c = __ldcg(T.child + node);
            const float4 l0 = ref_lo(T, c.x), h0 = ref_hi(T, c.x), l1 = ref_lo(T, c.y), h1 = ref_hi(T, c.y);
            const float4 lo = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
            const float4 hi = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
            T.nlo[node] = lo;
            T.nhi[node] = hi;
            T.cost[node] = kCostNode * half_area(lo, hi) + ref_cost(T, c.x) + ref_cost(T, c.y);
        }
        __threadfence();
    }
    __syncwarp();
}

// one restructuring pass: leaves walk up; each node whose second child finished
// is optimised by the warp of the thread that finished it
__global__ void __launch_bounds__(kBlock) k_treelets(Tree T)
{
    __shared__ Workspace ws[kWarps];
    Workspace& w = ws[threadIdx.x / 32];
    const unsigned lane = threadIdx.x & 31u;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t node = k < T.n_leaves ? T.par_l[k] : -1;
    bool active = node >= 0;
    for (int guard = 0; guard < kMaxWalk; ++guard) {
        bool ready = false;
        if (active) {
            if (atomicAdd(&T.visit[node], 1) == 0) active = false;  // the sibling subtree is not finished
            else ready = true;
        }
        if (ready) __threadfence();
        unsigned todo = __ballot_sync(0xffffffffu, ready);
        if (todo == 0 && __ballot_sync(0xffffffffu, active) == 0) break;
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int root = __shfl_sync(0xffffffffu, node, src);
            optimise_treelet(T, root, w);
        }
        if (ready) {
            node = __ldcg(T.par_i + node);
            active = node >= 0;
        }
    }
    (void)lane;
}

// leaves (and internal nodes) in depth-first order: the position of a node's
// first leaf is the number of leaves left of its path from the root
__global__ void k_counts(const int2* child, const int32_t* par_i, const int32_t* par_l, int64_t n_leaves, int* count,
                         int* visit)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_leaves) return;
    int32_t node = par_l[k];
    for (int guard = 0; node >= 0 && guard < kMaxWalk; ++guard) {
        if (atomicAdd(&visit[node], 1) == 0) return;
        __threadfence();
        const int2 c = child[node];
        count[node] = (c.x < 0 ? 1 : __ldcg(count + c.x)) + (c.y < 0 ? 1 : __ldcg(count + c.y));
        __threadfence();
        node = par_i[node];
    }
}

__device__ __forceinline__ int first_leaf(const int2* child, const int32_t* par_i, const int* count, int32_t self,
                                          int32_t parent)
{
    int pos = 0;
    for (int guard = 0; parent >= 0 && guard < kMaxWalk; ++guard) {
        const int2 c = child[parent];
        if (c.y == self) pos += c.x < 0 ? 1 : count[c.x];
        self = parent;
        parent = par_i[parent];
    }
    return pos;
}

__global__ void k_leaf_position(const int2* child, const int32_t* par_i, const int32_t* par_l, const int* count,
                                int64_t n_leaves, int32_t* pos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_leaves) return;
    pos[k] = first_leaf(child, par_i, count, ~(int32_t)k, par_l[k]);
}

__global__ void k_node_range(const int2* child, const int32_t* par_i, const int* count, int64_t n_int, int2* range)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const int first = first_leaf(child, par_i, count, (int32_t)i, par_i[i]);
    range[i] = make_int2(first, first + count[i] - 1);
}

// leaf k moves to position pos[k]: the triangle order, leaf boxes and references follow
__global__ void k_permute_leaves(const int32_t* pos, int64_t n_leaves, const int32_t* order, const float4* llo,
                                 const float4* lhi, int32_t* order2, float4* llo2, float4* lhi2, int32_t* par_l2,
                                 const int32_t* par_l)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_leaves) return;
    const int32_t p = pos[k];
    order2[p] = order[k];
    llo2[p] = llo[k];
    lhi2[p] = lhi[k];
    par_l2[p] = par_l[k];
}

__global__ void k_remap_children(int2* child, int64_t n_int, const int32_t* pos)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int2 c = child[i];
    if (c.x < 0) c.x = ~pos[~c.x];
    if (c.y < 0) c.y = ~pos[~c.y];
    child[i] = c;
}

unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace

rt_status rt_treelet_optimise(int64_t nt, int passes, int2* child, int2* range, int32_t* par_i, int32_t* par_l,
                              int32_t* order, float4* llo, float4* lhi, float4* nlo, float4* nhi, cudaStream_t s)
{
    if (nt < 3 || passes <= 0) return RT_OK;
    const int64_t ni = nt - 1;
    float* cost = nullptr;
    int* visit = nullptr;
    int* count = nullptr;
    int32_t* pos = nullptr;
    int32_t* order2 = nullptr;
    int32_t* par_l2 = nullptr;
    float4* llo2 = nullptr;
    float4* lhi2 = nullptr;
    rt_status st = RT_OK;
    cudaError_t e = cudaSuccess;
#define TRY_ALLOC(p, bytes) \
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&(p), (size_t)(bytes), s)
    TRY_ALLOC(cost, ni * sizeof(float));
    TRY_ALLOC(visit, ni * sizeof(int));
    TRY_ALLOC(count, ni * sizeof(int));
    TRY_ALLOC(pos, nt * sizeof(int32_t));
    TRY_ALLOC(order2, nt * sizeof(int32_t));
    TRY_ALLOC(par_l2, nt * sizeof(int32_t));
    TRY_ALLOC(llo2, nt * sizeof(float4));
    TRY_ALLOC(lhi2, nt * sizeof(float4));
#undef TRY_ALLOC
    if (e != cudaSuccess) st = rt_cuda_fail(e, "cudaMallocAsync");
    Tree T = {child, par_i, par_l, llo, lhi, nlo, nhi, cost, visit, nt};
    if (st == RT_OK) {
        e = cudaMemsetAsync(visit, 0, ni * sizeof(int), s);
        if (e == cudaSuccess) k_cost<<<grid_for(nt), kBlock, 0, s>>>(T);
        for (int pass = 0; pass < passes && e == cudaSuccess; ++pass) {
            e = cudaMemsetAsync(visit, 0, ni * sizeof(int), s);
            if (e == cudaSuccess) k_treelets<<<grid_for(nt), kBlock, 0, s>>>(T);
        }
        // depth-first leaf order
        if (e == cudaSuccess) e = cudaMemsetAsync(visit, 0, ni * sizeof(int), s);
        if (e == cudaSuccess) {
            k_counts<<<grid_for(nt), kBlock, 0, s>>>(child, par_i, par_l, nt, count, visit);
            k_leaf_position<<<grid_for(nt), kBlock, 0, s>>>(child, par_i, par_l, count, nt, pos);
            k_node_range<<<grid_for(ni), kBlock, 0, s>>>(child, par_i, count, ni, range);
            k_permute_leaves<<<grid_for(nt), kBlock, 0, s>>>(pos, nt, order, llo, lhi, order2, llo2, lhi2, par_l2,
                                                             par_l);
            k_remap_children<<<grid_for(ni), kBlock, 0, s>>>(child, ni, pos);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(order, order2, nt * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(par_l, par_l2, nt * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(llo, llo2, nt * sizeof(float4), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lhi, lhi2, nt * sizeof(float4), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = rt_cuda_fail(e, "treelet restructuring");
    }
    cudaFreeAsync(cost, s);
    cudaFreeAsync(visit, s);
    cudaFreeAsync(count, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(order2, s);
    cudaFreeAsync(par_l2, s);
    cudaFreeAsync(llo2, s);
    cudaFreeAsync(lhi2, s);
    return st;
}
