// Internal data layout and device helpers of the combined ray query library.
//
// HBM layout (built once per scene / per grid):
//   nodes  : n_tris-1 internal BVH nodes, 64 B each, read as two 32-byte loads:
//              a = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//              b = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//              c = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//              d = (child0, child1, -, -)   child >= 0: internal node,
//                                           child < 0 : leaf = triangle ~child
//   tris   : 48 B per triangle in leaf (Morton) order: v0.xyz|prim, v1.xyz|-, v2.xyz|-
//   wnodes : the same tree collapsed to 8-wide nodes of 80 B (five 16-byte vectors):
//              a  = (origin x, y, z, bits: exponent x | y << 8 | z << 16 | internal mask << 24)
//              b  = (first child node, first triangle, meta slots 0-3, meta slots 4-7)
//              q0 = (qlo.x[0..7], qlo.y[0..7]), q1 = (qlo.z[0..7], qhi.x[0..7]),
//              q2 = (qhi.y[0..7], qhi.z[0..7])   8-bit child bounds, box = origin + q * 2^(e-127)
//            meta byte: 0 empty, else leaf (count << 5 | first triangle offset) or, with the
//            internal-mask bit set, an inner child at first child + (inner children in lower slots)
//   wtris  : 48 B per triangle in wide-leaf order (each node's leaf triangles contiguous)
//   pn     : 112 B per triangle in leaf order: face normal, 3 edge and 3 vertex
//            pseudonormals (float4 each), read only by the distance bake
//   slot   : 4 B per triangle: input index -> leaf-order position (field build)
//   grid   : caller memory, dense n0*n1*n2 float32 or float16, x fastest
//   cells  : optional library copy of the grid with the 8 corners of every cell
//            stored together (32 B float32 / 16 B float16 per cell, cells x
//            fastest), so one march step is one vector load instead of eight
//            scalar ones; identical values, identical arithmetic
//   pairs  : optional library copy with the two x-neighbours (i, i+1) of every
//            sample stored together (8 B float32 / 4 B float16, (n0-1) x n1 x n2,
//            x fastest): a march step is four small loads from a copy twice the
//            grid's size, small enough to stay in L2 where the cell copy is not
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/rt_api.h"

#define RT_STACK_DEPTH 64

struct __align__(32) BNode {
    float4 a, b, c;
    int4 d;
};

struct __align__(16) WNode {
    float4 a;
    uint4 b, q0, q1, q2;
};

#define RT_WSTACK_DEPTH 32

struct rt_scene {
    int device;
    int64_t n_tris, n_verts, n_nodes;
    int32_t max_depth;
    BNode* nodes;
    float4* tris;   // 3 per triangle
    float4* pn;     // 7 per triangle
    int32_t* slot;  // input triangle index -> position in leaf order
    WNode* wnodes;  // null when the wide tree is not available
    float4* wtris;  // 3 per triangle
    int64_t n_wnodes;
    int32_t wide_depth;
    float lo[3], hi[3];
    int64_t bytes;
};

struct rt_sdf {
    const void* grid;
    int32_t dtype;
    float lo[3], hi[3], h[3], ih[3];  // one grid; on a cascade: the coarsest level's box
    int32_t n[3];
    void* cells;        // library-owned cell-corner copy (null until rt_sdf_prepare)
    int64_t cells_bytes;
    void* pairs;        // library-owned x-pair copy (null until rt_sdf_prepare)
    int64_t pairs_bytes;
    int device;
    // cascade (levels > 0): level k holds n^3 samples at (ilo[k] + i) * h0 * 2^k,
    // stored at grid + k * n^3, its cells at cells + k * (n-1)^3
    int32_t levels;
    float h0;
    int32_t ilo[RT_MAX_LEVELS][3];
    void* scratch;      // one level, for rt_cascade_recenter
    int64_t scratch_bytes;
    int32_t bake_method;  // method of the last rt_sdf_bake (RT_BAKE_JFA: sites kept)
    int32_t* sites;       // finished site of every sample after a field build (RT_BAKE_JFA): the
                          // seeds of finer levels when a rolling update rebuilds them
    int64_t sites_count;
};

// geometry of cascade level k as the queries see it (float, rounded once each)
struct CascLevel {
    float lo[3], hi[3];
    float ih, h, eps_hit, eps_min;
};

// Query order (rt_tuning.order_bits): each window of consecutive queries
// stably sorted by the cell of a 2^bits lattice over the box
// lo + [0, 2^bits / scale] that holds the query's origin (rt_order.cu).
// bits = 0, or fewer than kOrderMin queries: no ordering.
struct OrderBox {
    float lo[3], scale[3];
    int32_t bits;
};
constexpr int32_t kOrderMaxBits = 5;
constexpr int64_t kOrderMin = 64;

// The query order is applied where it was measured to pay: to queries whose
// first sub-interval is the near triangle one (closest hit, a split with
// 0 < m_near < inf).  Triangles-only, field-only and any-hit calls start with
// a kernel whose time the order does not change, and pay only its cost.
inline bool rt_order_applies(const rt_split_params& p)
{
    return (p.mode == RT_MODE_SPLIT1 || p.mode == RT_MODE_SPLIT2) && p.any_hit == 0 && p.m_near > 0.f &&
           !isinf(p.m_near);
}

// Everything one trace kernel needs, passed by value.
struct TraceArgs {
    const BNode* nodes;
    const float4* tris;
    const WNode* wnodes;  // null: binary traversal
    const float4* wtris;
    int32_t root;        // 0 (internal), ~0 (single leaf) or INT32_MIN (no triangles)
    const void* grid;    // null: no field
    const void* cells;   // null: read the plain grid (or the pairs)
    const void* pairs;   // null: no x-pair copy
    int32_t grid_f16;
    float glo[3], ghi[3], gih[3];
    int32_t gn[3];
    float hsplit, eps_hit, eps_min;
    int32_t max_steps;
    int32_t mode, any_hit, refine_root;
    float m_near, m_far;
    int32_t levels;        // 0: one grid; > 0: a cascade read through its cell copy
    int64_t level_cells;   // cells per cascade level
    CascLevel lv[RT_MAX_LEVELS];
    const float4* rays;
    rt_hit* hits;
    int64_t n;
    unsigned long long* counters;
    OrderBox ob;             // ob.bits = 0: queries in input order
    const int32_t* qorder;   // null: input order; else the first kernel's slot i traces query qorder[i]
};

// ---------------------------------------------------------------------------
// host-side error reporting (rt_api.cu)
// ---------------------------------------------------------------------------
rt_status rt_fail(rt_status s, const char* fmt, ...);
rt_status rt_cuda_fail(cudaError_t e, const char* what);
#define RT_CUDA_TRY(expr)                                         \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return rt_cuda_fail(_e, #expr);    \
    } while (0)

const rt_tuning& rt_current_tuning();

// which grid copy the march reads under a tuning: the cell copy, the x-pair copy
// or the plain grid (a copy is used only if rt_sdf_prepare has built it)
inline void rt_apply_layout(TraceArgs& a, const rt_tuning& tu)
{
    if (a.levels > 0) {  // a cascade has only its cell copy
        a.pairs = nullptr;
        return;
    }
    if (tu.grid_layout != RT_LAYOUT_CELLS) a.cells = nullptr;
    if (tu.grid_layout != RT_LAYOUT_PAIRS) a.pairs = nullptr;
}

// launchers implemented in the .cu files
// timing: when non-null, events[k] is recorded before launch k and events[n] after
// the last; kinds[k] receives the RT_STAGE_* of launch k; *n_launches the count
// Timed parts of one call (rt_trace_combined_timed): part k ran between
// events[2k] and events[2k+1], recorded on the stream that ran it.
constexpr int kMaxTimedParts = 6;
struct StageTiming {
    cudaEvent_t events[2 * kMaxTimedParts];
    int32_t kinds[kMaxTimedParts];
    int32_t n_launches;
};

// The queries' ray arrays as one index space: query g lies in segment b, the
// last with offset[b] <= g, at rays[b] + 2 (g - offset[b]).
struct OrderRays {
    const float4* rays[RT_MAX_BATCHES];
    int64_t offset[RT_MAX_BATCHES];
    int32_t count;
};
// Scratch bytes of the query order of n queries (a multiple of 256; 0 when
// there is nothing to order).
size_t rt_order_bytes(const OrderBox& ob, int64_t n);
// Order queries 0..n-1 of a (rt_order.cu) into `scratch` (rt_order_bytes,
// 256-byte aligned); on success a.qorder points into it.  Enqueued on s.
rt_status rt_launch_order(TraceArgs& a, const OrderRays& src, void* scratch, cudaStream_t s);
// The concurrent programs (rt_trace.cu for one call, rt_batch.cu for mixed
// batches): closest-hit near triangle sub-intervals run beside the field
// sub-intervals, which start at t_1 without waiting for the near result.  The
// near stage lists its hits; afterwards k_merge_hits writes each over the
// record the later stages left (a near hit lies before t_1, so it is the
// closest, Section 2).  A near miss that raised flags lists an entry with prim
// kFlagsOnly, whose flags are ORed into the record.
constexpr int32_t kFlagsOnly = -2;
struct HitEntry {
    rt_hit* dst;  // the query's record
    uint32_t flags;
    float t, u, v;
    int32_t prim;
    int32_t pad;
};
static_assert(sizeof(HitEntry) == 32, "one 32-byte entry per hit");
// Two library streams per device for the concurrent programs: near (highest
// priority) and field (lowest), with the events that fork and join them.
// Callers hold rt_conc_mutex() from the fork to the join.
struct ConcStreams {
    cudaStream_t near = nullptr, field = nullptr;
    cudaEvent_t fork = nullptr, ordered = nullptr, near_done = nullptr, field_done = nullptr;
    bool ready = false;
};
std::mutex& rt_conc_mutex();
rt_status rt_conc_streams(ConcStreams*& out);
// k_merge_hits over the *count entries of list, on s
rt_status rt_launch_merge_hits(const HitEntry* list, const unsigned* count, int sms, cudaStream_t s);
// Resident blocks of 128 threads per SM of the two concurrent stages when the
// tuning leaves them free.  Both kernels are persistent, so their blocks must
// fit in an SM side by side (registers: near 2 x 128 x 56 (64 for the batch
// kernel) + field 9 x 128 x 40, at most 62,464 of 65,536), or the later launch
// waits for the earlier one's end.  Measured on the 1080p GI workload, whole
// call: near 2 + field 9 0.595 ms, 3 + 9 0.608, 2 + 10 0.603, 2 + 8 0.611,
// 4 + 7 0.661, 1 + 11 1.015; the stages in sequence 0.662.
#ifndef RT_CONC_NEAR_BLOCKS
#define RT_CONC_NEAR_BLOCKS 2
#endif
#ifndef RT_CONC_FIELD_BLOCKS
#define RT_CONC_FIELD_BLOCKS 9
#endif
constexpr int kConcNearBlocks = RT_CONC_NEAR_BLOCKS;
constexpr int kConcFieldBlocks = RT_CONC_FIELD_BLOCKS;

// allow_concurrent = false: the stages of a closest-hit split call run in
// sequence on s (no internal streams), as the pieces of rt_trace_combined_host need
rt_status rt_launch_trace(const TraceArgs& a, bool counted, cudaStream_t s, StageTiming* timing = nullptr,
                          bool allow_concurrent = true);
rt_status rt_launch_backward(const TraceArgs& a, const float* grad_t, float* grad_grid, cudaStream_t s);
rt_status rt_build_scene(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, cudaStream_t s,
                         rt_scene* out);
rt_status rt_launch_bake(const rt_scene* sc, const rt_sdf* sdf, int32_t method, cudaStream_t s);
rt_status rt_build_wide(rt_scene* sc, const int2* child, const int2* range, const float4* node_lo,
                        const float4* node_hi, const float4* leaf_lo, const float4* leaf_hi, float pad,
                        cudaStream_t s);
rt_status rt_launch_prepare(rt_sdf* sdf, cudaStream_t s);
rt_status rt_treelet_optimise(int64_t nt, int passes, int2* child, int2* range, int32_t* par_i, int32_t* par_l,
                              int32_t* order, float4* llo, float4* lhi, float4* nlo, float4* nhi, cudaStream_t s);
rt_status rt_fill_trace_args(TraceArgs& a, const rt_scene* sc, const rt_sdf* sdf, const rt_split_params* p);
void rt_cascade_geometry(const rt_sdf* sdf, int k, float lo[3], float hi[3], float* h, float* ih);
rt_status rt_launch_cascade_bake(const rt_scene* sc, const rt_sdf* sdf, int k, int32_t method, const void* keep,
                                 const int32_t shift[3], cudaStream_t s);
rt_status rt_launch_cascade_cells(const rt_sdf* sdf, int k, cudaStream_t s);
rt_status rt_launch_df_sites(const rt_scene* sc, const rt_sdf* sdf, int32_t stage, int32_t* d_sites, cudaStream_t s);
rt_status rt_launch_df_levels(const rt_scene* sc, const rt_sdf* sdf, const int* lv, int nl, int32_t* jfa_store,
                              cudaStream_t s);
