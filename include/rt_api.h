/*
 * rt_api.h -- C interface of the GB300 (sm_103a) combined ray query library.
 *
 * The library answers ray queries (o, d, t_min, t_max, f) -- Eq. 1 of Bartels
 * & Harada, "Combining GPU Tracing Methods within a Single Ray Query"
 * (SIGGRAPH Asia 2022 Technical Communications) -- by splitting [t_min, t_max]
 * into mutually exclusive sub-intervals (Eq. 2) and tracing each one either
 * exactly against the triangles (BVH traversal with a watertight test) or
 * approximately through a dense signed distance field (sphere tracing).
 *
 * General rules for every entry point
 *   - All ray, hit and grid buffers are DEVICE memory owned by the caller,
 *     16-byte aligned.  Handles (rt_scene, rt_sdf) are owned by the library and
 *     released with the matching *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; argument errors are
 *     detected before anything is enqueued and returned synchronously.
 *   - Every call returns an rt_status.  On failure rt_last_error() gives a
 *     human-readable message (thread-local; valid until the next call on the
 *     same thread).
 *   - Device-side limits (traversal stack depth, march step budget) never
 *     abort a kernel: they set bits in rt_hit.flags.
 *   - Eq. 1 is defined for real numbers: a query with a NaN in o, d, t_min or
 *     t_max is answered with a miss.  t_min > t_max is an empty query (miss).
 *   - The library uses the current CUDA device of the calling thread; a handle
 *     must be used on the device it was created on.
 */
#ifndef GB300_RT_API_H
#define GB300_RT_API_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,    /* null pointer, negative size, misaligned buffer, bad mode */
    RT_ERR_CUDA = 2,           /* a CUDA runtime call failed (message has the CUDA error) */
    RT_ERR_OOM = 3,            /* device allocation failed */
    RT_ERR_DEVICE_LIMIT = 4,   /* a problem exceeds a device-side limit (e.g. tree depth) */
    RT_ERR_NOT_IMPLEMENTED = 5
} rt_status;

/* One query of Eq. 1: origin o, t_min, unit direction d, t_max.  32 bytes,
 * loaded as two 16-byte vectors.  The caller normalises d. */
typedef struct {
    float ox, oy, oz, tmin;
    float dx, dy, dz, tmax;
} rt_ray;

/* Result of one query.  24 bytes.
 *   t       hit distance along the ray (+inf on a miss)
 *   prim    triangle index in the mesh given to rt_scene_build; -1 for a miss
 *           or for a hit resolved by the distance field (the paper notes that
 *           surface information is not directly available from a distance
 *           field, Section 2 "Surface information")
 *   u, v    barycentric weights of the triangle's second and third vertex
 *           (hit = (1-u-v) v0 + u v1 + v v2); 0 for field hits
 *   tracer  RT_TRACER_* : which technique resolved the query
 *   flags   RT_FLAG_* */
typedef struct {
    float t;
    int32_t prim;
    float u, v;
    int32_t tracer;
    uint32_t flags;
} rt_hit;

enum { RT_TRACER_MISS = 0, RT_TRACER_BVH = 1, RT_TRACER_SDF = 2 };
enum {
    RT_FLAG_STACK_OVERFLOW = 1u, /* BVH traversal stack exhausted (result may miss a hit) */
    RT_FLAG_STEP_LIMIT = 2u,     /* distance-field march used all max_steps without hit or exit */
    RT_FLAG_ITER_LIMIT = 4u      /* traversal stopped by its iteration guard (corrupt structure) */
};

/* How [t_min, t_max] is split (Eq. 2) and processed (Section 2, after Eq. 2;
 * the split rules of Section 3).  h = largest edge of one grid voxel.
 *   mode 0  RT_MODE_BVH    : triangles on [t_min, t_max] (the pure technique)
 *   mode 1  RT_MODE_SPLIT1 : t_1 = clamp(t_min + m_near*h, t_min, t_max);
 *                            triangles on [t_min, t_1] (skipped if m_near == 0),
 *                            field on [t_1, t_max] (skipped if t_1 == t_max and
 *                            m_near > 0).  Section 3, occlusion queries and the
 *                            first GI pass.
 *   mode 2  RT_MODE_SPLIT2 : additionally t_2 = clamp(t_max - m_far*h, t_1, t_max);
 *                            triangles on [t_min, t_1] and [t_2, t_max] (each
 *                            skipped when its multiplier is 0), field on [t_1, t_2]
 *                            (skipped when empty, unless both multipliers are 0).
 *                            Section 3, shadow rays.
 *   mode 3  RT_MODE_SDF    : field on [t_min, t_max] (the pure technique)
 * any_hit = 0 (closest hit): sub-intervals in order, stop at the first that
 * hits.  any_hit = 1: field sub-interval first, then the triangle ones.
 * Triangle sub-intervals are closed: a hit exactly at t_1 belongs to them.
 * Multipliers may be +INFINITY; they must not be negative or NaN.
 * The field march (Section 1 names distance-field tracing; the step rule is
 * this library's): clip the sub-interval to the grid box, t = start; up to
 * max_steps times: phi = trilinear(o + t d); phi < hit_eps_vox*hmin -> hit at
 * t; t += max(phi, min_step_vox*hmin); t > end -> miss.  hmin = smallest voxel
 * edge.  refine_root = 1 replaces the hit t by the root of
 * phi = hit_eps_vox*hmin inside the last step (bisection, 24 halvings), the
 * point at which rt_trace_combined_backward differentiates. */
typedef struct {
    int32_t mode;
    int32_t any_hit;
    float m_near;
    float m_far;
    int32_t max_steps;
    float hit_eps_vox;
    float min_step_vox;
    int32_t refine_root;
} rt_split_params;

enum { RT_MODE_BVH = 0, RT_MODE_SPLIT1 = 1, RT_MODE_SPLIT2 = 2, RT_MODE_SDF = 3 };
enum { RT_GRID_F32 = 0, RT_GRID_F16 = 1 };
enum { RT_BAKE_AUTO = 0, RT_BAKE_BRUTE = 1, RT_BAKE_BVH = 2, RT_BAKE_JFA = 3 };

typedef struct rt_scene rt_scene;
typedef struct rt_sdf rt_sdf;

typedef struct {
    int64_t n_tris;
    int64_t n_verts;
    int64_t n_nodes;     /* internal BVH nodes (64 bytes each) */
    int32_t max_depth;   /* deepest leaf; traversal stack holds RT_STACK_DEPTH entries */
    int32_t stack_depth;
    int64_t n_wide_nodes;  /* 80-byte nodes of the 8-wide tree (0: not built) */
    int32_t wide_depth;    /* levels of the 8-wide tree */
    int32_t pad_;
    float lo[3], hi[3];  /* bounds of all triangles */
    int64_t device_bytes;
} rt_scene_info;

/* Build the triangle acceleration structure (a linear BVH from 63-bit Morton
 * codes of triangle centroids, hierarchy by Karras' split search, HPG 2012)
 * and the angle-weighted pseudonormals used by rt_sdf_bake.  The triangle
 * tracer stands in for the paper's hardware ray tracing (Section 3).
 *   d_verts  n_verts x 3 float32 (x,y,z), device
 *   d_tris   n_tris x 3 int32 vertex indices, device; winding gives the
 *            outward normal (counter-clockwise seen from outside)
 *   out      receives a new handle; inputs are copied and may be freed after
 *            the call returns (the call synchronises `stream`)
 * Errors: RT_ERR_INVALID_ARG (null pointers, n_tris < 1, n_verts < 3, more
 * than 2^31-1 triangles), RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_DEVICE_LIMIT (tree
 * deeper than the traversal stack). */
rt_status rt_scene_build(const float* d_verts, int64_t n_verts, const int32_t* d_tris, int64_t n_tris,
                         void* stream, rt_scene** out);
rt_status rt_scene_info_get(const rt_scene* scene, rt_scene_info* info);
rt_status rt_scene_destroy(rt_scene* scene);

/* Copy of the binary BVH for inspection (tests, debugging, visualisation).
 * d_nodes: n_nodes x 64 bytes (rt_scene_info.n_nodes), each node as 16 floats:
 *   c0.lo.x c0.hi.x c0.lo.y c0.hi.y | c1.lo.x c1.hi.x c1.lo.y c1.hi.y |
 *   c0.lo.z c0.hi.z c1.lo.z c1.hi.z | child0 child1 (int32) - -
 * where a child >= 0 is an internal node and a child < 0 the leaf ~child, a
 * position in the triangle array; node 0 is the root (a scene of one triangle
 * has no node: its root is leaf 0).  d_tris: n_tris x 48 bytes, triangles in
 * leaf order as v0.xyz, input index (int32 bits), v1.xyz, -, v2.xyz, -.  Both
 * caller device memory; either may be null.  Enqueued on `stream`. */
rt_status rt_scene_export(const rt_scene* scene, void* d_nodes, void* d_tris, void* stream);

/* Describe a dense distance-field grid held in caller memory (not copied;
 * the memory must outlive the handle).  Samples sit at lo + (i,j,k)*h with
 * h = (hi - lo) / (n - 1) per axis, x fastest: value (i,j,k) is at element
 * i + n0*(j + n1*k).  dtype RT_GRID_F32 or RT_GRID_F16 (converted exactly to
 * float for the arithmetic).  n >= 2 per axis, hi > lo.  The paper's field is
 * a set of camera-centred cascades (Section 3, "Distance Field Generation"):
 * see rt_cascade_create; this call describes one dense grid. */
rt_status rt_sdf_create(const void* d_grid, int32_t dtype, const float lo[3], const float hi[3],
                        const int32_t n[3], rt_sdf** out);
rt_status rt_sdf_destroy(rt_sdf* sdf);

/* Build (or rebuild) the library's cell-corner copy of the grid of `sdf`:
 * for every cell the 8 corner values stored together (32 bytes for float32,
 * 16 bytes for float16), so that a march step reads one vector instead of 8
 * scalars.  Same values, same arithmetic, same results.  rt_sdf_bake calls it
 * itself; call it after writing the grid memory any other way (for example
 * after an optimiser step), otherwise the traces keep reading the old copy.
 * Traces read the plain grid until the first prepare, or when the tuning
 * selects the plain layout.  Also builds the x-pair copy (see rt_tuning).
 * Memory: about 8x (cells) + 2x (pairs) the grid, owned by the handle,
 * released by rt_sdf_destroy.  On a cascade: the cell copy of every level
 * (no x-pair copy).  Enqueued on `stream`. */
rt_status rt_sdf_prepare(rt_sdf* sdf, void* stream);

/* Fill the grid of `sdf` with the signed distance to the nearest triangle of
 * `scene`: exact closest point on each triangle, sign from the angle-weighted
 * pseudonormal of the closest face, edge or vertex (positive on the side the
 * normals point to).  This replaces the paper's voxelisation + jump flooding +
 * fast sweeping build (Section 3, "Distance Field Generation") by its exact
 * definition.  method: RT_BAKE_BRUTE tests every triangle for every sample
 * (triangles staged through shared memory); RT_BAKE_BVH prunes with the BVH
 * (same result up to float rounding); RT_BAKE_AUTO picks by problem size.  Writes through the
 * grid pointer given to rt_sdf_create.  On a cascade (rt_cascade_create) every
 * level is baked at its lattice points (ilo_k + i) * h_k, each coordinate
 * rounded once from that product, so that a level moved by rt_cascade_recenter
 * holds the same values as one baked at its new place.
 * RT_BAKE_JFA is the paper's build instead (Section 3, "Distance Field
 * Generation"): conservative voxelisation, jump flooding and sweeping give
 * every sample a site triangle (see rt_sdf_sites), and the value is the signed
 * distance to that triangle.  It equals the exact bake where the site is the
 * nearest triangle and is larger elsewhere; triangles outside the grid's box
 * (the coarsest level's on a cascade) are not seen.  The handle keeps the
 * sites (4 bytes per sample) for rt_cascade_recenter, which then rebuilds each
 * moved level the same way. */
rt_status rt_sdf_bake(const rt_scene* scene, rt_sdf* sdf, int32_t method, void* stream);

/* Site map of the paper's field build: for every sample of `sdf` (level
 * after level on a cascade) the input index of its site triangle (-1: none)
 * after step `stage` of the build:
 *   1  conservative voxelisation: the sample's voxel box (side h (1 + 2^-8),
 *      centred on the sample) meets the triangle (separating-axis test,
 *      Akenine-Moller 2001); on a cascade level below the coarsest, the site of
 *      the nearest sample of the next coarser level is a candidate too
 *   2  jump flooding (Rong & Tan 2006): steps 2^(ceil(log2 n)-1) ... 1, each
 *      sample taking the best site of itself and its 26 neighbours at offsets
 *      {-k, 0, k}^3
 *   3  sweeps along every grid line, +x, -x, +y, -y, +z, -z (the fast-sweeping
 *      step), each sample taking the better of its site and the previous
 *      sample's
 * "Best" is the smallest (squared distance to the triangle, triangle index),
 * evaluated in single precision with every operation rounded once.  Cascade
 * levels are built one at a time, coarsest first: a level runs steps 1..stage
 * before the next finer level takes its sites as seeds.  d_sites: caller
 * memory, one int32 per
 * sample.  The grid values are not touched.  Enqueued on `stream`. */
rt_status rt_sdf_sites(const rt_scene* scene, const rt_sdf* sdf, int32_t stage, int32_t* d_sites, void* stream);

#define RT_MAX_LEVELS 8

/* Camera-centred cascade of distance-field grids (Section 3, "Distance Field
 * Generation": the field is built in cascades centred on the camera, with
 * smaller voxels close to it; 5 levels of 64^3 with a 0.1 m smallest voxel in
 * the paper's combined set-up, twice the resolution for field-only tracing).
 *   d_grid  caller memory of levels * n^3 values of `dtype` (RT_GRID_F32 or
 *           RT_GRID_F16), level after level, x fastest within a level, 16-byte
 *           aligned; not copied, must outlive the handle
 *   levels  1..RT_MAX_LEVELS;  n: samples per axis of every level, 2..1024
 *   h0      voxel edge of the finest level (finite, > 0); level k has
 *           h_k = h0 * 2^k, the same on all three axes
 *   center  the camera position (finite)
 * Level k's samples sit at (ilo_k + (i,j,l)) * h_k with, per axis,
 * ilo_k = floor(center / h_k) - floor((n-1)/2): the centre lies in the middle
 * cell of every level, and the levels nest.  The handle is accepted wherever
 * an rt_sdf is; on a cascade the queries use, at each march step, the
 * trilinear sample of the finest level whose closed box holds the point (the
 * coarsest level's outside all boxes), with eps_hit and eps_min scaled by
 * that level's voxel instead of the grid's smallest voxel edge; t_1 uses
 * the voxel at the query's start point o + t_min d and t_2 the voxel at its end
 * point o + t_max d (Section 3, "GI & Shadow Rays"); the march is clipped to
 * the coarsest level's box.  A cascade is always read through its cell-corner
 * copy: fill it with rt_sdf_bake (or write the values and call rt_sdf_prepare)
 * before tracing; a trace before that returns RT_ERR_INVALID_ARG, as does
 * rt_trace_combined_backward on a cascade.  Errors: RT_ERR_INVALID_ARG for
 * the argument rules above or |center / h0| >= 2^22. */
rt_status rt_cascade_create(const void* d_grid, int32_t dtype, int32_t levels, int32_t n, float h0,
                            const float center[3], rt_sdf** out);

/* Rolling update (Section 3, "Distance Field Generation": when the camera
 * moves, only the cascade slices that changed are rebuilt).  Moves the
 * cascade to a new centre.  Every level whose lattice origin changes keeps the
 * samples that the old and new lattices share (moved within its memory) and
 * fills only the new slices with the exact distance of rt_sdf_bake (BVH
 * method); a level that moved by n or more samples on an axis is baked
 * whole.  After an RT_BAKE_JFA bake, each moved level is rebuilt whole by the
 * paper's build instead, seeded from the next coarser level's sites.  The
 * cell-corner copy of each changed level is rebuilt.  The values equal those
 * of a full rt_sdf_bake at the new centre (with the same method).  Enqueued on
 * `stream`; uses a device scratch of one level owned by the handle (allocated
 * on the first call).  *moved (nullable) receives the number of levels that
 * changed.  Errors: RT_ERR_INVALID_ARG (not a cascade, null or non-finite
 * centre, |center / h0| >= 2^22), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_cascade_recenter(const rt_scene* scene, rt_sdf* sdf, const float center[3], void* stream,
                              int32_t* moved);

/* The combined query of rt_trace_combined for rays and hit records in host
 * memory: the rays are copied to d_rays, traced, and the records copied back
 * to h_hits, in `chunks` pieces (0: 4; 1..64; from 3 pieces on, the first and
 * last are half as large as the others) pipelined over two copy streams and
 * up to four compute streams owned by the library, so that the upload of one
 * piece, the traces of the previous ones and the download of the one before
 * overlap.  The
 * paper's queries start on the GPU (Section 3); this call serves callers whose
 * rays live in host memory.
 *   h_rays, h_hits  host memory of n rays / records; page-locked memory
 *                   (cudaHostAlloc, torch pin_memory) is needed for the copies
 *                   to overlap, pageable memory works but serialises them
 *   d_rays, d_hits  device memory of n rays / records (caller-owned staging)
 * Enqueued behind the work already on `stream`; when the call returns, all of
 * its work is ordered before later work on `stream`, and h_hits is complete
 * once `stream` is synchronised.  Overlapping calls on different streams share
 * the library's copy streams (they serialise there, results stay correct).
 * Errors as rt_trace_combined, plus RT_ERR_INVALID_ARG for a null host buffer
 * or chunks outside 0..64. */
rt_status rt_trace_combined_host(const rt_scene* scene, const rt_sdf* sdf, const rt_ray* h_rays, int64_t n,
                                 const rt_split_params* params, rt_hit* h_hits, rt_ray* d_rays, rt_hit* d_hits,
                                 int32_t chunks, void* stream);

/* Geometry of level k of a cascade: lattice origin ilo[3] and voxel edge *h.
 * Errors: RT_ERR_INVALID_ARG when sdf is not a cascade or k is out of range. */
rt_status rt_cascade_level(const rt_sdf* sdf, int32_t k, int32_t ilo[3], float* h);

/* The pure triangle technique: closest hit (any_hit = 0) or any hit
 * (any_hit = 1) on [t_min, t_max] for n rays.  d_rays: n rt_ray; d_hits: n
 * rt_hit (written).  n may be 0. */
rt_status rt_trace_bvh(const rt_scene* scene, const rt_ray* d_rays, int64_t n, int32_t any_hit,
                       rt_hit* d_hits, void* stream);

/* The pure distance-field technique on [t_min, t_max] (params->mode is
 * ignored and taken as RT_MODE_SDF; the other fields apply). */
rt_status rt_trace_sdf(const rt_sdf* sdf, const rt_ray* d_rays, int64_t n, const rt_split_params* params,
                       rt_hit* d_hits, void* stream);

/* The combined query (Eq. 2 and the rules of rt_split_params) for n rays.
 * `params` is read on the host during the call.  With the stage kernels, a
 * closest-hit split call with 0 < m_near < inf runs its near triangle stage
 * and its field stage at the same time, on two streams of the library forked
 * from `stream` and joined back into it by events (calls on one device share
 * these streams; a lock keeps each call's launches together).  The records
 * are those of the sub-intervals traced in order. */
rt_status rt_trace_combined(const rt_scene* scene, const rt_sdf* sdf, const rt_ray* d_rays, int64_t n,
                            const rt_split_params* params, rt_hit* d_hits, void* stream);

/* Same as rt_trace_combined, and also adds per-query work counts into
 * d_counters (device, 4 x uint64, caller zeroes): [0] BVH nodes visited,
 * [1] triangles tested, [2] field march steps, [3] queries that ran a field
 * sub-interval.  Slower; used to count algorithmic bytes. */
rt_status rt_trace_combined_counted(const rt_scene* scene, const rt_sdf* sdf, const rt_ray* d_rays,
                                    int64_t n, const rt_split_params* params, rt_hit* d_hits,
                                    unsigned long long* d_counters, void* stream);

/* Same as rt_trace_combined, and also reports how long each kernel of the
 * call ran: stage_ms[k] for the k-th part (at most 6: the query order where
 * it applies (see rt_tuning.order_bits), then one launch per sub-interval
 * kind with the wavefront kernels and, for closest-hit split calls, a second
 * near stage after the field (RT_STAGE_BVH_NEAR_REST) and the merge of the
 * near hits; or the one launch of the simple kernel), *n_stages
 * the number of parts, stage_kind[k] RT_STAGE_* (nullable).  stage_ms and
 * stage_kind hold 6 entries.  Each part is timed by CUDA events on the
 * stream that ran it; in a closest-hit split call with 0 < m_near < inf the
 * near and field stages run at the same time on two streams, so their times
 * overlap.  The call
 * synchronises `stream`.  Used to measure per-kernel throughput. */
enum { RT_STAGE_ALL = 0, RT_STAGE_BVH_FULL = 1, RT_STAGE_BVH_NEAR = 2, RT_STAGE_BVH_FAR = 3,
       RT_STAGE_FIELD_FULL = 4, RT_STAGE_FIELD_SPLIT = 5, RT_STAGE_ORDER = 6, RT_STAGE_MERGE = 7,
       RT_STAGE_BVH_NEAR_REST = 8 };
rt_status rt_trace_combined_timed(const rt_scene* scene, const rt_sdf* sdf, const rt_ray* d_rays, int64_t n,
                                  const rt_split_params* params, rt_hit* d_hits, float stage_ms[6],
                                  int32_t stage_kind[6], int32_t* n_stages, void* stream);

/* The combined query of rt_trace_combined, for callers that cannot allocate
 * device memory during the call: for example a renderer whose frame loop
 * forbids allocation, or a host that hands the library a fixed device-memory
 * budget and must not see it grow.  rt_trace_combined takes its per-call
 * scratch (work counters, the query order and two ray queues) from a memory
 * pool; this entry point allocates nothing and uses one fixed array compiled
 * into the library instead.  The paper has no counterpart: this is a
 * deployment variant.
 *   - At most 1,048,576 queries per call (the array holds 20 MiB + 256 bytes
 *     and every GPU that loads the library keeps it until the process ends);
 *     a larger n is rejected with RT_ERR_INVALID_ARG before any work.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 *   - All calls on a device share the one array.  Calls whose work overlaps on
 *     the GPU (other streams, other threads) race and corrupt each other's
 *     results: serialise them, e.g. on one stream.  The counters are cleared
 *     on `stream` at the start of every call.
 *   - Always runs the wavefront stage kernels (the tuning's block, residency,
 *     refill, layout and query order apply), their stages one after the other
 *     on `stream` (not on the library's two streams); results equal
 *     rt_trace_combined's.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
rt_status rt_trace_combined_noalloc(const rt_scene* scene, const rt_sdf* sdf, const rt_ray* d_rays, int64_t n,
                                    const rt_split_params* params, rt_hit* d_hits, void* stream);

/* One batch of queries for rt_trace_batches: its rays, its hit records, its
 * split parameters. */
typedef struct {
    const rt_ray* d_rays;
    rt_hit* d_hits;
    int64_t n;
    rt_split_params params;
} rt_batch;

enum { RT_MAX_BATCHES = 16 };

/* Several batches of queries in one call, for example the primary, shadow, AO
 * and GI rays of one frame (Section 3 uses one split for AO and GI rays and two
 * splits with any-hit for shadow rays).  The result equals one
 * rt_trace_combined per batch.  All batches run through one pipeline of four
 * persistent stage launches (triangles, field, triangles, triangles): every query follows
 * its own batch's sub-interval program through it, so uneven batches share the
 * kernels instead of each paying its own launches and tails, and a frame is a
 * fixed sequence of launches that can be captured in a CUDA graph.  When a
 * batch has closest-hit split queries with 0 < m_near < inf, the first two
 * launches run at the same time on the library's two streams, as in
 * rt_trace_combined, and the field launch starts those queries at t_1 without
 * waiting for their near result.
 *   - at most RT_MAX_BATCHES batches, at most 2^31-1 queries in total;
 *   - mode, any_hit, m_near and m_far may differ per batch; max_steps,
 *     hit_eps_vox, min_step_vox and refine_root must be equal in all batches;
 *   - always uses the wavefront stage kernels; the tuning's block, residency,
 *     refill and layout apply.
 * Errors: RT_ERR_INVALID_ARG before any work for bad batches. */
rt_status rt_trace_batches(const rt_scene* scene, const rt_sdf* sdf, const rt_batch* batches, int32_t n_batches,
                           void* stream);

/* Adjoint of the field-resolved hit distance.  For each query whose hit
 * record (from a forward call with the same params, refine_root = 1) has
 * tracer == RT_TRACER_SDF, the root p* = o + t d of phi = eps satisfies
 * phi_theta(p*) = eps; implicit differentiation gives
 *   dt/dtheta_k = -w_k(p*) / (grad phi(p*) . d)
 * with w_k the 8 trilinear weights.  Adds d_grad_t[i] * dt/dtheta_k into
 * d_grad_grid[k] (float32, same layout as the grid; the caller zeroes it).
 * Queries with grad phi . d > -1e-6 (tangent), a field hit at the start of
 * the sub-interval, or another tracer contribute nothing.  The forward pass
 * is not stored: the kernel re-marches each ray.  The grid must be
 * RT_GRID_F32 and not a cascade. */
rt_status rt_trace_combined_backward(const rt_scene* scene, const rt_sdf* sdf, const rt_ray* d_rays,
                                     int64_t n, const rt_split_params* params, const rt_hit* d_hits,
                                     const float* d_grad_t, float* d_grad_grid, void* stream);

/* Launch tuning of the trace kernels (process-wide; applies to later calls).
 *   kernel        RT_KERNEL_WAVEFRONT: persistent stage kernels, one per
 *                 sub-interval kind, with per-lane refill from a global queue,
 *                 so rays that switch tracer mid-query are regrouped across
 *                 the whole batch; RT_KERNEL_SIMPLE: one thread per query runs
 *                 all its sub-intervals; RT_KERNEL_AUTO (default): the stage
 *                 kernels (on triangles-only calls as well, where they were
 *                 measured at least as fast as one thread per query on GI,
 *                 primary and AO rays).
 *   block         threads per block (multiple of 32, 32..1024)
 *   blocks_per_sm persistent grid = SMs x this (0: as many as fit)
 *   refill_min    triangle stages: a warp fetches new queries when at least
 *                 this many lanes are idle (1..32), or when all are (32 keeps
 *                 the rays of a warp together, which suits coherent rays; a
 *                 lane then runs its segment to the end between two checks,
 *                 otherwise it checks every 8 traversal iterations)
 *   refill_min_field  the same for the distance-field stages, whose queries
 *                 end after very different step counts
 *   bvh_width     2 (default): the binary tree (64-byte nodes); 8: the 8-wide
 *                 compressed tree (80-byte nodes, 8-bit child bounds,
 *                 octant-ordered children).  Scenes whose wide tree would be
 *                 deeper than its traversal stack use the binary tree.
 *   grid_layout   RT_LAYOUT_CELLS (default): use the cell-corner copy when it
 *                 exists; RT_LAYOUT_PLAIN: always read the plain grid;
 *                 RT_LAYOUT_PAIRS: the copy of x-neighbour pairs (4 loads a
 *                 step, twice the grid's size) when it exists
 *   order_bits    0: the first kernel takes the queries in input order.
 *                 1..5 (default 4): it takes each window of 1024
 *                 consecutive queries grouped by the cell that holds the
 *                 query's origin, in a 2^b x 2^b x 2^b lattice over the
 *                 scene's box; windows keep their order.  A warp's queries
 *                 then start in one region and read the same nodes and
 *                 triangles.  It pays when input neighbours start at
 *                 different depths (a screen tile over several surfaces) and
 *                 costs one kernel per call that reads every ray's origin and
 *                 writes 4 bytes per query.  Applied only where the first
 *                 kernel traces near triangle sub-intervals (closest hit, a
 *                 split with 0 < m_near < +inf; in rt_trace_batches, when a
 *                 non-empty batch has such queries) and n >= 64; never to the
 *                 pieces of rt_trace_combined_host, whose copy pipeline an
 *                 extra kernel per piece slows down.
 * Results do not depend on the tuning. */
typedef struct {
    int32_t kernel;
    int32_t block;
    int32_t blocks_per_sm;
    int32_t refill_min;
    int32_t grid_layout;
    int32_t refill_min_field;
    int32_t bvh_width;
    int32_t order_bits;
} rt_tuning;

enum { RT_KERNEL_WAVEFRONT = 0, RT_KERNEL_SIMPLE = 1, RT_KERNEL_AUTO = 2 };
enum { RT_LAYOUT_CELLS = 0, RT_LAYOUT_PLAIN = 1, RT_LAYOUT_PAIRS = 2 };

rt_status rt_set_tuning(const rt_tuning* tuning);
rt_status rt_get_tuning(rt_tuning* tuning);

/* Message of the last failed call on this thread ("" if none). */
const char* rt_last_error(void);

/* Library version string. */
const char* rt_version(void);

#ifdef __cplusplus
}
#endif
#endif
