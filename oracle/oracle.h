/*
 * CPU checker for the combined ray query of Bartels & Harada, "Combining GPU
 * Tracing Methods within a Single Ray Query" (SIGGRAPH Asia 2022 Technical
 * Communications).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is loaded by the test-suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark, and by nothing
 * else.  It shares no source, header, table or helper with the device
 * library; the only thing both sides see is the seeded input (triangles,
 * rays, grid extents) produced by the separate `synth` generators.
 *
 * Plain, slow, obviously correct: double precision throughout (the "fp64"
 * ground truth), plus a float mode of the distance-field march that performs
 * the stated step rule operation by operation in IEEE single precision.
 *
 * Conventions
 *   rays   : float32, 8 per ray: ox oy oz t_min dx dy dz t_max (Eq. 1, d unit)
 *   mesh   : double vertices (nv*3), int32 triangles (nt*3)
 *   grid   : values at lo + (i,j,k)*h, h = (hi-lo)/(n-1), x fastest
 *   hits   : or_hit records; miss = {t=+inf, prim=-1, tracer=0}
 */
#ifndef GB300_RQ_ORACLE_H
#define GB300_RQ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double t, u, v;
    int32_t prim;      /* triangle index, -1 for a miss or a distance-field hit */
    int32_t tracer;    /* 0 miss, 1 triangle (BVH) segment, 2 distance-field segment */
    uint32_t flags;    /* OR_FLAG_* */
    int32_t steps;     /* distance-field march steps taken by this query */
    double margin;     /* smallest |phi - eps_hit| over the query's march steps
                          (+inf without a step): how near the hit test of any
                          step came to the other outcome */
} or_hit;

#define OR_FLAG_STEP_LIMIT 2u

typedef struct {
    int32_t mode;       /* 0 triangles only, 1 one split, 2 two splits, 3 distance field only */
    int32_t any_hit;    /* f of Eq. 1: 0 closest hit, 1 any hit */
    double m_near;      /* multiplier on the voxel size for t_1 (may be +inf) */
    double m_far;       /* multiplier on the voxel size for t_2 (mode 2, may be +inf) */
    int32_t max_steps;  /* march step limit */
    int32_t pad;
    double hit_eps_vox; /* hit threshold, in units of the smallest voxel edge */
    double min_step_vox;/* minimum march step, same units */
} or_params;

typedef struct or_bvh or_bvh;
typedef struct or_grid or_grid;
typedef struct or_cascade or_cascade;

/* Watertight ray/triangle test (Woop, Benthin & Wald, JCGT 2(1), 2013), fp64.
 * Returns 1 when the ray's line meets the triangle; out = {t, u, v}. */
int or_watertight(const double o[3], const double d[3], const double a[3], const double b[3],
                  const double c[3], double out[3]);

/* fp64 watertight test of ray i against triangle prim[i] alone (prim < 0 or
 * >= nt: no test).  out: 5 doubles per ray: hit (1 or 0), t, u, v, and
 * |n . d| with n the unit normal of the triangle.  On a miss t, u, v locate
 * where the ray's line meets the triangle's plane (u or v or 1-u-v < 0 there;
 * all 0 and t = +inf when the line is parallel to the plane). */
void or_tri_check(const double* V, const int32_t* F, int64_t nt, const float* rays, const int32_t* prim,
                  int64_t nr, int32_t nthreads, double* out);

/* Closest hit by definition: every triangle tested, t in [t_min, t_max]. */
void or_trace_brute(const double* V, const int32_t* F, int64_t nt, const float* rays, int64_t nr,
                    int32_t nthreads, or_hit* hits);

or_bvh* or_bvh_build(const double* V, int64_t nv, const int32_t* F, int64_t nt);
void or_bvh_free(or_bvh* b);
int64_t or_bvh_node_count(const or_bvh* b);
void or_trace_bvh(const or_bvh* b, const float* rays, int64_t nr, int32_t any_hit, int32_t nthreads,
                  or_hit* hits);

/* Signed distance: exact closest point on the nearest triangle, sign from the
 * angle-weighted pseudonormal of the closest feature.  feature[i] (nullable) =
 * tri*8 + region (0 face, 1..3 vertex a/b/c, 4 edge ab, 5 edge bc, 6 edge ca). */
void or_sdf_points_brute(const double* V, int64_t nv, const int32_t* F, int64_t nt, const double* P,
                         int64_t np, int32_t nthreads, double* out, int64_t* feature);
void or_sdf_points_bvh(const or_bvh* b, const double* P, int64_t np, int32_t nthreads, double* out,
                       int64_t* feature);

/* Grid of values at lo + (i,j,k)h.  values != NULL: dense copy; else values are
 * computed on first use from `src` by or_sdf_points_bvh. */
or_grid* or_grid_new(const double lo[3], const double hi[3], const int32_t n[3], const double* values,
                     const or_bvh* src);
/* Grid on an integer lattice: sample (i,j,k) at (ilo + (i,j,k)) * h, the same
 * spacing h on every axis (h is used as given, not recomputed from the box). */
or_grid* or_grid_new_lattice(const int64_t ilo[3], double h, const int32_t n[3], const double* values,
                             const or_bvh* src);
void or_grid_free(or_grid* g);
void or_grid_values(or_grid* g, const int64_t* idx, int64_t count, int32_t nthreads, double* out);
/* Every sample value (fp64) and whether it is known: all samples of a dense
 * grid, the samples evaluated so far of one computed on first use.  Unknown
 * samples are written as 0.  Either output may be NULL. */
void or_grid_export(const or_grid* g, double* values, uint8_t* known);

/* Queries.  precision 64: everything in double; precision 32: the distance-field
 * segment, the split and the trilinear sample in IEEE single precision (the
 * triangle segments stay in double). */
void or_trace_sdf(const or_grid* g, const float* rays, int64_t nr, const or_params* p, int32_t precision,
                  int32_t nthreads, or_hit* hits);
void or_trace_combined(const or_bvh* b, const or_grid* g, const float* rays, int64_t nr,
                       const or_params* p, int32_t precision, int32_t nthreads, or_hit* hits);

/* Camera-centred cascade of `levels` lattice grids of n^3 samples (Section 3,
 * "Distance Field Generation").  Level k has voxel h0 * 2^k and lattice origin
 * ilo_k = floor(center / h_k) - floor((n-1)/2) per axis.  values (nullable):
 * levels * n^3 doubles, level after level, x fastest; NULL evaluates them on
 * first use from `src`.  Tracing on a cascade samples, at each march step, the
 * finest level whose box holds the point, with eps_hit and eps_min scaled by
 * that level's voxel; the split points use the voxel at the query's start
 * (t_1) and end (t_2) points.  t12 (nullable, 2 per ray) receives t_1 and t_2
 * of split queries (mode 1 reports t_2 = t_max). */
or_cascade* or_cascade_new(const double center[3], double h0, int32_t n, int32_t levels, const double* values,
                           const or_bvh* src);
void or_cascade_free(or_cascade* c);
int32_t or_cascade_level_grid(const or_cascade* c, int32_t k, int64_t ilo[3], double* h, or_grid** grid);
void or_cascade_level_of(const or_cascade* c, const double* P, int64_t np, int32_t precision, int32_t* level);
void or_trace_combined_cascade(const or_bvh* b, const or_cascade* c, const float* rays, int64_t nr,
                               const or_params* p, int32_t precision, int32_t nthreads, or_hit* hits,
                               double* t12);

/* The paper's field build (Section 3, "Distance Field Generation"):
 * conservative voxelisation, jump flooding, axis sweeps (dfgen.inc states the
 * steps).  or_df_sites writes the site (triangle index, -1 for none) of every
 * sample of g after step `stage` (1 voxelisation, 2 jump flooding, 3 sweeps);
 * coarse / gc: the sites and grid of the next coarser cascade level (NULL
 * otherwise; a cascade is built one level at a time, coarsest first, and a
 * level is seeded from the coarser level's finished sites).  or_df_sweep:
 * step 3 alone, in place.  or_df_field: signed distance (double) from each sample to its
 * site triangle.  or_tri_box_overlap and or_tri_dist2_f expose the single
 * precision triangle/box test and point/triangle squared distance. */
void or_df_sites(const or_bvh* b, const or_grid* g, const int32_t* coarse, const or_grid* gc, int32_t stage,
                 int32_t nthreads, int32_t* sites);
void or_df_sweep(const or_bvh* b, const or_grid* g, int32_t* sites);
void or_df_field(const or_bvh* b, const or_grid* g, const int32_t* sites, double* phi);
int or_tri_box_overlap(const float c[3], const float hs[3], const float a[3], const float b[3], const float cc[3]);
float or_tri_dist2_f(const float p[3], const float a[3], const float b[3], const float c[3]);

/* Trilinear value and gradient of the grid interpolant at points (fp64). */
void or_grid_sample(const or_grid* g, const double* P, int64_t np, double* phi, double* grad);

/* Adjoint of the distance-field hit distance (implicit differentiation at the
 * root of phi = eps_hit inside the last march step).  For each ray with an SDF
 * hit: t_root[i], and the 8 corner indices / weights dt/dtheta. Rays that miss:
 * t_root = +inf, idx = -1. */
void or_sdf_root_adjoint(const or_grid* g, const float* rays, int64_t nr, const or_params* p,
                         double* t_root, int64_t* idx8, double* dtdtheta8);

#ifdef __cplusplus
}
#endif
#endif
