/*
 * CPU checker for the combined ray query (Bartels & Harada, SIGGRAPH Asia 2022
 * Technical Communications).  TEST INFRASTRUCTURE ONLY: loaded by the tests,
 * the smoke check and the CPU-baseline leg of the benchmark, never by the
 * product path.  Independent of the device library (no shared code).
 *
 * What it computes, and where each part comes from:
 *   - the query (o, d, t_min, t_max, f) of Eq. 1 and its split into mutually
 *     exclusive sub-intervals of Eq. 2, processed in order with early exit for
 *     a closest-hit query and distance-field parts first for an any-hit query
 *     (Section 2, text after Eq. 2);
 *   - the one-split rule [t_min, t_1] triangles / [t_1, t_max] distance field
 *     (Section 3, "Occlusion Queries", and the first GI pass) and the two-split
 *     rule triangles / field / triangles for shadow rays (Section 3, "GI &
 *     Shadow Rays"), t_i from the voxel size times a user multiplier;
 *   - the "pure" techniques the paper compares against (Section 3, first
 *     paragraph): triangles only and distance field only;
 *   - triangle tracing: the closest triangle hit by definition (brute force),
 *     and the same through a plain median-split BVH, with the watertight test
 *     of Woop, Benthin & Wald (JCGT 2013);
 *   - the distance field: exact closest point on each triangle (Voronoi
 *     regions of the triangle, Ericson, Real-Time Collision Detection 5.1.5),
 *     sign from the angle-weighted pseudonormal of the closest feature
 *     (Baerentzen & Aanaes, IEEE TVCG 2005);
 *   - distance-field tracing: sphere tracing on the trilinear interpolant
 *     (march.inc states the step rule).
 *
 * Compiled with -ffp-contract=off so that no multiply-add is fused unless it
 * is written as fma()/fmaf().
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* parallel for over index ranges                                            */
/* ------------------------------------------------------------------------ */
typedef void (*range_fn)(void* ctx, int64_t begin, int64_t end);
typedef struct {
    range_fn fn;
    void* ctx;
    int64_t n, chunk, next;
} pf_state;

static void* pf_worker(void* arg)
{
    pf_state* s = (pf_state*)arg;
    for (;;) {
        int64_t b = __atomic_fetch_add(&s->next, s->chunk, __ATOMIC_RELAXED);
        if (b >= s->n) break;
        int64_t e = b + s->chunk < s->n ? b + s->chunk : s->n;
        s->fn(s->ctx, b, e);
    }
    return NULL;
}

static void parallel_for(int64_t n, int32_t nthreads, int64_t chunk, range_fn fn, void* ctx)
{
    if (nthreads <= 1 || n <= chunk) {
        fn(ctx, 0, n);
        return;
    }
    enum { MAXT = 512 };
    pthread_t th[MAXT];
    pf_state s = {fn, ctx, n, chunk, 0};
    int k = nthreads > MAXT ? MAXT : nthreads;
    int started = 1;
    for (int i = 1; i < k; ++i)
        if (pthread_create(&th[i], NULL, pf_worker, &s) == 0) started = i + 1; else break;
    pf_worker(&s);
    for (int i = 1; i < started; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static inline void sub3(const double* a, const double* b, double* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double* a, const double* b, double* r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static void ray_load(const float* r, double o[3], double d[3], double* tmin, double* tmax)
{
    o[0] = r[0]; o[1] = r[1]; o[2] = r[2]; *tmin = r[3];
    d[0] = r[4]; d[1] = r[5]; d[2] = r[6]; *tmax = r[7];
}

/* Eq. 1 is defined for real o, d, t_min, t_max with t_min <= t_max (the paper
 * assumes this ordering, Section 2): any other query has no intersection and
 * is reported as a miss. */
static int ray_has_nan(const float* r)
{
    for (int k = 0; k < 8; ++k)
        if (isnan(r[k])) return 1;
    return !(r[3] <= r[7]);
}

static void hit_miss(or_hit* h)
{
    h->t = INFINITY;
    h->u = h->v = 0;
    h->prim = -1;
    h->tracer = 0;
    h->flags = 0;
    h->steps = 0;
    h->margin = INFINITY;
}

/* ------------------------------------------------------------------------ */
/* watertight ray/triangle test (Woop, Benthin & Wald 2013), fp64            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kx, ky, kz;
    double Sx, Sy, Sz;
} wt_ray;

static void wt_setup(const double d[3], wt_ray* w)
{
    /* the axis where |d| is largest becomes z; keep the winding by swapping x/y */
    int kz = 0;
    if (fabs(d[1]) > fabs(d[kz])) kz = 1;
    if (fabs(d[2]) > fabs(d[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0) { int s = kx; kx = ky; ky = s; }
    w->kx = kx; w->ky = ky; w->kz = kz;
    w->Sx = d[kx] / d[kz];
    w->Sy = d[ky] / d[kz];
    w->Sz = 1.0 / d[kz];
}

/* returns 1 on a hit of the ray's line; t, u (weight of b), v (weight of c) */
static int wt_test(const double o[3], const wt_ray* w, const double* a, const double* b, const double* c,
                   double* t, double* u, double* v)
{
    double A[3], B[3], C[3];
    sub3(a, o, A); sub3(b, o, B); sub3(c, o, C);
    /* shear and scale the vertices into the ray's frame */
    double Ax = A[w->kx] - w->Sx * A[w->kz], Ay = A[w->ky] - w->Sy * A[w->kz];
    double Bx = B[w->kx] - w->Sx * B[w->kz], By = B[w->ky] - w->Sy * B[w->kz];
    double Cx = C[w->kx] - w->Sx * C[w->kz], Cy = C[w->ky] - w->Sy * C[w->kz];
    /* scaled barycentric coordinates = 2D edge functions */
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0 || V < 0 || W < 0) && (U > 0 || V > 0 || W > 0)) return 0;
    double det = U + V + W;
    if (det == 0) return 0;
    double Az = w->Sz * A[w->kz], Bz = w->Sz * B[w->kz], Cz = w->Sz * C[w->kz];
    double T = U * Az + V * Bz + W * Cz;
    *t = T / det;
    *u = V / det;
    *v = W / det;
    return 1;
}

int or_watertight(const double o[3], const double d[3], const double a[3], const double b[3],
                  const double c[3], double out[3])
{
    wt_ray w;
    wt_setup(d, &w);
    return wt_test(o, &w, a, b, c, &out[0], &out[1], &out[2]);
}

typedef struct {
    const double* V;
    const int32_t* F;
    int64_t nt;
    const float* rays;
    const int32_t* prim;
    double* out;
} tc_ctx;

static void tc_range(void* vctx, int64_t s, int64_t e)
{
    tc_ctx* c = (tc_ctx*)vctx;
    for (int64_t i = s; i < e; ++i) {
        double* r = c->out + 5 * i;
        r[0] = 0; r[1] = INFINITY; r[2] = r[3] = r[4] = 0;
        int32_t k = c->prim[i];
        if (k < 0 || k >= c->nt) continue;
        double o[3], d[3], ta, tb;
        ray_load(c->rays + 8 * i, o, d, &ta, &tb);
        const int32_t* f = c->F + 3 * (int64_t)k;
        const double *a = c->V + 3 * (int64_t)f[0], *b = c->V + 3 * (int64_t)f[1], *cc = c->V + 3 * (int64_t)f[2];
        wt_ray w;
        wt_setup(d, &w);
        double t, u, v;
        double e1[3], e2[3], n[3];
        sub3(b, a, e1); sub3(cc, a, e2); cross3(e1, e2, n);
        if (wt_test(o, &w, a, b, cc, &t, &u, &v)) {
            r[0] = 1; r[1] = t; r[2] = u; r[3] = v;
        } else {
            /* a miss: where the ray's line meets the triangle's plane, in the
             * same barycentric weights (Cramer's rule on o + t d = a + u e1 + v e2),
             * so that the caller sees how far outside an edge it passes */
            double pv[3], tv[3], qv[3];
            cross3(d, e2, pv);
            double det = dot3(e1, pv);
            if (det != 0) {
                sub3(o, a, tv);
                cross3(tv, e1, qv);
                r[2] = dot3(tv, pv) / det;
                r[3] = dot3(d, qv) / det;
                r[1] = dot3(e2, qv) / det;
            }
        }
        double len = sqrt(dot3(n, n));
        r[4] = len > 0 ? fabs(dot3(n, d)) / len : 0;
    }
}

void or_tri_check(const double* V, const int32_t* F, int64_t nt, const float* rays, const int32_t* prim,
                  int64_t nr, int32_t nthreads, double* out)
{
    tc_ctx c = {V, F, nt, rays, prim, out};
    parallel_for(nr, nthreads, 256, tc_range, &c);
}

/* Accept a candidate into the running closest hit: t in [ta, tb], then the
 * smaller t, ties to the smaller triangle index. */
static inline void consider(or_hit* h, double t, double u, double v, int32_t prim, double ta, double tb)
{
    if (!(t >= ta && t <= tb)) return;
    if (h->tracer == 0 || t < h->t || (t == h->t && prim < h->prim)) {
        h->t = t; h->u = u; h->v = v; h->prim = prim; h->tracer = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* brute force: the definition of the closest hit                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double* V;
    const int32_t* F;
    int64_t nt;
    const float* rays;
    or_hit* hits;
} brute_ctx;

static void brute_range(void* vctx, int64_t b, int64_t e)
{
    brute_ctx* c = (brute_ctx*)vctx;
    for (int64_t i = b; i < e; ++i) {
        double o[3], d[3], ta, tb;
        ray_load(c->rays + 8 * i, o, d, &ta, &tb);
        or_hit h;
        hit_miss(&h);
        wt_ray w;
        wt_setup(d, &w);
        for (int64_t k = 0; k < c->nt; ++k) {
            double t, u, v;
            const int32_t* f = c->F + 3 * k;
            if (wt_test(o, &w, c->V + 3 * f[0], c->V + 3 * f[1], c->V + 3 * f[2], &t, &u, &v))
                consider(&h, t, u, v, (int32_t)k, ta, tb);
        }
        if (h.tracer == 0) h.t = INFINITY;
        c->hits[i] = h;
    }
}

void or_trace_brute(const double* V, const int32_t* F, int64_t nt, const float* rays, int64_t nr,
                    int32_t nthreads, or_hit* hits)
{
    brute_ctx c = {V, F, nt, rays, hits};
    parallel_for(nr, nthreads, 16, brute_range, &c);
}

/* ------------------------------------------------------------------------ */
/* plain median-split BVH (leaves of at most 4 triangles)                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
    int32_t left, right, first, count;
} onode;

struct or_bvh {
    int64_t nv, nt, nn;
    double* V;
    int32_t* F;
    int32_t* order;
    double* cen;
    onode* nodes;
    double* fn;  /* nt*3 unit face normals */
    double* en;  /* nt*9 edge pseudonormals (edges ab, bc, ca) */
    double* vpn; /* nv*3 vertex pseudonormals */
};

static inline double key_of(const or_bvh* b, int32_t t, int axis) { return b->cen[3 * (int64_t)t + axis]; }

static void qselect(const or_bvh* bv, int32_t* idx, int axis, int64_t lo, int64_t hi, int64_t k)
{
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        double a = key_of(bv, idx[lo], axis), b = key_of(bv, idx[mid], axis), c = key_of(bv, idx[hi - 1], axis);
        double pivot = (a < b) ? ((b < c) ? b : (a < c ? c : a)) : ((a < c) ? a : (b < c ? c : b));
        int64_t lt = lo, i = lo, gt = hi;
        while (i < gt) {
            double v = key_of(bv, idx[i], axis);
            if (v < pivot) { int32_t s = idx[lt]; idx[lt] = idx[i]; idx[i] = s; ++lt; ++i; }
            else if (v > pivot) { --gt; int32_t s = idx[gt]; idx[gt] = idx[i]; idx[i] = s; }
            else ++i;
        }
        if (k < lt) hi = lt;
        else if (k >= gt) lo = gt;
        else return;
    }
}

static int32_t build_rec(or_bvh* b, int64_t first, int64_t count, double pad)
{
    int32_t id = (int32_t)b->nn++;
    onode* n = &b->nodes[id];
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int a = 0; a < 3; ++a) { n->lo[a] = INFINITY; n->hi[a] = -INFINITY; }
    for (int64_t i = first; i < first + count; ++i) {
        int32_t t = b->order[i];
        for (int c = 0; c < 3; ++c) {
            const double* p = b->V + 3 * (int64_t)b->F[3 * (int64_t)t + c];
            for (int a = 0; a < 3; ++a) {
                if (p[a] < n->lo[a]) n->lo[a] = p[a];
                if (p[a] > n->hi[a]) n->hi[a] = p[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            double v = key_of(b, t, a);
            if (v < clo[a]) clo[a] = v;
            if (v > chi[a]) chi[a] = v;
        }
    }
    for (int a = 0; a < 3; ++a) { n->lo[a] -= pad; n->hi[a] += pad; }
    if (count <= 4) {
        n->left = n->right = -1;
        n->first = (int32_t)first;
        n->count = (int32_t)count;
        return id;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    int64_t half = count / 2;
    qselect(b, b->order, axis, first, first + count, first + half);
    int32_t l = build_rec(b, first, half, pad);
    int32_t r = build_rec(b, first + half, count - half, pad);
    n = &b->nodes[id];
    n->left = l;
    n->right = r;
    n->first = -1;
    n->count = 0;
    return id;
}

typedef struct {
    int32_t a, b; /* vertex pair, a < b */
    int32_t tri, edge;
} edge_rec;

static int edge_cmp(const void* x, const void* y)
{
    const edge_rec* p = (const edge_rec*)x;
    const edge_rec* q = (const edge_rec*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->tri != q->tri) return p->tri < q->tri ? -1 : 1;
    return 0;
}

/* Angle-weighted pseudonormals (Baerentzen & Aanaes 2005): face = unit normal;
 * edge = sum of the unit normals of the faces sharing it; vertex = sum over
 * incident faces of (corner angle) * unit normal. */
static void build_pseudonormals(or_bvh* b)
{
    int64_t nt = b->nt;
    b->fn = (double*)calloc((size_t)(3 * nt + 1), sizeof(double));
    b->en = (double*)calloc((size_t)(9 * nt + 1), sizeof(double));
    b->vpn = (double*)calloc((size_t)(3 * b->nv + 1), sizeof(double));
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* f = b->F + 3 * t;
        double e1[3], e2[3], n[3];
        sub3(b->V + 3 * (int64_t)f[1], b->V + 3 * (int64_t)f[0], e1);
        sub3(b->V + 3 * (int64_t)f[2], b->V + 3 * (int64_t)f[0], e2);
        cross3(e1, e2, n);
        double len = sqrt(dot3(n, n));
        if (len > 0)
            for (int a = 0; a < 3; ++a) b->fn[3 * t + a] = n[a] / len;
        for (int c = 0; c < 3; ++c) {
            const double* p = b->V + 3 * (int64_t)f[c];
            const double* q = b->V + 3 * (int64_t)f[(c + 1) % 3];
            const double* r = b->V + 3 * (int64_t)f[(c + 2) % 3];
            double x[3], y[3], cr[3];
            sub3(q, p, x);
            sub3(r, p, y);
            cross3(x, y, cr);
            double ang = atan2(sqrt(dot3(cr, cr)), dot3(x, y));
            for (int a = 0; a < 3; ++a) b->vpn[3 * (int64_t)f[c] + a] += ang * b->fn[3 * t + a];
        }
    }
    edge_rec* E = (edge_rec*)malloc(sizeof(edge_rec) * (size_t)(3 * nt + 1));
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 3; ++e) {
            int32_t p = b->F[3 * t + e], q = b->F[3 * t + (e + 1) % 3];
            edge_rec r = {p < q ? p : q, p < q ? q : p, (int32_t)t, e};
            E[3 * t + e] = r;
        }
    qsort(E, (size_t)(3 * nt), sizeof(edge_rec), edge_cmp);
    for (int64_t s = 0; s < 3 * nt;) {
        int64_t e = s;
        double sum[3] = {0, 0, 0};
        while (e < 3 * nt && E[e].a == E[s].a && E[e].b == E[s].b) {
            for (int a = 0; a < 3; ++a) sum[a] += b->fn[3 * (int64_t)E[e].tri + a];
            ++e;
        }
        for (int64_t k = s; k < e; ++k)
            for (int a = 0; a < 3; ++a) b->en[9 * (int64_t)E[k].tri + 3 * E[k].edge + a] = sum[a];
        s = e;
    }
    free(E);
}

or_bvh* or_bvh_build(const double* V, int64_t nv, const int32_t* F, int64_t nt)
{
    or_bvh* b = (or_bvh*)calloc(1, sizeof(or_bvh));
    b->nv = nv;
    b->nt = nt;
    b->V = (double*)malloc(sizeof(double) * (size_t)(3 * nv + 1));
    b->F = (int32_t*)malloc(sizeof(int32_t) * (size_t)(3 * nt + 1));
    memcpy(b->V, V, sizeof(double) * (size_t)(3 * nv));
    memcpy(b->F, F, sizeof(int32_t) * (size_t)(3 * nt));
    b->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt + 1));
    b->cen = (double*)malloc(sizeof(double) * (size_t)(3 * nt + 1));
    double ext = 0;
    for (int64_t t = 0; t < nt; ++t) {
        b->order[t] = (int32_t)t;
        for (int a = 0; a < 3; ++a) {
            double s = 0;
            for (int c = 0; c < 3; ++c) {
                double x = V[3 * (int64_t)F[3 * t + c] + a];
                s += x;
                if (fabs(x) > ext) ext = fabs(x);
            }
            b->cen[3 * t + a] = s / 3.0;
        }
    }
    b->nodes = (onode*)calloc((size_t)(2 * nt + 1), sizeof(onode));
    b->nn = 0;
    /* boxes are widened by a margin far above fp64 rounding so that the slab
     * test can never reject a box whose triangle is hit */
    double pad = 1e-9 * (1.0 + ext);
    if (nt > 0) build_rec(b, 0, nt, pad);
    build_pseudonormals(b);
    return b;
}

void or_bvh_free(or_bvh* b)
{
    if (!b) return;
    free(b->V); free(b->F); free(b->order); free(b->cen); free(b->nodes);
    free(b->fn); free(b->en); free(b->vpn);
    free(b);
}

int64_t or_bvh_node_count(const or_bvh* b) { return b->nn; }

static int box_hit(const onode* n, const double o[3], const double d[3], double ta, double tb)
{
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0) {
            if (o[a] < n->lo[a] || o[a] > n->hi[a]) return 0;
            continue;
        }
        double inv = 1.0 / d[a];
        double t0 = (n->lo[a] - o[a]) * inv, t1 = (n->hi[a] - o[a]) * inv;
        if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
        if (t0 > ta) ta = t0;
        if (t1 < tb) tb = t1;
        if (ta > tb) return 0;
    }
    return 1;
}

/* Closest (or any) triangle hit on [ta, tb] through the BVH; fills h when hit. */
static int bvh_segment(const or_bvh* b, const double o[3], const double d[3], double ta, double tb,
                       int any_hit, or_hit* h)
{
    if (b->nt == 0 || !(ta <= tb)) return 0;
    wt_ray w;
    wt_setup(d, &w);
    or_hit best;
    hit_miss(&best);
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode* n = &b->nodes[stack[--sp]];
        double lim = best.tracer ? best.t : tb;
        if (!box_hit(n, o, d, ta, lim)) continue;
        if (n->count > 0) {
            for (int32_t i = n->first; i < n->first + n->count; ++i) {
                int32_t tri = b->order[i];
                const int32_t* f = b->F + 3 * (int64_t)tri;
                double t, u, v;
                if (wt_test(o, &w, b->V + 3 * (int64_t)f[0], b->V + 3 * (int64_t)f[1], b->V + 3 * (int64_t)f[2], &t, &u, &v))
                    consider(&best, t, u, v, tri, ta, tb);
            }
            if (any_hit && best.tracer) break;
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    if (!best.tracer) return 0;
    h->t = best.t; h->u = best.u; h->v = best.v; h->prim = best.prim; h->tracer = 1;
    return 1;
}

typedef struct {
    const or_bvh* b;
    const float* rays;
    int any_hit;
    or_hit* hits;
} bvh_ctx;

static void bvh_range(void* vctx, int64_t s, int64_t e)
{
    bvh_ctx* c = (bvh_ctx*)vctx;
    for (int64_t i = s; i < e; ++i) {
        double o[3], d[3], ta, tb;
        ray_load(c->rays + 8 * i, o, d, &ta, &tb);
        or_hit h;
        hit_miss(&h);
        if (!ray_has_nan(c->rays + 8 * i)) bvh_segment(c->b, o, d, ta, tb, c->any_hit, &h);
        c->hits[i] = h;
    }
}

void or_trace_bvh(const or_bvh* b, const float* rays, int64_t nr, int32_t any_hit, int32_t nthreads,
                  or_hit* hits)
{
    bvh_ctx c = {b, rays, any_hit, hits};
    parallel_for(nr, nthreads, 64, bvh_range, &c);
}

/* ------------------------------------------------------------------------ */
/* exact signed distance                                                     */
/* ------------------------------------------------------------------------ */
/* Closest point on triangle abc to p by its Voronoi regions.  Returns the
 * region: 0 face, 1 vertex a, 2 vertex b, 3 vertex c, 4 edge ab, 5 edge bc,
 * 6 edge ca; q = closest point. */
static int closest_on_tri(const double* p, const double* a, const double* b, const double* c, double q[3])
{
    double ab[3], ac[3], ap[3];
    sub3(b, a, ab); sub3(c, a, ac); sub3(p, a, ap);
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0 && d2 <= 0) { memcpy(q, a, 3 * sizeof(double)); return 1; }
    double bp[3];
    sub3(p, b, bp);
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0 && d4 <= d3) { memcpy(q, b, 3 * sizeof(double)); return 2; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0 && d1 >= 0 && d3 <= 0) {
        double s = d1 / (d1 - d3);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + s * ab[k];
        return 4;
    }
    double cp[3];
    sub3(p, c, cp);
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0 && d5 <= d6) { memcpy(q, c, 3 * sizeof(double)); return 3; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0 && d2 >= 0 && d6 <= 0) {
        double s = d2 / (d2 - d6);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + s * ac[k];
        return 6;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
        double s = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int k = 0; k < 3; ++k) q[k] = b[k] + s * (c[k] - b[k]);
        return 5;
    }
    double den = 1.0 / (va + vb + vc);
    double v = vb * den, w = vc * den;
    for (int k = 0; k < 3; ++k) q[k] = a[k] + ab[k] * v + ac[k] * w;
    return 0;
}

/* pseudonormal of the feature (tri, region) */
static const double* feature_normal(const double* fn, const double* en, const double* vpn, const int32_t* F,
                                    int64_t tri, int region)
{
    switch (region) {
    case 0: return fn + 3 * tri;
    case 1: return vpn + 3 * (int64_t)F[3 * tri + 0];
    case 2: return vpn + 3 * (int64_t)F[3 * tri + 1];
    case 3: return vpn + 3 * (int64_t)F[3 * tri + 2];
    case 4: return en + 9 * tri + 0;
    case 5: return en + 9 * tri + 3;
    default: return en + 9 * tri + 6;
    }
}

typedef struct {
    double d2;
    int64_t tri;
    int region;
    double q[3];
} nearest_t;

static inline void nearest_consider(nearest_t* best, const double* p, const double* V, const int32_t* F, int64_t tri)
{
    double q[3], pq[3];
    const int32_t* f = F + 3 * tri;
    int r = closest_on_tri(p, V + 3 * (int64_t)f[0], V + 3 * (int64_t)f[1], V + 3 * (int64_t)f[2], q);
    sub3(p, q, pq);
    double d2 = dot3(pq, pq);
    if (best->tri < 0 || d2 < best->d2 || (d2 == best->d2 && tri < best->tri)) {
        best->d2 = d2; best->tri = tri; best->region = r;
        memcpy(best->q, q, sizeof(best->q));
    }
}

static double signed_from(const nearest_t* nb, const double* p, const double* fn, const double* en,
                          const double* vpn, const int32_t* F)
{
    if (nb->tri < 0) return INFINITY;
    const double* pn = feature_normal(fn, en, vpn, F, nb->tri, nb->region);
    double pq[3];
    sub3(p, nb->q, pq);
    double dist = sqrt(nb->d2);
    return dot3(pq, pn) >= 0 ? dist : -dist;
}

typedef struct {
    const double* V;
    const int32_t* F;
    int64_t nt;
    const double* P;
    double* out;
    int64_t* feature;
    const double *fn, *en, *vpn;
    const or_bvh* bvh;
} sdf_ctx;

static void sdf_brute_range(void* vctx, int64_t s, int64_t e)
{
    sdf_ctx* c = (sdf_ctx*)vctx;
    for (int64_t i = s; i < e; ++i) {
        nearest_t nb = {INFINITY, -1, 0, {0, 0, 0}};
        for (int64_t t = 0; t < c->nt; ++t) nearest_consider(&nb, c->P + 3 * i, c->V, c->F, t);
        c->out[i] = signed_from(&nb, c->P + 3 * i, c->fn, c->en, c->vpn, c->F);
        if (c->feature) c->feature[i] = nb.tri * 8 + nb.region;
    }
}

void or_sdf_points_brute(const double* V, int64_t nv, const int32_t* F, int64_t nt, const double* P,
                         int64_t np, int32_t nthreads, double* out, int64_t* feature)
{
    /* pseudonormals need the mesh adjacency; reuse the BVH container for them */
    or_bvh* tmp = (or_bvh*)calloc(1, sizeof(or_bvh));
    tmp->nv = nv; tmp->nt = nt;
    tmp->V = (double*)V;
    tmp->F = (int32_t*)F;
    build_pseudonormals(tmp);
    sdf_ctx c = {V, F, nt, P, out, feature, tmp->fn, tmp->en, tmp->vpn, NULL};
    parallel_for(np, nthreads, 8, sdf_brute_range, &c);
    free(tmp->fn); free(tmp->en); free(tmp->vpn); free(tmp);
}

static double box_dist2(const onode* n, const double* p)
{
    double s = 0;
    for (int a = 0; a < 3; ++a) {
        double d = 0;
        if (p[a] < n->lo[a]) d = n->lo[a] - p[a];
        else if (p[a] > n->hi[a]) d = p[a] - n->hi[a];
        s += d * d;
    }
    return s;
}

static void bvh_nearest(const or_bvh* b, const double* p, nearest_t* nb)
{
    nb->tri = -1;
    nb->d2 = INFINITY;
    if (b->nt == 0) return;
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode* n = &b->nodes[stack[--sp]];
        if (nb->tri >= 0 && box_dist2(n, p) > nb->d2) continue;
        if (n->count > 0) {
            for (int32_t i = n->first; i < n->first + n->count; ++i) nearest_consider(nb, p, b->V, b->F, b->order[i]);
        } else {
            double dl = box_dist2(&b->nodes[n->left], p), dr = box_dist2(&b->nodes[n->right], p);
            if (dl <= dr) { stack[sp++] = n->right; stack[sp++] = n->left; }
            else { stack[sp++] = n->left; stack[sp++] = n->right; }
        }
    }
}

static double bvh_sdf_point(const or_bvh* b, const double* p, int64_t* feature)
{
    nearest_t nb;
    bvh_nearest(b, p, &nb);
    if (feature) *feature = nb.tri * 8 + nb.region;
    return signed_from(&nb, p, b->fn, b->en, b->vpn, b->F);
}

static void sdf_bvh_range(void* vctx, int64_t s, int64_t e)
{
    sdf_ctx* c = (sdf_ctx*)vctx;
    for (int64_t i = s; i < e; ++i)
        c->out[i] = bvh_sdf_point(c->bvh, c->P + 3 * i, c->feature ? c->feature + i : NULL);
}

void or_sdf_points_bvh(const or_bvh* b, const double* P, int64_t np, int32_t nthreads, double* out,
                       int64_t* feature)
{
    sdf_ctx c = {0};
    c.P = P; c.out = out; c.feature = feature; c.bvh = b;
    parallel_for(np, nthreads, 16, sdf_bvh_range, &c);
}

/* ------------------------------------------------------------------------ */
/* grid (dense or evaluated on first use)                                    */
/* ------------------------------------------------------------------------ */
struct or_grid {
    double lo[3], hi[3], h[3], ih[3];
    float lo_f[3], hi_f[3], h_f[3], ih_f[3];
    int32_t n[3];
    int64_t count;
    double* val;
    uint8_t* known; /* NULL when dense */
    const or_bvh* src;
    int32_t lattice;  /* 1: sample (i,j,k) sits at (ilo + (i,j,k)) * h */
    int64_t ilo[3];
};

static void sample_position(const or_grid* g, int64_t ix, int64_t iy, int64_t iz, double p[3])
{
    const int64_t ii[3] = {ix, iy, iz};
    for (int a = 0; a < 3; ++a)
        p[a] = g->lattice ? (double)(g->ilo[a] + ii[a]) * g->h[a] : g->lo[a] + (double)ii[a] * g->h[a];
}

static double grid_get(const or_grid* g, int64_t i)
{
    if (!g->known || __atomic_load_n(&g->known[i], __ATOMIC_ACQUIRE)) return g->val[i];
    int64_t nx = g->n[0], ny = g->n[1];
    int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    double p[3];
    sample_position(g, ix, iy, iz, p);
    double v = bvh_sdf_point(g->src, p, NULL);
    /* identical values may be written by several threads; each store is whole */
    uint64_t bitsv;
    memcpy(&bitsv, &v, sizeof bitsv);
    __atomic_store_n((uint64_t*)&g->val[i], bitsv, __ATOMIC_RELAXED);
    __atomic_store_n(&g->known[i], (uint8_t)1, __ATOMIC_RELEASE);
    return v;
}

or_grid* or_grid_new(const double lo[3], const double hi[3], const int32_t n[3], const double* values,
                     const or_bvh* src)
{
    if (n[0] < 2 || n[1] < 2 || n[2] < 2) return NULL;
    if (!values && !src) return NULL;
    or_grid* g = (or_grid*)calloc(1, sizeof(or_grid));
    g->count = (int64_t)n[0] * n[1] * n[2];
    for (int a = 0; a < 3; ++a) {
        g->n[a] = n[a];
        g->lo[a] = lo[a];
        g->hi[a] = hi[a];
        g->h[a] = (hi[a] - lo[a]) / (double)(n[a] - 1);
        g->ih[a] = 1.0 / g->h[a];
        g->lo_f[a] = (float)lo[a];
        g->hi_f[a] = (float)hi[a];
        g->h_f[a] = (g->hi_f[a] - g->lo_f[a]) / (float)(n[a] - 1);
        g->ih_f[a] = 1.0f / g->h_f[a];
    }
    g->val = (double*)malloc(sizeof(double) * (size_t)g->count);
    if (values) {
        memcpy(g->val, values, sizeof(double) * (size_t)g->count);
    } else {
        g->known = (uint8_t*)calloc((size_t)g->count, 1);
        g->src = src;
    }
    return g;
}

or_grid* or_grid_new_lattice(const int64_t ilo[3], double h, const int32_t n[3], const double* values,
                             const or_bvh* src)
{
    if (!(h > 0)) return NULL;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)ilo[a] * h;
        hi[a] = (double)(ilo[a] + n[a] - 1) * h;
    }
    or_grid* g = or_grid_new(lo, hi, n, values, src);
    if (!g) return NULL;
    g->lattice = 1;
    for (int a = 0; a < 3; ++a) {
        /* the spacing is h itself, not (hi - lo) / (n - 1) rounded again */
        g->ilo[a] = ilo[a];
        g->h[a] = h;
        g->ih[a] = 1.0 / h;
        g->h_f[a] = (float)h;
        g->ih_f[a] = 1.0f / g->h_f[a];
    }
    return g;
}

void or_grid_free(or_grid* g)
{
    if (!g) return;
    free(g->val);
    free(g->known);
    free(g);
}

void or_grid_export(const or_grid* g, double* values, uint8_t* known)
{
    for (int64_t i = 0; i < g->count; ++i) {
        int k = g->known ? __atomic_load_n(&g->known[i], __ATOMIC_ACQUIRE) != 0 : 1;
        if (values) values[i] = k ? g->val[i] : 0.0;
        if (known) known[i] = (uint8_t)k;
    }
}

/* a sample as the single-precision march reads it: the fp64 value rounded
 * once to float (IEEE round to nearest even) */
static float fetch_f(const or_grid* g, int64_t i) { return (float)grid_get(g, i); }

typedef struct {
    or_grid* g;
    const int64_t* idx;
    double* out;
} gv_ctx;

static void gv_range(void* vctx, int64_t s, int64_t e)
{
    gv_ctx* c = (gv_ctx*)vctx;
    for (int64_t i = s; i < e; ++i) c->out[i] = grid_get(c->g, c->idx[i]);
}

void or_grid_values(or_grid* g, const int64_t* idx, int64_t count, int32_t nthreads, double* out)
{
    gv_ctx c = {g, idx, out};
    parallel_for(count, nthreads, 64, gv_range, &c);
}

/* ------------------------------------------------------------------------ */
/* camera-centred cascade (Section 3, "Distance Field Generation")           */
/* ------------------------------------------------------------------------ */
#define OR_MAX_LEVELS 16
struct or_cascade {
    int32_t levels, n;
    or_grid* lv[OR_MAX_LEVELS];
};

/* Level k: voxel h_k = h0 * 2^k; n samples per axis at (ilo_k + i) * h_k with
 * ilo_k = floor(center / h_k) - floor((n - 1) / 2), so that the centre lies in
 * the middle cell and a move of the centre by whole voxels moves the lattice
 * origin by whole samples. */
static void cascade_origin(const double center[3], double h0, int32_t n, int32_t k, int64_t ilo[3], double* h)
{
    *h = ldexp(h0, k);
    for (int a = 0; a < 3; ++a) ilo[a] = (int64_t)floor(center[a] / *h) - (int64_t)((n - 1) / 2);
}

or_cascade* or_cascade_new(const double center[3], double h0, int32_t n, int32_t levels, const double* values,
                           const or_bvh* src)
{
    if (levels < 1 || levels > OR_MAX_LEVELS || n < 2 || !(h0 > 0)) return NULL;
    if (!values && !src) return NULL;
    or_cascade* c = (or_cascade*)calloc(1, sizeof(or_cascade));
    c->levels = levels;
    c->n = n;
    const int32_t nn[3] = {n, n, n};
    const int64_t per = (int64_t)n * n * n;
    for (int32_t k = 0; k < levels; ++k) {
        int64_t ilo[3];
        double h;
        cascade_origin(center, h0, n, k, ilo, &h);
        c->lv[k] = or_grid_new_lattice(ilo, h, nn, values ? values + k * per : NULL, src);
    }
    return c;
}

void or_cascade_free(or_cascade* c)
{
    if (!c) return;
    for (int32_t k = 0; k < c->levels; ++k) or_grid_free(c->lv[k]);
    free(c);
}

int32_t or_cascade_level_grid(const or_cascade* c, int32_t k, int64_t ilo[3], double* h, or_grid** grid)
{
    if (k < 0 || k >= c->levels) return 0;
    for (int a = 0; a < 3; ++a) ilo[a] = c->lv[k]->ilo[a];
    *h = c->lv[k]->h[0];
    if (grid) *grid = c->lv[k];
    return 1;
}

/* the two precisions of the distance-field segment */
#define GRID_FETCH(g, i) grid_get((g), (i))
#define REAL double
#define SFX(x) x##_d
#define FMA fma
#define FMIN fmin
#define FMAX fmax
#define FLOOR floor
#define FABS fabs
#define GLO(g) ((g)->lo)
#define GHI(g) ((g)->hi)
#define GIH(g) ((g)->ih)
#define GH(g) ((g)->h)
#include "march.inc"
#undef REAL
#undef SFX
#undef FMA
#undef FMIN
#undef FMAX
#undef FLOOR
#undef FABS
#undef GLO
#undef GHI
#undef GIH
#undef GH
#undef GRID_FETCH
#define GRID_FETCH(g, i) fetch_f((g), (i))
#define REAL float
#define SFX(x) x##_f
#define FMA fmaf
#define FMIN fminf
#define FMAX fmaxf
#define FLOOR floorf
#define FABS fabsf
#define GLO(g) ((g)->lo_f)
#define GHI(g) ((g)->hi_f)
#define GIH(g) ((g)->ih_f)
#define GH(g) ((g)->h_f)
#include "march.inc"
#undef REAL
#undef SFX
#undef FMA
#undef FMIN
#undef FMAX
#undef FLOOR
#undef FABS
#undef GLO
#undef GHI
#undef GIH
#undef GH

/* distance-field segment [ta, tb] in the requested precision, on one grid or
 * on a cascade */
static int sdf_segment(const or_grid* g, const or_cascade* cas, const float* ray, double ta, double tb,
                       const or_params* p, int precision, or_hit* h)
{
    if (cas) {
        if (precision == 32) {
            float o[3] = {ray[0], ray[1], ray[2]}, d[3] = {ray[4], ray[5], ray[6]};
            return march_cascade_f(cas, o, d, (float)ta, (float)tb, (float)p->hit_eps_vox, (float)p->min_step_vox,
                                   p->max_steps, h);
        }
        double o[3] = {ray[0], ray[1], ray[2]}, d[3] = {ray[4], ray[5], ray[6]};
        return march_cascade_d(cas, o, d, ta, tb, p->hit_eps_vox, p->min_step_vox, p->max_steps, h);
    }
    if (precision == 32) {
        float o[3] = {ray[0], ray[1], ray[2]}, d[3] = {ray[4], ray[5], ray[6]};
        float hmin = fminf(fminf(g->h_f[0], g->h_f[1]), g->h_f[2]);
        float eh = (float)p->hit_eps_vox * hmin, em = (float)p->min_step_vox * hmin;
        return march_f(g, o, d, (float)ta, (float)tb, eh, em, p->max_steps, g->lo_f, g->hi_f, g->ih_f, h);
    }
    double o[3] = {ray[0], ray[1], ray[2]}, d[3] = {ray[4], ray[5], ray[6]};
    double hmin = fmin(fmin(g->h[0], g->h[1]), g->h[2]);
    double eh = p->hit_eps_vox * hmin, em = p->min_step_vox * hmin;
    return march_d(g, o, d, ta, tb, eh, em, p->max_steps, g->lo, g->hi, g->ih, h);
}

typedef struct {
    const or_bvh* b;
    const or_grid* g;
    const float* rays;
    const or_params* p;
    int precision;
    or_hit* hits;
    const or_cascade* cas; /* when set, the field is this cascade instead of g */
    double* t12;           /* optional: the split points t_1, t_2 of each query */
} comb_ctx;

/* Eq. 2 split and the ordering rules of Section 2 for one query. */
static void combined_one(const comb_ctx* c, int64_t i)
{
    const float* r = c->rays + 8 * i;
    const or_params* p = c->p;
    double o[3], d[3], tmin, tmax;
    ray_load(r, o, d, &tmin, &tmax);
    or_hit h;
    hit_miss(&h);
    if (ray_has_nan(r)) {
        c->hits[i] = h;
        return;
    }
    int mode = p->mode;
    const int have_field = c->g || c->cas;
    if (mode == 0 || !have_field) {
        bvh_segment(c->b, o, d, tmin, tmax, p->any_hit, &h);
        c->hits[i] = h;
        return;
    }
    if (mode == 3 || !c->b) {
        sdf_segment(c->g, c->cas, r, tmin, tmax, p, c->precision, &h);
        c->hits[i] = h;
        return;
    }
    /* split points t_1 (and t_2) from the voxel size times the multipliers.
     * One grid: its largest voxel edge.  Cascade (Section 3, "GI & Shadow
     * Rays"): the voxel size at the start point o + t_min d for t_1 and at the
     * end point o + t_max d for t_2. */
    double t1, t2;
    if (c->precision == 32) {
        float a = (float)tmin, bb = (float)tmax;
        float hn, hf;
        if (c->cas) {
            float of[3] = {r[0], r[1], r[2]}, df[3] = {r[4], r[5], r[6]};
            hn = voxel_at_f(c->cas, of, df, a);
            hf = voxel_at_f(c->cas, of, df, bb);
        } else {
            hn = hf = fmaxf(fmaxf(c->g->h_f[0], c->g->h_f[1]), c->g->h_f[2]);
        }
        float x1 = fminf(fmaxf(fmaf((float)p->m_near, hn, a), a), bb);
        float x2 = fminf(fmaxf(fmaf(-(float)p->m_far, hf, bb), x1), bb);
        t1 = x1;
        t2 = x2;
    } else {
        double hn, hf;
        if (c->cas) {
            hn = voxel_at_d(c->cas, o, d, tmin);
            hf = voxel_at_d(c->cas, o, d, tmax);
        } else {
            hn = hf = fmax(fmax(c->g->h[0], c->g->h[1]), c->g->h[2]);
        }
        t1 = fmin(fmax(fma(p->m_near, hn, tmin), tmin), tmax);
        t2 = fmin(fmax(fma(-p->m_far, hf, tmax), t1), tmax);
    }
    if (c->t12) {
        c->t12[2 * i] = t1;
        c->t12[2 * i + 1] = mode == 1 ? tmax : t2;
    }
    int near_bvh = p->m_near > 0;
    if (mode == 1) {
        int field = (p->m_near == 0) || (t1 < tmax);
        if (p->any_hit) {
            if (field && sdf_segment(c->g, c->cas, r, t1, tmax, p, c->precision, &h)) { c->hits[i] = h; return; }
            if (near_bvh) bvh_segment(c->b, o, d, tmin, t1, 1, &h);
        } else {
            if (near_bvh && bvh_segment(c->b, o, d, tmin, t1, 0, &h)) { c->hits[i] = h; return; }
            if (field) sdf_segment(c->g, c->cas, r, t1, tmax, p, c->precision, &h);
        }
        c->hits[i] = h;
        return;
    }
    /* mode 2: triangles [t_min, t_1], field [t_1, t_2], triangles [t_2, t_max] */
    int field = (t1 < t2) || (p->m_near == 0 && p->m_far == 0);
    int far_bvh = p->m_far > 0;
    if (p->any_hit) {
        if (field && sdf_segment(c->g, c->cas, r, t1, t2, p, c->precision, &h)) { c->hits[i] = h; return; }
        if (near_bvh && bvh_segment(c->b, o, d, tmin, t1, 1, &h)) { c->hits[i] = h; return; }
        if (far_bvh) bvh_segment(c->b, o, d, t2, tmax, 1, &h);
    } else {
        if (near_bvh && bvh_segment(c->b, o, d, tmin, t1, 0, &h)) { c->hits[i] = h; return; }
        if (field && sdf_segment(c->g, c->cas, r, t1, t2, p, c->precision, &h)) { c->hits[i] = h; return; }
        if (far_bvh) bvh_segment(c->b, o, d, t2, tmax, 0, &h);
    }
    c->hits[i] = h;
}

static void comb_range(void* vctx, int64_t s, int64_t e)
{
    comb_ctx* c = (comb_ctx*)vctx;
    for (int64_t i = s; i < e; ++i) combined_one(c, i);
}

void or_trace_sdf(const or_grid* g, const float* rays, int64_t nr, const or_params* p, int32_t precision,
                  int32_t nthreads, or_hit* hits)
{
    or_params q = *p;
    q.mode = 3;
    comb_ctx c = {NULL, g, rays, &q, precision, hits, NULL, NULL};
    parallel_for(nr, nthreads, 16, comb_range, &c);
}

void or_trace_combined(const or_bvh* b, const or_grid* g, const float* rays, int64_t nr,
                       const or_params* p, int32_t precision, int32_t nthreads, or_hit* hits)
{
    comb_ctx c = {b, g, rays, p, precision, hits, NULL, NULL};
    parallel_for(nr, nthreads, 16, comb_range, &c);
}

void or_trace_combined_cascade(const or_bvh* b, const or_cascade* cas, const float* rays, int64_t nr,
                               const or_params* p, int32_t precision, int32_t nthreads, or_hit* hits,
                               double* t12)
{
    comb_ctx c = {b, NULL, rays, p, precision, hits, cas, t12};
    parallel_for(nr, nthreads, 16, comb_range, &c);
}

void or_cascade_level_of(const or_cascade* c, const double* P, int64_t np, int32_t precision, int32_t* level)
{
    for (int64_t i = 0; i < np; ++i) {
        if (precision == 32) {
            float q[3] = {(float)P[3 * i], (float)P[3 * i + 1], (float)P[3 * i + 2]};
            level[i] = level_of_f(c, q);
        } else {
            level[i] = level_of_d(c, P + 3 * i);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* interpolant value, gradient and the adjoint of the hit distance           */
/* ------------------------------------------------------------------------ */
/* Trilinear weights of the 8 corners at p (order: x fastest), their flat
 * indices, the value and the gradient d(phi)/dp (zero along a clamped axis). */
static double interp_full(const or_grid* g, const double* p, int64_t idx[8], double w[8], double grad[3])
{
    int64_t i0[3];
    double f[3];
    int clamped[3];
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] - g->lo[a]) * g->ih[a];
        double top = (double)(g->n[a] - 1);
        clamped[a] = (u < 0) || (u > top);
        u = fmin(fmax(u, 0.0), top);
        int64_t ii = (int64_t)floor(u);
        if (ii > g->n[a] - 2) ii = g->n[a] - 2;
        f[a] = u - (double)ii;
        i0[a] = ii;
    }
    const int64_t sy = g->n[0], sz = (int64_t)g->n[0] * g->n[1];
    double v[8];
    double phi = 0;
    for (int k = 0; k < 8; ++k) {
        int bx = k & 1, by = (k >> 1) & 1, bz = (k >> 2) & 1;
        idx[k] = (i0[0] + bx) + sy * (i0[1] + by) + sz * (i0[2] + bz);
        v[k] = grid_get(g, idx[k]);
        double wx = bx ? f[0] : 1 - f[0], wy = by ? f[1] : 1 - f[1], wz = bz ? f[2] : 1 - f[2];
        w[k] = wx * wy * wz;
        phi += w[k] * v[k];
    }
    for (int a = 0; a < 3; ++a) {
        double s = 0;
        for (int k = 0; k < 8; ++k) {
            int bit[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
            double dw = bit[a] ? 1.0 : -1.0;
            for (int q = 0; q < 3; ++q)
                if (q != a) dw *= bit[q] ? f[q] : 1 - f[q];
            s += dw * v[k];
        }
        grad[a] = clamped[a] ? 0.0 : s * g->ih[a];
    }
    return phi;
}

void or_grid_sample(const or_grid* g, const double* P, int64_t np, double* phi, double* grad)
{
    for (int64_t i = 0; i < np; ++i) {
        int64_t idx[8];
        double w[8];
        phi[i] = interp_full(g, P + 3 * i, idx, w, grad + 3 * i);
    }
}

void or_sdf_root_adjoint(const or_grid* g, const float* rays, int64_t nr, const or_params* p,
                         double* t_root, int64_t* idx8, double* dtdtheta8)
{
    double hmin = fmin(fmin(g->h[0], g->h[1]), g->h[2]);
    double eh = p->hit_eps_vox * hmin, em = p->min_step_vox * hmin;
    for (int64_t i = 0; i < nr; ++i) {
        const float* r = rays + 8 * i;
        double o[3] = {r[0], r[1], r[2]}, d[3] = {r[4], r[5], r[6]};
        double ta = r[3], tb = r[7];
        t_root[i] = INFINITY;
        for (int k = 0; k < 8; ++k) { idx8[8 * i + k] = -1; dtdtheta8[8 * i + k] = 0; }
        if (!clip_box_d(o, d, g->lo, g->hi, &ta, &tb)) continue;
        /* the march of march.inc, remembering the last point above the threshold */
        double t = ta, t_prev = NAN;
        int hit = 0;
        for (int32_t k = 0; k < p->max_steps; ++k) {
            double q[3] = {fma(t, d[0], o[0]), fma(t, d[1], o[1]), fma(t, d[2], o[2])};
            double phi = trilinear_d(g, q[0], q[1], q[2], g->lo, g->ih);
            if (phi < eh) { hit = 1; break; }
            t_prev = t;
            t = t + fmax(phi, em);
            if (t > tb) break;
        }
        if (!hit) continue;
        if (isnan(t_prev)) { t_root[i] = t; continue; } /* started inside: no bracket, no gradient */
        /* root of phi(o + s d) = eps_hit in [t_prev, t] by bisection */
        double a = t_prev, b = t;
        for (int it = 0; it < 200 && b - a > 1e-13 * (1.0 + fabs(b)); ++it) {
            double m = 0.5 * (a + b);
            double q[3] = {o[0] + m * d[0], o[1] + m * d[1], o[2] + m * d[2]};
            double phi = trilinear_d(g, q[0], q[1], q[2], g->lo, g->ih);
            if (phi < eh) b = m; else a = m;
        }
        double ts = 0.5 * (a + b);
        t_root[i] = ts;
        double q[3] = {o[0] + ts * d[0], o[1] + ts * d[1], o[2] + ts * d[2]};
        int64_t ix[8];
        double w[8], gr[3];
        interp_full(g, q, ix, w, gr);
        double gd = dot3(gr, d);
        if (gd > -1e-6) continue; /* tangent: the root does not move smoothly */
        for (int k = 0; k < 8; ++k) {
            idx8[8 * i + k] = ix[k];
            dtdtheta8[8 * i + k] = -w[k] / gd;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* the paper's field build: voxelisation, jump flooding, sweeping             */
/* ------------------------------------------------------------------------ */
#include "dfgen.inc"
