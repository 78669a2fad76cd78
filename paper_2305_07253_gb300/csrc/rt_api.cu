// C entry points: argument checks, handle bookkeeping and launch set-up.
// Every step of the query itself runs in the kernels of rt_trace.cu,
// rt_scene.cu, rt_bake.cu and rt_backward.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "rt_internal.cuh"
#include "rt_trace_dev.cuh"

static thread_local char g_err[512] = "";

// process-wide launch tuning (see rt_set_tuning)
static rt_tuning g_tuning = {RT_KERNEL_AUTO, 128, 0, 32, RT_LAYOUT_CELLS, 16, 2, 4};

const rt_tuning& rt_current_tuning() { return g_tuning; }

extern "C" rt_status rt_set_tuning(const rt_tuning* t)
{
    if (!t) return rt_fail(RT_ERR_INVALID_ARG, "tuning is null");
    if (t->kernel != RT_KERNEL_WAVEFRONT && t->kernel != RT_KERNEL_SIMPLE && t->kernel != RT_KERNEL_AUTO)
        return rt_fail(RT_ERR_INVALID_ARG, "kernel %d", t->kernel);
    if (t->block < 32 || t->block > 1024 || t->block % 32)
        return rt_fail(RT_ERR_INVALID_ARG, "block %d must be a multiple of 32 in [32, 1024]", t->block);
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 64) return rt_fail(RT_ERR_INVALID_ARG, "blocks_per_sm %d", t->blocks_per_sm);
    if (t->refill_min < 1 || t->refill_min > 32) return rt_fail(RT_ERR_INVALID_ARG, "refill_min %d", t->refill_min);
    if (t->refill_min_field < 1 || t->refill_min_field > 32)
        return rt_fail(RT_ERR_INVALID_ARG, "refill_min_field %d", t->refill_min_field);
    if (t->bvh_width != 2 && t->bvh_width != 8) return rt_fail(RT_ERR_INVALID_ARG, "bvh_width %d", t->bvh_width);
    if (t->grid_layout != RT_LAYOUT_CELLS && t->grid_layout != RT_LAYOUT_PLAIN && t->grid_layout != RT_LAYOUT_PAIRS)
        return rt_fail(RT_ERR_INVALID_ARG, "grid_layout %d", t->grid_layout);
    if (t->order_bits < 0 || t->order_bits > kOrderMaxBits)
        return rt_fail(RT_ERR_INVALID_ARG, "order_bits %d not in 0..%d", t->order_bits, kOrderMaxBits);
    g_tuning = *t;
    return RT_OK;
}

extern "C" rt_status rt_get_tuning(rt_tuning* t)
{
    if (!t) return rt_fail(RT_ERR_INVALID_ARG, "tuning is null");
    *t = g_tuning;
    return RT_OK;
}

rt_status rt_fail(rt_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

rt_status rt_cuda_fail(cudaError_t e, const char* what)
{
    cudaGetLastError();  // clear a non-sticky error so the next call starts clean
    return rt_fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "%s: %s (%s)", what,
                   cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" const char* rt_last_error(void) { return g_err; }
extern "C" const char* rt_version(void) { return "gb300-rayquery 0.1 (sm_103a)"; }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static rt_status check_params(const rt_split_params* p)
{
    if (!p) return rt_fail(RT_ERR_INVALID_ARG, "params is null");
    if (p->mode < 0 || p->mode > 3) return rt_fail(RT_ERR_INVALID_ARG, "mode %d not in 0..3", p->mode);
    if (!(p->m_near >= 0.f) || !(p->m_far >= 0.f))
        return rt_fail(RT_ERR_INVALID_ARG, "multipliers must be >= 0 (got %g, %g)", p->m_near, p->m_far);
    if (p->max_steps < 1) return rt_fail(RT_ERR_INVALID_ARG, "max_steps must be >= 1");
    if (!(p->hit_eps_vox >= 0.f) || !(p->min_step_vox > 0.f) || isinf(p->hit_eps_vox) || isinf(p->min_step_vox))
        return rt_fail(RT_ERR_INVALID_ARG, "hit_eps_vox must be >= 0 and min_step_vox > 0, both finite");
    if (p->any_hit != 0 && p->any_hit != 1) return rt_fail(RT_ERR_INVALID_ARG, "any_hit must be 0 or 1");
    return RT_OK;
}

static rt_status check_io(const rt_ray* rays, int64_t n, const rt_hit* hits)
{
    if (n < 0) return rt_fail(RT_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n == 0) return RT_OK;
    if (!rays || !hits) return rt_fail(RT_ERR_INVALID_ARG, "null ray or hit buffer");
    if (!aligned16(rays)) return rt_fail(RT_ERR_INVALID_ARG, "ray buffer not 16-byte aligned");
    if (((uintptr_t)hits & 7u) != 0) return rt_fail(RT_ERR_INVALID_ARG, "hit buffer not 8-byte aligned");
    return RT_OK;
}

// Cascade level k as the queries see it: h = h0 * 2^k (exact), box corners
// (float)ilo * h and (float)(ilo + n - 1) * h rounded once, ih = 1 / h rounded once.
void rt_cascade_geometry(const rt_sdf* sdf, int k, float lo[3], float hi[3], float* h, float* ih)
{
    const float hk = ldexpf(sdf->h0, k);
    for (int a = 0; a < 3; ++a) {
        volatile float l = (float)sdf->ilo[k][a] * hk;
        volatile float u = (float)(sdf->ilo[k][a] + sdf->n[a] - 1) * hk;
        lo[a] = l;
        hi[a] = u;
    }
    *h = hk;
    *ih = 1.0f / hk;
}

// Host-side set-up of the split (the same float operations the queries use).
rt_status rt_fill_trace_args(TraceArgs& a, const rt_scene* sc, const rt_sdf* sdf, const rt_split_params* p)
{
    memset(&a, 0, sizeof(a));
    if (sc) {
        a.nodes = sc->nodes;
        a.tris = sc->tris;
        if (g_tuning.bvh_width == 8 && sc->wnodes) {
            a.wnodes = sc->wnodes;
            a.wtris = sc->wtris;
        }
        a.root = sc->n_tris == 0 ? INT32_MIN : (sc->n_tris == 1 ? ~0 : 0);
    } else {
        a.root = INT32_MIN;
    }
    if (sdf) {
        a.grid = sdf->grid;
        a.cells = sdf->cells;
        a.pairs = sdf->pairs;
        a.grid_f16 = sdf->dtype == RT_GRID_F16;
        for (int k = 0; k < 3; ++k) {
            a.glo[k] = sdf->lo[k];
            a.ghi[k] = sdf->hi[k];
            a.gih[k] = sdf->ih[k];
            a.gn[k] = sdf->n[k];
        }
        float hmin = fminf(fminf(sdf->h[0], sdf->h[1]), sdf->h[2]);
        a.hsplit = fmaxf(fmaxf(sdf->h[0], sdf->h[1]), sdf->h[2]);
        a.eps_hit = p->hit_eps_vox * hmin;
        a.eps_min = p->min_step_vox * hmin;
        if (sdf->levels > 0) {
            if (!sdf->cells)
                return rt_fail(RT_ERR_INVALID_ARG, "cascade has no cell copy yet: call rt_sdf_bake or rt_sdf_prepare");
            a.levels = sdf->levels;
            a.level_cells = rtdev::cell_count(sdf->n[0], sdf->n[0], sdf->n[0]);
            for (int k = 0; k < sdf->levels; ++k) {
                CascLevel& v = a.lv[k];
                rt_cascade_geometry(sdf, k, v.lo, v.hi, &v.h, &v.ih);
                v.eps_hit = p->hit_eps_vox * v.h;
                v.eps_min = p->min_step_vox * v.h;
            }
        }
    }
    a.max_steps = p->max_steps;
    a.mode = p->mode;
    a.any_hit = p->any_hit;
    a.refine_root = p->refine_root;
    a.m_near = p->m_near;
    a.m_far = p->m_far;
    // query order (where rt_order_applies; the caller clears ob.bits elsewhere):
    // cells over the scene's box
    if (g_tuning.order_bits > 0 && sc) {
        a.ob.bits = g_tuning.order_bits;
        for (int k = 0; k < 3; ++k) {
            const float ext = sc->hi[k] - sc->lo[k];
            a.ob.lo[k] = sc->lo[k];
            a.ob.scale[k] = ext > 0.f ? (float)(1 << a.ob.bits) / ext : 0.f;
        }
    }
    return RT_OK;
}

static rt_status device_matches(int dev)
{
    int cur = -1;
    RT_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != dev) return rt_fail(RT_ERR_INVALID_ARG, "handle belongs to device %d, current device is %d", dev, cur);
    return RT_OK;
}

extern "C" rt_status rt_scene_build(const float* d_verts, int64_t n_verts, const int32_t* d_tris, int64_t n_tris,
                                    void* stream, rt_scene** out)
{
    if (!out) return rt_fail(RT_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!d_verts || !d_tris) return rt_fail(RT_ERR_INVALID_ARG, "null vertex or triangle buffer");
    if (n_tris < 1 || n_verts < 3) return rt_fail(RT_ERR_INVALID_ARG, "need n_tris >= 1 and n_verts >= 3");
    if (n_tris > (int64_t)INT32_MAX / 2 || n_verts > (int64_t)INT32_MAX)
        return rt_fail(RT_ERR_INVALID_ARG, "mesh too large (n_tris %lld)", (long long)n_tris);
    if (((uintptr_t)d_verts & 3u) || ((uintptr_t)d_tris & 3u))
        return rt_fail(RT_ERR_INVALID_ARG, "vertex/triangle buffers must be 4-byte aligned");
    rt_scene* sc = new (std::nothrow) rt_scene();
    if (!sc) return rt_fail(RT_ERR_OOM, "host allocation failed");
    memset(sc, 0, sizeof(*sc));
    cudaGetDevice(&sc->device);
    rt_status st = rt_build_scene(d_verts, n_verts, d_tris, n_tris, (cudaStream_t)stream, sc);
    if (st != RT_OK) {
        rt_scene_destroy(sc);
        return st;
    }
    *out = sc;
    return RT_OK;
}

extern "C" rt_status rt_scene_info_get(const rt_scene* sc, rt_scene_info* info)
{
    if (!sc || !info) return rt_fail(RT_ERR_INVALID_ARG, "null argument");
    info->n_tris = sc->n_tris;
    info->n_verts = sc->n_verts;
    info->n_nodes = sc->n_nodes;
    info->max_depth = sc->max_depth;
    info->stack_depth = RT_STACK_DEPTH;
    info->n_wide_nodes = sc->wnodes ? sc->n_wnodes : 0;
    info->wide_depth = sc->wide_depth;
    info->pad_ = 0;
    for (int k = 0; k < 3; ++k) {
        info->lo[k] = sc->lo[k];
        info->hi[k] = sc->hi[k];
    }
    info->device_bytes = sc->bytes;
    return RT_OK;
}

extern "C" rt_status rt_scene_export(const rt_scene* sc, void* d_nodes, void* d_tris, void* stream)
{
    if (!sc) return rt_fail(RT_ERR_INVALID_ARG, "scene is null");
    rt_status st = device_matches(sc->device);
    if (st != RT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_nodes && sc->n_tris > 1)
        RT_CUDA_TRY(cudaMemcpyAsync(d_nodes, sc->nodes, (size_t)(sc->n_tris - 1) * sizeof(BNode),
                                    cudaMemcpyDeviceToDevice, s));
    if (d_tris)
        RT_CUDA_TRY(cudaMemcpyAsync(d_tris, sc->tris, (size_t)sc->n_tris * 3 * sizeof(float4),
                                    cudaMemcpyDeviceToDevice, s));
    return RT_OK;
}

extern "C" rt_status rt_scene_destroy(rt_scene* sc)
{
    if (!sc) return RT_OK;
    cudaFree(sc->nodes);
    cudaFree(sc->tris);
    cudaFree(sc->pn);
    cudaFree(sc->slot);
    cudaFree(sc->wnodes);
    cudaFree(sc->wtris);
    delete sc;
    return RT_OK;
}

extern "C" rt_status rt_sdf_create(const void* d_grid, int32_t dtype, const float lo[3], const float hi[3],
                                   const int32_t n[3], rt_sdf** out)
{
    if (!out) return rt_fail(RT_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!d_grid || !lo || !hi || !n) return rt_fail(RT_ERR_INVALID_ARG, "null argument");
    if (dtype != RT_GRID_F32 && dtype != RT_GRID_F16) return rt_fail(RT_ERR_INVALID_ARG, "dtype %d", dtype);
    if (!aligned16(d_grid)) return rt_fail(RT_ERR_INVALID_ARG, "grid not 16-byte aligned");
    int64_t cnt = 1;
    for (int k = 0; k < 3; ++k) {
        if (n[k] < 2) return rt_fail(RT_ERR_INVALID_ARG, "n[%d] = %d < 2", k, n[k]);
        if (!(hi[k] > lo[k]) || isinf(lo[k]) || isinf(hi[k]))
            return rt_fail(RT_ERR_INVALID_ARG, "need finite hi > lo on axis %d", k);
        cnt *= n[k];
    }
    if (cnt > ((int64_t)1 << 40)) return rt_fail(RT_ERR_INVALID_ARG, "grid too large");
    rt_sdf* g = new (std::nothrow) rt_sdf();
    if (!g) return rt_fail(RT_ERR_OOM, "host allocation failed");
    memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    g->grid = d_grid;
    g->dtype = dtype;
    for (int k = 0; k < 3; ++k) {
        g->lo[k] = lo[k];
        g->hi[k] = hi[k];
        g->n[k] = n[k];
        // spacing and its reciprocal, rounded once each in float
        volatile float ext = hi[k] - lo[k];
        g->h[k] = ext / (float)(n[k] - 1);
        g->ih[k] = 1.0f / g->h[k];
    }
    *out = g;
    return RT_OK;
}

extern "C" rt_status rt_sdf_destroy(rt_sdf* sdf)
{
    if (!sdf) return RT_OK;
    if (sdf->cells) cudaFree(sdf->cells);
    if (sdf->pairs) cudaFree(sdf->pairs);
    if (sdf->scratch) cudaFree(sdf->scratch);
    if (sdf->sites) cudaFree(sdf->sites);
    delete sdf;
    return RT_OK;
}

// lattice origin of level k around `center` (floor taken in double)
static bool cascade_origin(const float center[3], float h0, int32_t n, int k, int32_t ilo[3])
{
    const double hk = ldexp((double)h0, k);
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(center[a]) || !(fabs((double)center[a] / (double)h0) < 4194304.0)) return false;
        ilo[a] = (int32_t)floor((double)center[a] / hk) - (n - 1) / 2;
    }
    return true;
}

extern "C" rt_status rt_cascade_create(const void* d_grid, int32_t dtype, int32_t levels, int32_t n, float h0,
                                       const float center[3], rt_sdf** out)
{
    if (!out) return rt_fail(RT_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!d_grid || !center) return rt_fail(RT_ERR_INVALID_ARG, "null argument");
    if (dtype != RT_GRID_F32 && dtype != RT_GRID_F16) return rt_fail(RT_ERR_INVALID_ARG, "dtype %d", dtype);
    if (!aligned16(d_grid)) return rt_fail(RT_ERR_INVALID_ARG, "grid not 16-byte aligned");
    if (levels < 1 || levels > RT_MAX_LEVELS)
        return rt_fail(RT_ERR_INVALID_ARG, "levels %d not in 1..%d", levels, RT_MAX_LEVELS);
    if (n < 2 || n > 1024) return rt_fail(RT_ERR_INVALID_ARG, "n %d not in 2..1024", n);
    if (!(h0 > 0.f) || isinf(h0)) return rt_fail(RT_ERR_INVALID_ARG, "h0 must be finite and > 0");
    rt_sdf* g = new (std::nothrow) rt_sdf();
    if (!g) return rt_fail(RT_ERR_OOM, "host allocation failed");
    memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    g->grid = d_grid;
    g->dtype = dtype;
    g->levels = levels;
    g->h0 = h0;
    for (int k = 0; k < levels; ++k) {
        if (!cascade_origin(center, h0, n, k, g->ilo[k])) {
            delete g;
            return rt_fail(RT_ERR_INVALID_ARG, "centre must be finite with |center / h0| < 2^22");
        }
    }
    for (int a = 0; a < 3; ++a) g->n[a] = n;
    // the coarsest level's box clips every march
    float lo[3], hi[3], h, ih;
    rt_cascade_geometry(g, levels - 1, lo, hi, &h, &ih);
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = lo[a];
        g->hi[a] = hi[a];
        g->h[a] = h;
        g->ih[a] = ih;
    }
    *out = g;
    return RT_OK;
}

extern "C" rt_status rt_cascade_level(const rt_sdf* sdf, int32_t k, int32_t ilo[3], float* h)
{
    if (!sdf || !ilo || !h) return rt_fail(RT_ERR_INVALID_ARG, "null argument");
    if (sdf->levels < 1) return rt_fail(RT_ERR_INVALID_ARG, "not a cascade");
    if (k < 0 || k >= sdf->levels) return rt_fail(RT_ERR_INVALID_ARG, "level %d not in 0..%d", k, sdf->levels - 1);
    for (int a = 0; a < 3; ++a) ilo[a] = sdf->ilo[k][a];
    *h = ldexpf(sdf->h0, k);
    return RT_OK;
}

extern "C" rt_status rt_cascade_recenter(const rt_scene* sc, rt_sdf* sdf, const float center[3], void* stream,
                                         int32_t* moved)
{
    if (moved) *moved = 0;
    if (!sc || !sdf || !center) return rt_fail(RT_ERR_INVALID_ARG, "null argument");
    if (sdf->levels < 1) return rt_fail(RT_ERR_INVALID_ARG, "not a cascade");
    rt_status st = device_matches(sc->device);
    if (st != RT_OK) return st;
    int32_t ilo[RT_MAX_LEVELS][3];
    for (int k = 0; k < sdf->levels; ++k)
        if (!cascade_origin(center, sdf->h0, sdf->n[0], k, ilo[k]))
            return rt_fail(RT_ERR_INVALID_ARG, "centre must be finite with |center / h0| < 2^22");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = sdf->n[0];
    const int64_t level_bytes = n * n * n * (sdf->dtype == RT_GRID_F16 ? 2 : 4);
    if (!sdf->cells) {
        st = rt_launch_prepare(sdf, s);  // allocates the cell copy
        if (st != RT_OK) return st;
    }
    int32_t count = 0;
    const bool jfa = sdf->bake_method == RT_BAKE_JFA && sdf->sites;
    int rebuilt[RT_MAX_LEVELS];
    int n_rebuilt = 0;
    // coarsest first: a level baked whole is bounded (exact bake) or seeded (the
    // paper's build) by the next coarser one at its new place
    for (int k = sdf->levels - 1; k >= 0; --k) {
        int32_t shift[3];
        bool same = true, far = false;
        for (int a = 0; a < 3; ++a) {
            shift[a] = ilo[k][a] - sdf->ilo[k][a];
            same = same && shift[a] == 0;
            far = far || shift[a] >= n || shift[a] <= -n;
        }
        if (same) continue;
        const void* keep = nullptr;
        if (!far && !jfa) {
            if (!sdf->scratch) {
                RT_CUDA_TRY(cudaMalloc(&sdf->scratch, (size_t)level_bytes));
                sdf->scratch_bytes = level_bytes;
            }
            const char* src = static_cast<const char*>(sdf->grid) + k * level_bytes;
            RT_CUDA_TRY(cudaMemcpyAsync(sdf->scratch, src, (size_t)level_bytes, cudaMemcpyDeviceToDevice, s));
            keep = sdf->scratch;
        }
        for (int a = 0; a < 3; ++a) sdf->ilo[k][a] = ilo[k][a];
        ++count;
        if (jfa) {  // the paper's build: moved levels are rebuilt whole, together, below
            rebuilt[n_rebuilt++] = k;
            continue;
        }
        st = rt_launch_cascade_bake(sc, sdf, k, RT_BAKE_BVH, keep, shift, s);
        if (st != RT_OK) return st;
        st = rt_launch_cascade_cells(sdf, k, s);
        if (st != RT_OK) return st;
    }
    if (n_rebuilt > 0) {
        st = rt_launch_df_levels(sc, sdf, rebuilt, n_rebuilt, sdf->sites, s);
        for (int l = 0; l < n_rebuilt && st == RT_OK; ++l) st = rt_launch_cascade_cells(sdf, rebuilt[l], s);
        if (st != RT_OK) return st;
    }
    float lo[3], hi[3], h, ih;
    rt_cascade_geometry(sdf, sdf->levels - 1, lo, hi, &h, &ih);
    for (int a = 0; a < 3; ++a) {
        sdf->lo[a] = lo[a];
        sdf->hi[a] = hi[a];
    }
    if (moved) *moved = count;
    return RT_OK;
}

extern "C" rt_status rt_sdf_prepare(rt_sdf* sdf, void* stream)
{
    if (!sdf) return rt_fail(RT_ERR_INVALID_ARG, "grid is null");
    rt_status st = device_matches(sdf->device);
    if (st != RT_OK) return st;
    return rt_launch_prepare(sdf, (cudaStream_t)stream);
}

static int64_t sample_count(const rt_sdf* sdf)
{
    return (int64_t)(sdf->levels > 0 ? sdf->levels : 1) * sdf->n[0] * sdf->n[1] * sdf->n[2];
}

extern "C" rt_status rt_sdf_bake(const rt_scene* sc, rt_sdf* sdf, int32_t method, void* stream)
{
    if (!sc || !sdf) return rt_fail(RT_ERR_INVALID_ARG, "null scene or grid");
    if (method < 0 || method > 3) return rt_fail(RT_ERR_INVALID_ARG, "bake method %d", method);
    rt_status st = device_matches(sc->device);
    if (st != RT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (method == RT_BAKE_JFA) {
        const int64_t count = sample_count(sdf);
        if (!sdf->sites || sdf->sites_count != count) {
            if (sdf->sites) cudaFree(sdf->sites);
            sdf->sites = nullptr;
            sdf->sites_count = 0;
            RT_CUDA_TRY(cudaMalloc(&sdf->sites, (size_t)count * sizeof(int32_t)));
            sdf->sites_count = count;
        }
        int lv[RT_MAX_LEVELS];
        const int nl = sdf->levels > 0 ? sdf->levels : 1;
        for (int l = 0; l < nl; ++l) lv[l] = nl - 1 - l;  // coarsest first
        st = rt_launch_df_levels(sc, sdf, lv, nl, sdf->sites, s);
    } else {
        st = rt_launch_bake(sc, sdf, method, s);
    }
    if (st != RT_OK) return st;
    sdf->bake_method = method;
    return rt_launch_prepare(sdf, s);
}

extern "C" rt_status rt_sdf_sites(const rt_scene* sc, const rt_sdf* sdf, int32_t stage, int32_t* d_sites,
                                  void* stream)
{
    if (!sc || !sdf || !d_sites) return rt_fail(RT_ERR_INVALID_ARG, "null argument");
    if (stage < 1 || stage > 3) return rt_fail(RT_ERR_INVALID_ARG, "stage %d not in 1..3", stage);
    if (((uintptr_t)d_sites & 3u) != 0) return rt_fail(RT_ERR_INVALID_ARG, "site buffer not 4-byte aligned");
    rt_status st = device_matches(sc->device);
    if (st != RT_OK) return st;
    return rt_launch_df_sites(sc, sdf, stage, d_sites, (cudaStream_t)stream);
}

// allow_order = false: trace in input order whatever the tuning, and the
// stages in sequence on `stream` (the pieces of rt_trace_combined_host, whose
// pipeline an extra kernel per piece slows down, and whose pieces run on
// streams of their own)
static rt_status trace_common(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* rays, int64_t n,
                              const rt_split_params* p, rt_hit* hits, unsigned long long* counters,
                              void* stream, StageTiming* timing = nullptr, bool allow_order = true)
{
    rt_status st = check_params(p);
    if (st != RT_OK) return st;
    st = check_io(rays, n, hits);
    if (st != RT_OK) return st;
    if (p->mode != RT_MODE_SDF && !sc) return rt_fail(RT_ERR_INVALID_ARG, "mode %d needs a scene", p->mode);
    if (p->mode != RT_MODE_BVH && !sdf) return rt_fail(RT_ERR_INVALID_ARG, "mode %d needs a grid", p->mode);
    if (counters && ((uintptr_t)counters & 7u)) return rt_fail(RT_ERR_INVALID_ARG, "counters misaligned");
    if (n == 0) return RT_OK;
    TraceArgs a;
    st = rt_fill_trace_args(a, p->mode == RT_MODE_SDF ? nullptr : sc, p->mode == RT_MODE_BVH ? nullptr : sdf, p);
    if (st != RT_OK) return st;
    if (sc && p->mode != RT_MODE_SDF) {
        st = device_matches(sc->device);
        if (st != RT_OK) return st;
    }
    if (sdf && p->mode != RT_MODE_BVH) {
        st = device_matches(sdf->device);
        if (st != RT_OK) return st;
    }
    a.rays = reinterpret_cast<const float4*>(rays);
    a.hits = hits;
    a.n = n;
    a.counters = counters;
    if (!allow_order || !rt_order_applies(*p)) a.ob.bits = 0;
    return rt_launch_trace(a, counters != nullptr, (cudaStream_t)stream, timing, allow_order);
}

extern "C" rt_status rt_trace_combined_timed(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* rays, int64_t n,
                                             const rt_split_params* params, rt_hit* hits, float stage_ms[6],
                                             int32_t stage_kind[6], int32_t* n_stages, void* stream)
{
    if (!stage_ms || !n_stages) return rt_fail(RT_ERR_INVALID_ARG, "null stage_ms or n_stages");
    *n_stages = 0;
    if (n == 0) return trace_common(sc, sdf, rays, n, params, hits, nullptr, stream);
    StageTiming tm = {};
    int made = 0;
    rt_status st = RT_OK;
    for (; made < 2 * kMaxTimedParts; ++made) {
        cudaError_t e = cudaEventCreate(&tm.events[made]);
        if (e != cudaSuccess) { st = rt_cuda_fail(e, "cudaEventCreate"); break; }
    }
    if (st == RT_OK) st = trace_common(sc, sdf, rays, n, params, hits, nullptr, stream, &tm);
    if (st == RT_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = rt_cuda_fail(e, "cudaStreamSynchronize");
    }
    if (st == RT_OK) {
        for (int k = 0; k < tm.n_launches; ++k) {
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, tm.events[2 * k], tm.events[2 * k + 1]);
            if (e != cudaSuccess) { st = rt_cuda_fail(e, "cudaEventElapsedTime"); break; }
            stage_ms[k] = ms;
            if (stage_kind) stage_kind[k] = tm.kinds[k];
        }
        if (st == RT_OK) *n_stages = tm.n_launches;
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(tm.events[k]);
    return st;
}

extern "C" rt_status rt_trace_bvh(const rt_scene* sc, const rt_ray* rays, int64_t n, int32_t any_hit, rt_hit* hits,
                                  void* stream)
{
    if (!sc) return rt_fail(RT_ERR_INVALID_ARG, "scene is null");
    rt_split_params p = {RT_MODE_BVH, any_hit, 0.f, 0.f, 1, 0.f, 1.f, 0};
    return trace_common(sc, nullptr, rays, n, &p, hits, nullptr, stream);
}

extern "C" rt_status rt_trace_sdf(const rt_sdf* sdf, const rt_ray* rays, int64_t n, const rt_split_params* params,
                                  rt_hit* hits, void* stream)
{
    if (!sdf || !params) return rt_fail(RT_ERR_INVALID_ARG, "null grid or params");
    rt_split_params p = *params;
    p.mode = RT_MODE_SDF;
    return trace_common(nullptr, sdf, rays, n, &p, hits, nullptr, stream);
}

extern "C" rt_status rt_trace_combined(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* rays, int64_t n,
                                       const rt_split_params* params, rt_hit* hits, void* stream)
{
    return trace_common(sc, sdf, rays, n, params, hits, nullptr, stream);
}

// copy streams and events of the host-to-host pipeline, per device
namespace {
constexpr int kMaxChunks = 64;
constexpr int kComputeStreams = 4;
struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr;
    cudaStream_t comp[kComputeStreams] = {};
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t ev_in[kMaxChunks] = {}, ev_tr[kMaxChunks] = {};
    bool ready = false;
};
std::mutex g_pipe_mu;
HostPipe g_pipe[64];

rt_status host_pipe(HostPipe*& out)
{
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return rt_fail(RT_ERR_INVALID_ARG, "device %d out of range", dev);
    HostPipe& p = g_pipe[dev];
    if (!p.ready) {
        RT_CUDA_TRY(cudaStreamCreateWithFlags(&p.in, cudaStreamNonBlocking));
        RT_CUDA_TRY(cudaStreamCreateWithFlags(&p.out, cudaStreamNonBlocking));
        for (int c = 0; c < kComputeStreams; ++c) RT_CUDA_TRY(cudaStreamCreateWithFlags(&p.comp[c], cudaStreamNonBlocking));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming));
        for (int c = 0; c < kMaxChunks; ++c) {
            RT_CUDA_TRY(cudaEventCreateWithFlags(&p.ev_in[c], cudaEventDisableTiming));
            RT_CUDA_TRY(cudaEventCreateWithFlags(&p.ev_tr[c], cudaEventDisableTiming));
        }
        p.ready = true;
    }
    out = &p;
    return RT_OK;
}
}  // namespace

extern "C" rt_status rt_trace_combined_host(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* h_rays, int64_t n,
                                            const rt_split_params* params, rt_hit* h_hits, rt_ray* d_rays,
                                            rt_hit* d_hits, int32_t chunks, void* stream)
{
    rt_status st = check_params(params);
    if (st != RT_OK) return st;
    st = check_io(d_rays, n, d_hits);
    if (st != RT_OK) return st;
    if (n > 0 && (!h_rays || !h_hits)) return rt_fail(RT_ERR_INVALID_ARG, "null host ray or hit buffer");
    if (chunks < 0 || chunks > kMaxChunks) return rt_fail(RT_ERR_INVALID_ARG, "chunks %d not in 0..%d", chunks, kMaxChunks);
    if (n == 0) return RT_OK;
    if (chunks == 0) chunks = 4;
    if (chunks > n) chunks = (int32_t)n;
    // the library's copy streams are shared by all callers on this device
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe* p = nullptr;
    st = host_pipe(p);
    if (st != RT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RT_CUDA_TRY(cudaEventRecord(p->start, s));
    RT_CUDA_TRY(cudaStreamWaitEvent(p->in, p->start, 0));
    RT_CUDA_TRY(cudaStreamWaitEvent(p->out, p->start, 0));
    // pieces are traced on alternating compute streams: the tail of one piece's
    // persistent stage kernels (its slowest queries) overlaps the next piece
    const int ncomp = chunks < kComputeStreams ? chunks : kComputeStreams;
    for (int c = 0; c < ncomp; ++c) RT_CUDA_TRY(cudaStreamWaitEvent(p->comp[c], p->start, 0));
    // the first and last pieces are half as large as the others: the pipeline
    // fills (first upload) and drains (last download) sooner
    const int64_t weight_total = chunks >= 3 ? 2 * (int64_t)chunks - 2 : chunks;
    int64_t done_w = 0;
    for (int c = 0; c < chunks; ++c) {
        const int64_t w = (chunks >= 3 && (c == 0 || c == chunks - 1)) ? 1 : (chunks >= 3 ? 2 : 1);
        const int64_t b = n * done_w / weight_total;
        done_w += w;
        const int64_t m = n * done_w / weight_total - b;
        if (m <= 0) continue;
        cudaStream_t cs = p->comp[c % ncomp];
        RT_CUDA_TRY(cudaMemcpyAsync(d_rays + b, h_rays + b, (size_t)m * sizeof(rt_ray), cudaMemcpyHostToDevice, p->in));
        RT_CUDA_TRY(cudaEventRecord(p->ev_in[c], p->in));
        RT_CUDA_TRY(cudaStreamWaitEvent(cs, p->ev_in[c], 0));
        st = trace_common(sc, sdf, d_rays + b, m, params, d_hits + b, nullptr, cs, nullptr, false);
        if (st != RT_OK) return st;
        RT_CUDA_TRY(cudaEventRecord(p->ev_tr[c], cs));
        RT_CUDA_TRY(cudaStreamWaitEvent(p->out, p->ev_tr[c], 0));
        RT_CUDA_TRY(cudaMemcpyAsync(h_hits + b, d_hits + b, (size_t)m * sizeof(rt_hit), cudaMemcpyDeviceToHost, p->out));
    }
    RT_CUDA_TRY(cudaEventRecord(p->done, p->out));
    RT_CUDA_TRY(cudaStreamWaitEvent(s, p->done, 0));
    return RT_OK;
}

extern "C" rt_status rt_trace_combined_counted(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* rays, int64_t n,
                                               const rt_split_params* params, rt_hit* hits,
                                               unsigned long long* counters, void* stream)
{
    if (!counters) return rt_fail(RT_ERR_INVALID_ARG, "counters is null");
    return trace_common(sc, sdf, rays, n, params, hits, counters, stream);
}

extern "C" rt_status rt_trace_combined_backward(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* rays, int64_t n,
                                                const rt_split_params* params, const rt_hit* hits,
                                                const float* grad_t, float* grad_grid, void* stream)
{
    rt_status st = check_params(params);
    if (st != RT_OK) return st;
    st = check_io(rays, n, hits);
    if (st != RT_OK) return st;
    if (!sdf) return rt_fail(RT_ERR_INVALID_ARG, "grid is null");
    if (sdf->dtype != RT_GRID_F32) return rt_fail(RT_ERR_INVALID_ARG, "backward needs a float32 grid");
    if (sdf->levels > 0) return rt_fail(RT_ERR_INVALID_ARG, "backward does not take a cascade");
    if (n > 0 && (!grad_t || !grad_grid)) return rt_fail(RT_ERR_INVALID_ARG, "null gradient buffer");
    if (params->mode != RT_MODE_SDF && params->mode != RT_MODE_BVH && !sc)
        return rt_fail(RT_ERR_INVALID_ARG, "combined modes need the scene");
    if (n == 0) return RT_OK;
    TraceArgs a;
    st = rt_fill_trace_args(a, params->mode == RT_MODE_SDF ? nullptr : sc, sdf, params);
    if (st != RT_OK) return st;
    a.rays = reinterpret_cast<const float4*>(rays);
    a.hits = const_cast<rt_hit*>(hits);
    a.n = n;
    return rt_launch_backward(a, grad_t, grad_grid, (cudaStream_t)stream);
}
