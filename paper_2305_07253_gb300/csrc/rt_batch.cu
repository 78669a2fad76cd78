// Mixed batches in one wavefront pipeline (rt_trace_batches).
//
// Each query follows the sub-interval program of its batch (Section 2: closest
// hit in order with early exit, any hit field first; Section 3: one split for
// AO/GI rays, two splits for shadow rays):
//   mode 0            : triangles [t_min, t_max]
//   mode 3            : field [t_min, t_max]
//   mode 1, closest   : triangles near, field
//   mode 1, any hit   : field, triangles near
//   mode 2, closest   : triangles near, field, triangles far
//   mode 2, any hit   : field, triangles near, triangles far
// The pipeline is four persistent launches -- triangles, field, triangles,
// triangles -- which covers every program above.  A query whose next sub-interval is not of
// a launch's kind passes through it to the next launch's queue.
//
// When some batch has closest-hit near sub-intervals (0 < m_near < inf), the
// first two launches run at the same time instead (the concurrent program,
// rt_internal.cuh): the triangle launch takes the queries that start with
// triangles, writes the records of triangles-only queries and lists the near
// hits; the field launch takes every query with a field sub-interval straight
// from the input, a closest-hit split query from t_1 as if its near
// sub-interval had missed.  The last two launches follow the field launch, a
// second triangle launch takes what the first left, and k_merge_hits puts the
// near hits over the records.
#include <mutex>

#include "rt_trace_dev.cuh"

using namespace rtdev;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBatchSteps = 4;  // march steps between refill checks

enum Seg { SEG_NONE = 0, SEG_B_FULL, SEG_F_FULL, SEG_B_NEAR, SEG_F_SPLIT, SEG_B_FAR };
constexpr int kLaunches = 4;  // triangles, field, triangles, triangles

struct BatchEntry {
    const float4* rays;
    rt_hit* hits;
    int64_t offset;
    int32_t mode, any_hit;
    float m_near, m_far;
};

struct BatchTable {
    BatchEntry e[RT_MAX_BATCHES];
    int32_t count;
};

struct Pipe {
    const int2* in_items;     // null: first launch, every query
    const unsigned* in_count;
    unsigned n_first;         // total queries (first launch)
    int2* out_items;          // null: last launch
    unsigned* out_count;
    unsigned* fetch;
    int32_t refill_min;
    int32_t trip;             // traversal iterations between refill checks (trip_budget)
    int32_t conc;             // kSequential, or the first triangle / field launch of the concurrent program
    HitEntry* hit_list;       // kConcTri: near hits of closest-hit split queries
    unsigned* hit_count;
};
constexpr int32_t kSequential = 0, kConcTri = 1, kConcField = 2;

__device__ __forceinline__ unsigned lane() { return threadIdx.x & 31u; }

__device__ __forceinline__ int seg_at(int mode, int any_hit, int p)
{
    switch (mode) {
    case RT_MODE_BVH: return p == 0 ? SEG_B_FULL : SEG_NONE;
    case RT_MODE_SDF: return p == 0 ? SEG_F_FULL : SEG_NONE;
    case RT_MODE_SPLIT1:
        if (any_hit) return p == 0 ? SEG_F_SPLIT : (p == 1 ? SEG_B_NEAR : SEG_NONE);
        return p == 0 ? SEG_B_NEAR : (p == 1 ? SEG_F_SPLIT : SEG_NONE);
    default:
        if (any_hit) return p == 0 ? SEG_F_SPLIT : (p == 1 ? SEG_B_NEAR : (p == 2 ? SEG_B_FAR : SEG_NONE));
        return p == 0 ? SEG_B_NEAR : (p == 1 ? SEG_F_SPLIT : (p == 2 ? SEG_B_FAR : SEG_NONE));
    }
}

__device__ __forceinline__ bool seg_is_field(int s) { return s == SEG_F_FULL || s == SEG_F_SPLIT; }

// the batch table, staged in shared memory once per block (lanes index it freely)
__device__ __forceinline__ void stage_table(const BatchTable& tb, BatchEntry* stb)
{
    for (int k = threadIdx.x; k < tb.count; k += blockDim.x) stb[k] = tb.e[k];
    __syncthreads();
}

__device__ __forceinline__ int find_batch(const BatchEntry* stb, int count, int64_t g)
{
    int lo = 0, hi = count - 1;  // last batch whose offset <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (stb[mid].offset <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void forward_item(const Pipe& pp, bool fwd, int2 item)
{
    const unsigned m = __ballot_sync(kFull, fwd);
    if (m == 0) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane() == (unsigned)leader) base = atomicAdd(pp.out_count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (fwd) pp.out_items[base + __popc(m & ((1u << lane()) - 1u))] = item;
}

__device__ __forceinline__ void take(const Pipe& pp, unsigned n_in, bool idle, bool& drained, bool& got, unsigned& slot)
{
    got = false;
    const unsigned want = __ballot_sync(kFull, idle && !drained);
    const unsigned busy = __ballot_sync(kFull, !idle);
    if (want == 0 || (__popc(want) < pp.refill_min && busy != 0)) return;
    const int leader = __ffs(want) - 1;
    unsigned base = 0;
    if (lane() == (unsigned)leader) base = atomicAdd(pp.fetch, (unsigned)__popc(want));
    base = __shfl_sync(kFull, base, leader);
    if (idle && !drained) {
        const unsigned k = base + __popc(want & ((1u << lane()) - 1u));
        if (k < n_in) { got = true; slot = k; } else drained = true;
    }
}

// queue item: x = global query index, y = flags | (program position << 8)
__device__ __forceinline__ int2 pack_item(int g, uint32_t flags, int p) { return make_int2(g, (int)(flags | (p << 8))); }

template <bool COUNT, bool WIDE>
__global__ void k_batch_bvh(const TraceArgs a, const BatchTable tb, const Pipe pp)
{
    __shared__ BatchEntry stb[RT_MAX_BATCHES];
    stage_table(tb, stb);
    const unsigned n_in = pp.in_items ? *pp.in_count : pp.n_first;
    rt_hit* hits = nullptr;  // this lane's batch output
    bool has_next = false;   // the query's program continues after this sub-interval
    typename TravOf<WIDE>::entry stack[TravOf<WIDE>::depth];
    Counts cnt = {0, 0, 0, 0};
    bool drained = false, live = false;
    int g = -1, p = 0, b = 0;
    int64_t qi = 0;
    uint32_t flags = 0;
    bool any_hit = false;
    bool listed = false;     // kConcTri: a closest-hit near sub-interval, whose hit goes to the list
    BvhRay r;
    typename TravOf<WIDE>::state s;
    Hit best;
    for (;;) {
        bool got;
        unsigned slot = 0;
        take(pp, n_in, !live, drained, got, slot);
        bool done = false, found = false, pass = false;
        if (got) {
            const int2 item = pp.in_items ? pp.in_items[slot] : make_int2((int)first_query(a, slot), 0);
            g = item.x;
            flags = (uint32_t)item.y & 0xffu;
            p = (item.y >> 8) & 0xff;
            b = find_batch(stb, tb.count, g);
            const BatchEntry e = stb[b];
            qi = g - e.offset;
            hits = e.hits;
            const int seg = seg_at(e.mode, e.any_hit, p);
            listed = pp.conc == kConcTri && seg == SEG_B_NEAR;
            const float4 r0 = __ldg(e.rays + 2 * qi), r1 = __ldg(e.rays + 2 * qi + 1);
            const float3 o = make_float3(r0.x, r0.y, r0.z), d = make_float3(r1.x, r1.y, r1.z);
            const float tmin = r0.w, tmax = r1.w;
            has_next = false;
            if (pp.conc == kConcTri && seg_is_field(seg)) {
                // the field launch beside this one takes the query
            } else if (!pp.in_items && !valid_query(o, d, tmin, tmax)) {
                // an invalid split query's miss is written by the field launch
                done = !listed;
                done = true;       // invalid: a miss, program over
            } else if (seg_is_field(seg)) {
                pass = true;       // not this launch's kind: hand on unchanged
                has_next = true;
            } else {
                has_next = seg_at(e.mode, e.any_hit, p + 1) != SEG_NONE;
                float ta = tmin, tb2 = tmax;
                bool active = true;
                if (seg != SEG_B_FULL) {
                    float hn, hf;
                    split_voxels(a, o, d, tmin, tmax, hn, hf);
                    const Split sp = make_split(e.mode, e.m_near, e.m_far, hn, hf, tmin, tmax);
                    if (seg == SEG_B_NEAR) { ta = tmin; tb2 = sp.t1; active = sp.near_bvh; }
                    else { ta = sp.t2; tb2 = tmax; active = sp.far_bvh; }
                }
                any_hit = e.any_hit != 0;
                if (active && ta <= tb2 && a.root != INT32_MIN) {
                    r = bvh_ray(o, d);
                    s = tbegin<WIDE>(a, r, ta, tb2);
                    best.prim = -1;
                    live = true;
                } else {
                    done = true;
                }
            }
        } else if (live) {
            if (ttrip<COUNT, WIDE>(a, r, s, stack, any_hit, best, flags, cnt, pp.trip)) {
                live = false;
                done = true;
                found = s.found;
            }
        }
        // after a miss the query moves to its next sub-interval, if any
        const bool more = (pass || (done && !found)) && has_next;
        const bool fwd = more && pp.out_items != nullptr;
        forward_item(pp, fwd, pack_item(g, flags, pass ? p : p + 1));
        if (pp.conc == kConcTri) {
            // a listed near sub-interval writes no record: its hit, or the flags
            // of its miss, go to the list
            if (done && listed && !found) best.prim = kFlagsOnly;
            append_hit_entry(pp.hit_list, pp.hit_count, done && listed && (found || flags != 0u), hits + qi, best, flags);
        }
        if ((done || pass) && !fwd && !listed) {
            if (found) store_hit(hits + qi, best.t, best.prim, best.u, best.v, RT_TRACER_BVH, flags);
            else store_hit(hits + qi, __int_as_float(0x7f800000), -1, 0.f, 0.f, RT_TRACER_MISS, flags);
        }
        if (__ballot_sync(kFull, live || !drained) == 0) break;
    }
    if (COUNT) {
        if (cnt.nodes) atomicAdd(&a.counters[0], (unsigned long long)cnt.nodes);
        if (cnt.tris) atomicAdd(&a.counters[1], (unsigned long long)cnt.tris);
    }
}

template <bool COUNT, int L>
__global__ void __maxnreg__(40) k_batch_field(const TraceArgs a, const BatchTable tb, const Pipe pp)
{
    __shared__ BatchEntry stb[RT_MAX_BATCHES];
    stage_table(tb, stb);
    const unsigned n_in = pp.in_items ? *pp.in_count : pp.n_first;
    rt_hit* hits = nullptr;
    bool has_next = false;
    Counts cnt = {0, 0, 0, 0};
    bool drained = false, live = false;
    int g = -1, p = 0, b = 0, k = 0;
    int64_t qi = 0;
    uint32_t flags = 0;
    float3 o = make_float3(0.f, 0.f, 0.f), d = o;
    float t = 0.f, tb2 = 0.f, t_prev = 0.f;
    for (;;) {
        bool got;
        unsigned slot = 0;
        take(pp, n_in, !live, drained, got, slot);
        bool done = false, found = false, pass = false;
        if (got) {
            const int2 item = pp.in_items ? pp.in_items[slot] : make_int2((int)first_query(a, slot), 0);
            g = item.x;
            flags = (uint32_t)item.y & 0xffu;
            p = (item.y >> 8) & 0xff;
            b = find_batch(stb, tb.count, g);
            const BatchEntry e = stb[b];
            qi = g - e.offset;
            hits = e.hits;
            int seg = seg_at(e.mode, e.any_hit, p);
            bool skip = false;
            if (pp.conc == kConcField) {
                // a closest-hit split query from t_1, as if its near sub-interval
                // had missed (the triangle launch beside this one traces that);
                // triangles-only queries are the triangle launch's alone
                if (seg == SEG_B_NEAR) seg = seg_at(e.mode, e.any_hit, ++p);
                skip = seg == SEG_B_FULL;
            }
            const float4 r0 = __ldg(e.rays + 2 * qi), r1 = __ldg(e.rays + 2 * qi + 1);
            o = make_float3(r0.x, r0.y, r0.z);
            d = make_float3(r1.x, r1.y, r1.z);
            const float tmin = r0.w, tmax = r1.w;
            has_next = false;
            if (skip) {
                // nothing to do here
            } else if (!pp.in_items && !valid_query(o, d, tmin, tmax)) {
                done = true;
            } else if (!seg_is_field(seg)) {
                pass = true;
                has_next = true;
            } else {
                has_next = seg_at(e.mode, e.any_hit, p + 1) != SEG_NONE;
                float ta = tmin;
                tb2 = tmax;
                bool active = true;
                if (seg == SEG_F_SPLIT) {
                    float hn, hf;
                    split_voxels(a, o, d, tmin, tmax, hn, hf);
                    const Split sp = make_split(e.mode, e.m_near, e.m_far, hn, hf, tmin, tmax);
                    ta = sp.t1;
                    tb2 = sp.t2;
                    active = sp.field;
                }
                if (active && clip_grid(a, o, d, ta, tb2)) {
                    if (COUNT) ++cnt.field;
                    t = ta;
                    t_prev = __int_as_float(0x7fc00000);
                    k = 0;
                    live = true;
                } else {
                    done = true;
                }
            }
        } else if (live) {
            for (int it = 0; it < kBatchSteps; ++it) {
                if (COUNT) ++cnt.steps;
                const int res = march_step<L>(a, o, d, t, tb2, t_prev);
                ++k;
                if (res == 1) { done = true; found = true; }
                else if (res == 2) done = true;
                else if (k >= a.max_steps) { flags |= RT_FLAG_STEP_LIMIT; done = true; }
                if (done) break;
            }
            if (done) live = false;
        }
        const bool more = (pass || (done && !found)) && has_next;
        const bool fwd = more && pp.out_items != nullptr;
        forward_item(pp, fwd, pack_item(g, flags, pass ? p : p + 1));
        if ((done || pass) && !fwd) {
            if (found) {
                const float th = (a.refine_root && !isnan(t_prev)) ? refine<L>(a, o, d, t_prev, t) : t;
                store_hit(hits + qi, th, -1, 0.f, 0.f, RT_TRACER_SDF, flags);
            } else {
                store_hit(hits + qi, __int_as_float(0x7f800000), -1, 0.f, 0.f, RT_TRACER_MISS, flags);
            }
        }
        if (__ballot_sync(kFull, live || !drained) == 0) break;
    }
    if (COUNT) {
        if (cnt.steps) atomicAdd(&a.counters[2], (unsigned long long)cnt.steps);
        if (cnt.field) atomicAdd(&a.counters[3], (unsigned long long)cnt.field);
    }
}

struct BatchDevice {
    int sms = 0;
    cudaMemPool_t pool = nullptr;
};
std::mutex g_bmu;
BatchDevice g_bdev[64];

rt_status batch_device(BatchDevice*& out)
{
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return rt_fail(RT_ERR_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchDevice& d = g_bdev[dev];
    if (d.sms == 0) {
        RT_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        RT_CUDA_TRY(cudaMemPoolCreate(&d.pool, &props));
        uint64_t keep = ~0ull;
        RT_CUDA_TRY(cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    out = &d;
    return RT_OK;
}

template <class K>
int grid_for(K kernel, const rt_tuning& tu, int sms)
{
    int per_sm = tu.blocks_per_sm;
    if (per_sm <= 0) {
        int fit = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, tu.block, 0) != cudaSuccess || fit < 1) fit = 1;
        per_sm = fit;
    }
    return sms * per_sm;
}

}  // namespace

extern "C" rt_status rt_trace_batches(const rt_scene* sc, const rt_sdf* sdf, const rt_batch* batches, int32_t n_batches,
                                      void* stream)
{
    if (!batches && n_batches > 0) return rt_fail(RT_ERR_INVALID_ARG, "batches is null");
    if (n_batches < 0 || n_batches > RT_MAX_BATCHES)
        return rt_fail(RT_ERR_INVALID_ARG, "n_batches %d not in 0..%d", n_batches, RT_MAX_BATCHES);
    BatchTable tb = {};
    int64_t total = 0;
    bool need_scene = false, need_grid = false;
    const rt_split_params* p0 = nullptr;
    for (int k = 0; k < n_batches; ++k) {
        const rt_batch& bt = batches[k];
        const rt_split_params& p = bt.params;
        if (p.mode < 0 || p.mode > 3) return rt_fail(RT_ERR_INVALID_ARG, "batch %d: mode %d", k, p.mode);
        if (!(p.m_near >= 0.f) || !(p.m_far >= 0.f)) return rt_fail(RT_ERR_INVALID_ARG, "batch %d: negative multiplier", k);
        if (p.any_hit != 0 && p.any_hit != 1) return rt_fail(RT_ERR_INVALID_ARG, "batch %d: any_hit", k);
        if (p.max_steps < 1 || !(p.hit_eps_vox >= 0.f) || !(p.min_step_vox > 0.f) || isinf(p.hit_eps_vox) ||
            isinf(p.min_step_vox))
            return rt_fail(RT_ERR_INVALID_ARG, "batch %d: bad march parameters", k);
        if (bt.n < 0) return rt_fail(RT_ERR_INVALID_ARG, "batch %d: n < 0", k);
        if (bt.n > 0 && (!bt.d_rays || !bt.d_hits)) return rt_fail(RT_ERR_INVALID_ARG, "batch %d: null buffer", k);
        if (((uintptr_t)bt.d_rays & 15u) || ((uintptr_t)bt.d_hits & 7u))
            return rt_fail(RT_ERR_INVALID_ARG, "batch %d: misaligned buffer", k);
        if (!p0) p0 = &p;
        else if (p.max_steps != p0->max_steps || p.hit_eps_vox != p0->hit_eps_vox ||
                 p.min_step_vox != p0->min_step_vox || p.refine_root != p0->refine_root)
            return rt_fail(RT_ERR_INVALID_ARG, "batch %d: march parameters differ from batch 0", k);
        need_scene |= p.mode != RT_MODE_SDF;
        need_grid |= p.mode != RT_MODE_BVH;
        tb.e[k].rays = reinterpret_cast<const float4*>(bt.d_rays);
        tb.e[k].hits = bt.d_hits;
        tb.e[k].offset = total;
        tb.e[k].mode = p.mode;
        tb.e[k].any_hit = p.any_hit;
        tb.e[k].m_near = p.m_near;
        tb.e[k].m_far = p.m_far;
        total += bt.n;
    }
    tb.count = n_batches;
    if (total > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "more than 2^31-1 queries");
    if (need_scene && !sc) return rt_fail(RT_ERR_INVALID_ARG, "a batch needs the scene");
    if (need_grid && !sdf) return rt_fail(RT_ERR_INVALID_ARG, "a batch needs the grid");
    if (total == 0) return RT_OK;
    int cur = -1;
    RT_CUDA_TRY(cudaGetDevice(&cur));
    if (need_scene && sc->device != cur) return rt_fail(RT_ERR_INVALID_ARG, "scene belongs to another device");
    if (need_grid && sdf->device != cur) return rt_fail(RT_ERR_INVALID_ARG, "grid belongs to another device");
    BatchDevice* dev = nullptr;
    rt_status st = batch_device(dev);
    if (st != RT_OK) return st;

    TraceArgs a;
    st = rt_fill_trace_args(a, need_scene ? sc : nullptr, need_grid ? sdf : nullptr, p0);
    if (st != RT_OK) return st;
    const rt_tuning& tu = rt_current_tuning();
    rt_apply_layout(a, tu);
    a.n = total;
    a.counters = nullptr;
    // closest-hit near sub-intervals in some batch: the query order (unless the
    // tuning turns it off) and the concurrent program
    bool near_split = false;
    int64_t n_listed = 0;  // queries whose near hit may be listed
    for (int k = 0; k < n_batches; ++k) {
        const bool ns = batches[k].n > 0 && rt_order_applies(batches[k].params);
        near_split |= ns;
        const rt_split_params& p = batches[k].params;
        if ((p.mode == RT_MODE_SPLIT1 || p.mode == RT_MODE_SPLIT2) && !p.any_hit) n_listed += batches[k].n;
    }
    if (!near_split) a.ob.bits = 0;
    const bool conc = near_split;
    cudaStream_t s = (cudaStream_t)stream;

    const size_t ctr_bytes = 256, qbytes = (size_t)total * sizeof(int2), order_bytes = rt_order_bytes(a.ob, total);
    const size_t list_bytes = conc ? (size_t)n_listed * sizeof(HitEntry) : 0;
    void* scratch = nullptr;
    RT_CUDA_TRY(cudaMallocFromPoolAsync(&scratch, ctr_bytes + order_bytes + 2 * qbytes + list_bytes, dev->pool, s));
    char* base = static_cast<char*>(scratch);
    unsigned* ctr = reinterpret_cast<unsigned*>(base);
    int2* q[2] = {reinterpret_cast<int2*>(base + ctr_bytes + order_bytes),
                  reinterpret_cast<int2*>(base + ctr_bytes + order_bytes + qbytes)};
    HitEntry* list = reinterpret_cast<HitEntry*>(base + ctr_bytes + order_bytes + 2 * qbytes);
    unsigned* hit_count = &ctr[16];
    rt_status rs = RT_OK;
    cudaError_t e = cudaMemsetAsync(ctr, 0, ctr_bytes, s);
    if (e != cudaSuccess) rs = rt_cuda_fail(e, "cudaMemsetAsync");

    ConcStreams* cs = nullptr;
    std::unique_lock<std::mutex> lk(rt_conc_mutex(), std::defer_lock);
    cudaStream_t s_tri = s, s_field = s;  // the streams of the first two launches
    if (conc && rs == RT_OK) {
        lk.lock();
        rs = rt_conc_streams(cs);
        if (rs == RT_OK) {
            e = cudaEventRecord(cs->fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs->near, cs->fork, 0);
            if (e != cudaSuccess) rs = rt_cuda_fail(e, "concurrent program set-up");
            s_tri = cs->near;
            s_field = cs->field;
        }
    }
    if (order_bytes && rs == RT_OK) {
        // the queries of every batch in one order, as one index space
        OrderRays src = {};
        for (int k = 0; k < n_batches; ++k) {
            src.rays[k] = tb.e[k].rays;
            src.offset[k] = tb.e[k].offset;
        }
        src.count = n_batches;
        rs = rt_launch_order(a, src, base + ctr_bytes, s_tri);
    }
    if (conc && rs == RT_OK) {
        // the field launch starts after the order kernel, whose SMs its blocks would take
        e = cudaEventRecord(cs->ordered, cs->near);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs->field, cs->ordered, 0);
        if (e != cudaSuccess) rs = rt_cuda_fail(e, "concurrent program set-up");
    }
    TraceArgs af = a;  // the concurrent field launch reads the input in its own order
    if (conc) af.qorder = nullptr;
    // launches: triangles, field, triangles, triangles; ctr[k] = fetch counter of
    // launch k, ctr[8 + k] = number of queries launch k hands on (queues ping-pong);
    // in the concurrent program the first launch hands nothing on, and a fifth
    // (a second first launch, sharing its counter and list) follows the fourth
    const int n_launch = conc ? kLaunches + 1 : kLaunches;
    for (int k = 0; k < n_launch && rs == RT_OK; ++k) {
        const bool helper = k == kLaunches;
        const int kk = helper ? 0 : k;
        Pipe pp;
        // the concurrent field launch, like the first, takes every query from the input
        const bool from_input = kk == 0 || (conc && kk == 1);
        pp.in_items = from_input ? nullptr : q[(kk - 1) & 1];
        pp.in_count = from_input ? nullptr : &ctr[8 + kk - 1];
        pp.n_first = (unsigned)total;
        pp.out_items = kk + 1 < kLaunches && !(conc && kk == 0) ? q[kk & 1] : nullptr;
        pp.out_count = pp.out_items ? &ctr[8 + kk] : nullptr;
        pp.fetch = &ctr[kk];
        pp.refill_min = kk == 1 ? tu.refill_min_field : tu.refill_min;
        pp.trip = trip_budget(pp.refill_min);
        pp.conc = !conc ? kSequential : (kk == 0 ? kConcTri : (kk == 1 ? kConcField : kSequential));
        pp.hit_list = list;
        pp.hit_count = hit_count;
        rt_tuning tk = tu;
        if (conc && tu.blocks_per_sm == 0 && !helper && kk <= 1) tk.blocks_per_sm = kk == 0 ? kConcNearBlocks : kConcFieldBlocks;
        const cudaStream_t sk = !conc ? s : (k == 0 ? s_tri : s_field);
        const TraceArgs& ak = kk == 1 ? af : a;
        if (kk == 1 && need_grid) {
            switch (grid_layout_of(a)) {
#define RT_BATCH_FIELD(LL)                                                                                     \
    case LL:                                                                                                   \
        k_batch_field<false, LL><<<grid_for(k_batch_field<false, LL>, tk, dev->sms), tu.block, 0, sk>>>(ak, tb, pp); \
        break;
                RT_BATCH_FIELD(GL_PLAIN_F32)
                RT_BATCH_FIELD(GL_PLAIN_F16)
                RT_BATCH_FIELD(GL_CELLS_F32)
                RT_BATCH_FIELD(GL_CELLS_F16)
                RT_BATCH_FIELD(GL_PAIRS_F32)
                RT_BATCH_FIELD(GL_PAIRS_F16)
                RT_BATCH_FIELD(GL_CASC_F32)
                RT_BATCH_FIELD(GL_CASC_F16)
#undef RT_BATCH_FIELD
            }
        } else if (kk == 1) {
            // no batch uses the field: pass everything through an empty field launch
            k_batch_field<false, GL_PLAIN_F32><<<grid_for(k_batch_field<false, GL_PLAIN_F32>, tk, dev->sms), tu.block, 0, sk>>>(
                ak, tb, pp);
        } else if (a.wnodes) {
            k_batch_bvh<false, true><<<grid_for(k_batch_bvh<false, true>, tk, dev->sms), tu.block, 0, sk>>>(ak, tb, pp);
        } else {
            k_batch_bvh<false, false><<<grid_for(k_batch_bvh<false, false>, tk, dev->sms), tu.block, 0, sk>>>(ak, tb, pp);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) rs = rt_cuda_fail(e, "stage launch");
    }
    if (conc && cs) {
        // join (also after a failed launch, so that no library stream is left
        // waiting on this call), then the near hits over the records
        e = cudaEventRecord(cs->near_done, cs->near);
        if (e == cudaSuccess) e = cudaEventRecord(cs->field_done, cs->field);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, cs->near_done, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, cs->field_done, 0);
        if (rs == RT_OK && e != cudaSuccess) rs = rt_cuda_fail(e, "concurrent program join");
        if (rs == RT_OK) rs = rt_launch_merge_hits(list, hit_count, dev->sms, s);
    }
    e = cudaFreeAsync(scratch, s);
    if (rs == RT_OK && e != cudaSuccess) rs = rt_cuda_fail(e, "cudaFreeAsync");
    return rs;
}
