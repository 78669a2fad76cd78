// Trace kernels.  A query (Eq. 1) is split into the sub-intervals of Eq. 2 and
// processed by the ordering rule of Section 2: a closest-hit query runs its
// sub-intervals in order and stops at the first that hits; an any-hit query
// runs the distance-field sub-interval first.
//
// Two implementations with identical results:
//   * wavefront (stage kernels): one persistent kernel per sub-interval kind
//     (triangles near, field, triangles far); a kind no query of the call has
//     is not launched.  Each lane holds one query and takes a new one from a
//     global counter once enough lanes of its warp are idle (per-lane refill:
//     all 32 for triangles, which keeps coherent rays together, 16 for the
//     field, whose marches end after very different step counts).  Queries
//     that miss a sub-interval are appended to the queue of the next kind:
//     rays that switch tracer mid-query are regrouped across the whole batch
//     instead of diverging inside a warp.
//   * simple: one thread per query runs all of its sub-intervals.
// The default (RT_KERNEL_AUTO) takes the stage kernels.
#include <mutex>

#include "rt_trace_dev.cuh"

using namespace rtdev;

namespace {

constexpr unsigned kFull = 0xffffffffu;
#ifndef RT_FIELD_BUDGET
#define RT_FIELD_BUDGET 4
#endif
constexpr int kFieldBudget = RT_FIELD_BUDGET;  // march steps between two refill checks

// ---------------------------------------------------------------------------
// simple kernel: one thread per query
// ---------------------------------------------------------------------------
template <bool COUNT, int L, bool WIDE>
__device__ __forceinline__ void trace_one(const TraceArgs& a, int64_t i, Counts& cnt)
{
    const float4 r0 = __ldg(a.rays + 2 * i), r1 = __ldg(a.rays + 2 * i + 1);
    const float3 o = make_float3(r0.x, r0.y, r0.z), d = make_float3(r1.x, r1.y, r1.z);
    const float tmin = r0.w, tmax = r1.w;
    Hit h = {__int_as_float(0x7f800000), -1, 0.f, 0.f};
    uint32_t flags = 0;
    int32_t tracer = RT_TRACER_MISS;

    if (!valid_query(o, d, tmin, tmax)) {
    } else if (a.mode == RT_MODE_BVH) {
        if (bvh_segment<COUNT, WIDE>(a, o, d, tmin, tmax, a.any_hit, h, flags, cnt)) tracer = RT_TRACER_BVH;
    } else if (a.mode == RT_MODE_SDF) {
        March m = sdf_march<COUNT, L>(a, o, d, tmin, tmax, flags, cnt);
        if (m.hit) {
            tracer = RT_TRACER_SDF;
            h.t = (a.refine_root && !isnan(m.t_prev)) ? refine<L>(a, o, d, m.t_prev, m.t) : m.t;
        }
    } else {
        const Split s = make_split(a, o, d, tmin, tmax);
        if (a.any_hit) {
            if (s.field) {
                March m = sdf_march<COUNT, L>(a, o, d, s.t1, s.t2, flags, cnt);
                if (m.hit) {
                    tracer = RT_TRACER_SDF;
                    h.t = (a.refine_root && !isnan(m.t_prev)) ? refine<L>(a, o, d, m.t_prev, m.t) : m.t;
                }
            }
            if (tracer == RT_TRACER_MISS && s.near_bvh && bvh_segment<COUNT, WIDE>(a, o, d, tmin, s.t1, true, h, flags, cnt))
                tracer = RT_TRACER_BVH;
            if (tracer == RT_TRACER_MISS && s.far_bvh && bvh_segment<COUNT, WIDE>(a, o, d, s.t2, tmax, true, h, flags, cnt))
                tracer = RT_TRACER_BVH;
        } else {
            if (s.near_bvh && bvh_segment<COUNT, WIDE>(a, o, d, tmin, s.t1, false, h, flags, cnt)) tracer = RT_TRACER_BVH;
            if (tracer == RT_TRACER_MISS && s.field) {
                March m = sdf_march<COUNT, L>(a, o, d, s.t1, s.t2, flags, cnt);
                if (m.hit) {
                    tracer = RT_TRACER_SDF;
                    h.t = (a.refine_root && !isnan(m.t_prev)) ? refine<L>(a, o, d, m.t_prev, m.t) : m.t;
                }
            }
            if (tracer == RT_TRACER_MISS && s.far_bvh && bvh_segment<COUNT, WIDE>(a, o, d, s.t2, tmax, false, h, flags, cnt))
                tracer = RT_TRACER_BVH;
        }
    }
    if (tracer != RT_TRACER_BVH) {
        h.prim = -1;
        h.u = h.v = 0.f;
    }
    store_hit(a.hits + i, h.t, h.prim, h.u, h.v, tracer, flags);
}

__device__ __forceinline__ void flush_counts(const TraceArgs& a, const Counts& cnt)
{
    if (cnt.nodes) atomicAdd(&a.counters[0], (unsigned long long)cnt.nodes);
    if (cnt.tris) atomicAdd(&a.counters[1], (unsigned long long)cnt.tris);
    if (cnt.steps) atomicAdd(&a.counters[2], (unsigned long long)cnt.steps);
    if (cnt.field) atomicAdd(&a.counters[3], (unsigned long long)cnt.field);
}

template <bool COUNT, int L, bool WIDE>
__global__ void k_trace(const TraceArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Counts cnt = {0, 0, 0, 0};
    if (i < a.n) trace_one<COUNT, L, WIDE>(a, first_query(a, i), cnt);
    if (COUNT) flush_counts(a, cnt);
}

// ---------------------------------------------------------------------------
// wavefront stage kernels
// ---------------------------------------------------------------------------
enum StageKind { ST_BVH_FULL = 0, ST_BVH_NEAR = 1, ST_BVH_FAR = 2, ST_FIELD_FULL = 3, ST_FIELD_SPLIT = 4 };

struct StageArgs {
    int32_t kind;
    int32_t first;             // input = every query 0..n-1 (validity is checked here)
    const int2* in_items;      // (query, flags) appended by the previous stage
    const unsigned* in_count;
    int2* out_items;           // null: last stage, a miss is final
    unsigned* out_count;
    unsigned* fetch;           // work counter of this stage
    int32_t refill_min;
    int32_t trip;              // traversal iterations between refill checks (trip_budget)
    HitEntry* hit_list;        // non-null (near stage of the concurrent program): hits go here, misses write nothing
    unsigned* hit_count;
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// The bounds of this stage's sub-interval of the query (o, d, t_min, t_max).
// Returns false when the sub-interval is not part of the query (or the query
// is invalid).  more: the query has a later sub-interval in its program
// (Section 2: closest hit near, field, far; any hit field, near, far), so a
// miss here goes on to the next stage; otherwise the miss is final here.
__device__ __forceinline__ bool segment_bounds(const TraceArgs& a, int kind, float3 o, float3 d, float tmin,
                                               float tmax, float& ta, float& tb, bool& more)
{
    more = false;
    if (!valid_query(o, d, tmin, tmax)) return false;
    if (kind == ST_BVH_FULL || kind == ST_FIELD_FULL) {
        ta = tmin;
        tb = tmax;
        return true;
    }
    const Split s = make_split(a, o, d, tmin, tmax);
    if (kind == ST_BVH_NEAR) {
        ta = tmin;
        tb = s.t1;
        more = a.any_hit ? s.far_bvh : (s.field || s.far_bvh);
        return s.near_bvh;
    }
    if (kind == ST_BVH_FAR) { ta = s.t2; tb = tmax; return s.far_bvh; }
    ta = s.t1;
    tb = s.t2;
    more = a.any_hit ? (s.near_bvh || s.far_bvh) : s.far_bvh;
    return s.field;
}

// Load query q and the bounds of this stage's sub-interval.
__device__ __forceinline__ bool stage_segment(const TraceArgs& a, int kind, int64_t q, float3& o, float3& d,
                                              float& ta, float& tb, bool& more)
{
    const float4 r0 = __ldg(a.rays + 2 * q), r1 = __ldg(a.rays + 2 * q + 1);
    o = make_float3(r0.x, r0.y, r0.z);
    d = make_float3(r1.x, r1.y, r1.z);
    return segment_bounds(a, kind, o, d, r0.w, r1.w, ta, tb, more);
}

// Append the lanes with `fwd` set to the next stage's queue (one atomic per warp).
__device__ __forceinline__ void forward(const StageArgs& st, bool fwd, int query, uint32_t flags)
{
    const unsigned m = __ballot_sync(kFull, fwd);
    if (m == 0) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane_id() == (unsigned)leader) base = atomicAdd(st.out_count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (fwd) st.out_items[base + __popc(m & ((1u << lane_id()) - 1u))] = make_int2(query, (int)flags);
}

// Take new queries for the idle lanes when enough of them are idle (or all are).
// Sets `got` for the lanes that received query `slot`.
__device__ __forceinline__ void refill(const StageArgs& st, unsigned n_in, bool idle, bool& drained, bool& got,
                                       unsigned& slot)
{
    got = false;
    const unsigned want = __ballot_sync(kFull, idle && !drained);
    const unsigned busy = __ballot_sync(kFull, !idle);
    if (want == 0 || (__popc(want) < st.refill_min && busy != 0)) return;
    const int leader = __ffs(want) - 1;
    unsigned base = 0;
    if (lane_id() == (unsigned)leader) base = atomicAdd(st.fetch, (unsigned)__popc(want));
    base = __shfl_sync(kFull, base, leader);
    if (idle && !drained) {
        const unsigned k = base + __popc(want & ((1u << lane_id()) - 1u));
        if (k < n_in) {
            got = true;
            slot = k;
        } else {
            drained = true;
        }
    }
}

// 56 registers: 9 resident blocks of 128 per SM (61 without the cap, 8 blocks);
// measured on the 1080p GI workload: near stage 0.238 -> 0.224 ms
#ifndef RT_BVH_REGS
#define RT_BVH_REGS 56
#endif
template <bool COUNT, bool WIDE>
__global__ void __maxnreg__(RT_BVH_REGS) k_stage_bvh(const TraceArgs a, const StageArgs st)
{
    const unsigned n_in = st.first ? (unsigned)a.n : *st.in_count;
    const bool any_hit = a.any_hit != 0;
    typename TravOf<WIDE>::entry stack[TravOf<WIDE>::depth];
    Counts cnt = {0, 0, 0, 0};
    bool drained = false, live = false, more = false;
    int query = -1;
    uint32_t flags = 0;
    BvhRay r;
    typename TravOf<WIDE>::state s;
    Hit best;
    for (;;) {
        bool got;
        unsigned slot = 0;
        refill(st, n_in, !live, drained, got, slot);
        bool done = false, found = false;
        if (got) {
            int2 item = st.first ? make_int2((int)first_query(a, slot), 0) : st.in_items[slot];
            query = item.x;
            flags = (uint32_t)item.y;
            float3 o, d;
            float ta, tb;
            bool active = stage_segment(a, st.kind, query, o, d, ta, tb, more);
            if (active && ta <= tb && a.root != INT32_MIN) {
                r = bvh_ray(o, d);
                s = tbegin<WIDE>(a, r, ta, tb);
                best.prim = -1;
                live = true;
            } else {
                done = true;
            }
        } else if (live) {
            if (ttrip<COUNT, WIDE>(a, r, s, stack, any_hit, best, flags, cnt, st.trip)) {
                done = true;
                found = s.found;
                live = false;
            }
        }
        const bool fwd = done && !found && more && st.out_items != nullptr;
        forward(st, fwd, query, flags);
        if (st.hit_list) {
            // concurrent program: the field stage writes every record; a near hit
            // replaces it, a near miss's flags join it (k_merge_hits)
            if (done && !found) best.prim = kFlagsOnly;
            append_hit_entry(st.hit_list, st.hit_count, done && (found || flags != 0u), a.hits + query, best, flags);
        } else if (done && !fwd) {
            if (found) store_hit(a.hits + query, best.t, best.prim, best.u, best.v, RT_TRACER_BVH, flags);
            else store_hit(a.hits + query, __int_as_float(0x7f800000), -1, 0.f, 0.f, RT_TRACER_MISS, flags);
        }
        if (__ballot_sync(kFull, live || (!drained)) == 0) break;
    }
    if (COUNT) flush_counts(a, cnt);
}

// The near hits of the concurrent program over the field's records: a hit in
// the near sub-interval is the closest hit (Section 2: sub-intervals in order)
__global__ void __launch_bounds__(256) k_merge_hits(const HitEntry* __restrict__ list, const unsigned* __restrict__ count)
{
    const unsigned n = *count;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const HitEntry e = list[i];
        if (e.prim == kFlagsOnly) {
            uint32_t* f = reinterpret_cast<uint32_t*>(e.dst) + 5;  // the record's flags word
            *f |= e.flags;
        } else {
            store_hit(e.dst, e.t, e.prim, e.u, e.v, RT_TRACER_BVH, e.flags);
        }
    }
}

// 40 registers: 12 resident blocks of 128 threads per SM; more march chains in
// flight hide more of the cell-load latency (measured: 0.596 vs 0.616 ms field-only)
#ifndef RT_FIELD_REGS
#define RT_FIELD_REGS 40
#endif
template <bool COUNT, int L>
__global__ void __maxnreg__(RT_FIELD_REGS) k_stage_field(const TraceArgs a, const StageArgs st)
{
    const unsigned n_in = st.first ? (unsigned)a.n : *st.in_count;
    Counts cnt = {0, 0, 0, 0};
    bool drained = false, live = false, more = false;
    int query = -1;
    uint32_t flags = 0;
    float3 o = make_float3(0.f, 0.f, 0.f), d = o;
    float t = 0.f, tb = 0.f, t_prev = 0.f;
    int k = 0;
    for (;;) {
        bool got;
        unsigned slot = 0;
        refill(st, n_in, !live, drained, got, slot);
        bool done = false, found = false;
        if (got) {
            int2 item = st.first ? make_int2((int)first_query(a, slot), 0) : st.in_items[slot];
            query = item.x;
            flags = (uint32_t)item.y;
            float ta;
            bool active = stage_segment(a, st.kind, query, o, d, ta, tb, more);
            if (active && clip_grid(a, o, d, ta, tb)) {
                if (COUNT) ++cnt.field;
                t = ta;
                t_prev = __int_as_float(0x7fc00000);
                k = 0;
                live = true;
            } else {
                done = true;
            }
        } else if (live) {
            // several march steps between two refill checks
            for (int it = 0; it < kFieldBudget; ++it) {
                if (COUNT) ++cnt.steps;
                const int res = march_step<L>(a, o, d, t, tb, t_prev);
                ++k;
                if (res == 1) {
                    done = true;
                    found = true;
                } else if (res == 2) {
                    done = true;
                } else if (k >= a.max_steps) {
                    flags |= RT_FLAG_STEP_LIMIT;
                    done = true;
                }
                if (done) break;
            }
            if (done) live = false;
        }
        const bool fwd = done && !found && more && st.out_items != nullptr;
        forward(st, fwd, query, flags);
        if (done && !fwd) {
            if (found) {
                const float th = (a.refine_root && !isnan(t_prev)) ? refine<L>(a, o, d, t_prev, t) : t;
                store_hit(a.hits + query, th, -1, 0.f, 0.f, RT_TRACER_SDF, flags);
            } else {
                store_hit(a.hits + query, __int_as_float(0x7f800000), -1, 0.f, 0.f, RT_TRACER_MISS, flags);
            }
        }
        if (__ballot_sync(kFull, live || (!drained)) == 0) break;
    }
    if (COUNT) flush_counts(a, cnt);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct DeviceInfo {
    int sms = 0;
    cudaMemPool_t pool = nullptr;
};

std::mutex g_mu;
DeviceInfo g_dev[64];

rt_status device_info(DeviceInfo*& out)
{
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return rt_fail(RT_ERR_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo& d = g_dev[dev];
    if (d.sms == 0) {
        RT_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        RT_CUDA_TRY(cudaMemPoolCreate(&d.pool, &props));
        // keep freed scratch in the pool between calls instead of returning it
        uint64_t keep = ~0ull;
        RT_CUDA_TRY(cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    out = &d;
    return RT_OK;
}

template <class K>
int persistent_blocks(K kernel, int block, const rt_tuning& tu, int sms)
{
    int per_sm = tu.blocks_per_sm;
    if (per_sm <= 0) {
        int fit = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, block, 0) != cudaSuccess || fit < 1) fit = 1;
        per_sm = fit;
    }
    return sms * per_sm;
}

template <bool COUNT>
rt_status launch_stage(const TraceArgs& a, const StageArgs& st, const rt_tuning& tu, int sms, cudaStream_t s)
{
    const bool field = st.kind == ST_FIELD_FULL || st.kind == ST_FIELD_SPLIT;
    if (field) {
        switch (grid_layout_of(a)) {
#define RT_FIELD_CASE(LL)                                                                  \
    case LL: {                                                                             \
        int blocks = persistent_blocks(k_stage_field<COUNT, LL>, tu.block, tu, sms);       \
        k_stage_field<COUNT, LL><<<blocks, tu.block, 0, s>>>(a, st);                       \
        break;                                                                             \
    }
            RT_FIELD_CASE(GL_PLAIN_F32)
            RT_FIELD_CASE(GL_PLAIN_F16)
            RT_FIELD_CASE(GL_CELLS_F32)
            RT_FIELD_CASE(GL_CELLS_F16)
            RT_FIELD_CASE(GL_PAIRS_F32)
            RT_FIELD_CASE(GL_PAIRS_F16)
            RT_FIELD_CASE(GL_CASC_F32)
            RT_FIELD_CASE(GL_CASC_F16)
#undef RT_FIELD_CASE
        }
    } else if (a.wnodes) {
        int blocks = persistent_blocks(k_stage_bvh<COUNT, true>, tu.block, tu, sms);
        k_stage_bvh<COUNT, true><<<blocks, tu.block, 0, s>>>(a, st);
    } else {
        int blocks = persistent_blocks(k_stage_bvh<COUNT, false>, tu.block, tu, sms);
        k_stage_bvh<COUNT, false><<<blocks, tu.block, 0, s>>>(a, st);
    }
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// the sub-interval kinds of a query, in the order Section 2 processes them
int stage_program(const TraceArgs& a, int kinds[3])
{
    switch (a.mode) {
    case RT_MODE_BVH: kinds[0] = ST_BVH_FULL; return 1;
    case RT_MODE_SDF: kinds[0] = ST_FIELD_FULL; return 1;
    default: {
        // a triangle sub-interval whose multiplier is 0 is empty for every query:
        // its stage would only pass the queries on, so it is not launched (the
        // neighbouring field stage then takes every query, or writes the final misses)
        const bool near = a.m_near > 0.f, far = a.mode == RT_MODE_SPLIT2 && a.m_far > 0.f;
        int n = 0;
        if (a.any_hit) {
            kinds[n++] = ST_FIELD_SPLIT;
            if (near) kinds[n++] = ST_BVH_NEAR;
        } else {
            if (near) kinds[n++] = ST_BVH_NEAR;
            kinds[n++] = ST_FIELD_SPLIT;
        }
        if (far) kinds[n++] = ST_BVH_FAR;
        return n;
    }
    }
}

int32_t public_kind(int k)
{
    switch (k) {
    case ST_BVH_FULL: return RT_STAGE_BVH_FULL;
    case ST_BVH_NEAR: return RT_STAGE_BVH_NEAR;
    case ST_BVH_FAR: return RT_STAGE_BVH_FAR;
    case ST_FIELD_FULL: return RT_STAGE_FIELD_FULL;
    default: return RT_STAGE_FIELD_SPLIT;
    }
}

// Streams and events of the concurrent programs, one set per device, and the
// lock that keeps one call's fork-to-join sequence of launches together.
std::mutex g_conc_mu;
ConcStreams g_conc[64];

// Work counters sit 128 bytes apart: atomics of different counters, from one
// kernel or from two running side by side, then never share an L2 line.
constexpr int kCtrStride = 32;

// start / end of timed part k on stream s
struct Marks {
    StageTiming* t;
    int part = 0;
    rt_status begin(cudaStream_t s, int32_t kind)
    {
        if (!t) return RT_OK;
        if (part >= kMaxTimedParts) return rt_fail(RT_ERR_INVALID_ARG, "too many timed parts");
        t->kinds[part] = kind;
        cudaError_t e = cudaEventRecord(t->events[2 * part], s);
        return e == cudaSuccess ? RT_OK : rt_cuda_fail(e, "cudaEventRecord");
    }
    rt_status end(cudaStream_t s)
    {
        if (!t) return RT_OK;
        cudaError_t e = cudaEventRecord(t->events[2 * part + 1], s);
        ++part;
        t->n_launches = part;
        return e == cudaSuccess ? RT_OK : rt_cuda_fail(e, "cudaEventRecord");
    }
};

StageArgs stage_args(int kind, const rt_tuning& tu)
{
    StageArgs sa = {};
    sa.kind = kind;
    sa.refill_min = (kind == ST_FIELD_FULL || kind == ST_FIELD_SPLIT) ? tu.refill_min_field : tu.refill_min;
    sa.trip = trip_budget(sa.refill_min);
    return sa;
}

// The concurrent program of a closest-hit split call (near triangles, field[,
// far triangles]): the near stage and the field stage are independent except
// for which record wins, so they run at the same time on two streams.  The
// near stage (after the query order) traces every query's near sub-interval
// and lists its hits; the field stage traces every query's field sub-interval
// from t_1 in input order and writes every record (passing its misses to the
// far stage, which writes theirs); then k_merge_hits puts each near hit over
// its query's record, since a near hit is the closest hit.  The records equal
// those of the stages run in sequence.
template <bool COUNT>
rt_status run_concurrent(const TraceArgs& a, const int kinds[3], int n_st, const rt_tuning& tu, DeviceInfo* dev,
                         cudaStream_t s, Marks& marks)
{
    ConcStreams* cs = nullptr;
    std::lock_guard<std::mutex> lk(g_conc_mu);
    rt_status st = rt_conc_streams(cs);
    if (st != RT_OK) return st;
    const bool far = n_st > 2;
    const size_t counters_bytes = 8 * kCtrStride * sizeof(unsigned);
    const size_t order_bytes = rt_order_bytes(a.ob, a.n);
    const size_t list_bytes = (size_t)a.n * sizeof(HitEntry);
    const size_t queue_bytes = far ? (size_t)a.n * sizeof(int2) : 0;
    void* scratch = nullptr;
    RT_CUDA_TRY(cudaMallocFromPoolAsync(&scratch, counters_bytes + order_bytes + list_bytes + queue_bytes, dev->pool, s));
    char* base = static_cast<char*>(scratch);
    unsigned* ctr = reinterpret_cast<unsigned*>(base);
    HitEntry* list = reinterpret_cast<HitEntry*>(base + counters_bytes + order_bytes);
    int2* queue = reinterpret_cast<int2*>(base + counters_bytes + order_bytes + list_bytes);
    rt_status rs = RT_OK;
    cudaError_t e = cudaMemsetAsync(ctr, 0, counters_bytes, s);
    if (e == cudaSuccess) e = cudaEventRecord(cs->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs->near, cs->fork, 0);
    if (e != cudaSuccess) rs = rt_cuda_fail(e, "concurrent program set-up");
    rt_tuning tn = tu, tf = tu;
    if (tu.blocks_per_sm == 0) {
        tn.blocks_per_sm = kConcNearBlocks;
        tf.blocks_per_sm = kConcFieldBlocks;
    }
    // near stream: the order, then the near stage
    TraceArgs ao = a;
    if (rs == RT_OK && order_bytes) {
        rs = marks.begin(cs->near, RT_STAGE_ORDER);
        OrderRays src = {};
        src.rays[0] = a.rays;
        src.count = 1;
        if (rs == RT_OK) rs = rt_launch_order(ao, src, base + counters_bytes, cs->near);
        if (rs == RT_OK) rs = marks.end(cs->near);
    }
    // the field stage starts with the near stage, after the order: started
    // beside the order kernel, its blocks would hold the SMs the order and then
    // the near stage need
    if (rs == RT_OK) {
        e = cudaEventRecord(cs->ordered, cs->near);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs->field, cs->ordered, 0);
        if (e != cudaSuccess) rs = rt_cuda_fail(e, "concurrent program set-up");
    }
    if (rs == RT_OK) {
        StageArgs sa = stage_args(kinds[0], tu);
        sa.first = 1;
        sa.fetch = &ctr[0 * kCtrStride];
        sa.hit_list = list;
        sa.hit_count = &ctr[6 * kCtrStride];
        rs = marks.begin(cs->near, public_kind(kinds[0]));
        if (rs == RT_OK) rs = launch_stage<COUNT>(ao, sa, tn, dev->sms, cs->near);
        if (rs == RT_OK) rs = marks.end(cs->near);
    }
    // field stream: the field stage over every query in input order, then the far stage
    TraceArgs af = a;
    af.qorder = nullptr;
    if (rs == RT_OK) {
        StageArgs sa = stage_args(kinds[1], tu);
        sa.first = 1;
        sa.fetch = &ctr[1 * kCtrStride];
        if (far) {
            sa.out_items = queue;
            sa.out_count = &ctr[3 * kCtrStride];
        }
        rs = marks.begin(cs->field, public_kind(kinds[1]));
        if (rs == RT_OK) rs = launch_stage<COUNT>(af, sa, tf, dev->sms, cs->field);
        if (rs == RT_OK) rs = marks.end(cs->field);
    }
    if (rs == RT_OK && far) {
        StageArgs sa = stage_args(kinds[2], tu);
        sa.in_items = queue;
        sa.in_count = &ctr[3 * kCtrStride];
        sa.fetch = &ctr[2 * kCtrStride];
        rs = marks.begin(cs->field, public_kind(kinds[2]));
        if (rs == RT_OK) rs = launch_stage<COUNT>(af, sa, tf, dev->sms, cs->field);
        if (rs == RT_OK) rs = marks.end(cs->field);
    }
    // then a second near stage on the field stream, at full residency, sharing
    // the first's work counter and hit list: when the near sub-intervals are the
    // larger share of the work (short rays), it finishes them once the field
    // is done; otherwise it finds the counter drained and ends at once
    if (rs == RT_OK) {
        StageArgs sa = stage_args(kinds[0], tu);
        sa.first = 1;
        sa.fetch = &ctr[0 * kCtrStride];
        sa.hit_list = list;
        sa.hit_count = &ctr[6 * kCtrStride];
        rs = marks.begin(cs->field, RT_STAGE_BVH_NEAR_REST);
        if (rs == RT_OK) rs = launch_stage<COUNT>(ao, sa, tu, dev->sms, cs->field);
        if (rs == RT_OK) rs = marks.end(cs->field);
    }
    // join, then the near hits over the field's records
    e = cudaEventRecord(cs->near_done, cs->near);
    if (e == cudaSuccess) e = cudaEventRecord(cs->field_done, cs->field);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, cs->near_done, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, cs->field_done, 0);
    if (rs == RT_OK && e != cudaSuccess) rs = rt_cuda_fail(e, "concurrent program join");
    if (rs == RT_OK) {
        rs = marks.begin(s, RT_STAGE_MERGE);
        if (rs == RT_OK) rs = rt_launch_merge_hits(list, &ctr[6 * kCtrStride], dev->sms, s);
        if (rs == RT_OK) rs = marks.end(s);
    }
    e = cudaFreeAsync(scratch, s);
    if (rs == RT_OK && e != cudaSuccess) rs = rt_cuda_fail(e, "cudaFreeAsync");
    return rs;
}

template <bool COUNT>
rt_status run_wavefront(const TraceArgs& a, const rt_tuning& tu, cudaStream_t s, StageTiming* timing,
                        bool allow_concurrent)
{
    DeviceInfo* dev = nullptr;
    rt_status st = device_info(dev);
    if (st != RT_OK) return st;
    if (a.n > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "at most 2^31-1 queries per call");
    int kinds[3];
    const int n_st = stage_program(a, kinds);
    Marks marks{timing};
    if (timing) timing->n_launches = 0;
    // closest-hit split calls: the near and field stages at the same time (not
    // with m_near = +inf, where the field sub-interval is empty for every query)
    if (allow_concurrent && n_st >= 2 && kinds[0] == ST_BVH_NEAR && !a.any_hit && !isinf(a.m_near))
        return run_concurrent<COUNT>(a, kinds, n_st, tu, dev, s, marks);
    // scratch: counters (fetch x3, queue sizes x2), the query order, and two
    // ping-pong queues
    const size_t counters_bytes = 8 * kCtrStride * sizeof(unsigned);
    const size_t order_bytes = rt_order_bytes(a.ob, a.n);
    const size_t queue_bytes = n_st > 1 ? (size_t)a.n * sizeof(int2) : 0;
    const size_t total = counters_bytes + order_bytes + (n_st > 1 ? queue_bytes : 0) + (n_st > 2 ? queue_bytes : 0);
    void* scratch = nullptr;
    RT_CUDA_TRY(cudaMallocFromPoolAsync(&scratch, total, dev->pool, s));
    char* base = static_cast<char*>(scratch);
    unsigned* ctr = reinterpret_cast<unsigned*>(base);
    int2* q[2] = {reinterpret_cast<int2*>(base + counters_bytes + order_bytes),
                  reinterpret_cast<int2*>(base + counters_bytes + order_bytes + queue_bytes)};
    rt_status rs = RT_OK;
    cudaError_t e = cudaMemsetAsync(ctr, 0, counters_bytes, s);
    if (e != cudaSuccess) rs = rt_cuda_fail(e, "cudaMemsetAsync");
    TraceArgs ao = a;  // with the query order
    if (order_bytes && rs == RT_OK) {
        rs = marks.begin(s, RT_STAGE_ORDER);
        OrderRays src = {};
        src.rays[0] = a.rays;
        src.count = 1;
        if (rs == RT_OK) rs = rt_launch_order(ao, src, base + counters_bytes, s);
        if (rs == RT_OK) rs = marks.end(s);
    }
    for (int k = 0; k < n_st && rs == RT_OK; ++k) {
        StageArgs sa = stage_args(kinds[k], tu);
        sa.first = k == 0;
        sa.in_items = k > 0 ? q[(k - 1) & 1] : nullptr;
        sa.in_count = k > 0 ? &ctr[(3 + ((k - 1) & 1)) * kCtrStride] : nullptr;
        sa.out_items = k + 1 < n_st ? q[k & 1] : nullptr;
        sa.out_count = k + 1 < n_st ? &ctr[(3 + (k & 1)) * kCtrStride] : nullptr;
        sa.fetch = &ctr[k * kCtrStride];
        rs = marks.begin(s, public_kind(kinds[k]));
        if (rs == RT_OK) rs = launch_stage<COUNT>(ao, sa, tu, dev->sms, s);
        if (rs == RT_OK) rs = marks.end(s);
    }
    e = cudaFreeAsync(scratch, s);
    if (rs == RT_OK && e != cudaSuccess) rs = rt_cuda_fail(e, "cudaFreeAsync");
    return rs;
}

template <bool C, bool W>
void launch_simple(const TraceArgs& a, int L, unsigned nb, int block, cudaStream_t s)
{
    switch (L) {
    case GL_PLAIN_F32: k_trace<C, GL_PLAIN_F32, W><<<nb, block, 0, s>>>(a); break;
    case GL_PLAIN_F16: k_trace<C, GL_PLAIN_F16, W><<<nb, block, 0, s>>>(a); break;
    case GL_CELLS_F32: k_trace<C, GL_CELLS_F32, W><<<nb, block, 0, s>>>(a); break;
    case GL_CELLS_F16: k_trace<C, GL_CELLS_F16, W><<<nb, block, 0, s>>>(a); break;
    case GL_PAIRS_F32: k_trace<C, GL_PAIRS_F32, W><<<nb, block, 0, s>>>(a); break;
    case GL_PAIRS_F16: k_trace<C, GL_PAIRS_F16, W><<<nb, block, 0, s>>>(a); break;
    case GL_CASC_F32: k_trace<C, GL_CASC_F32, W><<<nb, block, 0, s>>>(a); break;
    default: k_trace<C, GL_CASC_F16, W><<<nb, block, 0, s>>>(a); break;
    }
}

}  // namespace

std::mutex& rt_conc_mutex() { return g_conc_mu; }

rt_status rt_conc_streams(ConcStreams*& out)
{
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return rt_fail(RT_ERR_INVALID_ARG, "device %d out of range", dev);
    ConcStreams& c = g_conc[dev];
    if (!c.ready) {
        // the near stream at the highest priority: when both stages have blocks
        // waiting for room (after the order kernel), the near stage's are placed
        // first, and the field stage's fill the rest of each SM
        int least = 0, greatest = 0;
        RT_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        RT_CUDA_TRY(cudaStreamCreateWithPriority(&c.near, cudaStreamNonBlocking, greatest));
        RT_CUDA_TRY(cudaStreamCreateWithPriority(&c.field, cudaStreamNonBlocking, least));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&c.ordered, cudaEventDisableTiming));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&c.near_done, cudaEventDisableTiming));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&c.field_done, cudaEventDisableTiming));
        c.ready = true;
    }
    out = &c;
    return RT_OK;
}

rt_status rt_launch_merge_hits(const HitEntry* list, const unsigned* count, int sms, cudaStream_t s)
{
    k_merge_hits<<<sms * 4, 256, 0, s>>>(list, count);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

rt_status rt_launch_trace(const TraceArgs& a0, bool counted, cudaStream_t s, StageTiming* timing,
                          bool allow_concurrent)
{
    const rt_tuning& tu = rt_current_tuning();
    TraceArgs a = a0;
    rt_apply_layout(a, tu);
    // AUTO: the stage kernels for every call; on triangles-only calls too they
    // were measured at least as fast as one thread per query on every ray kind
    const bool wavefront = tu.kernel == RT_KERNEL_WAVEFRONT || tu.kernel == RT_KERNEL_AUTO;
    if (wavefront)
        return counted ? run_wavefront<true>(a, tu, s, timing, allow_concurrent)
                       : run_wavefront<false>(a, tu, s, timing, allow_concurrent);
    const int64_t blocks = (a.n + tu.block - 1) / tu.block;
    if (blocks > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "too many rays");
    Marks marks{timing};
    if (timing) timing->n_launches = 0;
    void* scratch = nullptr;
    const size_t order_bytes = rt_order_bytes(a.ob, a.n);
    if (order_bytes) {
        // the query order, read by the kernel through a.qorder
        DeviceInfo* dev = nullptr;
        rt_status st = device_info(dev);
        if (st != RT_OK) return st;
        RT_CUDA_TRY(cudaMallocFromPoolAsync(&scratch, order_bytes, dev->pool, s));
        st = marks.begin(s, RT_STAGE_ORDER);
        OrderRays src = {};
        src.rays[0] = a.rays;
        src.count = 1;
        if (st == RT_OK) st = rt_launch_order(a, src, scratch, s);
        if (st == RT_OK) st = marks.end(s);
        if (st != RT_OK) {
            cudaFreeAsync(scratch, s);
            return st;
        }
    }
    rt_status st = marks.begin(s, RT_STAGE_ALL);
    cudaError_t e = cudaSuccess;
    if (st == RT_OK) {
        const unsigned nb = (unsigned)blocks;
        const int L = grid_layout_of(a);
        if (a.wnodes) {
            if (counted) launch_simple<true, true>(a, L, nb, tu.block, s);
            else launch_simple<false, true>(a, L, nb, tu.block, s);
        } else {
            if (counted) launch_simple<true, false>(a, L, nb, tu.block, s);
            else launch_simple<false, false>(a, L, nb, tu.block, s);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) st = marks.end(s);
    }
    if (scratch) {
        const cudaError_t ef = cudaFreeAsync(scratch, s);
        if (e == cudaSuccess) e = ef;
    }
    if (e != cudaSuccess) return rt_cuda_fail(e, "simple trace launch");
    return st;
}

// ---------------------------------------------------------------------------
// rt_trace_combined_noalloc: the wavefront trace with its scratch (the stage
// counters and the two queues) in one fixed device array of this file instead
// of memory taken from the pool on every call.  The array is sized for
// kNoAllocMaxRays queries and is part of the module: every device that loads
// the library holds it until the process exits.  Host code reaches it only
// through the address returned by cudaGetSymbolAddress (the array's name is a
// host-side stand-in, not a device address).
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxRays = (int64_t)1 << 20;
constexpr size_t kNoAllocCounterBytes = 256;
// the query order at its largest: one 4-byte entry per query of the largest call
constexpr size_t kNoAllocOrderBytes = (size_t)kNoAllocMaxRays * sizeof(int32_t);
constexpr size_t kNoAllocQueueBytes = (size_t)kNoAllocMaxRays * sizeof(int2);
constexpr size_t kNoAllocBytes = kNoAllocCounterBytes + kNoAllocOrderBytes + 2 * kNoAllocQueueBytes;
static_assert(kNoAllocOrderBytes % 256 == 0, "the queues stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    void* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sms = 0;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// once per device, with that device current: look up the array's device address
rt_status noalloc_setup(NoAllocDevice*& out)
{
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return rt_fail(RT_ERR_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.scratch) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return rt_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return rt_cuda_fail(e, "cudaDeviceGetAttribute");
        d.sms = sms;
        d.scratch = p;
    }
    out = &d;
    return RT_OK;
}

}  // namespace

extern "C" rt_status rt_trace_combined_noalloc(const rt_scene* sc, const rt_sdf* sdf, const rt_ray* rays, int64_t n,
                                               const rt_split_params* p, rt_hit* hits, void* stream)
{
    if (!p) return rt_fail(RT_ERR_INVALID_ARG, "params is null");
    if (p->mode < 0 || p->mode > 3) return rt_fail(RT_ERR_INVALID_ARG, "mode %d not in 0..3", p->mode);
    if (!(p->m_near >= 0.f) || !(p->m_far >= 0.f))
        return rt_fail(RT_ERR_INVALID_ARG, "multipliers must be >= 0 (got %g, %g)", p->m_near, p->m_far);
    if (p->max_steps < 1) return rt_fail(RT_ERR_INVALID_ARG, "max_steps must be >= 1");
    if (!(p->hit_eps_vox >= 0.f) || !(p->min_step_vox > 0.f) || isinf(p->hit_eps_vox) || isinf(p->min_step_vox))
        return rt_fail(RT_ERR_INVALID_ARG, "hit_eps_vox must be >= 0 and min_step_vox > 0, both finite");
    if (p->any_hit != 0 && p->any_hit != 1) return rt_fail(RT_ERR_INVALID_ARG, "any_hit must be 0 or 1");
    if (n < 0) return rt_fail(RT_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n > kNoAllocMaxRays)
        return rt_fail(RT_ERR_INVALID_ARG,
                       "rt_trace_combined_noalloc takes at most %lld queries per call (got %lld); split the batch "
                       "or use rt_trace_combined", (long long)kNoAllocMaxRays, (long long)n);
    if (p->mode != RT_MODE_SDF && !sc) return rt_fail(RT_ERR_INVALID_ARG, "mode %d needs a scene", p->mode);
    if (p->mode != RT_MODE_BVH && !sdf) return rt_fail(RT_ERR_INVALID_ARG, "mode %d needs a grid", p->mode);
    if (n == 0) return RT_OK;
    if (!rays || !hits) return rt_fail(RT_ERR_INVALID_ARG, "null ray or hit buffer");
    if (((uintptr_t)rays & 15u) != 0) return rt_fail(RT_ERR_INVALID_ARG, "ray buffer not 16-byte aligned");
    if (((uintptr_t)hits & 7u) != 0) return rt_fail(RT_ERR_INVALID_ARG, "hit buffer not 8-byte aligned");
    int cur = -1;
    RT_CUDA_TRY(cudaGetDevice(&cur));
    if (sc && p->mode != RT_MODE_SDF && sc->device != cur)
        return rt_fail(RT_ERR_INVALID_ARG, "scene belongs to device %d, current is %d", sc->device, cur);
    if (sdf && p->mode != RT_MODE_BVH && sdf->device != cur)
        return rt_fail(RT_ERR_INVALID_ARG, "grid belongs to device %d, current is %d", sdf->device, cur);
    NoAllocDevice* dev = nullptr;
    rt_status st = noalloc_setup(dev);
    if (st != RT_OK) return st;

    TraceArgs a;
    st = rt_fill_trace_args(a, p->mode == RT_MODE_SDF ? nullptr : sc, p->mode == RT_MODE_BVH ? nullptr : sdf, p);
    if (st != RT_OK) return st;
    a.rays = reinterpret_cast<const float4*>(rays);
    a.hits = hits;
    a.n = n;
    a.counters = nullptr;
    if (!rt_order_applies(*p)) a.ob.bits = 0;
    const rt_tuning& tu = rt_current_tuning();
    rt_apply_layout(a, tu);
    cudaStream_t s = (cudaStream_t)stream;

    int kinds[3];
    const int n_st = stage_program(a, kinds);
    unsigned char* base = static_cast<unsigned char*>(dev->scratch);
    unsigned* ctr = reinterpret_cast<unsigned*>(base);
    int2* q[2] = {reinterpret_cast<int2*>(base + kNoAllocCounterBytes + kNoAllocOrderBytes),
                  reinterpret_cast<int2*>(base + kNoAllocCounterBytes + kNoAllocOrderBytes + kNoAllocQueueBytes)};
    // every call starts from zeroed counters (the array keeps the last call's contents)
    RT_CUDA_TRY(cudaMemsetAsync(ctr, 0, kNoAllocCounterBytes, s));
    if (rt_order_bytes(a.ob, a.n) > kNoAllocOrderBytes)
        return rt_fail(RT_ERR_INVALID_ARG, "query order larger than its fixed scratch");
    OrderRays src = {};
    src.rays[0] = a.rays;
    src.count = 1;
    st = rt_launch_order(a, src, base + kNoAllocCounterBytes, s);
    if (st != RT_OK) return st;
    for (int k = 0; k < n_st; ++k) {
        StageArgs sa = stage_args(kinds[k], tu);
        sa.first = k == 0;
        sa.in_items = k > 0 ? q[(k - 1) & 1] : nullptr;
        sa.in_count = k > 0 ? &ctr[3 + ((k - 1) & 1)] : nullptr;
        sa.out_items = k + 1 < n_st ? q[k & 1] : nullptr;
        sa.out_count = k + 1 < n_st ? &ctr[3 + (k & 1)] : nullptr;
        sa.fetch = &ctr[k];
        sa.refill_min = (kinds[k] == ST_FIELD_FULL || kinds[k] == ST_FIELD_SPLIT) ? tu.refill_min_field : tu.refill_min;
        sa.trip = trip_budget(sa.refill_min);
        st = launch_stage<false>(a, sa, tu, dev->sms, s);
        if (st != RT_OK) return st;
    }
    return RT_OK;
}
