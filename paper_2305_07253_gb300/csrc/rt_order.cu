// Query order for the trace kernels (rt_tuning.order_bits).
//
// A call's records do not depend on the order in which its queries are
// traced; its speed does.  A warp runs 32 queries at once, and a warp whose
// queries start in one region of the scene reads the same tree nodes,
// triangles and field cells in all its lanes.  Queries that are neighbours in
// the input are not always neighbours in space: those of one screen tile, for
// instance, can start on surfaces at very different depths.
//
// The order groups each window of kOrderWindow (1024) consecutive queries by
// a key: the cell that holds the query's origin, in a 2^b x 2^b x 2^b lattice
// over the scene's box (origins outside the box fall in the nearest cell).  Windows keep their order, and within a window the
// queries of one cell become neighbours; the first kernel of the call then
// takes query qorder[0], qorder[1], ...
//
// One persistent launch: each block takes windows in turn and copies the
// next window's origins into shared memory (cp.async) while it groups the
// current one.  A window holds few distinct keys, so the block counts them in
// a shared-memory hash table (open addressing, one slot per query; a key that
// finds no slot is counted apart, after all others), lists the slots in use,
// scans their counts, and writes each query at its key's start plus its rank.
// The groups come in the order their keys were first met, and a group's
// queries in about input order.
#include <algorithm>
#include <atomic>

#include "rt_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
#ifndef RT_ORDER_THREADS
#define RT_ORDER_THREADS 128
#endif
constexpr int kOrderThreads = RT_ORDER_THREADS;
constexpr int kOrderItems = 1024 / kOrderThreads;
constexpr int kOrderWindow = kOrderThreads * kOrderItems;  // queries per window
constexpr int kSlots = kOrderWindow;
static_assert(kSlots == 1 << 10, "slot_of hashes to 10 bits");

__device__ __forceinline__ int32_t order_key(const OrderBox& ob, float4 r0)
{
    const float p[3] = {r0.x, r0.y, r0.z};
    const float top = (float)((1 << ob.bits) - 1);
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // fmaxf returns the other operand for a NaN: such an origin lands in cell 0
        const float f = fminf(fmaxf((p[a] - ob.lo[a]) * ob.scale[a], 0.f), top);
        c[a] = (uint32_t)f;
    }
    // only equality of keys matters within a window: the cell's coordinates, packed
    return (int32_t)(c[0] | (c[1] << ob.bits) | (c[2] << (2 * ob.bits)));
}

// the slot of key (inserted if new; fresh = this call inserted it), -1 if
// every slot holds another key
__device__ __forceinline__ int slot_of(int32_t* skey, int32_t key, bool& fresh)
{
    uint32_t h = ((uint32_t)key * 0x9e3779b1u) >> 22;
    for (int probe = 0; probe < kSlots; ++probe, h = (h + 1u) & (kSlots - 1)) {
        const int32_t prev = atomicCAS(&skey[h], -1, key);
        fresh = prev == -1;
        if (fresh || prev == key) return (int)h;
    }
    fresh = false;
    return -1;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_last() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// start copying the origins (first float4 of each ray) of window w into buf;
// item j of thread t is query w kOrderWindow + j kOrderThreads + t
__device__ __forceinline__ void fetch_window(const OrderRays& src, int64_t n, int64_t w, float4* buf)
{
#pragma unroll
    for (int j = 0; j < kOrderItems; ++j) {
        const int64_t g = w * kOrderWindow + (int64_t)j * kOrderThreads + threadIdx.x;
        if (g < n) {
            int b = 0;
            for (int k = 1; k < src.count; ++k)
                if (src.offset[k] <= g) b = k;
            cp_async16(&buf[j * kOrderThreads + threadIdx.x], src.rays[b] + 2 * (g - src.offset[b]));
        }
    }
}

__global__ void __launch_bounds__(kOrderThreads) k_order_local(const OrderRays src, const OrderBox ob, int64_t n,
                                                               int64_t windows, int32_t* __restrict__ qorder)
{
    __shared__ float4 sray[2][kOrderWindow];
    __shared__ int32_t skey[kSlots];
    __shared__ unsigned scount[kSlots];      // queries per slot, then the slot's start
    __shared__ int16_t slist[kOrderWindow];  // the slots in use, in the order they were taken
    __shared__ unsigned nused, nover, warp_sum[kOrderThreads / 32];
    const unsigned lane = threadIdx.x & 31u;
    int64_t w = blockIdx.x;
    if (w >= windows) return;
    int cur = 0;
    fetch_window(src, n, w, sray[0]);
    cp_async_commit();
    for (; w < windows; w += gridDim.x, cur ^= 1) {
        // the next window's copy runs while this one is grouped; the buffer it
        // fills was last read before the previous window's second barrier
        if (w + gridDim.x < windows) fetch_window(src, n, w + gridDim.x, sray[cur ^ 1]);
        cp_async_commit();
        for (int i = threadIdx.x; i < kSlots; i += kOrderThreads) {
            skey[i] = -1;
            scount[i] = 0u;
        }
        if (threadIdx.x == 0) nused = nover = 0u;
        cp_async_wait_all_but_last();
        __syncthreads();  // this window's origins are in sray[cur]; the table is clear

        const int64_t w0 = w * kOrderWindow;
        int sl[kOrderItems];         // slot; -1: counted apart; -2: no query
        unsigned rank[kOrderItems];  // rank among the slot's queries (or among those counted apart)
#pragma unroll
        for (int j = 0; j < kOrderItems; ++j) {
            const int64_t g = w0 + (int64_t)j * kOrderThreads + threadIdx.x;
            const int32_t key = g < n ? order_key(ob, sray[cur][j * kOrderThreads + threadIdx.x]) : -1;
            const unsigned peers = __match_any_sync(kFull, key);
            const int leader = __ffs(peers) - 1;
            int s = -1;
            unsigned base = 0u;
            if (key >= 0 && (int)lane == leader) {
                bool fresh;
                s = slot_of(skey, key, fresh);
                if (fresh) slist[atomicAdd(&nused, 1u)] = (int16_t)s;
                base = s >= 0 ? atomicAdd(&scount[s], (unsigned)__popc(peers))
                              : atomicAdd(&nover, (unsigned)__popc(peers));
            }
            s = __shfl_sync(kFull, s, leader);
            base = __shfl_sync(kFull, base, leader);
            sl[j] = key >= 0 ? s : -2;
            rank[j] = base + __popc(peers & ((1u << lane) - 1u));
        }
        __syncthreads();

        // starts of the slots in use: an exclusive scan of their counts in list
        // order; thread t owns list entries kOrderItems t ...
        const unsigned nu = nused;
        unsigned c[kOrderItems], sum = 0u;
#pragma unroll
        for (int k = 0; k < kOrderItems; ++k) {
            const unsigned i = threadIdx.x * kOrderItems + k;
            c[k] = i < nu ? scount[slist[i]] : 0u;
            sum += c[k];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31u) warp_sum[threadIdx.x >> 5] = incl;
        __syncthreads();
        unsigned run = incl - sum, total = 0u;
#pragma unroll
        for (int v = 0; v < kOrderThreads / 32; ++v) {
            if (v < (int)(threadIdx.x >> 5)) run += warp_sum[v];
            total += warp_sum[v];
        }
        // each slot is listed once, so every thread writes only its own entries' slots
#pragma unroll
        for (int k = 0; k < kOrderItems; ++k) {
            const unsigned i = threadIdx.x * kOrderItems + k;
            if (i < nu) scount[slist[i]] = run;
            run += c[k];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kOrderItems; ++j) {
            if (sl[j] == -2) continue;
            const unsigned pos = sl[j] >= 0 ? scount[sl[j]] + rank[j] : total + rank[j];
            qorder[w0 + pos] = (int32_t)(w0 + (int64_t)j * kOrderThreads + threadIdx.x);
        }
        __syncthreads();  // the table and warp_sum are read above before the next window clears them
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy left in flight
}

constexpr int kMaxDevices = 64;
std::atomic<int> g_resident[kMaxDevices];  // resident blocks of k_order_local per device (0: not looked up)

}  // namespace

size_t rt_order_bytes(const OrderBox& ob, int64_t n)
{
    if (ob.bits < 1 || n < kOrderMin) return 0;
    return ((size_t)n * sizeof(int32_t) + 255) & ~(size_t)255;
}

rt_status rt_launch_order(TraceArgs& a, const OrderRays& src, void* scratch, cudaStream_t s)
{
    const OrderBox& ob = a.ob;
    a.qorder = nullptr;
    if (ob.bits < 1 || a.n < kOrderMin) return RT_OK;  // nothing to sort
    if (ob.bits > kOrderMaxBits) return rt_fail(RT_ERR_INVALID_ARG, "query order: %d bits", ob.bits);
    if (a.n > 0x7fffffffLL) return rt_fail(RT_ERR_INVALID_ARG, "query order: n = %lld", (long long)a.n);
    if (src.count < 1 || src.count > RT_MAX_BATCHES || src.offset[0] != 0)
        return rt_fail(RT_ERR_INVALID_ARG, "query order: %d ray segments", src.count);
    if (!scratch || ((uintptr_t)scratch & 255u) != 0)
        return rt_fail(RT_ERR_INVALID_ARG, "query order: scratch not 256-byte aligned");
    int32_t* qorder = static_cast<int32_t*>(scratch);
    const int64_t windows = (a.n + kOrderWindow - 1) / kOrderWindow;
    // persistent: as many blocks as fit at once (or one per window); the
    // figure is looked up once per device
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return rt_fail(RT_ERR_INVALID_ARG, "device %d out of range", dev);
    int resident = g_resident[dev].load(std::memory_order_relaxed);
    if (resident == 0) {
        int sms = 0, per_sm = 0;
        RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        RT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_order_local, kOrderThreads, 0));
        resident = sms * std::max(per_sm, 1);
        g_resident[dev].store(resident, std::memory_order_relaxed);
    }
    const int64_t blocks = std::min<int64_t>(windows, resident);
    k_order_local<<<(unsigned)blocks, kOrderThreads, 0, s>>>(src, ob, a.n, windows, qorder);
    RT_CUDA_TRY(cudaGetLastError());
    a.qorder = qorder;
    return RT_OK;
}
