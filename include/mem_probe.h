/*
 * mem_probe.h -- memory-system probes that give the roofline of the combined
 * ray query library its denominators.  Measurement only: none of these is a
 * query, and the query library (rt_api.h) does not use them.  Built as a
 * library of its own (libmem_probe.so).
 *
 * Rules shared by every entry point
 *   - Buffers are DEVICE memory owned by the caller; `stream` is a
 *     cudaStream_t passed as void* (NULL = legacy default stream); the work is
 *     enqueued asynchronously on it.
 *   - Return 0 on success, 1 for an invalid argument (detected on the host,
 *     before anything is enqueued), 2 when a CUDA call fails;
 *     mp_last_error() then gives a message (thread-local).
 */
#ifndef GB300_MEM_PROBE_H
#define GB300_MEM_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Dependent random 32-byte gathers: the access of one march step of the
 * field tracer (Section 3 of the paper; sphere tracing reads one 32-byte cell
 * whose address depends on the previous step), with no locality.  blocks x 128
 * chains of `steps` gathers each over d_cells:
 *   d_cells  n_cells x 32 bytes (8 float32), 32-byte aligned; n_cells a power
 *            of two in [1, 2^31]
 *   chain i  starts at cell fmix32(i + 1) & (n_cells - 1) (fmix32: the 32-bit
 *            finaliser of MurmurHash3); a step at cell c loads its 8 floats v,
 *            adds v[0] + v[7] to the chain's sum (float32, in order) and moves
 *            to fmix32(c ^ bits(v[3]) ^ s) & (n_cells - 1), s the step number
 *   d_out    blocks x 128 float32, 4-byte aligned: each chain's sum
 * Errors: 1 for null or misaligned buffers, n_cells not a power of two,
 * steps < 1, blocks outside [1, 2^20]. */
int mp_random_gather(const void* d_cells, int64_t n_cells, int32_t steps, int32_t blocks, float* d_out,
                     void* stream);

/* L2 read bandwidth: blocks x 256 threads read the n_bytes of d_buf `reps`
 * times over, 16 bytes per load, through L2 only (ld.global.cg: not cached in
 * L1), thread t taking the 16-byte words t, t + T, t + 2T, ... (T threads in
 * all), so every warp load is one coalesced 512-byte request.  With n_bytes
 * well below the L2 size every pass after the first is served from L2.
 *   d_buf   n_bytes, 16-byte aligned, n_bytes a multiple of 16 in [16, 2^40]
 *   d_out   blocks x 256 float32: each thread's sum of the x lanes it read
 * Errors: 1 for null or misaligned buffers, bad n_bytes, reps < 1, blocks
 * outside [1, 2^20]. */
int mp_l2_read(const void* d_buf, int64_t n_bytes, int32_t reps, int32_t blocks, float* d_out, void* stream);

/* L1 read bandwidth: block b reads its own window of `window` bytes of d_buf
 * (starting at b * window) `reps` times over, 16 bytes per load, cached in L1
 * (ld.global.ca); with a window that fits in L1 every pass after the first is
 * served from the SM's L1.
 *   d_buf   blocks x window bytes, 16-byte aligned; window a multiple of 4096
 *           in [4096, 131072]
 *   d_out   blocks x 256 float32
 * Errors: 1 for null or misaligned buffers, bad window, reps < 1, blocks
 * outside [1, 2^20]. */
int mp_l1_read(const void* d_buf, int32_t window, int32_t reps, int32_t blocks, float* d_out, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* mp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
