/*
 * radix_gb300 — MSD radix sorting of fixed-size records on one GPU (sm_103a).
 *
 * The method is RADULS2 (M. Kokot, S. Deorowicz, M. Dlugosz, "Even faster sorting of
 * (not only) integers", 2017), re-designed for the GPU.  Section 1 of the paper states the
 * problem (order records by a key made of digits; radix sort processes one digit per phase
 * with a counting sort), section 3.1 the method (an MSD radix sort with 1-byte digits:
 * distribute the whole array by the first digit, then process the bins independently, and
 * hand tiny bins to a dedicated sorter), sections 3.2-3.3 the small- and tiny-bin steps.
 *
 * Records.  A record is rec_size bytes (a multiple of 8, at most 256).  Its key is bytes
 * [0, key_size) read as a little-endian unsigned integer (1 <= key_size <= 16, and
 * key_size <= rec_size): byte key_size-1 is the most significant, so for key_size = 8 the key
 * is the native uint64 at offset 0, and for key_size = 16 the word at bytes 8..15 is compared
 * before the word at bytes 0..7.  The other bytes are data that moves with the key.
 *
 * Order.  The result is the stable sort by key: keys are non-decreasing and records with
 * equal keys keep their input order.  It is therefore unique and byte-identical to a stable
 * LSD radix sort of the same records.
 *
 * Memory.  All record buffers are device memory owned by the caller; the library never
 * allocates, frees or keeps them.  The library owns a metadata workspace per (device,
 * stream) — histograms, bucket bases, per-segment run starts, bin and chunk lists, a status word —
 * allocated on first use with cudaMalloc (so the first call for a given size must not be
 * made while the stream is being captured into a CUDA graph), grown when a larger call
 * needs it, reused, and freed by radix_sort_release().
 *
 * Asynchrony.  Every call validates its arguments on the host and returns at once; the
 * work runs asynchronously on `stream` (NULL = the legacy default stream).  Errors found on
 * the device (a list that overflowed, a destination that failed its range check) set the
 * status word and are reported by radix_sort_status() after the stream has drained; no
 * kernel traps.  No kernel waits for another CTA; the only device-side waits are those of a
 * CTA for its own bulk copies into shared memory, each bounded (rs_plan.watchdog_polls) and
 * reported as RS_ERR_DEVICE_TIMEOUT when it runs out.  Once a step of a call has failed, the
 * call's later kernels do nothing (its result is undefined; `in` is left as the failed step
 * left it).  Calls on one stream run in order; calls on different streams use different
 * workspaces and may overlap.
 *
 * Errors.  A call that returns anything but RS_OK launched no work.
 */
#ifndef RADIX_GB300_H
#define RADIX_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *rs_stream_t; /* a cudaStream_t */

typedef enum rs_status {
  RS_OK = 0,
  RS_ERR_INVALID_ARG = 1,    /* a size or pointer argument is out of range */
  RS_ERR_MISALIGNED = 2,     /* a record buffer is not 16-byte aligned */
  RS_ERR_OVERLAP = 3,        /* the two record buffers overlap */
  RS_ERR_TOO_LARGE = 4,      /* n * rec_size does not fit in 64 bits / in the address space */
  RS_ERR_NO_MEMORY = 5,      /* the workspace could not be allocated */
  RS_ERR_CUDA = 6,           /* a CUDA runtime call failed (launch, memcpy, sync) */
  RS_ERR_DEVICE_TIMEOUT = 7, /* a bulk copy into shared memory did not land within its bounded wait */
  RS_ERR_QUEUE_OVERFLOW = 8, /* a device-side list overflowed (result undefined) */
  RS_ERR_UNSUPPORTED = 9,    /* a valid request this build does not handle (key_size > 16) */
  RS_ERR_INTERNAL = 10       /* a device-side consistency check failed (result undefined) */
} rs_status;

/*
 * Sort n records in place.
 *   in        device pointer, n * rec_size bytes, 16-byte aligned: the records; on
 *             completion they are in key order (section 1: the sorted sequence).
 *   tmp       device pointer, n * rec_size bytes, 16-byte aligned, not overlapping `in`:
 *             scratch (the other buffer of every distribution pass); contents undefined after.
 *   n         number of records (n <= 1: nothing is launched).
 *   rec_size  bytes per record: a multiple of 8, 8..256.
 *   key_size  key bytes: 1..16, <= rec_size.
 *   stream    CUDA stream for all work.
 */
rs_status radix_sort(void *in, void *tmp, uint64_t n, uint32_t rec_size, uint32_t key_size,
                     rs_stream_t stream);

/*
 * Sort n records that live in HOST memory: copy them to the device, sort, copy them back.
 *   h_in      HOST pointer, n * rec_size bytes: the records (read).
 *   h_out     HOST pointer, n * rec_size bytes: receives the sorted records; may equal h_in.
 *             Page-locked (pinned) host memory makes both copies asynchronous; with pageable
 *             memory the CUDA runtime stages them and the call may return later.
 *   d_buf     DEVICE pointer, n * rec_size bytes, 16-byte aligned: holds the records on the
 *             device (sorted there, then copied out).
 *   d_tmp     DEVICE pointer, n * rec_size bytes, 16-byte aligned, not overlapping d_buf.
 *   n, rec_size, key_size, stream: as for radix_sort.  The copies and the sort are enqueued on
 *   `stream`; h_out holds the result once the stream has reached this point.  The caller
 *   owns all four buffers.  Errors as for radix_sort, plus RS_ERR_INVALID_ARG for a null
 *   host pointer with n > 0 and RS_ERR_CUDA if a copy cannot be enqueued.
 */
rs_status radix_sort_host(const void *h_in, void *h_out, void *d_buf, void *d_tmp, uint64_t n, uint32_t rec_size,
                          uint32_t key_size, rs_stream_t stream);

/*
 * Sort many independent instances in one call: segment s is records
 * [seg_offsets[s], seg_offsets[s+1]) of `in`, sorted on its own, in place.
 *   seg_offsets  DEVICE pointer to n_segs + 1 uint64 values: non-decreasing, [0] = 0,
 *                [n_segs] = total records (not checked on the host; violating it is
 *                undefined behaviour).
 *   n_segs       number of segments (0: nothing is launched).
 *   total        seg_offsets[n_segs], passed by the caller so no device read is needed.
 *   in, tmp, rec_size, key_size, stream: as for radix_sort, with n = total.
 */
rs_status radix_sort_segmented(void *in, void *tmp, const uint64_t *seg_offsets, uint64_t n_segs,
                               uint64_t total, uint32_t rec_size, uint32_t key_size,
                               rs_stream_t stream);

/*
 * One stable counting-sort phase (section 1) on one digit: the records of `src` are written
 * to `dst` ordered by key bits [bit_lo, bit_lo + width), ties in input order.  This is the
 * distribution pass that every level of the sort makes on each large bin (section 3.1, step 1).
 *   src, dst   device pointers, n * rec_size bytes each, 16-byte aligned, not overlapping.
 *   width      1..10; bit_lo + width <= 8 * key_size.
 */
rs_status radix_partition(const void *src, void *dst, uint64_t n, uint32_t rec_size, uint32_t key_size,
                          uint32_t bit_lo, uint32_t width, rs_stream_t stream);

/*
 * Histogram of one digit (the counting step of a phase, section 1):
 * counts[v] = number of records whose key bits [bit_lo, bit_lo + width) equal v.
 *   counts   DEVICE pointer to 2^width uint64 values (written, not accumulated).
 *   width    1..10; bit_lo + width <= 8 * key_size.
 */
rs_status radix_histogram(const void *src, uint64_t n, uint32_t rec_size, uint32_t key_size, uint32_t bit_lo,
                          uint32_t width, uint64_t *counts, rs_stream_t stream);

/*
 * Run-length count of equal keys in records that are already sorted by key: the counting
 * step that follows the sort in k-mer counting (KMC3, the application of section 4).  A run
 * is a maximal range of consecutive records with equal keys (key_size bytes).
 *   in        DEVICE pointer to n sorted records (not modified); 16-byte aligned.
 *   out       DEVICE pointer with room for n records: receives the first record of each run,
 *             in order.
 *   counts    DEVICE pointer with room for n uint64 values: counts[r] = records in run r.
 *   d_nruns   DEVICE pointer to one uint64: the number of runs (0 for n = 0).
 * Asynchronous on `stream`; uses a small part of the stream's library workspace (its
 * status word is kept).  Records that are not sorted give runs of the unsorted sequence.
 */
rs_status radix_count_runs(const void *in, uint64_t n, uint32_t rec_size, uint32_t key_size, void *out,
                           uint64_t *counts, uint64_t *d_nruns, rs_stream_t stream);

/*
 * Waits for `stream` to drain, then reports (and clears) the device-side status of the
 * calls made on it: RS_OK, RS_ERR_DEVICE_TIMEOUT, RS_ERR_QUEUE_OVERFLOW, RS_ERR_INTERNAL
 * (a destination or range check failed; the offending writes were skipped), or RS_ERR_CUDA.
 */
rs_status radix_sort_status(rs_stream_t stream);

/* Human-readable name of a status code (static storage). */
const char *radix_sort_strerror(rs_status status);

/* Frees every library-owned workspace (after synchronising the device). */
rs_status radix_sort_release(void);

/*
 * Tuning knobs (process-wide; a zero field means "automatic").  They change speed only,
 * never the result.
 */
typedef struct rs_plan {
  uint32_t digit_bits_max;  /* widest digit of a distribution pass: 8..10 (default 9, or 10 when
                               that saves a level; each bin takes the fewest levels, then the
                               narrowest digit for them) */
  uint32_t tile_records;    /* records per distribution tile: 256, 512, 1024, 2048 or 4096 */
  uint32_t chunk_records;   /* largest bin sorted on chip: 64.. the shared-memory maximum */
  uint32_t sm_limit;        /* use at most this many SMs for the persistent grids */
  uint32_t watchdog_polls;  /* limit of every device-side wait (a CTA waiting for its own bulk
                               copy into shared memory): this many suspended polls of the
                               barrier, then the call reports RS_ERR_DEVICE_TIMEOUT
                               (default 2^20, about a second) */
  uint32_t tiny_records;    /* chunks (small bins or segments) of at most this many records are
                               sorted by warps with sorting networks, larger ones by a CTA:
                               2..64 (default 64) */
  uint32_t enum_records;    /* largest bucket of the on-chip sorter finished by enumeration sort
                               (larger ones are distributed again): 8..64 (default 48) */
} rs_plan;

rs_status radix_sort_set_plan(const rs_plan *plan);
rs_status radix_sort_get_plan(rs_plan *plan);

/* Kernels launched by this process through the library so far (all entry points). */
uint64_t radix_sort_launch_count(void);

/*
 * Largest bin (in records of rec_size bytes) that the current plan sorts in one on-chip
 * pass: bins and segments up to this size skip the distribution levels.  0 for an invalid
 * rec_size.  Host only; no GPU needed.
 */
uint32_t radix_sort_chunk_records(uint32_t rec_size);

/*
 * Bytes of the library-owned workspace that a call of n records (n_segs segments; 0 for
 * radix_sort) needs under the current plan; 0 for invalid sizes.  Host only.
 */
uint64_t radix_sort_workspace_bytes(uint64_t n, uint32_t rec_size, uint32_t key_size, uint64_t n_segs);

/*
 * Makes the workspace of (current device, stream) large enough for calls of up to n records
 * and n_segs segments, so that later calls of that size neither allocate nor synchronise
 * (growing a workspace drains its stream and frees the old one; cudaMalloc and cudaFree can
 * stall every stream of the device).  Call it before capturing a stream into a CUDA graph.
 * Returns RS_ERR_NO_MEMORY if the allocation fails, RS_ERR_INVALID_ARG for a bad layout.
 */
rs_status radix_sort_reserve(uint64_t n, uint32_t rec_size, uint32_t key_size, uint64_t n_segs,
                             rs_stream_t stream);

/*
 * Per-launch timing (for benchmarks).  radix_sort_profile(1) starts a session: every kernel
 * the library launches from then on is bracketed by two CUDA events recorded on the
 * launching stream; radix_sort_profile(0) stops recording.  radix_sort_profile_read() waits
 * for the recorded events and writes up to `max` records (kernel id, level, milliseconds)
 * in launch order; it returns how many it wrote (out = NULL: how many there are), or -1 on
 * a CUDA error.  Kernel ids: RS_K_*.
 */
enum {
  RS_K_INIT = 0,      /* set-up of the control block, first bin list or chunk */
  RS_K_HIST = 1,      /* histogram of a level's digit (+ bucket bases) */
  RS_K_HIST_REDO = 2, /* recount of the bins whose digit had to move after the count */
  RS_K_SCATTER = 3,   /* stable distribution of a level's bins (the dominant kernel) */
  RS_K_CLASSIFY = 4,  /* sub-bin classification and the next level's bin list */
  RS_K_CHUNK = 5,     /* on-chip sorts of small bins */
  RS_K_COPY = 6,      /* copy-back of finished ranges left in tmp */
  RS_K_TINY = 7       /* warp sorts of tiny chunks (at most 64 records) */
};
typedef struct rs_kernel_time {
  uint32_t kernel;
  uint32_t level;
  float ms;
} rs_kernel_time;

rs_status radix_sort_profile(int enable);
int64_t radix_sort_profile_read(rs_kernel_time *out, int64_t max);

/*
 * Which kernels radix_sort_profile brackets with events: bit k set = kernel id k (RS_K_*) is
 * timed (default: all).  Fewer events disturb the timed work less: a benchmark can time the
 * whole call and one kernel together.  Applies to launches made after the call.
 */
rs_status radix_sort_profile_kernels(uint32_t mask);

/*
 * radix_sort without any allocation.  (No counterpart in the paper: this is an interface
 * for callers that cannot allocate.)
 *
 * Some callers must not have a library allocate device memory behind their back: a
 * framework whose caching allocator owns the GPU's memory (an outside cudaMalloc can fail
 * or fragment it), a latency-critical path where cudaMalloc/cudaFree would add an implicit
 * device synchronisation, or a process with a fixed device-memory budget.  radix_sort
 * allocates its metadata workspace on first use; this entry point instead uses a fixed
 * array of 64 MiB in device memory that the library declares statically.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  The CUDA runtime reserves the array on
 * a device when it loads the array's module there: under lazy module loading (the CUDA 12+
 * default) that happens during the first radix_sort_noalloc call on that device, which can
 * therefore return RS_ERR_NO_MEMORY when the device is full; from then on the device holds
 * the array until the process exits, and later calls reserve nothing.
 *
 * Arguments and result are those of radix_sort; the sort is the same (byte-identical
 * output).  Additionally:
 *   d_status  optional DEVICE pointer to one uint32: when the call's work has run it holds
 *             the call's device-side error bits, 0 = ok, else the OR of 1 (a bounded wait
 *             ran out: RS_ERR_DEVICE_TIMEOUT), 2 (a list outgrew its bound:
 *             RS_ERR_QUEUE_OVERFLOW) and 4 (a destination range check failed:
 *             RS_ERR_INTERNAL), the conditions radix_sort_status reports for radix_sort.
 *             NULL: none.  (radix_sort_status does not see calls made through this entry
 *             point.)
 * Limits:
 *   The workspace needed for (n, rec_size, key_size) must fit the 64 MiB array, else the
 *   call returns RS_ERR_TOO_LARGE and launches nothing.  With the default plan that is about
 *   3.0 x 10^7 records of 8 or 16 bytes (8-byte keys), 2.4 x 10^7 of 24 bytes (16-byte
 *   keys); radix_sort_workspace_bytes tells for any shape.
 * Sharing:
 *   Every call uses the same array, on every stream.  Calls whose work overlaps on the GPU
 *   (on different streams, or from different host threads without ordering) race on it and
 *   produce undefined results: order them on one stream or synchronise between them.
 *   The array keeps the previous call's contents; each call resets what it relies on.
 * Set-up:
 *   The first call on a device looks up the array's device address on that device (the
 *   address is then kept).  Make that first call on each device before capturing a stream
 *   into a CUDA graph.
 */
rs_status radix_sort_noalloc(void *in, void *tmp, uint64_t n, uint32_t rec_size, uint32_t key_size,
                             uint32_t *d_status, rs_stream_t stream);

/*
 * Testing only; the flags apply to the next radix_sort / radix_sort_segmented / radix_partition
 * / radix_sort_noalloc call on any stream, then clear (flags = 0 clears them at once).  For
 * radix_sort_noalloc the failure reaches the caller's status word (value 4 or 1) instead of
 * radix_sort_status().
 *   bit 0 (1): each distribution pass treats the first non-empty digit run of its first tile as
 *          failing the destination range check, so that run is not written: the call's later
 *          kernels do nothing, and radix_sort_status() reports RS_ERR_INTERNAL.
 *   bit 1 (2): the first bulk-copy wait of the first distribution CTA waits on a shared-memory
 *          barrier that nothing completes, so it runs out after rs_plan.watchdog_polls polls:
 *          the call's later kernels do nothing, and radix_sort_status() reports
 *          RS_ERR_DEVICE_TIMEOUT.  (The CTA still waits, with the default limit, for its own
 *          copy before it exits.)
 */
rs_status radix_sort_test_inject(uint32_t flags);

#ifdef __cplusplus
}
#endif

#endif /* RADIX_GB300_H */
