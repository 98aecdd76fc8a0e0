// Internal declarations shared by the sorter's CUDA translation units.
//
// The method is the MSD radix sort of Kokot, Deorowicz and Dlugosz ("Even faster sorting
// of (not only) integers", section 3.1): distribute the records of a bin by a digit of the
// key into sub-bins (a stable counting sort: histogram, exclusive prefix sum, scatter),
// recurse into every sub-bin independently, and switch to an on-chip sorter once a bin is
// small.  Here a "bin" is a contiguous range of records; a level is one distribution pass
// over every large bin at once.
//
// Record layout: rec_size bytes = RW 8-byte words.  The key is bytes [0, key_size) read as
// a little-endian unsigned integer: key bit b is bit (b mod 64) of word floor(b / 64), so
// word 1 (bytes 8..15) is more significant than word 0.  Only key_size <= 16 is supported
// (the paper's keys are 8 and 16 bytes, section 3.3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rsg {

using u64 = unsigned long long;
using u32 = unsigned int;
using u16 = unsigned short;
using u8 = unsigned char;

constexpr int kThreads = 512;                 // threads of every sorting CTA
constexpr int kWarps = kThreads / 32;
constexpr int kWMax = 10;                     // widest digit (bits) a distribution pass supports
constexpr int kWMin = 8;                      // narrowest digit of a pass that has 8 key bits to use
constexpr u32 kFull = 0xffffffffu;

// device error bits (reported by radix_sort_status)
enum : u32 { kErrTimeout = 1u, kErrOverflow = 2u, kErrInternal = 4u };

// testing hooks (radix_sort_test_inject): one digit run of the first scatter tile fails its
// range check; the first scatter tile waits on a barrier that nothing completes
enum : u32 { kInjectRange = 1u, kInjectWait = 2u };

// default limit of a device-side wait: 2^20 suspended polls (about a second)
constexpr u32 kWaitPolls = 1u << 20;

// Bin flags
enum : u32 { kBinRedo = 1u, kBinEqual = 2u, kBinDom = 4u };

// Chunk flags
enum : u32 { kChSrcTmp = 1u, kChCopyOnly = 2u };

// Chunks of at most this many records can be tiny: warps sort them with sorting networks in
// registers (k_tiny) instead of a CTA (the limit of a job, Job::tiny_max, is at most this).
// They are listed from the top of the chunk array down.
constexpr u32 kTinyMax = 64;
// largest bucket the on-chip sorter finishes by enumeration sort (Job::es_max: 8..kEsLimit)
constexpr u32 kEsDefault = 48, kEsLimit = 64;

// A bin handled by a multi-CTA distribution pass.
struct Bin {
  u64 begin;        // first record
  u64 size;         // records
  u64 tile_start;   // number of the bin's first tile within its level
  u64 base_off;     // first of its 2^bucket_bits entries in the level's bucket-base pool
  u64 kand[2];      // AND / OR of the bin's keys, gathered by the histogram pass: they tell
  u64 kor[2];       // whether the digit starts at the highest differing bit, or all keys are equal
  u64 dom[2];       // kBinDom: the key that holds most of the bin (its bucket is finished)
  u32 lo, W;        // the digit is key bits [lo, lo + W)
  u32 parity;       // 0: the bin's records are in `in`; 1: in `tmp`
  u32 flags;
  u32 done;         // tiles counted by the histogram pass (finds the last CTA of the bin)
  u32 pad;
};

// A contiguous range of records sorted completely by one CTA in shared memory.  It is one
// small bin, or several consecutive small sub-bins of the same parent (they share every key
// bit above the parent's digit and are already in digit order, so sorting the whole range
// by key sorts each of them).
struct Chunk {
  u64 begin;
  u32 size;
  u32 flags;        // kChSrcTmp: records are in tmp (else in); kChCopyOnly: already sorted
  u32 p;            // every key bit >= p is shared by the chunk (0: unknown, compute it)
  // A chunk packed from several sub-bins of one parent: they differ in the parent's digit
  // (key bits [p, p + pw)), whose values lie in [v0, v0 + 2^sb).  The chunk's first
  // distribution then uses (digit - v0) above the bits right below p.  sb = 0: one sub-bin.
  u32 v0;
  u16 pw, sb;
};

// A range of finished records that lives in tmp and must be copied to in.
struct Piece {
  u64 begin, size;
};

// Control block in device memory.  Lists are double-buffered by level parity.
// `err` collects the error bits of every call on the stream until radix_sort_status reads
// it; `cerr` holds those of the current call only (the call's first kernel clears it), and
// every kernel after the one that set it returns at once: nothing computed from records that
// a failed step left unwritten reaches a later kernel.
struct Ctl {
  u32 err, cerr;
  u64 nbins[2];
  u64 ntiles[2];
  u64 base_used[2];
  u32 cls_done;     // classify CTAs finished (the last one finalises the next list)
  u32 nredo;        // bins of this level whose digit moved after the count (recount needed)
  u64 nchunks, chunk_ticket;
  u64 ntiny;        // tiny chunks, at chunks[cap_chunks - 1 - t] for t < ntiny
  u64 npieces, piece_ticket;
};

// Everything a kernel needs about one call, passed by value.
struct Job {
  u64* buf[2];        // [0] = in, [1] = tmp
  u64 n;              // records
  u32 RW;             // words per record
  u32 K;              // key bytes
  u32 KW;             // key words (1 or 2)
  u32 T;              // records per tile of a distribution pass
  u32 chunk_max;      // largest range one CTA sorts on chip
  u32 wmax;           // widest digit of a pass (<= kWMax)
  u32 lanes;          // tile ranges of a distribution level (one per histogram CTA)
  u32 inject;         // testing: kInjectRange / kInjectWait (one call)
  u32 wd_polls;       // limit of a device-side wait (suspended polls of a shared-memory barrier)
  u32 tiny_max;       // chunks of at most this many records go to the warp sorter (<= kTinyMax)
  u32 es_max;         // largest bucket the on-chip sorter finishes by enumeration sort

  u64 keymask[2];     // key bits of words 0 and 1
  Ctl* ctl;
  Bin* bins[2];
  u64 cap_bins;
  u64* base[2];       // bucket counts, then (after the scan) bucket bases
  u64 cap_base;
  u64* seg;           // per (lane, bin) segment and digit: counts, then run starts (2^wmax each)
  u64 cap_seg;        // segments
  Chunk* chunks;
  u64 cap_chunks;
  Piece* pieces;
  u64 cap_pieces;
  const u64* seg_off; // segmented mode: n_segs + 1 record offsets
  u64 n_segs;
};

// Records an error of the current call (and in the stream's sticky word).
__device__ __forceinline__ void report(Ctl* ctl, u32 bits) {
  atomicOr(&ctl->err, bits);
  atomicOr(&ctl->cerr, bits);
}
// Whether an earlier step of the current call failed (then a kernel does nothing).
__device__ __forceinline__ bool call_failed(const Ctl* ctl) { return *(volatile const u32*)&ctl->cerr != 0; }

constexpr u64 kPieceRecords = 1ull << 16;      // copy-back granularity
constexpr u32 kMaxLanes = 1024;                // tile ranges per level, at most

// Lane of tile t: level tiles are split into j.lanes contiguous ranges of `per` tiles.  The
// part of bin b inside lane c is segment c + b (unique: a later lane never reaches back to an
// earlier bin), so a level needs at most lanes + bins segments.
__host__ __device__ inline u64 lane_tiles(u64 ntiles, u32 lanes) { return (ntiles + lanes - 1) / lanes; }

// ---------------------------------------------------------------------------- keys
template <int KW>
struct Key {
  u64 w[KW];
};

template <int KW>
__device__ __forceinline__ Key<KW> load_key(const u64* rec, const Job& j) {
  Key<KW> k;
#pragma unroll
  for (int i = 0; i < KW; i++) k.w[i] = rec[i] & j.keymask[i];
  return k;
}

// Buckets of a bin.  A plain bin has one bucket per digit value (key bits [lo, lo + W)).  A bin
// that one key K dominates (kBinDom; seen in a sample when the bin was formed) splits K's
// digit dK in three -- keys below K, K itself, keys above K -- so that K's records are
// finished by this pass instead of being moved again at every later level: digits below dK
// keep their number, dK becomes dK (below K), dK + 1 (K) and dK + 2 (above K), digits above
// dK move up by two.  Its bucket numbers fit W + 1 bits.
__host__ __device__ inline u32 bucket_bits(u32 W, u32 flags) { return W + ((flags & kBinDom) ? 1u : 0u); }

// Digit = key bits [lo, lo + W), W <= 16.
template <int KW>
__device__ __forceinline__ u32 digit_of(const Key<KW>& k, u32 lo, u32 W) {
  u64 v;
  if (KW == 1) {
    v = k.w[0] >> lo;
  } else {
    const u32 sh = lo & 63;
    if (lo >= 64) {
      v = k.w[KW - 1] >> sh;
    } else {
      v = k.w[0] >> sh;
      if (sh != 0 && sh + W > 64) v |= k.w[KW - 1] << (64 - sh);
    }
  }
  return (u32)v & ((1u << W) - 1u);
}

template <int KW>
__device__ __forceinline__ bool key_less(const Key<KW>& a, const Key<KW>& b) {
  if (KW == 2 && a.w[KW - 1] != b.w[KW - 1]) return a.w[KW - 1] < b.w[KW - 1];
  return a.w[0] < b.w[0];
}

template <int KW>
__device__ __forceinline__ bool key_eq(const Key<KW>& a, const Key<KW>& b) {
  bool e = a.w[0] == b.w[0];
  if (KW == 2) e = e && a.w[KW - 1] == b.w[KW - 1];
  return e;
}

// Bucket of key k in a bin with digit [lo, lo + W): the digit, or for a dominated bin (dom)
// the three-way split of K's digit dK (see bucket_bits).
template <int KW>
__device__ __forceinline__ u32 bucket_of(const Key<KW>& k, u32 lo, u32 W, bool dom, const Key<KW>& K, u32 dK) {
  const u32 d = digit_of<KW>(k, lo, W);
  if (!dom) return d;
  if (d != dK) return d < dK ? d : d + 2;
  return key_less<KW>(k, K) ? dK : key_eq<KW>(k, K) ? dK + 1 : dK + 2;
}

// Position of the highest set bit plus one (0 if none) over a KW-word value.
__host__ __device__ inline u32 top_bit_plus1(u64 w0, u64 w1) {
#ifdef __CUDA_ARCH__
  if (w1) return 128u - (u32)__clzll((long long)w1);
  if (w0) return 64u - (u32)__clzll((long long)w0);
#else
  if (w1) return 128u - (u32)__builtin_clzll(w1);
  if (w0) return 64u - (u32)__builtin_clzll(w0);
#endif
  return 0;
}

// Digit plan for a bin of `size` records whose highest differing key bit is p - 1: enough
// bits that an average sub-bin fits one on-chip sort, spread evenly over the passes still
// needed, at least kWMin (bounds the number of levels) and at most wmax.
__host__ __device__ inline void plan_digit(u64 size, u32 p, u32 chunk_max, u32 wmax, u32* lo, u32* W) {
  u32 need = 0;
  while (need < 63 && (size >> need) > chunk_max) need++;
  u32 passes = (need + wmax - 1) / wmax;
  if (passes == 0) passes = 1;
  u32 w = (need + passes - 1) / passes;
  if (w < (u32)kWMin) w = kWMin;
  if (w > wmax) w = wmax;
  if (w > p) w = p;
  if (w == 0) w = 1;
  *W = w;
  *lo = p >= w ? p - w : 0;
}

__host__ __device__ inline u64 ceil_div(u64 a, u64 b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------- warp helpers
__device__ __forceinline__ u32 lanemask_lt() {
  u32 m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Bin of a tile: the last bin whose tile_start <= t (bins are in tile order).
__device__ __forceinline__ u64 find_bin(const Bin* bins, u64 nb, u64 t) {
  u64 lo = 0, hi = nb;  // invariant: bins[lo].tile_start <= t < bins[hi].tile_start
  while (hi - lo > 1) {
    u64 mid = (lo + hi) >> 1;
    if (bins[mid].tile_start <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Asynchronous global -> shared copies (cp.async, completed by cp_async_wait_all): all of a
// tile's loads are in flight at once, without staging through registers.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most one (the most recent) group of this thread's copies is still pending
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Bulk copies global -> shared by the copy engine of the SM (one instruction for a whole
// tile), completed on a shared-memory barrier that counts the bytes that have landed.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this CTA's earlier ordinary accesses of shared memory (made visible to this thread by
// a barrier) before the copy engine's writes that follow.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// One thread: announce `bytes` on the barrier and start the copy (dst, src, bytes: multiples
// of 16 bytes and 16-byte aligned).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, u64* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// One arrival on the barrier without a copy (completes a phase that has nothing to load).
__device__ __forceinline__ void mbar_arrive(u64* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Wait until the barrier's phase `parity` has completed, at most `tries` waits (each one
// suspends the thread for a bounded time); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(u64* bar, unsigned parity, unsigned tries) {
  for (unsigned i = 0; i < tries; i++) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Exclusive prefix sum over the CTA of one value per thread (NT threads); ends with a barrier.
template <int NT>
__device__ __forceinline__ u32 block_exclusive_sum(u32 x, u32* scr) {
  constexpr int kW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32 incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scr[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const u32 v = lane < kW ? scr[lane] : 0;
    u32 t = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kW) scr[lane] = t - v;
  }
  __syncthreads();
  return scr[warp] + incl - x;
}

// Ask for [p, p + bytes) to be brought into L2 with one bulk request (the range shrunk to
// 16-byte boundaries, so nothing outside it is touched).  Nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p, u64 bytes) {
  const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// Start copying `words` 8-byte words global -> shared (16-byte copies when the source is
// 16-byte aligned; the destination always is).  Call cp_async_wait_all + __syncthreads
// before reading them.
// NT = threads of the calling CTA (all of them call it).
template <int NT = kThreads>
__device__ __forceinline__ void load_words_async(u64* dst, const u64* src, u64 words) {
  const int tid = threadIdx.x;
  if ((((uintptr_t)src) & 15) == 0) {
    const u64 pairs = words >> 1;
    for (u64 i = tid; i < pairs; i += NT) cp_async16(dst + 2 * i, src + 2 * i);
    if ((words & 1) && tid == 0) cp_async8(dst + words - 1, src + words - 1);
  } else {
    for (u64 i = tid; i < words; i += NT) cp_async8(dst + i, src + i);
  }
}


// Shared memory of k_hist: two buffers of a tile's keys (tile t+1 streams in while tile t
// is counted).
__host__ __device__ inline size_t hist_smem_bytes_for(u32 T, u32 KW) { return 2ull * T * KW * 8; }

// ------------------------------------------------------------------ launch helpers
// Host (rs_api.cu): a kernel's dynamic shared-memory limit, set once per (device, kernel) and
// raised when a larger size is needed, and its occupancy, cached per (device, kernel,
// threads, size): both are driver calls of microseconds, and a sort makes dozens of launches.
void ensure_smem(const void* fn, size_t smem);
int occupancy(const void* fn, int threads, size_t smem);

// Host-side launchers implemented in the kernel translation units.  Each returns the
// number of kernels it launched (or -1 on a launch error).
int launch_init_plain(const Job& j, u32 lo, u32 W, cudaStream_t s);
int launch_init_single_chunk(const Job& j, cudaStream_t s);
int launch_init_segments(const Job& j, u32 grid, cudaStream_t s);
int launch_hist(const Job& j, int level, int mode, cudaStream_t s);  // grid = j.lanes
int launch_scatter(const Job& j, int level, u32 grid, cudaStream_t s);
int launch_classify(const Job& j, int level, u32 grid, cudaStream_t s);
int launch_chunks(const Job& j, u32 grid, cudaStream_t s);
int launch_tiny(const Job& j, u32 sms, cudaStream_t s);
int launch_copy(const Job& j, u32 grid, cudaStream_t s);
int launch_read_counts(const Job& j, u64* d_counts, u32 W, cudaStream_t s);

// smem bytes and CTAs per SM of the tile/chunk kernels for a job
size_t scatter_smem_bytes(const Job& j);
size_t chunk_smem_bytes(const Job& j);
int scatter_ctas_per_sm(const Job& j);
int chunk_ctas_per_sm(const Job& j);
int hist_ctas_per_sm(const Job& j);
int classify_ctas_per_sm();

}  // namespace rsg
