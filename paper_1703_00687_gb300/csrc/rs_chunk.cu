// On-chip sorting of small bins (Kokot et al., sections 3.2-3.3) and the final copy-back.
//
// One CTA sorts a chunk (one small bin, or several consecutive small sub-bins of one parent)
// completely in shared memory: the records are staged once, a permutation of their indices
// is sorted, and the records are written once, in order, to `in`.  Because every record is
// staged before any is written, the chunk may be sorted in place.
//
// The index sort follows the paper's small/tiny-bin scheme on chip:
//   * skip the key bits every record of the range shares (AND/OR of the keys);
//   * one counting-sort distribution on the next kWinBits bits (fewer for a small chunk),
//     with shared-memory atomic counters (the order inside a bucket is arbitrary here);
//   * every bucket of up to es_max records (the plan's enumeration limit, 48 by default) is
//     finished by enumeration sort (section 2.2, 3.3): a record's place is the number of
//     records of the bucket that must precede it, comparing (key, input position) -- so
//     equal keys come out in input order;
//   * a larger bucket is processed again the same way; if all its keys are equal it is put
//     back in input order (ranks of its input positions, from a bitmap of them);
//   * a chunk of at most es_max records is one enumeration sort, without a distribution.
// The result is therefore the stable order, and the whole sorter is stable.
//
// Chunks of at most the plan's tiny limit (at most kTinyMax) records are kept in a list of
// their own and sorted by k_tiny: warps, not CTAs, with bitonic sorting networks over lane
// shuffles (several chunks per warp).
#include <algorithm>

#include "rs_internal.cuh"

namespace rsg {

// Two CTAs of 512 threads per SM, each with one stage buffer: one CTA's load and write overlap
// the other's sort.
constexpr int kCThreads = 512;   // threads of a chunk CTA
constexpr int kChunkCtas = 2;    // chunk CTAs per SM
constexpr int kCWarps = kCThreads / 32;
constexpr int kWinBits = 12;     // digit of the on-chip distribution pass
constexpr int kIdxBits = 13;     // input positions of a chunk (chunk_max <= 2^13)
constexpr int kChunkItems = 8;   // positions per thread (chunk_max <= kCThreads * this)
constexpr int kCntWords = 1 << (kWinBits - 1);  // counters of a distribution, two 16-bit per word
// dynamic shared memory of the chunk CTA (two CTAs and their static shared memory fit an SM)
constexpr size_t kChunkSmem = 111 * 1024;
constexpr size_t kChunkFixed = kCntWords * 4 + 256;

// stage: the chunk's records; aux: one composite key (u64) per record in the first round, or
// the two index arrays (u16) and the bucket stack of the general rounds; cnt: the counters.
struct ChunkLayout {
  size_t stage, aux, cnt, total;
};

__host__ __device__ inline ChunkLayout chunk_layout(u32 m, u32 RW) {
  ChunkLayout c;
  size_t o = 0;
  c.stage = o; o += (size_t)m * RW * 8;
  c.aux = o; o += (size_t)m * 8;  // >= 4m (perm, out) + the stack of at most m / 9 + 2 pairs (es_max >= 8)
  o = (o + 15) & ~(size_t)15;
  c.cnt = o; o += (size_t)kCntWords * 4;
  c.total = (o + 127) & ~(size_t)127;
  return c;
}

template <int KW, int RWT>
struct ChunkCtx {
  u64 km0, km1;  // key bits of words 0 and 1
  u32 RW;
  const u64* stage;
  u16* perm;     // the current order (record indices)
  u16* out;      // scratch order
  u32* cnt;      // 2^kWinBits 16-bit counters, two per word
  u32* stack;    // pairs (begin, size) of buckets still to sort
  u32 stack_cap;
  u32 es_max;    // largest bucket finished by enumeration sort

  __device__ __forceinline__ Key<KW> key(u32 r) const {
    const u64* p = stage + r * (RWT ? (u32)RWT : RW);
    Key<KW> k;
    k.w[0] = p[0] & km0;
    if (KW == 2) k.w[KW - 1] = p[1] & km1;
    return k;
  }
  __device__ __forceinline__ u32 count_of(u32 d) const { return (cnt[d >> 1] >> ((d & 1) * 16)) & 0xffffu; }
};

// Exclusive scan, in place, of nd (even, <= 2^kWinBits) 16-bit counters packed two per word.
// Returns (the same in every thread) whether some counter exceeded `big`.
template <int KW, int RWT>
__device__ bool scan_counts(const ChunkCtx<KW, RWT>& c, u32 nd, u32 big = 0xffffu) {
  __shared__ u32 scr[kCWarps + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 words = nd >> 1;
  const u32 per = (words + kCThreads - 1) / kCThreads;
  const u32 w0 = min(words, tid * per), w1 = min(words, w0 + per);
  // a full window's counters: 16-byte accesses (four words each) instead of accesses of
  // consecutive words per lane, which meet a 4-way bank conflict
  constexpr u32 kV = kCntWords / kCThreads / 4 > 0 ? kCntWords / kCThreads / 4 : 1;
  u32 sum = 0, mx = 0;
  uint4 v4[kV];
  const bool vec = per == 4 * kV && w1 - w0 == 4 * kV;
  auto take = [&](u32 x) {
    sum += (x & 0xffffu) + (x >> 16);
    mx = max(mx, max(x & 0xffffu, x >> 16));
  };
  if (vec) {
#pragma unroll
    for (u32 q = 0; q < kV; q++) {
      v4[q] = reinterpret_cast<const uint4*>(c.cnt + w0)[q];
      take(v4[q].x);
      take(v4[q].y);
      take(v4[q].z);
      take(v4[q].w);
    }
  } else {
    for (u32 w = w0; w < w1; w++) take(c.cnt[w]);
  }
  u32 x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scr[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const u32 v = lane < kCWarps ? scr[lane] : 0;
    u32 t = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kCWarps) scr[lane] = t - v;
  }
  __syncthreads();
  u32 run = scr[warp] + x - sum;
  if (vec) {
    // word = (first slot of its even digit) | (first slot of its odd digit) << 16
    auto starts = [&run](u32 v) {
      const u32 hi = run + (v & 0xffffu), w = run | (hi << 16);
      run = hi + (v >> 16);
      return w;
    };
#pragma unroll
    for (u32 q = 0; q < kV; q++) {
      uint4 o;
      o.x = starts(v4[q].x);
      o.y = starts(v4[q].y);
      o.z = starts(v4[q].z);
      o.w = starts(v4[q].w);
      reinterpret_cast<uint4*>(c.cnt + w0)[q] = o;
    }
  } else {
    for (u32 w = w0; w < w1; w++) {
      const u32 v = c.cnt[w];
      const u32 lo = run, hi = run + (v & 0xffffu);
      c.cnt[w] = lo | (hi << 16);
      run = hi + (v >> 16);
    }
  }
  return __syncthreads_or(mx > big) != 0;
}

// The digit of an on-chip distribution: key bits [lo, lo + w), optionally preceded (as more
// significant bits) by a packed chunk's sub-bin number, (parent digit - v0) on sb bits.
struct DigitSpec {
  u32 lo, w;        // window below the shared bits
  u32 plo, pw, v0;  // the parent digit of a packed chunk: key bits [plo, plo + pw)
  u32 sb;           // bits of the sub-bin number (0: not packed)
  __device__ __forceinline__ u32 bits() const { return sb + w; }
  template <int KW>
  __device__ __forceinline__ u32 of(const Key<KW>& k) const {
    u32 d = digit_of<KW>(k, lo, w);
    // (masked: a record whose parent digit lies outside the chunk's sub-bins -- possible
    // only after a reported error -- must still index inside the counters)
    if (sb) d |= ((digit_of<KW>(k, plo, pw) - v0) & ((1u << sb) - 1)) << w;
    return d;
  }
};

// Window right below bit p (all bits >= p shared), no sub-bin number: kWinBits bits, or
// fewer for a range of s records (about 2 to 4 buckets per record: the counters to scan
// then scale with the range).
__device__ __forceinline__ DigitSpec window_below(u32 p, u32 s = 1u << kIdxBits) {
  u32 w = kWinBits;
  if (s < (1u << (kWinBits - 2))) {
    w = 4;
    while ((1u << (w - 2)) < s) w++;
  }
  DigitSpec d = {};
  d.w = p > w ? w : p;
  d.lo = p - d.w;
  return d;
}

// The first on-chip round of a chunk sorts 64-bit composite keys: the record's relevant key
// bits -- a packed chunk's sub-bin number (sb bits) above key bits [0, p), every higher key bit
// being shared by the chunk -- cut from below to their top kCompKeyBits bits, then the record's
// position in the chunk (kIdxBits).  Composite keys are distinct (positions are), so ranking a
// bucket needs one comparison of neighbouring words per pair; their order is the (key,
// position) order, except between two records whose kept key bits are equal while dropped
// ones (t > 0) differ: those compare their whole keys.
constexpr u32 kCompKeyBits = 64 - kIdxBits;

struct CompSpec {
  u64 m0, m1;         // key bits [0, p) of words 0 and 1
  u32 p, sb, plo, pw, v0;
  u32 t;              // relevant key bits dropped from below (0: the composite order is exact)
  u32 dshift, dmask;  // the round's digit = (composite >> dshift) & dmask (= DigitSpec::of)

  // relevant key bits [t, p + sb) of a key, at bit 0
  template <int KW>
  __device__ __forceinline__ u64 keypart(const Key<KW>& k) const {
    u64 lo = k.w[0] & m0, hi = KW == 2 ? (k.w[KW - 1] & m1) : 0ull;
    if (sb) {
      const u64 sub = (u64)((digit_of<KW>(k, plo, pw) - v0) & ((1u << sb) - 1u));
      if (p < 64) {
        lo |= sub << p;
        if (p + sb > 64) hi |= sub >> (64 - p);
      } else {
        hi |= sub << (p - 64);
      }
    }
    if (t == 0) return lo;
    if (t < 64) return (lo >> t) | (hi << (64 - t));
    return hi >> (t - 64);
  }
};

// Composite keys for a round whose digit `dig` sits right below bit p (dig.lo + dig.w = p).
__device__ __forceinline__ CompSpec comp_spec(const DigitSpec& dig, u32 p, u64 km0, u64 km1) {
  CompSpec cs;
  cs.p = p;
  cs.sb = dig.sb;
  cs.plo = dig.plo;
  cs.pw = dig.pw;
  cs.v0 = dig.v0;
  cs.m0 = (p >= 64 ? ~0ull : ((1ull << p) - 1ull)) & km0;
  cs.m1 = (p <= 64 ? 0ull : p >= 128 ? ~0ull : ((1ull << (p - 64)) - 1ull)) & km1;
  const u32 kb = p + dig.sb;
  cs.t = kb > kCompKeyBits ? kb - kCompKeyBits : 0u;
  cs.dshift = kIdxBits + dig.lo - cs.t;  // (the digit lies inside the kept bits)
  cs.dmask = (1u << dig.bits()) - 1u;
  return cs;
}

// Distributes positions [a, a + s) of c.perm into c.out by a digit of the record (any order
// inside a bucket); afterwards c.cnt holds every bucket's first position (relative to a).
// identity: c.perm is the identity over the range (not read).  zeroed: c.cnt is already 0.
template <int KW, int RWT>
__device__ void distribute(const ChunkCtx<KW, RWT>& c, u32 a, u32 s, const DigitSpec& dig,
                           bool identity, bool zeroed) {
  const int tid = threadIdx.x;
  const u32 nd = 1u << dig.bits();
  const u32 words = (nd + 1) >> 1;
  if (!zeroed) {
    for (u32 i = tid; i < words; i += kCThreads) c.cnt[i] = 0;
    __syncthreads();
  }
  u32 held[kChunkItems];
#pragma unroll
  for (int k = 0; k < kChunkItems; k++) {
    const u32 i = tid + k * kCThreads;
    held[k] = 0xffffffffu;
    if (i < s) {
      const u32 r = identity ? a + i : c.perm[a + i];
      const u32 d = dig.of<KW>(c.key(r));
      const u32 old = atomicAdd(&c.cnt[d >> 1], 1u << ((d & 1) * 16));
      held[k] = (((old >> ((d & 1) * 16)) & 0xffffu)) | (d << 16);
    }
  }
  __syncthreads();
  scan_counts(c, nd < 2 ? 2 : nd);
#pragma unroll
  for (int k = 0; k < kChunkItems; k++) {
    if (held[k] != 0xffffffffu) {
      const u32 d = held[k] >> 16;
      const u32 i = tid + k * kCThreads;
      c.out[a + c.count_of(d) + (held[k] & 0xffffu)] = identity ? (u16)(a + i) : c.perm[a + i];
    }
  }
  __syncthreads();
}

// After a distribution of positions [a, a + s) by `dig` into c.out (bucket starts in c.cnt):
// enumeration sort of every bucket of up to es_max records into c.perm; the positions of a
// larger bucket are copied as they are and the bucket goes on the stack.  Ends with a
// barrier, after which *s_top is final.
template <int KW, int RWT>
__device__ void finish_round(const ChunkCtx<KW, RWT>& c, u32 a, u32 s, const DigitSpec& dig, u32* s_top) {
  const int tid = threadIdx.x;
  const u32 nd = 1u << dig.bits();
  for (u32 i = tid; i < s; i += kCThreads) {
    const u32 r = c.out[a + i];
    const Key<KW> kr = c.key(r);
    const u32 d = dig.of<KW>(kr);
    const u32 st = c.count_of(d);
    const u32 en = d + 1 < nd ? c.count_of(d + 1) : s;
    const u32 sz = en - st;
    if (sz == 1) {
      c.perm[a + i] = (u16)r;
    } else if (sz <= c.es_max) {
      // enumeration sort: rank = records of the bucket that must precede this one
      u32 rank = 0;
      for (u32 q = st; q < en; q++) {
        const u32 r2 = c.out[a + q];
        const Key<KW> k2 = c.key(r2);
        rank += key_less<KW>(k2, kr) || (key_eq<KW>(k2, kr) && r2 < r);
      }
      c.perm[a + st + rank] = (u16)r;
    } else {
      c.perm[a + i] = (u16)r;
      if (i == st) {
        const u32 t = atomicAdd(s_top, 1u);
        if (t < c.stack_cap) {
          c.stack[2 * t] = a + st;
          c.stack[2 * t + 1] = sz;
        }
      }
    }
  }
  __syncthreads();
}

// Sorts positions [a, a + s) of c.perm by (key, input position): one distribution by `dig`,
// then finish_round.
template <int KW, int RWT>
__device__ void sort_round(const ChunkCtx<KW, RWT>& c, u32 a, u32 s, const DigitSpec& dig, u32* s_top) {
  distribute(c, a, s, dig, false, false);
  finish_round(c, a, s, dig, s_top);
}

// Highest differing key bit + 1 over positions [a, a + s) (through c.perm, or the identity)
// (0: all keys equal).
template <int KW, int RWT>
__device__ u32 range_top_bit(const ChunkCtx<KW, RWT>& c, u32 a, u32 s, bool through_perm) {
  __shared__ u64 red[kCWarps][4];
  __shared__ u32 s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  u64 kand[2] = {~0ull, ~0ull}, kor[2] = {0, 0};
  for (u32 i = tid; i < s; i += kCThreads) {
    const Key<KW> k = c.key(through_perm ? c.perm[a + i] : a + i);
#pragma unroll
    for (int q = 0; q < KW; q++) {
      kand[q] &= k.w[q];
      kor[q] |= k.w[q];
    }
  }
#pragma unroll
  for (int q = 0; q < KW; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kand[q] &= __shfl_xor_sync(kFull, kand[q], o);
      kor[q] |= __shfl_xor_sync(kFull, kor[q], o);
    }
    if (lane == 0) {
      red[warp][q] = kand[q];
      red[warp][2 + q] = kor[q];
    }
  }
  __syncthreads();
  if (tid == 0) {
    u64 a2[2] = {~0ull, ~0ull}, o2[2] = {0, 0};
    for (int wq = 0; wq < kCWarps; wq++)
      for (int q = 0; q < KW; q++) {
        a2[q] &= red[wq][q];
        o2[q] |= red[wq][2 + q];
      }
    s_p = top_bit_plus1(a2[0] ^ o2[0], KW == 2 ? a2[1] ^ o2[1] : 0);
  }
  __syncthreads();
  const u32 p = s_p;
  __syncthreads();
  return p;
}

// Positions [a, a + s) of c.perm hold records with equal keys in some order: put them back in
// input order (increasing record index).  A bitmap of the chunk's record indices (borrowing
// the counters, which are cleared before their next use) marks the bucket's records; a
// record's new place is the number of marked indices below its own.  Ends with a barrier.
template <int KW, int RWT>
__device__ void restore_input_order(const ChunkCtx<KW, RWT>& c, u32 a, u32 s) {
  __shared__ u32 scr[kCWarps];
  constexpr u32 kWords = (1u << kIdxBits) / 32;  // bitmap words over every possible index
  static_assert(kWords <= (u32)kCThreads, "one bitmap word per thread");
  static_assert(2 * kWords <= (u32)kCntWords, "bitmap and prefix fit the counters");
  u32* bm = c.cnt;             // [kWords] the bitmap
  u32* below = c.cnt + kWords;  // [kWords] marked indices in the words before
  const u32 tid = threadIdx.x;
  for (u32 w = tid; w < kWords; w += kCThreads) bm[w] = 0;
  __syncthreads();
  for (u32 i = tid; i < s; i += kCThreads) {
    const u32 r = c.perm[a + i];
    atomicOr(&bm[r >> 5], 1u << (r & 31));
  }
  __syncthreads();
  const u32 mine = tid < kWords ? bm[tid] : 0u;
  const u32 ex = block_exclusive_sum<kCThreads>(__popc(mine), scr);  // ends with a barrier
  if (tid < kWords) below[tid] = ex;
  __syncthreads();
  for (u32 i = tid; i < s; i += kCThreads) {
    const u32 r = c.perm[a + i];
    c.out[a + below[r >> 5] + __popc(bm[r >> 5] & ((1u << (r & 31)) - 1u))] = (u16)r;
  }
  __syncthreads();
  for (u32 i = tid; i < s; i += kCThreads) c.perm[a + i] = c.out[a + i];
  __syncthreads();
}

// A chunk of at most es_max records: enumeration sort of the whole range at once (each
// record's rank among all of them by (key, input position)); the counters stay untouched.
// Kept out of line so that it does not disturb the code of the common path.
template <int KW, int RWT>
__device__ __noinline__ void small_chunk_sort(const ChunkCtx<KW, RWT>& c, u32 sz) {
  for (u32 i = threadIdx.x; i < sz; i += kCThreads) {
    const Key<KW> kr = c.key(i);
    u32 rank = 0;
    for (u32 q = 0; q < sz; q++) {
      const Key<KW> k2 = c.key(q);
      rank += key_less<KW>(k2, kr) || (key_eq<KW>(k2, kr) && q < i);
    }
    c.perm[rank] = (u16)i;
  }
  __syncthreads();
}

// Persistent CTAs take chunks by ticket; the two CTAs of an SM overlap each other's load,
// sort and write.  Per chunk: one bulk copy of its records into shared memory (bounded wait;
// the next chunk's records are meanwhile prefetched into L2), then
//   * more than es_max records: the first distribution counts the digit right below the
//     chunk's shared bits and keeps every record's composite key (CompSpec).  If no bucket
//     holds more than es_max records, the composite keys go to their buckets and a record's
//     place is its bucket's start plus the number of smaller composite keys in the bucket;
//     records of 8 or 16 bytes are written straight there, larger ones through the order
//     array.  Otherwise the round goes on with record indices (finish_round) and recurses on
//     the buckets it leaves on the stack;
//   * at most es_max records: one enumeration sort of the whole chunk;
//   * already in order: copied to `in` if it lives in tmp.
template <int KW, int RWT>
__global__ void __launch_bounds__(kCThreads, kChunkCtas) k_chunk(Job j) {
  Ctl* ctl = j.ctl;
  const u64 nch = ctl->nchunks;
  if (nch == 0 || call_failed(ctl)) return;
  if (nch + ctl->ntiny > j.cap_chunks) {  // the two lists met (reported when they were filled)
    if (blockIdx.x == 0 && threadIdx.x == 0) report(ctl, kErrOverflow);
    return;
  }
  const u32 RW = RWT ? (u32)RWT : j.RW;
  const u32 m = j.chunk_max;
  const ChunkLayout lay = chunk_layout(m, RW);
  extern __shared__ __align__(16) unsigned char smem[];
  ChunkCtx<KW, RWT> c;
  c.km0 = j.keymask[0];
  c.km1 = j.keymask[1];
  c.RW = RW;
  u64* stage = (u64*)(smem + lay.stage);
  c.stage = stage;
  u64* comp = (u64*)(smem + lay.aux);  // first round: composite keys
  c.perm = (u16*)(smem + lay.aux);     // general rounds: two order arrays and the stack
  c.out = c.perm + m;
  c.stack = (u32*)(smem + lay.aux + (size_t)m * 4);
  c.es_max = j.es_max;
  c.stack_cap = m / (c.es_max + 1) + 2;
  c.cnt = (u32*)(smem + lay.cnt);
  __shared__ Chunk s_ch;
  __shared__ __align__(16) Chunk s_next;  // the next ticket's descriptor, copied in by cp.async
  __shared__ u64 s_t, s_nt;
  __shared__ u32 s_top;
  __shared__ __align__(8) u64 s_bar[kCWarps];  // bar w: warp w's strip of the chunk has landed
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr u32 kIdxMask = (1u << kIdxBits) - 1u;
  u32 bar_phase = 0;

  // thread 0: publish ticket t with its descriptor `raw` (an unusable one is reported, not
  // used) and ask for its records to be brought into L2
  auto fetch = [&](u64 t, Chunk raw) {
    Chunk ch = {};
    if (t < nch) {
      ch = raw;
      if (ch.size > m || ch.begin > j.n || ch.begin + ch.size > j.n) {
        report(ctl, kErrInternal);
        ch.size = 0;
      }
      if (ch.size) prefetch_l2(j.buf[(ch.flags & kChSrcTmp) ? 1 : 0] + ch.begin * RW, (u64)ch.size * RW * 8);
    }
    s_ch = ch;
    s_t = t;
  };
  // Tickets are dispensed in batches when chunks are many (many tiny segments): thread 0
  // owns tickets [t_next, t_end) and takes the next batch with one atomic.
  const u64 batch = nch >= (u64)gridDim.x * 2048 ? 8 : 1;
  u64 t_next = 0, t_end = 0;
  auto take = [&]() -> u64 {
    if (t_next == t_end) {
      t_next = atomicAdd(&ctl->chunk_ticket, batch);
      t_end = t_next + batch;
    }
    return t_next++;
  };
  for (u32 i = tid; i < (u32)kCntWords; i += kCThreads) c.cnt[i] = 0;
  if (tid < kCWarps) mbar_init(&s_bar[tid], 1);
  if (tid == 0) {
    const u64 t = take();
    Chunk raw = {};
    if (t < nch) raw = j.chunks[t];
    fetch(t, raw);
  }
  __syncthreads();
  for (;;) {
    if (s_t >= nch) break;  // a CTA's tickets only grow: no later chunk either
    const Chunk ch = s_ch;
    const u32 sz = ch.size;
    const bool in_place = !(ch.flags & kChSrcTmp), copy_only = (ch.flags & kChCopyOnly) != 0;
    // the records come in by bulk copies when they start on a 16-byte boundary (an even word
    // count per record: always), one per warp strip of S records, each completing on its
    // own barrier; else by 16- or 8-byte copies of every thread
    const u64* src = j.buf[in_place ? 0 : 1] + ch.begin * RW;
    const u32 bytes = sz * RW * 8;
    const bool load = sz && !(copy_only && in_place);
    const bool bulk = load && ((((uintptr_t)src) | bytes) & 15) == 0;
    // strips of S records, a multiple of 32: the warps share the chunk evenly, S <= 32 *
    // kChunkItems (kCWarps * 32 * kChunkItems >= chunk_max)
    const u32 S = 32u * ((sz + kCThreads - 1) / kCThreads);
    if (load && !bulk) load_words_async<kCThreads>(stage, src, (u64)sz * RW);
    if (bulk && lane == 0) {
      // (strip boundaries are multiples of 32 records: 16-byte aligned, as is the chunk's end)
      const u32 a = min(sz, warp * S), e = min(sz, a + S);
      fence_proxy_async_smem();  // the last chunk's reads of the stage are done (barrier)
      if (e > a) bulk_load(stage + (u64)a * RW, src + (u64)a * RW, (e - a) * RW * 8, &s_bar[warp]);
      else mbar_arrive(&s_bar[warp]);
    }
    if (tid == 0) {  // the next ticket; its descriptor comes into s_next (published after the wait)
      const u64 nt = take();
      s_nt = nt;
      static_assert(sizeof(Chunk) == 32, "a descriptor is two 16-byte copies");
      if (nt < nch) {
        cp_async16(&s_next, j.chunks + nt);
        cp_async16(reinterpret_cast<char*>(&s_next) + 16, reinterpret_cast<const char*>(j.chunks + nt) + 16);
      }
      cp_async_commit();
    }
    u64* dst = j.buf[0] + ch.begin * RW;
    DigitSpec dig = {};
    u32 p = ch.p;
    bool sort = sz && !copy_only;
    if (sort && p) {  // shared bits known from the level that produced the chunk
      dig = window_below(p, sz);
      if (ch.sb) {
        dig.sb = ch.sb;
        dig.plo = p;
        dig.pw = ch.pw;
        dig.v0 = ch.v0;
        dig.w = p > (u32)kWinBits - ch.sb ? (u32)kWinBits - ch.sb : p;
        dig.lo = p - dig.w;
      }
    }
    // bounded waits, each warp for its own strip (a copy cannot be cancelled: after a timeout
    // the CTA still waits for every strip, with the default limit, before it leaves)
    bool failed = false;
    if (bulk) failed = !mbar_wait(&s_bar[warp], bar_phase, j.wd_polls);
    if (!bulk) cp_async_wait_all();
    auto give_up = [&]() {
      if (tid == 0) report(ctl, kErrTimeout);
      if (bulk) mbar_wait(&s_bar[warp], bar_phase, kWaitPolls);
    };
    // the first round counts each warp's own strip as soon as it has landed; every other path
    // reads the whole chunk and waits for all strips first
    const bool strips = bulk && sort && p && sz > c.es_max;
    if (!strips) {
      if (__syncthreads_or(failed)) {
        give_up();
        return;
      }
      if (bulk) bar_phase ^= 1;
      if (tid == 0) {  // every thread has read s_ch and s_t (barrier above)
        cp_async_wait_all();
        fetch(s_nt, s_next);
      }
      if (sort && !p) {
        p = range_top_bit(c, 0, sz, false);  // (ends with a barrier)
        sort = p != 0;
        dig = window_below(p, sz);
      }
    }
    bool via_perm = false;  // the sorted order is in c.perm (else the records are written)
    if (sort && sz > c.es_max) {
      // first round: count the digit, keeping every record's composite key
      const CompSpec cs = comp_spec(dig, p, c.km0, c.km1);
      u64 ck[kChunkItems];
      u32 held[kChunkItems];  // (digit << 16) | rank among the digit's records counted before
#pragma unroll
      for (int k = 0; k < kChunkItems; k++) {
        const u32 i = warp * S + k * 32 + lane;  // (this warp's strip)
        held[k] = 0xffffffffu;
        ck[k] = 0;
        if (i < sz && k * 32 < S) {
          ck[k] = (cs.keypart<KW>(c.key(i)) << kIdxBits) | i;
          const u32 d = (u32)(ck[k] >> cs.dshift) & cs.dmask;
          const u32 old = atomicAdd(&c.cnt[d >> 1], 1u << ((d & 1) * 16));
          held[k] = ((old >> ((d & 1) * 16)) & 0xffffu) | (d << 16);
        }
      }
      if (tid == 0) s_top = 0;
      if (strips) {
        if (__syncthreads_or(failed)) {
          give_up();
          return;
        }
        bar_phase ^= 1;
        if (tid == 0) {  // every thread has read s_ch and s_t (barrier above)
        cp_async_wait_all();
        fetch(s_nt, s_next);
      }
      } else {
        __syncthreads();
      }
      const u32 nd = cs.dmask + 1;
      const bool big = scan_counts(c, nd < 2 ? 2 : nd, c.es_max);  // (ends with a barrier)
      if (!big) {
#pragma unroll
        for (int k = 0; k < kChunkItems; k++)
          if (held[k] != 0xffffffffu) comp[c.count_of(held[k] >> 16) + (held[k] & 0xffffu)] = ck[k];
        __syncthreads();
        // a record's place: its bucket's start + the smaller composite keys of its bucket
        u32 placed[kChunkItems];  // (place << 16) | record, for records of more than 16 bytes
#pragma unroll
        for (int k = 0; k < kChunkItems; k++) {
          const u32 i = tid + k * kCThreads;
          placed[k] = 0xffffffffu;
          if (i < sz) {
            const u64 cm = comp[i];
            const u32 d = (u32)(cm >> cs.dshift) & cs.dmask;
            const u32 st = c.count_of(d), en = d < cs.dmask ? c.count_of(d + 1) : sz;
            u32 rank = 0;
            if (cs.t == 0) {
              for (u32 q = st; q < en; q++) rank += comp[q] < cm;
            } else {
              for (u32 q = st; q < en; q++) {
                const u64 cq = comp[q];
                bool lt = cq < cm;
                if (cq != cm && (cq ^ cm) <= (u64)kIdxMask) {  // equal kept key bits: whole keys
                  const Key<KW> kq = c.key((u32)cq & kIdxMask), km = c.key((u32)cm & kIdxMask);
                  lt = key_less<KW>(kq, km) || (key_eq<KW>(kq, km) && cq < cm);
                }
                rank += lt;
              }
            }
            const u32 r = (u32)cm & kIdxMask, pos = st + rank;
            if (RW <= 2) {
              const u64* sp = stage + (u64)r * RW;
              u64* dp = dst + (u64)pos * RW;
              if (RW == 2)
                *reinterpret_cast<ulonglong2*>(dp) = *reinterpret_cast<const ulonglong2*>(sp);
              else
                *dp = sp[0];
            } else {
              placed[k] = (pos << 16) | r;
            }
          }
        }
        __syncthreads();  // composite keys and counters are read
        if (RW > 2) {
#pragma unroll
          for (int k = 0; k < kChunkItems; k++)
            if (placed[k] != 0xffffffffu) c.perm[placed[k] >> 16] = (u16)(placed[k] & 0xffffu);
          via_perm = true;
        }
      } else {
        // a bucket of more than es_max records: the general rounds, on record indices
#pragma unroll
        for (int k = 0; k < kChunkItems; k++)
          if (held[k] != 0xffffffffu)
            c.out[c.count_of(held[k] >> 16) + (held[k] & 0xffffu)] = (u16)(warp * S + k * 32 + lane);
        __syncthreads();
        finish_round(c, 0, sz, dig, &s_top);
        while (s_top) {  // s_top is final after the barrier that ends every round
          const u32 top = s_top;
          if (top > c.stack_cap) {  // cannot happen: buckets on the stack are disjoint and > es_max
            if (tid == 0) report(ctl, kErrInternal);
            break;
          }
          const u32 a = c.stack[2 * (top - 1)], s = c.stack[2 * (top - 1) + 1];
          __syncthreads();
          if (tid == 0) s_top = top - 1;
          __syncthreads();
          const u32 pp = range_top_bit(c, a, s, true);
          if (pp) {
            sort_round(c, a, s, window_below(pp), &s_top);
          } else {  // all keys equal: back to input order
            restore_input_order(c, a, s);
          }
        }
        via_perm = true;
      }
      // counters back to zero for the next chunk's first distribution
      for (u32 i = tid; i < (u32)kCntWords; i += kCThreads) c.cnt[i] = 0;
      __syncthreads();  // (the order array is complete)
    } else if (sort) {
      small_chunk_sort(c, sz);  // (ends with a barrier)
      via_perm = true;
    }
    if (via_perm) {
      // write the records in sorted order
      if (RW == 2) {
        for (u32 s = tid; s < sz; s += kCThreads) {
          const u32 r = c.perm[s];
          const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(stage + 2 * (u64)r);
          __stcs(reinterpret_cast<ulonglong2*>(dst + 2 * (u64)s), v);
        }
      } else if (RWT != 0 && (RW & 1)) {
        for (u32 q = tid; q < sz * RW; q += kCThreads) {
          const u32 s = q / RW, w = q - s * RW;
          __stcs(dst + q, stage[(u64)c.perm[s] * RW + w]);
        }
      } else {
        // whole warps write consecutive records: lane k * P + piece moves one piece (16 bytes
        // if RW is even, else 8) of record s0 + k (P <= 32: records are at most 256 bytes)
        const bool pairs = (RW & 1) == 0;
        const u32 P = pairs ? RW >> 1 : RW, rpw = 32 / P;
        const u32 k = lane / P, piece = lane - k * P;
        for (u32 s0 = warp * rpw; s0 < sz; s0 += kCWarps * rpw) {
          const u32 s = s0 + k;
          if (k >= rpw || s >= sz) continue;
          const u64* sp = stage + (u64)c.perm[s] * RW;
          u64* d = dst + (u64)s * RW;
          if (pairs)
            __stcs(reinterpret_cast<ulonglong2*>(d) + piece, reinterpret_cast<const ulonglong2*>(sp)[piece]);
          else
            __stcs(d + piece, sp[piece]);
        }
      }
    } else if (!sort && sz && !in_place) {  // already in order, but in tmp
      const u64 words = (u64)sz * RW;
      for (u64 i = tid; i < words; i += kCThreads) __stcs(dst + i, stage[i]);
    }
    __syncthreads();  // the stage is free and s_ch describes the next chunk
  }
}

// Finished ranges that live in tmp: copy to in.
__global__ void __launch_bounds__(kThreads) k_copy(Job j) {
  Ctl* ctl = j.ctl;
  const u64 np = ctl->npieces;
  if (np == 0 || call_failed(ctl)) return;
  __shared__ u64 s_ticket;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(&ctl->piece_ticket, 1ull);
    __syncthreads();
    const u64 t = s_ticket;
    __syncthreads();
    if (t >= np) break;
    const Piece pc = j.pieces[t];
    if (pc.begin > j.n || pc.size > j.n - pc.begin) {
      if (threadIdx.x == 0) report(ctl, kErrInternal);
      continue;
    }
    const u64 words = pc.size * j.RW;
    const u64* src = j.buf[1] + pc.begin * j.RW;
    u64* dst = j.buf[0] + pc.begin * j.RW;
    if (((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0) {
      const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(src);
      ulonglong2* d2 = reinterpret_cast<ulonglong2*>(dst);
      for (u64 i = threadIdx.x; i < words / 2; i += kThreads) __stcs(d2 + i, __ldcs(s2 + i));
      if ((words & 1) && threadIdx.x == 0) dst[words - 1] = src[words - 1];
    } else {
      for (u64 i = threadIdx.x; i < words; i += kThreads) __stcs(dst + i, __ldcs(src + i));
    }
  }
}

size_t chunk_smem_bytes(const Job& j) { return chunk_layout(j.chunk_max, j.RW).total; }

template <int KW>
static cudaError_t launch_chunks_kw(const Job& j, u32 grid, cudaStream_t s) {
  const size_t sm = chunk_smem_bytes(j);
#define RS_CH(R)                                                                     \
  do {                                                                               \
    ensure_smem((const void*)k_chunk<KW, R>, sm);                                    \
    k_chunk<KW, R><<<grid, kCThreads, sm, s>>>(j);                                  \
  } while (0)
  switch (j.RW) {
    case 1: RS_CH(1); break;
    case 2: RS_CH(2); break;
    case 3: RS_CH(3); break;
    case 4: RS_CH(4); break;
    default: RS_CH(0); break;
  }
#undef RS_CH
  return cudaGetLastError();
}

int chunk_ctas_per_sm(const Job& j) {
  int n = 0;
  const size_t sm = chunk_smem_bytes(j);
  if (j.KW == 1) {
    n = occupancy((const void*)k_chunk<1, 0>, kCThreads, sm);
  } else {
    n = occupancy((const void*)k_chunk<2, 0>, kCThreads, sm);
  }
  return n < 1 ? 1 : n;
}

int launch_chunks(const Job& j, u32 grid, cudaStream_t s) {
  cudaError_t e = j.KW == 1 ? launch_chunks_kw<1>(j, grid, s) : launch_chunks_kw<2>(j, grid, s);
  return e == cudaSuccess ? 1 : -1;
}

// ------------------------------------------------------------------------------ tiny
// Chunks of at most kTinyMax = 64 records (tiny segments of a batched sort, short packed runs):
// warps instead of CTAs (the paper's tiny-array sorter, section 2.2).  A warp reads the
// descriptors of 32 consecutive tiny chunks at once (one per lane), then sorts them in rounds:
// a chunk of more than 32 records takes the whole warp (tiny_sort64); otherwise a round takes
// the next G chunks that all fit in w = 32 / G records (w a power of two), one group of w
// lanes per chunk, and
//   * stages each lane's record in the warp's slice of shared memory (so a chunk may be sorted
//     in place),
//   * sorts every group's pairs (key, input position) ascending with a bitonic network over
//     its w lanes -- compare-exchange partners by shuffles; the position breaks ties, so the
//     order is the stable one; lanes past a chunk's end hold the largest key and positions
//     past every real one, so they sort last --
//   * and writes lane r's output record r of its chunk from the slice.
// Warps take batches of chunks by a static stride (tiny chunks are all alike).
constexpr int kTinyThreads = 256;
constexpr int kTinyWarps = kTinyThreads / 32;

// One chunk of 33..64 records by one warp: lane l holds records l and l + 32 (the second pair
// of the bitonic network's elements); the stages that pair element e with e + 32 compare
// within a lane, the others exchange both elements by shuffles.
template <int KW>
__device__ __forceinline__ void tiny_sort64(const Job& j, u64 begin, u32 size, u32 flags, const u64* slice,
                                            u32 lane) {
  const u32 RW = j.RW;
  u64* sl = const_cast<u64*>(slice);
  const u64* src = j.buf[(flags & kChSrcTmp) ? 1 : 0] + begin * RW;
  u64* dst = j.buf[0] + begin * RW;
  if (flags & kChCopyOnly) {  // in order already; copy it to `in` if it lives in tmp
    if (flags & kChSrcTmp)
      for (u32 q = lane; q < size * RW; q += 32) __stcs(dst + q, src[q]);
    return;
  }
  for (u32 q = lane; q < size * RW; q += 32) sl[q] = src[q];
  __syncwarp();
  Key<KW> ka, kb;
  u32 ia = lane, ib = lane + 32;
#pragma unroll
  for (int q = 0; q < KW; q++) ka.w[q] = kb.w[q] = ~0ull;
  if (ia < size) {
    ka.w[0] = sl[ia * RW] & j.keymask[0];
    if (KW == 2) ka.w[KW - 1] = sl[ia * RW + 1] & j.keymask[1];
  }
  if (ib < size) {
    kb.w[0] = sl[ib * RW] & j.keymask[0];
    if (KW == 2) kb.w[KW - 1] = sl[ib * RW + 1] & j.keymask[1];
  }
  auto less = [](const Key<KW>& x, u32 xi, const Key<KW>& y, u32 yi) {
    return key_less<KW>(x, y) || (key_eq<KW>(x, y) && xi < yi);
  };
  // one compare-exchange of element e (key k, position i) with its partner across lanes
  auto cross = [&](Key<KW>& k, u32& i, u32 e, u32 blk, u32 d) {
    Key<KW> o;
#pragma unroll
    for (int q = 0; q < KW; q++) o.w[q] = __shfl_xor_sync(kFull, k.w[q], d);
    const u32 oi = __shfl_xor_sync(kFull, i, d);
    const bool o_less = less(o, oi, k, i);
    const bool ascending = (e & blk) == 0, lower = (e & d) == 0;
    if (ascending == lower ? o_less : !o_less) {
      k = o;
      i = oi;
    }
  };
#pragma unroll
  for (u32 blk = 2; blk <= 64; blk <<= 1) {
#pragma unroll
    for (u32 d = blk >> 1; d > 0; d >>= 1) {
      if (d == 32) {  // elements lane and lane + 32: the lower one keeps the smaller (blk = 64)
        if (less(kb, ib, ka, ia)) {
          const Key<KW> tk = ka;
          ka = kb;
          kb = tk;
          const u32 ti = ia;
          ia = ib;
          ib = ti;
        }
      } else {
        cross(ka, ia, lane, blk, d);
        cross(kb, ib, lane + 32, blk, d);
      }
    }
  }
  // output record e = input record i_e
  const u32 outs[2] = {lane, lane + 32}, from[2] = {ia, ib};
#pragma unroll
  for (int h = 0; h < 2; h++) {
    if (outs[h] >= size) continue;
    const u64* sp = slice + (size_t)from[h] * RW;
    u64* dp = dst + (u64)outs[h] * RW;
    if ((RW & 1) == 0) {
      for (u32 q = 0; q < RW; q += 2)
        __stcs(reinterpret_cast<ulonglong2*>(dp + q), *reinterpret_cast<const ulonglong2*>(sp + q));
    } else {
      for (u32 q = 0; q < RW; q++) __stcs(dp + q, sp[q]);
    }
  }
  __syncwarp();  // the slice is reused by the next chunk
}

template <int KW>
__global__ void __launch_bounds__(kTinyThreads) k_tiny(Job j) {
  Ctl* ctl = j.ctl;
  const u64 nt = ctl->ntiny;
  if (nt == 0 || call_failed(ctl)) return;
  if (ctl->nchunks + nt > j.cap_chunks) {  // the two lists met (reported when they were filled)
    if (blockIdx.x == 0 && threadIdx.x == 0) report(ctl, kErrOverflow);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  const u32 RW = j.RW;
  const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* mine = reinterpret_cast<u64*>(smem) + ((size_t)warp * kTinyMax + lane) * RW;  // this lane's record
  const u64* slice = reinterpret_cast<const u64*>(smem) + (size_t)warp * kTinyMax * RW;
  const u64 warps = (u64)gridDim.x * kTinyWarps;
  for (u64 t0 = ((u64)blockIdx.x * kTinyWarps + warp) * 32; t0 < nt; t0 += warps * 32) {
    const u32 nb = (u32)min((u64)32, nt - t0);
    // lane i: descriptor of chunk t0 + i (an unusable one is reported and left out)
    u64 c_begin = 0;
    u32 c_size = 0, c_flags = 0;
    if (lane < nb) {
      const Chunk ch = j.chunks[j.cap_chunks - 1 - (t0 + lane)];
      if (ch.size > kTinyMax || ch.begin > j.n || ch.begin + ch.size > j.n) {
        report(ctl, kErrInternal);
      } else {
        c_begin = ch.begin;
        c_size = ch.size;
        c_flags = ch.flags;
      }
    }
    // fits[q]: lanes whose chunk holds at most 2^q records
    u32 fits[6];
#pragma unroll
    for (int q = 1; q <= 5; q++) fits[q] = __ballot_sync(kFull, c_size <= (1u << q)) | ~((nb < 32 ? (1u << nb) : 0u) - 1u);
    for (u32 p = 0; p < nb;) {
      if (!((fits[5] >> p) & 1u)) {  // 33..64 records: the whole warp, two records per lane
        tiny_sort64<KW>(j, __shfl_sync(kFull, c_begin, p), __shfl_sync(kFull, c_size, p),
                        __shfl_sync(kFull, c_flags, p), slice, lane);
        p++;
        continue;
      }
      // widest grouping: G = 32 / w chunks starting at p, each of at most w records
      u32 lw = 5;
      for (u32 q = 1; q < 5; q++) {
        const u32 G = 32u >> q;
        const u32 span = G >= 32 ? kFull : ((1u << G) - 1u);
        if (p + G <= 32 && ((fits[q] >> p) & span) == span) {
          lw = q;
          break;
        }
      }
      const u32 w = 1u << lw, G = 32u >> lw;
      const u32 g = lane >> lw, r = lane & (w - 1), c = p + g;
      const u32 src_lane = c < 32 ? c : 31;  // (always c < 32: p + G <= 32, or G = 1)
      const u64 begin = __shfl_sync(kFull, c_begin, src_lane);
      const u32 size_c = __shfl_sync(kFull, c_size, src_lane), size = c < nb ? size_c : 0u;
      const u32 flags = __shfl_sync(kFull, c_flags, src_lane);
      const bool live = c < nb && r < size;
      const u64* src = j.buf[(flags & kChSrcTmp) ? 1 : 0] + (begin + r) * RW;
      u64* dst = j.buf[0] + (begin + r) * RW;
      if (live)
        for (u32 q = 0; q < RW; q++) mine[q] = src[q];
      __syncwarp();
      Key<KW> key;
      u32 idx = r;
      if (live) {
        key.w[0] = mine[0] & j.keymask[0];
        if (KW == 2) key.w[KW - 1] = mine[1] & j.keymask[1];
      } else {
#pragma unroll
        for (int q = 0; q < KW; q++) key.w[q] = ~0ull;
      }
      for (u32 blk = 2; blk <= w; blk <<= 1) {
        for (u32 d = blk >> 1; d > 0; d >>= 1) {
          Key<KW> o;
#pragma unroll
          for (int q = 0; q < KW; q++) o.w[q] = __shfl_xor_sync(kFull, key.w[q], d);
          const u32 oi = __shfl_xor_sync(kFull, idx, d);
          const bool o_less = key_less<KW>(o, key) || (key_eq<KW>(o, key) && oi < idx);
          // an ascending block keeps the smaller pair in its lower lane, a descending one the
          // larger; the last merge of a group is ascending
          const bool ascending = (r & blk) == 0, lower = (lane & d) == 0;
          if (ascending == lower ? o_less : !o_less) {
            key = o;
            idx = oi;
          }
        }
      }
      // lane r writes its chunk's output record r: input record idx of the group (a chunk
      // already in order keeps every record where it is, copied to `in` if it lives in tmp)
      const bool copy_only = (flags & kChCopyOnly) != 0;
      if (live && !(copy_only && (flags & kChSrcTmp) == 0)) {
        const u64* sp = slice + (size_t)((g << lw) + (copy_only ? r : idx)) * RW;
        if ((RW & 1) == 0) {
          for (u32 q = 0; q < RW; q += 2)
            __stcs(reinterpret_cast<ulonglong2*>(dst + q), *reinterpret_cast<const ulonglong2*>(sp + q));
        } else {
          for (u32 q = 0; q < RW; q++) __stcs(dst + q, sp[q]);
        }
      }
      __syncwarp();  // the slice is reused by the next round
      p += G;
    }
  }
}

int launch_tiny(const Job& j, u32 sms, cudaStream_t s) {
  const size_t sm = (size_t)kTinyWarps * kTinyMax * j.RW * 8;
  const u32 per_sm = (u32)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / sm));
  cudaError_t e;
  if (j.KW == 1) {
    ensure_smem((const void*)k_tiny<1>, sm);
    k_tiny<1><<<sms * per_sm, kTinyThreads, sm, s>>>(j);
  } else {
    ensure_smem((const void*)k_tiny<2>, sm);
    k_tiny<2><<<sms * per_sm, kTinyThreads, sm, s>>>(j);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? 1 : -1;
}

int launch_copy(const Job& j, u32 grid, cudaStream_t s) {
  k_copy<<<grid, kThreads, 0, s>>>(j);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// chunk_max for a record size: the largest range whose staged records and composite keys fit
// the shared memory of the chunk CTA (and whose positions fit kIdxBits bits).
u32 chunk_capacity(u32 RW) {
  const size_t budget = kChunkSmem - kChunkFixed;
  u32 m = (u32)(budget / (RW * 8 + 8));  // the staged record + its composite key (or two u16 indices)
  m &= ~63u;
  if (m > (u32)kCThreads * kChunkItems) m = kCThreads * kChunkItems;
  if (m > (1u << kIdxBits)) m = 1u << kIdxBits;
  return m;
}

}  // namespace rsg
