// On-chip sorting of small bins (Kokot et al., sections 3.2-3.3) and the final copy-back.
//
// One CTA sorts a chunk (one small bin, or several consecutive small sub-bins of one parent)
// completely in shared memory: the records are staged once, a permutation of their indices
// is sorted, and the records are written once, in order, to `in`.  Because every record is
// staged before any is written, the chunk may be sorted in place.
//
// The index sort follows the paper's small/tiny-bin scheme on chip: skip the key bits that
// every record of the range shares (AND/OR of the keys), then a counting-sort distribution on
// the next 16 bits (two stable 8-bit passes), then the runs of records equal in those bits:
// runs of up to kEsMax records are finished by enumeration sort (each record's rank = the
// number of records that must precede it, section 2.2 and 3.3); longer runs go through the
// same steps again (a run whose keys are all equal is already in order).  Ties are broken by the record's input
// position, so the chunk sort is stable and the whole sorter is stable.
#include "rs_internal.cuh"

namespace rsg {

constexpr int kEsMax = 48;           // longest run finished by enumeration sort
constexpr int kChunkItems = 12;      // index-sort items per thread (chunk_max <= 512 * 12)
// per-CTA shared memory the chunk kernel may use (two CTAs per SM), and what is not per record
constexpr size_t kChunkSmem = 112 * 1024;
constexpr size_t kChunkFixed = 2 * 1024 + kWarps * 256 * 2 + 1024;

struct ChunkLayout {
  size_t stage, permA, permB, win, whist, stack, total;
};

__host__ __device__ inline ChunkLayout chunk_layout(u32 m, u32 RW) {
  ChunkLayout c;
  size_t o = 0;
  c.stage = o; o += (size_t)m * RW * 8;
  c.permA = o; o += (size_t)m * 2;
  c.permB = o; o += (size_t)m * 2;
  c.win = o; o += (size_t)(m + 1) * 2 + 2;
  o = (o + 15) & ~(size_t)15;
  c.whist = o; o += (size_t)kWarps * 256 * 2;
  c.stack = o; o += (size_t)(m / (kEsMax + 1) + 2) * 8;
  c.total = (o + 127) & ~(size_t)127;
  return c;
}

template <int KW, int RWT>
struct ChunkCtx {
  u64 km0, km1;   // key bits of words 0 and 1
  u32 RW;
  const u64* stage;
  u16* permA;
  u16* permB;
  u16* win;       // window digit of each position of the range being sorted
  u16* whist;
  u32* stack;  // pairs (begin, size)
  u32 stack_cap;

  __device__ __forceinline__ Key<KW> key(u32 r) const {
    const u64* p = stage + r * (RWT ? (u32)RWT : RW);
    Key<KW> k;
    k.w[0] = p[0] & km0;
    if (KW == 2) k.w[KW - 1] = p[1] & km1;
    return k;
  }
};

// Stable counting sort of positions [a, a + s) of `src` into `dst` by key bits [lo, lo + w).
template <int KW, int RWT>
__device__ void lsd_pass(const ChunkCtx<KW, RWT>& c, const u16* src, u16* dst, u32 a, u32 s, u32 lo, u32 w) {
  __shared__ u32 tcount[256];
  __shared__ u32 scan_scr[kWarps + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 nd = 1u << w;
  for (u32 i = tid; i < (u32)kWarps * nd; i += kThreads) c.whist[i] = 0;
  __syncthreads();
  const u32 per_warp = ((s + kWarps * 32 - 1) / (kWarps * 32)) * 32;
  const u32 items = per_warp / 32;
  u16* wh = c.whist + warp * nd;
  u32 packed[kChunkItems];
#pragma unroll
  for (int it = 0; it < kChunkItems; it++) {
    packed[it] = 0xffffffffu;
    if ((u32)it < items) {
      const u32 pos = warp * per_warp + it * 32 + lane;
      const bool valid = pos < s;
      u32 d = 0;
      if (valid) d = digit_of<KW>(c.key(src[a + pos]), lo, w);
      const u32 peers = __match_any_sync(kFull, valid ? d : (0x10000u | lane));
      const u32 before = __popc(peers & lanemask_lt());
      u32 old = 0;
      if (valid) old = wh[d];
      __syncwarp();
      if (valid && before == 0) wh[d] = (u16)(old + __popc(peers));
      __syncwarp();
      if (valid) packed[it] = (old + before) | (d << 16);
    }
  }
  __syncthreads();
  for (u32 v = tid; v < nd; v += kThreads) {
    u32 run = 0;
    for (int q = 0; q < kWarps; q++) {
      const u32 x = c.whist[q * nd + v];
      c.whist[q * nd + v] = (u16)run;
      run += x;
    }
    tcount[v] = run;
  }
  __syncthreads();
  block_exclusive_scan(tcount, nd, scan_scr);
#pragma unroll
  for (int it = 0; it < kChunkItems; it++) {
    if (packed[it] != 0xffffffffu) {
      const u32 d = packed[it] >> 16;
      const u32 pos = warp * per_warp + it * 32 + lane;
      dst[a + tcount[d] + wh[d] + (packed[it] & 0xffffu)] = src[a + pos];
    }
  }
  __syncthreads();
}

// Sort positions [a, a + s) of permA by the full key, given that every key bit >= p is
// shared by the range.  Runs longer than kEsMax go on the stack for another round.
template <int KW, int RWT>
__device__ void sort_round(const ChunkCtx<KW, RWT>& c, u32 a, u32 s, u32 p, u32* s_top) {
  const int tid = threadIdx.x;
  const u32 lo1 = p > 16 ? p - 16 : 0;
  const u32 wall = p - lo1;
  const u32 wlo = wall > 8 ? wall - 8 : 0;
  const u32 whi = wall - wlo;
  if (wlo) {
    lsd_pass(c, c.permA, c.permB, a, s, lo1, wlo);
    lsd_pass(c, c.permB, c.permA, a, s, lo1 + wlo, whi);
  } else {
    lsd_pass(c, c.permA, c.permB, a, s, lo1, whi);
    for (u32 i = tid; i < s; i += kThreads) c.permA[a + i] = c.permB[a + i];
    __syncthreads();
  }
  // window digit (key bits [lo1, p)) of every position: non-decreasing along the range, so a
  // run of equal digits is found by looking at neighbours and by binary search
  u16* win = c.win;
  for (u32 i = tid; i < s; i += kThreads) win[i] = (u16)digit_of<KW>(c.key(c.permA[a + i]), lo1, wall);
  __syncthreads();
  for (u32 i = tid; i < s; i += kThreads) {
    const u32 d = win[i];
    const u32 r = c.permA[a + i];
    const bool head = i == 0 || win[i - 1] != d;
    const bool last = i + 1 == s || win[i + 1] != d;
    if (head && last) {  // a run of one record
      c.permB[a + i] = (u16)r;
      continue;
    }
    // run start: first position with digit d in [i - kEsMax, i]
    bool lng = false;
    u32 st = i, en = i + 1;
    const u32 L = i >= (u32)kEsMax ? i - kEsMax : 0;
    if (i >= (u32)kEsMax && win[L] == d) {
      lng = true;
    } else {
      u32 lo = L, hi = i;
      while (lo < hi) {
        const u32 mid = (lo + hi) >> 1;
        if (win[mid] < d) lo = mid + 1; else hi = mid;
      }
      st = lo;
      const u32 H = min(s - 1, i + kEsMax);
      if (i + kEsMax < s && win[H] == d) {
        lng = true;
      } else {
        u32 lo2 = i + 1, hi2 = H + 1;
        while (lo2 < hi2) {
          const u32 mid = (lo2 + hi2) >> 1;
          if (win[mid] <= d) lo2 = mid + 1; else hi2 = mid;
        }
        en = lo2;
        lng = en - st > (u32)kEsMax;
      }
    }
    if (lng) {  // stays in place for now; its head measures it and pushes it
      c.permB[a + i] = (u16)r;
      if (head) {
        u32 lo2 = i + 1, hi2 = s;
        while (lo2 < hi2) {
          const u32 mid = (lo2 + hi2) >> 1;
          if (win[mid] <= d) lo2 = mid + 1; else hi2 = mid;
        }
        const u32 t = atomicAdd(s_top, 1u);
        if (t < c.stack_cap) {
          c.stack[2 * t] = a + i;
          c.stack[2 * t + 1] = lo2 - i;
        }
      }
      continue;
    }
    // enumeration sort: rank = records of the run that must precede this one
    const Key<KW> kr = c.key(r);
    u32 rank = 0;
    for (u32 q = st; q < en; q++) {
      const u32 r2 = c.permA[a + q];
      const Key<KW> k2 = c.key(r2);
      rank += key_less<KW>(k2, kr) || (key_eq<KW>(k2, kr) && r2 < r);
    }
    c.permB[a + st + rank] = (u16)r;
  }
  __syncthreads();
  for (u32 i = tid; i < s; i += kThreads) c.permA[a + i] = c.permB[a + i];
  __syncthreads();
}

// Highest differing key bit + 1 over positions [a, a + s) of permA (0: all keys equal).
template <int KW, int RWT>
__device__ u32 range_top_bit(const ChunkCtx<KW, RWT>& c, u32 a, u32 s, bool through_perm) {
  __shared__ u64 red[kWarps][4];
  __shared__ u32 s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  u64 kand[2] = {~0ull, ~0ull}, kor[2] = {0, 0};
  for (u32 i = tid; i < s; i += kThreads) {
    const Key<KW> k = c.key(through_perm ? c.permA[a + i] : a + i);
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
    for (int w = 0; w < kWarps; w++)
      for (int q = 0; q < KW; q++) {
        a2[q] &= red[w][q];
        o2[q] |= red[w][2 + q];
      }
    s_p = top_bit_plus1(a2[0] ^ o2[0], KW == 2 ? a2[1] ^ o2[1] : 0);
  }
  __syncthreads();
  const u32 p = s_p;
  __syncthreads();
  return p;
}

template <int KW, int RWT>
__global__ void __launch_bounds__(kThreads, 2) k_chunk(Job j) {
  Ctl* ctl = j.ctl;
  const u64 nch = ctl->nchunks;
  if (nch == 0) return;
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
  c.permA = (u16*)(smem + lay.permA);
  c.permB = (u16*)(smem + lay.permB);
  c.win = (u16*)(smem + lay.win);
  c.whist = (u16*)(smem + lay.whist);
  c.stack = (u32*)(smem + lay.stack);
  c.stack_cap = m / (kEsMax + 1) + 2;
  __shared__ u64 s_ticket;
  __shared__ u32 s_top;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_ticket = atomicAdd(&ctl->chunk_ticket, 1ull);
    __syncthreads();
    const u64 t = s_ticket;
    __syncthreads();  // every thread has its ticket before thread 0 may take the next
    if (t >= nch) break;
    const Chunk ch = j.chunks[t];
    const u32 sz = ch.size;
    if (sz > m || ch.begin > j.n || ch.begin + sz > j.n) {  // never produced; reported, not touched
      if (tid == 0) atomicOr(&ctl->err, kErrInternal);
      continue;
    }
    const u64* src = j.buf[(ch.flags & kChSrcTmp) ? 1 : 0] + ch.begin * RW;
    u64* dst = j.buf[0] + ch.begin * RW;
    load_words_async(stage, src, (u64)sz * RW);
    cp_async_wait_all();
    __syncthreads();
    u32 p = 0;
    if (!(ch.flags & kChCopyOnly)) p = range_top_bit(c, 0, sz, false);
    if (p == 0) {  // already in order
      if (src != dst) store_words(dst, stage, (u64)sz * RW);
      __syncthreads();
      continue;
    }
    for (u32 i = tid; i < sz; i += kThreads) c.permA[i] = (u16)i;
    if (tid == 0) s_top = 0;
    __syncthreads();
    sort_round(c, 0, sz, p, &s_top);
    for (;;) {
      __syncthreads();
      const u32 top = s_top;
      if (top == 0) break;
      if (top > c.stack_cap) {  // cannot happen: runs on the stack are disjoint and > kEsMax
        if (tid == 0) atomicOr(&ctl->err, kErrInternal);
        break;
      }
      const u32 a = c.stack[2 * (top - 1)], s = c.stack[2 * (top - 1) + 1];
      __syncthreads();
      if (tid == 0) s_top = top - 1;
      __syncthreads();
      const u32 pp = range_top_bit(c, a, s, true);
      if (pp) sort_round(c, a, s, pp, &s_top);
    }
    // write the records in sorted order
    if (RW == 2) {
      for (u32 s = tid; s < sz; s += kThreads) {
        const u32 r = c.permA[s];
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(stage + 2 * (u64)r);
        __stcs(reinterpret_cast<ulonglong2*>(dst + 2 * (u64)s), v);
      }
    } else if (RWT != 0) {
      for (u32 q = tid; q < sz * RW; q += kThreads) {
        const u32 s = q / RW, w = q - s * RW;
        __stcs(dst + q, stage[(u64)c.permA[s] * RW + w]);
      }
    } else {
      for (u32 s = tid; s < sz; s += kThreads) {
        const u64* sp = stage + (u64)c.permA[s] * RW;
        for (u32 w = 0; w < RW; w++) __stcs(dst + (u64)s * RW + w, sp[w]);
      }
    }
    __syncthreads();
  }
}

// Finished ranges that live in tmp: copy to in.
__global__ void __launch_bounds__(kThreads) k_copy(Job j) {
  Ctl* ctl = j.ctl;
  const u64 np = ctl->npieces;
  __shared__ u64 s_ticket;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(&ctl->piece_ticket, 1ull);
    __syncthreads();
    const u64 t = s_ticket;
    __syncthreads();
    if (t >= np) break;
    const Piece pc = j.pieces[t];
    if (pc.begin > j.n || pc.size > j.n - pc.begin) {
      if (threadIdx.x == 0) atomicOr(&ctl->err, kErrInternal);
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
    cudaFuncSetAttribute(k_chunk<KW, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)sm);                                                   \
    k_chunk<KW, R><<<grid, kThreads, sm, s>>>(j);                                   \
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
  cudaError_t e;
  if (j.KW == 1) {
    cudaFuncSetAttribute(k_chunk<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chunk<1, 0>, kThreads, sm);
  } else {
    cudaFuncSetAttribute(k_chunk<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chunk<2, 0>, kThreads, sm);
  }
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

int launch_chunks(const Job& j, u32 grid, cudaStream_t s) {
  cudaError_t e = j.KW == 1 ? launch_chunks_kw<1>(j, grid, s) : launch_chunks_kw<2>(j, grid, s);
  return e == cudaSuccess ? 1 : -1;
}

int launch_copy(const Job& j, u32 grid, cudaStream_t s) {
  k_copy<<<grid, kThreads, 0, s>>>(j);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// chunk_max for a record size: the largest range whose staging and index arrays fit the
// shared memory of two CTAs per SM.
u32 chunk_capacity(u32 RW) {
  const size_t budget = kChunkSmem - kChunkFixed;
  u32 m = (u32)(budget / (RW * 8 + 6));   // the record + three u16 index arrays
  m &= ~63u;
  if (m > (u32)kThreads * kChunkItems) m = kThreads * kChunkItems;
  return m;
}

}  // namespace rsg
