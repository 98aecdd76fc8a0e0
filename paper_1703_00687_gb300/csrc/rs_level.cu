// Distribution passes of the MSD radix sort (Kokot et al., section 3.1, steps 1-2): for
// every large bin of a level, a histogram of its digit, the exclusive prefix sum of the
// histogram (bucket bases), and a stable scatter of its records into the other buffer.
// Then every sub-bin is classified: finished, sorted on chip (chunk), or large again.
//
// Kernels, all launched on the caller's stream:
//   k_hist      histogram of each bin's digit, plus the AND/OR of the bin's keys.  The last
//               CTA to count a bin checks that the digit starts at the bin's highest
//               differing key bit (digits shared by every key are skipped, the paper's
//               remark in section 1 that bins of equal keys do not shrink), flags a recount
//               if not, marks a bin of equal keys finished, and turns counts into bases.
//   k_scatter   tile-wise stable scatter with a decoupled look-back across the tiles of a bin.
//   k_classify  sub-bin classification, chunk packing, the next level's bin list.
#include "rs_internal.cuh"

namespace rsg {

// Exclusive scan of one u64 per thread (kThreads threads); returns the exclusive prefix and
// the total in *total.
__device__ inline u64 block_scan_value64(u64 x, u64* scratch, u64* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 s = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(kFull, s, o);
    if (lane >= o) s += y;
  }
  if (lane == 31) scratch[warp] = s;
  __syncthreads();
  if (warp == 0) {
    u64 w = lane < kWarps ? scratch[lane] : 0, t = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) scratch[lane] = t - w;
    if (lane == kWarps - 1) scratch[kWarps] = t;
  }
  __syncthreads();
  u64 r = scratch[warp] + s - x;
  *total = scratch[kWarps];
  __syncthreads();
  return r;
}

// Tile numbering of bin list L: tile_start = exclusive prefix of ceil(size / T) in list order.
// One CTA of kThreads threads.
__device__ void finalize_list(const Job& j, int L) {
  __shared__ u64 scr[kWarps + 1];
  Ctl* ctl = j.ctl;
  u64 nb = *(volatile u64*)&ctl->nbins[L];
  if (nb > j.cap_bins) nb = j.cap_bins;
  Bin* bins = j.bins[L];
  u64 carry = 0;
  for (u64 base = 0; base < nb; base += kThreads) {
    const u64 i = base + threadIdx.x;
    const u64 t = i < nb ? ceil_div(bins[i].size, j.T) : 0;
    u64 tot;
    const u64 ex = block_scan_value64(t, scr, &tot);
    if (i < nb) bins[i].tile_start = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    ctl->ntiles[L] = carry;
    if (*(volatile u64*)&ctl->nbins[L] > j.cap_bins) ctl->nbins[L] = j.cap_bins;
  }
}

// ------------------------------------------------------------------------ init
__global__ void __launch_bounds__(kThreads) k_init_plain(Job j, u32 lo, u32 W) {
  Ctl* ctl = j.ctl;
  const u32 nd = 1u << W;
  if (threadIdx.x == 0) {
    const u64 tiles = ceil_div(j.n, j.T);
    Ctl c = {};
    c.err = ctl->err;
    c.nbins[0] = 1;
    c.ntiles[0] = tiles;
    c.base_used[0] = nd;
    c.status_used[0] = tiles * nd;
    *ctl = c;
    Bin b = {};
    b.begin = 0;
    b.size = j.n;
    b.kand[0] = b.kand[1] = ~0ull;
    b.lo = lo;
    b.W = W;
    j.bins[0][0] = b;
  }
  for (u32 v = threadIdx.x; v < nd; v += kThreads) j.base[0][v] = 0;
}

__global__ void k_init_single_chunk(Job j) {
  if (threadIdx.x == 0) {
    Ctl c = {};
    c.err = j.ctl->err;
    c.nchunks = 1;
    *j.ctl = c;
    Chunk ch = {};
    ch.begin = 0;
    ch.size = (u32)j.n;
    j.chunks[0] = ch;
  }
}

__global__ void k_reset(Job j) {
  if (threadIdx.x == 0) {
    Ctl c = {};
    c.err = j.ctl->err;
    *j.ctl = c;
  }
}

// Segmented (batched) start: every segment is a level-0 bin (if large) or a chunk.
__global__ void __launch_bounds__(kThreads) k_init_segments(Job j) {
  Ctl* ctl = j.ctl;
  for (u64 s = blockIdx.x * (u64)kThreads + threadIdx.x; s < j.n_segs; s += (u64)gridDim.x * kThreads) {
    const u64 a = j.seg_off[s], e = j.seg_off[s + 1];
    if (e < a || e > j.n) {  // offsets not non-decreasing within [0, total]: skip, report
      atomicOr(&ctl->err, kErrInternal);
      continue;
    }
    if (e <= a + 1) continue;
    const u64 c = e - a;
    if (c <= j.chunk_max) {
      const u64 idx = atomicAdd(&ctl->nchunks, 1ull);
      if (idx >= j.cap_chunks) { atomicOr(&ctl->err, kErrOverflow); continue; }
      Chunk ch = {};
      ch.begin = a;
      ch.size = (u32)c;
      j.chunks[idx] = ch;
      continue;
    }
    u32 lo, W;
    plan_digit(c, 8 * j.K, j.chunk_max, j.wmax, &lo, &W);
    const u32 nd = 1u << W;
    const u64 tiles = ceil_div(c, j.T);
    const u64 idx = atomicAdd(&ctl->nbins[0], 1ull);
    const u64 bo = atomicAdd(&ctl->base_used[0], (u64)nd);
    const u64 so = atomicAdd(&ctl->status_used[0], tiles * nd);
    if (idx >= j.cap_bins || bo + nd > j.cap_base || so + tiles * nd > j.cap_status) {
      atomicOr(&ctl->err, kErrOverflow);
      continue;
    }
    Bin b = {};
    b.begin = a;
    b.size = c;
    b.base_off = bo;
    b.status_off = so;
    b.kand[0] = b.kand[1] = ~0ull;
    b.lo = lo;
    b.W = W;
    j.bins[0][idx] = b;
    for (u32 v = 0; v < nd; v++) j.base[0][bo + v] = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_finalize0(Job j) { finalize_list(j, 0); }

// ------------------------------------------------------------------- histogram
constexpr int kHistCopies = 2;  // privatised histogram copies (by warp parity)

// mode 0: count + key AND/OR, then check the digit; mode 1: recount bins flagged kBinRedo;
// mode 2: counts only (histogram entry point); mode 3: count + bases (given digit).
//
// The last CTA to count a bin finishes it: in mode 0, if every key is equal the bin is
// finished as it is; if the digit does not start at the bin's highest differing bit, it is
// moved there (never widened: the bin's pools were sized for W) and a recount is requested.
// Otherwise the counts become exclusive bucket bases.
template <int KW>
__device__ void finish_bin(const Job& j, int L, u64 b, int mode) {
  __shared__ u64 scr[kWarps + 1];
  __shared__ int s_ret;
  Ctl* ctl = j.ctl;
  Bin* bp = &j.bins[L][b];
  const u32 W = bp->W;
  const u32 nd = 1u << W;
  const u64 size = bp->size;
  u64* base = j.base[L] + bp->base_off;
  if (threadIdx.x == 0) {
    s_ret = 0;
    if (mode == 0) {
      const u64 v0 = (__ldcg(&bp->kand[0]) ^ __ldcg(&bp->kor[0])) & j.keymask[0];
      const u64 v1 = KW == 2 ? (__ldcg(&bp->kand[1]) ^ __ldcg(&bp->kor[1])) & j.keymask[1] : 0;
      const u32 p = top_bit_plus1(v0, v1);
      if (p == 0) {
        bp->flags |= kBinEqual;
        s_ret = 1;
      } else if (bp->lo + W != p) {
        u32 nlo, nW;
        plan_digit(size, p, j.chunk_max, j.wmax, &nlo, &nW);
        if (nW > W) {
          nW = W;
          nlo = p - W;
        }
        bp->lo = nlo;
        bp->W = nW;
        bp->flags |= kBinRedo;
        bp->done = 0;
        atomicAdd(&ctl->nredo, 1u);
        s_ret = 2;
      }
    }
  }
  __syncthreads();
  if (s_ret) {
    if (s_ret == 2)
      for (u32 v = threadIdx.x; v < nd; v += kThreads) base[v] = 0;
    return;
  }
  if (mode == 2) return;
  // nd <= 1024: two entries per thread
  const u32 v0 = 2 * threadIdx.x;
  const u64 c0 = v0 < nd ? __ldcg(base + v0) : 0;
  const u64 c1 = v0 + 1 < nd ? __ldcg(base + v0 + 1) : 0;
  u64 tot;
  const u64 ex = block_scan_value64(c0 + c1, scr, &tot);
  if (v0 < nd) base[v0] = ex;
  if (v0 + 1 < nd) base[v0 + 1] = ex + c0;
  if (mode == 1 && threadIdx.x == 0) bp->flags &= ~kBinRedo;
}

// Shared memory of k_hist: two buffers of a tile's keys (tile t+1 streams in while tile t
// is counted).
__host__ __device__ inline size_t hist_smem_bytes_for(u32 T, u32 KW) { return 2ull * T * KW * 8; }


template <int KW>
__global__ void __launch_bounds__(kThreads, 2) k_hist(Job j, int level, int mode) {
  const int L = level & 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0) return;
  if (mode == 1 && ctl->nredo == 0) return;
  const u64 ntiles = ctl->ntiles[L];
  Bin* bins = j.bins[L];
  extern __shared__ __align__(16) unsigned char smem[];
  u64* kbuf = (u64*)smem;  // [2][T][KW]
  __shared__ u32 hist[kHistCopies << kWMax];
  __shared__ u64 red[kWarps][4];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool want_masks = mode == 0;
  const u32 T = j.T;
  const u64 per = ceil_div(ntiles, gridDim.x);
  const u64 t0 = blockIdx.x * per;
  const u64 t1 = min(ntiles, t0 + per);
  if (t0 >= t1) return;
  for (u32 v = tid; v < (kHistCopies << kWMax); v += kThreads) hist[v] = 0;
  u32* my_hist = hist + ((warp & (kHistCopies - 1)) << kWMax);
  u32 counted = 0;
  u64 kand[2] = {~0ull, ~0ull}, kor[2] = {0ull, 0ull};
  __syncthreads();

  auto flush = [&](u64 b) {
    __syncthreads();
    const Bin* bb = &bins[b];
    const u32 nd = 1u << bb->W;
    const u64 bo = bb->base_off;
    for (u32 v = tid; v < nd; v += kThreads) {
      u32 h = 0;
#pragma unroll
      for (int c = 0; c < kHistCopies; c++) {
        h += hist[(c << kWMax) + v];
        hist[(c << kWMax) + v] = 0;
      }
      if (h) atomicAdd(&j.base[L][bo + v], (u64)h);
    }
    if (want_masks) {
#pragma unroll
      for (int k = 0; k < KW; k++) {
        u64 a = kand[k], o = kor[k];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
          a &= __shfl_xor_sync(kFull, a, s);
          o |= __shfl_xor_sync(kFull, o, s);
        }
        if (lane == 0) {
          red[warp][k] = a;
          red[warp][2 + k] = o;
        }
        kand[k] = ~0ull;
        kor[k] = 0;
      }
      __syncthreads();
      if (tid < KW) {
        u64 a = ~0ull, o = 0;
        for (int w = 0; w < kWarps; w++) {
          a &= red[w][tid];
          o |= red[w][2 + tid];
        }
        atomicAnd(&bins[b].kand[tid], a);
        atomicOr(&bins[b].kor[tid], o);
      }
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const u32 old = atomicAdd(&bins[b].done, counted);
      s_last = (u64)(old + counted) == ceil_div(bins[b].size, (u64)T);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finish_bin<KW>(j, L, b, mode);
    }
    __syncthreads();
    counted = 0;
  };

  struct TileRef {
    u64 b;
    u32 cnt, lo, W, skip;
  };
  u64 walk = find_bin(bins, nb, t0);
  // locate tile t, clear its look-back words, and start copying its keys into buffer `buf`
  auto issue = [&](u64 t, int buf) {
    while (walk + 1 < nb && bins[walk + 1].tile_start <= t) walk++;
    const Bin* bp = &bins[walk];
    TileRef tr;
    tr.b = walk;
    tr.skip = (mode == 1 && !(bp->flags & kBinRedo)) ? 1u : 0u;
    tr.lo = bp->lo;
    tr.W = bp->W;
    const u64 tib = t - bp->tile_start;
    const u64 r0 = tib * T;
    tr.cnt = (u32)min((u64)T, bp->size - r0);
    if ((mode == 0 || mode == 3) && tid == 0 && t < j.cap_tiles) j.tile_bin[t] = (u32)walk;
    if (mode == 0 || mode == 3) {  // the scatter pass's look-back words of this tile start cleared
      const u32 nd = 1u << tr.W;
      const u64 so = bp->status_off + tib * nd;
      if (j.wide) {
        u64* st = (u64*)j.status[L] + so;
        for (u32 v = tid; v < nd; v += kThreads) st[v] = 0;
      } else {
        u32* st = (u32*)j.status[L] + so;
        for (u32 v = tid; v < nd; v += kThreads) st[v] = 0;
      }
    }
    if (!tr.skip) {
      const u64* src = j.buf[bp->parity] + (bp->begin + r0) * j.RW;
      u64* dst = kbuf + (size_t)buf * T * KW;
      for (u32 r = tid; r < tr.cnt; r += kThreads) {
        if (KW == 2 && ((((uintptr_t)(src + (u64)r * j.RW)) & 15) == 0)) {
          cp_async16(dst + 2 * r, src + (u64)r * j.RW);
        } else {
#pragma unroll
          for (int q = 0; q < KW; q++) cp_async8(dst + KW * r + q, src + (u64)r * j.RW + q);
        }
      }
    }
    cp_async_commit();
    return tr;
  };

  TileRef tn = issue(t0, 0);
  u64 cur = tn.b;
  for (u64 t = t0; t < t1; t++) {
    const TileRef tc = tn;
    const int buf = (int)((t - t0) & 1);
    if (t + 1 < t1) tn = issue(t + 1, buf ^ 1);
    else cp_async_commit();  // keep one group per iteration
    cp_async_wait_one();     // tile t's keys have landed
    __syncthreads();
    if (tc.b != cur) {
      if (counted) flush(cur);
      cur = tc.b;
    }
    if (!tc.skip) {
      const u64* kb = kbuf + (size_t)buf * T * KW;
      for (u32 r = tid; r < tc.cnt; r += kThreads) {
        Key<KW> k;
#pragma unroll
        for (int q = 0; q < KW; q++) k.w[q] = kb[KW * r + q] & j.keymask[q];
        atomicAdd(&my_hist[digit_of<KW>(k, tc.lo, tc.W)], 1u);
        if (want_masks) {
#pragma unroll
          for (int q = 0; q < KW; q++) {
            kand[q] &= k.w[q];
            kor[q] |= k.w[q];
          }
        }
      }
      counted++;
    }
    __syncthreads();  // buffer `buf` is refilled by the next issue
  }
  if (counted) flush(cur);
}

// --------------------------------------------------------------------- scatter
constexpr int kSThreads = 256;  // threads of a scatter CTA
constexpr int kSWarps = kSThreads / 32;

// Shared memory of k_scatter: T records, per-warp 16-bit digit counters (row stride 2^wmax),
// the tile's permutation, per-digit counts / run bases / global bases.
struct ScatterLayout {
  size_t stage, whist, perm, sdig, tcount, tbase, gbase, total;
};

__host__ __device__ inline ScatterLayout scatter_layout(u32 T, u32 RW, u32 wmax) {
  ScatterLayout s;
  const size_t nd = (size_t)1 << wmax;
  size_t o = 0;
  s.stage = o; o += (size_t)T * RW * 8;
  s.whist = o; o += (size_t)kSWarps * nd * 2;
  s.perm = o; o += (size_t)T * 2;
  s.sdig = o; o += (size_t)T * 2;
  o = (o + 15) & ~(size_t)15;
  s.tcount = o; o += nd * 4;
  s.tbase = o; o += nd * 4;
  s.gbase = o; o += nd * 8;
  s.total = (o + 127) & ~(size_t)127;
  return s;
}

// Look-back word: 2-bit state (0 none, 1 tile count, 2 inclusive prefix) above the value.
template <typename S>
struct LB;
template <>
struct LB<u32> {
  static constexpr int kShift = 30;
  static constexpr u32 kVal = (1u << 30) - 1;
};
template <>
struct LB<u64> {
  static constexpr int kShift = 62;
  static constexpr u64 kVal = (1ull << 62) - 1;
};

// Publishes this tile's count of one digit and returns the number of records with that digit
// in the bin's earlier tiles (decoupled look-back).  A look-back word carries its state and its
// count together, so plain relaxed accesses suffice (no fences).  The words of up to
// LookAhead<S>::n earlier tiles are read together, one round trip per group.  Every wait is bounded.
template <typename S>
struct LookAhead {  // predecessors read per round trip (fewer for the rare 64-bit words: registers)
  static constexpr int n = sizeof(S) == 4 ? 8 : 3;
};

template <typename S>
__device__ __forceinline__ void lb_publish(S* st, u64 self, u64 tib, u32 c) {
  st_relaxed(st + self, (S)(((S)(tib == 0 ? 2 : 1) << LB<S>::kShift) | (S)c));
}

template <typename S>
__device__ __forceinline__ S lb_word(const S* st, u64 at, bool stall, Ctl* ctl) {
  return stall ? (S)ld_relaxed(&ctl->never) : ld_relaxed(st + at);
}

// Reads the words of the LookAhead<S>::n tiles before this one (one round trip).
template <typename S>
__device__ __forceinline__ void lb_first(const S* st, u64 self, u32 nd, u64 tib, bool stall, Ctl* ctl, S (&w)[LookAhead<S>::n]) {
#pragma unroll
  for (int q = 0; q < LookAhead<S>::n; q++)
    if ((u64)q < tib) w[q] = lb_word(st, self - (u64)(q + 1) * nd, stall && q == 0, ctl);
}

// Walks back from the words lb_first read, waiting (bounded) for tiles not yet published and
// reading further groups while only aggregates are found; then publishes the inclusive prefix.
template <typename S>
__device__ __forceinline__ u64 lb_collect(S* st, u64 self, u32 nd, u64 tib, u32 c, const Job& j, bool stall, S (&w)[LookAhead<S>::n]) {
  Ctl* ctl = j.ctl;
  if (tib == 0) return 0;
  u64 excl = 0;
  u64 back = 1;  // distance of w[0]
  bool done = false;
  for (;;) {
    const u64 n = min((u64)LookAhead<S>::n, tib - back + 1);
#pragma unroll
    for (int q = 0; q < LookAhead<S>::n && !done; q++) {
      if ((u64)q >= n) break;
      u32 polls = 0;
      while ((w[q] >> LB<S>::kShift) == 0) {  // a tile not yet published
        if (++polls > j.watchdog || ((polls & 255) == 0 && (*(volatile u32*)&ctl->err & kErrTimeout))) {
          atomicOr(&ctl->err, kErrTimeout);
          break;
        }
        __nanosleep(100);
        w[q] = lb_word(st, self - (back + q) * nd, stall && back + q == 1, ctl);
      }
      excl += (u64)(w[q] & LB<S>::kVal);
      if ((w[q] >> LB<S>::kShift) != 1) done = true;  // inclusive prefix (or gave up)
    }
    back += n;
    if (done || back > tib) break;
#pragma unroll
    for (int q = 0; q < LookAhead<S>::n; q++)
      if ((u64)q < tib - back + 1) w[q] = ld_relaxed(st + self - (back + q) * nd);
  }
  st_relaxed(st + self, (S)(((S)2 << LB<S>::kShift) | (S)(excl + c)));
  return excl;
}

// Lanes of the warp whose digit equals this lane's (d has W significant bits): one vote per
// digit bit.  Lanes with valid == false get a mask of their own.
__device__ __forceinline__ u32 peers_of(u32 d, u32 W, bool valid) {
  u32 peers = __ballot_sync(kFull, valid);
  for (u32 b = 0; b < W; b++) {
    const bool bit = (d >> b) & 1u;
    const u32 v = __ballot_sync(kFull, bit);
    peers &= bit ? v : ~v;
  }
  return valid ? peers : (1u << (threadIdx.x & 31));
}

// Digit of a staged record.  No key mask is needed: a digit window never reaches past the key.
template <int KW>
__device__ __forceinline__ u32 staged_digit(const u64* rec, u32 lo, u32 W) {
  Key<KW> k;
  k.w[0] = rec[0];
  if (KW == 2) k.w[KW - 1] = rec[1];
  return digit_of<KW>(k, lo, W);
}

constexpr u64 kSkip = ~0ull;  // gbase of a digit whose run would leave its bin

// Turns the tile's digit counts into destinations: the exclusive scan over digits (tbase) and,
// per digit, the records of that digit in the bin's earlier tiles (decoupled look-back).  The
// first look-back words of all of a thread's digits are read together (one round trip).  A
// digit run that would leave the bin (possible only after a failed wait or a corrupted
// histogram) gets kSkip and is not written.
template <typename S, u32 Q>
__device__ __forceinline__ void tile_offsets(S* st, u64 status_off, u64 tib, u32 nd, const u32* tcount, u32* tbase,
                                             u32* scan_scr, const u64 (&mybase)[Q], u64 begin, u64 size, const Job& j,
                                             u64* gbase) {
  const u32 tid = threadIdx.x;
  block_exclusive_scan<kSThreads>(tbase, nd, scan_scr);
  S w[Q][LookAhead<S>::n];
#pragma unroll
  for (u32 q = 0; q < Q; q++) {
    const u32 v = tid + q * kSThreads;
    if (v < nd) lb_first<S>(st, status_off + tib * nd + v, nd, tib, j.inject && v == 0 && tib == 1, j.ctl, w[q]);
  }
#pragma unroll
  for (u32 q = 0; q < Q; q++) {
    const u32 v = tid + q * kSThreads;
    if (v >= nd) break;
    const u32 c = tcount[v];
    const u64 excl = lb_collect<S>(st, status_off + tib * nd + v, nd, tib, c, j, j.inject && v == 0 && tib == 1, w[q]);
    const u64 first = mybase[q] + excl;  // the run's first record, relative to the bin
    u64 g = begin + first - tbase[v];
    if (c && (first > size || c > size - first)) {
      atomicOr(&j.ctl->err, kErrInternal);
      g = kSkip;
    }
    gbase[v] = g;
  }
}

// IT = records per thread (T = kSThreads * IT).  Tiles are taken one at a time from a ticket
// dispenser, in order, so that every tile a look-back waits for is already held by a running
// CTA that will publish its counts without waiting for anything later.
template <int KW, int RWT, int IT>
__global__ void __launch_bounds__(kSThreads) k_scatter(Job j, int level) {
  const int L = level & 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0) return;
  const u64 ntiles = ctl->ntiles[L];
  const Bin* bins = j.bins[L];
  const u32 RW = RWT ? (u32)RWT : j.RW;
  constexpr u32 T = kSThreads * IT;
  constexpr u32 PW = T / kSWarps;  // records per warp strip
  constexpr u32 kDigitsPerThread = (1u << kWMax) / kSThreads;
  const u32 WS = 1u << j.wmax;     // row stride of the per-warp counters
  const ScatterLayout lay = scatter_layout(T, RW, j.wmax);
  extern __shared__ __align__(16) unsigned char smem[];
  u64* stage = (u64*)(smem + lay.stage);
  u16* whist = (u16*)(smem + lay.whist);
  u16* perm = (u16*)(smem + lay.perm);
  u16* sdig = (u16*)(smem + lay.sdig);
  u32* tcount = (u32*)(smem + lay.tcount);
  u32* tbase = (u32*)(smem + lay.tbase);
  u64* gbase = (u64*)(smem + lay.gbase);
  __shared__ u64 s_ticket;
  __shared__ u32 s_bin;
  __shared__ u32 scan_scr[kSWarps + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 ltmask = lanemask_lt();
  // per-warp digit counters: counts while ranking, then each warp's offset inside the digit's
  // run; they are zeroed again while the tile is written out
  for (u32 i = tid; i < kSWarps * WS; i += kSThreads) whist[i] = 0;
  u16* wh = whist + warp * WS;
  for (;;) {
    if (tid == 0) {
      const u64 tk = atomicAdd(&ctl->s_ticket, 1ull);
      s_ticket = tk;
      s_bin = tk < ntiles && tk < j.cap_tiles ? j.tile_bin[tk] : 0;
    }
    __syncthreads();
    const u64 t = s_ticket;
    const u32 b = s_bin;
    __syncthreads();  // every thread has its ticket before thread 0 may take the next
    if (t >= ntiles) break;
    const Bin* bp = &bins[b < nb ? b : 0];
    const u32 lo = bp->lo, W = bp->W, nd = 1u << W;
    const u64 begin = bp->begin, size = bp->size;
    const u64 tib = t - bp->tile_start;
    const u64 status_off = bp->status_off;
    const u32 parity = bp->parity;
    if ((bp->flags & kBinEqual) || tib * T >= size) continue;  // finished bin (or inconsistent map)
    const u64 r0 = tib * T;
    const u32 cnt = (u32)min((u64)T, size - r0);
    u64* dstb = j.buf[parity ^ 1];
    const u64* bbase = j.base[L] + bp->base_off;

    load_words_async<kSThreads>(stage, j.buf[parity] + (begin + r0) * RW, (u64)cnt * RW);
    u64 mybase[kDigitsPerThread];  // this thread's digits' bucket bases, fetched during the load
#pragma unroll
    for (u32 q = 0; q < kDigitsPerThread; q++) {
      const u32 v = tid + q * kSThreads;
      mybase[q] = v < nd ? bbase[v] : 0;
    }
    cp_async_wait_all();
    __syncthreads();

    // stable rank: warp w owns records [w*PW, (w+1)*PW), visited in order
    u32 packed[IT];
    if (cnt == T) {
      // first every item's digit and peers (independent of each other), then the counters
      u32 dg[IT], pr[IT];
#pragma unroll
      for (int it = 0; it < IT; it++) {
        dg[it] = staged_digit<KW>(stage + (u64)(warp * PW + it * 32 + lane) * RW, lo, W);
        pr[it] = peers_of(dg[it], W, true);
      }
#pragma unroll
      for (int it = 0; it < IT; it++) {
        const u32 d = dg[it], peers = pr[it];
        const u32 before = __popc(peers & ltmask);
        const u32 old = wh[d];
        __syncwarp();
        if (before == 0) wh[d] = (u16)(old + __popc(peers));
        __syncwarp();
        packed[it] = (old + before) | (d << 16);
      }
    } else {
#pragma unroll
      for (int it = 0; it < IT; it++) {
        const u32 r = warp * PW + it * 32 + lane;
        const bool valid = r < cnt;
        u32 d = 0;
        if (valid) d = staged_digit<KW>(stage + (u64)r * RW, lo, W);
        const u32 peers = peers_of(d, W, valid);
        const u32 before = __popc(peers & ltmask);
        u32 old = 0;
        if (valid) old = wh[d];
        __syncwarp();
        if (valid && before == 0) wh[d] = (u16)(old + __popc(peers));
        __syncwarp();
        packed[it] = valid ? ((old + before) | (d << 16)) : 0xffffffffu;
      }
    }
    __syncthreads();
    for (u32 v = tid; v < nd; v += kSThreads) {
      u32 run = 0;
#pragma unroll
      for (int w = 0; w < kSWarps; w++) {
        const u32 x = whist[w * WS + v];
        whist[w * WS + v] = (u16)run;
        run += x;
      }
      tcount[v] = run;
      tbase[v] = run;
      // publish this tile's count at once: later tiles of the bin may be waiting for it
      if (j.wide) lb_publish<u64>((u64*)j.status[L], status_off + tib * nd + v, tib, run);
      else lb_publish<u32>((u32*)j.status[L], status_off + tib * nd + v, tib, run);
    }
    __syncthreads();
    if (j.wide) tile_offsets<u64, kDigitsPerThread>((u64*)j.status[L], status_off, tib, nd, tcount, tbase, scan_scr, mybase, begin, size, j, gbase);
    else tile_offsets<u32, kDigitsPerThread>((u32*)j.status[L], status_off, tib, nd, tcount, tbase, scan_scr, mybase, begin, size, j, gbase);
    if (cnt == T) {
#pragma unroll
      for (int it = 0; it < IT; it++) {
        const u32 d = packed[it] >> 16;
        const u32 slot = tbase[d] + wh[d] + (packed[it] & 0xffffu);
        perm[slot] = (u16)(warp * PW + it * 32 + lane);
        sdig[slot] = (u16)d;
      }
    } else {
#pragma unroll
      for (int it = 0; it < IT; it++) {
        if (packed[it] != 0xffffffffu) {
          const u32 d = packed[it] >> 16;
          const u32 slot = tbase[d] + wh[d] + (packed[it] & 0xffffu);
          perm[slot] = (u16)(warp * PW + it * 32 + lane);
          sdig[slot] = (u16)d;
        }
      }
    }
    __syncthreads();
    // per-warp counters back to zero for the next tile (nothing reads them before then)
    for (u32 v = tid; v < nd; v += kSThreads) {
#pragma unroll
      for (int w = 0; w < kSWarps; w++) whist[w * WS + v] = 0;
    }
    // write the tile in digit order: consecutive slots of one digit go to consecutive records
    if (RW == 2) {
      for (u32 s = tid; s < cnt; s += kSThreads) {
        const u64 g = gbase[sdig[s]];
        if (g == kSkip) continue;
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(stage + 2 * (u32)perm[s]);
        __stcs(reinterpret_cast<ulonglong2*>(dstb + 2 * (g + s)), v);
      }
    } else {
      for (u32 s = tid; s < cnt; s += kSThreads) {
        const u64 g = gbase[sdig[s]];
        if (g == kSkip) continue;
        const u64* sp = stage + (u64)perm[s] * RW;
        u64* d = dstb + (g + s) * RW;
        for (u32 w = 0; w < RW; w++) __stcs(d + w, sp[w]);
      }
    }
    __syncthreads();
  }
}

// -------------------------------------------------------------------- classify
// Highest differing key bit + 1 over 32 records spread over a sub-bin (the sample tells where
// the sub-bin's next digit probably starts; the next histogram pass checks, and moves it).
template <int KW>
__device__ u32 sample_top_bit(const Job& j, const u64* rec, u64 c) {
  u64 a[2] = {~0ull, ~0ull}, o[2] = {0, 0};
  const int ns = 32;
  for (int i = 0; i < ns; i++) {
    const u64 r = (c * (u64)i) / ns;
    const Key<KW> k = load_key<KW>(rec + r * j.RW, j);
#pragma unroll
    for (int q = 0; q < KW; q++) {
      a[q] &= k.w[q];
      o[q] |= k.w[q];
    }
  }
  return top_bit_plus1(a[0] ^ o[0], KW == 2 ? a[1] ^ o[1] : 0);
}

__device__ void push_pieces(const Job& j, u64 begin, u64 c) {
  Ctl* ctl = j.ctl;
  const u64 np = ceil_div(c, kPieceRecords);
  const u64 idx = atomicAdd(&ctl->npieces, np);
  if (idx + np > j.cap_pieces) {
    atomicOr(&ctl->err, kErrOverflow);
    return;
  }
  for (u64 q = 0; q < np; q++) {
    Piece pc;
    pc.begin = begin + q * kPieceRecords;
    pc.size = min(kPieceRecords, c - q * kPieceRecords);
    j.pieces[idx + q] = pc;
  }
}

template <int KW>
__global__ void __launch_bounds__(kThreads) k_classify(Job j, int level) {
  const int L = level & 1, N = L ^ 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0) return;
  const Bin* bins = j.bins[L];
  __shared__ u8 cls[1 << kWMax];
  __shared__ u32 cnt[1 << kWMax];
  __shared__ u64 boff[1 << kWMax];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  for (u64 b = blockIdx.x; b < nb; b += gridDim.x) {
    const Bin bin = bins[b];
    if (bin.flags & kBinEqual) {  // finished without moving; copy back if it lives in tmp
      if (tid == 0 && bin.parity) push_pieces(j, bin.begin, bin.size);
      continue;
    }
    const u32 nd = 1u << bin.W;
    const u32 p1 = bin.parity ^ 1;
    const u64* bbase = j.base[L] + bin.base_off;
    for (u32 v = tid; v < nd; v += kThreads) {
      u64 bv = bbase[v];
      u64 next = v + 1 < nd ? bbase[v + 1] : bin.size;
      if (next < bv || next > bin.size) {  // inconsistent bases (only after a reported error)
        atomicOr(&ctl->err, kErrInternal);
        next = bv = min(bv, bin.size);
      }
      const u64 c = next - bv;
      boff[v] = bv;
      cnt[v] = (u32)min(c, (u64)j.chunk_max + 1);
      u8 k;
      if (c == 0) {
        k = 0;
      } else if (c == 1) {
        k = 1;
      } else if (c <= j.chunk_max) {
        k = 2;
      } else {
        k = 3;
        const u64 rb = bin.begin + bv;
        // every key bit >= bin.lo is shared by the sub-bin; guess where its next digit
        // starts from a sample
        u32 p = sample_top_bit<KW>(j, j.buf[p1] + rb * j.RW, c);
        if (p == 0 || p > bin.lo) p = bin.lo;
        if (p == 0) p = 1;
        u32 nlo, nW;
        plan_digit(c, p, j.chunk_max, j.wmax, &nlo, &nW);
        const u32 nnd = 1u << nW;
        const u64 tiles = ceil_div(c, j.T);
        const u64 idx = atomicAdd(&ctl->nbins[N], 1ull);
        const u64 bo = atomicAdd(&ctl->base_used[N], (u64)nnd);
        const u64 so = atomicAdd(&ctl->status_used[N], tiles * nnd);
        if (idx >= j.cap_bins || bo + nnd > j.cap_base || so + tiles * nnd > j.cap_status) {
          atomicOr(&ctl->err, kErrOverflow);
        } else {
          Bin nbn = {};
          nbn.begin = rb;
          nbn.size = c;
          nbn.base_off = bo;
          nbn.status_off = so;
          nbn.kand[0] = nbn.kand[1] = ~0ull;
          nbn.lo = nlo;
          nbn.W = nW;
          nbn.parity = p1;
          j.bins[N][idx] = nbn;
          for (u32 q = 0; q < nnd; q++) j.base[N][bo + q] = 0;
        }
      }
      cls[v] = k;
    }
    __syncthreads();
    if (tid == 0) {
      // greedy packing of consecutive small sub-bins into on-chip chunks
      u64 cb = 0;
      u32 csz = 0, nsub = 0, vfirst = 0, vlast = 0;
      bool open = false, uns = false;
      auto emit = [&]() {
        if (open && (uns || p1)) {
          const u64 idx = atomicAdd(&ctl->nchunks, 1ull);
          if (idx >= j.cap_chunks) {
            atomicOr(&ctl->err, kErrOverflow);
          } else {
            Chunk ch = {};
            ch.begin = bin.begin + cb;
            ch.size = csz;
            ch.flags = (p1 ? kChSrcTmp : 0u) | (uns ? 0u : kChCopyOnly);
            // one sub-bin shares every bit >= lo; several differ in the digit itself
            ch.p = bin.lo;
            ch.pw = (u16)bin.W;
            ch.v0 = vfirst;
            u32 sb = 0;
            while ((1u << sb) < vlast - vfirst + 1) sb++;
            ch.sb = (u16)(nsub == 1 ? 0 : sb);
            j.chunks[idx] = ch;
          }
        }
        open = false;
      };
      for (u32 v = 0; v < nd; v++) {
        const u8 k = cls[v];
        if (k == 0) continue;
        if (k <= 2) {
          const u32 sz = cnt[v];
          if (open && csz + sz > j.chunk_max) emit();
          if (!open) {
            cb = boff[v];
            csz = 0;
            nsub = 0;
            vfirst = v;
            uns = false;
            open = true;
          }
          csz += sz;
          nsub++;
          vlast = v;
          if (k == 2) uns = true;
        } else {
          emit();
        }
      }
      emit();
    }
    __syncthreads();
  }
  // the last CTA numbers the tiles of the next level's bins and resets per-level counters
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&ctl->cls_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    finalize_list(j, N);
    if (tid == 0) {
      ctl->s_ticket = 0;
      ctl->cls_done = 0;
      ctl->nredo = 0;
      ctl->nbins[L] = 0;
      ctl->ntiles[L] = 0;
      ctl->base_used[L] = 0;
      ctl->status_used[L] = 0;
      __threadfence();
    }
  }
}

// Histogram entry point: copy the raw counts (u64) of bin 0 out.
__global__ void k_read_counts(Job j, u64* out, u32 nd) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < nd; v += gridDim.x * blockDim.x) out[v] = j.base[0][v];
}

// ------------------------------------------------------------------- launchers
size_t scatter_smem_bytes(const Job& j) { return scatter_layout(j.T, j.RW, j.wmax).total; }

// Largest shared memory either level kernel needs for tiles of T records.
size_t level_smem_for(u32 T, u32 RW, u32 KW, u32 wmax) {
  const size_t a = scatter_layout(T, RW, wmax).total, b = hist_smem_bytes_for(T, KW);
  return a > b ? a : b;
}

template <int KW, int RWT, int IT>
static cudaError_t launch_scatter_t(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  const size_t sm = scatter_smem_bytes(j);
  cudaFuncSetAttribute(k_scatter<KW, RWT, IT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (occ) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_scatter<KW, RWT, IT>, kSThreads, sm) != cudaSuccess ||
        *occ < 1)
      *occ = 1;
    return cudaSuccess;
  }
  k_scatter<KW, RWT, IT><<<grid, kSThreads, sm, s>>>(j, level);
  return cudaGetLastError();
}

template <int KW, int IT>
static cudaError_t scatter_rw(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  switch (j.RW) {
    case 1: return launch_scatter_t<KW, 1, IT>(j, level, grid, s, occ);
    case 2: return launch_scatter_t<KW, 2, IT>(j, level, grid, s, occ);
    case 3: return launch_scatter_t<KW, 3, IT>(j, level, grid, s, occ);
    case 4: return launch_scatter_t<KW, 4, IT>(j, level, grid, s, occ);
    default: return launch_scatter_t<KW, 0, IT>(j, level, grid, s, occ);
  }
}

template <int KW>
static cudaError_t scatter_it(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  switch (j.T / kSThreads) {
    case 16: return scatter_rw<KW, 16>(j, level, grid, s, occ);
    case 8: return scatter_rw<KW, 8>(j, level, grid, s, occ);
    case 4: return scatter_rw<KW, 4>(j, level, grid, s, occ);
    case 2: return scatter_rw<KW, 2>(j, level, grid, s, occ);
    default: return scatter_rw<KW, 1>(j, level, grid, s, occ);
  }
}

int scatter_ctas_per_sm(const Job& j, bool) {
  int n = 1;
  if (j.KW == 1) scatter_it<1>(j, 0, 0, 0, &n);
  else scatter_it<2>(j, 0, 0, 0, &n);
  return n;
}

static size_t hist_smem(const Job& j) { return hist_smem_bytes_for(j.T, j.KW); }

int hist_ctas_per_sm(const Job& j) {
  int n = 0;
  const size_t sm = hist_smem(j);
  cudaError_t e;
  if (j.KW == 1) {
    cudaFuncSetAttribute(k_hist<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hist<1>, kThreads, sm);
  } else {
    cudaFuncSetAttribute(k_hist<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hist<2>, kThreads, sm);
  }
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

int launch_init_plain(const Job& j, u32 lo, u32 W, cudaStream_t s) {
  k_init_plain<<<1, kThreads, 0, s>>>(j, lo, W);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_init_single_chunk(const Job& j, cudaStream_t s) {
  k_init_single_chunk<<<1, 32, 0, s>>>(j);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_init_segments(const Job& j, u32 grid, cudaStream_t s) {
  k_reset<<<1, 32, 0, s>>>(j);
  const u64 need = ceil_div(j.n_segs, kThreads);
  const u32 g = (u32)(need < grid ? (need ? need : 1) : grid);
  k_init_segments<<<g, kThreads, 0, s>>>(j);
  k_finalize0<<<1, kThreads, 0, s>>>(j);
  return cudaGetLastError() == cudaSuccess ? 3 : -1;
}

int launch_hist(const Job& j, int level, int mode, u32 grid, cudaStream_t s) {
  const size_t sm = hist_smem(j);
  if (j.KW == 1) {
    cudaFuncSetAttribute(k_hist<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_hist<1><<<grid, kThreads, sm, s>>>(j, level, mode);
  } else {
    cudaFuncSetAttribute(k_hist<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_hist<2><<<grid, kThreads, sm, s>>>(j, level, mode);
  }
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_scatter(const Job& j, int level, bool, u32 grid, cudaStream_t s) {
  cudaError_t e = j.KW == 1 ? scatter_it<1>(j, level, grid, s, nullptr) : scatter_it<2>(j, level, grid, s, nullptr);
  return e == cudaSuccess ? 1 : -1;
}

int launch_classify(const Job& j, int level, u32 grid, cudaStream_t s) {
  if (j.KW == 1) k_classify<1><<<grid, kThreads, 0, s>>>(j, level);
  else k_classify<2><<<grid, kThreads, 0, s>>>(j, level);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_read_counts(const Job& j, u64* d_counts, u32 W, cudaStream_t s) {
  const u32 nd = 1u << W;
  k_read_counts<<<(nd + 255) / 256, 256, 0, s>>>(j, d_counts, nd);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace rsg
