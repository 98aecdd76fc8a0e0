// Distribution passes of the MSD radix sort (Kokot et al., section 3.1, steps 1-2): for
// every large bin of a level, a histogram of its digit, the exclusive prefix sum of the
// histogram (bucket bases), and a stable scatter of its records into the other buffer.
// Then every sub-bin is classified: finished, sorted on chip (chunk), or large again.
//
// Kernels, all launched on the caller's stream:
//   k_hist      histogram of each bin's digit (+ the bin's key AND/OR at level 0); the
//               last CTA of a bin turns the counts into bucket bases.
//   k_scatter   tile-wise stable scatter with a decoupled look-back across the tiles of a
//               bin; also the key AND/OR of every sub-bin that stays large (digit skip).
//   k_classify  sub-bin classification, chunk packing, next level's bin list.
#include "rs_internal.cuh"

namespace rsg {

// Exclusive scan of one u64 per thread; returns the exclusive prefix, total in *total.
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
// One CTA.
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
constexpr int kHistItems = 8;  // records per thread per tile (T <= kThreads * kHistItems)

// The last CTA to count a bin: at level 0 check that the digit starts at the bin's highest
// differing key bit (else move it there and ask for a recount); then counts -> bases, and a
// mask slot for every sub-bin that will need another pass.
template <int KW>
__device__ void finish_bin(const Job& j, int L, u64 b, int level, int mode) {
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
    if (level == 0 && mode == 0) {
      const u64 v0 = (__ldcg(&bp->kand[0]) ^ __ldcg(&bp->kor[0])) & j.keymask[0];
      const u64 v1 = KW == 2 ? (__ldcg(&bp->kand[1]) ^ __ldcg(&bp->kor[1])) & j.keymask[1] : 0;
      const u32 p = top_bit_plus1(v0, v1);
      if (p == 0) {
        bp->flags |= kBinEqual;  // every key equal: already sorted, nothing to move
        s_ret = 1;
      } else if (bp->lo + W != p) {
        u32 nlo, nW;
        plan_digit(size, p, j.chunk_max, j.wmax, &nlo, &nW);
        if (nW > W) nW = W, nlo = p - W;
        bp->lo = nlo;
        bp->W = nW;
        bp->flags |= kBinRedo;
        bp->done = 0;
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
  const u64 nk = 2ull * KW;
  for (int q = 0; q < 2; q++) {
    const u32 v = v0 + q;
    if (v >= nd) break;
    const u64 c = q ? c1 : c0;
    const u64 e = q ? ex + c0 : ex;
    u64 tag = 0;
    if (c > j.chunk_max) {
      const u64 s = atomicAdd(&ctl->mslot_used, 1ull);
      if (s < j.cap_mslots) {
        u64* m = j.masks + s * nk;
        for (int k = 0; k < KW; k++) {
          m[k] = ~0ull;
          m[KW + k] = 0;
        }
        tag = s + 1;
      }
    }
    base[v] = e | (tag << kSlotShift);
  }
  if (mode == 1 && threadIdx.x == 0) bp->flags &= ~kBinRedo;
}

// mode 0: count (+ key AND/OR at level 0), finish bins; mode 1: recount level-0 bins flagged
// kBinRedo; mode 2: counts only; mode 3: count and finish a bin whose digit is given.
template <int KW>
__global__ void __launch_bounds__(kThreads) k_hist(Job j, int level, int mode) {
  const int L = level & 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0) return;
  const u64 ntiles = ctl->ntiles[L];
  Bin* bins = j.bins[L];
  __shared__ u32 hist[1 << kWMax];
  __shared__ u64 red[kWarps][4];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool want_masks = level == 0 && mode == 0;
  const u64 per = ceil_div(ntiles, gridDim.x);
  const u64 t0 = blockIdx.x * per;
  const u64 t1 = min(ntiles, t0 + per);
  if (t0 >= t1) return;
  for (u32 v = tid; v < (1u << kWMax); v += kThreads) hist[v] = 0;
  u64 cur = find_bin(bins, nb, t0);
  u32 counted = 0;
  u64 kand[2] = {~0ull, ~0ull}, kor[2] = {0ull, 0ull};
  __syncthreads();

  auto flush = [&](u64 b) {
    __syncthreads();
    const Bin* bb = &bins[b];
    const u32 nd = 1u << bb->W;
    const u64 bo = bb->base_off;
    for (u32 v = tid; v < nd; v += kThreads) {
      const u32 h = hist[v];
      if (h) atomicAdd(&j.base[L][bo + v], (u64)h);
      hist[v] = 0;
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
      s_last = (u64)(old + counted) == ceil_div(bins[b].size, j.T);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finish_bin<KW>(j, L, b, level, mode);
    }
    __syncthreads();
    counted = 0;
  };

  for (u64 t = t0; t < t1; t++) {
    u64 b = cur;
    while (b + 1 < nb && bins[b + 1].tile_start <= t) b++;
    if (b != cur) {
      if (counted) flush(cur);
      cur = b;
    }
    const Bin* bp = &bins[b];
    const u32 flags = bp->flags;
    if (mode == 1 && !(flags & kBinRedo)) continue;
    const u32 lo = bp->lo, W = bp->W, nd = 1u << W;
    const u64 tib = t - bp->tile_start;
    const u64 r0 = tib * j.T;
    const u64 r1 = min(bp->size, r0 + j.T);
    if (mode == 0 || mode == 3) {  // the scatter pass's look-back words of this tile start cleared
      const u64 so = bp->status_off + tib * nd;
      if (j.wide) {
        u64* st = (u64*)j.status[L] + so;
        for (u32 v = tid; v < nd; v += kThreads) st[v] = 0;
      } else {
        u32* st = (u32*)j.status[L] + so;
        for (u32 v = tid; v < nd; v += kThreads) st[v] = 0;
      }
    }
    const u64* src = j.buf[bp->parity] + bp->begin * j.RW;
    // all of the tile's key loads in flight before any is used
    Key<KW> keys[kHistItems];
#pragma unroll
    for (int it = 0; it < kHistItems; it++) {
      const u64 r = r0 + (u64)it * kThreads + tid;
      if (r < r1) keys[it] = load_key<KW>(src + r * j.RW, j);
    }
#pragma unroll
    for (int it = 0; it < kHistItems; it++) {
      const u64 r = r0 + (u64)it * kThreads + tid;
      if (r0 + (u64)it * kThreads >= r1) break;  // uniform
      const bool valid = r < r1;
      u32 d = 0;
      if (valid) {
        d = digit_of<KW>(keys[it], lo, W);
        if (want_masks) {
#pragma unroll
          for (int q = 0; q < KW; q++) {
            kand[q] &= keys[it].w[q];
            kor[q] |= keys[it].w[q];
          }
        }
      }
      const u32 peers = __match_any_sync(kFull, valid ? d : (0x10000u | lane));
      if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&hist[d], (u32)__popc(peers));
    }
    counted++;
  }
  if (counted) flush(cur);
}

// --------------------------------------------------------------------- scatter
// Shared memory of k_scatter for digit width <= wmax and T records per tile.
struct ScatterLayout {
  size_t stage, gbase, sand, sor, tcount, tbase, need, whist, perm, sdig, total;
};

__host__ __device__ inline ScatterLayout scatter_layout(u32 T, u32 RW, u32 KW, u32 wmax) {
  ScatterLayout s;
  const size_t nd = (size_t)1 << wmax;
  size_t o = 0;
  s.stage = o; o += (size_t)T * RW * 8;
  s.gbase = o; o += nd * 8;
  s.sand = o; o += nd * KW * 8;   // AND of the keys per digit, as 2*KW 32-bit halves
  s.sor = o; o += nd * KW * 8;
  s.tcount = o; o += nd * 4;
  s.tbase = o; o += nd * 4;
  s.need = o; o += (nd / 32 + 1) * 4;
  s.whist = o; o += (size_t)kWarps * nd * 2;
  s.perm = o; o += (size_t)T * 2;
  s.sdig = o; o += (size_t)T * 2;
  s.total = (o + 127) & ~(size_t)127;
  return s;
}

constexpr int kMaxItems = 8;  // records per thread per tile (T <= kThreads * kMaxItems)

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

template <typename S>
__device__ __forceinline__ u64 look_back(S* st, u64 self, u32 nd, u64 tib, u32 c, const Job& j, bool stall) {
  Ctl* ctl = j.ctl;
  if (tib == 0) {
    st_release(st + self, (S)(((S)2 << LB<S>::kShift) | (S)c));
    return 0;
  }
  st_release(st + self, (S)(((S)1 << LB<S>::kShift) | (S)c));
  u64 excl = 0;
  u64 idx = self - nd;
  for (u64 back = 1; back <= tib; back++, idx -= nd) {
    // a stalled wait (testing) polls a word that no tile ever writes
    const S* wp = stall && back == 1 ? (const S*)nullptr : st + idx;
    S w = wp ? ld_acquire(wp) : (S)ld_acquire(&ctl->never);
    u32 polls = 0;
    while ((w >> LB<S>::kShift) == 0) {
      // bounded wait: give up after `watchdog` polls, or at once when any wait of this
      // call has already given up (the result is then undefined and reported)
      if (++polls > j.watchdog || ((polls & 255) == 0 && (*(volatile u32*)&ctl->err & kErrTimeout))) {
        atomicOr(&ctl->err, kErrTimeout);
        break;
      }
      __nanosleep(100);
      w = wp ? ld_acquire(wp) : (S)ld_acquire(&ctl->never);
    }
    excl += (u64)(w & LB<S>::kVal);
    if ((w >> LB<S>::kShift) != 1) break;  // inclusive prefix (or gave up): done
  }
  st_release(st + self, (S)(((S)2 << LB<S>::kShift) | (S)(excl + c)));
  return excl;
}

template <int KW, int RWT>
__global__ void __launch_bounds__(kThreads) k_scatter(Job j, int level) {
  const int L = level & 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0) return;
  const u64 ntiles = ctl->ntiles[L];
  const Bin* bins = j.bins[L];
  const u32 RW = RWT ? (u32)RWT : j.RW;
  const u32 T = j.T;
  const ScatterLayout lay = scatter_layout(T, RW, KW, j.wmax);
  extern __shared__ __align__(16) unsigned char smem[];
  u64* stage = (u64*)(smem + lay.stage);
  u64* gbase = (u64*)(smem + lay.gbase);
  u32* sand = (u32*)(smem + lay.sand);  // [v][2*KW] 32-bit halves: native shared atomics
  u32* sor = (u32*)(smem + lay.sor);
  u32* tcount = (u32*)(smem + lay.tcount);
  u32* tbase = (u32*)(smem + lay.tbase);
  u32* need = (u32*)(smem + lay.need);
  u16* whist = (u16*)(smem + lay.whist);
  u16* perm = (u16*)(smem + lay.perm);
  u16* sdig = (u16*)(smem + lay.sdig);
  __shared__ u64 s_ticket, s_bin;
  __shared__ u32 scan_scr[kWarps + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 its = T / kThreads;
  const u32 per_warp = T / kWarps;
  // Sub-bin key AND/OR accumulate in shared memory over all tiles this CTA takes from one
  // bin, and go to global memory once per (CTA, bin).
  u64 mask_bin = ~0ull;
  auto flush_masks = [&](u64 mb) {
    const Bin* mp = &bins[mb];
    const u32 mnd = 1u << mp->W;
    const u64* mbase = j.base[L] + mp->base_off;
    for (u32 v = tid; v < mnd; v += kThreads) {
      if (!((need[v >> 5] >> (v & 31)) & 1u)) continue;
      const u64 slot = mbase[v] >> kSlotShift;
      u64* m = j.masks + (slot - 1) * 2 * KW;
#pragma unroll
      for (int q = 0; q < KW; q++) {
        const u64 a = ((u64)sand[v * 2 * KW + 2 * q + 1] << 32) | sand[v * 2 * KW + 2 * q];
        const u64 o = ((u64)sor[v * 2 * KW + 2 * q + 1] << 32) | sor[v * 2 * KW + 2 * q];
        if (o | ~a) {  // skip untouched entries
          atomicAnd(&m[q], a);
          atomicOr(&m[KW + q], o);
        }
      }
    }
  };

  for (;;) {
    if (tid == 0) {
      const u64 tk = atomicAdd(&ctl->s_ticket, 1ull);
      s_ticket = tk;
      s_bin = tk < ntiles ? find_bin(bins, nb, tk) : 0;
    }
    __syncthreads();
    const u64 t = s_ticket;
    const u64 b = s_bin;
    __syncthreads();  // every thread has its ticket before thread 0 may take the next
    if (t >= ntiles) break;
    const Bin bin = bins[b];
    const Bin* bp = &bin;
    if (bp->flags & kBinEqual) continue;
    const u32 lo = bp->lo, W = bp->W, nd = 1u << W;
    const u64 tib = t - bp->tile_start;
    const u64 r0 = tib * T;
    const u32 cnt = (u32)min((u64)T, bp->size - r0);
    const u64* src = j.buf[bp->parity] + (bp->begin + r0) * RW;
    u64* dstb = j.buf[bp->parity ^ 1];
    const u64* bbase = j.base[L] + bp->base_off;

    load_words_async(stage, src, (u64)cnt * RW);
    for (u32 i = tid; i < (u32)kWarps * nd; i += kThreads) whist[i] = 0;
    if (b != mask_bin) {
      if (mask_bin != ~0ull) flush_masks(mask_bin);
      __syncthreads();
      for (u32 i = tid; i < nd / 32 + 1; i += kThreads) need[i] = 0;
      __syncthreads();
      for (u32 v = tid; v < nd; v += kThreads) {
        if (bbase[v] >> kSlotShift) {
          atomicOr(&need[v >> 5], 1u << (v & 31));
#pragma unroll
          for (int k = 0; k < 2 * KW; k++) {
            sand[v * 2 * KW + k] = ~0u;
            sor[v * 2 * KW + k] = 0;
          }
        }
      }
      mask_bin = b;
    }
    cp_async_wait_all();
    __syncthreads();

    // stable rank: warp w owns records [w*per_warp, (w+1)*per_warp), visited in order
    u32 packed[kMaxItems];
    u16* wh = whist + warp * nd;
#pragma unroll
    for (int it = 0; it < kMaxItems; it++) {
      packed[it] = 0xffffffffu;
      if ((u32)it < its) {
        const u32 r = warp * per_warp + it * 32 + lane;
        const bool valid = r < cnt;
        Key<KW> k;
        u32 d = 0;
        if (valid) {
          k = load_key<KW>(stage + (u64)r * RW, j);
          d = digit_of<KW>(k, lo, W);
        }
        const u32 peers = __match_any_sync(kFull, valid ? d : (0x10000u | lane));
        const u32 before = __popc(peers & lanemask_lt());
        u32 old = 0;
        if (valid) old = wh[d];
        __syncwarp();
        if (valid && before == 0) wh[d] = (u16)(old + __popc(peers));
        __syncwarp();
        if (valid) {
          packed[it] = (old + before) | (d << 16);
          if ((need[d >> 5] >> (d & 31)) & 1u) {
#pragma unroll
            for (int q = 0; q < KW; q++) {
              const u32 alo = __reduce_and_sync(peers, (u32)k.w[q]);
              const u32 ahi = __reduce_and_sync(peers, (u32)(k.w[q] >> 32));
              const u32 olo = __reduce_or_sync(peers, (u32)k.w[q]);
              const u32 ohi = __reduce_or_sync(peers, (u32)(k.w[q] >> 32));
              if (before == 0) {
                atomicAnd(&sand[d * 2 * KW + 2 * q], alo);
                atomicAnd(&sand[d * 2 * KW + 2 * q + 1], ahi);
                atomicOr(&sor[d * 2 * KW + 2 * q], olo);
                atomicOr(&sor[d * 2 * KW + 2 * q + 1], ohi);
              }
            }
          }
        }
      }
    }
    __syncthreads();
    // per digit: offsets of each warp's run, and the tile's count
    for (u32 v = tid; v < nd; v += kThreads) {
      u32 run = 0;
      for (int w = 0; w < kWarps; w++) {
        const u32 c = whist[w * nd + v];
        whist[w * nd + v] = (u16)run;
        run += c;
      }
      tcount[v] = run;
      tbase[v] = run;
    }
    __syncthreads();
    block_exclusive_scan(tbase, nd, scan_scr);
    // decoupled look-back over the earlier tiles of this bin: records of digit v before this tile
    for (u32 v = tid; v < nd; v += kThreads) {
      const u64 self = bp->status_off + tib * nd + v;
      u64 excl;
      const bool stall = j.inject && v == 0 && tib == 1;
      if (j.wide)
        excl = look_back<u64>((u64*)j.status[L], self, nd, tib, tcount[v], j, stall);
      else
        excl = look_back<u32>((u32*)j.status[L], self, nd, tib, tcount[v], j, stall);
      gbase[v] = bp->begin + (bbase[v] & kBaseMask) + excl - tbase[v];
    }
#pragma unroll
    for (int it = 0; it < kMaxItems; it++) {
      if (packed[it] != 0xffffffffu) {
        const u32 d = packed[it] >> 16;
        const u32 slot = tbase[d] + whist[warp * nd + d] + (packed[it] & 0xffffu);
        perm[slot] = (u16)(warp * per_warp + it * 32 + lane);
        sdig[slot] = (u16)d;
      }
    }
    __syncthreads();
    // write the tile in digit order: consecutive slots of one digit go to consecutive
    // records.  A destination outside the bin (possible only after a failed wait or a
    // corrupted histogram, both reported) is skipped, never written.
    const u64 lo_rec = bp->begin, hi_rec = bp->begin + bp->size;
    bool bad = false;
    if (RW == 2) {
      for (u32 s = tid; s < cnt; s += kThreads) {
        const u32 r = perm[s];
        const u64 dst = gbase[sdig[s]] + s;
        if (dst < lo_rec || dst >= hi_rec) { bad = true; continue; }
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(stage + 2 * (u64)r);
        __stcs(reinterpret_cast<ulonglong2*>(dstb + 2 * dst), v);
      }
    } else if (RWT != 0) {
      for (u32 q = tid; q < cnt * RW; q += kThreads) {
        const u32 s = q / RW, w = q - s * RW;
        const u32 r = perm[s];
        const u64 dst = gbase[sdig[s]] + s;
        if (dst < lo_rec || dst >= hi_rec) { bad = true; continue; }
        __stcs(dstb + dst * RW + w, stage[(u64)r * RW + w]);
      }
    } else {
      for (u32 s = tid; s < cnt; s += kThreads) {
        const u32 r = perm[s];
        const u64 dst = gbase[sdig[s]] + s;
        if (dst < lo_rec || dst >= hi_rec) { bad = true; continue; }
        u64* d = dstb + dst * RW;
        const u64* sp = stage + (u64)r * RW;
        for (u32 w = 0; w < RW; w++) __stcs(d + w, sp[w]);
      }
    }
    if (bad) atomicOr(&ctl->err, kErrInternal);
    __syncthreads();
  }
  if (mask_bin != ~0ull) flush_masks(mask_bin);
}

// -------------------------------------------------------------------- classify
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
    if (bin.flags & kBinEqual) continue;
    const u32 nd = 1u << bin.W;
    const u32 p1 = bin.parity ^ 1;
    const u64* bbase = j.base[L] + bin.base_off;
    for (u32 v = tid; v < nd; v += kThreads) {
      const u64 e = bbase[v];
      u64 bv = e & kBaseMask;
      u64 next = v + 1 < nd ? (bbase[v + 1] & kBaseMask) : bin.size;
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
        const u64 slot = e >> kSlotShift;
        u32 p = bin.lo;  // without masks: every bit below the digit may differ
        bool equal = false;
        if (slot) {
          const u64* m = j.masks + (slot - 1) * 2 * KW;
          const u64 v0 = (m[0] ^ m[KW]) & j.keymask[0];
          const u64 v1 = KW == 2 ? (m[1] ^ m[KW + 1]) & j.keymask[1] : 0;
          p = top_bit_plus1(v0, v1);
          equal = p == 0;
        }
        const u64 rb = bin.begin + bv;
        if (equal) {
          k = 4;
          if (p1) {  // finished, but in tmp: copy back
            const u64 np = ceil_div(c, kPieceRecords);
            const u64 idx = atomicAdd(&ctl->npieces, np);
            if (idx + np > j.cap_pieces) {
              atomicOr(&ctl->err, kErrOverflow);
            } else {
              for (u64 q = 0; q < np; q++) {
                Piece pc;
                pc.begin = rb + q * kPieceRecords;
                pc.size = min(kPieceRecords, c - q * kPieceRecords);
                j.pieces[idx + q] = pc;
              }
            }
          }
        } else {
          k = 3;
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
            nbn.lo = nlo;
            nbn.W = nW;
            nbn.parity = p1;
            j.bins[N][idx] = nbn;
            for (u32 q = 0; q < nnd; q++) j.base[N][bo + q] = 0;
          }
        }
      }
      cls[v] = k;
    }
    __syncthreads();
    if (tid == 0) {
      // greedy packing of consecutive small sub-bins into on-chip chunks
      u64 cb = 0;
      u32 csz = 0;
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
            uns = false;
            open = true;
          }
          csz += sz;
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
      ctl->mslot_used = 0;
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
size_t scatter_smem_bytes(const Job& j) { return scatter_layout(j.T, j.RW, j.KW, j.wmax).total; }

template <int KW, int RWT>
static void set_scatter_attr(const Job& j) {
  cudaFuncSetAttribute(k_scatter<KW, RWT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem_bytes(j));
}

template <int KW>
static cudaError_t launch_scatter_kw(const Job& j, int level, u32 grid, cudaStream_t s) {
  const size_t sm = scatter_smem_bytes(j);
#define RS_SCAT(R)                                                                      \
  do {                                                                                  \
    cudaFuncSetAttribute(k_scatter<KW, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)sm);                                                      \
    k_scatter<KW, R><<<grid, kThreads, sm, s>>>(j, level);                             \
  } while (0)
  switch (j.RW) {
    case 1: RS_SCAT(1); break;
    case 2: RS_SCAT(2); break;
    case 3: RS_SCAT(3); break;
    case 4: RS_SCAT(4); break;
    default: RS_SCAT(0); break;
  }
#undef RS_SCAT
  return cudaGetLastError();
}

int scatter_ctas_per_sm(const Job& j, bool) {
  int n = 0;
  const size_t sm = scatter_smem_bytes(j);
  cudaError_t e;
  if (j.KW == 1) {
    cudaFuncSetAttribute(k_scatter<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_scatter<1, 0>, kThreads, sm);
  } else {
    cudaFuncSetAttribute(k_scatter<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_scatter<2, 0>, kThreads, sm);
  }
  if (e != cudaSuccess || n < 1) n = 1;
  return n;
}

int hist_ctas_per_sm(const Job& j) {
  int n = 0;
  cudaError_t e = j.KW == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hist<1>, kThreads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hist<2>, kThreads, 0);
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
  if (j.KW == 1) k_hist<1><<<grid, kThreads, 0, s>>>(j, level, mode);
  else k_hist<2><<<grid, kThreads, 0, s>>>(j, level, mode);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_scatter(const Job& j, int level, bool, u32 grid, cudaStream_t s) {
  cudaError_t e = j.KW == 1 ? launch_scatter_kw<1>(j, level, grid, s) : launch_scatter_kw<2>(j, level, grid, s);
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
