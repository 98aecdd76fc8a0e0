// The distribution pass of the MSD radix sort (Kokot et al., section 3.1, step 1, and the
// buffered scatter of sections 2.1 / 3.2): a stable scatter of every large bin of a level into
// the other buffer, tile by tile, with the destinations that the histogram pass (rs_level.cu)
// prepared per lane.
#include <algorithm>

#include "rs_internal.cuh"

namespace rsg {

// --------------------------------------------------------------------- scatter
constexpr int kSThreads = 256;  // threads of a scatter CTA
// 8-byte records at the default tile (4,096 records) with 10-bit digit tables take CTAs of
// 512 threads: each warp ranks half as many records in a row, and twice as many warps hide
// the shared-memory latency of the ranking (measured at 2e9 x 8 B, two 10-bit levels: 31.3 vs
// 33.8 ms of scatter per sort).  Not with 9-bit tables (1e9 x 8 B: 13.3 vs 12.5 ms), nor for
// larger records (16 to 32 bytes: 1-2% slower), where 256 threads keep the lane masks.
constexpr int kSThreadsWide = 512;
__host__ __device__ inline u32 scatter_threads(u32 T, u32 RW, u32 wmax) {
  return RW == 1 && T == 4096 && wmax >= 10 ? (u32)kSThreadsWide : (u32)kSThreads;
}

// Shared memory of k_scatter: T records, per-warp 16-bit digit counters (row stride 2^wmax),
// the tile's permutation (sharing its room with one byte per warp and bucket, used while
// ranking to find the lanes that share a bucket: see rank_item), per-digit counts / run bases
// / global bases, and, when two CTAs per SM still fit, a 32-bit lane mask per warp and bucket
// (the other way rank_item finds them).
struct ScatterLayout {
  size_t stage, whist, slot, tbase, gbase, winner, pmask, total;
  bool masks;
};

// shared memory of a scatter CTA that still lets two of them (and their static shared memory)
// share an SM
constexpr size_t kScatterPairSmem = 112 * 1024;

__host__ __device__ inline ScatterLayout scatter_layout(u32 T, u32 RW, u32 wmax) {
  const size_t kSWarps = scatter_threads(T, RW, wmax) / 32;
  ScatterLayout s;
  const size_t nd = (size_t)1 << wmax;
  size_t o = 0;
  s.stage = o; o += (size_t)T * RW * 8;
  s.whist = o; o += (size_t)kSWarps * nd * 2;
  // (the winner bytes are used only while ranking, before the permutation is written)
  s.slot = s.winner = o; o += std::max((size_t)T * 4, (size_t)kSWarps * nd);
  o = (o + 15) & ~(size_t)15;
  s.tbase = o; o += nd * 4;
  s.gbase = o; o += nd * 8;
  const size_t with_masks = ((o + kSWarps * nd * 4) + 127) & ~(size_t)127;
  s.masks = with_masks <= kScatterPairSmem;
  s.pmask = o;
  if (s.masks) o += kSWarps * nd * 4;
  s.total = (o + 127) & ~(size_t)127;
  return s;
}

// Digit of a staged record.  No key mask is needed: a digit window never reaches past the key.
template <int KW>
__device__ __forceinline__ u32 staged_digit(const u64* rec, u32 lo, u32 W) {
  Key<KW> k;
  k.w[0] = rec[0];
  if (KW == 2) k.w[KW - 1] = rec[1];
  return digit_of<KW>(k, lo, W);
}

// Digits per thread in the scatter's prefix pass: nd / NT, at least 2 (the per-warp counters
// are read two at a time).
template <int NT>
__device__ __forceinline__ u32 digits_per_thread(u32 nd) { return nd > 2u * NT ? nd / NT : 2u; }

constexpr u64 kSkip = ~0ull;  // gbase of a digit whose run would leave its bin

// Stable scatter of every large bin of the level into the other buffer.  The level's tiles
// are split into the same lanes as in the histogram pass (contiguous tile ranges); a CTA
// takes its lanes in turn and walks each lane's tiles in order.  The histogram pass left,
// for every (lane, bin) segment and digit, where the segment's records of that digit start
// (bucket base + the digit's records in the bin's earlier lanes), so a tile's destinations
// are known from those starts plus the digit counts of the lane's earlier tiles of the bin,
// which the CTA keeps in registers: no tile waits for another.
//
// Per tile of T = NT * IT records: the records are staged in shared memory; warp w
// ranks its strip of records in order (lanes sharing a bucket found through per-warp lane
// masks or bytes per bucket, per-warp 16-bit counters), so the order inside a digit is the
// input order (stable); the digit counts are scanned; then the tile is written in digit
// order, so consecutive threads write consecutive records of a run with 16-byte streaming
// stores.
// MASKS: the layout has the per-warp lane masks (chosen at launch from scatter_layout).
// NT: threads of the CTA (scatter_threads).
template <int KW, int RWT, int IT, bool MASKS, int NT>
__global__ void __launch_bounds__(NT, 2) k_scatter(Job j, int level) {
  constexpr int kSWarps = NT / 32;
  const int L = level & 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0 || call_failed(ctl)) return;
  const u64 ntiles = ctl->ntiles[L];
  const Bin* bins = j.bins[L];
  const u32 RW = RWT ? (u32)RWT : j.RW;
  constexpr u32 T = NT * IT;
  constexpr u32 PW = T / kSWarps;  // records per warp strip
  constexpr u32 kDigitsPerThread = (1u << kWMax) / NT;
  const u32 WSMAX = 1u << j.wmax;  // room for the per-warp counters: kSWarps rows of 2^wmax
  const ScatterLayout lay = scatter_layout(T, RW, j.wmax);
  if (MASKS != lay.masks) {  // (cannot happen: the launcher picks MASKS from the same layout)
    if (blockIdx.x == 0 && threadIdx.x == 0) report(ctl, kErrInternal);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  u64* stage = (u64*)(smem + lay.stage);
  u16* whist = (u16*)(smem + lay.whist);
  u8* winner = (u8*)(smem + lay.winner);
  u32* peermask = (u32*)(smem + lay.pmask);  // (lay.masks: zero between uses)
  u32* slotw = (u32*)(smem + lay.slot);  // per output slot: staged record | digit << 16
  u32* tbase = (u32*)(smem + lay.tbase);
  u64* gbase = (u64*)(smem + lay.gbase);
  __shared__ u32 scan_scr[kSWarps + 1];
  __shared__ __align__(8) u64 s_bar[kSWarps];  // bar w: warp w's strip of a tile has landed
  __shared__ __align__(8) u64 s_never;          // testing (kInjectWait): a barrier nothing completes
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 ltmask = lanemask_lt();
  u32 bar_phase = 0;
  if (tid < kSWarps) mbar_init(&s_bar[tid], 1);
  if (tid == 0) mbar_init(&s_never, 1);
  // per-warp digit counters: counts while ranking, then each warp's offset inside the digit's
  // run; they are zeroed again while the tile is written out
  for (u32 i = tid; i < kSWarps * WSMAX; i += NT) whist[i] = 0;
  if (MASKS)
    for (u32 i = tid; i < kSWarps * WSMAX; i += NT) peermask[i] = 0;
  const u64 per = lane_tiles(ntiles, j.lanes);
  bool inject = (j.inject & kInjectRange) && blockIdx.x == 0 && tid == 0;  // testing: fail one run check
  bool inject_wait = (j.inject & kInjectWait) && blockIdx.x == 0;  // testing: one wait runs out
  __syncthreads();

  for (u64 ln = blockIdx.x; ln < j.lanes; ln += gridDim.x) {
    const u64 t0 = ln * per, t1 = min(ntiles, t0 + per);
    if (t0 >= t1) break;  // later lanes are empty too
    u64 b = find_bin(bins, nb, t0);
    u64 cur = ~0ull;
    u64 run[kDigitsPerThread];    // this thread's digits: start of the next run, bin-relative
    for (u64 t = t0; t < t1; t++) {
      while (b + 1 < nb && bins[b + 1].tile_start <= t) b++;
      const Bin* bp = &bins[b];
      const u32 lo = bp->lo, W = bp->W, BW = bucket_bits(W, bp->flags), nd = 1u << BW;
      const bool dom = (bp->flags & kBinDom) != 0;
      Key<KW> K = {};
      u32 dK = 0;
      if (dom) {
#pragma unroll
        for (int q = 0; q < KW; q++) K.w[q] = bp->dom[q];
        dK = digit_of<KW>(K, lo, W);
      }
      // bucket of a staged record (a digit window never reaches past the key, so only the
      // comparisons with a dominant key need the key mask)
      auto bucket = [&](const u64* rec) -> u32 {
        if (!dom) return staged_digit<KW>(rec, lo, W);
        Key<KW> k;
#pragma unroll
        for (int q = 0; q < KW; q++) k.w[q] = rec[q] & j.keymask[q];
        return bucket_of<KW>(k, lo, W, true, K, dK);
      };
      // per-warp counters with a row stride of this bin's bucket count (every tile zeroes the
      // rows it used, so the rows of a narrower or wider digit start at zero too)
      const u32 WS = nd < 2 ? 2 : nd;
      u16* wh = whist + warp * WS;
      const u64 begin = bp->begin, size = bp->size;
      const u64 tib = t - bp->tile_start;
      const u32 parity = bp->parity;
      if ((bp->flags & kBinEqual) || tib * T >= size) continue;  // finished bin (or inconsistent list)
      const u64 r0 = tib * T;
      const u32 cnt = (u32)min((u64)T, size - r0);
      u64* dstb = j.buf[parity ^ 1];

      // the tile comes in by bulk copies when it starts on a 16-byte boundary (an even word
      // count per record: always), one per warp strip, each completing on its own barrier so
      // that a warp starts ranking as soon as its strip has landed; else by 16- or 8-byte
      // copies of every thread
      const u64* src = j.buf[parity] + (begin + r0) * RW;
      const u32 bytes = cnt * RW * 8;
      const bool bulk = ((((uintptr_t)src) | bytes) & 15) == 0;
      if (!bulk) {
        load_words_async<NT>(stage, src, (u64)cnt * RW);
      } else if (lane == 0) {
        // (strip boundaries are multiples of PW records: 16-byte aligned, as is the tile's end)
        const u32 a = warp * PW, e = min(cnt, a + PW);
        fence_proxy_async_smem();  // the last tile's reads of the stage are done (barrier)
        if (e > a) bulk_load(stage + (u64)a * RW, src + (u64)a * RW, (e - a) * RW * 8, &s_bar[warp]);
        else mbar_arrive(&s_bar[warp]);
      }
      // the lane's next tile of this bin comes into L2 while this one is processed
      if (tid == 0 && t + 1 < t1 && r0 + T < size)
        prefetch_l2(j.buf[parity] + (begin + r0 + T) * RW, min((u64)T, size - r0 - T) * RW * 8);
      if (b != cur) {  // first tile of this lane's part of the bin: its run starts
        cur = b;
        const u64* sg = j.seg + ((ln + b) << j.wmax);
        const u32 D = digits_per_thread<NT>(nd);
#pragma unroll
        for (u32 q = 0; q < kDigitsPerThread; q++) {
          const u32 v = D * tid + q;
          run[q] = (q < D && v < nd) ? sg[v] : 0;
        }
      }
      // bounded: a strip that has not landed after j.wd_polls suspended waits is reported after
      // the ranking (its warp ranks nothing; the copies cannot be cancelled, so the CTA waits
      // for every strip once more, with the default limit, before it gives up); every thread
      // takes the same way out
      bool failed = false;
      if (bulk) {
        failed = !mbar_wait(inject_wait && warp == 0 ? &s_never : &s_bar[warp], inject_wait && warp == 0 ? 0u : bar_phase,
                            j.wd_polls);
        inject_wait = false;
        failed = __any_sync(kFull, failed);  // (the whole warp skips its strip)
      } else {
        cp_async_wait_all();
        __syncthreads();
      }

      // Stable rank of one item (one record per lane, lanes in record order) among the warp's
      // records of its bucket: the count before this item (per-warp counter) + the lanes below
      // it with the same bucket.  The lanes sharing a bucket are found without a vote per digit
      // bit, in one of two ways:
      //   * masks (when the room fits): every lane ORs its bit into its bucket's 32-bit mask,
      //     which then holds exactly the lanes of the bucket; the bucket's first lane clears it;
      //   * winner bytes: every lane writes its id into its bucket's byte and all lanes of a
      //     bucket read back the same winner.  With 2^9 buckets and 32 lanes most items share
      //     no bucket (every lane reads its own id back: one vote tells); otherwise lanes are
      //     grouped by their winner's id (5 votes).
      // Lanes without a record (valid = false) touch neither and form groups of their own.
      // Returns (rank | bucket << 16), or all ones.
      u8* wn = winner + warp * WS;
      u32* wm = peermask + warp * WS;
      constexpr bool masks = MASKS;
      auto rank_item = [&](u32 d, bool valid) -> u32 {
        u32 peers = 1u << lane, old = 0;
        if (masks) {
          __syncwarp();  // (the last item's first lanes have cleared their masks)
          if (valid) atomicOr(&wm[d], 1u << lane);
          __syncwarp();
          if (valid) {
            peers = wm[d];
            old = wh[d];
          }
        } else {
          if (valid) wn[d] = (u8)lane;
          __syncwarp();
          const u32 w = valid ? (u32)wn[d] : (u32)lane;
          if (valid) old = wh[d];
          if (__any_sync(kFull, w != (u32)lane)) {
            u32 x = 0;
#pragma unroll
            for (int b = 0; b < 5; b++) {
              const u32 v = __ballot_sync(kFull, (w >> b) & 1u);
              x |= v ^ (0u - ((w >> b) & 1u));
            }
            peers = ~x;
          }
        }
        const u32 before = __popc(peers & ltmask);
        __syncwarp();  // (every lane has read its bucket's mask or byte, and its counter)
        if (valid && before == 0) {
          wh[d] = (u16)(old + __popc(peers));
          if (masks) wm[d] = 0;
        }
        return valid ? ((old + before) | (d << 16)) : 0xffffffffu;
      };
      // stable rank: warp w owns records [w*PW, (w+1)*PW), visited in order
      u32 packed[IT];
      if (failed) {
#pragma unroll
        for (int it = 0; it < IT; it++) packed[it] = 0xffffffffu;
      } else if (cnt == T) {
        // first every item's bucket, then the ranks
        u32 dg[IT];
        if (!dom) {  // (the two loops differ in the bucket function only)
#pragma unroll
          for (int it = 0; it < IT; it++) dg[it] = staged_digit<KW>(stage + (u64)(warp * PW + it * 32 + lane) * RW, lo, W);
        } else {
#pragma unroll
          for (int it = 0; it < IT; it++) dg[it] = bucket(stage + (u64)(warp * PW + it * 32 + lane) * RW);
        }
#pragma unroll
        for (int it = 0; it < IT; it++) packed[it] = rank_item(dg[it], true);
      } else {
#pragma unroll
        for (int it = 0; it < IT; it++) {
          const u32 r = warp * PW + it * 32 + lane;
          const bool valid = r < cnt;
          packed[it] = rank_item(valid ? bucket(stage + (u64)r * RW) : 0u, valid);
        }
      }
      if (__syncthreads_or(failed)) {
        if (tid == 0) report(ctl, kErrTimeout);
        if (lane == 0) mbar_wait(&s_bar[warp], bar_phase, kWaitPolls);
        __syncwarp();
        return;
      }
      if (bulk) bar_phase ^= 1;
      // Thread tid owns digits [D*tid, D*tid + D): it turns their per-warp counts into each
      // warp's offset inside the digit's run (two 16-bit counters per 32-bit access), then one
      // block scan of the threads' totals gives the digits' first slots in the tile.
      const u32 D = digits_per_thread<NT>(nd);
      const u32 v0 = D * tid;
      u32 c[kDigitsPerThread];
#pragma unroll
      for (u32 q = 0; q < kDigitsPerThread; q++) c[q] = 0;
      if (v0 < nd) {
        u32* wh32 = (u32*)whist;
#pragma unroll
        for (u32 p2 = 0; p2 < kDigitsPerThread / 2; p2++) {
          if (2 * p2 >= D) break;
          u32 a0 = 0, a1 = 0;
#pragma unroll
          for (int w = 0; w < kSWarps; w++) {
            u32* x = wh32 + w * (WS >> 1) + (v0 >> 1) + p2;
            const u32 y = *x;
            *x = a0 | (a1 << 16);
            a0 += y & 0xffffu;
            a1 += y >> 16;
          }
          c[2 * p2] = a0;
          c[2 * p2 + 1] = a1;
        }
      }
      u32 mine = 0;
#pragma unroll
      for (u32 q = 0; q < kDigitsPerThread; q++) mine += c[q];
      u32 tb = block_exclusive_sum<NT>(mine, scan_scr);
      // destinations of this thread's runs; a run that would leave its bin (possible only with
      // corrupted counts) is reported and not written
#pragma unroll
      for (u32 q = 0; q < kDigitsPerThread; q++) {
        const u32 v = v0 + q;
        if (q >= D || v >= nd) break;
        const u32 cq = c[q];
        const u64 first = run[q];
        run[q] += cq;
        u64 g = begin + first - tb;
        bool bad = cq && (first > size || cq > size - first);
        if (cq && inject) {
          bad = true;
          inject = false;
        }
        if (bad) {
          report(ctl, kErrInternal);
          g = kSkip;
        }
        tbase[v] = tb;
        gbase[v] = g;
        tb += cq;
      }
      __syncthreads();
      if (cnt == T) {
        // 8 items at a time: their counter loads first, then the stores (measured: 0.06 to
        // 0.14 ms less scatter per sort on uniform, Zipf and k-mer records)
        constexpr int B = IT < 8 ? IT : 8;
#pragma unroll
        for (int b0 = 0; b0 < IT; b0 += B) {
          u32 sl[B];
#pragma unroll
          for (int q = 0; q < B; q++) {
            const u32 d = packed[b0 + q] >> 16;
            sl[q] = tbase[d] + wh[d] + (packed[b0 + q] & 0xffffu);
          }
#pragma unroll
          for (int q = 0; q < B; q++)
            slotw[sl[q]] = (warp * PW + (b0 + q) * 32 + lane) | ((packed[b0 + q] >> 16) << 16);
        }
      } else {
#pragma unroll
        for (int it = 0; it < IT; it++) {
          if (packed[it] != 0xffffffffu) {
            const u32 d = packed[it] >> 16;
            const u32 slot = tbase[d] + wh[d] + (packed[it] & 0xffffu);
            slotw[slot] = (warp * PW + it * 32 + lane) | (d << 16);
          }
        }
      }
      __syncthreads();
      // per-warp counters back to zero for the next tile (nothing reads them before then)
      for (u32 v = tid; v < nd; v += NT) {
#pragma unroll
        for (int w = 0; w < kSWarps; w++) whist[w * WS + v] = 0;
      }
      // write the tile in digit order: consecutive slots of one digit go to consecutive records
      if (RW == 2 && cnt == T) {
        // a full tile: every thread's IT slots, 8 at a time with all their loads in flight
        // (measured: 0.27 ms less scatter per sort of 1e9 x 16 B than one slot at a time)
        constexpr int B = IT < 8 ? IT : 8;
#pragma unroll
        for (int b0 = 0; b0 < IT; b0 += B) {
          u32 swv[B];
#pragma unroll
          for (int q = 0; q < B; q++) swv[q] = slotw[tid + (b0 + q) * NT];
          ulonglong2 v[B];
          u64 g[B];
#pragma unroll
          for (int q = 0; q < B; q++) {
            g[q] = gbase[swv[q] >> 16];
            v[q] = *reinterpret_cast<const ulonglong2*>(stage + 2 * (swv[q] & 0xffffu));
          }
#pragma unroll
          for (int q = 0; q < B; q++)
            if (g[q] != kSkip) __stcs(reinterpret_cast<ulonglong2*>(dstb + 2 * (g[q] + tid + (b0 + q) * NT)), v[q]);
        }
      } else if (RW == 2) {
        for (u32 s = tid; s < cnt; s += NT) {
          const u32 sw = slotw[s];
          const u64 g = gbase[sw >> 16];
          const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(stage + 2 * (sw & 0xffffu));
          if (g == kSkip) continue;
          __stcs(reinterpret_cast<ulonglong2*>(dstb + 2 * (g + s)), v);
        }
      } else {
        // whole warps write consecutive slots: lane k * P + piece moves one piece (16 bytes if
        // RW is even, else 8) of slot s0 + k, so a store instruction covers whole records of a run
        // (P <= 32: records are at most 256 bytes)
        const bool pairs = (RW & 1) == 0;
        const u32 P = pairs ? RW >> 1 : RW, rpw = 32 / P;
        const u32 k = lane / P, piece = lane - k * P;
        for (u32 s0 = warp * rpw; s0 < cnt; s0 += kSWarps * rpw) {
          const u32 s = s0 + k;
          if (k >= rpw || s >= cnt) continue;
          const u32 sw = slotw[s];
          const u64 g = gbase[sw >> 16];
          if (g == kSkip) continue;
          const u64* sp = stage + (u64)(sw & 0xffffu) * RW;
          u64* d = dstb + (g + s) * RW;
          if (pairs)
            __stcs(reinterpret_cast<ulonglong2*>(d) + piece, reinterpret_cast<const ulonglong2*>(sp)[piece]);
          else
            __stcs(d + piece, sp[piece]);
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------- launchers
size_t scatter_smem_bytes(const Job& j) { return scatter_layout(j.T, j.RW, j.wmax).total; }

// Largest shared memory either level kernel needs for tiles of T records.
size_t level_smem_for(u32 T, u32 RW, u32 KW, u32 wmax) {
  const size_t a = scatter_layout(T, RW, wmax).total, b = hist_smem_bytes_for(T, KW);
  return a > b ? a : b;
}

template <int KW, int RWT, int IT, bool MASKS, int NT>
static cudaError_t launch_scatter_m(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  const size_t sm = scatter_smem_bytes(j);
  if (occ) {
    *occ = occupancy((const void*)k_scatter<KW, RWT, IT, MASKS, NT>, NT, sm);
    return cudaSuccess;
  }
  ensure_smem((const void*)k_scatter<KW, RWT, IT, MASKS, NT>, sm);
  k_scatter<KW, RWT, IT, MASKS, NT><<<grid, NT, sm, s>>>(j, level);
  return cudaGetLastError();
}

template <int KW, int RWT, int IT, int NT = kSThreads>
static cudaError_t launch_scatter_t(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  return scatter_layout(j.T, j.RW, j.wmax).masks ? launch_scatter_m<KW, RWT, IT, true, NT>(j, level, grid, s, occ)
                                                  : launch_scatter_m<KW, RWT, IT, false, NT>(j, level, grid, s, occ);
}

// Record sizes of 8 to 32 bytes at their default tile (T * rec_size = 64 KB at most) have
// instances of their own; every other (size, tile) pair takes the instance for any size.
template <int KW, int IT>
static cudaError_t scatter_rw(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  if constexpr (IT == 16) {
    if (j.RW == 2) return launch_scatter_t<KW, 2, 16>(j, level, grid, s, occ);
  }
  if constexpr (IT == 8) {
    if (j.RW == 3) return launch_scatter_t<KW, 3, 8>(j, level, grid, s, occ);
    if (j.RW == 4) return launch_scatter_t<KW, 4, 8>(j, level, grid, s, occ);
  }
  return launch_scatter_t<KW, 0, IT>(j, level, grid, s, occ);
}

template <int KW>
static cudaError_t scatter_it(const Job& j, int level, u32 grid, cudaStream_t s, int* occ) {
  if constexpr (KW == 1)  // (8-byte records hold 8-byte keys at most)
    if (scatter_threads(j.T, j.RW, j.wmax) == (u32)kSThreadsWide)
      return launch_scatter_t<KW, 1, 4096 / kSThreadsWide, kSThreadsWide>(j, level, grid, s, occ);
  switch (j.T / kSThreads) {
    case 16: return scatter_rw<KW, 16>(j, level, grid, s, occ);
    case 8: return scatter_rw<KW, 8>(j, level, grid, s, occ);
    case 4: return scatter_rw<KW, 4>(j, level, grid, s, occ);
    case 2: return scatter_rw<KW, 2>(j, level, grid, s, occ);
    default: return scatter_rw<KW, 1>(j, level, grid, s, occ);
  }
}

int scatter_ctas_per_sm(const Job& j) {
  int n = 1;
  if (j.KW == 1) scatter_it<1>(j, 0, 0, 0, &n);
  else scatter_it<2>(j, 0, 0, 0, &n);
  return n;
}

int launch_scatter(const Job& j, int level, u32 grid, cudaStream_t s) {
  cudaError_t e = j.KW == 1 ? scatter_it<1>(j, level, grid, s, nullptr) : scatter_it<2>(j, level, grid, s, nullptr);
  return e == cudaSuccess ? 1 : -1;
}

}  // namespace rsg
