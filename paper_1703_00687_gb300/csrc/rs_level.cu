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
//               It counts per lane (a contiguous range of the level's tiles), and the last
//               CTA of a bin also turns every lane's counts into that lane's run starts.
//   k_scatter   (rs_scatter.cu) tile-wise stable scatter, lane by lane: a tile's destinations
//               follow from its lane's run starts and the lane's earlier tiles.
//   k_classify  sub-bin classification, chunk packing (chunks of at most kTinyMax records go
//               to the tiny list), the next level's bin list.
//
// A bin that a sample showed to be mostly one key (kBinDom) is counted and scattered with
// that key's digit split in three (below, equal, above; see bucket_of), and classify
// finishes the equal part at once: heavy keys are not moved again at later levels.
#include "rs_internal.cuh"

namespace rsg {

// Exclusive scan of one u64 per thread (NT threads); returns the exclusive prefix and the
// total in *total.  scratch holds NT / 32 + 1 words.
template <int NT = kThreads>
__device__ inline u64 block_scan_value64(u64 x, u64* scratch, u64* total) {
  constexpr int kW = NT / 32;
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
    u64 w = lane < kW ? scratch[lane] : 0, t = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kW) scratch[lane] = t - w;
    if (lane == kW - 1) scratch[kW] = t;
  }
  __syncthreads();
  u64 r = scratch[warp] + s - x;
  *total = scratch[kW];
  __syncthreads();
  return r;
}

// Tile numbering of bin list L: tile_start = exclusive prefix of ceil(size / T) in list order.
// One CTA of NT threads; each thread takes kItems consecutive bins per round, so that their
// loads are in flight together.
template <int NT = kThreads>
__device__ void finalize_list(const Job& j, int L) {
  constexpr int kItems = 4;
  __shared__ u64 scr[NT / 32 + 1];
  Ctl* ctl = j.ctl;
  u64 nb = *(volatile u64*)&ctl->nbins[L];
  if (nb > j.cap_bins) nb = j.cap_bins;
  Bin* bins = j.bins[L];
  u64 carry = 0;
  for (u64 base = 0; base < nb; base += (u64)NT * kItems) {
    const u64 i0 = base + (u64)threadIdx.x * kItems;
    u64 t[kItems], sum = 0;
#pragma unroll
    for (int q = 0; q < kItems; q++) {
      t[q] = i0 + q < nb ? ceil_div(bins[i0 + q].size, j.T) : 0;
      sum += t[q];
    }
    u64 tot;
    u64 ex = carry + block_scan_value64<NT>(sum, scr, &tot);
#pragma unroll
    for (int q = 0; q < kItems; q++) {
      if (i0 + q < nb) bins[i0 + q].tile_start = ex;
      ex += t[q];
    }
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
    *ctl = c;
    Bin b = {};
    b.begin = 0;
    b.size = j.n;
    b.kand[0] = b.kand[1] = ~0ull;
    b.lo = lo;
    b.W = W;
    j.bins[0][0] = b;
  }
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

// Segmented (batched) start: every segment is a level-0 bin (if large) or a chunk.  Chunk
// slots are reserved with one atomic per warp (batches hold up to millions of small segments).
__global__ void __launch_bounds__(kThreads) k_init_segments(Job j) {
  Ctl* ctl = j.ctl;
  const u32 lane = threadIdx.x & 31;
  for (u64 base = blockIdx.x * (u64)kThreads; base < j.n_segs; base += (u64)gridDim.x * kThreads) {
    const u64 s = base + threadIdx.x;
    u64 a = 0, c = 0;
    bool to_tiny = false, to_chunk = false, to_bin = false;
    if (s < j.n_segs) {
      const u64 e = j.seg_off[s + 1];
      a = j.seg_off[s];
      if (e < a || e > j.n) {  // offsets not non-decreasing within [0, total]: skip, report
        report(ctl, kErrInternal);
      } else if (e > a + 1) {
        c = e - a;
        to_tiny = c <= j.tiny_max;
        to_chunk = !to_tiny && c <= j.chunk_max;
        to_bin = c > j.chunk_max;
      }
    }
    // one slot reservation per warp and list: chunks count up from 0, tiny chunks from the top
    const u32 want = __ballot_sync(kFull, to_chunk), want_t = __ballot_sync(kFull, to_tiny);
    u64 first = 0, first_t = 0;
    if (want) {
      const int leader = __ffs(want) - 1;
      if ((int)lane == leader) first = atomicAdd(&ctl->nchunks, (u64)__popc(want));
      first = __shfl_sync(kFull, first, leader);
    }
    if (want_t) {
      const int leader = __ffs(want_t) - 1;
      if ((int)lane == leader) first_t = atomicAdd(&ctl->ntiny, (u64)__popc(want_t));
      first_t = __shfl_sync(kFull, first_t, leader);
    }
    if (to_chunk || to_tiny) {
      const u64 t = to_tiny ? first_t + __popc(want_t & lanemask_lt()) : first + __popc(want & lanemask_lt());
      if (t >= j.cap_chunks) {
        report(ctl, kErrOverflow);
      } else {
        Chunk ch = {};
        ch.begin = a;
        ch.size = (u32)c;
        j.chunks[to_tiny ? j.cap_chunks - 1 - t : t] = ch;
      }
    }
    if (!to_bin) continue;
    u32 lo, W;
    plan_digit(c, 8 * j.K, j.chunk_max, j.wmax, &lo, &W);
    const u32 nd = 1u << W;
    const u64 idx = atomicAdd(&ctl->nbins[0], 1ull);
    const u64 bo = atomicAdd(&ctl->base_used[0], (u64)nd);
    if (idx >= j.cap_bins || bo + nd > j.cap_base) {
      report(ctl, kErrOverflow);
      continue;
    }
    Bin bn = {};
    bn.begin = a;
    bn.size = c;
    bn.base_off = bo;
    bn.kand[0] = bn.kand[1] = ~0ull;
    bn.lo = lo;
    bn.W = W;
    j.bins[0][idx] = bn;
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
  const u32 nd = 1u << bucket_bits(W, bp->flags);  // buckets (the digit moves, the split stays)
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
  if (s_ret) return;
  // Every lane that holds tiles of the bin (lanes cfirst..clast: its tiles are consecutive) has
  // stored its digit counts in its segment; their sums are the bucket counts.  nd <= 1024:
  // two entries per thread.
  const u64 per = lane_tiles(j.ctl->ntiles[L], j.lanes);
  const u64 ts = bp->tile_start, nt = ceil_div(size, (u64)j.T);
  const u64 cfirst = ts / per, clast = (ts + nt - 1) / per;
  if (clast + b >= j.cap_seg) {  // cannot happen: lanes + bins segments are allocated
    if (threadIdx.x == 0) report(j.ctl, kErrOverflow);
    return;
  }
  const u32 v0 = 2 * threadIdx.x;
  u64 c0 = 0, c1 = 0;
  for (u64 c = cfirst; c <= clast; c++) {
    const u64* sg = j.seg + ((c + b) << j.wmax);
    if (v0 < nd) c0 += __ldcg(sg + v0);
    if (v0 + 1 < nd) c1 += __ldcg(sg + v0 + 1);
  }
  if (mode == 2) {  // the counts themselves
    if (v0 < nd) base[v0] = c0;
    if (v0 + 1 < nd) base[v0 + 1] = c1;
    return;
  }
  u64 tot;
  const u64 ex = block_scan_value64(c0 + c1, scr, &tot);
  if (v0 < nd) base[v0] = ex;
  if (v0 + 1 < nd) base[v0 + 1] = ex + c0;
  if (mode == 1 && threadIdx.x == 0) bp->flags &= ~kBinRedo;
  // Run starts of the scatter: the part of the bin inside lane c writes digit v from
  // bucket base + (records of digit v in the bin's earlier lanes).
  u64 r0 = ex, r1 = ex + c0;
  for (u64 c = cfirst; c <= clast; c++) {
    u64* sg = j.seg + ((c + b) << j.wmax);
    if (v0 < nd) {
      const u64 t = __ldcg(sg + v0);
      sg[v0] = r0;
      r0 += t;
    }
    if (v0 + 1 < nd) {
      const u64 t = __ldcg(sg + v0 + 1);
      sg[v0 + 1] = r1;
      r1 += t;
    }
  }
}



template <int KW>
__global__ void __launch_bounds__(kThreads, 2) k_hist(Job j, int level, int mode) {
  const int L = level & 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0 || call_failed(ctl)) return;
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
  const u64 per = lane_tiles(ntiles, j.lanes);  // one CTA per lane
  const u64 lane_id = blockIdx.x;
  const u64 t0 = lane_id * per;
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
    const u32 nd = 1u << bucket_bits(bb->W, bb->flags);
    const u64 sid = lane_id + b;  // segment of (lane, bin)
    if (sid >= j.cap_seg) {    // cannot happen: lanes + bins segments are allocated
      if (tid == 0) report(ctl, kErrOverflow);
      return;
    }
    u64* sg = j.seg + (sid << j.wmax);
    for (u32 v = tid; v < nd; v += kThreads) {
      u32 h = 0;
#pragma unroll
      for (int c = 0; c < kHistCopies; c++) {
        h += hist[(c << kWMax) + v];
        hist[(c << kWMax) + v] = 0;
      }
      sg[v] = h;  // this lane's counts of the bin (summed when the bin is finished)
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
    bool dom;  // kBinDom: buckets split around the dominant key
  };
  u64 walk = find_bin(bins, nb, t0);
  // locate tile t and start copying its keys into buffer `buf`
  auto issue = [&](u64 t, int buf) {
    while (walk + 1 < nb && bins[walk + 1].tile_start <= t) walk++;
    const Bin* bp = &bins[walk];
    TileRef tr;
    tr.b = walk;
    tr.skip = (mode == 1 && !(bp->flags & kBinRedo)) ? 1u : 0u;
    tr.lo = bp->lo;
    tr.W = bp->W;
    tr.dom = (bp->flags & kBinDom) != 0;
    const u64 tib = t - bp->tile_start;
    const u64 r0 = tib * T;
    tr.cnt = (u32)min((u64)T, bp->size - r0);
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
      auto count = [&](auto&& bucket) {
        for (u32 r = tid; r < tc.cnt; r += kThreads) {
          Key<KW> k;
#pragma unroll
          for (int q = 0; q < KW; q++) k.w[q] = kb[KW * r + q] & j.keymask[q];
          atomicAdd(&my_hist[bucket(k)], 1u);
          if (want_masks) {
#pragma unroll
            for (int q = 0; q < KW; q++) {
              kand[q] &= k.w[q];
              kor[q] |= k.w[q];
            }
          }
        }
      };
      if (!tc.dom) {
        count([&](const Key<KW>& k) { return digit_of<KW>(k, tc.lo, tc.W); });
      } else {  // (rare: a bin that a sample showed to be mostly one key)
        Key<KW> K;
#pragma unroll
        for (int q = 0; q < KW; q++) K.w[q] = bins[tc.b].dom[q];
        const u32 dK = digit_of<KW>(K, tc.lo, tc.W);
        count([&](const Key<KW>& k) { return bucket_of<KW>(k, tc.lo, tc.W, true, K, dK); });
      }
      counted++;
    }
    __syncthreads();  // buffer `buf` is refilled by the next issue
  }
  if (counted) flush(cur);
}

// -------------------------------------------------------------------- classify
// 32 records spread over a sub-bin: their highest differing key bit + 1 (where the sub-bin's
// next digit probably starts; the next histogram pass checks, and moves it), and the key that
// most of them share (of the first and the middle sample), with how many share it.
constexpr u32 kSamples = 32;
constexpr u32 kDomSamples = 16;  // samples sharing one key that make a bin dominated (half)

template <int KW>
__device__ u32 sample_sub_bin(const Job& j, const u64* rec, u64 c, Key<KW>* kdom, u32* ndom) {
  const Key<KW> c0 = load_key<KW>(rec, j), c1 = load_key<KW>(rec + (c * (kSamples / 2) / kSamples) * j.RW, j);
  u64 a[2] = {~0ull, ~0ull}, o[2] = {0, 0};
  u32 n0 = 0, n1 = 0;
#pragma unroll(8 / KW)
  for (u32 i = 0; i < kSamples; i++) {
    const u64 r = (c * (u64)i) / kSamples;
    const Key<KW> k = load_key<KW>(rec + r * j.RW, j);
#pragma unroll
    for (int q = 0; q < KW; q++) {
      a[q] &= k.w[q];
      o[q] |= k.w[q];
    }
    n0 += key_eq<KW>(k, c0);
    n1 += key_eq<KW>(k, c1);
  }
  *kdom = n1 > n0 ? c1 : c0;
  *ndom = n1 > n0 ? n1 : n0;
  return top_bit_plus1(a[0] ^ o[0], KW == 2 ? a[1] ^ o[1] : 0);
}

__device__ void push_pieces(const Job& j, u64 begin, u64 c) {
  Ctl* ctl = j.ctl;
  const u64 np = ceil_div(c, kPieceRecords);
  const u64 idx = atomicAdd(&ctl->npieces, np);
  if (idx + np > j.cap_pieces) {
    report(ctl, kErrOverflow);
    return;
  }
  for (u64 q = 0; q < np; q++) {
    Piece pc;
    pc.begin = begin + q * kPieceRecords;
    pc.size = min(kPieceRecords, c - q * kPieceRecords);
    j.pieces[idx + q] = pc;
  }
}

// Bit sets of sub-bins, 32 to a word.
// First member >= u of a set of nb bits, nb if none.
__device__ __forceinline__ u32 next_member(const u32* m, u32 u, u32 nb) {
  if (u >= nb) return nb;
  const u32 nw = (nb + 31) >> 5;
  u32 w = u >> 5, x = m[w] & (~0u << (u & 31));
  while (x == 0) {
    if (++w >= nw) return nb;
    x = m[w];
  }
  return (w << 5) + __ffs(x) - 1;
}
// Last member <= u (u itself if none is found before word 0 runs out).
__device__ __forceinline__ u32 prev_member(const u32* m, u32 u) {
  u32 w = u >> 5, x = m[w] & ((u & 31) == 31 ? ~0u : (2u << (u & 31)) - 1);
  while (x == 0) {
    if (w == 0) return u;
    x = m[--w];
  }
  return (w << 5) + 31 - __clz(x);
}
// Whether any of [a, b] is a member.
__device__ __forceinline__ bool any_member(const u32* m, u32 a, u32 b) {
  const u32 wa = a >> 5, wb = b >> 5;
  for (u32 w = wa; w <= wb; w++) {
    u32 x = m[w];
    if (w == wa) x &= ~0u << (a & 31);
    if (w == wb) x &= (b & 31) == 31 ? ~0u : (2u << (b & 31)) - 1;
    if (x) return true;
  }
  return false;
}

constexpr int kClsThreads = 256;
constexpr int kClsCtas = 4;  // per SM: a bin is a chain of dependent loads and barriers
constexpr u16 kKeepChunk = 0x8000;
constexpr u16 kTinyChunk = 0x8000;

// Per bin of the level, for every sub-bin v of its digit: empty, one record (finished where
// it is), 2..chunk_max records (sorted on chip), or more (a bin of the next level, whose
// digit is guessed from a sample).  Consecutive sub-bins of at most chunk_max records are
// packed greedily into chunks of at most chunk_max records: a chunk opens at a non-empty
// small sub-bin and takes the following ones while they fit; a large sub-bin closes it.
// The packing runs in parallel: S = inclusive prefix of the sizes (a large sub-bin counts
// chunk_max + 1, so no chunk reaches past it), the chunk opened at v ends at the last e with
// S[e] <= S[v - 1] + chunk_max, and the next chunk opens at the first small sub-bin after e;
// one thread then follows that chain from the first small sub-bin.  A chunk made only of
// single records that are already in `in` is finished and not kept.
template <int KW>
__global__ void __launch_bounds__(kClsThreads, kClsCtas) k_classify(Job j, int level) {
  const int L = level & 1, N = L ^ 1;
  Ctl* ctl = j.ctl;
  const u64 nb = ctl->nbins[L];
  if (nb == 0 || call_failed(ctl)) return;
  const Bin* bins = j.bins[L];
  constexpr u32 kMaxD = 1u << kWMax;
  __shared__ u32 S[kMaxD];              // inclusive prefix of sub-bin sizes
  __shared__ u64 boff[kMaxD];           // first record of sub-bin v within the bin
  __shared__ u16 vlast[kMaxD];          // chunk opened at v: its last non-empty sub-bin
  __shared__ u16 vnext[kMaxD];          // chunk opened at v: where the next opens | kKeepChunk
  __shared__ u16 pk[kMaxD];             // the bin's kept chunks: first sub-bin
  __shared__ u16 pkr[kMaxD];            // ... and its place in its list | kTinyChunk
  __shared__ u32 m12[kMaxD / 32];       // sub-bins of 1..chunk_max records
  __shared__ u32 m2[kMaxD / 32];        // sub-bins of 2..chunk_max records
  __shared__ u32 scr[kClsThreads / 32];
  __shared__ u32 s_npk, s_nn, s_nt;
  __shared__ u64 s_base, s_tbase;
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31;
  const u32 cm = j.chunk_max;
  // Large sub-bins (the next level's bins) first, spread over every warp of the grid: unit u
  // is bin u / 32 and its group u % 32 of 32 sub-bins, one per lane, so that the samples
  // (random reads) of a bin with many large sub-bins are taken by many warps at once.
  {
    const u64 nw = (u64)gridDim.x * (kClsThreads / 32);
    for (u64 u = (u64)blockIdx.x * (kClsThreads / 32) + (tid >> 5); u < nb * 32; u += nw) {
      const Bin& bin = bins[u >> 5];
      const u32 flags = bin.flags, W = bin.W;
      const u32 nd = 1u << bucket_bits(W, flags), v = (u32)(u & 31) * 32 + lane;
      if ((flags & kBinEqual) || v >= nd) continue;
      const u64 size = bin.size;
      const u64* bbase = j.base[L] + bin.base_off;
      const u64 bv = bbase[v], next = v + 1 < nd ? bbase[v + 1] : size;
      if (next < bv || next > size || next - bv <= cm) continue;  // (inconsistent bases: reported below)
      u32 vdom = nd;  // a dominated bin's own key bucket is finished in the packing loop
      if (flags & kBinDom) {
        Key<KW> K;
#pragma unroll
        for (int q = 0; q < KW; q++) K.w[q] = bin.dom[q];
        vdom = digit_of<KW>(K, bin.lo, W) + 1;
      }
      if (v == vdom) continue;
      const u64 c = next - bv, rb = bin.begin + bv;
      const u32 p1 = bin.parity ^ 1, blo = bin.lo;
      // every key bit >= bin.lo is shared by the sub-bin; guess where its next digit starts
      // from a sample, and whether one key holds most of it
      Key<KW> K2;
      u32 ndom;
      u32 p = sample_sub_bin<KW>(j, j.buf[p1] + rb * j.RW, c, &K2, &ndom);
      if (p == 0 || p > blo) p = blo;
      if (p == 0) p = 1;
      u32 nlo, nW;
      plan_digit(c, p, cm, j.wmax, &nlo, &nW);
      // a dominated bin takes one digit bit less, so its 2^(W+1) buckets need no more room
      // than a plain bin's (the other keys are at most half of it)
      const bool dom2 = ndom >= kDomSamples && nW >= 2;
      if (dom2) {
        nW -= 1;
        nlo += 1;
      }
      const u32 nnd = 1u << bucket_bits(nW, dom2 ? kBinDom : 0u);
      const u64 idx = atomicAdd(&ctl->nbins[N], 1ull);
      const u64 bo = atomicAdd(&ctl->base_used[N], (u64)nnd);
      if (idx >= j.cap_bins || bo + nnd > j.cap_base) {
        report(ctl, kErrOverflow);
        continue;
      }
      Bin nbn = {};
      nbn.begin = rb;
      nbn.size = c;
      nbn.base_off = bo;
      nbn.kand[0] = nbn.kand[1] = ~0ull;
      nbn.lo = nlo;
      nbn.W = nW;
      nbn.parity = p1;
      if (dom2) {
        nbn.flags = kBinDom;
#pragma unroll
        for (int q = 0; q < KW; q++) nbn.dom[q] = K2.w[q];
      }
      j.bins[N][idx] = nbn;
    }
  }
  // Then, per bin, the small sub-bins: finished records and chunk packing.
  for (u64 b = blockIdx.x; b < nb; b += gridDim.x) {
    const Bin bin = bins[b];
    if (bin.flags & kBinEqual) {  // finished without moving; copy back if it lives in tmp
      if (tid == 0 && bin.parity) push_pieces(j, bin.begin, bin.size);
      continue;
    }
    const u32 nd = 1u << bucket_bits(bin.W, bin.flags);
    const u32 p1 = bin.parity ^ 1;
    const u64* bbase = j.base[L] + bin.base_off;
    const bool dom = (bin.flags & kBinDom) != 0;
    u32 vdom = nd;  // the dominant key's bucket: finished here
    if (dom) {
      Key<KW> K;
#pragma unroll
      for (int q = 0; q < KW; q++) K.w[q] = bin.dom[q];
      vdom = digit_of<KW>(K, bin.lo, bin.W) + 1;
    }
    for (u32 v0 = tid & ~31u; v0 < nd; v0 += kClsThreads) {
      const u32 v = v0 + lane;
      u32 k = 0;
      if (v < nd) {
        u64 bv = bbase[v];
        u64 next = v + 1 < nd ? bbase[v + 1] : bin.size;
        if (next < bv || next > bin.size) {  // inconsistent bases (only after a reported error)
          report(ctl, kErrInternal);
          next = bv = min(bv, bin.size);
        }
        const u64 c = next - bv;
        boff[v] = bv;
        k = c == 0 ? 0 : c == 1 ? 1 : c <= cm ? 2 : 3;
        S[v] = k == 3 ? cm + 1 : (u32)c;
        if (v == vdom) {  // all the dominant key: finished (copied back if it lives in tmp); no
          k = 0;          // chunk may reach across it
          S[v] = c ? cm + 1 : 0;
          if (c && p1) push_pieces(j, bin.begin + bv, c);
        }
      }
      const u32 small = __ballot_sync(kFull, k == 1 || k == 2), multi = __ballot_sync(kFull, k == 2);
      if (lane == 0) {
        m12[v0 >> 5] = small;
        m2[v0 >> 5] = multi;
      }
    }
    __syncthreads();
    {  // S: sizes -> inclusive prefix (at most 2^kWMax * (chunk_max + 1), well inside u32)
      const u32 ipt = (nd + kClsThreads - 1) / kClsThreads, v0 = tid * ipt;
      u32 own = 0;
      for (u32 q = 0; q < ipt; q++)
        if (v0 + q < nd) own += S[v0 + q];
      u32 run = block_exclusive_sum<kClsThreads>(own, scr);  // ends with a barrier
      for (u32 q = 0; q < ipt; q++)
        if (v0 + q < nd) S[v0 + q] = run += S[v0 + q];
    }
    __syncthreads();
    for (u32 v = tid; v < nd; v += kClsThreads) {
      if (!(m12[v >> 5] >> (v & 31) & 1u)) continue;
      const u32 lim = (v ? S[v - 1] : 0) + cm;
      u32 lo = v, hi = nd;  // S[lo] <= lim (a small sub-bin fits alone), S[hi] > lim or hi = nd
      while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (S[mid] <= lim) lo = mid; else hi = mid;
      }
      const u32 vl = prev_member(m12, lo);
      const bool keep = p1 || any_member(m2, v, vl);
      vlast[v] = (u16)vl;
      vnext[v] = (u16)(next_member(m12, lo + 1, nd) | (keep ? kKeepChunk : 0u));
    }
    __syncthreads();
    if (tid == 0) {  // (chunks of at most j.tiny_max records go to the tiny list)
      u32 npk = 0, nn = 0, nt = 0;
      for (u32 v = next_member(m12, 0, nd); v < nd;) {
        const u32 x = vnext[v];
        if (x & kKeepChunk) {
          const u32 size = S[vlast[v]] - (v ? S[v - 1] : 0);
          pk[npk] = (u16)v;
          pkr[npk++] = (u16)(size <= j.tiny_max ? (nt++ | kTinyChunk) : nn++);
        }
        const u32 w = x & ~(u32)kKeepChunk;
        v = w > v ? w : nd;
      }
      s_npk = npk;
      s_nn = nn;
      s_nt = nt;
      s_base = nn ? atomicAdd(&ctl->nchunks, (u64)nn) : 0;
      s_tbase = nt ? atomicAdd(&ctl->ntiny, (u64)nt) : 0;
    }
    __syncthreads();
    {
      const u32 npk = s_npk;
      const u64 base = s_base, tbase = s_tbase;
      const bool ok = base + s_nn <= j.cap_chunks, ok_t = tbase + s_nt <= j.cap_chunks;
      if (tid == 0 && !(ok && ok_t)) report(ctl, kErrOverflow);
      for (u32 q = tid; q < npk; q += kClsThreads) {
        const u32 vf = pk[q], vl = vlast[vf], r = pkr[q];
        const bool tiny = (r & kTinyChunk) != 0;
        if (tiny ? !ok_t : !ok) continue;
        Chunk ch = {};
        ch.begin = bin.begin + boff[vf];
        ch.size = S[vl] - (vf ? S[vf - 1] : 0);
        ch.flags = (p1 ? kChSrcTmp : 0u) | (any_member(m2, vf, vl) ? 0u : kChCopyOnly);
        // one sub-bin shares every bit >= lo; several differ in the digit itself (the bucket
        // numbers of a dominated bin are not key bits: its chunks find their shared bits)
        if (!dom) {
          ch.p = bin.lo;
          ch.pw = (u16)bin.W;
          ch.v0 = vf;
          u32 sb = 0;
          while ((1u << sb) < vl - vf + 1) sb++;
          ch.sb = (u16)(vl == vf ? 0 : sb);
        }
        const u32 rank = r & ~(u32)kTinyChunk;
        j.chunks[tiny ? j.cap_chunks - 1 - (tbase + rank) : base + rank] = ch;
      }
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
    finalize_list<kClsThreads>(j, N);
    if (tid == 0) {
      ctl->cls_done = 0;
      ctl->nredo = 0;
      ctl->nbins[L] = 0;
      ctl->ntiles[L] = 0;
      ctl->base_used[L] = 0;
      __threadfence();
    }
  }
}

// Histogram entry point: copy the raw counts (u64) of bin 0 out.
__global__ void k_read_counts(Job j, u64* out, u32 nd) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < nd; v += gridDim.x * blockDim.x) out[v] = j.base[0][v];
}

// ------------------------------------------------------------------- launchers
static size_t hist_smem(const Job& j) { return hist_smem_bytes_for(j.T, j.KW); }

int hist_ctas_per_sm(const Job& j) {
  int n = 0;
  const size_t sm = hist_smem(j);
  if (j.KW == 1) {
    n = occupancy((const void*)k_hist<1>, kThreads, sm);
  } else {
    n = occupancy((const void*)k_hist<2>, kThreads, sm);
  }
  return n < 1 ? 1 : n;
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

int launch_hist(const Job& j, int level, int mode, cudaStream_t s) {
  const size_t sm = hist_smem(j);
  const u32 grid = j.lanes;  // one CTA per lane (the scatter pass uses the same lanes)
  if (j.KW == 1) {
    ensure_smem((const void*)k_hist<1>, sm);
    k_hist<1><<<grid, kThreads, sm, s>>>(j, level, mode);
  } else {
    ensure_smem((const void*)k_hist<2>, sm);
    k_hist<2><<<grid, kThreads, sm, s>>>(j, level, mode);
  }
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int classify_ctas_per_sm() { return kClsCtas; }

int launch_classify(const Job& j, int level, u32 grid, cudaStream_t s) {
  if (j.KW == 1) k_classify<1><<<grid, kClsThreads, 0, s>>>(j, level);
  else k_classify<2><<<grid, kClsThreads, 0, s>>>(j, level);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_read_counts(const Job& j, u64* d_counts, u32 W, cudaStream_t s) {
  const u32 nd = 1u << W;
  k_read_counts<<<(nd + 255) / 256, 256, 0, s>>>(j, d_counts, nd);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace rsg
