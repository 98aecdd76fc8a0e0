// Run-length counting of equal keys in sorted records: the step that follows the sort when
// it serves k-mer counting (KMC3, the application of Kokot et al., section 4): every distinct
// key once, with the number of records that carry it.
//
//   k_runs_tiles   per tile of kRTile records: how many runs start in it (a run starts at
//                  record 0 and wherever the key differs from the previous record's)
//   k_runs_scan    exclusive scan of the tile counts (one CTA), and the number of runs
//   k_runs_write   per tile: the first record of every run that starts in it goes to
//                  out[run], the index of that record to counts[run]
//   k_runs_len     counts[run] = start of the next run - start of this one (in place)
#include "rs_internal.cuh"

namespace rsg {

constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr u32 kRRange = 4096;                  // runs per range of k_runs_len
constexpr u32 kRItems = 16;                    // rounds of 32 records per warp and tile
constexpr u32 kRTile = kRThreads * kRItems;    // records per tile (warp w: records [w*512, w*512+512))

template <int KW>
__device__ __forceinline__ Key<KW> run_key(const u64* recs, u64 i, u32 RW, u64 km0, u64 km1) {
  Key<KW> k;
  k.w[0] = recs[i * RW] & km0;
  if (KW == 2) k.w[KW - 1] = recs[i * RW + 1] & km1;
  return k;
}

// One round of a warp over records [r, r + 32) (lane l: record r + l, coalesced): which lanes
// start a run.  prev = key of record r - 1 (any value when r == 0), passed round to round.
template <int KW>
__device__ __forceinline__ u32 run_start_mask(const u64* recs, u64 n, u64 r, u32 RW, u64 km0, u64 km1,
                                              Key<KW>& prev) {
  const u32 lane = threadIdx.x & 31;
  const u64 i = r + lane;
  Key<KW> k = prev;
  if (i < n) k = run_key<KW>(recs, i, RW, km0, km1);
  Key<KW> before;
#pragma unroll
  for (int q = 0; q < KW; q++) {
    before.w[q] = __shfl_up_sync(kFull, k.w[q], 1);
    if (lane == 0) before.w[q] = prev.w[q];
    prev.w[q] = __shfl_sync(kFull, k.w[q], 31);
  }
  return __ballot_sync(kFull, i < n && (i == 0 || !key_eq<KW>(k, before)));
}

// Runs starting in the warp's part of a tile (records [r0, r0 + 32 * kRItems)).
template <int KW>
__device__ __forceinline__ u32 warp_run_starts(const u64* recs, u64 n, u64 r0, u32 RW, u64 km0, u64 km1) {
  Key<KW> prev = {};
  if (r0 > 0 && r0 - 1 < n) prev = run_key<KW>(recs, r0 - 1, RW, km0, km1);
  u32 c = 0;
  for (u32 it = 0; it < kRItems; it++) c += __popc(run_start_mask<KW>(recs, n, r0 + 32 * it, RW, km0, km1, prev));
  return c;
}

template <int KW>
__global__ void __launch_bounds__(kRThreads) k_runs_tiles(const u64* recs, u64 n, u32 RW, u64 km0, u64 km1,
                                                          u32* tile_cnt, u64 ntiles) {
  __shared__ u32 scr[kRWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (u64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 r0 = tile * kRTile + (u64)warp * 32 * kRItems;
    const u32 c = warp_run_starts<KW>(recs, n, r0, RW, km0, km1);
    if (lane == 0) scr[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 t = 0;
      for (int w = 0; w < kRWarps; w++) t += scr[w];
      tile_cnt[tile] = t;
    }
    __syncthreads();
  }
}

// One CTA of 1,024 threads: tile_off[t] = runs starting before tile t; *nruns = all runs.
__global__ void __launch_bounds__(1024) k_runs_scan(const u32* tile_cnt, u64 ntiles, u64* tile_off, u64* nruns) {
  __shared__ u64 scr[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 carry = 0;
  for (u64 base = 0; base < ntiles; base += 1024) {
    const u64 t = base + threadIdx.x;
    const u64 x = t < ntiles ? tile_cnt[t] : 0;
    u64 incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) scr[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const u64 v = scr[lane];
      u64 s = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += y;
      }
      scr[lane] = s - v;
      if (lane == 31) scr[32] = s;
    }
    __syncthreads();
    if (t < ntiles) tile_off[t] = carry + scr[warp] + incl - x;
    carry += scr[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) *nruns = carry;
}


// Per tile: the first record of every run that starts in it goes to out[run]; counts[run]
// receives the index of that record (turned into lengths by k_runs_len), and the start of
// every kRRange-th run also goes to bound[run / kRRange].
template <int KW>
__global__ void __launch_bounds__(kRThreads) k_runs_write(const u64* recs, u64 n, u32 RW, u64 km0, u64 km1,
                                                          const u64* tile_off, u64 ntiles, u64* out, u64* counts,
                                                          u64* bound) {
  __shared__ u32 scr[kRWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 ltmask = lanemask_lt();
  for (u64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 r0 = tile * kRTile + (u64)warp * 32 * kRItems;
    // runs starting in the warps before this one, then this warp's rounds in order
    const u32 mine = warp_run_starts<KW>(recs, n, r0, RW, km0, km1);
    if (lane == 0) scr[warp] = mine;
    __syncthreads();
    u64 p = tile_off[tile];
    for (int w = 0; w < warp; w++) p += scr[w];
    __syncthreads();  // scr is reused by the next tile
    if (mine == 0) continue;
    Key<KW> prev = {};
    if (r0 > 0 && r0 - 1 < n) prev = run_key<KW>(recs, r0 - 1, RW, km0, km1);
    for (u32 it = 0; it < kRItems; it++) {
      const u64 r = r0 + 32 * it;
      const u32 m = run_start_mask<KW>(recs, n, r, RW, km0, km1, prev);
      if (m >> lane & 1u) {
        const u64 q = p + __popc(m & ltmask), i = r + lane;
        for (u32 w = 0; w < RW; w++) out[q * RW + w] = recs[i * RW + w];
        counts[q] = i;
        if (q % kRRange == 0) bound[q / kRRange] = i;
      }
      p += __popc(m);
    }
  }
}

// counts[p] = start(p + 1) - start(p) for every run, start(nruns) = n.  A CTA reads its whole
// range of starts before writing any length; the start after its range comes from bound[],
// which no CTA writes here, so the in-place update has no race.
__global__ void __launch_bounds__(kRThreads) k_runs_len(u64* counts, const u64* bound, const u64* nruns_p, u64 n) {
  __shared__ u64 st[kRRange];
  const u64 nruns = *nruns_p;
  const u64 nranges = (nruns + kRRange - 1) / kRRange;
  for (u64 r = blockIdx.x; r < nranges; r += gridDim.x) {
    const u64 p0 = r * kRRange, p1 = min(nruns, p0 + kRRange);
    for (u64 p = p0 + threadIdx.x; p < p1; p += kRThreads) st[p - p0] = counts[p];
    __syncthreads();
    const u64 after = p1 < nruns ? bound[p1 / kRRange] : n;
    for (u64 p = p0 + threadIdx.x; p < p1; p += kRThreads)
      counts[p] = (p + 1 < p1 ? st[p + 1 - p0] : after) - st[p - p0];
    __syncthreads();
  }
}

// host side ------------------------------------------------------------------------------
u64 runs_tiles(u64 n) { return (n + kRTile - 1) / kRTile; }
u64 runs_bounds(u64 n) { return n / kRRange + 2; }

int launch_count_runs(const u64* recs, u64 n, u32 RW, u32 KW, u64 km0, u64 km1, u32* tile_cnt, u64* tile_off,
                      u64* bound, u64* out, u64* counts, u64* nruns, u32 grid, cudaStream_t s) {
  const u64 ntiles = runs_tiles(n);
  if (KW == 1) k_runs_tiles<1><<<grid, kRThreads, 0, s>>>(recs, n, RW, km0, km1, tile_cnt, ntiles);
  else k_runs_tiles<2><<<grid, kRThreads, 0, s>>>(recs, n, RW, km0, km1, tile_cnt, ntiles);
  k_runs_scan<<<1, 1024, 0, s>>>(tile_cnt, ntiles, tile_off, nruns);
  if (KW == 1) k_runs_write<1><<<grid, kRThreads, 0, s>>>(recs, n, RW, km0, km1, tile_off, ntiles, out, counts, bound);
  else k_runs_write<2><<<grid, kRThreads, 0, s>>>(recs, n, RW, km0, km1, tile_off, ntiles, out, counts, bound);
  k_runs_len<<<grid, kRThreads, 0, s>>>(counts, bound, nruns, n);
  return cudaGetLastError() == cudaSuccess ? 4 : -1;
}

}  // namespace rsg
