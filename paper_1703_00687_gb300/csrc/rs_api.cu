// C ABI of the sorter: argument validation, the per-(device, stream) workspace, and the
// host driver that launches the levels of the MSD radix sort (Kokot et al., section 3.1).
//
// The driver never reads device memory: it launches a fixed sequence of kernels per level
// and every kernel reads the amount of work left for it from the device control block,
// returning at once when there is none.  A level uses a digit of at least kWMin bits that
// starts at the bin's highest differing key bit, so a key of key_size bytes needs at most
// key_size levels.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <algorithm>
#include <vector>

#include "radix_gb300.h"
#include "rs_internal.cuh"

namespace rsg {

u32 chunk_capacity(u32 RW);
u64 runs_tiles(u64 n);
u64 runs_bounds(u64 n);
int launch_count_runs(const u64* recs, u64 n, u32 RW, u32 KW, u64 km0, u64 km1, u32* tile_cnt, u64* tile_off,
                      u64* bound, u64* out, u64* counts, u64* nruns, u32 grid, cudaStream_t s);
size_t level_smem_for(u32 T, u32 RW, u32 KW, u32 wmax);
constexpr size_t kMaxSmemPerCta = 227 * 1024;

struct Workspace {
  void* mem = nullptr;
  size_t bytes = 0;
  Ctl* ctl = nullptr;
};

static std::mutex g_mu;
static std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;
static rs_plan g_plan = {0, 0, 0, 0, 0, 0, 0};
static std::atomic<unsigned long long> g_launches{0};
static std::map<int, int> g_sms;
static std::atomic<unsigned> g_inject{0};

static std::mutex g_sms_mu;

// kernel attribute and occupancy caches (keyed by device and kernel)
static std::mutex g_attr_mu;
static std::map<std::pair<int, const void*>, size_t> g_smem_set;
static std::map<std::tuple<int, const void*, int, size_t>, int> g_occ;

static int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  return dev;
}

void ensure_smem(const void* fn, size_t smem) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mu);
  size_t& have = g_smem_set[std::make_pair(dev, fn)];
  if (smem > have) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) have = smem;
    else cudaGetLastError();  // (the launch then reports the error)
  }
}

int occupancy(const void* fn, int threads, size_t smem) {
  ensure_smem(fn, smem);
  const int dev = current_device();
  const auto key = std::make_tuple(dev, fn, threads, smem);
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  std::lock_guard<std::mutex> lk(g_attr_mu);
  g_occ[key] = n;
  return n;
}

static int sm_count(int dev) {
  std::lock_guard<std::mutex> lk(g_sms_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  g_sms[dev] = n;
  return n;
}

// Sizes of every workspace region for a job.
struct Caps {
  u64 bins, base, seg, chunks, pieces;
  size_t bytes;
  size_t off_ctl, off_bins0, off_bins1, off_base0, off_base1, off_seg, off_chunks, off_pieces;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static Caps caps_for(u64 n, u32 cm, u32 wmax, u64 n_segs) {
  Caps c;
  c.bins = n / ((u64)cm + 1) + 2;  // large bins of one level (each holds > cm records)
  c.base = 256ull * c.bins + 2 * (n / cm) + (1ull << wmax) + 64;
  c.seg = kMaxLanes + c.bins;       // (lane, bin) segments of one level
  c.chunks = 6 * (n / cm) + n_segs + 16;
  c.pieces = n / kPieceRecords + n / ((u64)cm + 1) + 16;
  size_t o = 0;
  c.off_ctl = o; o = al(o + sizeof(Ctl));
  c.off_bins0 = o; o = al(o + c.bins * sizeof(Bin));
  c.off_bins1 = o; o = al(o + c.bins * sizeof(Bin));
  c.off_base0 = o; o = al(o + c.base * 8);
  c.off_base1 = o; o = al(o + c.base * 8);
  c.off_seg = o; o = al(o + (c.seg << wmax) * 8);
  c.off_chunks = o; o = al(o + c.chunks * sizeof(Chunk));
  c.off_pieces = o; o = al(o + c.pieces * sizeof(Piece));
  c.bytes = o;
  return c;
}

// Tile size, on-chip limit and digit width of a job under a plan.
struct Shape {
  u32 T, chunk_max, wmax;
};

static Shape shape_for(u64 n, u32 rec_size, u32 key_size, const rs_plan& p) {
  Shape sh;
  const u32 cap = chunk_capacity(rec_size / 8);
  sh.chunk_max = p.chunk_records && p.chunk_records < cap ? p.chunk_records : cap;
  // widest digit a level may use (it sizes the per-digit tables; each bin's digit is chosen by
  // plan_digit: as few levels as possible, then the narrowest digit for them).  By default 9
  // bits, or 10 when that saves a level for the whole input.
  if (p.digit_bits_max) {
    sh.wmax = p.digit_bits_max;
  } else {
    u32 need = 0;
    while (need < 63 && (n >> need) > sh.chunk_max) need++;
    sh.wmax = (need + 9) / 10 < (need + 8) / 9 ? 10 : 9;
  }
  u32 T = 4096;  // 64 KB of 16-byte records per tile (measured best of 1024..4096)
  while (T > 256 && (u64)T * rec_size > 65536) T >>= 1;
  if (p.tile_records) T = p.tile_records;
  // a planned tile too large for one CTA's shared memory is halved until it fits
  const u32 KW = key_size > 8 ? 2 : 1;
  while (T > 256 && level_smem_for(T, rec_size / 8, KW, sh.wmax) > kMaxSmemPerCta) T >>= 1;
  sh.T = T;
  return sh;
}

static rs_plan current_plan() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_plan;
}

static rs_status get_workspace(int dev, cudaStream_t s, size_t bytes, Workspace** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace& w = g_ws[std::make_pair(dev, s)];
  if (w.bytes < bytes) {
    u32 err_keep = 0;
    if (w.mem) {
      // keep the sticky error bits of earlier calls on this stream
      if (cudaStreamSynchronize(s) != cudaSuccess) return RS_ERR_CUDA;
      cudaMemcpy(&err_keep, &w.ctl->err, sizeof(u32), cudaMemcpyDeviceToHost);
      cudaFree(w.mem);
      w.mem = nullptr;
      w.bytes = 0;
    }
    size_t want = bytes + bytes / 4;  // head room so that slightly larger calls reuse it
    void* m = nullptr;
    if (cudaMalloc(&m, want) != cudaSuccess) {
      cudaGetLastError();
      want = bytes;
      if (cudaMalloc(&m, want) != cudaSuccess) {
        cudaGetLastError();
        return RS_ERR_NO_MEMORY;
      }
    }
    if (cudaMemset(m, 0, sizeof(Ctl)) != cudaSuccess) return RS_ERR_CUDA;
    w.mem = m;
    w.bytes = want;
    w.ctl = (Ctl*)m;
    if (err_keep) cudaMemcpy(&w.ctl->err, &err_keep, sizeof(u32), cudaMemcpyHostToDevice);
  }
  *out = &w;
  return RS_OK;
}

// Tile ranges of a level: as many as histogram or scatter CTAs fit on the GPU at once,
// whichever is more (every scatter CTA needs a lane of its own; histogram CTAs beyond the
// resident ones simply run in a second wave).
static u32 lanes_for(const Job& j, int sms) {
  const int per_sm = std::max(hist_ctas_per_sm(j), scatter_ctas_per_sm(j));
  const u64 l = (u64)sms * (u64)per_sm;
  return (u32)(l < 1 ? 1 : l > kMaxLanes ? kMaxLanes : l);
}

struct Setup {
  Job j;
  Caps c;
  int dev;
  int sms;
};

static rs_status validate_layout(uint32_t rec_size, uint32_t key_size) {
  if (rec_size == 0 || rec_size % 8 != 0 || rec_size > 256) return RS_ERR_INVALID_ARG;
  if (key_size == 0 || key_size > rec_size) return RS_ERR_INVALID_ARG;
  if (key_size > 16) return RS_ERR_UNSUPPORTED;
  return RS_OK;
}

static bool overlap(const void* a, const void* b, u64 bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

static rs_status validate_buffers(const void* a, const void* b, u64 n, uint32_t rec_size) {
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  const u64 bytes = n * rec_size;
  if (bytes > (u64)UINTPTR_MAX / 2) return RS_ERR_TOO_LARGE;
  if (!a || !b) return RS_ERR_INVALID_ARG;
  if ((((uintptr_t)a) | ((uintptr_t)b)) & 15) return RS_ERR_MISALIGNED;
  if (overlap(a, b, bytes)) return RS_ERR_OVERLAP;
  return RS_OK;
}

static rs_status check_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return RS_ERR_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return RS_ERR_INVALID_ARG;
  return RS_OK;
}

static rs_status setup_job(void* in, void* tmp, u64 n, u32 rec_size, u32 key_size, u64 n_segs,
                           cudaStream_t stream, Setup* st) {
  if (check_device_ptr(in) != RS_OK || check_device_ptr(tmp) != RS_OK) return RS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  Job& j = st->j;
  memset(&j, 0, sizeof j);
  j.buf[0] = (u64*)in;
  j.buf[1] = (u64*)tmp;
  j.n = n;
  j.RW = rec_size / 8;
  j.K = key_size;
  j.KW = key_size > 8 ? 2 : 1;
  for (u32 w = 0; w < 2; w++) {
    const int bytes = (int)key_size - 8 * (int)w;
    j.keymask[w] = bytes >= 8 ? ~0ull : bytes <= 0 ? 0ull : ((1ull << (8 * bytes)) - 1);
  }
  const rs_plan p = current_plan();
  const Shape sh = shape_for(n, rec_size, key_size, p);
  j.wmax = sh.wmax;
  j.T = sh.T;
  j.chunk_max = sh.chunk_max;
  j.inject = g_inject.exchange(0);
  j.wd_polls = p.watchdog_polls ? p.watchdog_polls : kWaitPolls;
  j.tiny_max = p.tiny_records ? p.tiny_records : kTinyMax;
  j.es_max = p.enum_records ? p.enum_records : kEsDefault;
  j.n_segs = n_segs;
  int sms = sm_count(dev);
  if (p.sm_limit && (int)p.sm_limit < sms) sms = (int)p.sm_limit;
  j.lanes = lanes_for(j, sms);
  Caps c = caps_for(n, j.chunk_max, j.wmax, n_segs);
  Workspace* w = nullptr;
  rs_status r = get_workspace(dev, stream, c.bytes, &w);
  if (r != RS_OK) return r;
  char* base = (char*)w->mem;
  j.ctl = (Ctl*)(base + c.off_ctl);
  j.bins[0] = (Bin*)(base + c.off_bins0);
  j.bins[1] = (Bin*)(base + c.off_bins1);
  j.cap_bins = c.bins;
  j.base[0] = (u64*)(base + c.off_base0);
  j.base[1] = (u64*)(base + c.off_base1);
  j.cap_base = c.base;
  j.seg = (u64*)(base + c.off_seg);
  j.cap_seg = c.seg;
  j.chunks = (Chunk*)(base + c.off_chunks);
  j.cap_chunks = c.chunks;
  j.pieces = (Piece*)(base + c.off_pieces);
  j.cap_pieces = c.pieces;
  st->c = c;
  st->dev = dev;
  st->sms = sms;
  return RS_OK;
}

static void count(int k) {
  if (k > 0) g_launches += (unsigned long long)k;
}

// Optional per-launch timing: CUDA events recorded on the launching stream around each
// kernel of the sort (enabled by radix_sort_profile).
struct ProfRec {
  cudaEvent_t a, b;
  u32 kernel, level;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static uint32_t g_prof_mask = ~0u;  // kernels (bit RS_K_*) that get events while profiling
static std::vector<ProfRec> g_prof;     // records of this profiling session
static std::vector<cudaEvent_t> g_evpool;
static size_t g_evnext = 0;

static cudaEvent_t prof_event() {
  if (g_evnext == g_evpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_evpool.push_back(e);
  }
  return g_evpool[g_evnext++];
}

template <typename F>
static int timed(u32 kernel, u32 level, cudaStream_t s, F&& launch) {
  ProfRec r = {nullptr, nullptr, kernel, level};
  bool on;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    on = g_prof_on && ((g_prof_mask >> kernel) & 1u);
    if (on) {
      r.a = prof_event();
      r.b = prof_event();
      on = r.a && r.b;
    }
  }
  if (on) cudaEventRecord(r.a, s);
  const int k = launch();
  if (on) {
    cudaEventRecord(r.b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(r);
  }
  count(k);
  return k;
}

// Levels 0..K-1 of distribution passes, then the on-chip sorts and the copy-back.
// levels = 0 when no bin can exceed the on-chip limit (then only chunks exist).
static rs_status run_levels(const Setup& st, cudaStream_t s, bool levels_needed = true) {
  const Job& j = st.j;
  const u32 gs = (u32)st.sms * (u32)scatter_ctas_per_sm(j);
  const u32 gc = (u32)st.sms * (u32)classify_ctas_per_sm();
  const int levels = levels_needed ? (int)j.K : 0;  // each level consumes >= 8 key bits
  for (int lv = 0; lv < levels; lv++) {
    if (timed(RS_K_HIST, lv, s, [&] { return launch_hist(j, lv, 0, s); }) < 0) return RS_ERR_CUDA;
    if (timed(RS_K_HIST_REDO, lv, s, [&] { return launch_hist(j, lv, 1, s); }) < 0) return RS_ERR_CUDA;
    if (timed(RS_K_SCATTER, lv, s, [&] { return launch_scatter(j, lv, gs, s); }) < 0) return RS_ERR_CUDA;
    if (timed(RS_K_CLASSIFY, lv, s, [&] { return launch_classify(j, lv, gc, s); }) < 0) return RS_ERR_CUDA;
  }
  const u32 gch = (u32)st.sms * (u32)chunk_ctas_per_sm(j);
  if (timed(RS_K_CHUNK, levels, s, [&] { return launch_chunks(j, gch, s); }) < 0) return RS_ERR_CUDA;
  if (timed(RS_K_TINY, levels, s, [&] { return launch_tiny(j, (u32)st.sms, s); }) < 0) return RS_ERR_CUDA;
  if (levels == 0) return RS_OK;  // (ranges left in tmp come from the levels only)
  if (timed(RS_K_COPY, levels, s, [&] { return launch_copy(j, (u32)st.sms * 2, s); }) < 0) return RS_ERR_CUDA;
  return RS_OK;
}

// ------------------------------------------------------------- no-allocation variant
// Workspace of radix_sort_noalloc: a fixed array in device memory.  CUDA loads the module
// that holds it on a device when it is first needed there (lazy loading: the first
// radix_sort_noalloc call on that device, whose address look-up loads it), or with the other
// modules when lazy loading is off; from then on the device holds the array until the
// process exits.  Its size bounds the sorts that entry point accepts (see noalloc_setup).
constexpr size_t kNoAllocBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_na_mu;
static void* g_na_ptr[kNoAllocMaxDevices];  // device address of g_noalloc_ws, per device

// The array's address on the current device.  In host code g_noalloc_ws names a host-side
// stand-in, not device memory, so the address is looked up once per device (with that device
// current) and kept.
static rs_status noalloc_address(int dev, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return RS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      // (under lazy module loading this first look-up is what loads the array's module and
      // reserves its memory on the device, so it can fail for lack of memory)
      return e == cudaErrorMemoryAllocation ? RS_ERR_NO_MEMORY : RS_ERR_CUDA;
    }
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return RS_OK;
}

// The job of radix_sort_noalloc: the same plan as radix_sort, its workspace carved from the
// fixed array.  RS_ERR_TOO_LARGE when that workspace would not fit.
static rs_status noalloc_setup(void* in, void* tmp, u64 n, u32 rec_size, u32 key_size, Setup* st) {
  Job& j = st->j;
  memset(&j, 0, sizeof j);
  j.buf[0] = (u64*)in;
  j.buf[1] = (u64*)tmp;
  j.n = n;
  j.RW = rec_size / 8;
  j.K = key_size;
  j.KW = key_size > 8 ? 2 : 1;
  for (u32 w = 0; w < 2; w++) {
    const int bytes = (int)key_size - 8 * (int)w;
    j.keymask[w] = bytes >= 8 ? ~0ull : bytes <= 0 ? 0ull : ((1ull << (8 * bytes)) - 1);
  }
  const rs_plan p = current_plan();
  const Shape sh = shape_for(n, rec_size, key_size, p);
  j.wmax = sh.wmax;
  j.T = sh.T;
  j.chunk_max = sh.chunk_max;
  j.wd_polls = p.watchdog_polls ? p.watchdog_polls : kWaitPolls;
  j.tiny_max = p.tiny_records ? p.tiny_records : kTinyMax;
  j.es_max = p.enum_records ? p.enum_records : kEsDefault;
  const Caps c = caps_for(n, j.chunk_max, j.wmax, 0);
  if (c.bytes > kNoAllocBytes) return RS_ERR_TOO_LARGE;
  st->c = c;
  return RS_OK;
}

static void noalloc_carve(Setup* st, char* base) {
  Job& j = st->j;
  const Caps& c = st->c;
  j.ctl = (Ctl*)(base + c.off_ctl);
  j.bins[0] = (Bin*)(base + c.off_bins0);
  j.bins[1] = (Bin*)(base + c.off_bins1);
  j.cap_bins = c.bins;
  j.base[0] = (u64*)(base + c.off_base0);
  j.base[1] = (u64*)(base + c.off_base1);
  j.cap_base = c.base;
  j.seg = (u64*)(base + c.off_seg);
  j.cap_seg = c.seg;
  j.chunks = (Chunk*)(base + c.off_chunks);
  j.cap_chunks = c.chunks;
  j.pieces = (Piece*)(base + c.off_pieces);
  j.cap_pieces = c.pieces;
}

// The level sequence of run_levels, launched without the optional timing events.
static rs_status noalloc_levels(const Setup& st, cudaStream_t s) {
  const Job& j = st.j;
  const u32 gs = (u32)st.sms * (u32)scatter_ctas_per_sm(j);
  const u32 gc = (u32)st.sms * (u32)classify_ctas_per_sm();
  int k;
  for (int lv = 0; lv < (int)j.K; lv++) {
    if ((k = launch_hist(j, lv, 0, s)) < 0) return RS_ERR_CUDA;
    count(k);
    if ((k = launch_hist(j, lv, 1, s)) < 0) return RS_ERR_CUDA;
    count(k);
    if ((k = launch_scatter(j, lv, gs, s)) < 0) return RS_ERR_CUDA;
    count(k);
    if ((k = launch_classify(j, lv, gc, s)) < 0) return RS_ERR_CUDA;
    count(k);
  }
  if ((k = launch_chunks(j, (u32)st.sms * (u32)chunk_ctas_per_sm(j), s)) < 0) return RS_ERR_CUDA;
  count(k);
  if ((k = launch_tiny(j, (u32)st.sms, s)) < 0) return RS_ERR_CUDA;
  count(k);
  if ((k = launch_copy(j, (u32)st.sms * 2, s)) < 0) return RS_ERR_CUDA;
  count(k);
  return RS_OK;
}

// radix_sort in two halves: every check and the workspace (sort_prepare), then the launches
// (sort_launch).  *work = false: nothing to sort (n <= 1).
static rs_status sort_prepare(void* in, void* tmp, uint64_t n, uint32_t rec_size, uint32_t key_size,
                              cudaStream_t s, Setup* st, bool* work) {
  *work = false;
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  if (n <= 1) return RS_OK;
  if ((r = validate_buffers(in, tmp, n, rec_size)) != RS_OK) return r;
  if ((r = setup_job(in, tmp, n, rec_size, key_size, 0, s, st)) != RS_OK) return r;
  *work = true;
  return RS_OK;
}

static rs_status sort_launch(const Setup& st, cudaStream_t s) {
  const Job& j = st.j;
  const u64 n = j.n;
  if (n <= j.chunk_max) {
    if (timed(RS_K_INIT, 0, s, [&] { return launch_init_single_chunk(j, s); }) < 0) return RS_ERR_CUDA;
    if (timed(RS_K_CHUNK, 0, s, [&] { return launch_chunks(j, 1, s); }) < 0) return RS_ERR_CUDA;
    return RS_OK;
  }
  u32 lo, W;
  plan_digit(n, 8 * j.K, j.chunk_max, j.wmax, &lo, &W);
  if (timed(RS_K_INIT, 0, s, [&] { return launch_init_plain(j, lo, W, s); }) < 0) return RS_ERR_CUDA;
  return run_levels(st, s);
}

}  // namespace rsg

using namespace rsg;

extern "C" {

rs_status radix_sort(void* in, void* tmp, uint64_t n, uint32_t rec_size, uint32_t key_size, rs_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  Setup st;
  bool work = false;
  const rs_status r = sort_prepare(in, tmp, n, rec_size, key_size, s, &st, &work);
  if (r != RS_OK || !work) return r;
  return sort_launch(st, s);
}

rs_status radix_sort_host(const void* h_in, void* h_out, void* d_buf, void* d_tmp, uint64_t n, uint32_t rec_size,
                          uint32_t key_size, rs_stream_t stream) {
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  if (n == 0) return RS_OK;
  if (!h_in || !h_out) return RS_ERR_INVALID_ARG;
  if ((r = validate_buffers(d_buf, d_tmp, n, rec_size)) != RS_OK) return r;
  if (check_device_ptr(d_buf) != RS_OK || check_device_ptr(d_tmp) != RS_OK) return RS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // every check (and the workspace) before the first copy is enqueued: a call that fails
  // launches nothing
  Setup st;
  bool work = false;
  if ((r = sort_prepare(d_buf, d_tmp, n, rec_size, key_size, s, &st, &work)) != RS_OK) return r;
  const size_t bytes = (size_t)(n * rec_size);
  if (cudaMemcpyAsync(d_buf, h_in, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return RS_ERR_CUDA;
  if (work && (r = sort_launch(st, s)) != RS_OK) return r;
  if (cudaMemcpyAsync(h_out, d_buf, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return RS_ERR_CUDA;
  return RS_OK;
}

rs_status radix_sort_segmented(void* in, void* tmp, const uint64_t* seg_offsets, uint64_t n_segs, uint64_t total,
                               uint32_t rec_size, uint32_t key_size, rs_stream_t stream) {
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (total > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  if (n_segs == 0 || total <= 1) return RS_OK;
  if (!seg_offsets) return RS_ERR_INVALID_ARG;
  if ((r = validate_buffers(in, tmp, total, rec_size)) != RS_OK) return r;
  if (check_device_ptr(seg_offsets) != RS_OK) return RS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Setup st;
  if ((r = setup_job(in, tmp, total, rec_size, key_size, n_segs, s, &st)) != RS_OK) return r;
  st.j.seg_off = (const u64*)seg_offsets;
  if (timed(RS_K_INIT, 0, s, [&] { return launch_init_segments(st.j, (u32)st.sms * 4, s); }) < 0) return RS_ERR_CUDA;
  // no segment can exceed the on-chip limit when all of them together do not: no levels
  return run_levels(st, s, total > st.j.chunk_max);
}

static rs_status one_pass(const void* src, void* dst, uint64_t n, uint32_t rec_size, uint32_t key_size,
                          uint32_t bit_lo, uint32_t width, uint64_t* counts, rs_stream_t stream) {
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (width == 0 || width > (uint32_t)kWMax || bit_lo + width > 8 * key_size) return RS_ERR_INVALID_ARG;
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)stream;
  if (counts) {  // histogram
    if (n == 0) {
      if (cudaMemsetAsync(counts, 0, sizeof(uint64_t) << width, s) != cudaSuccess) return RS_ERR_CUDA;
      return RS_OK;
    }
    if (!src) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)src) & 15) return RS_ERR_MISALIGNED;
  } else {
    if (n == 0) return RS_OK;
    if ((r = validate_buffers(src, dst, n, rec_size)) != RS_OK) return r;
    if (n == 1) {
      if (cudaMemcpyAsync(dst, src, rec_size, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return RS_ERR_CUDA;
      return RS_OK;
    }
  }
  Setup st;
  // the histogram has no destination: point the second buffer at the source (never written)
  if ((r = setup_job(const_cast<void*>(src), counts ? const_cast<void*>(src) : dst, n, rec_size, key_size, 0, s, &st)) != RS_OK)
    return r;
  Job& j = st.j;
  j.wmax = kWMax;  // the requested width, whatever the plan says
  int k;
  if ((k = launch_init_plain(j, bit_lo, width, s)) < 0) return RS_ERR_CUDA;
  count(k);
  if (counts) {
    if ((k = launch_hist(j, 0, 2, s)) < 0) return RS_ERR_CUDA;
    count(k);
    if ((k = launch_read_counts(j, (u64*)counts, width, s)) < 0) return RS_ERR_CUDA;
    count(k);
    return RS_OK;
  }
  if ((k = launch_hist(j, 0, 3, s)) < 0) return RS_ERR_CUDA;
  count(k);
  if ((k = launch_scatter(j, 0, (u32)st.sms * (u32)scatter_ctas_per_sm(j), s)) < 0)
    return RS_ERR_CUDA;
  count(k);
  return RS_OK;
}

rs_status radix_partition(const void* src, void* dst, uint64_t n, uint32_t rec_size, uint32_t key_size,
                          uint32_t bit_lo, uint32_t width, rs_stream_t stream) {
  return one_pass(src, dst, n, rec_size, key_size, bit_lo, width, nullptr, stream);
}

rs_status radix_histogram(const void* src, uint64_t n, uint32_t rec_size, uint32_t key_size, uint32_t bit_lo,
                          uint32_t width, uint64_t* counts, rs_stream_t stream) {
  if (!counts) return RS_ERR_INVALID_ARG;
  return one_pass(src, nullptr, n, rec_size, key_size, bit_lo, width, counts, stream);
}

rs_status radix_count_runs(const void* in, uint64_t n, uint32_t rec_size, uint32_t key_size, void* out,
                           uint64_t* counts, uint64_t* d_nruns, rs_stream_t stream) {
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  if (!d_nruns) return RS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (check_device_ptr(d_nruns) != RS_OK) return RS_ERR_INVALID_ARG;
  if (n == 0) return cudaMemsetAsync(d_nruns, 0, sizeof(uint64_t), s) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
  if (!in || !out || !counts) return RS_ERR_INVALID_ARG;
  if ((((uintptr_t)in) | ((uintptr_t)out)) & 15) return RS_ERR_MISALIGNED;
  if (overlap(in, out, n * rec_size)) return RS_ERR_OVERLAP;
  if (check_device_ptr(in) != RS_OK || check_device_ptr(out) != RS_OK || check_device_ptr(counts) != RS_OK)
    return RS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  // tile counts, tile offsets and range bounds, after the workspace's control block
  const u64 nt = runs_tiles(n), nbd = runs_bounds(n);
  const size_t o_cnt = al(sizeof(Ctl)), o_off = al(o_cnt + nt * 4), o_bd = al(o_off + nt * 8), bytes = al(o_bd + nbd * 8);
  Workspace* w = nullptr;
  if ((r = get_workspace(dev, s, bytes, &w)) != RS_OK) return r;
  char* base = (char*)w->mem;
  const u32 KW = key_size > 8 ? 2 : 1;
  u64 km[2];
  for (u32 q = 0; q < 2; q++) {
    const int b = (int)key_size - 8 * (int)q;
    km[q] = b >= 8 ? ~0ull : b <= 0 ? 0ull : ((1ull << (8 * b)) - 1);
  }
  const u32 grid = (u32)sm_count(dev) * 8;
  const int k = launch_count_runs((const u64*)in, n, rec_size / 8, KW, km[0], km[1], (u32*)(base + o_cnt),
                                  (u64*)(base + o_off), (u64*)(base + o_bd), (u64*)out, (u64*)counts, (u64*)d_nruns, grid, s);
  if (k < 0) return RS_ERR_CUDA;
  count(k);
  return RS_OK;
}

rs_status radix_sort_status(rs_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return RS_ERR_CUDA;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  Ctl* ctl = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find(std::make_pair(dev, s));
    if (it == g_ws.end() || !it->second.mem) return RS_OK;
    ctl = it->second.ctl;
  }
  // read and clear the word on the stream itself, so no other stream of the device waits
  u32 err = 0;
  if (cudaMemcpyAsync(&err, &ctl->err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RS_ERR_CUDA;
  if (err) {
    if (cudaMemsetAsync(&ctl->err, 0, sizeof(u32), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return RS_ERR_CUDA;
  }
  if (err & kErrTimeout) return RS_ERR_DEVICE_TIMEOUT;
  if (err & kErrOverflow) return RS_ERR_QUEUE_OVERFLOW;
  if (err) return RS_ERR_INTERNAL;
  return RS_OK;
}

const char* radix_sort_strerror(rs_status s) {
  switch (s) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_MISALIGNED: return "record buffer not 16-byte aligned";
    case RS_ERR_OVERLAP: return "record buffers overlap";
    case RS_ERR_TOO_LARGE: return "size too large";
    case RS_ERR_NO_MEMORY: return "workspace allocation failed";
    case RS_ERR_CUDA: return "CUDA error";
    case RS_ERR_DEVICE_TIMEOUT: return "device-side wait hit its limit";
    case RS_ERR_QUEUE_OVERFLOW: return "device-side list overflowed";
    case RS_ERR_UNSUPPORTED: return "unsupported (key_size > 16)";
    case RS_ERR_INTERNAL: return "device-side consistency check failed";
  }
  return "unknown status";
}

rs_status radix_sort_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ws.empty()) return RS_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
  }
  rs_status r = RS_OK;
  for (auto& kv : g_ws)
    if (kv.second.mem && cudaFree(kv.second.mem) != cudaSuccess) r = RS_ERR_CUDA;
  g_ws.clear();
  return r;
}

rs_status radix_sort_set_plan(const rs_plan* plan) {
  if (!plan) return RS_ERR_INVALID_ARG;
  rs_plan p = *plan;
  if (p.digit_bits_max && (p.digit_bits_max < (u32)kWMin || p.digit_bits_max > (u32)kWMax)) return RS_ERR_INVALID_ARG;
  if (p.tile_records && p.tile_records != 256 && p.tile_records != 512 && p.tile_records != 1024 &&
      p.tile_records != 2048 && p.tile_records != 4096)
    return RS_ERR_INVALID_ARG;
  if (p.chunk_records && p.chunk_records < 64) return RS_ERR_INVALID_ARG;
  if (p.tiny_records && (p.tiny_records < 2 || p.tiny_records > kTinyMax)) return RS_ERR_INVALID_ARG;
  if (p.enum_records && (p.enum_records < 8 || p.enum_records > kEsLimit)) return RS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  g_plan = p;
  return RS_OK;
}

rs_status radix_sort_get_plan(rs_plan* plan) {
  if (!plan) return RS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  *plan = g_plan;
  return RS_OK;
}

uint64_t radix_sort_launch_count(void) { return (uint64_t)g_launches.load(); }

uint32_t radix_sort_chunk_records(uint32_t rec_size) {
  if (rec_size == 0 || rec_size % 8 != 0 || rec_size > 256) return 0;
  return shape_for(1, rec_size, 8, current_plan()).chunk_max;
}

uint64_t radix_sort_workspace_bytes(uint64_t n, uint32_t rec_size, uint32_t key_size, uint64_t n_segs) {
  if (validate_layout(rec_size, key_size) != RS_OK || n > UINT64_MAX / rec_size) return 0;
  const Shape sh = shape_for(n, rec_size, key_size, current_plan());
  return (uint64_t)caps_for(n, sh.chunk_max, sh.wmax, n_segs).bytes;
}

rs_status radix_sort_reserve(uint64_t n, uint32_t rec_size, uint32_t key_size, uint64_t n_segs, rs_stream_t stream) {
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  const Shape sh = shape_for(n, rec_size, key_size, current_plan());
  const Caps c = caps_for(n, sh.chunk_max, sh.wmax, n_segs);
  Workspace* w = nullptr;
  return get_workspace(dev, (cudaStream_t)stream, c.bytes, &w);
}

rs_status radix_sort_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (enable) {
    g_prof.clear();
    g_evnext = 0;
  }
  g_prof_on = enable != 0;
  return RS_OK;
}

rs_status radix_sort_profile_kernels(uint32_t mask) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_mask = mask;
  return RS_OK;
}

int64_t radix_sort_profile_read(rs_kernel_time* out, int64_t max) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int64_t k = 0;
  for (const ProfRec& r : g_prof) {
    if (k >= max || !out) break;
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    out[k].kernel = r.kernel;
    out[k].level = r.level;
    out[k].ms = ms;
    k++;
  }
  return out ? k : (int64_t)g_prof.size();
}

rs_status radix_sort_noalloc(void* in, void* tmp, uint64_t n, uint32_t rec_size, uint32_t key_size,
                             uint32_t* d_status, rs_stream_t stream) {
  rs_status r = validate_layout(rec_size, key_size);
  if (r != RS_OK) return r;
  if (n > UINT64_MAX / rec_size) return RS_ERR_TOO_LARGE;
  Setup st;
  if ((r = noalloc_setup(in, tmp, n, rec_size, key_size, &st)) != RS_OK) return r;  // size check first
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 1) {
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s) != cudaSuccess) return RS_ERR_CUDA;
    return RS_OK;
  }
  if ((r = validate_buffers(in, tmp, n, rec_size)) != RS_OK) return r;
  if (check_device_ptr(in) != RS_OK || check_device_ptr(tmp) != RS_OK) return RS_ERR_INVALID_ARG;
  if (d_status && check_device_ptr(d_status) != RS_OK) return RS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  void* ws = nullptr;
  if ((r = noalloc_address(dev, &ws)) != RS_OK) return r;
  noalloc_carve(&st, (char*)ws);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return RS_ERR_CUDA;
  rs_plan p;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    p = g_plan;
  }
  if (p.sm_limit && (int)p.sm_limit < sms) sms = (int)p.sm_limit;
  st.sms = sms;
  st.dev = dev;
  st.j.lanes = lanes_for(st.j, sms);
  st.j.inject = g_inject.exchange(0);  // testing only (radix_sort_test_inject)
  const Job& j = st.j;
  // the array keeps the previous call's contents: its error word starts this call at zero,
  // and the init kernels rewrite the rest of the control block and the first bin list
  if (cudaMemsetAsync(&j.ctl->err, 0, sizeof(u32), s) != cudaSuccess) return RS_ERR_CUDA;
  int k;
  if (n <= j.chunk_max) {
    if ((k = launch_init_single_chunk(j, s)) < 0) return RS_ERR_CUDA;
    count(k);
    if ((k = launch_chunks(j, 1, s)) < 0) return RS_ERR_CUDA;
    count(k);
  } else {
    u32 lo, W;
    plan_digit(n, 8 * key_size, j.chunk_max, j.wmax, &lo, &W);
    if ((k = launch_init_plain(j, lo, W, s)) < 0) return RS_ERR_CUDA;
    count(k);
    if ((r = noalloc_levels(st, s)) != RS_OK) return r;
  }
  if (d_status && cudaMemcpyAsync(d_status, &j.ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RS_ERR_CUDA;
  return RS_OK;
}

rs_status radix_sort_test_inject(uint32_t flags) {
  if (flags > (kInjectRange | kInjectWait)) return RS_ERR_INVALID_ARG;
  g_inject = flags;
  return RS_OK;
}

}  // extern "C"
