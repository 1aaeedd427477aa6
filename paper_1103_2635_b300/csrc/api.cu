// C ABI of librbc.so and the host-side orchestration of the kernels.
//
// Every search is a sequence of BF calls (Section 3) on the device:
//   bf_search   : BF(Q, X)                                     (Section 3)
//   rbc_build   : BF(X, R) -> owners -> lists, radii            (Sections 4, 5.2)
//   rbc_search  : BF(Q, R) keeping all distances, pruning, then BF over the
//                 union of surviving lists per query tile        (Section 5.2)
// Host code only validates arguments, allocates stream-ordered workspace and
// launches kernels; every arithmetic step of the search runs on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {
thread_local char g_err[512] = "";
}

thread_local long long t_launches = 0;

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? RBC_ERR_OOM : RBC_ERR_CUDA;
}

const char* last_error_text() { return g_err; }

}  // namespace rbc

// the index object (opaque to callers): index.cuh

namespace rbc {
namespace {

#define RBC_TRY(x)               \
  do {                           \
    int _r = (x);                \
    if (_r != RBC_OK) return _r; \
  } while (0)

// ---------------------------------------------------------------------------
// representative sampler (Section 4, fixed-size reading): partial
// Fisher-Yates over [0, n) driven by SplitMix64 (Steele, Lea & Flood 2014)
// ---------------------------------------------------------------------------
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform in [0, bound): draws >= 2^64 - (2^64 mod bound) are rejected
  uint64_t below(uint64_t bound) {
    uint64_t rem = (0 - bound) % bound;  // 2^64 mod bound
    for (;;) {
      uint64_t x = next();
      if (rem == 0 || x < (0 - rem)) return x % bound;
    }
  }
};

std::vector<int64_t> sample_reps_host(int64_t n, int32_t n_r, uint64_t seed) {
  SplitMix64 g{seed};
  std::unordered_map<int64_t, int64_t> moved;  // positions no longer holding their own index
  moved.reserve((size_t)n_r * 2 + 1);
  auto at = [&](int64_t p) {
    auto it = moved.find(p);
    return it == moved.end() ? p : it->second;
  };
  std::vector<int64_t> out((size_t)n_r);
  for (int32_t i = 0; i < n_r; ++i) {
    int64_t j = i + (int64_t)g.below((uint64_t)(n - i));
    int64_t vi = at(i), vj = at(j);
    moved[i] = vj;
    moved[j] = vi;
    out[(size_t)i] = vj;
  }
  std::sort(out.begin(), out.end());
  return out;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

// Workspace memory comes from a library-owned stream-ordered pool per device
// whose release threshold is unlimited: freed blocks stay mapped and are
// reused by the next call instead of being unmapped at every
// synchronisation (a search's workspace is a few GB).  rbc_trim_workspace()
// hands the cached memory back.
constexpr int MAX_POOL_DEVICES = 64;
cudaMemPool_t g_pools[MAX_POOL_DEVICES] = {};
std::mutex g_pool_mu;

cudaMemPool_t workspace_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_POOL_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

// Stream-ordered scratch released when the arena goes out of scope.
// whether work enqueued on `st` is being recorded into a graph
bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Workspace bytes this thread's arenas hold, and the peak since the last
// reset (reported per search as rbc_search_stats::workspace_bytes).
thread_local int64_t t_ws_cur = 0;
thread_local int64_t t_ws_peak = 0;

struct Arena {
  cudaStream_t st;
  cudaMemPool_t pool;
  std::vector<void*> ptrs;
  int64_t held = 0;
  // under stream capture the allocations become graph memory nodes of the
  // default pool
  explicit Arena(cudaStream_t s)
      : st(s), pool(stream_capturing(s) ? nullptr : workspace_pool()) {}
  ~Arena() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    t_ws_cur -= held;
  }
  template <typename T>
  int alloc(T** out, int64_t count) {
    *out = nullptr;
    if (count <= 0) count = 1;
    void* p = nullptr;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, (size_t)count * sizeof(T), pool, st)
                         : cudaMallocAsync(&p, (size_t)count * sizeof(T), st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("workspace allocation of %lld bytes failed: %s",
                (long long)((size_t)count * sizeof(T)), cudaGetErrorString(e));
      return RBC_ERR_OOM;
    }
    ptrs.push_back(p);
    held += count * (int64_t)sizeof(T);
    t_ws_cur += count * (int64_t)sizeof(T);
    if (t_ws_cur > t_ws_peak) t_ws_peak = t_ws_cur;
    *out = static_cast<T*>(p);
    return RBC_OK;
  }
};

constexpr float U32 = 5.9604645e-08f;
// relative bound of rho from the FP32 tile kernel (sequential fused sums)
float simt_eps(int d) { return (float)(d + 8) * U32; }
// relative bound of rho from the FP32 re-rank (interleaved partial sums)
float rerank_eps_host(int d) { return (0.25f * d + 8.0f) * U32; }
int pad64(int d) { return (d + 63) / 64 * 64; }

// Stage one BF(Q, R) as dense work items: the representatives are split into
// column chunks (at least 256 each) so that every SM gets at least six items
// (three per resident CTA), which keeps the last wave's tail a small part of
// the pass; a batch with that many 128-query tiles keeps one item per tile.
void set_stage1_splits(TileWork& w, int64_t tiles, int n_r, int sms) {
  int64_t splits = tiles > 0 ? (6LL * sms + tiles - 1) / tiles : 1;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, (n_r + 255) / 256));
  int64_t chunk = (n_r + splits - 1) / splits;
  splits = (n_r + chunk - 1) / chunk;
  w.dense_splits = (int)splits;
  w.dense_chunk = chunk;
  w.num_items = (int)(tiles * splits);
}
// low-precision row length: 128-byte K blocks of 64 16-bit or 128 FP8 elements
int lp_pad(int d, int storage) {
  return storage == RBC_FP8E4M3 ? (d + 127) / 128 * 128 : pad64(d);
}
// the tensor-core kernel reads whole tiles of norms past the last row
constexpr int64_t NORM_PAD = 512;

// ---- per-thread statistics ----
struct StatsBlock {
  unsigned long long v[8];
};
thread_local cudaStream_t t_stats_stream = nullptr;
thread_local bool t_stats_pending = false;
// pinned landing block of a thread's statistics, freed when the thread ends
// (serving workers come and go with their servers)
struct StatsHost {
  StatsBlock* p = nullptr;
  ~StatsHost() {
    if (!p) return;
    if (t_stats_pending && t_stats_stream) cudaStreamSynchronize(t_stats_stream);
    cudaFreeHost(p);
  }
};
thread_local StatsHost t_stats_holder;
thread_local rbc_search_stats t_stats_fixed;

// device counters: ints [0] uncertified [1] fp64 ties [2] boundary ties,
// [4..6] the same for the FP32 re-search; u64 sums [0] kept reps
// [1] tile points [2] (query, point) pairs of the main pass [3] emitted
// candidates (windowed search)
struct Counters {
  int* c = nullptr;
  unsigned long long* sums = nullptr;
};

// Optional per-phase device timing (rbc_set_timing).  Marks 0..4 bound the
// phases: [0,1) preparation + stage one, [1,2) main BF kernel, [2,3) merge +
// re-rank + certification, [3,4) FP32 re-search.
struct Timing {
  bool on = false;
  bool ready = false;
  cudaEvent_t ev[5];
  double ms[4] = {0, 0, 0, 0};
};
thread_local Timing t_timing;

void tmark(int i, cudaStream_t st) {
  if (!t_timing.on) return;
  if (!t_timing.ready) {
    for (auto& e : t_timing.ev) cudaEventCreate(&e);
    t_timing.ready = true;
  }
  cudaEventRecord(t_timing.ev[i], st);
}

// after the stream has passed mark 4: add the phase times
void taccumulate() {
  if (!t_timing.on || !t_timing.ready) return;
  cudaEventSynchronize(t_timing.ev[4]);
  for (int i = 0; i < 4; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t_timing.ev[i], t_timing.ev[i + 1]) == cudaSuccess)
      t_timing.ms[i] += ms;
  }
  cudaGetLastError();
}

__global__ void stats_pack_kernel(const int* c, const unsigned long long* sums,
                                  unsigned long long* out) {
  if (threadIdx.x == 0) {
    out[0] = sums[0];
    out[1] = sums[1];
    out[2] = (unsigned long long)c[0];
    out[3] = (unsigned long long)(c[1] + c[5]);
    out[4] = (unsigned long long)(c[2] + c[6]);
    out[5] = (unsigned long long)c[4];
    out[6] = sums[2];
    out[7] = sums[3];
  }
}

int counters_alloc(Counters& cn, Arena& ar, cudaStream_t st) {
  RBC_TRY(ar.alloc(&cn.c, 8));
  RBC_TRY(ar.alloc(&cn.sums, 4));
  RBC_CUDA(cudaMemsetAsync(cn.c, 0, 8 * sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(cn.sums, 0, 4 * sizeof(unsigned long long), st));
  t_launches = 0;
  for (double& v : t_timing.ms) v = 0;
  return RBC_OK;
}

thread_local int64_t t_stats_host_kept = -1;  // >= 0: kept_reps known on the host
// set by bf_search_noalloc: its counters ([0] uncertified, [1] FP64 ties,
// [2] boundary ties) live in the library's static scratch and are read there
thread_local const int* t_stats_counters_dev = nullptr;

int stats_publish(const Counters& cn, int64_t queries, int64_t items, int64_t host_pairs, Arena& ar,
                  cudaStream_t st, int64_t host_kept = -1) {
  StatsBlock*& t_stats_host = t_stats_holder.p;
  if (!t_stats_host && stream_capturing(st)) {
    // no pinned landing block yet, and none can be allocated while a graph
    // is recorded: this search reports host-side statistics only
    memset(&t_stats_fixed, 0, sizeof(t_stats_fixed));
    t_stats_fixed.queries = queries;
    t_stats_fixed.stage2_items = items;
    t_stats_fixed.kernel_launches = t_launches;
    t_stats_pending = false;
    t_stats_counters_dev = nullptr;
    return RBC_OK;
  }
  if (!t_stats_host) {
    void* p = nullptr;
    RBC_CUDA(cudaMallocHost(&p, sizeof(StatsBlock)));
    t_stats_host = static_cast<StatsBlock*>(p);
  }
  unsigned long long* packed;
  RBC_TRY(ar.alloc(&packed, 8));
  stats_pack_kernel<<<1, 32, 0, st>>>(cn.c, cn.sums, packed);
  RBC_LAUNCH_CHECK("stats_pack_kernel");
  RBC_CUDA(cudaMemcpyAsync(t_stats_host->v, packed, sizeof(StatsBlock), cudaMemcpyDeviceToHost,
                           st));
  memset(&t_stats_fixed, 0, sizeof(t_stats_fixed));
  t_stats_fixed.queries = queries;
  t_stats_fixed.stage2_items = items;
  t_stats_fixed.pairs = host_pairs;
  t_stats_host_kept = host_kept;
  t_stats_fixed.kernel_launches = t_launches;
  t_stats_fixed.stage1_ms = t_timing.ms[0];
  t_stats_fixed.stage2_ms = t_timing.ms[1];
  t_stats_fixed.select_ms = t_timing.ms[2];
  t_stats_fixed.fallback_ms = t_timing.ms[3];
  t_stats_stream = st;
  t_stats_pending = true;
  t_stats_counters_dev = nullptr;
  return RBC_OK;
}

// ---- inputs / outputs that may live in host memory ----
struct IoPlan {
  const float* Qdev = nullptr;
  const float* Qhost = nullptr;  // set when the batches copy their own rows (defer_copy)
  int64_t* ids_dev = nullptr;
  float* dist_dev = nullptr;
  bool ids_host = false, dist_host = false;
};

// Host query rows: copied here in one piece, or (defer_copy) only given
// their device buffer, each batch then copying its own rows beside stage 1.
int io_prepare(const float* Q, int64_t m, int d, int k, int64_t* out_ids, float* out_dist,
               IoPlan& io, Arena& ar, cudaStream_t st, bool defer_copy = false) {
  if (m > 0 && !is_device_ptr(Q)) {
    float* q;
    RBC_TRY(ar.alloc(&q, m * d));
    if (defer_copy)
      io.Qhost = Q;
    else
      RBC_CUDA(cudaMemcpyAsync(q, Q, (size_t)m * d * sizeof(float), cudaMemcpyHostToDevice, st));
    io.Qdev = q;
  } else {
    io.Qdev = Q;
  }
  io.ids_host = m > 0 && !is_device_ptr(out_ids);
  io.dist_host = m > 0 && !is_device_ptr(out_dist);
  if (io.ids_host) {
    RBC_TRY(ar.alloc(&io.ids_dev, m * k));
  } else {
    io.ids_dev = out_ids;
  }
  if (io.dist_host) {
    RBC_TRY(ar.alloc(&io.dist_dev, m * k));
  } else {
    io.dist_dev = out_dist;
  }
  return RBC_OK;
}

// Query rows from host memory in FEED_CHUNKS row chunks on a second stream
// (one per thread and device), each chunk's per-row steps (stage 1, row
// statistics, low-precision copy) waiting only for its own rows: they
// overlap the copy of later rows.  Batches below FEED_MIN_ROWS copy in one
// piece on the search's stream.
constexpr int FEED_CHUNKS = 8;
constexpr int64_t FEED_MIN_ROWS = 8192;
constexpr int FEED_MAX_DEVICES = 64;

struct FeedStreams {
  cudaStream_t s[FEED_MAX_DEVICES] = {};
  ~FeedStreams() {
    for (cudaStream_t x : s)
      if (x) cudaStreamDestroy(x);
  }
};
thread_local FeedStreams t_feed;

cudaStream_t feed_stream() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= FEED_MAX_DEVICES) {
    cudaGetLastError();
    return nullptr;
  }
  if (!t_feed.s[dev] &&
      cudaStreamCreateWithFlags(&t_feed.s[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    t_feed.s[dev] = nullptr;
  }
  return t_feed.s[dev];
}

// the events of one batch's chunk copies (released once they complete)
struct FeedEvents {
  cudaEvent_t ev[FEED_CHUNKS + 1] = {};
  ~FeedEvents() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

int io_finish(int64_t m, int k, int64_t* out_ids, float* out_dist, const IoPlan& io,
              cudaStream_t st) {
  if (m == 0) return RBC_OK;
  if (io.ids_host)
    RBC_CUDA(cudaMemcpyAsync(out_ids, io.ids_dev, (size_t)m * k * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, st));
  if (io.dist_host)
    RBC_CUDA(cudaMemcpyAsync(out_dist, io.dist_dev, (size_t)m * k * sizeof(float),
                             cudaMemcpyDeviceToHost, st));
  if (io.ids_host || io.dist_host) RBC_CUDA(cudaStreamSynchronize(st));
  return RBC_OK;
}

int valid_enums(int metric, int storage) {
  if (metric != RBC_L2 && metric != RBC_L1) {
    set_error("unknown metric %d", metric);
    return RBC_ERR_ARG;
  }
  if (storage != RBC_F32 && storage != RBC_BF16 && storage != RBC_F16 &&
      storage != RBC_FP8E4M3) {
    set_error("unknown storage %d", storage);
    return RBC_ERR_ARG;
  }
  return RBC_OK;
}

bool uses_lp(int storage, int metric) { return storage != RBC_F32 && metric == RBC_L2; }

int choose_c(int k, bool lp, int rerank_c) {
  int c = k + 1;
  if (lp) c = rerank_c > 0 ? std::max(rerank_c, k + 1) : (k <= 1 ? 16 : 32);
  return std::min(c, MAX_C);
}

// Candidates kept per (row, half) by the tensor-core kernel: half of c_out.
// The certificate also bounds what full half-lists dropped, so a row's c_out
// candidates need not fit in one half.
int lp_width(int c) { return c <= 16 ? 8 : (c <= 32 ? 16 : 32); }

// FP32 paths: the CUDA-core kernel keeps the C best per (row, half), C the
// smallest list width >= k + 1, and the select merges up to 2C of them (at
// most MAX_C): the extra candidates widen the certificate's margin at no
// cost to the distance kernel.
int f32_list_width(int k) { return simt_list_width(k + 1); }
int f32_c_out(int k) { return std::min(2 * f32_list_width(k), MAX_C); }

// The exact finish (band.cu) of the rows a select launch could not certify:
// rows fb[0 .. *nfb) of the query buffer Qbuf, results at qorig[row].
BandArgs band_args(const int* fb, const int* nfb, const float* Qbuf, const int* qorig,
                   const float* X32, const int* xid, int64_t n, int d, int k, int metric,
                   int64_t* out_ids, float* out_dist) {
  BandArgs b{};
  b.rows = fb;
  b.nrows_dev = nfb;
  b.Q32 = Qbuf;
  b.qorig = qorig;
  b.X32 = X32;
  b.xid = xid;
  b.n = n;
  b.d = d;
  b.ld = d;
  b.k = k;
  b.metric = metric;
  b.eps = rerank_eps_host(d);
  b.out_ids = out_ids;
  b.out_dist = out_dist;
  return b;
}

// scratch of the band pass's chunked rows (a few hundred KB)
int band_split_alloc(BandArgs& b, Arena& ar) {
  const int64_t n = band_split_scratch_entries();
  RBC_TRY(ar.alloc(&b.split_r, n));
  RBC_TRY(ar.alloc(&b.split_i, n));
  return RBC_OK;
}

// ---------------------------------------------------------------------------
// database views for the BF core
// ---------------------------------------------------------------------------
struct DbView {
  const float* X32 = nullptr;  // [rows, d] FP32 rows
  const int* xid = nullptr;    // row -> original id (nullptr = identity)
  int64_t rows = 0;
  const void* Xlp = nullptr;   // [rows, dpad]
  const float* xnorm = nullptr;
  const float* xscale = nullptr;  // FP8: per-row scales
  int dpad = 0;
  const unsigned* lp_max = nullptr;  // [0] max |x - x~|, [1] max |x~| (float bits)
  const void* nblock = nullptr;      // bf16 / fp16: [rows + pad, 16] norm block
};

// Dense BF(Q, DB) with the FP32 CUDA-core kernel; results for query row i go
// to output row qorig[i] (identity when null).  `cnt` = 3 counters.
int bf_dense_f32(const float* Qdev, int64_t m, const DbView& db, int d, int k, int metric,
                 const int* qorig, int64_t* out_ids, float* out_dist, int* cnt, Arena& ar,
                 cudaStream_t st, bool marks = true) {
  if (m == 0) return RBC_OK;
  const int C = f32_list_width(k);
  const int c_out = f32_c_out(k);
  const int64_t tiles = (m + TQ - 1) / TQ;
  const int sms = sm_count();
  int64_t splits = (8LL * sms + tiles - 1) / tiles;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, db.rows / 512)));
  int64_t chunk = (db.rows + splits - 1) / splits;
  splits = (db.rows + chunk - 1) / chunk;
  const int64_t items = tiles * splits;
  float* ps;
  int* pi;
  RBC_TRY(ar.alloc(&ps, items * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pi, items * TQ * 2 * C));
  TileWork w{};
  w.num_items = (int)items;
  w.m = m;
  w.n = db.rows;
  w.dense_splits = (int)splits;
  w.dense_chunk = chunk;
  int grid = (int)std::min<int64_t>(items, (int64_t)sms * 2 * 16);
  // l2: the expansion form |x|^2 - 2 q.x (one FFMA per dimension) with FP32
  // norms, certified with its absolute rounding bound; l1: the difference form
  const bool exp32 = metric == RBC_L2;
  float *xn = nullptr, *qn = nullptr;
  unsigned* xmax = nullptr;
  if (exp32) {
    RBC_TRY(ar.alloc(&xn, db.rows));
    RBC_TRY(ar.alloc(&qn, m));
    RBC_TRY(ar.alloc(&xmax, 1));
    RBC_CUDA(cudaMemsetAsync(xmax, 0, sizeof(unsigned), st));
    RBC_TRY(launch_row_norms(db.X32, db.rows, d, xn, xmax, st));
    RBC_TRY(launch_row_norms(Qdev, m, d, qn, nullptr, st));
  }
  if (marks) tmark(1, st);
  if (exp32)
    RBC_TRY(launch_bf_simt_topc_exp(Qdev, db.X32, xn, d, C, w, TopOut{ps, pi, nullptr}, grid, st));
  else
    RBC_TRY(launch_bf_simt_topc(Qdev, db.X32, d, metric, C, w, TopOut{ps, pi, nullptr}, grid, st));
  if (marks) tmark(2, st);
  SelectArgs a{};
  if (exp32) {
    a.lp = 1;
    a.exp32 = 1;
    a.q_lpnorm = qn;
    a.x_norm_max_bits = xmax;
  }
  a.part_score = ps;
  a.part_idx = pi;
  a.C = C;
  a.nsub = 2;
  a.dense_splits = (int)splits;
  a.m = m;
  a.Q32 = Qdev;
  a.d = d;
  a.metric = metric;
  a.qorig = qorig;
  a.X32 = db.X32;
  a.xid = db.xid;
  a.simt_eps = simt_eps(d);
  a.k = k;
  a.c_out = c_out;
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  int* fb;
  int* lc;  // [0] rows appended to fb, [1..2] ties
  RBC_TRY(ar.alloc(&fb, m));
  RBC_TRY(ar.alloc(&lc, 8));
  RBC_CUDA(cudaMemsetAsync(lc, 0, 8 * sizeof(int), st));
  a.fallback_rows = fb;
  a.counters = lc;
  RBC_TRY(launch_select(a, st));
  RBC_TRY(launch_add_ints(cnt, lc, 3, st));
  if (marks) tmark(3, st);
  BandArgs bb = band_args(fb, lc, Qdev, qorig, db.X32, db.xid, db.rows, d, k, metric, out_ids,
                          out_dist);
  RBC_TRY(band_split_alloc(bb, ar));
  RBC_TRY(launch_band(bb, (int)m, st));
  if (marks) tmark(4, st);
  return RBC_OK;
}

// Rows of a query buffer that failed certification are searched again with
// the FP32 kernel over every row of `db` (a superset of what they needed).
int fallback_f32(const float* Qbuf, const int* rows_dev, int nrows, const int* qorig,
                 const DbView& db, int d, int k, int metric, int64_t* out_ids, float* out_dist,
                 int* cnt, Arena& ar, cudaStream_t st) {
  if (nrows <= 0) return RBC_OK;
  float* Qf;
  int* forig;
  RBC_TRY(ar.alloc(&Qf, (int64_t)nrows * d));
  RBC_TRY(ar.alloc(&forig, nrows));
  RBC_TRY(launch_gather_rows(Qbuf, nullptr, rows_dev, nrows, d, Qf, st));
  RBC_TRY(launch_map_rows(rows_dev, nullptr, nrows, qorig, forig, st));
  // nested pass: its phases belong to the caller's "re-search" phase
  return bf_dense_f32(Qf, nrows, db, d, k, metric, forig, out_ids, out_dist, cnt, ar, st, false);
}

// Low-precision copy of a query buffer.
struct LpQueries {
  void* lp = nullptr;
  float* norm = nullptr;
  float* err = nullptr;
  float* scale = nullptr;  // FP8 only
  int storage = RBC_BF16;
};

int lp_queries_alloc(int64_t m, int dpad, int storage, LpQueries& q, Arena& ar) {
  uint8_t* buf;
  RBC_TRY(ar.alloc(&buf, std::max<int64_t>(m, 1) * dpad * lp_elem_bytes(storage)));
  RBC_TRY(ar.alloc(&q.norm, m));
  RBC_TRY(ar.alloc(&q.err, m));
  if (storage == RBC_FP8E4M3) RBC_TRY(ar.alloc(&q.scale, m));
  q.lp = buf;
  q.storage = storage;
  return RBC_OK;
}

// rows [r0, r0 + mr) of Qdev into the same rows of q
int lp_queries_rows(const float* Qdev, int64_t r0, int64_t mr, int d, int dpad,
                    const LpQueries& q, cudaStream_t st) {
  const int64_t rb = (int64_t)dpad * lp_elem_bytes(q.storage);
  return launch_to_lowp(Qdev + r0 * d, mr, d, dpad, q.storage,
                        static_cast<uint8_t*>(q.lp) + r0 * rb, q.norm + r0, q.err + r0, nullptr,
                        nullptr, st, q.scale ? q.scale + r0 : nullptr);
}

int lp_queries(const float* Qdev, int64_t m, int d, int dpad, int storage, LpQueries& q,
               Arena& ar, cudaStream_t st) {
  RBC_TRY(lp_queries_alloc(m, dpad, storage, q, ar));
  return lp_queries_rows(Qdev, 0, m, d, dpad, q, st);
}

int bf_dense_lp(const float* Qdev, int64_t m, const DbView& db, int d, int k, int storage,
                int rerank_c, int64_t* out_ids, float* out_dist, int* cnt, Arena& ar,
                cudaStream_t st, const int* qorig = nullptr, int level = 0);

// Select (merge + re-rank + certification) for the low-precision pass, then
// the re-search of uncertified rows (one host read of their count): first on
// the tensor cores with the widest candidate lists (level 0 only), then, for
// rows that still fail, with the FP32 kernel over every row of `db`.
int fallback_rbc_f32(const rbc_index* ix, const float* Qbuf, const int* rows_dev, int nrows,
                     const int* qorig, int k, int64_t* out_ids, float* out_dist, int* cnt,
                     Arena& ar, cudaStream_t st, const float* g_rows = nullptr);

int select_lp_and_fallback(const float* ps, const int* pi, const int* pv, int C,
                           const int* tile_slot_off,
                           int dense_splits, int64_t m, const float* Qbuf, const LpQueries& ql,
                           const DbView& db, int d, int k, int c_out, const int* qorig,
                           int64_t* out_ids, float* out_dist, int* cnt, Arena& ar,
                           cudaStream_t st, int level = 0, const rbc_index* rbc_ix = nullptr,
                           const float* g_rows = nullptr) {
  int* fb_rows;
  int* lc;  // this call's counters: [0] rows appended to fb_rows, [1..2] ties
  RBC_TRY(ar.alloc(&fb_rows, m));
  RBC_TRY(ar.alloc(&lc, 8));
  RBC_CUDA(cudaMemsetAsync(lc, 0, 8 * sizeof(int), st));
  SelectArgs a{};
  a.part_score = ps;
  a.part_idx = pi;
  a.slot_valid = pv;
  a.C = C;
  a.nsub = 2;
  a.tile_slot_off = tile_slot_off;
  a.dense_splits = dense_splits;
  a.m = m;
  a.Q32 = Qbuf;
  a.d = d;
  a.metric = RBC_L2;
  a.qorig = qorig;
  a.X32 = db.X32;
  a.xid = db.xid;
  a.lp = 1;
  a.q_lpnorm = ql.norm;
  a.q_err = ql.err;
  a.x_err_max_bits = db.lp_max;
  a.x_norm_max_bits = db.lp_max + 1;
  a.k = k;
  a.c_out = c_out;
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.fallback_rows = fb_rows;
  a.counters = lc;
  if (level == 0) tmark(2, st);
  RBC_TRY(launch_select(a, st));
  if (level == 0) tmark(3, st);
  RBC_TRY(launch_add_ints(cnt, lc, 3, st));
  int nfb = 0;
  RBC_CUDA(cudaMemcpyAsync(&nfb, lc, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  if (nfb > 0) {
    if (rbc_ix) {
      // exact RBC: the FP32 exact search over the rows' surviving lists
      RBC_TRY(fallback_rbc_f32(rbc_ix, Qbuf, fb_rows, nfb, qorig, k, out_ids, out_dist, cnt + 4,
                               ar, st, g_rows));
    } else if (level == 0 && db.Xlp) {
      float* Qf;
      int* forig;
      RBC_TRY(ar.alloc(&Qf, (int64_t)nfb * d));
      RBC_TRY(ar.alloc(&forig, nfb));
      RBC_TRY(launch_gather_rows(Qbuf, nullptr, fb_rows, nfb, d, Qf, st));
      RBC_TRY(launch_map_rows(fb_rows, nullptr, nfb, qorig, forig, st));
      RBC_TRY(bf_dense_lp(Qf, nfb, db, d, k, ql.storage, MAX_C, out_ids, out_dist, cnt + 4, ar, st,
                          forig, 1));
    } else {
      RBC_TRY(fallback_f32(Qbuf, fb_rows, nfb, qorig, db, d, k, RBC_L2, out_ids, out_dist,
                           cnt + 4, ar, st));
    }
  }
  if (level == 0) tmark(4, st);
  return RBC_OK;
}

// Dense BF(Q, DB) on the tensor cores (L2, bf16 / fp16).  Level 1 is the
// re-search of rows that failed certification: the widest lists, output rows
// mapped through qorig, no phase marks.
int bf_dense_lp(const float* Qdev, int64_t m, const DbView& db, int d, int k, int storage,
                int rerank_c, int64_t* out_ids, float* out_dist, int* cnt, Arena& ar,
                cudaStream_t st, const int* qorig, int level) {
  if (m == 0) return RBC_OK;
  const int c_out = choose_c(k, true, rerank_c);
  const int C = level ? MAX_C : lp_width(c_out);
  LpQueries ql;
  RBC_TRY(lp_queries(Qdev, m, d, db.dpad, storage, ql, ar, st));
  if (level == 0) tmark(1, st);
  const int64_t tiles = (m + TQ - 1) / TQ;
  const int sms = sm_count();
  int64_t splits = (16LL * sms + tiles - 1) / tiles;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, db.rows / 8192)));
  // a query merges splits x 2C partial entries: keep that within 2048
  splits = std::min<int64_t>(splits, std::max(1, 2048 / (2 * C)));
  int64_t chunk = (db.rows + splits - 1) / splits;
  chunk = (chunk + 255) / 256 * 256;
  splits = (db.rows + chunk - 1) / chunk;
  const int64_t items = tiles * splits;
  float* ps;
  int* pi;
  int* pv;
  RBC_TRY(ar.alloc(&ps, items * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pi, items * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pv, items));
  TileWork w{};
  w.num_items = (int)items;
  w.m = m;
  w.n = db.rows;
  w.dense_splits = (int)splits;
  w.dense_chunk = chunk;
  LpMatrix Qm{ql.lp, ql.norm, m, db.dpad, storage, nullptr, ql.scale};
  LpMatrix Xm{db.Xlp, db.xnorm, db.rows, db.dpad, storage, db.nblock, db.xscale};
  uint32_t* dev_err;
  RBC_TRY(ar.alloc(&dev_err, 1));
  RBC_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(uint32_t), st));
  int grid = (int)std::min<int64_t>(items, (int64_t)sms);
  RBC_TRY(launch_bf_tc_topc(Qm, Xm, C, w, TopOut{ps, pi, pv}, grid, st, dev_err));
  RBC_TRY(select_lp_and_fallback(ps, pi, pv, C, nullptr, (int)splits, m, Qdev, ql, db, d, k,
                                 c_out, qorig, out_ids, out_dist, cnt, ar, st, level));
  if (level == 0) taccumulate();
  uint32_t herr = 0;
  RBC_CUDA(cudaMemcpyAsync(&herr, dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error("tensor-core kernel reported device error flags 0x%x", herr);
    return (herr & DEV_ERR_TIMEOUT) ? RBC_ERR_TIMEOUT : RBC_ERR_CUDA;
  }
  return RBC_OK;
}

// ---------------------------------------------------------------------------
// build (Sections 4, 5.2)
// ---------------------------------------------------------------------------
// Low-precision copies of the list rows and the representatives (L2 with
// bf16 / fp16 storage): rows padded to dpad, squared norms, error maxima.
int make_lp_copies(rbc_index* ix, cudaStream_t st) {
  if (ix->storage == RBC_F32 || ix->metric != RBC_L2) return RBC_OK;
  const int64_t n = ix->list_entries;
  const int d = ix->d, n_r = ix->n_r;
  const bool fp8 = ix->storage == RBC_FP8E4M3;
  const int eb = lp_elem_bytes(ix->storage);
  ix->dpad = lp_pad(d, ix->storage);
  uint8_t* xl;
  uint8_t* rl;
  RBC_TRY(ix->alloc(&xl, n * ix->dpad * eb));
  RBC_TRY(ix->alloc(&ix->xnorm, n + NORM_PAD));
  RBC_CUDA(cudaMemsetAsync(ix->xnorm + n, 0, NORM_PAD * sizeof(float), st));
  RBC_TRY(ix->alloc(&ix->lp_max, 4));
  RBC_TRY(ix->alloc(&rl, (int64_t)n_r * ix->dpad * eb));
  RBC_TRY(ix->alloc(&ix->rnorm, n_r));
  if (fp8) {
    RBC_TRY(ix->alloc(&ix->xscale, n + NORM_PAD));
    RBC_CUDA(cudaMemsetAsync(ix->xscale + n, 0, NORM_PAD * sizeof(float), st));
    RBC_TRY(ix->alloc(&ix->rscale, n_r));
  }
  RBC_CUDA(cudaMemsetAsync(ix->lp_max, 0, 4 * sizeof(unsigned), st));
  RBC_TRY(launch_to_lowp(ix->X32, n, d, ix->dpad, ix->storage, xl, ix->xnorm, nullptr,
                         ix->lp_max, ix->lp_max + 1, st, ix->xscale));
  if (!fp8) {
    // -|x~|^2 / 2 as a bf16 (high, low) block: the windowed kernel adds it to
    // its accumulators with one extra MMA instead of a per-column FMA
    RBC_TRY(ix->alloc(reinterpret_cast<uint16_t**>(&ix->xnblock), (n + NORM_PAD) * NBLOCK_COLS));
    RBC_TRY(launch_norm_block(ix->xnorm, n, n + NORM_PAD, ix->xnblock, st));
    // with two spare padding columns the pair goes into the rows themselves
    // (an fp16 pair only while -|x~|^2 / 2 stays well inside its range)
    if (d % 2 == 0 && ix->dpad - d >= 2) {
      unsigned nmax_bits = 0;
      RBC_CUDA(cudaMemcpyAsync(&nmax_bits, ix->lp_max + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                               st));
      RBC_CUDA(cudaStreamSynchronize(st));
      float nmax = 0.f;
      std::memcpy(&nmax, &nmax_bits, sizeof(float));
      if (ix->storage == RBC_BF16 || 0.5 * (double)nmax * nmax < 16384.0) {
        RBC_TRY(launch_fold_norm(xl, ix->xnorm, n, ix->dpad, d, ix->storage, st));
        ix->norm_fold_col = d;
      }
    }
  }
  RBC_TRY(launch_to_lowp(ix->R32, n_r, d, ix->dpad, ix->storage, rl, ix->rnorm, nullptr,
                         ix->lp_max + 2, ix->lp_max + 3, st, ix->rscale));
  ix->Xlp = xl;
  ix->Rlp = rl;
  if (ix->plan == RBC_PLAN_WINDOW_OFFSET && ix->mode == RBC_EXACT && ix->storage == RBC_BF16 &&
      d % 8 == 0 && ix->offsets) {
    // list rows as offsets from their representative: y~ = bf16(x - r)
    float* y32 = nullptr;
    RBC_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&y32), (size_t)n * (d + 1) * sizeof(float),
                             st));
    float* yerr = y32 + n * d;  // per-row |y - y~|
    uint8_t* yl;
    unsigned* ymax;
    int rc = ix->alloc(&yl, n * ix->dpad * eb);
    if (rc == RBC_OK) rc = ix->alloc(&ix->ynorm, n + NORM_PAD);
    if (rc == RBC_OK) rc = ix->alloc(&ix->yerr_list, n_r);
    if (rc == RBC_OK) rc = ix->alloc(&ymax, 2);
    if (rc == RBC_OK)
      rc = ix->alloc(reinterpret_cast<uint16_t**>(&ix->ynblock), (n + NORM_PAD) * NBLOCK_COLS);
    if (rc == RBC_OK) rc = launch_offset_rows(ix->X32, ix->R32, ix->offsets, n_r, d, y32, st);
    if (rc == RBC_OK) {
      cudaError_t e = cudaMemsetAsync(ix->ynorm + n, 0, NORM_PAD * sizeof(float), st);
      if (e == cudaSuccess) e = cudaMemsetAsync(ymax, 0, 2 * sizeof(unsigned), st);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
    }
    if (rc == RBC_OK)
      rc = launch_to_lowp(y32, n, d, ix->dpad, ix->storage, yl, ix->ynorm, yerr, ymax, ymax + 1,
                          st);
    if (rc == RBC_OK) rc = launch_list_max(yerr, ix->offsets, n_r, ix->yerr_list, st);
    if (rc == RBC_OK) rc = launch_norm_block(ix->ynorm, n, n + NORM_PAD, ix->ynblock, st);
    if (rc == RBC_OK && ix->norm_fold_col >= 0)
      rc = launch_fold_norm(yl, ix->ynorm, n, ix->dpad, d, ix->storage, st);
    cudaFreeAsync(y32, st);
    RBC_TRY(rc);
    ix->Ylp = yl;
  }
  return RBC_OK;
}

int build_exact(rbc_index* ix, const float* Xdev, const std::vector<int64_t>& reps,
                cudaStream_t st) {
  const int64_t n = ix->n;
  const int d = ix->d, n_r = ix->n_r, metric = ix->metric;
  Arena ar(st);
  RBC_TRY(ix->alloc(&ix->reps, n_r));
  RBC_CUDA(cudaMemcpyAsync(ix->reps, reps.data(), n_r * sizeof(int64_t), cudaMemcpyHostToDevice,
                           st));
  RBC_TRY(ix->alloc(&ix->R32, (int64_t)n_r * d));
  RBC_TRY(launch_gather_rows(Xdev, ix->reps, nullptr, n_r, d, ix->R32, st));
  // BF(X, R): owner = nearest representative ordinal (ties to the smaller
  // ordinal = smaller id since R is sorted), owner distance
  int64_t* owner;
  float* odist;
  RBC_TRY(ar.alloc(&owner, n));
  RBC_TRY(ar.alloc(&odist, n));
  Counters cn;
  RBC_TRY(counters_alloc(cn, ar, st));
  DbView dbR;
  dbR.X32 = ix->R32;
  dbR.rows = n_r;
  RBC_TRY(bf_dense_f32(Xdev, n, dbR, d, 1, metric, nullptr, owner, odist, cn.c, ar, st, false));
  // lists: stable counting sort by owner
  ix->list_entries = n;
  RBC_TRY(ix->alloc(&ix->offsets, n_r + 1));
  RBC_TRY(ix->alloc(&ix->members, n));
  // lists by owner, each ordered by (rho(x, r), id): the order the stage-two
  // window search (Section 5.2's sorted lists) cuts ranges from
  int* scratch;
  RBC_TRY(ix->alloc(&ix->xdist, n));
  RBC_TRY(ar.alloc(&scratch, sort_lists_scratch_ints(n, n_r)));
  RBC_TRY(launch_sort_lists(owner, odist, n, n_r, ix->members, ix->offsets, ix->xdist, scratch,
                            st));
  RBC_TRY(ix->alloc(&ix->X32, n * d));
  RBC_TRY(launch_gather_rows(Xdev, nullptr, ix->members, n, d, ix->X32, st));
  // radii psi_r, inflated by the FP32 bound of the owner distances
  RBC_TRY(ix->alloc(&ix->psi, n_r));
  RBC_TRY(launch_list_radii(odist, ix->members, ix->offsets, n_r, 2.0f * rerank_eps_host(d),
                            ix->psi, st));
  RBC_TRY(make_lp_copies(ix, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  return RBC_OK;
}

// ---------------------------------------------------------------------------
// exact search (Section 5.2)
// ---------------------------------------------------------------------------
constexpr int64_t MAX_BATCH = 131072;  // queries per internal batch (bounds workspace)
constexpr int64_t WINDOW_MAX_PAIRS = 1LL << 28;  // windowed search: batch x n_r bound
constexpr int64_t ARENA_MIN_LANE = 256;  // hit records per epilogue thread, at least

int own_list_bound(const rbc_index* ix, const float* Qb, int64_t mb, const int64_t* nearest,
                   const LpQueries& ql, int k, float* own, uint32_t* dev_err, Arena& ar,
                   cudaStream_t st, int** order = nullptr);

int search_exact_batch(const rbc_index* ix, const float* Qb, int64_t mb, int k, int64_t* ids,
                       float* dist, const Counters& cn, int64_t* items_total, Arena& ar,
                       cudaStream_t st, bool f32_only = false, const float* g_cap = nullptr) {
  const int d = ix->d, n_r = ix->n_r, metric = ix->metric;
  const int64_t n = ix->list_entries;
  const int sms = sm_count();
  const bool lp = !f32_only && uses_lp(ix->storage, metric) && ix->Xlp != nullptr;
  const int64_t tiles = (mb + TQ - 1) / TQ;

  tmark(0, st);
  // stage 1: BF(Q, R) keeping every distance
  float* D;
  RBC_TRY(ar.alloc(&D, mb * n_r));
  TileWork w1{};
  w1.num_items = (int)tiles;
  w1.m = mb;
  w1.n = n_r;
  set_stage1_splits(w1, tiles, n_r, sms);
  RBC_TRY(launch_bf_simt_store(Qb, ix->R32, d, metric, w1, D, n_r,
                               (int)std::min<int64_t>(w1.num_items, (int64_t)sms * 2 * 16), st));
  float *g1, *gk;
  int64_t* nearest;
  RBC_TRY(ar.alloc(&g1, mb));
  RBC_TRY(ar.alloc(&gk, mb));
  RBC_TRY(ar.alloc(&nearest, mb));
  RBC_TRY(launch_row_stats(D, mb, n_r, k, g1, gk, nearest, st));
  // a caller that already knows an upper bound of each query's k-th neighbour
  // distance (the windowed search's own-list bound) tightens gamma_k with it
  if (g_cap) RBC_TRY(launch_gbound(g_cap, gk, mb, 0.0f, gk, st));
  // low-precision search: the own-list bound g = min(gamma_k, the k-th
  // distance inside the nearest representative's list) prunes more
  // surviving lists and bounds the FP32 re-search of uncertified queries
  uint32_t* dev_err;
  RBC_TRY(ar.alloc(&dev_err, 1));
  RBC_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(uint32_t), st));
  if (lp) {
    LpQueries qb;
    RBC_TRY(lp_queries(Qb, mb, d, ix->dpad, ix->storage, qb, ar, st));
    float* own;
    RBC_TRY(ar.alloc(&own, mb));
    RBC_TRY(own_list_bound(ix, Qb, mb, nearest, qb, k, own, dev_err, ar, st));
    RBC_TRY(launch_gbound(own, gk, mb, simt_eps(d), gk, st));
  }
  // queries ordered by nearest representative, so each tile holds nearby queries
  int *qperm, *qoff, *scratch;
  RBC_TRY(ar.alloc(&qperm, mb));
  RBC_TRY(ar.alloc(&qoff, n_r + 1));
  RBC_TRY(ar.alloc(&scratch, counting_sort_scratch_ints(mb, n_r)));
  RBC_TRY(launch_counting_sort(nearest, mb, n_r, qperm, qoff, scratch, st));
  float* Qp;
  RBC_TRY(ar.alloc(&Qp, mb * d));
  RBC_TRY(launch_gather_rows(Qb, nullptr, qperm, mb, d, Qp, st));
  // pruning -> per tile union of surviving lists
  const int words = (n_r + 31) / 32;
  uint32_t* tmask;
  int64_t* tpts;
  int* qkept;
  RBC_TRY(ar.alloc(&tmask, tiles * words));
  RBC_TRY(ar.alloc(&tpts, tiles));
  RBC_TRY(ar.alloc(&qkept, mb));
  RBC_TRY(launch_prune(D, qperm, mb, n_r, g1, gk, ix->psi, ix->offsets, simt_eps(d), tmask, tpts,
                       qkept, st));
  RBC_TRY(launch_sum_i32(qkept, mb, cn.sums, st));
  RBC_TRY(launch_sum_i64(tpts, tiles, cn.sums + 1, st));
  RBC_TRY(launch_sum_pairs(tpts, mb, cn.sums + 2, st));
  // work items
  int64_t W = (tiles * n + 16LL * sms - 1) / (16LL * sms);
  W = std::max<int64_t>(W, 4096);
  W = std::min<int64_t>(W, std::max<int64_t>(n, 1));
  W = (W + 255) / 256 * 256;
  const int item_cap = (int)((n + W - 1) / W) + 1;
  const int seg_cap = n_r + item_cap + 1;
  int *toff, *tcnt;
  RBC_TRY(ar.alloc(&toff, tiles + 1));
  RBC_TRY(ar.alloc(&tcnt, tiles));
  RBC_TRY(launch_item_offsets(tpts, (int)tiles, (int)W, tcnt, toff, st));
  WorkItem* items;
  Seg* segs;
  RBC_TRY(ar.alloc(&items, tiles * item_cap));
  RBC_TRY(ar.alloc(&segs, tiles * seg_cap));
  RBC_TRY(launch_workgen_items(tmask, ix->offsets, n_r, mb, (int)W, item_cap, seg_cap, toff, items,
                               segs, dev_err, st));
  *items_total += tiles * item_cap;
  TileWork w2{};
  w2.items = items;
  w2.num_items_dev = toff + tiles;
  w2.num_items = (int)(tiles * item_cap);
  w2.segs = segs;
  w2.m = mb;
  w2.n = n;
  DbView db;
  db.X32 = ix->X32;
  db.xid = ix->members;
  db.rows = n;
  db.Xlp = ix->Xlp;
  db.xnorm = ix->xnorm;
  db.xscale = ix->xscale;
  db.dpad = ix->dpad;
  db.lp_max = ix->lp_max;
  db.nblock = ix->xnblock;
  const int64_t cap_items = tiles * item_cap;
  if (!lp) {
    const int C = f32_list_width(k);
    const int c_out = f32_c_out(k);
    float* ps;
    int* pi;
    RBC_TRY(ar.alloc(&ps, cap_items * TQ * 2 * C));
    RBC_TRY(ar.alloc(&pi, cap_items * TQ * 2 * C));
    tmark(1, st);
    RBC_TRY(launch_bf_simt_topc(Qp, ix->X32, d, metric, C, w2, TopOut{ps, pi, nullptr},
                                (int)std::min<int64_t>(cap_items, (int64_t)sms * 2 * 8), st));
    tmark(2, st);
    SelectArgs a{};
    a.part_score = ps;
    a.part_idx = pi;
    a.C = C;
    a.nsub = 2;
    a.tile_slot_off = toff;
    a.m = mb;
    a.Q32 = Qp;
    a.d = d;
    a.metric = metric;
    a.qorig = qperm;
    a.X32 = ix->X32;
    a.xid = ix->members;
    a.simt_eps = simt_eps(d);
    a.k = k;
    a.c_out = c_out;
    a.out_ids = ids;
    a.out_dist = dist;
    int* fb;
    int* lc;  // [0] rows appended to fb, [1..2] ties
    RBC_TRY(ar.alloc(&fb, mb));
    RBC_TRY(ar.alloc(&lc, 8));
    RBC_CUDA(cudaMemsetAsync(lc, 0, 8 * sizeof(int), st));
    a.fallback_rows = fb;
    a.counters = lc;
    RBC_TRY(launch_select(a, st));
    RBC_TRY(launch_add_ints(cn.c, lc, 3, st));
    tmark(3, st);
    // uncertified rows: the FP64 band over the whole index (a superset of
    // their surviving lists)
    BandArgs bb = band_args(fb, lc, Qp, qperm, ix->X32, ix->members, n, d, k, metric, ids, dist);
    RBC_TRY(band_split_alloc(bb, ar));
    RBC_TRY(launch_band(bb, (int)mb, st));
    tmark(4, st);
  } else {
    const int c_out = choose_c(k, true, ix->rerank_c);
    const int C = lp_width(c_out);
    LpQueries ql;
    RBC_TRY(lp_queries(Qp, mb, d, ix->dpad, ix->storage, ql, ar, st));
    float* ps;
    int* pi;
    int* pv;
    RBC_TRY(ar.alloc(&ps, cap_items * TQ * 2 * C));
    RBC_TRY(ar.alloc(&pi, cap_items * TQ * 2 * C));
    RBC_TRY(ar.alloc(&pv, cap_items));
    LpMatrix Qm{ql.lp, ql.norm, mb, ix->dpad, ix->storage, nullptr, ql.scale};
    LpMatrix Xm{ix->Xlp, ix->xnorm, n, ix->dpad, ix->storage, ix->xnblock, ix->xscale};
    tmark(1, st);
    RBC_TRY(launch_bf_tc_topc(Qm, Xm, C, w2, TopOut{ps, pi, pv}, sms, st, dev_err));
    // the bound g of each sorted row, for the re-search of uncertified rows
    float* gp;
    RBC_TRY(ar.alloc(&gp, mb));
    RBC_TRY(launch_gather_rows(gk, nullptr, qperm, mb, 1, gp, st));
    RBC_TRY(select_lp_and_fallback(ps, pi, pv, C, toff, 0, mb, Qp, ql, db, d, k, c_out, qperm,
                                   ids, dist, cn.c, ar, st, 0, ix, gp));
  }
  uint32_t herr = 0;
  RBC_CUDA(cudaMemcpyAsync(&herr, dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  taccumulate();
  if (herr) {
    set_error("stage-two work generation / kernel reported device error flags 0x%x", herr);
    return (herr & DEV_ERR_TIMEOUT) ? RBC_ERR_TIMEOUT : RBC_ERR_CUDA;
  }
  return RBC_OK;
}

// Rows of a query buffer whose low-precision candidates could not be
// certified in an exact search are searched again by the FP32 exact search
// (CUDA cores) over the union of their own surviving lists -- a superset of
// what they need, and far less than every point of the index.  Row i's
// result goes to output row qorig[rows_dev[i]] (rows_dev[i] when qorig is
// null).  g_rows (optional, per row of the query buffer) bounds each
// query's k-th neighbour distance and tightens the pruning.  The nested
// search's phases count as the caller's re-search phase.
int fallback_rbc_f32(const rbc_index* ix, const float* Qbuf, const int* rows_dev, int nrows,
                     const int* qorig, int k, int64_t* out_ids, float* out_dist, int* cnt,
                     Arena& ar, cudaStream_t st, const float* g_rows) {
  if (nrows <= 0) return RBC_OK;
  const int d = ix->d;
  float* Qf;
  int* forig;
  int64_t* tid;
  float* tds;
  RBC_TRY(ar.alloc(&Qf, (int64_t)nrows * d));
  RBC_TRY(ar.alloc(&forig, nrows));
  RBC_TRY(ar.alloc(&tid, (int64_t)nrows * k));
  RBC_TRY(ar.alloc(&tds, (int64_t)nrows * k));
  RBC_TRY(launch_gather_rows(Qbuf, nullptr, rows_dev, nrows, d, Qf, st));
  RBC_TRY(launch_map_rows(rows_dev, nullptr, nrows, qorig, forig, st));
  float* gsub = nullptr;
  if (g_rows) {
    RBC_TRY(ar.alloc(&gsub, nrows));
    RBC_TRY(launch_gather_rows(g_rows, nullptr, rows_dev, nrows, 1, gsub, st));
  }
  Counters c2;
  RBC_TRY(ar.alloc(&c2.c, 8));
  RBC_TRY(ar.alloc(&c2.sums, 4));
  RBC_CUDA(cudaMemsetAsync(c2.c, 0, 8 * sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(c2.sums, 0, 4 * sizeof(unsigned long long), st));
  int64_t items = 0;
  const bool timing = t_timing.on;
  t_timing.on = false;
  const int rc = search_exact_batch(ix, Qf, nrows, k, tid, tds, c2, &items, ar, st, true, gsub);
  t_timing.on = timing;
  RBC_TRY(rc);
  RBC_TRY(launch_add_ints(cnt, c2.c, 3, st));
  return launch_scatter_result_rows(tid, tds, forig, nrows, k, out_ids, out_dist, st);
}


// ---------------------------------------------------------------------------
// one-shot build and search (Sections 4 and 5.1)
// ---------------------------------------------------------------------------
constexpr int ONESHOT_MAX_CAP = 16384;             // candidates a refine block can sort
constexpr int64_t ONESHOT_D_BYTES = 4LL << 30;     // distance block of the build

// BF(R, X) with k = s: L_r = the s nearest points of r by (rho, id), psi_r
// the s-th distance.  Representatives are processed in blocks whose FP32
// distance rows fit ONESHOT_D_BYTES.
int build_oneshot(rbc_index* ix, const float* Xdev, const std::vector<int64_t>& reps,
                  cudaStream_t st) {
  const int64_t n = ix->n;
  const int d = ix->d, n_r = ix->n_r, metric = ix->metric, s = ix->s;
  const int64_t entries = (int64_t)n_r * s;
  if (entries >= (1LL << 31)) {
    set_error("rbc_build: one-shot lists hold n_r * s = %lld entries (limit 2^31 - 1)",
              (long long)entries);
    return RBC_ERR_UNSUPPORTED;
  }
  Arena ar(st);
  RBC_TRY(ix->alloc(&ix->reps, n_r));
  RBC_CUDA(cudaMemcpyAsync(ix->reps, reps.data(), n_r * sizeof(int64_t), cudaMemcpyHostToDevice,
                           st));
  RBC_TRY(ix->alloc(&ix->R32, (int64_t)n_r * d));
  RBC_TRY(launch_gather_rows(Xdev, ix->reps, nullptr, n_r, d, ix->R32, st));
  ix->list_entries = entries;
  RBC_TRY(ix->alloc(&ix->members, entries));
  RBC_TRY(ix->alloc(&ix->psi, n_r));
  RBC_TRY(ix->alloc(&ix->offsets, n_r + 1));
  {
    std::vector<int> off((size_t)n_r + 1);
    for (int r = 0; r <= n_r; ++r) off[(size_t)r] = r * s;
    RBC_CUDA(cudaMemcpyAsync(ix->offsets, off.data(), off.size() * sizeof(int),
                             cudaMemcpyHostToDevice, st));
    RBC_CUDA(cudaStreamSynchronize(st));  // `off` leaves scope
  }
  int64_t rb = std::max<int64_t>(1, ONESHOT_D_BYTES / (n * (int64_t)sizeof(float)));
  rb = std::min<int64_t>(rb, n_r);
  if (rb > TQ) rb = rb / TQ * TQ;
  float* D;
  RBC_TRY(ar.alloc(&D, rb * n));
  uint32_t* dev_err;
  RBC_TRY(ar.alloc(&dev_err, 1));
  const int sms = sm_count();
  int cap = oneshot_candidate_cap(s);
  for (;;) {
    if (cap > ONESHOT_MAX_CAP) {
      set_error("rbc_build: more than %d points tie within rounding of a representative's s-th "
                "distance (s=%d)",
                ONESHOT_MAX_CAP, s);
      return RBC_ERR_UNSUPPORTED;
    }
    Arena car(st);
    int *cand, *ccnt;
    RBC_TRY(car.alloc(&cand, rb * cap));
    RBC_TRY(car.alloc(&ccnt, rb));
    RBC_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(uint32_t), st));
    for (int64_t r0 = 0; r0 < n_r; r0 += rb) {
      const int nb = (int)std::min<int64_t>(rb, n_r - r0);
      const int64_t tiles = (nb + TQ - 1) / TQ;
      int64_t splits = (8LL * sms + tiles - 1) / tiles;
      splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, n / 512)));
      int64_t chunk = (n + splits - 1) / splits;
      splits = (n + chunk - 1) / chunk;
      TileWork w{};
      w.num_items = (int)(tiles * splits);
      w.m = nb;
      w.n = n;
      w.dense_splits = (int)splits;
      w.dense_chunk = chunk;
      RBC_TRY(launch_bf_simt_store(ix->R32 + r0 * d, Xdev, d, metric, w, D, n,
                                   (int)std::min<int64_t>(w.num_items, (int64_t)sms * 2 * 16),
                                   st));
      RBC_TRY(launch_oneshot_select(D, n, n, nb, s, simt_eps(d), cap, cand, ccnt, dev_err, st));
      RBC_TRY(launch_oneshot_refine(Xdev, ix->R32, d, metric, s, cap, cand, ccnt, (int)r0, nb,
                                    ix->members, ix->psi, dev_err, st));
    }
    uint32_t herr = 0;
    RBC_CUDA(cudaMemcpyAsync(&herr, dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RBC_CUDA(cudaStreamSynchronize(st));
    if (herr & DEV_ERR_BOUNDS) {
      set_error("rbc_build: non-finite distances (X holds inf or NaN)");
      return RBC_ERR_ARG;
    }
    if (!(herr & DEV_ERR_CAPACITY)) break;
    cap = cap < ONESHOT_MAX_CAP ? std::min(ONESHOT_MAX_CAP, cap * 4) : cap * 2;
  }
  RBC_TRY(ix->alloc(&ix->X32, entries * d));
  RBC_TRY(launch_gather_rows(Xdev, nullptr, ix->members, entries, d, ix->X32, st));
  RBC_TRY(make_lp_copies(ix, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  return RBC_OK;
}

// Stage two of the one-shot search: query rows of `Qsrc` (mq of them) against
// the list of their representative rep_of[i]; results go to output row
// orig[i] (i when orig is null).  Lists are [r s, (r + 1) s) of the index's
// list storage, or [list_off[r], list_off[r + 1]) when list_off is given (the
// exact index's own lists, used by the windowed search for gamma bounds).  Queries are grouped by representative and
// every group padded to whole TQ-row tiles, so each tile is one dense item
// against exactly one list.  Low-precision rows that fail certification are
// searched again against their own list with the FP32 kernel.
// Queries grouped by representative: a counting sort by rep_of, each group
// padded to whole TQ-row tiles (padded rows map to -1), the gathered FP32
// query rows, and one work item per tile against its representative's list.
struct Grouped {
  int64_t max_tiles = 0, rows_cap = 0;
  int* qsrc = nullptr;      // padded row -> source row (or -1)
  int* qout = nullptr;      // padded row -> output row (or -1)
  int* tile_rep = nullptr;  // tile -> representative
  float* Qp = nullptr;      // [rows_cap, d]
  TileWork w{};             // the tiles as work items
};

int group_queries(const rbc_index* ix, const float* Qsrc, int64_t mq, const int64_t* rep_of,
                  const int* orig, const int* list_off, unsigned long long* points_sum, Grouped& gq,
                  Arena& ar, cudaStream_t st, bool gather_fp32 = true, int** order = nullptr) {
  const int d = ix->d, n_r = ix->n_r, s = ix->s;
  int *qperm, *qoff, *scratch;
  RBC_TRY(ar.alloc(&qperm, mq));
  RBC_TRY(ar.alloc(&qoff, n_r + 1));
  RBC_TRY(ar.alloc(&scratch, counting_sort_scratch_ints(mq, n_r)));
  RBC_TRY(launch_counting_sort(rep_of, mq, n_r, qperm, qoff, scratch, st));
  if (order) *order = qperm;
  gq.max_tiles = (mq + TQ - 1) / TQ + std::min<int64_t>(n_r, mq);
  gq.rows_cap = gq.max_tiles * TQ;
  int *pad_cnt, *pad_off;
  RBC_TRY(ar.alloc(&pad_cnt, n_r));
  RBC_TRY(ar.alloc(&pad_off, n_r + 1));
  RBC_TRY(ar.alloc(&gq.qsrc, gq.rows_cap));
  int* qsrc = gq.qsrc;
  RBC_TRY(ar.alloc(&gq.qout, gq.rows_cap));
  RBC_TRY(ar.alloc(&gq.tile_rep, gq.max_tiles));
  RBC_CUDA(cudaMemsetAsync(qsrc, 0xff, gq.rows_cap * sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(gq.qout, 0xff, gq.rows_cap * sizeof(int), st));
  RBC_TRY(launch_oneshot_layout(qoff, n_r, qperm, orig, pad_cnt, pad_off, qsrc, gq.qout,
                                gq.tile_rep, st));
  if (gather_fp32) {
    RBC_TRY(ar.alloc(&gq.Qp, gq.rows_cap * d));
    RBC_TRY(launch_gather_padded(Qsrc, qsrc, gq.rows_cap, d, gq.Qp, st));
  }
  WorkItem* items;
  Seg* segs;
  int* nitems;
  RBC_TRY(ar.alloc(&items, gq.max_tiles));
  RBC_TRY(ar.alloc(&segs, gq.max_tiles));
  RBC_TRY(ar.alloc(&nitems, 1));
  RBC_TRY(launch_oneshot_items(pad_off, n_r, gq.tile_rep, qoff, s, list_off, items, segs, nitems,
                               (int)gq.max_tiles, points_sum, st));
  gq.w = TileWork{};
  gq.w.items = items;
  gq.w.num_items_dev = nitems;
  gq.w.num_items = (int)gq.max_tiles;
  gq.w.segs = segs;
  gq.w.m = gq.rows_cap;
  gq.w.n = ix->list_entries;
  return RBC_OK;
}

// own[q] = the k-th smallest FP32 distance among the k best low-precision
// scores of q inside its nearest representative's list -- the distances of
// k actual points, so an upper bound of q's k-th neighbour distance (INF if
// that list holds fewer than k points).  Queries grouped by nearest
// representative, one tensor-core top-C pass over the own lists, FP32
// distances of the selected rows.  ql holds the batch's low-precision rows.
int own_list_bound(const rbc_index* ix, const float* Qb, int64_t mb, const int64_t* nearest,
                   const LpQueries& ql, int k, float* own, uint32_t* dev_err, Arena& ar,
                   cudaStream_t st, int** order) {
  Grouped gq;
  RBC_TRY(
      group_queries(ix, Qb, mb, nearest, nullptr, ix->offsets, nullptr, gq, ar, st, false, order));
  const int row_bytes = ix->dpad * lp_elem_bytes(ix->storage);
  uint8_t* alp;
  float *anorm, *aerr, *ascale = nullptr;
  RBC_TRY(ar.alloc(&alp, gq.rows_cap * row_bytes));
  RBC_TRY(ar.alloc(&anorm, gq.rows_cap));
  RBC_TRY(ar.alloc(&aerr, gq.rows_cap));
  if (ql.scale) RBC_TRY(ar.alloc(&ascale, gq.rows_cap));
  RBC_TRY(launch_gather_lp_rows(ql.lp, ql.norm, ql.err, gq.qsrc, gq.rows_cap, row_bytes, alp,
                                anorm, aerr, st, ql.scale, ascale));
  // 16-wide half-lists for k <= 16: with 8-wide ones the k best-scored
  // points of a row missed some of its k nearest often enough to loosen g
  // (measured: 107 of 100,000 queries overflowed, stage two 4.8 -> 7.0 ms)
  const int C = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  float* ps;
  int* pi;
  RBC_TRY(ar.alloc(&ps, gq.max_tiles * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pi, gq.max_tiles * TQ * 2 * C));
  LpMatrix Qm{alp, anorm, gq.rows_cap, ix->dpad, ix->storage, nullptr, ascale};
  LpMatrix Xm{ix->Xlp, ix->xnorm, ix->list_entries, ix->dpad, ix->storage, ix->xnblock,
              ix->xscale};
  TileWork wo = gq.w;
  wo.strided = true;  // one item per query tile: a popular list's tiles spread over CTAs
  RBC_TRY(launch_bf_tc_topc(Qm, Xm, C, wo, TopOut{ps, pi, nullptr}, sm_count(), st, dev_err));
  return launch_own_kth_lp(ps, pi, C, gq.qsrc, gq.rows_cap, k, Qb, ix->X32, ix->d, ix->metric,
                           rerank_eps_host(ix->d) + 8.0f * U32, own, st);
}

// The same bound from the FP32 CUDA-core top-C pass (FP32 storage or l1):
// the k best FP32 values of q inside its nearest representative's list,
// re-ranked, the largest of them rounded up.
int own_list_bound_f32(const rbc_index* ix, const float* Qb, int64_t mb, const int64_t* nearest,
                       int k, float* own, Arena& ar, cudaStream_t st, int** order = nullptr) {
  Grouped gq;
  RBC_TRY(
      group_queries(ix, Qb, mb, nearest, nullptr, ix->offsets, nullptr, gq, ar, st, true, order));
  const int C = simt_list_width((k + 1) / 2);  // half-lists: 2C >= k
  float* ps;
  int* pi;
  RBC_TRY(ar.alloc(&ps, gq.max_tiles * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pi, gq.max_tiles * TQ * 2 * C));
  const int sms = sm_count();
  RBC_TRY(launch_bf_simt_topc(gq.Qp, ix->X32, ix->d, ix->metric, C, gq.w, TopOut{ps, pi, nullptr},
                              (int)std::min<int64_t>(gq.max_tiles, (int64_t)sms * 2 * 8), st));
  return launch_own_kth_lp(ps, pi, C, gq.qsrc, gq.rows_cap, k, Qb, ix->X32, ix->d, ix->metric,
                           rerank_eps_host(ix->d) + 8.0f * U32, own, st);
}

int oneshot_stage2(const rbc_index* ix, const float* Qsrc, int64_t mq, const int64_t* rep_of,
                   const int* orig, bool lp, int k, int64_t* ids, float* dist, int* cnt,
                   unsigned long long* points_sum, int64_t* items_total, Arena& ar,
                   cudaStream_t st, bool marks, const int* list_off = nullptr) {
  if (mq == 0) return RBC_OK;
  const int d = ix->d, metric = ix->metric;
  const int64_t entries = ix->list_entries;
  const int sms = sm_count();
  Grouped gq;
  RBC_TRY(group_queries(ix, Qsrc, mq, rep_of, orig, list_off, points_sum, gq, ar, st));
  const int64_t max_tiles = gq.max_tiles, rows_cap = gq.rows_cap;
  float* Qp = gq.Qp;
  int* qout = gq.qout;
  int* tile_rep = gq.tile_rep;
  const TileWork& w = gq.w;
  if (items_total) *items_total += max_tiles;
  SelectArgs a{};
  a.nsub = 2;
  a.dense_splits = 1;  // slot of tile t is t
  a.m = rows_cap;
  a.Q32 = Qp;
  a.d = d;
  a.metric = metric;
  a.qorig = qout;
  a.X32 = ix->X32;
  a.xid = ix->members;
  a.k = k;
  a.out_ids = ids;
  a.out_dist = dist;
  if (!lp) {
    const int C = f32_list_width(k);
    const int c_out = f32_c_out(k);
    float* ps;
    int* pi;
    RBC_TRY(ar.alloc(&ps, max_tiles * TQ * 2 * C));
    RBC_TRY(ar.alloc(&pi, max_tiles * TQ * 2 * C));
    if (marks) tmark(1, st);
    RBC_TRY(launch_bf_simt_topc(Qp, ix->X32, d, metric, C, w, TopOut{ps, pi, nullptr},
                                (int)std::min<int64_t>(max_tiles, (int64_t)sms * 2 * 8), st));
    if (marks) tmark(2, st);
    a.part_score = ps;
    a.part_idx = pi;
    a.C = C;
    a.simt_eps = simt_eps(d);
    a.c_out = c_out;
    int* fb;
    int* lc;  // [0] rows appended to fb, [1..2] ties
    RBC_TRY(ar.alloc(&fb, rows_cap));
    RBC_TRY(ar.alloc(&lc, 8));
    RBC_CUDA(cudaMemsetAsync(lc, 0, 8 * sizeof(int), st));
    a.fallback_rows = fb;
    a.counters = lc;
    RBC_TRY(launch_select(a, st));
    RBC_TRY(launch_add_ints(cnt, lc, 3, st));
    if (marks) tmark(3, st);
    // uncertified rows: the FP64 band over the row's own list
    BandArgs b = band_args(fb, lc, Qp, qout, ix->X32, ix->members, entries, d, k, metric, ids,
                           dist);
    b.tile_list = tile_rep;
    b.list_off = list_off;
    b.list_len = ix->s;
    RBC_TRY(band_split_alloc(b, ar));
    RBC_TRY(launch_band(b, (int)rows_cap, st));
    if (marks) tmark(4, st);
    return RBC_OK;
  }
  const int c_out = choose_c(k, true, ix->rerank_c);
  const int C = lp_width(c_out);
  LpQueries ql;
  RBC_TRY(lp_queries(Qp, rows_cap, d, ix->dpad, ix->storage, ql, ar, st));
  float* ps;
  int* pi;
  int* pv;
  RBC_TRY(ar.alloc(&ps, max_tiles * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pi, max_tiles * TQ * 2 * C));
  RBC_TRY(ar.alloc(&pv, max_tiles));
  uint32_t* dev_err;
  RBC_TRY(ar.alloc(&dev_err, 1));
  RBC_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(uint32_t), st));
  LpMatrix Qm{ql.lp, ql.norm, rows_cap, ix->dpad, ix->storage, nullptr, ql.scale};
  LpMatrix Xm{ix->Xlp, ix->xnorm, entries, ix->dpad, ix->storage, ix->xnblock, ix->xscale};
  if (marks) tmark(1, st);
  RBC_TRY(launch_bf_tc_topc(Qm, Xm, C, w, TopOut{ps, pi, pv}, sms, st, dev_err));
  if (marks) tmark(2, st);
  int* fb_rows;
  int* lc;  // [0] rows appended to fb_rows, [1..2] ties
  RBC_TRY(ar.alloc(&fb_rows, rows_cap));
  RBC_TRY(ar.alloc(&lc, 8));
  RBC_CUDA(cudaMemsetAsync(lc, 0, 8 * sizeof(int), st));
  a.part_score = ps;
  a.part_idx = pi;
  a.slot_valid = pv;
  a.C = C;
  a.lp = 1;
  a.q_lpnorm = ql.norm;
  a.q_err = ql.err;
  a.x_err_max_bits = ix->lp_max;
  a.x_norm_max_bits = ix->lp_max + 1;
  a.c_out = c_out;
  a.fallback_rows = fb_rows;
  a.counters = lc;
  RBC_TRY(launch_select(a, st));
  if (marks) tmark(3, st);
  RBC_TRY(launch_add_ints(cnt, lc, 3, st));
  int nfb = 0;
  uint32_t herr = 0;
  RBC_CUDA(cudaMemcpyAsync(&nfb, lc, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBC_CUDA(cudaMemcpyAsync(&herr, dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    set_error("one-shot tensor-core pass reported device error flags 0x%x", herr);
    return (herr & DEV_ERR_TIMEOUT) ? RBC_ERR_TIMEOUT : RBC_ERR_CUDA;
  }
  if (nfb > 0) {
    int64_t* frep;
    int* forig;
    float* Qf;
    RBC_TRY(ar.alloc(&frep, nfb));
    RBC_TRY(ar.alloc(&forig, nfb));
    RBC_TRY(ar.alloc(&Qf, (int64_t)nfb * d));
    RBC_TRY(launch_oneshot_fallback_map(fb_rows, nfb, tile_rep, qout, frep, forig, st));
    RBC_TRY(launch_gather_rows(Qp, nullptr, fb_rows, nfb, d, Qf, st));
    RBC_TRY(oneshot_stage2(ix, Qf, nfb, frep, forig, false, k, ids, dist, cnt + 4, nullptr,
                           nullptr, ar, st, false, list_off));
  }
  if (marks) tmark(4, st);
  return RBC_OK;
}

// One-shot search of one query batch: r(q) = nearest representative by
// BF(Q, R) (k = 1, ties to the smaller ordinal, i.e. the smaller id), then
// BF(q, X[L_r(q)]).
int search_oneshot_batch(const rbc_index* ix, const float* Qb, int64_t mb, int k, int64_t* ids,
                         float* dist, const Counters& cn, int64_t* items_total, Arena& ar,
                         cudaStream_t st) {
  tmark(0, st);
  int64_t* nearest;
  float* ndist;
  int* c1;  // stage-one select counters (not part of the search statistics)
  RBC_TRY(ar.alloc(&nearest, mb));
  RBC_TRY(ar.alloc(&ndist, mb));
  RBC_TRY(ar.alloc(&c1, 8));
  RBC_CUDA(cudaMemsetAsync(c1, 0, 8 * sizeof(int), st));
  DbView dbR;
  dbR.X32 = ix->R32;
  dbR.rows = ix->n_r;
  RBC_TRY(bf_dense_f32(Qb, mb, dbR, ix->d, 1, ix->metric, nullptr, nearest, ndist, c1, ar, st,
                       false));
  const bool lp = uses_lp(ix->storage, ix->metric) && ix->Xlp != nullptr;
  RBC_TRY(oneshot_stage2(ix, Qb, mb, nearest, nullptr, lp, k, ids, dist, cn.c, cn.sums + 1,
                         items_total, ar, st, true));
  taccumulate();
  return RBC_OK;
}


// ---------------------------------------------------------------------------
// windowed exact search (Section 5.2 with lists sorted by rho(x, r))
// ---------------------------------------------------------------------------
// Qhost: the batch's rows in host memory, copied here into Qb (the batch's
// device buffer) chunk by chunk beside stage 1; null when Qb already holds them.
int search_window_batch(const rbc_index* ix, const float* Qb, int64_t mb, int k, int64_t* ids,
                        float* dist, const Counters& cn, int64_t* items_total, Arena& ar,
                        cudaStream_t st, const float* Qhost = nullptr) {
  const int d = ix->d, n_r = ix->n_r;
  const int64_t n = ix->list_entries;
  const int sms = sm_count();
  tmark(0, st);
  // stage 1: BF(Q, R) keeping every distance; gamma_1, gamma_k, nearest
  float* D;
  RBC_TRY(ar.alloc(&D, mb * n_r));
  float *g1, *gk;
  int64_t* nearest;
  RBC_TRY(ar.alloc(&g1, mb));
  RBC_TRY(ar.alloc(&gk, mb));
  RBC_TRY(ar.alloc(&nearest, mb));
  // bf16 / fp16 storage with l2: tensor-core passes on the low-precision rows;
  // otherwise (FP32 storage, l1) the same plan on the CUDA cores in FP32
  const bool lp = uses_lp(ix->storage, ix->metric) && ix->Xlp != nullptr;
  const int metric = ix->metric;
  const float f32_eps = simt_eps(d);
  // low-precision copy of the batch (pass A and the emission pass)
  LpQueries ql;
  if (lp) RBC_TRY(lp_queries_alloc(mb, ix->dpad, ix->storage, ql, ar));
  // every step up to here is per query row: with host rows, chunk by chunk
  // behind each chunk's copy
  cudaStream_t side = (Qhost && mb >= FEED_MIN_ROWS) ? feed_stream() : nullptr;
  const int64_t crows =
      side ? ((mb + FEED_CHUNKS - 1) / FEED_CHUNKS + TQ - 1) / TQ * TQ : std::max<int64_t>(mb, 1);
  FeedEvents fe;
  if (side) {
    for (cudaEvent_t& e : fe.ev) RBC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // the copies land in workspace allocated on the search's stream
    RBC_CUDA(cudaEventRecord(fe.ev[FEED_CHUNKS], st));
    RBC_CUDA(cudaStreamWaitEvent(side, fe.ev[FEED_CHUNKS], 0));
  }
  for (int64_t c0 = 0, ci = 0; c0 < mb; c0 += crows, ++ci) {
    const int64_t mc = std::min(crows, mb - c0);
    if (Qhost) {
      RBC_CUDA(cudaMemcpyAsync(const_cast<float*>(Qb) + c0 * d, Qhost + c0 * d,
                               (size_t)mc * d * sizeof(float), cudaMemcpyHostToDevice,
                               side ? side : st));
      if (side) {
        RBC_CUDA(cudaEventRecord(fe.ev[ci], side));
        RBC_CUDA(cudaStreamWaitEvent(st, fe.ev[ci], 0));
      }
    }
    const int64_t tiles = (mc + TQ - 1) / TQ;
    TileWork w1{};
    w1.num_items = (int)tiles;
    w1.m = mc;
    w1.n = n_r;
    set_stage1_splits(w1, tiles, n_r, sms);
    RBC_TRY(launch_bf_simt_store(Qb + c0 * d, ix->R32, d, ix->metric, w1, D + c0 * n_r, n_r,
                                 (int)std::min<int64_t>(w1.num_items, (int64_t)sms * 2 * 16),
                                 st));
    RBC_TRY(launch_row_stats(D + c0 * n_r, mc, n_r, k, g1 + c0, gk + c0, nearest + c0, st));
    if (lp) RBC_TRY(lp_queries_rows(Qb, c0, mc, d, ix->dpad, ql, st));
  }
  // device error flags of both tensor-core passes
  uint32_t* dev_err;
  RBC_TRY(ar.alloc(&dev_err, 1));
  RBC_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(uint32_t), st));
  // pass A: the k-th distance inside the nearest representative's own list
  // (and the batch's queries ordered by nearest representative)
  float* own;
  int* qorder = nullptr;
  RBC_TRY(ar.alloc(&own, mb));
  if (lp)
    RBC_TRY(own_list_bound(ix, Qb, mb, nearest, ql, k, own, dev_err, ar, st, &qorder));
  else
    RBC_TRY(own_list_bound_f32(ix, Qb, mb, nearest, k, own, ar, st, &qorder));
  float* g;
  RBC_TRY(ar.alloc(&g, mb));
  RBC_TRY(launch_gbound(own, gk, mb, simt_eps(d), g, st));
  // surviving (q, r) pairs binned by (r, bucket of rho(q, r))
  const int NB = window_buckets();
  const int64_t nbins = (int64_t)n_r * NB;
  int *totals, *bin_off, *blk_off;
  RBC_TRY(ar.alloc(&totals, nbins));
  RBC_TRY(ar.alloc(&bin_off, nbins + 1));
  RBC_TRY(ar.alloc(&blk_off, window_block_offsets(mb, n_r)));
  int* scan_scratch;
  RBC_TRY(ar.alloc(&scan_scratch, exclusive_scan_scratch_ints((int)nbins)));
  // representative offsets (an index built for them, FP32 queries 16-byte
  // aligned): the count pass also takes each query's largest pair M
  const bool offs = lp && ix->Ylp != nullptr && (reinterpret_cast<uintptr_t>(Qb) & 15) == 0;
  if (offs && stream_capturing(st)) {
    set_error("rbc_search: the offset plan reads its pair count back and cannot be recorded");
    return RBC_ERR_UNSUPPORTED;
  }
  unsigned *mq = nullptr, *meps = nullptr;  // per query: M, and eps of its rows (emission)
  if (offs) {
    RBC_TRY(ar.alloc(&mq, 2 * mb));
    meps = mq + mb;
    RBC_CUDA(cudaMemsetAsync(mq, 0, 2 * mb * sizeof(unsigned), st));
  }
  RBC_TRY(launch_window_pairs_count(D, mb, n_r, g, g1, ix->psi, simt_eps(d), totals, bin_off,
                                    blk_off, cn.sums, st, scan_scratch, mq));
  // pair arrays sized by the bound mb x n_r (batches are cut so that it stays
  // within WINDOW_MAX_PAIRS), so no count needs to come back to the host
  const int64_t pair_cap = mb * n_r;
  // score thresholds of the queries
  float* thr;
  RBC_TRY(ar.alloc(&thr, mb));
  RBC_TRY(launch_score_threshold(g, ql.norm, ql.err, ix->lp_max, d, mb, thr, st, f32_eps, metric));
  int2* pairs;  // (query, rho(q, r) bits)
  RBC_TRY(ar.alloc(&pairs, pair_cap));
  RBC_TRY(launch_window_pairs_scatter(D, mb, n_r, g, g1, ix->psi, simt_eps(d), bin_off, blk_off,
                                      pairs, st));
  // work items: chunks of TQ pairs, each with the union of its windows
  const int max_items = (int)std::min<int64_t>(pair_cap / TQ + n_r, INT32_MAX);
  int *ccount, *choff;
  EmitItem* items;
  RBC_TRY(ar.alloc(&ccount, n_r));
  RBC_TRY(ar.alloc(&choff, n_r + 1));
  RBC_TRY(ar.alloc(&items, std::max(max_items, 1)));
  RBC_TRY(launch_window_items(bin_off, NB, n_r, pairs, g, ix->offsets, ix->xdist, simt_eps(d),
                              2.0f * rerank_eps_host(d) + 8.0f * U32, ccount, choff, max_items,
                              items, cn.sums + 1, st));
  *items_total += max_items;
  // the tensor-core pass emitting candidates
  float* cs;
  int *cr, *cc;
  RBC_TRY(ar.alloc(&cs, mb * CAND_CAP));
  RBC_TRY(ar.alloc(&cr, mb * CAND_CAP));
  RBC_TRY(ar.alloc(&cc, mb));
  LpMatrix Qm{ql.lp, ql.norm, mb, ix->dpad, ix->storage};
  LpMatrix Xm{ix->Xlp, ix->xnorm, n, ix->dpad, ix->storage, ix->xnblock};
  // the main pass's database rows: the offsets y~ = bf16(x - r) on the offset plan
  LpMatrix Ym = offs ? LpMatrix{ix->Ylp, ix->ynorm, n, ix->dpad, ix->storage, ix->ynblock} : Xm;
  EmitOffsets eoff;
  if (offs) {
    // the kept pairs' query rows as offsets a~ = bf16(q - r), sized by the
    // pair count (read back: the one host wait this plan adds)
    int npairs = 0;
    RBC_CUDA(cudaMemcpyAsync(&npairs, bin_off + nbins, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBC_CUDA(cudaStreamSynchronize(st));
    uint8_t* arows;
    float *rowt, *rown;
    RBC_TRY(ar.alloc(&arows, (int64_t)std::max(npairs, 1) * ix->dpad * 2));
    RBC_TRY(ar.alloc(&rowt, npairs));
    RBC_TRY(ar.alloc(&rown, npairs));
    RBC_TRY(launch_offset_pair_rows(pairs, npairs, bin_off, NB, n_r, Qb, ix->R32, ix->psi,
                                    ix->yerr_list, g, d, ix->dpad, arows, rowt, rown, meps, sms,
                                    st));
    eoff.a_rows = arows;
    eoff.row_t = rowt;
    eoff.row_n = rown;
  }
  // hit arena: each epilogue thread appends its emissions to its own slice
  // (no atomics in the kernel); a post-pass fills the per-query buffers.  The
  // slices together hold 256 records per query of the batch (about 5x the
  // candidates of clustered 64-d data) and at least ARENA_MIN_LANE each: in a
  // small batch a chunk holds few queries, so a query with thousands of
  // candidates fills the slices of the few rows it occupies.  If one
  // overflows, the batch is emitted again with direct per-query appends, and
  // so are the index's next few searches.
  const int64_t nslices = (int64_t)sms * ARENA_SUBSEG * 32;
  const int arena_lane = (int)std::min<int64_t>(
      INT32_MAX / (4 * ARENA_SUBSEG * 32), std::max<int64_t>(ARENA_MIN_LANE, (mb * 256 + nslices - 1) / nslices));
  const int arena_seg = arena_lane * 32 * ARENA_SUBSEG;  // per CTA
  int4* arena;
  int *arena_cnt, *arena_ovf;
  if (lp) {
    RBC_TRY(ar.alloc(&arena, (int64_t)sms * arena_seg));
    RBC_TRY(ar.alloc(&arena_cnt, nslices));
    RBC_CUDA(cudaMemsetAsync(arena_cnt, 0, nslices * sizeof(int), st));
  } else {
    arena = nullptr;
    arena_cnt = nullptr;
  }
  RBC_TRY(ar.alloc(&arena_ovf, 1));
  int* fb_rows;
  int *lc, *lc2, *fb2, *srows, *srows2, *n_dense;
  RBC_TRY(ar.alloc(&fb_rows, mb));
  RBC_TRY(ar.alloc(&lc, 8));
  RBC_TRY(ar.alloc(&fb2, mb));
  RBC_TRY(ar.alloc(&lc2, 8));
  RBC_TRY(ar.alloc(&n_dense, 1));
  RBC_TRY(ar.alloc(&srows, mb));  // queries whose survivors are re-ranked in a stream
  RBC_TRY(ar.alloc(&srows2, mb));
  const int xspan = (int)std::max<int64_t>(4096, (n + 2 * sms - 1) / (2 * sms) / 256 * 256);
  const int nsplit = (int)((n + xspan - 1) / xspan);
  const int max2 = (int)std::min<int64_t>((mb + TQ - 1) / TQ * nsplit, INT32_MAX);
  EmitItem* items2;
  int* n_items2;
  RBC_TRY(ar.alloc(&items2, max2));
  RBC_TRY(ar.alloc(&n_items2, 1));
  CandSelectArgs a{};
  a.cand_score = cs;
  a.cand_row = cr;
  a.cand_cnt = cc;
  a.cap = CAND_CAP;
  a.m = mb;
  a.Q32 = Qb;
  a.d = d;
  a.metric = ix->metric;
  a.q_lpnorm = ql.norm;
  a.q_err = ql.err;
  a.x_err_max_bits = ix->lp_max;
  a.x_norm_max_bits = ix->lp_max + 1;
  a.X32 = ix->X32;
  a.xid = ix->members;
  a.k = k;
  a.c_out = std::min(k + 1, MAX_C);
  a.out_ids = ids;
  a.out_dist = dist;
  a.fallback_rows = fb_rows;
  a.counters = lc;
  a.stream_rows = srows;
  a.stream_count = lc + 4;
  a.f32 = lp ? 0 : 1;
  a.f32_eps = f32_eps;
  a.mq_bits = mq;  // offset estimates (the overflow pass's raw scores: a2 clears them)
  a.eps_bits = meps;
  // queries in nearest-representative order: the warps that run together
  // re-rank points of the same few lists, whose FP32 rows then come from L2
  a.rows = qorder;
  a.nrows = (int)mb;
  RBC_CUDA(cudaMemsetAsync(cc, 0, mb * sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(arena_ovf, 0, sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(lc, 0, 8 * sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(lc2, 0, 8 * sizeof(int), st));
  EmitOut eo{thr, cs, cr, cc, CAND_CAP};
  EmitOut eo_arena = eo;
  if (lp) {
    eo_arena.arena = arena;
    eo_arena.arena_seg = arena_seg;
    eo_arena.arena_cnt = arena_cnt;
    eo_arena.arena_ovf = arena_ovf;
  }
  tmark(1, st);
  // the CUDA-core emission appends to the per-query buffers directly
  if (lp)
    RBC_TRY(launch_bf_tc_emit(Qm, Ym, items, choff + n_r, max_items,
                              reinterpret_cast<const int*>(pairs), 2, eo_arena, sms, st, dev_err,
                              ix->norm_fold_col, offs ? &eoff : nullptr));
  else
    RBC_TRY(launch_bf_simt_emit(Qb, ix->X32, d, metric, items, choff + n_r, max_items,
                                reinterpret_cast<const int*>(pairs), 2, eo, 2 * sms, st));
  if (lp)
    RBC_TRY(launch_scatter_hits(arena, arena_lane, arena_cnt, (int)nslices, cs, cr, cc, CAND_CAP,
                                st));
  tmark(2, st);
  // exact re-rank of the candidates; overflowing queries are collected,
  // queries with more survivors than shared memory holds are streamed
  RBC_TRY(launch_select_cands(a, st));
  RBC_TRY(launch_select_stream(a, (int)mb, st));
  tmark(3, st);
  // Overflowing queries (count lc[0], on the device).  Up to mb / 16 + 64 of
  // them: k of their stored candidates give a much tighter threshold; they
  // are emitted again alone against the whole list storage (direct appends)
  // and finished.  More than that (clustered data whose points tie within
  // the rounding slack by the thousand: a dense pass would overflow again)
  // go straight to the exact finish below.  Every launch here reads its
  // count on the device, so with no overflow they find no work.
  RBC_TRY(launch_overflow_split(fb_rows, lc, (int)mb, (int)(mb / 16 + 64), n_dense, fb2, lc2, st));
  RBC_TRY(launch_overflow_rethreshold(fb_rows, n_dense, mb, cs, cc, CAND_CAP, k, ql.norm, ql.err,
                                      ix->lp_max, d, thr, st, f32_eps, metric, mq, meps));
  RBC_TRY(launch_dense_emit_items(n_dense, n, xspan, max2, items2, n_items2, st));
  if (lp)
    RBC_TRY(launch_bf_tc_emit(Qm, Xm, items2, n_items2, max2, fb_rows, 1, eo, sms, st, dev_err,
                              ix->norm_fold_col));
  else
    RBC_TRY(launch_bf_simt_emit(Qb, ix->X32, d, metric, items2, n_items2, max2, fb_rows, 1, eo,
                                2 * sms, st));
  CandSelectArgs a2 = a;
  a2.mq_bits = nullptr;
  a2.eps_bits = nullptr;
  a2.rows = fb_rows;
  a2.nrows_dev = n_dense;
  a2.nrows = (int)mb;
  a2.fallback_rows = fb2;
  a2.counters = lc2;
  a2.stream_rows = srows2;
  a2.stream_count = lc2 + 4;
  RBC_TRY(launch_select_cands(a2, st));
  RBC_TRY(launch_select_stream(a2, (int)mb, st));
  RBC_TRY(launch_add_ints(cn.c, lc, 3, st));
  RBC_TRY(launch_add_ints(cn.c + 4, lc2, 3, st));
  RBC_TRY(launch_sum_i32(cc, mb, cn.sums + 3, st));
  // Rows still left (fb2, count lc2[0]): more points than a buffer holds tie
  // within rounding.  Outside stream capture the count comes back and they
  // take the FP32 exact search over their surviving lists; a recorded
  // search reads nothing back: they are finished on the device by the FP64
  // band pass over the whole database, with g(q) bounding the band, and the
  // device error flags go to the index for rbc_search_check.
  if (stream_capturing(st)) {
    BandArgs bb = band_args(fb2, lc2, Qb, nullptr, ix->X32, ix->members, n, d, k, metric, ids,
                            dist);
    bb.kth_bound = g;
    RBC_TRY(band_split_alloc(bb, ar));
    RBC_TRY(launch_band(bb, (int)mb, st));
    RBC_TRY(launch_or_flags(ix->dev_status, dev_err, st));
  } else {
    int host[2] = {0, 0};  // rows left for the FP32 search, device error flags
    RBC_CUDA(cudaMemcpyAsync(&host[0], lc2, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBC_CUDA(cudaMemcpyAsync(&host[1], dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RBC_CUDA(cudaStreamSynchronize(st));
    if (host[1]) {
      set_error("windowed stage two reported device error flags 0x%x", (unsigned)host[1]);
      return (host[1] & DEV_ERR_TIMEOUT) ? RBC_ERR_TIMEOUT : RBC_ERR_CUDA;
    }
    if (host[0] > 0)
      RBC_TRY(fallback_rbc_f32(ix, Qb, fb2, host[0], nullptr, k, ids, dist, cn.c + 4, ar, st, g));
  }
  tmark(4, st);
  taccumulate();
  return RBC_OK;
}

// ---------------------------------------------------------------------------
// Workspace upper bound of rbc_search: the sum of every workspace request a
// call may make, term by term as the batch functions above allocate, with
// every data-dependent size at its maximum (all candidate lists MAX_C wide,
// every query of a batch falling back to the FP32 search).  A call holds the
// I/O copies and counters for its duration and one batch's arena at a time.
// ---------------------------------------------------------------------------
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// the band pass's chunk scratch, (rho64, id) entries
int64_t bound_band() { return band_split_scratch_entries() * 12; }
// bf_dense_f32 over `rows` queries against `db_rows` database rows (items =
// tiles x splits <= tiles + 8 SMs): partial lists, FP32 norms of both (l2),
// the rows to finish exactly, counters and the band pass's scratch
int64_t bound_dense_f32(int64_t rows, int sms, int64_t db_rows) {
  if (rows <= 0) return 0;
  return (cdiv(rows, TQ) + 8LL * sms) * TQ * 2 * MAX_C * 8 + db_rows * 4 + rows * 8 + 64 +
         bound_band();
}
int64_t bound_exact_batch(const rbc_index* ix, int64_t mb, int k, bool f32_only = false);
// fallback_rbc_f32 over `rows` rows: gathered rows, results, counters and the
// FP32 exact search
int64_t bound_fallback_rbc(const rbc_index* ix, int64_t rows, int k) {
  if (rows <= 0) return 0;
  return rows * ((int64_t)ix->d * 4 + 8 + (int64_t)k * 12) + 96 +
         bound_exact_batch(ix, rows, k, true);
}
// select_lp_and_fallback at level 0 over `rows` rows of an exact search
int64_t bound_select_lp(const rbc_index* ix, int64_t rows, int k) {
  return rows * 4 + 32 + bound_fallback_rbc(ix, rows, k);
}
// group_queries over mq rows
int64_t bound_group(const rbc_index* ix, int64_t mq, bool gather_fp32) {
  const int64_t n_r = ix->n_r;
  const int64_t max_tiles = cdiv(mq, TQ) + std::min<int64_t>(n_r, mq);
  const int64_t rows_cap = max_tiles * TQ;
  return mq * 4 + (n_r + 1) * 4 + counting_sort_scratch_ints(mq, (int)n_r) * 4 + n_r * 4 +
         (n_r + 1) * 4 + rows_cap * 8 + max_tiles * 4 + (gather_fp32 ? rows_cap * ix->d * 4 : 0) +
         max_tiles * (int64_t)(sizeof(WorkItem) + sizeof(Seg)) + 4;
}

// own_list_bound over mb queries (with its output own[mb])
int64_t bound_own_list(const rbc_index* ix, int64_t mb) {
  const int64_t max_tiles = cdiv(mb, TQ) + std::min<int64_t>(ix->n_r, mb);
  const int64_t rows_cap = max_tiles * TQ;
  return mb * 4 + bound_group(ix, mb, false) + rows_cap * ((int64_t)ix->dpad * 2 + 12) +
         rows_cap * 2 * MAX_C * 8;
}

int64_t bound_window_batch(const rbc_index* ix, int64_t mb, int k) {
  const int dpad = ix->dpad, sms = sm_count();
  const int64_t n_r = ix->n_r, n = ix->list_entries;
  const int64_t nbins = n_r * window_buckets();
  const int64_t nslices = (int64_t)sms * ARENA_SUBSEG * 32;
  const int64_t arena_lane = std::max<int64_t>(ARENA_MIN_LANE, cdiv(mb * 256, nslices));
  const int64_t xspan = std::max<int64_t>(4096, cdiv(n, 2LL * sms) / 256 * 256);
  const int64_t max2 = cdiv(mb, TQ) * cdiv(n, xspan);
  int64_t b = mb * n_r * 4;                                  // D
  b += mb * 16 + 4;                                          // g1, gk, nearest, dev_err
  b += mb * ((int64_t)dpad * 2 + 12);                         // low-precision batch
  b += bound_own_list(ix, mb);                               // pass A (tensor cores)
  b += bound_group(ix, mb, true) + cdiv(mb, TQ) * TQ * 2 * MAX_C * 8 +
       std::min<int64_t>(ix->n_r, mb) * TQ * 2 * MAX_C * 8;  // pass A (CUDA cores)
  b += mb * 4 + (ix->Ylp ? mb * 8 : 0);                      // g, offset M and eps per query
  if (ix->Ylp) b += mb * n_r * ((int64_t)dpad * 2 + 8) + 256;  // offset rows of the pairs
  b += nbins * 8 + 4 + window_block_offsets(mb, n_r) * 4;   // totals, offsets, block offsets
  b += ((int64_t)exclusive_scan_scratch_ints((int)nbins)) * 4; // their scan
  b += mb * 4 + mb * n_r * 8;                                // thr, pairs
  b += n_r * 8 + 4 + (mb * n_r / TQ + n_r) * (int64_t)sizeof(EmitItem);  // chunks, items
  b += mb * (int64_t)CAND_CAP * 8 + mb * 4;                  // candidate buffers
  b += nslices * arena_lane * 16 + nslices * 4 + 4;          // hit arena
  b += mb * 16 + 64;                                         // fallback / stream rows, counters
  b += max2 * (int64_t)sizeof(EmitItem) + 4;                 // overflow items
  b += bound_fallback_rbc(ix, mb, k);                       // FP32 exact search of the rest
  b += bound_band();                                         // band pass (recorded searches)
  return b;
}

int64_t bound_exact_batch(const rbc_index* ix, int64_t mb, int k, bool f32_only) {
  const int d = ix->d, dpad = ix->dpad, sms = sm_count();
  const int64_t n_r = ix->n_r, n = ix->list_entries;
  const int64_t tiles = cdiv(mb, TQ);
  int64_t W = (tiles * n + 16LL * sms - 1) / (16LL * sms);
  W = std::max<int64_t>(W, 4096);
  W = std::min<int64_t>(W, std::max<int64_t>(n, 1));
  W = (W + 255) / 256 * 256;
  const int64_t item_cap = cdiv(n, W) + 1, seg_cap = n_r + item_cap + 1;
  const int64_t cap_items = tiles * item_cap;
  int64_t b = mb * n_r * 4 + mb * 16;                        // D, g1, gk, nearest
  b += mb * 4 + (n_r + 1) * 4 + counting_sort_scratch_ints(mb, (int)n_r) * 4;
  b += mb * (int64_t)d * 4;                                  // ordered queries
  b += tiles * cdiv(n_r, 32) * 4 + tiles * 8 + mb * 4;       // masks, points, kept
  b += (tiles + 1) * 4 + tiles * 4;                          // item offsets
  b += cap_items * (int64_t)sizeof(WorkItem) + tiles * seg_cap * (int64_t)sizeof(Seg) + 4;
  b += cap_items * TQ * 2 * MAX_C * 8 + cap_items * 4;       // partial lists
  b += bound_band();                                         // band pass (FP32 lists)
  if (!f32_only && uses_lp(ix->storage, ix->metric) && ix->Xlp) {
    b += 2 * mb * ((int64_t)dpad * 2 + 12);                   // low-precision batch, twice
    b += bound_own_list(ix, mb) + mb * 4;                      // own-list bound, sorted g
    b += bound_select_lp(ix, mb, k);
  }
  return b;
}

int64_t bound_oneshot_stage2(const rbc_index* ix, int64_t mq, bool lp, int level) {
  if (mq <= 0) return 0;
  const int d = ix->d, dpad = ix->dpad, sms = sm_count();
  const int64_t max_tiles = cdiv(mq, TQ) + std::min<int64_t>(ix->n_r, mq);
  const int64_t rows_cap = max_tiles * TQ;
  int64_t b = bound_group(ix, mq, true);
  b += max_tiles * TQ * 2 * MAX_C * 8 + max_tiles * 4 + 4;   // partial lists, valid, dev_err
  b += bound_band();                                         // band pass (FP32 lists)
  if (lp) {
    b += rows_cap * ((int64_t)dpad * 2 + 12);                 // low-precision rows
    b += rows_cap * 4 + 32;                                  // fallback rows, counters
    b += rows_cap * (8 + 4 + (int64_t)d * 4);                // fallback gather
    if (level == 0) b += bound_oneshot_stage2(ix, rows_cap, false, 1);
  }
  (void)sms;
  return b;
}

int64_t bound_oneshot_batch(const rbc_index* ix, int64_t mb) {
  const bool lp = uses_lp(ix->storage, ix->metric) && ix->Xlp != nullptr;
  return mb * 12 + 32 + bound_dense_f32(mb, sm_count(), ix->n_r) + bound_oneshot_stage2(ix, mb, lp, 0);
}

// the batch size rbc_search cuts a call into
int64_t search_batch_size(const rbc_index* ix, bool window) {
  return window ? std::max<int64_t>(TQ, std::min<int64_t>(MAX_BATCH, WINDOW_MAX_PAIRS / ix->n_r))
                : MAX_BATCH;
}
// the windowed plan's emission kernel folds -|x~|^2/2 into the MMA and tests
// row maxima, which needs one scale per row: FP8 (a scale per column too)
// takes the tile-union plan
bool search_uses_window(const rbc_index* ix) {
  if (ix->mode != RBC_EXACT || ix->plan == RBC_PLAN_TILE_UNION) return false;
  // FP32 storage or l1: the windowed plan on the CUDA cores
  if (!uses_lp(ix->storage, ix->metric)) return true;
  return ix->Xlp && ix->storage != RBC_FP8E4M3;
}

int64_t search_workspace_bound(const rbc_index* ix, int64_t m, int k) {
  const bool window = search_uses_window(ix);
  const int64_t mb = std::min<int64_t>(std::max<int64_t>(m, 1), search_batch_size(ix, window));
  int64_t b = m * ((int64_t)ix->d * 4 + (int64_t)k * 12);   // host I/O copies
  b += 64 + 64;                                              // counters, packed statistics
  if (ix->mode == RBC_ONESHOT)
    b += bound_oneshot_batch(ix, mb);
  else if (window)
    b += bound_window_batch(ix, mb, k);
  else
    b += bound_exact_batch(ix, mb, k);
  return b;
}

}  // namespace

void stats_publish_static(const int* counters_dev, int64_t queries, int64_t pairs,
                          cudaStream_t st) {
  memset(&t_stats_fixed, 0, sizeof(t_stats_fixed));
  t_stats_fixed.queries = queries;
  t_stats_fixed.pairs = pairs;
  t_stats_fixed.kernel_launches = t_launches;
  t_stats_host_kept = -1;
  t_stats_stream = st;
  t_stats_pending = true;
  t_stats_counters_dev = counters_dev;
}

}  // namespace rbc

// ===========================================================================
// C ABI
// ===========================================================================
using namespace rbc;

extern "C" {

void rbc_default_opts(rbc_opts* o) {
  if (o) memset(o, 0, sizeof(*o));
}

const char* rbc_last_error(void) { return last_error_text(); }

int rbc_sample_reps(int64_t n, int32_t n_r, uint64_t seed, int64_t* out) {
  if (n < 1 || n_r < 1 || n_r > n || !out) {
    set_error("rbc_sample_reps: need 1 <= n_r <= n and out != NULL (n=%lld n_r=%d)",
              (long long)n, n_r);
    return RBC_ERR_ARG;
  }
  std::vector<int64_t> r = sample_reps_host(n, n_r, seed);
  memcpy(out, r.data(), r.size() * sizeof(int64_t));
  return RBC_OK;
}

int rbc_last_stats(rbc_search_stats* out) {
  if (!out) {
    set_error("rbc_last_stats: NULL");
    return RBC_ERR_ARG;
  }
  if (t_stats_pending && t_stats_counters_dev) {
    cudaError_t e = cudaStreamSynchronize(t_stats_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    int c[8] = {0};
    e = cudaMemcpy(c, t_stats_counters_dev, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy", __FILE__, __LINE__);
    t_stats_fixed.uncertified = c[0];
    t_stats_fixed.fp64_ties = c[1];
    t_stats_fixed.boundary_ties = c[2];
    t_stats_pending = false;
    t_stats_counters_dev = nullptr;
  }
  if (t_stats_pending) {
    cudaError_t e = cudaStreamSynchronize(t_stats_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    const unsigned long long* v = t_stats_holder.p->v;
    t_stats_fixed.kept_reps = t_stats_host_kept >= 0 ? t_stats_host_kept : (int64_t)v[0];
    t_stats_fixed.tile_points = (int64_t)v[1];
    t_stats_fixed.candidates = (int64_t)v[7];
    t_stats_fixed.uncertified = (int64_t)v[2];
    t_stats_fixed.fp64_ties = (int64_t)v[3];
    t_stats_fixed.boundary_ties = (int64_t)v[4];
    if (v[6]) t_stats_fixed.pairs = (int64_t)v[6];
    t_stats_pending = false;
  }
  *out = t_stats_fixed;
  return RBC_OK;
}

int bf_search(const float* Q, int64_t m, const float* X, int64_t n, int32_t d, int32_t k,
              int32_t metric, int32_t storage, int64_t* out_ids, float* out_dist, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (m < 0 || n < 1 || d < 1 || k < 1 || n >= (1LL << 31) || m >= (1LL << 31)) {
    set_error("bf_search: bad sizes m=%lld n=%lld d=%d k=%d", (long long)m, (long long)n, d, k);
    return RBC_ERR_ARG;
  }
  RBC_TRY(valid_enums(metric, storage));
  if (!X || (m > 0 && (!Q || !out_ids || !out_dist))) {
    set_error("bf_search: NULL pointer");
    return RBC_ERR_ARG;
  }
  if (k > MAX_C - 1) {
    set_error("bf_search: k=%d exceeds the supported maximum %d", k, MAX_C - 1);
    return RBC_ERR_UNSUPPORTED;
  }
  if (d > MAX_D) {
    set_error("bf_search: d=%d exceeds %d", d, MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  Arena ar(st);
  IoPlan io;
  RBC_TRY(io_prepare(Q, m, d, k, out_ids, out_dist, io, ar, st));
  const float* Xdev = X;
  if (!is_device_ptr(X)) {
    float* x;
    RBC_TRY(ar.alloc(&x, n * d));
    RBC_CUDA(cudaMemcpyAsync(x, X, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, st));
    Xdev = x;
  }
  Counters cn;
  RBC_TRY(counters_alloc(cn, ar, st));
  DbView db;
  db.X32 = Xdev;
  db.rows = n;
  tmark(0, st);
  if (!uses_lp(storage, metric)) {
    RBC_TRY(bf_dense_f32(io.Qdev, m, db, d, k, metric, nullptr, io.ids_dev, io.dist_dev, cn.c,
                         ar, st));
    taccumulate();
  } else {
    db.dpad = lp_pad(d, storage);
    uint8_t* xl;
    float* xn;
    float* xs = nullptr;
    unsigned* mx;
    RBC_TRY(ar.alloc(&xl, n * db.dpad * lp_elem_bytes(storage)));
    RBC_TRY(ar.alloc(&xn, n + NORM_PAD));
    RBC_CUDA(cudaMemsetAsync(xn + n, 0, NORM_PAD * sizeof(float), st));
    if (storage == RBC_FP8E4M3) {
      RBC_TRY(ar.alloc(&xs, n + NORM_PAD));
      RBC_CUDA(cudaMemsetAsync(xs + n, 0, NORM_PAD * sizeof(float), st));
    }
    RBC_TRY(ar.alloc(&mx, 2));
    RBC_CUDA(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned), st));
    RBC_TRY(launch_to_lowp(Xdev, n, d, db.dpad, storage, xl, xn, nullptr, mx, mx + 1, st, xs));
    if (storage != RBC_FP8E4M3) {
      // -|x~|^2 / 2 as a bf16 (high, low) block: the tensor-core pass adds it
      // to its accumulators with one extra MMA
      uint16_t* nb;
      RBC_TRY(ar.alloc(&nb, (n + NORM_PAD) * NBLOCK_COLS));
      RBC_TRY(launch_norm_block(xn, n, n + NORM_PAD, nb, st));
      db.nblock = nb;
    }
    db.Xlp = xl;
    db.xnorm = xn;
    db.xscale = xs;
    db.lp_max = mx;
    RBC_TRY(bf_dense_lp(io.Qdev, m, db, d, k, storage, 0, io.ids_dev, io.dist_dev, cn.c, ar, st));
  }
  RBC_TRY(stats_publish(cn, m, 0, m * n, ar, st));
  RBC_TRY(io_finish(m, k, out_ids, out_dist, io, st));
  return RBC_OK;
}

int rbc_set_timing(int on) {
  int prev = t_timing.on ? 1 : 0;
  t_timing.on = on != 0;
  return prev;
}

int rbc_build(const float* X, int64_t n, int32_t d, int32_t n_r, int32_t s, int32_t metric,
              const rbc_opts* opts, void* stream, rbc_index** out) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!out || !X) {
    set_error("rbc_build: NULL pointer");
    return RBC_ERR_ARG;
  }
  *out = nullptr;
  rbc_opts o;
  rbc_default_opts(&o);
  if (opts) o = *opts;
  if (n < 1 || d < 1 || n_r < 1 || n_r > n || n >= (1LL << 31)) {
    set_error("rbc_build: bad sizes n=%lld d=%d n_r=%d", (long long)n, d, n_r);
    return RBC_ERR_ARG;
  }
  RBC_TRY(valid_enums(metric, o.storage));
  if (o.mode != RBC_EXACT && o.mode != RBC_ONESHOT) {
    set_error("rbc_build: unknown mode %d", o.mode);
    return RBC_ERR_ARG;
  }
  if (o.mode == RBC_ONESHOT && (s < 1 || s > n)) {
    set_error("rbc_build: one-shot needs 1 <= s <= n (s=%d)", s);
    return RBC_ERR_ARG;
  }
  if (o.rerank_c < 0 || o.rerank_c > MAX_C ||
      (o.plan != RBC_PLAN_WINDOW && o.plan != RBC_PLAN_TILE_UNION &&
       o.plan != RBC_PLAN_WINDOW_OFFSET)) {
    set_error("rbc_build: rerank_c must be in [0, %d] and plan RBC_PLAN_WINDOW, "
              "RBC_PLAN_TILE_UNION or RBC_PLAN_WINDOW_OFFSET", MAX_C);
    return RBC_ERR_ARG;
  }
  if (d > MAX_D) {
    set_error("rbc_build: d=%d exceeds %d", d, MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  std::vector<int64_t> reps;
  if (o.rep_ids) {
    reps.assign(o.rep_ids, o.rep_ids + n_r);
    for (int i = 0; i < n_r; ++i)
      if (reps[i] < 0 || reps[i] >= n || (i && reps[i] <= reps[i - 1])) {
        set_error("rbc_build: rep_ids must be ascending, distinct and inside [0, n)");
        return RBC_ERR_ARG;
      }
  } else {
    reps = sample_reps_host(n, n_r, o.seed);
  }
  rbc_index* ix = new (std::nothrow) rbc_index();
  if (!ix) {
    set_error("rbc_build: host allocation failed");
    return RBC_ERR_OOM;
  }
  ix->n = n;
  ix->d = d;
  ix->n_r = n_r;
  ix->s = s;
  ix->metric = metric;
  ix->mode = o.mode;
  ix->storage = o.storage;
  ix->rerank_c = o.rerank_c;
  ix->plan = o.plan;
  cudaGetDevice(&ix->device);
  int rc;
  {
    Arena ar(st);
    const float* Xdev = X;
    rc = ix->alloc(&ix->dev_status, 1);
    if (rc == RBC_OK) {
      cudaError_t e = cudaMemsetAsync(ix->dev_status, 0, sizeof(uint32_t), st);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
    }
    if (rc == RBC_OK && !is_device_ptr(X)) {
      float* x = nullptr;
      rc = ar.alloc(&x, n * d);
      if (rc == RBC_OK) {
        cudaError_t e =
            cudaMemcpyAsync(x, X, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
      }
      Xdev = x;
    }
    if (rc == RBC_OK)
      rc = o.mode == RBC_ONESHOT ? build_oneshot(ix, Xdev, reps, st)
                                 : build_exact(ix, Xdev, reps, st);
  }
  if (rc != RBC_OK) {
    cudaStreamSynchronize(st);
    delete ix;
    return rc;
  }
  *out = ix;
  return RBC_OK;
}

int rbc_search(const rbc_index* ix, const float* Q, int64_t m, int32_t k, int64_t* out_ids,
               float* out_dist, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!ix || (m > 0 && (!Q || !out_ids || !out_dist))) {
    set_error("rbc_search: NULL pointer");
    return RBC_ERR_ARG;
  }
  if (m < 0 || k < 1 || k > ix->n || m >= (1LL << 31)) {
    set_error("rbc_search: bad sizes m=%lld k=%d (n=%lld)", (long long)m, k, (long long)ix->n);
    return RBC_ERR_ARG;
  }
  if (ix->mode == RBC_ONESHOT && k > ix->s) {
    set_error("rbc_search: one-shot lists hold s=%d points, k=%d", ix->s, k);
    return RBC_ERR_ARG;
  }
  if (k > MAX_C - 1) {
    set_error("rbc_search: k=%d exceeds the supported maximum %d", k, MAX_C - 1);
    return RBC_ERR_UNSUPPORTED;
  }
  const int64_t ws0 = t_ws_cur;
  t_ws_peak = t_ws_cur;
  int64_t items = 0;
  const bool window = search_uses_window(ix);
  if (stream_capturing(st)) {
    // a recorded search may read nothing back: the windowed plan only, with
    // device-resident inputs and outputs and no phase timing
    if (!window || ix->Ylp) {
      set_error("rbc_search: under stream capture the index must use the windowed plan "
                "without offsets (exact mode, FP32 / bf16 / fp16 storage)");
      return RBC_ERR_UNSUPPORTED;
    }
    if (m > 0 && (!is_device_ptr(Q) || !is_device_ptr(out_ids) || !is_device_ptr(out_dist))) {
      set_error("rbc_search: under stream capture Q and the outputs must be device memory");
      return RBC_ERR_ARG;
    }
    if (t_timing.on) {
      set_error("rbc_search: phase timing (rbc_set_timing) cannot be recorded in a graph");
      return RBC_ERR_UNSUPPORTED;
    }
  }
  // the windowed search sizes its pair arrays by batch x n_r
  const int64_t batch = search_batch_size(ix, window);
  {
    Arena ar(st);
    IoPlan io;
    // the windowed plan copies host query rows batch by batch, beside stage 1
    RBC_TRY(io_prepare(Q, m, ix->d, k, out_ids, out_dist, io, ar, st, window));
    Counters cn;
    RBC_TRY(counters_alloc(cn, ar, st));
    for (int64_t b0 = 0; b0 < m; b0 += batch) {
      int64_t mb = std::min<int64_t>(batch, m - b0);
      Arena bar(st);
      if (ix->mode == RBC_ONESHOT)
        RBC_TRY(search_oneshot_batch(ix, io.Qdev + b0 * ix->d, mb, k, io.ids_dev + b0 * k,
                                     io.dist_dev + b0 * k, cn, &items, bar, st));
      else if (window)
        RBC_TRY(search_window_batch(ix, io.Qdev + b0 * ix->d, mb, k, io.ids_dev + b0 * k,
                                    io.dist_dev + b0 * k, cn, &items, bar, st,
                                    io.Qhost ? io.Qhost + b0 * ix->d : nullptr));
      else
        RBC_TRY(search_exact_batch(ix, io.Qdev + b0 * ix->d, mb, k, io.ids_dev + b0 * k,
                                   io.dist_dev + b0 * k, cn, &items, bar, st));
    }
    if (ix->mode == RBC_ONESHOT)
      RBC_TRY(stats_publish(cn, m, items, m * (int64_t)ix->s, ar, st, m));
    else
      RBC_TRY(stats_publish(cn, m, items, 0, ar, st));
    RBC_TRY(io_finish(m, k, out_ids, out_dist, io, st));
  }
  t_stats_fixed.workspace_bytes = t_ws_peak - ws0;
  return RBC_OK;
}

int rbc_search_check(const rbc_index* ix, void* stream) {
  if (!ix) {
    set_error("rbc_search_check: NULL index");
    return RBC_ERR_ARG;
  }
  RBC_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  uint32_t f = 0;
  RBC_CUDA(cudaMemcpy(&f, ix->dev_status, sizeof(f), cudaMemcpyDeviceToHost));
  if (!f) return RBC_OK;
  RBC_CUDA(cudaMemset(ix->dev_status, 0, sizeof(f)));
  set_error("a recorded search reported device error flags 0x%x", (unsigned)f);
  return (f & DEV_ERR_TIMEOUT) ? RBC_ERR_TIMEOUT : RBC_ERR_CUDA;
}

int rbc_search_workspace(const rbc_index* ix, int64_t m, int32_t k, int64_t* bytes) {
  if (!ix || !bytes || m < 0 || k < 1) {
    set_error("rbc_search_workspace: NULL pointer or bad sizes (m=%lld k=%d)", (long long)m, k);
    return RBC_ERR_ARG;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != ix->device) cudaSetDevice(ix->device);  // the bound reads this device's SM count
  *bytes = search_workspace_bound(ix, m, k);
  if (dev != ix->device) cudaSetDevice(dev);
  return RBC_OK;
}

int rbc_index_info(const rbc_index* ix, rbc_index_desc* out) {
  if (!ix || !out) {
    set_error("rbc_index_info: NULL");
    return RBC_ERR_ARG;
  }
  out->n = ix->n;
  out->d = ix->d;
  out->n_r = ix->n_r;
  out->s = ix->s;
  out->metric = ix->metric;
  out->mode = ix->mode;
  out->storage = ix->storage;
  out->list_entries = ix->list_entries;
  out->device_bytes = ix->bytes;
  out->device = ix->device;
  return RBC_OK;
}

int rbc_index_export(const rbc_index* ix, int64_t* reps, int64_t* offsets, int64_t* members,
                     float* psi) {
  if (!ix) {
    set_error("rbc_index_export: NULL index");
    return RBC_ERR_ARG;
  }
  // the build synchronised its stream before returning, so the index is complete
  if (reps)
    RBC_CUDA(cudaMemcpy(reps, ix->reps, ix->n_r * sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (offsets) {
    std::vector<int> o(ix->n_r + 1);
    RBC_CUDA(cudaMemcpy(o.data(), ix->offsets, o.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < o.size(); ++i) offsets[i] = o[i];
  }
  if (members) {
    std::vector<int> mm((size_t)ix->list_entries);
    RBC_CUDA(cudaMemcpy(mm.data(), ix->members, mm.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < mm.size(); ++i) members[i] = mm[i];
  }
  if (psi) RBC_CUDA(cudaMemcpy(psi, ix->psi, ix->n_r * sizeof(float), cudaMemcpyDeviceToHost));
  return RBC_OK;
}

int rbc_trim_workspace(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_POOL_DEVICES) {
    cudaGetLastError();
    set_error("rbc_trim_workspace: no current device");
    return RBC_ERR_CUDA;
  }
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    pool = g_pools[dev];
  }
  if (!pool) return RBC_OK;
  RBC_CUDA(cudaDeviceSynchronize());
  RBC_CUDA(cudaMemPoolTrimTo(pool, 0));
  return RBC_OK;
}

void rbc_free(rbc_index* ix) {
  // cudaFree waits for outstanding device work that may still read the index
  delete ix;
}

}  // extern "C"
