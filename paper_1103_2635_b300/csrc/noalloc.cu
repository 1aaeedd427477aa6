// bf_search_noalloc: the FP32 brute-force search for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: for example a serving
// process whose engine has already reserved the device memory budget for its
// own pool, or a latency-critical path where an allocation (which may
// synchronise the device or fail under memory pressure) is not acceptable.
// This entry point gives them BF(Q, X) with the FP32 CUDA-core kernels and no
// allocation at all: every buffer the search needs besides its inputs and
// outputs lives in one file-scope static device array of fixed size.
//
// The array belongs to the library's module: every GPU that loads the library
// holds it until the process exits, and every call shares it, so calls that
// overlap on the GPU (different streams, threads or processes sharing a
// context) race on it and must be serialised by the caller.  Its contents
// persist between calls; the counters that must start at zero are cleared at
// the start of each call (a memset of the array, not an allocation).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace rbc {
namespace {

// Scratch shared by all bf_search_noalloc calls on a device.
constexpr size_t NOALLOC_SCRATCH_BYTES = 32u << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array for the current device.  In host code
// `g_noalloc_scratch` is only a host-side stand-in for the symbol, so the
// address is looked up once per device (with that device current, on the
// first call there) and cached for the life of the process.
int scratch_for_current_device(int dev, void** out) {
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("bf_search_noalloc: device ordinal %d out of range", dev);
    return RBC_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RBC_OK;
}

// A device (or managed) pointer usable on the current device: the scratch
// belongs to the current device, so buffers of another GPU are refused
// rather than reached through unified addressing.
bool on_current_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Scratch layout of a call: [256-byte head: 8 int counters] [re-search rows:
// m ints, rounded up to 256 bytes] [partial candidate lists: items x 128
// rows x 2 halves x C x (score, column)].
constexpr size_t NOALLOC_HEAD = 256;
size_t rows_bytes(int64_t m) { return ((size_t)m * 4 + 255) / 256 * 256; }

}  // namespace
}  // namespace rbc

using namespace rbc;

extern "C" int bf_search_noalloc(const float* Q, int64_t m, const float* X, int64_t n, int32_t d,
                                 int32_t k, int32_t metric, int64_t* out_ids, float* out_dist,
                                 void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (m < 0 || n < 1 || d < 1 || k < 1 || n >= (1LL << 31) || m >= (1LL << 31)) {
    set_error("bf_search_noalloc: bad sizes m=%lld n=%lld d=%d k=%d", (long long)m, (long long)n,
              d, k);
    return RBC_ERR_ARG;
  }
  if (metric != RBC_L2 && metric != RBC_L1) {
    set_error("bf_search_noalloc: unknown metric %d", metric);
    return RBC_ERR_ARG;
  }
  if (k > MAX_C - 1) {
    set_error("bf_search_noalloc: k=%d exceeds the supported maximum %d", k, MAX_C - 1);
    return RBC_ERR_UNSUPPORTED;
  }
  if (d > SIMT_MAX_D) {
    set_error("bf_search_noalloc: d=%d exceeds %d", d, SIMT_MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  if (m == 0) return RBC_OK;
  if (!Q || !X || !out_ids || !out_dist) {
    set_error("bf_search_noalloc: NULL pointer");
    return RBC_ERR_ARG;
  }
  int dev = 0;
  RBC_CUDA(cudaGetDevice(&dev));
  if (!on_current_device(Q, dev) || !on_current_device(X, dev) ||
      !on_current_device(out_ids, dev) || !on_current_device(out_dist, dev)) {
    set_error("bf_search_noalloc: Q, X, out_ids and out_dist must be device pointers on the "
              "current device %d (host buffers would need device copies, i.e. an allocation)",
              dev);
    return RBC_ERR_ARG;
  }

  const int C = simt_list_width(k + 1);
  const int c_out = std::min(2 * C, MAX_C);
  const int64_t tiles = (m + TQ - 1) / TQ;
  const int64_t per_item = (int64_t)TQ * 2 * C;  // entries per work item
  const size_t fixed = NOALLOC_HEAD + rows_bytes(m);
  const int64_t max_items =
      fixed < NOALLOC_SCRATCH_BYTES
          ? (int64_t)((NOALLOC_SCRATCH_BYTES - fixed) / (size_t)(per_item * 8))
          : 0;
  if (tiles > max_items) {
    set_error("bf_search_noalloc: m=%lld needs %lld query tiles of candidate lists plus %zu "
              "bytes of re-search rows, but the %zu-byte scratch holds only %lld tiles at k=%d",
              (long long)m, (long long)tiles, rows_bytes(m), NOALLOC_SCRATCH_BYTES,
              (long long)max_items, k);
    return RBC_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  int rc = scratch_for_current_device(dev, &base);
  if (rc != RBC_OK) return rc;

  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // database splits: enough work items for the GPU, within the scratch
  int64_t splits = (8LL * sms + tiles - 1) / tiles;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, n / 512)));
  splits = std::min<int64_t>(splits, max_items / tiles);
  int64_t chunk = (n + splits - 1) / splits;
  splits = (n + chunk - 1) / chunk;
  const int64_t items = tiles * splits;

  unsigned char* b8 = static_cast<unsigned char*>(base);
  int* counters = reinterpret_cast<int*>(b8);
  int* fb_rows = reinterpret_cast<int*>(b8 + NOALLOC_HEAD);
  float* ps = reinterpret_cast<float*>(b8 + fixed);
  int* pi = reinterpret_cast<int*>(ps + items * per_item);
  RBC_CUDA(cudaMemsetAsync(counters, 0, 8 * sizeof(int), st));
  t_launches = 0;

  TileWork w{};
  w.num_items = (int)items;
  w.m = m;
  w.n = n;
  w.dense_splits = (int)splits;
  w.dense_chunk = chunk;
  int grid = (int)std::min<int64_t>(items, (int64_t)sms * 2 * 16);
  rc = launch_bf_simt_topc(Q, X, d, metric, C, w, TopOut{ps, pi, nullptr}, grid, st);
  if (rc != RBC_OK) return rc;

  SelectArgs a{};
  a.part_score = ps;
  a.part_idx = pi;
  a.C = C;
  a.nsub = 2;
  a.dense_splits = (int)splits;
  a.m = m;
  a.Q32 = Q;
  a.d = d;
  a.metric = metric;
  a.X32 = X;
  a.lp = 0;
  a.simt_eps = (float)(d + 8) * 5.9604645e-08f;
  a.k = k;
  a.c_out = c_out;
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.fallback_rows = fb_rows;
  a.counters = counters;
  rc = launch_select(a, st);
  if (rc != RBC_OK) return rc;
  // rows the certificate could not decide: the FP64 band over X (band.cu),
  // with the row list and its count in the scratch
  BandArgs b{};
  b.rows = fb_rows;
  b.nrows_dev = counters;
  b.Q32 = Q;
  b.X32 = X;
  b.n = n;
  b.d = d;
  b.ld = d;
  b.k = k;
  b.metric = metric;
  b.eps = (0.25f * d + 8.0f) * 5.9604645e-08f;
  b.out_ids = out_ids;
  b.out_dist = out_dist;
  rc = launch_band(b, (int)m, st);
  if (rc != RBC_OK) return rc;
  stats_publish_static(counters, m, m * n, st);
  return RBC_OK;
}
