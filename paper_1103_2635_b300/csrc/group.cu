// Grouped multi-index search: many independent Random Ball Covers searched
// together.
//
// The paper searches one database at a time (Sections 5, 7).  A deployment
// that holds many small indexes (one per tenant, shard or category) pays,
// per index and per batch, the fixed cost of a search: launches, host
// synchronisation, a tensor-core pass too small to fill the GPU.  A group
// concatenates the indexes into one resident layout and runs every step of the
// exact search (Section 5.2) for all of them at once:
//
//   * layout: every index's FP32 rows (list order), low-precision rows,
//     representatives, list offsets and radii are concatenated, each row
//     zero-padded to the group's widest dimension (zeros change no distance);
//     list offsets are global rows, representative ids global ordinals;
//   * stage one, BF(Q_i, R_i): one launch of the register-tiled FP32 kernel
//     over work items of 128 queries of one index against that index's
//     representatives; gamma_1, gamma_k, nearest rep;
//   * queries ordered by (index, nearest representative), each index's run
//     padded to whole 128-query tiles, so a tile never mixes indexes;
//   * pruning (Section 5.2, generalised to k) and work generation per tile
//     over its own index's lists;
//   * stage two, the ragged owned-list BF of every tile of every index: ONE
//     launch of the persistent tcgen05 top-C kernel over all work items;
//   * merge, FP32 re-rank, certification, FP64 ties for all queries in one
//     launch; uncertified queries searched by FP32 brute force over their own
//     index (device-side count, no host round trip).
//
// Nothing reads a count back to the host, so the whole search is captured
// once per batch shape (the per-index query counts and k) as a CUDA graph and
// replayed.  An autotuner times the stage-two work-item size on the caller's
// batch and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "kernels.cuh"

namespace rbc {
namespace {

constexpr int GROUP_PRUNE_WARPS = 8;
constexpr int64_t GROUP_NORM_PAD = 512;  // rows past the end the tensor-core kernel may read

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// dst [rows, dd] = src [rows, ds] zero-padded (ds <= dd); one warp per row
__global__ void pad_rows_kernel(const float* __restrict__ src, int64_t rows, int ds, int dd,
                                float* __restrict__ dst) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  for (int i = lane; i < dd; i += 32) dst[w * dd + i] = i < ds ? src[w * ds + i] : 0.f;
}

// Packed queries (index i's m_i rows of d_i floats, index after index) ->
// [M, DG] zero-padded rows; row r belongs to index row_index[r].
__global__ void group_pad_queries_kernel(const float* __restrict__ Q, const int* __restrict__ row_index,
                                         const int64_t* __restrict__ q_row_base,
                                         const int64_t* __restrict__ q_elem_base,
                                         const int* __restrict__ d_of, int64_t M, int DG,
                                         float* __restrict__ Qp) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= M) return;
  const int g = row_index[w];
  const int d = d_of[g];
  const float* src = Q + q_elem_base[g] + (w - q_row_base[g]) * d;
  for (int i = lane; i < DG; i += 32) Qp[w * DG + i] = i < d ? src[i] : 0.f;
}

// Stage one runs as the register-tiled FP32 kernel over work items (one per
// 128 packed queries of an index, against that index's representatives: one
// segment), which writes D[q, local r]; the columns past the index's n_r are
// set to +inf here.
__global__ void group_fill_pad_kernel(const int* __restrict__ row_index, const int* __restrict__ nr_of,
                                      int64_t M, int NRMAX, float* __restrict__ D) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= M) return;
  for (int r = nr_of[row_index[w]] + lane; r < NRMAX; r += 32) D[w * NRMAX + r] = INFINITY;
}

// Queries ordered by (index, nearest representative): a stable counting sort
// by the nearest representative's ordinal within its index, then a stable
// one by index (two small histograms instead of one over every
// representative of the group).  key2[s] = index of the s-th query of the
// first order; qperm[pos] = perm1[perm2[pos]].
__global__ void group_key2_kernel(const int* __restrict__ perm1, const int* __restrict__ row_index,
                                  int64_t M, int64_t* __restrict__ key2) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < M) key2[s] = row_index[perm1[s]];
}
__global__ void compose_perm_kernel(const int* __restrict__ perm1, const int* __restrict__ perm2,
                                    int64_t M, int* __restrict__ qperm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) qperm[i] = perm1[perm2[i]];
}

// Padded layout: index g's queries, in sorted order, occupy padded rows
// [pad_base_g, pad_base_g + m_g); its tiles end at a multiple of TQ.
__global__ void group_layout_kernel(const int* __restrict__ qperm, const int* __restrict__ tile_index,
                                    const int64_t* __restrict__ pad_base,
                                    const int64_t* __restrict__ q_row_base,
                                    const int64_t* __restrict__ m_of, int64_t MP,
                                    int* __restrict__ qsrc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MP) return;
  const int g = tile_index[p / TQ];
  const int64_t local = p - pad_base[g];
  qsrc[p] = local < m_of[g] ? qperm[q_row_base[g] + local] : -1;
}

// Pruning per tile (Section 5.2, generalised to k, with the FP32 bound of
// stage one): representative r of the tile's index is kept for query q iff
// rho(q, r) <= gamma_k + psi_r and rho(q, r) <= 2 gamma_k + gamma_1.  The
// tile keeps the union; its point count is the sum of the kept list sizes.
__global__ void __launch_bounds__(GROUP_PRUNE_WARPS * 32)
group_prune_kernel(const float* __restrict__ D, const int* __restrict__ qsrc,
                   const int* __restrict__ tile_index, const int* __restrict__ rep_base,
                   const int* __restrict__ nr_of, const float* __restrict__ psi,
                   const int* __restrict__ offsets, int NRMAX, const float* __restrict__ g1,
                   const float* __restrict__ gk, float rel, uint32_t* __restrict__ tile_mask,
                   int64_t* __restrict__ tile_points, int* __restrict__ q_kept) {
  extern __shared__ uint32_t mask[];
  const int words = (NRMAX + 31) / 32;
  const int t = blockIdx.x;
  const int g = tile_index[t];
  const int rb = rep_base[g], nr = nr_of[g];
  for (int i = threadIdx.x; i < words; i += blockDim.x) mask[i] = 0;
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float up = 1.0f + rel, lo = 1.0f - rel, slack = 1.0f + 2.4e-7f;
  for (int r = wid; r < TQ; r += GROUP_PRUNE_WARPS) {
    const int q = qsrc[(int64_t)t * TQ + r];
    if (q < 0) continue;
    const float gkh = gk[q] * up, g1h = g1[q] * up;
    const float lemma = (2.0f * gkh + g1h) * slack;
    const float* row = D + (int64_t)q * NRMAX;
    int kept = 0;
    for (int c0 = 0; c0 < nr; c0 += 32) {
      const int c = c0 + lane;
      bool keep = false;
      if (c < nr) {
        const float dl = row[c] * lo;
        keep = dl <= (gkh + psi[rb + c]) * slack && dl <= lemma;
      }
      const unsigned bits = __ballot_sync(0xffffffffu, keep);
      kept += __popc(bits);
      if (lane == 0 && bits) atomicOr(&mask[c0 >> 5], bits);
    }
    if (lane == 0 && q_kept) q_kept[q] = kept;
  }
  __syncthreads();
  long long pts = 0;
  for (int r = threadIdx.x; r < nr; r += blockDim.x)
    if (mask[r >> 5] & (1u << (r & 31))) pts += offsets[rb + r + 1] - offsets[rb + r];
  for (int o = 16; o > 0; o >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o);
  __shared__ long long part[GROUP_PRUNE_WARPS];
  if (lane == 0) part[wid] = pts;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int i = 0; i < GROUP_PRUNE_WARPS; ++i) s += part[i];
    tile_points[t] = s;
  }
  for (int i = threadIdx.x; i < words; i += blockDim.x) tile_mask[(int64_t)t * words + i] = mask[i];
}

// One thread per tile: the kept lists of its index (adjacent lists merged into
// runs of global rows) cut into work items of at most W points.
__global__ void group_workgen_kernel(const uint32_t* __restrict__ tile_mask,
                                     const int* __restrict__ tile_index, const int* __restrict__ rep_base,
                                     const int* __restrict__ nr_of, const int* __restrict__ offsets,
                                     int NRMAX, int tiles, int W, int seg_cap,
                                     const int* __restrict__ tile_item_off,
                                     const int* __restrict__ tile_item_cap, WorkItem* __restrict__ items,
                                     Seg* __restrict__ segs, uint32_t* dev_err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tiles) return;
  const int words = (NRMAX + 31) / 32;
  const uint32_t* mk = tile_mask + (int64_t)t * words;
  const int g = tile_index[t];
  const int rb = rep_base[g], nr = nr_of[g];
  const int q0 = t * TQ;
  int item = tile_item_off[t];
  const int item_end = tile_item_off[t + 1];
  if (item_end - item > tile_item_cap[t]) {
    atomicOr(dev_err, DEV_ERR_CAPACITY);
    return;
  }
  const int seg0 = t * seg_cap;
  int seg = seg0, acc = 0, item_seg0 = seg;
  auto close_item = [&]() {
    if (item < item_end) items[item] = WorkItem{q0, TQ, item_seg0, seg, item, t};
    ++item;
    item_seg0 = seg;
    acc = 0;
  };
  for (int r = 0; r < nr; ++r) {
    if (!(mk[r >> 5] & (1u << (r & 31)))) continue;
    int b = offsets[rb + r];
    const int e = offsets[rb + r + 1];
    while (b < e) {
      const int take = min(e - b, W - acc);
      if (seg > item_seg0 && segs[seg - 1].x_end == b) {
        segs[seg - 1].x_end = b + take;
      } else {
        if (seg - seg0 >= seg_cap) {
          atomicOr(dev_err, DEV_ERR_CAPACITY);
          return;
        }
        segs[seg++] = Seg{b, b + take};
      }
      acc += take;
      b += take;
      if (acc == W) close_item();
    }
  }
  if (acc > 0) close_item();
}

__global__ void add_offset_kernel(const int* __restrict__ src, int n, int add, int* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + add;
}

// ---- one batch shape: host tables, workspace, CUDA graph ----
struct Plan {
  std::vector<int64_t> m;  // queries per index
  int k = 0;
  int W = 0;               // stage-two work-item size (points)
  int64_t M = 0, MP = 0, tiles = 0, item_cap_total = 0;
  int seg_cap = 0, C = 0, c_sel = 0;
  std::vector<void*> dev;  // device allocations
  // device arrays
  int *row_index = nullptr, *tile_index = nullptr, *tile_item_cap = nullptr;
  int8_t* tile_kb = nullptr;   // per tile: 64-column K blocks holding its index's columns
  int16_t* tile_dim = nullptr; // per tile: its index's dimension
  WorkItem* items1 = nullptr;  // stage one: 128 packed queries of one index x its reps
  Seg* segs1 = nullptr;        // stage one: index i's representatives
  int64_t items1_n = 0;
  int64_t *q_row_base = nullptr, *q_elem_base = nullptr, *pad_base = nullptr, *m_of = nullptr;
  float *Qin = nullptr, *Qp = nullptr, *D = nullptr, *g1 = nullptr, *gk = nullptr, *Qs = nullptr;
  int64_t *nearest = nullptr, *key = nullptr;
  int *qperm = nullptr, *qoff = nullptr, *scratch = nullptr, *qsrc = nullptr, *qkept = nullptr;
  int *perm1 = nullptr, *perm2 = nullptr;
  void* qlp = nullptr;
  float *qnorm = nullptr, *qerr = nullptr;
  uint32_t* tmask = nullptr;
  int64_t* tpts = nullptr;
  int *tcnt = nullptr, *toff = nullptr;
  WorkItem* items = nullptr;
  Seg* segs = nullptr;
  float* ps = nullptr;
  int *pi = nullptr, *pv = nullptr;
  int64_t* out_ids = nullptr;
  float* out_dist = nullptr;
  int *fb_rows = nullptr, *counters = nullptr;
  uint32_t* dev_err = nullptr;
  int64_t in_floats = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t replays = 0;
  ~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
    for (void* p : dev) cudaFree(p);
  }
  template <typename T>
  int alloc(T** out, int64_t count) {
    void* p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("group workspace allocation of %lld bytes failed: %s",
                (long long)(count * (int64_t)sizeof(T)), cudaGetErrorString(e));
      return RBC_ERR_OOM;
    }
    dev.push_back(p);
    *out = static_cast<T*>(p);
    return RBC_OK;
  }
};

}  // namespace
}  // namespace rbc

using namespace rbc;

struct rbc_group {
  int count = 0, DG = 0, dpad = 0, storage = 0, NRMAX = 0, device = 0;
  int64_t N = 0, R = 0, nmax = 0;
  std::vector<int64_t> row_base, n_of;   // per index: first row, rows
  std::vector<int> rep_base, nr_of, d_of;
  std::vector<void*> dev;
  float *X32 = nullptr, *R32 = nullptr, *psi = nullptr, *xnorm = nullptr;
  int *members = nullptr, *offsets = nullptr, *rep_base_d = nullptr, *nr_of_d = nullptr,
      *d_of_d = nullptr;
  int64_t *row_base_d = nullptr, *n_of_d = nullptr;
  void* Xlp = nullptr;
  void* xnblock = nullptr;  // [N + pad, 16] bf16: -|x~|^2 / 2 as (high, low), the norm MMA's B
  unsigned* lp_max = nullptr;
  int W = 0;  // tuned work-item size (0: default)
  std::mutex mu;
  std::map<std::pair<int, std::vector<int64_t>>, std::unique_ptr<Plan>> plans;
  rbc_grouped_stats last{};

  template <typename T>
  int alloc(T** out, int64_t count) {
    void* p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("group allocation of %lld bytes failed: %s",
                (long long)(count * (int64_t)sizeof(T)), cudaGetErrorString(e));
      return RBC_ERR_OOM;
    }
    dev.push_back(p);
    *out = static_cast<T*>(p);
    return RBC_OK;
  }
  ~rbc_group() {
    plans.clear();
    for (void* p : dev) cudaFree(p);
  }
};

namespace rbc {
namespace {

#define G_TRY(x)                 \
  do {                           \
    int _r = (x);                \
    if (_r != RBC_OK) return _r; \
  } while (0)

template <typename T>
int upload(Plan& P, T** out, const std::vector<T>& v, cudaStream_t st) {
  G_TRY(P.alloc(out, (int64_t)v.size()));
  RBC_CUDA(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return RBC_OK;
}

int default_W(const rbc_group* g) {
  return g->W > 0 ? g->W : (int)std::max<int64_t>(2048, std::min<int64_t>(16384, g->nmax / 4 / 256 * 256));
}

// Host tables and workspace of one batch shape.
int make_plan(rbc_group* g, const std::vector<int64_t>& m, int k, int W, cudaStream_t st,
              std::unique_ptr<Plan>& out) {
  std::unique_ptr<Plan> P(new (std::nothrow) Plan());
  if (!P) {
    set_error("group plan: host allocation failed");
    return RBC_ERR_OOM;
  }
  P->m = m;
  P->k = k;
  P->W = W;
  const int n = g->count;
  std::vector<int64_t> q_row_base(n), q_elem_base(n), pad_base(n);
  std::vector<int> row_index, tile_index, tile_cap;
  std::vector<int8_t> tile_kb;
  std::vector<int16_t> tile_dim;
  std::vector<WorkItem> items1;
  std::vector<Seg> segs1;
  int64_t M = 0, E = 0, MP = 0, cap_total = 0, cap_max = 1;
  for (int i = 0; i < n; ++i) {
    segs1.push_back(Seg{g->rep_base[i], g->rep_base[i] + g->nr_of[i]});
    for (int64_t j = 0; j < m[i]; j += TQ) {
      const int it = (int)items1.size();
      items1.push_back(WorkItem{(int32_t)(M + j), (int32_t)std::min<int64_t>(TQ, m[i] - j), i, i + 1,
                                it, it});
    }
    q_row_base[i] = M;
    q_elem_base[i] = E;
    pad_base[i] = MP;
    const int64_t ti = cdiv64(m[i], TQ);
    const int64_t cap = cdiv64(g->n_of[i], W) + 1;  // a tile holds at most all of its index
    for (int64_t t = 0; t < ti; ++t) {
      tile_index.push_back(i);
      tile_cap.push_back((int)cap);
      tile_kb.push_back((int8_t)((g->d_of[i] + 63) / 64));
      tile_dim.push_back((int16_t)g->d_of[i]);
    }
    for (int64_t r = 0; r < m[i]; ++r) row_index.push_back(i);
    cap_total += ti * cap;
    cap_max = std::max(cap_max, cap);
    M += m[i];
    E += m[i] * g->d_of[i];
    MP += ti * TQ;
  }
  P->M = M;
  P->MP = MP;
  P->tiles = MP / TQ;
  P->item_cap_total = std::max<int64_t>(cap_total, 1);
  P->seg_cap = g->NRMAX + (int)cap_max + 2;
  P->in_floats = E;
  const int c_out = std::min(k <= 1 ? 16 : 32, MAX_C);  // low-precision candidate lists
  P->c_sel = c_out;
  P->C = c_out <= 16 ? 8 : 16;
  if (M == 0) {
    out = std::move(P);
    return RBC_OK;
  }
  Plan& p = *P;
  std::vector<int64_t> m64(m.begin(), m.end());
  G_TRY(upload(p, &p.row_index, row_index, st));
  G_TRY(upload(p, &p.items1, items1, st));
  G_TRY(upload(p, &p.segs1, segs1, st));
  p.items1_n = (int64_t)items1.size();
  G_TRY(upload(p, &p.tile_index, tile_index, st));
  G_TRY(upload(p, &p.tile_item_cap, tile_cap, st));
  G_TRY(upload(p, &p.tile_kb, tile_kb, st));
  G_TRY(upload(p, &p.tile_dim, tile_dim, st));
  G_TRY(upload(p, &p.q_row_base, q_row_base, st));
  G_TRY(upload(p, &p.q_elem_base, q_elem_base, st));
  G_TRY(upload(p, &p.pad_base, pad_base, st));
  G_TRY(upload(p, &p.m_of, m64, st));
  const int DG = g->DG;
  G_TRY(p.alloc(&p.Qin, E));
  G_TRY(p.alloc(&p.Qp, M * DG));
  G_TRY(p.alloc(&p.D, M * g->NRMAX));
  G_TRY(p.alloc(&p.g1, M));
  G_TRY(p.alloc(&p.gk, M));
  G_TRY(p.alloc(&p.nearest, M));
  G_TRY(p.alloc(&p.key, M));
  G_TRY(p.alloc(&p.qperm, M));
  G_TRY(p.alloc(&p.perm1, M));
  G_TRY(p.alloc(&p.perm2, M));
  const int bins = std::max(g->NRMAX, g->count);
  G_TRY(p.alloc(&p.qoff, bins + 1));
  G_TRY(p.alloc(&p.scratch, counting_sort_scratch_ints(M, bins)));
  G_TRY(p.alloc(&p.qsrc, MP));
  G_TRY(p.alloc(&p.qkept, M));
  G_TRY(p.alloc(&p.Qs, MP * DG));
  uint16_t* ql;
  G_TRY(p.alloc(&ql, MP * g->dpad));
  p.qlp = ql;
  G_TRY(p.alloc(&p.qnorm, MP));
  G_TRY(p.alloc(&p.qerr, MP));
  G_TRY(p.alloc(&p.tmask, p.tiles * ((g->NRMAX + 31) / 32)));
  G_TRY(p.alloc(&p.tpts, p.tiles));
  G_TRY(p.alloc(&p.tcnt, p.tiles));
  G_TRY(p.alloc(&p.toff, p.tiles + 1));
  G_TRY(p.alloc(&p.items, p.item_cap_total));
  G_TRY(p.alloc(&p.segs, p.tiles * p.seg_cap));
  G_TRY(p.alloc(&p.ps, p.item_cap_total * TQ * 2 * p.C));
  G_TRY(p.alloc(&p.pi, p.item_cap_total * TQ * 2 * p.C));
  G_TRY(p.alloc(&p.pv, p.item_cap_total));
  G_TRY(p.alloc(&p.out_ids, M * k));
  G_TRY(p.alloc(&p.out_dist, M * k));
  G_TRY(p.alloc(&p.fb_rows, MP));
  G_TRY(p.alloc(&p.counters, 8));
  G_TRY(p.alloc(&p.dev_err, 1));
  out = std::move(P);
  return RBC_OK;
}

// Every device step of one grouped search, on `st` (no host synchronisation;
// capturable).  Reads p.Qin, writes p.out_ids / p.out_dist and p.counters.
int run_plan(rbc_group* g, Plan& p, cudaStream_t st) {
  const int DG = g->DG, NRMAX = g->NRMAX;
  const int64_t M = p.M, MP = p.MP;
  const int tiles = (int)p.tiles;
  RBC_CUDA(cudaMemsetAsync(p.counters, 0, 8 * sizeof(int), st));
  RBC_CUDA(cudaMemsetAsync(p.dev_err, 0, sizeof(uint32_t), st));
  group_pad_queries_kernel<<<(unsigned)cdiv64(M * 32, 256), 256, 0, st>>>(
      p.Qin, p.row_index, p.q_row_base, p.q_elem_base, g->d_of_d, M, DG, p.Qp);
  RBC_LAUNCH_CHECK("group_pad_queries_kernel");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
  // stage one, BF(Q_i, R_i) for every index: FP32, every distance kept
  group_fill_pad_kernel<<<(unsigned)cdiv64(M * 32, 256), 256, 0, st>>>(p.row_index, g->nr_of_d, M,
                                                                       NRMAX, p.D);
  RBC_LAUNCH_CHECK("group_fill_pad_kernel");
  TileWork w1{};
  w1.items = p.items1;
  w1.num_items = (int)p.items1_n;
  w1.segs = p.segs1;
  w1.m = M;
  w1.n = g->R;
  G_TRY(launch_bf_simt_store(p.Qp, g->R32, DG, RBC_L2, w1, p.D, NRMAX,
                             (int)std::min<int64_t>(p.items1_n, (int64_t)sms * 2 * 16), st));
  G_TRY(launch_row_stats(p.D, M, NRMAX, p.k, p.g1, p.gk, p.nearest, st));
  G_TRY(launch_counting_sort(p.nearest, M, NRMAX, p.perm1, p.qoff, p.scratch, st));
  group_key2_kernel<<<(unsigned)cdiv64(M, 256), 256, 0, st>>>(p.perm1, p.row_index, M, p.key);
  RBC_LAUNCH_CHECK("group_key2_kernel");
  G_TRY(launch_counting_sort(p.key, M, g->count, p.perm2, p.qoff, p.scratch, st));
  compose_perm_kernel<<<(unsigned)cdiv64(M, 256), 256, 0, st>>>(p.perm1, p.perm2, M, p.qperm);
  RBC_LAUNCH_CHECK("compose_perm_kernel");
  group_layout_kernel<<<(unsigned)cdiv64(MP, 256), 256, 0, st>>>(p.qperm, p.tile_index, p.pad_base,
                                                                 p.q_row_base, p.m_of, MP, p.qsrc);
  RBC_LAUNCH_CHECK("group_layout_kernel");
  G_TRY(launch_gather_padded(p.Qp, p.qsrc, MP, DG, p.Qs, st));
  G_TRY(launch_to_lowp(p.Qs, MP, DG, g->dpad, g->storage, p.qlp, p.qnorm, p.qerr, nullptr, nullptr,
                       st));
  const int words = (NRMAX + 31) / 32;
  const float eps1 = (float)(DG + 8) * 5.9604645e-08f;  // FP32 stage-one bound (sequential sums)
  group_prune_kernel<<<tiles, GROUP_PRUNE_WARPS * 32, words * sizeof(uint32_t), st>>>(
      p.D, p.qsrc, p.tile_index, g->rep_base_d, g->nr_of_d, g->psi, g->offsets, NRMAX, p.g1, p.gk,
      eps1, p.tmask, p.tpts, p.qkept);
  RBC_LAUNCH_CHECK("group_prune_kernel");
  G_TRY(launch_item_offsets(p.tpts, tiles, p.W, p.tcnt, p.toff, st));
  group_workgen_kernel<<<(unsigned)cdiv64(tiles, 128), 128, 0, st>>>(
      p.tmask, p.tile_index, g->rep_base_d, g->nr_of_d, g->offsets, NRMAX, tiles, p.W, p.seg_cap,
      p.toff, p.tile_item_cap, p.items, p.segs, p.dev_err);
  RBC_LAUNCH_CHECK("group_workgen_kernel");
  // stage two: one persistent launch over the work items of every index
  TileWork w{};
  w.items = p.items;
  w.num_items_dev = p.toff + tiles;
  w.num_items = (int)p.item_cap_total;
  w.segs = p.segs;
  w.m = MP;
  w.n = g->N;
  w.tile_kb = p.tile_kb;  // an index of d <= 64 multiplies one K block, not two
  LpMatrix Qm{p.qlp, p.qnorm, MP, g->dpad, g->storage};
  LpMatrix Xm{g->Xlp, g->xnorm, g->N, g->dpad, g->storage, g->xnblock};
  G_TRY(launch_bf_tc_topc(Qm, Xm, p.C, w, TopOut{p.ps, p.pi, p.pv}, sms, st, p.dev_err));
  // merge + FP32 re-rank + certification + FP64 ties for every query
  SelectArgs a{};
  a.part_score = p.ps;
  a.part_idx = p.pi;
  a.slot_valid = p.pv;
  a.C = p.C;
  a.nsub = 2;
  a.tile_slot_off = p.toff;
  a.m = MP;
  a.Q32 = p.Qs;
  a.d = DG;
  a.metric = RBC_L2;
  a.qorig = p.qsrc;
  a.X32 = g->X32;
  a.xid = g->members;
  a.lp = 1;
  a.q_lpnorm = p.qnorm;
  a.q_err = p.qerr;
  a.x_err_max_bits = g->lp_max;
  a.x_norm_max_bits = g->lp_max + 1;
  a.k = p.k;
  a.c_out = p.c_sel;
  a.out_ids = p.out_ids;
  a.out_dist = p.out_dist;
  a.fallback_rows = p.fb_rows;
  a.counters = p.counters;
  a.tile_dim = p.tile_dim;  // re-rank over each index's own columns
  G_TRY(launch_select(a, st));
  // uncertified rows: the FP64 band over their own index (band.cu)
  BandArgs b{};
  b.rows = p.fb_rows;
  b.nrows_dev = p.counters;
  b.Q32 = p.Qs;
  b.qorig = p.qsrc;
  b.X32 = g->X32;
  b.xid = g->members;
  b.n = g->N;
  b.tile_grp = p.tile_index;
  b.grp_base = g->row_base_d;
  b.grp_len = g->n_of_d;
  b.d = DG;
  b.ld = DG;
  b.k = p.k;
  b.metric = RBC_L2;
  b.eps = (0.25f * DG + 8.0f) * 5.9604645e-08f;  // the re-rank's bound at the widest rows
  b.out_ids = p.out_ids;
  b.out_dist = p.out_dist;
  G_TRY(launch_band(b, (int)MP, st));
  return RBC_OK;
}

int plan_for(rbc_group* g, const std::vector<int64_t>& m, int k, int W, cudaStream_t st, Plan** out) {
  auto key = std::make_pair(k * 1000003 + W, m);
  auto it = g->plans.find(key);
  if (it != g->plans.end()) {
    *out = it->second.get();
    return RBC_OK;
  }
  if (g->plans.size() >= 8) g->plans.erase(g->plans.begin());  // bounded cache
  std::unique_ptr<Plan> P;
  G_TRY(make_plan(g, m, k, W, st, P));
  Plan* raw = P.get();
  g->plans.emplace(key, std::move(P));
  *out = raw;
  return RBC_OK;
}

// Capture the plan's steps as a CUDA graph (once), then launch it.
int launch_plan(rbc_group* g, Plan& p, cudaStream_t st, bool use_graph) {
  if (p.M == 0) return RBC_OK;
  if (!use_graph) return run_plan(g, p, st);
  if (!p.exec) {
    cudaStream_t cs;
    RBC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cs);
      return cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
    }
    const int rc = run_plan(g, p, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (rc != RBC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(&p.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p.exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
  }
  RBC_CUDA(cudaGraphLaunch(p.exec, st));
  ++p.replays;
  return RBC_OK;
}

// Q: the queries packed index after index; or (Q null) Qs[i]: index i's rows
// alone, each copied to its place in the plan's input buffer.
int group_search(rbc_group* g, const float* Q, const int64_t* m, int k, int64_t* out_ids,
                 float* out_dist, cudaStream_t st, int W, bool use_graph, Plan** used,
                 const float* const* Qs = nullptr) {
  std::vector<int64_t> mv(m, m + g->count);
  Plan* p = nullptr;
  G_TRY(plan_for(g, mv, k, W, st, &p));
  if (used) *used = p;
  if (p->M == 0) return RBC_OK;
  if (Q) {
    RBC_CUDA(cudaMemcpyAsync(p->Qin, Q, p->in_floats * sizeof(float), cudaMemcpyDefault, st));
  } else {
    int64_t off = 0;
    for (int i = 0; i < g->count; ++i) {
      const int64_t f = mv[i] * g->d_of[i];
      if (f > 0)
        RBC_CUDA(cudaMemcpyAsync(p->Qin + off, Qs[i], f * sizeof(float), cudaMemcpyDefault, st));
      off += f;
    }
  }
  G_TRY(launch_plan(g, *p, st, use_graph));
  RBC_CUDA(cudaMemcpyAsync(out_ids, p->out_ids, p->M * k * sizeof(int64_t), cudaMemcpyDefault, st));
  RBC_CUDA(cudaMemcpyAsync(out_dist, p->out_dist, p->M * k * sizeof(float), cudaMemcpyDefault, st));
  return RBC_OK;
}

// rbc_group_search and rbc_group_search_split: Q packed, or Qs per index
int group_search_entry(rbc_group* g, const float* Q, const float* const* Qs, const int64_t* m,
                       int32_t k, int64_t* out_ids, float* out_dist, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!g || !m) {
    set_error("rbc_group_search: NULL group or m");
    return RBC_ERR_ARG;
  }
  int64_t M = 0;
  for (int i = 0; i < g->count; ++i) {
    if (m[i] < 0 || m[i] >= (1LL << 31)) {
      set_error("rbc_group_search: m[%d] = %lld out of range", i, (long long)m[i]);
      return RBC_ERR_ARG;
    }
    M += m[i];
  }
  if (k < 1 || k > MAX_C - 1 || M >= (1LL << 31)) {
    set_error("rbc_group_search: k=%d must be in [1, %d]; total queries %lld < 2^31", k,
              MAX_C - 1, (long long)M);
    return RBC_ERR_ARG;
  }
  for (int i = 0; i < g->count; ++i)
    if (m[i] > 0 && k > g->n_of[i]) {
      set_error("rbc_group_search: k=%d exceeds the %lld points of index %d", k,
                (long long)g->n_of[i], i);
      return RBC_ERR_ARG;
    }
  if (M > 0 && ((!Q && !Qs) || !out_ids || !out_dist)) {
    set_error("rbc_group_search: NULL pointer");
    return RBC_ERR_ARG;
  }
  if (!Q)
    for (int i = 0; i < g->count; ++i)
      if (m[i] > 0 && !Qs[i]) {
        set_error("rbc_group_search_split: NULL query pointer of index %d", i);
        return RBC_ERR_ARG;
      }
  std::lock_guard<std::mutex> lk(g->mu);
  Plan* p = nullptr;
  G_TRY(group_search(g, Q, m, k, out_ids, out_dist, st, default_W(g), true, &p, Qs));
  g->last.queries = M;
  g->last.work_item_points = p->W;
  g->last.graph_replays = p->replays;
  if (M > 0) {
    // the call's one read-back: the device error flags of the batch
    uint32_t err = 0;
    RBC_CUDA(cudaMemcpyAsync(&err, p->dev_err, sizeof(err), cudaMemcpyDeviceToHost, st));
    RBC_CUDA(cudaStreamSynchronize(st));
    if (err) {
      set_error("rbc_group_search: device error flags 0x%x (capacity or bounded wait)", err);
      return (err & DEV_ERR_TIMEOUT) ? RBC_ERR_TIMEOUT : RBC_ERR_CUDA;
    }
  }
  return RBC_OK;
}

}  // namespace
}  // namespace rbc

extern "C" {

int rbc_group_create(const rbc_index* const* indexes, int32_t count, void* stream,
                     rbc_group** out) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!indexes || !out || count < 1) {
    set_error("rbc_group_create: NULL pointer or count < 1");
    return RBC_ERR_ARG;
  }
  *out = nullptr;
  const rbc_index* first = indexes[0];
  for (int i = 0; i < count; ++i) {
    const rbc_index* ix = indexes[i];
    if (!ix) {
      set_error("rbc_group_create: index %d is NULL", i);
      return RBC_ERR_ARG;
    }
    if (ix->mode != RBC_EXACT || ix->metric != RBC_L2 ||
        (ix->storage != RBC_BF16 && ix->storage != RBC_F16) || !ix->Xlp) {
      set_error("rbc_group_create: index %d must be an exact L2 index with bf16 or fp16 storage", i);
      return RBC_ERR_UNSUPPORTED;
    }
    if (ix->storage != first->storage || ix->device != first->device) {
      set_error("rbc_group_create: index %d differs in storage or device from index 0", i);
      return RBC_ERR_ARG;
    }
  }
  std::unique_ptr<rbc_group> G(new (std::nothrow) rbc_group());
  if (!G) {
    set_error("rbc_group_create: host allocation failed");
    return RBC_ERR_OOM;
  }
  rbc_group& g = *G;
  g.count = count;
  g.storage = first->storage;
  g.device = first->device;
  int dmax = 0;
  for (int i = 0; i < count; ++i) {
    const rbc_index* ix = indexes[i];
    g.row_base.push_back(g.N);
    g.n_of.push_back(ix->list_entries);
    g.rep_base.push_back((int)g.R);
    g.nr_of.push_back(ix->n_r);
    g.d_of.push_back(ix->d);
    g.N += ix->list_entries;
    g.R += ix->n_r;
    g.nmax = std::max<int64_t>(g.nmax, ix->list_entries);
    g.NRMAX = std::max(g.NRMAX, ix->n_r);
    dmax = std::max(dmax, ix->d);
  }
  if (g.NRMAX > 12000 || count > 12000) {
    set_error("rbc_group_create: at most 12000 indexes of at most 12000 representatives each");
    return RBC_ERR_UNSUPPORTED;
  }
  if (g.N >= (1LL << 31) || g.R >= (1LL << 31)) {
    set_error("rbc_group_create: %lld rows / %lld representatives exceed 2^31", (long long)g.N,
              (long long)g.R);
    return RBC_ERR_UNSUPPORTED;
  }
  g.DG = (dmax + 3) / 4 * 4;
  g.dpad = (g.DG + 63) / 64 * 64;
  int prev = 0;
  cudaGetDevice(&prev);
  RBC_CUDA(cudaSetDevice(g.device));
  G_TRY(g.alloc(&g.X32, g.N * g.DG));
  G_TRY(g.alloc(&g.members, g.N));
  G_TRY(g.alloc(&g.offsets, g.R + 1));
  G_TRY(g.alloc(&g.psi, g.R));
  G_TRY(g.alloc(&g.R32, g.R * g.DG));
  for (int i = 0; i < count; ++i) {
    const rbc_index* ix = indexes[i];
    const int64_t n = ix->list_entries;
    if (n > 0)
      pad_rows_kernel<<<(unsigned)cdiv64(n * 32, 256), 256, 0, st>>>(ix->X32, n, ix->d, g.DG,
                                                                     g.X32 + g.row_base[i] * g.DG);
    pad_rows_kernel<<<(unsigned)cdiv64((int64_t)ix->n_r * 32, 256), 256, 0, st>>>(
        ix->R32, ix->n_r, ix->d, g.DG, g.R32 + (int64_t)g.rep_base[i] * g.DG);
    RBC_LAUNCH_CHECK("pad_rows_kernel");
    RBC_CUDA(cudaMemcpyAsync(g.members + g.row_base[i], ix->members, n * sizeof(int),
                             cudaMemcpyDeviceToDevice, st));
    RBC_CUDA(cudaMemcpyAsync(g.psi + g.rep_base[i], ix->psi, ix->n_r * sizeof(float),
                             cudaMemcpyDeviceToDevice, st));
    add_offset_kernel<<<(ix->n_r + 1 + 255) / 256, 256, 0, st>>>(
        ix->offsets, ix->n_r + 1, (int)g.row_base[i], g.offsets + g.rep_base[i]);
    RBC_LAUNCH_CHECK("add_offset_kernel");
  }
  uint16_t* xl;
  G_TRY(g.alloc(&xl, g.N * g.dpad));
  g.Xlp = xl;
  G_TRY(g.alloc(&g.xnorm, g.N + GROUP_NORM_PAD));
  RBC_CUDA(cudaMemsetAsync(g.xnorm + g.N, 0, GROUP_NORM_PAD * sizeof(float), st));
  G_TRY(g.alloc(&g.lp_max, 2));
  RBC_CUDA(cudaMemsetAsync(g.lp_max, 0, 2 * sizeof(unsigned), st));
  G_TRY(launch_to_lowp(g.X32, g.N, g.DG, g.dpad, g.storage, g.Xlp, g.xnorm, nullptr, g.lp_max,
                       g.lp_max + 1, st));
  uint16_t* nb;
  G_TRY(g.alloc(&nb, (g.N + GROUP_NORM_PAD) * NBLOCK_COLS));
  G_TRY(launch_norm_block(g.xnorm, g.N, g.N + GROUP_NORM_PAD, nb, st));
  g.xnblock = nb;
  G_TRY(g.alloc(&g.rep_base_d, count));
  G_TRY(g.alloc(&g.nr_of_d, count));
  G_TRY(g.alloc(&g.d_of_d, count));
  G_TRY(g.alloc(&g.row_base_d, count));
  G_TRY(g.alloc(&g.n_of_d, count));
  RBC_CUDA(cudaMemcpyAsync(g.rep_base_d, g.rep_base.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
  RBC_CUDA(cudaMemcpyAsync(g.nr_of_d, g.nr_of.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
  RBC_CUDA(cudaMemcpyAsync(g.d_of_d, g.d_of.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
  RBC_CUDA(cudaMemcpyAsync(g.row_base_d, g.row_base.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  RBC_CUDA(cudaMemcpyAsync(g.n_of_d, g.n_of.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  RBC_CUDA(cudaStreamSynchronize(st));
  cudaSetDevice(prev);
  *out = G.release();
  return RBC_OK;
}

int rbc_group_search(rbc_group* g, const float* Q, const int64_t* m, int32_t k, int64_t* out_ids,
                     float* out_dist, void* stream) {
  return rbc::group_search_entry(g, Q, nullptr, m, k, out_ids, out_dist, stream);
}

int rbc_group_search_split(rbc_group* g, const float* const* Q, const int64_t* m, int32_t k,
                           int64_t* out_ids, float* out_dist, void* stream) {
  if (!Q) {
    rbc::set_error("rbc_group_search_split: NULL query pointer array");
    return RBC_ERR_ARG;
  }
  return rbc::group_search_entry(g, nullptr, Q, m, k, out_ids, out_dist, stream);
}

int rbc_group_tune(rbc_group* g, const float* Q, const int64_t* m, int32_t k, void* stream,
                   int32_t* chosen) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!g || !m || !Q) {
    set_error("rbc_group_tune: NULL pointer");
    return RBC_ERR_ARG;
  }
  int64_t M = 0;
  for (int i = 0; i < g->count; ++i) M += std::max<int64_t>(m[i], 0);
  if (M == 0 || k < 1 || k > MAX_C - 1) {
    set_error("rbc_group_tune: needs queries and 1 <= k <= %d", MAX_C - 1);
    return RBC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g->mu);
  int64_t* ids = nullptr;
  float* dist = nullptr;
  RBC_CUDA(cudaMalloc(&ids, M * k * sizeof(int64_t)));
  if (cudaMalloc(&dist, M * k * sizeof(float)) != cudaSuccess) {
    cudaFree(ids);
    set_error("rbc_group_tune: output allocation failed");
    return RBC_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // candidate work-item sizes: a quarter to a sixteenth of the largest index,
  // bounded to [1024, 32768] rows, plus the fixed choices
  std::vector<int> cand = {1024, 2048, 4096, 8192, 16384, 32768};
  int best = 0;
  float best_ms = 1e30f;
  int rc = RBC_OK;
  for (int W : cand) {
    if (W > std::max<int64_t>(g->nmax, 1024) * 2) continue;
    Plan* p = nullptr;
    rc = group_search(g, Q, m, k, ids, dist, st, W, true, &p);  // capture + warm-up
    if (rc != RBC_OK) break;
    float tot = 0.f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0, st);
      rc = group_search(g, Q, m, k, ids, dist, st, W, true, nullptr);
      cudaEventRecord(e1, st);
      if (rc != RBC_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (rc != RBC_OK) break;
    uint32_t err = 0;
    cudaMemcpy(&err, p->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (err) continue;  // this size overflowed a capacity: not a candidate
    if (tot < best_ms) {
      best_ms = tot;
      best = W;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(ids);
  cudaFree(dist);
  if (rc != RBC_OK) return rc;
  if (!best) {
    set_error("rbc_group_tune: no candidate size completed");
    return RBC_ERR_CUDA;
  }
  g->W = best;
  // keep only the chosen size's plans
  for (auto it = g->plans.begin(); it != g->plans.end();)
    it = it->second->W != best ? g->plans.erase(it) : std::next(it);
  if (chosen) *chosen = best;
  return RBC_OK;
}

int rbc_group_stats(rbc_group* g, rbc_grouped_stats* out) {
  if (!g || !out) {
    set_error("rbc_group_stats: NULL");
    return RBC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g->mu);
  *out = g->last;
  out->indexes = g->count;
  out->rows = g->N;
  out->representatives = g->R;
  out->dim = g->DG;
  // device counters and error flags of the most recent batch shape searched
  for (auto& kv : g->plans) {
    Plan& p = *kv.second;
    if (p.M != g->last.queries || p.W != g->last.work_item_points) continue;
    int c[8] = {0};
    uint32_t err = 0;
    RBC_CUDA(cudaMemcpy(c, p.counters, sizeof(c), cudaMemcpyDeviceToHost));
    RBC_CUDA(cudaMemcpy(&err, p.dev_err, sizeof(err), cudaMemcpyDeviceToHost));
    out->uncertified = c[0];
    out->fp64_ties = c[1] + c[5];
    out->device_errors = err;
    int nitems = 0;
    RBC_CUDA(cudaMemcpy(&nitems, p.toff + p.tiles, sizeof(int), cudaMemcpyDeviceToHost));
    out->work_items = nitems;
    out->tiles = p.tiles;
    break;
  }
  return RBC_OK;
}

void rbc_group_free(rbc_group* g) {
  if (!g) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  delete g;
  cudaSetDevice(prev);
}

}  // extern "C"
