// One-shot Random Ball Cover (Sections 4 and 5.1).
//
// Build: BF(R, X) with k = s.  Every representative's list L_r is the s
// nearest database points of r in (rho, id) order and psi_r the s-th
// distance.  The distances come from the FP32 tile kernel (store mode) one
// block of representatives at a time; per representative an exact radix
// select finds the s-th smallest FP32 distance t, every point within the FP32
// rounding bound of t is kept as a candidate (a superset of the true s
// nearest), the candidates are recomputed in FP64 and sorted by (rho, id) with
// a bitonic network in shared memory, and the first s form L_r.
//
// Search: BF(q, R) gives q's nearest representative r (ties to the smaller
// ordinal), and BF(q, X[L_r]) the answer.  Queries are regrouped so that every
// 128-query tile belongs to one representative (tiles are padded), which makes
// stage two a dense tile against exactly one list.
#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int SEL_THREADS = 1024;
constexpr int RADIX_BITS = 11;
constexpr int RADIX_BINS = 1 << RADIX_BITS;

// Block-wide exclusive search in a histogram: the bin in which the running
// count reaches `want` (1-based rank), and the count of entries before it.
__device__ void find_bin(const int* hist, int want, int* s_bin, int* s_before) {
  __shared__ int warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // each thread owns two consecutive bins
  const int b0 = 2 * t;
  const int c0 = hist[b0], c1 = hist[b0 + 1];
  int x = c0 + c1;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = warp_tot[lane];
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, iv, o);
      if (lane >= o) iv += y;
    }
    warp_tot[lane] = iv - v;  // exclusive over warps
  }
  __syncthreads();
  const int before = warp_tot[wid] + incl - x;  // entries before bin b0
  if (before < want && before + c0 >= want) {
    *s_bin = b0;
    *s_before = before;
  } else if (before + c0 < want && before + c0 + c1 >= want) {
    *s_bin = b0 + 1;
    *s_before = before + c0;
  }
  __syncthreads();
}

// Per representative row of D (non-negative FP32 distances): the s-th
// smallest value t (exact, by radix select over the float bit patterns) and
// every column whose distance is <= t (1 + 3 eps) appended to cand[r].
__global__ void __launch_bounds__(SEL_THREADS)
oneshot_select_kernel(const float* __restrict__ D, int64_t ld, int64_t n, int s, float eps,
                      int cap, int* __restrict__ cand, int* __restrict__ cand_cnt,
                      uint32_t* dev_err) {
  __shared__ int hist[RADIX_BINS];
  __shared__ int s_bin, s_before, s_cnt;
  const unsigned* row = reinterpret_cast<const unsigned*>(D + (int64_t)blockIdx.x * ld);
  unsigned prefix = 0, pmask = 0;
  int want = s;
  // 32-bit keys in three digits: bits 31..21, 20..10, 9..0
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  for (int pass = 0; pass < 3; ++pass) {
    for (int i = threadIdx.x; i < RADIX_BINS; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int sh = shifts[pass];
    const unsigned dmask = (1u << widths[pass]) - 1u;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      unsigned key = row[i];
      if ((key & pmask) == prefix) atomicAdd(&hist[(key >> sh) & dmask], 1);
    }
    __syncthreads();
    find_bin(hist, want, &s_bin, &s_before);
    prefix |= (unsigned)s_bin << sh;
    pmask |= dmask << sh;
    want -= s_before;
    __syncthreads();
  }
  const float t = __uint_as_float(prefix);
  const float lim = t * (1.0f + 3.0f * eps) + 1e-30f;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  int* out = cand + (int64_t)blockIdx.x * cap;
  const float* rowf = D + (int64_t)blockIdx.x * ld;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    if (rowf[i] <= lim) {
      int pos = atomicAdd(&s_cnt, 1);
      if (pos < cap) out[pos] = (int)i;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cand_cnt[blockIdx.x] = min(s_cnt, cap);
    if (s_cnt > cap) atomicOr(dev_err, DEV_ERR_CAPACITY);
  }
}

// FP64 distances of the candidates (difference form, dimensions summed in
// order), bitonic sort by (rho64, id), first s.
// The candidate capacity is a power of two <= 8192 (shared memory: 12 bytes each).
__global__ void __launch_bounds__(SEL_THREADS)
oneshot_refine_kernel(const float* __restrict__ X, const float* __restrict__ R, int d, int metric,
                      int s, int cap, const int* __restrict__ cand,
                      const int* __restrict__ cand_cnt, int r0, int* __restrict__ members,
                      float* __restrict__ psi, uint32_t* dev_err) {
  extern __shared__ unsigned char sm[];
  double* key = reinterpret_cast<double*>(sm);
  int* id = reinterpret_cast<int*>(key + cap);
  const int r = blockIdx.x;
  const int cnt = cand_cnt[r];
  const int* cr = cand + (int64_t)r * cap;
  const float* rv = R + (int64_t)(r0 + r) * d;
  for (int i = threadIdx.x; i < cap; i += blockDim.x) {
    if (i < cnt) {
      const int xi = cr[i];
      const float* xv = X + (int64_t)xi * d;
      double acc = 0.0;
      for (int j = 0; j < d; ++j) {
        double t = (double)rv[j] - (double)xv[j];
        acc += metric == RBC_L2 ? t * t : fabs(t);
      }
      key[i] = metric == RBC_L2 ? sqrt(acc) : acc;
      id[i] = xi;
    } else {
      key[i] = INFINITY;
      id[i] = INT32_MAX;
    }
  }
  __syncthreads();
  for (int size = 2; size <= cap; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const bool gt = key[i] > key[j] || (key[i] == key[j] && id[i] > id[j]);
          if (gt == up) {
            double tk = key[i];
            key[i] = key[j];
            key[j] = tk;
            int ti = id[i];
            id[i] = id[j];
            id[j] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  int* mr = members + (int64_t)(r0 + r) * s;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    int v = id[i];
    if (v == INT32_MAX) {  // fewer than s candidates (non-finite distances)
      v = 0;
      atomicOr(dev_err, DEV_ERR_BOUNDS);
    }
    mr[i] = v;
  }
  if (threadIdx.x == 0) psi[r0 + r] = (float)key[s - 1];
}

// Queries regrouped by nearest representative with every representative's
// run padded to a multiple of TQ: padded row -> source row and output row (or
// -1), and per tile its representative.
__global__ void oneshot_layout_kernel(const int* __restrict__ qoff, int n_r,
                                      const int* __restrict__ qperm, const int* __restrict__ orig,
                                      const int* __restrict__ pad_off, int* __restrict__ qsrc_pad,
                                      int* __restrict__ qout_pad, int* __restrict__ tile_rep) {
  const int r = blockIdx.x;
  if (r >= n_r) return;
  const int b = qoff[r], e = qoff[r + 1];
  const int pb = pad_off[r], pe = pad_off[r + 1];
  for (int i = threadIdx.x; i < pe - pb; i += blockDim.x) {
    const int src = (b + i < e) ? qperm[b + i] : -1;
    qsrc_pad[pb + i] = src;
    qout_pad[pb + i] = src < 0 ? -1 : (orig ? orig[src] : src);
  }
  for (int t = pb / TQ + threadIdx.x; t < pe / TQ; t += blockDim.x) tile_rep[t] = r;
}

__global__ void fallback_map_kernel(const int* __restrict__ rows, int n,
                                    const int* __restrict__ tile_rep,
                                    const int* __restrict__ qout_pad, int64_t* __restrict__ rep64,
                                    int* __restrict__ out_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int row = rows[i];
  rep64[i] = tile_rep[row / TQ];
  out_row[i] = qout_pad[row];
}

__global__ void padded_counts_kernel(const int* __restrict__ qoff, int n_r, int* __restrict__ out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_r) out[r] = (qoff[r + 1] - qoff[r] + TQ - 1) / TQ * TQ;
}

__global__ void oneshot_items_kernel(const int* __restrict__ pad_off, int n_r,
                                     const int* __restrict__ tile_rep,
                                     const int* __restrict__ qoff, int s,
                                     const int* __restrict__ list_off,
                                     WorkItem* __restrict__ items,
                                     Seg* __restrict__ segs, int* __restrict__ num_items,
                                     int max_tiles, unsigned long long* points_sum) {
  const int tiles = pad_off[n_r] / TQ;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *num_items = min(tiles, max_tiles);
    if (points_sum && !list_off)
      atomicAdd(points_sum, (unsigned long long)min(tiles, max_tiles) * s);
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles && t < max_tiles;
       t += gridDim.x * blockDim.x) {
    const int r = tile_rep[t];
    const int valid = qoff[r + 1] - qoff[r] - (t * TQ - pad_off[r]);
    items[t] = WorkItem{t * TQ, min(TQ, valid), t, t + 1, t, t};
    const Seg sg = list_off ? Seg{list_off[r], list_off[r + 1]} : Seg{r * s, (r + 1) * s};
    segs[t] = sg;
    if (points_sum && list_off) atomicAdd(points_sum, (unsigned long long)(sg.x_end - sg.x_begin));
  }
}

__global__ void gather_padded_kernel(const float* __restrict__ Q, const int* __restrict__ src,
                                     int64_t rows, int d, float* __restrict__ out) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const int q = src[w];
  for (int i = lane; i < d; i += 32) out[w * d + i] = q >= 0 ? Q[(int64_t)q * d + i] : 0.f;
}

}  // namespace

int oneshot_candidate_cap(int s) {
  int cap = 1;
  while (cap < s + s / 4 + 64) cap <<= 1;
  return cap;
}

int launch_oneshot_select(const float* D, int64_t ld, int64_t n, int reps, int s, float eps,
                          int cap, int* cand, int* cand_cnt, uint32_t* dev_err, cudaStream_t st) {
  if (reps <= 0) return RBC_OK;
  oneshot_select_kernel<<<reps, SEL_THREADS, 0, st>>>(D, ld, n, s, eps, cap, cand, cand_cnt,
                                                      dev_err);
  RBC_LAUNCH_CHECK("oneshot_select_kernel");
  return RBC_OK;
}

int launch_oneshot_refine(const float* X, const float* R, int d, int metric, int s, int cap,
                          const int* cand, const int* cand_cnt, int r0, int reps, int* members,
                          float* psi, uint32_t* dev_err, cudaStream_t st) {
  if (reps <= 0) return RBC_OK;
  size_t smem = (size_t)cap * (sizeof(double) + sizeof(int));
  RBC_CUDA(cudaFuncSetAttribute(oneshot_refine_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  oneshot_refine_kernel<<<reps, SEL_THREADS, smem, st>>>(X, R, d, metric, s, cap, cand, cand_cnt,
                                                         r0, members, psi, dev_err);
  RBC_LAUNCH_CHECK("oneshot_refine_kernel");
  return RBC_OK;
}

int launch_oneshot_layout(const int* qoff, int n_r, const int* qperm, const int* orig,
                          int* counts_scratch, int* pad_off, int* qsrc_pad, int* qout_pad,
                          int* tile_rep, cudaStream_t st) {
  padded_counts_kernel<<<(n_r + 255) / 256, 256, 0, st>>>(qoff, n_r, counts_scratch);
  RBC_LAUNCH_CHECK("padded_counts_kernel");
  int rc = launch_exclusive_scan(counts_scratch, n_r, pad_off, st);
  if (rc != RBC_OK) return rc;
  oneshot_layout_kernel<<<n_r, 128, 0, st>>>(qoff, n_r, qperm, orig, pad_off, qsrc_pad, qout_pad,
                                             tile_rep);
  RBC_LAUNCH_CHECK("oneshot_layout_kernel");
  return RBC_OK;
}

int launch_oneshot_fallback_map(const int* rows, int n, const int* tile_rep, const int* qout_pad,
                                int64_t* rep64, int* out_row, cudaStream_t st) {
  if (n <= 0) return RBC_OK;
  fallback_map_kernel<<<(n + 255) / 256, 256, 0, st>>>(rows, n, tile_rep, qout_pad, rep64,
                                                       out_row);
  RBC_LAUNCH_CHECK("fallback_map_kernel");
  return RBC_OK;
}

int launch_oneshot_items(const int* pad_off, int n_r, const int* tile_rep, const int* qoff, int s,
                         const int* list_off, WorkItem* items, Seg* segs, int* num_items,
                         int max_tiles, unsigned long long* points_sum, cudaStream_t st) {
  oneshot_items_kernel<<<64, 256, 0, st>>>(pad_off, n_r, tile_rep, qoff, s, list_off, items, segs,
                                           num_items, max_tiles, points_sum);
  RBC_LAUNCH_CHECK("oneshot_items_kernel");
  return RBC_OK;
}

int launch_gather_padded(const float* Q, const int* src, int64_t rows, int d, float* out,
                         cudaStream_t st) {
  if (rows <= 0) return RBC_OK;
  gather_padded_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(Q, src, rows, d, out);
  RBC_LAUNCH_CHECK("gather_padded_kernel");
  return RBC_OK;
}

}  // namespace rbc
