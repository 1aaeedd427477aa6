// Exact finish of the query rows whose FP32 candidate set could not be
// certified (Section 3: BF returns the k nearest points; Section 5.2: the
// exact search always returns them).
//
// Every FP32 path ends in the select step (select.cu), which writes for each
// query k distinct database points ordered by their FP32 re-ranked distance
// and certifies that nothing outside its candidate set can still be among
// the k nearest.  A row fails that certificate when more points than the
// candidate set holds lie within the FP32 rounding bound of its k-th
// distance.  Such a row is finished here, with no candidate buffer and no
// capacity limit:
//
//   Let r_k be the row's k-th FP32 distance as written by the select step
//   and eps the relative bound of the FP32 re-rank.  The k written points are
//   k distinct database points, so the true k-th neighbour distance is at
//   most r_k / (1 - eps).  A point x can be among the k nearest only if
//   rho(q, x) <= r_k / (1 - eps), hence only if its own FP32 value satisfies
//   rho32(q, x) <= r_k (1 + eps) / (1 - eps).
//
// One CTA takes one row at a time (rows from a device-side list, so no count
// has to reach the host).  Groups of eight lanes evaluate one database point
// each in FP32 difference form (coalesced 16-byte reads); the few points
// inside the band above are evaluated again in FP64 and kept per group as
// the k smallest (rho64, id) pairs in shared memory.  A warp then merges the
// 32 group lists and overwrites the row's answer: the k nearest points of
// the FP64 brute force over the row's database range, in (rho, id) order.
// A band of any size is handled (a thousand equidistant duplicates are all
// evaluated in FP64 and ordered by id); it only costs time, and the band is
// empty but for the row's near-ties whenever the row's answer was right.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int BAND_THREADS = 256;
constexpr int BAND_GROUPS = BAND_THREADS / 8;  // one point per 8-lane group
constexpr int BAND_MAXK = 32;
constexpr float BAND_U32 = 5.9604645e-08f;  // 2^-24
constexpr int BAND_U = 4;                    // rows per group and step
// A launch with at most BAND_SPLIT_ROWS rows cuts each into BAND_SPLIT chunks
// of its range, one CTA each: a few rows over a large database would
// otherwise each stream it through one SM.
constexpr int BAND_SPLIT = 16;
constexpr int BAND_SPLIT_ROWS = 64;

__device__ __forceinline__ bool lt64(double a, int ia, double b, int ib) {
  return a < b || (a == b && ia < ib);
}

// two CTAs per SM: up to 128 registers, so the four-row steps do not spill
__global__ void __launch_bounds__(BAND_THREADS, 2) band_kernel(BandArgs a) {
  __shared__ __align__(16) float sq[MAX_D];
  __shared__ double s_r[BAND_GROUPS][BAND_MAXK];
  __shared__ int s_i[BAND_GROUPS][BAND_MAXK];
  __shared__ int s_n[BAND_GROUPS];
  const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 3, g8 = tid & 7;
  const int k = a.k, d = a.d;
  const int nrows = *a.nrows_dev;
  // work units: up to BAND_SPLIT_ROWS rows in BAND_SPLIT chunks of their
  // range (their chunk lists go to the split scratch, merged by
  // band_merge_kernel); more rows than that keep every SM busy whole (the
  // scan is then bound by HBM, not by one SM's reads)
  const int nsplit = (a.split_r && nrows <= BAND_SPLIT_ROWS) ? nrows : 0;
  const int units = nsplit * BAND_SPLIT + (nrows - nsplit);
  for (int un = blockIdx.x; un < units; un += gridDim.x) {
    const bool split = un < nsplit * BAND_SPLIT;
    const int fi = split ? un / BAND_SPLIT : nsplit + (un - nsplit * BAND_SPLIT);
    const int chunk = split ? un % BAND_SPLIT : 0;
    const int p = a.rows[fi];
    const int64_t orow = a.qorig ? (int64_t)a.qorig[p] : (int64_t)p;
    if (orow < 0) continue;  // padding row (the same for every thread)
    int64_t b = 0, e = a.n;
    if (a.tile_grp) {
      const int g = a.tile_grp[p / TQ];
      b = a.grp_base[g];
      e = b + a.grp_len[g];
    } else if (a.tile_list) {
      const int r = a.tile_list[p / TQ];
      b = a.list_off ? a.list_off[r] : (int64_t)r * a.list_len;
      e = a.list_off ? a.list_off[r + 1] : b + a.list_len;
    }
    if (split) {
      const int64_t len = e - b;
      const int64_t cb = b + len * chunk / BAND_SPLIT, ce = b + len * (chunk + 1) / BAND_SPLIT;
      b = cb;
      e = ce;
    }
    __syncthreads();  // the previous row's readers of sq and the lists are done
    for (int i = tid; i < d; i += BAND_THREADS) sq[i] = a.Q32[(int64_t)p * a.ld + i];
    if (tid < BAND_GROUPS) s_n[tid] = 0;
    // the band: FP32 values at most r_k (1 + eps) / (1 - eps), rounded up;
    // given a bound U of the true k-th distance instead: U (1 + eps)
    float thr;
    if (a.kth_bound) {
      const float ub = a.kth_bound[p];
      thr = ub < INFINITY ? ub * (1.0f + a.eps) * (1.0f + 8.0f * BAND_U32) : INFINITY;
    } else {
      const float rk = a.out_dist[orow * k + k - 1];
      thr = rk < INFINITY ? rk * (1.0f + a.eps) / (1.0f - a.eps) * (1.0f + 8.0f * BAND_U32)
                          : INFINITY;
    }
    __syncthreads();
    // BAND_U rows per group and step, their loads issued together (the
    // scan of a whole database is latency-bound otherwise)
    const bool vec = (d & 3) == 0 && (a.ld & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(a.X32) & 15) == 0;
    const int64_t iters = (e - b + BAND_GROUPS * BAND_U - 1) / (BAND_GROUPS * BAND_U);
    for (int64_t it = 0; it < iters; ++it) {
      float vu[BAND_U];
      if (vec) {
        rho8_rows<BAND_U>(sq, a.X32, a.ld, b, e, b + it * BAND_GROUPS * BAND_U + grp,
                          BAND_GROUPS, d, a.metric, g8, vu);
      } else {
#pragma unroll
        for (int u = 0; u < BAND_U; ++u) {
          const int64_t x = b + (it * BAND_U + u) * BAND_GROUPS + grp;
          vu[u] = rerank_rho8(sq, a.X32 + (x < e ? x : b) * a.ld, d, a.metric, g8);
        }
      }
#pragma unroll
      for (int u = 0; u < BAND_U; ++u) {
      const int64_t x = b + (it * BAND_U + u) * BAND_GROUPS + grp;
      const bool valid = x < e;
      const float* xr = a.X32 + (valid ? x : b) * a.ld;
      const float v = vu[u];
      const bool in = valid && v <= thr;
      if (__any_sync(0xffffffffu, in)) {
        const double r64 = rho64_8(sq, xr, d, a.metric, g8);
        if (in && g8 == 0) {
          // sorted insert into this group's list of at most k (one writer)
          const int id = a.xid ? a.xid[x] : (int)x;
          double* R = s_r[grp];
          int* I = s_i[grp];
          const int nn = s_n[grp];
          if (nn < k || lt64(r64, id, R[nn - 1], I[nn - 1])) {
            int j = nn < k ? nn : k - 1;
            while (j > 0 && lt64(r64, id, R[j - 1], I[j - 1])) {
              R[j] = R[j - 1];
              I[j] = I[j - 1];
              --j;
            }
            R[j] = r64;
            I[j] = id;
            if (nn < k) s_n[grp] = nn + 1;
          }
        }
      }
      }
    }
    __syncthreads();
    if (tid < 32) {
      // lane l holds group l's sorted list; k rounds of a warp arg-min
      const int cnt = s_n[lane];
      int head = 0;
      double myr = INFINITY;
      int myi = INT32_MAX;
      for (int j = 0; j < k; ++j) {
        double bv = head < cnt ? s_r[lane][head] : INFINITY;
        int bi = head < cnt ? s_i[lane][head] : INT32_MAX;
        int bl = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
          if (ov < bv || (ov == bv && (oi < bi || (oi == bi && ol < bl)))) {
            bv = ov;
            bi = oi;
            bl = ol;
          }
        }
        if (lane == bl) ++head;
        if (lane == j) {
          myr = bv;
          myi = bi;
        }
      }
      if (split) {
        // this chunk's k best, sorted, to the row's slot of the scratch
        const int64_t so = ((int64_t)fi * BAND_SPLIT + chunk) * BAND_MAXK;
        if (lane < k) {
          a.split_r[so + lane] = myr;
          a.split_i[so + lane] = myi;
        }
      } else if (lane < k) {
        const bool ok = myr < INFINITY;
        a.out_ids[orow * k + lane] = ok ? (int64_t)myi : (int64_t)-1;
        a.out_dist[orow * k + lane] = ok ? (float)myr : INFINITY;
      }
    }
  }
}

// The split rows: one warp per row merges its BAND_SPLIT sorted chunk lists
// (lane c holds chunk c's head) by k rounds of a warp arg-min over (rho64, id)
// and writes the row's answer.
__global__ void band_merge_kernel(BandArgs a) {
  const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int nrows = *a.nrows_dev;
  const int nsplit = nrows <= BAND_SPLIT_ROWS ? nrows : 0;
  if (w >= nsplit) return;
  const int p = a.rows[w];
  const int64_t orow = a.qorig ? (int64_t)a.qorig[p] : (int64_t)p;
  if (orow < 0) return;
  const int k = a.k;
  const int64_t so = ((int64_t)w * BAND_SPLIT + lane) * BAND_MAXK;
  int head = 0;
  double myr = INFINITY;
  int myi = INT32_MAX;
  for (int j = 0; j < k; ++j) {
    double bv = INFINITY;
    int bi = INT32_MAX;
    if (lane < BAND_SPLIT && head < k) {
      bv = a.split_r[so + head];
      bi = a.split_i[so + head];
    }
    int bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (ov < bv || (ov == bv && (oi < bi || (oi == bi && ol < bl)))) {
        bv = ov;
        bi = oi;
        bl = ol;
      }
    }
    if (lane == bl) ++head;
    if (lane == j) {
      myr = bv;
      myi = bi;
    }
  }
  if (lane < k) {
    const bool ok = myr < INFINITY;
    a.out_ids[orow * k + lane] = ok ? (int64_t)myi : (int64_t)-1;
    a.out_dist[orow * k + lane] = ok ? (float)myr : INFINITY;
  }
}

}  // namespace

int64_t band_split_scratch_entries() { return (int64_t)BAND_SPLIT_ROWS * BAND_SPLIT * BAND_MAXK; }

int launch_band(const BandArgs& a, int max_rows, cudaStream_t st) {
  if (max_rows <= 0) return RBC_OK;
  if (a.k < 1 || a.k > BAND_MAXK || a.d < 1 || a.d > MAX_D || a.ld < a.d || !a.rows ||
      !a.nrows_dev || !a.Q32 || !a.X32 || !a.out_ids || !a.out_dist) {
    set_error("band re-search: bad arguments (k=%d d=%d ld=%d)", a.k, a.d, a.ld);
    return RBC_ERR_ARG;
  }
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t units =
      a.split_r ? std::max<int64_t>((int64_t)std::min(max_rows, BAND_SPLIT_ROWS) * BAND_SPLIT,
                                    max_rows)
                : max_rows;
  const int grid = (int)std::min<int64_t>(units, (int64_t)sms * 4);
  band_kernel<<<grid, BAND_THREADS, 0, st>>>(a);
  RBC_LAUNCH_CHECK("band_kernel");
  if (a.split_r) {
    const int nw = std::min(max_rows, BAND_SPLIT_ROWS);
    band_merge_kernel<<<(nw * 32 + 255) / 256, 256, 0, st>>>(a);
    RBC_LAUNCH_CHECK("band_merge_kernel");
  }
  return RBC_OK;
}

}  // namespace rbc
