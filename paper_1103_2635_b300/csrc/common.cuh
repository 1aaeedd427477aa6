// Shared device/host definitions for the RBC library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cfloat>
#include <cmath>

#include "../../include/rbc.h"

namespace rbc {

// Query tile height: every distance kernel processes queries in tiles of this
// many rows, and the exact search forms one union of kept lists per tile.
constexpr int TQ = 128;

// One contiguous run of database rows [x_begin, x_end) in a database buffer.
struct Seg {
  int32_t x_begin;
  int32_t x_end;
};

// A unit of distance work: queries [q_row0, q_row0 + nq) of the query buffer
// against the union of segs[seg_begin .. seg_end); results go to partial slot
// `slot`.
struct WorkItem {
  int32_t q_row0;
  int32_t nq;
  int32_t seg_begin;
  int32_t seg_end;
  int32_t slot;
  int32_t tile;
};

// Ordering used by every selection: (score, index) lexicographic.
__device__ __forceinline__ bool pair_lt(float a, int ia, float b, int ib) {
  return a < b || (a == b && ia < ib);
}

// Sorted register list of C (score, index) pairs, ascending.  Insert walks the
// list once, carrying the larger element of each compare-swap downwards; the
// last element falls off.  Fully unrolled so the arrays stay in registers.
template <int C>
struct TopList {
  float s[C];
  int i[C];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      s[j] = INFINITY;
      i[j] = INT32_MAX;
    }
  }
  __device__ __forceinline__ float worst() const { return s[C - 1]; }
  __device__ __forceinline__ bool admits(float v, int id) const {
    return pair_lt(v, id, s[C - 1], i[C - 1]);
  }
  __device__ __forceinline__ void insert(float v, int id) {
    float cv = v;
    int ci = id;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      bool lt = pair_lt(cv, ci, s[j], i[j]);
      float ts = lt ? s[j] : cv;
      int ti = lt ? i[j] : ci;
      s[j] = lt ? cv : s[j];
      i[j] = lt ? ci : i[j];
      cv = ts;
      ci = ti;
    }
  }
};

// rho(q, x) of a candidate row by the eight lanes of a group (g8 = lane % 8):
// lane g8 sums elements g8, g8 + 8, ... (float4 steps when rows allow it),
// then the group adds its eight partial sums as a tree; every lane of the
// group returns the result.  FP32 error: d / 8 + 3 roundings of the sum.
__device__ __forceinline__ float rerank_rho8(const float* qr, const float* xr, int d, int metric,
                                             int g8) {
  float p = 0.f;
  if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(qr) | reinterpret_cast<uintptr_t>(xr)) & 15) == 0) {
    const float4* q4 = reinterpret_cast<const float4*>(qr);
    const float4* x4 = reinterpret_cast<const float4*>(xr);
    for (int i = g8; i < d / 4; i += 8) {
      const float4 a = q4[i], b = x4[i];
      const float t0 = a.x - b.x, t1 = a.y - b.y, t2 = a.z - b.z, t3 = a.w - b.w;
      if (metric == RBC_L2) {
        p = fmaf(t0, t0, p);
        p = fmaf(t1, t1, p);
        p = fmaf(t2, t2, p);
        p = fmaf(t3, t3, p);
      } else {
        p += fabsf(t0) + fabsf(t1) + fabsf(t2) + fabsf(t3);
      }
    }
  } else {
    for (int i = g8; i < d; i += 8) {
      const float t = qr[i] - xr[i];
      p = metric == RBC_L2 ? fmaf(t, t, p) : p + fabsf(t);
    }
  }
  p += __shfl_xor_sync(0xffffffffu, p, 1);
  p += __shfl_xor_sync(0xffffffffu, p, 2);
  p += __shfl_xor_sync(0xffffffffu, p, 4);
  return metric == RBC_L2 ? sqrtf(p) : p;
}

// rerank_rho8 of U gathered rows xr[u] by the eight lanes of a group (d a
// multiple of 4, rows and query 16-byte aligned): the float4 elements of all
// U rows, up to four per lane and row (all of a row for d <= 128), are loaded
// before any is used, so a group keeps up to 4 U loads in flight.  Every sum
// runs in rerank_rho8's order (ascending element, then the same shuffle
// tree), so the values are bit-identical to it.
template <int U>
__device__ __forceinline__ void rho8_gather(const float* qr, const float* const (&xr)[U], int d,
                                            int metric, int g8, float (&out)[U]) {
  const float4* q4 = reinterpret_cast<const float4*>(qr);
  const int n4 = d / 4;
#pragma unroll
  for (int u = 0; u < U; ++u) out[u] = 0.f;
  for (int i0 = g8; i0 < n4; i0 += 32) {
    float4 v[4][U];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = i0 + 8 * s;
#pragma unroll
      for (int u = 0; u < U; ++u)
        v[s][u] = i < n4 ? reinterpret_cast<const float4*>(xr[u])[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = i0 + 8 * s;
      if (i < n4) {
        const float4 qa = q4[i];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float t0 = qa.x - v[s][u].x, t1 = qa.y - v[s][u].y, t2 = qa.z - v[s][u].z,
                      t3 = qa.w - v[s][u].w;
          if (metric == RBC_L2) {
            out[u] = fmaf(t0, t0, out[u]);
            out[u] = fmaf(t1, t1, out[u]);
            out[u] = fmaf(t2, t2, out[u]);
            out[u] = fmaf(t3, t3, out[u]);
          } else {
            out[u] += fabsf(t0) + fabsf(t1) + fabsf(t2) + fabsf(t3);
          }
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    float p = out[u];
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    p += __shfl_xor_sync(0xffffffffu, p, 4);
    out[u] = metric == RBC_L2 ? sqrtf(p) : p;
  }
}

// FP32 distances of the rows rows[0 .. n) (shared memory) to the query, into
// out[0 .. n) (shared memory), by the whole warp: 4 U rows per round (U per
// group of eight lanes, gathered loads; a larger U keeps more loads in flight
// for long lists, a smaller one fewer registers for short ones), or
// rerank_rho8 row by row when the layout does not allow 16-byte loads.
template <int U>
__device__ __forceinline__ void rerank_rows(const float* qr, const float* X32, int d, int metric,
                                            const int* rows, int n, float* out, int lane) {
  const int g = lane >> 3, g8 = lane & 7;
  if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(qr) | reinterpret_cast<uintptr_t>(X32)) & 15) == 0) {
    for (int e0 = 0; e0 < n; e0 += 4 * U) {
      const float* xr[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + g + 4 * u;
        xr[u] = X32 + (int64_t)rows[e < n ? e : 0] * d;
      }
      float v[U];
      rho8_gather<U>(qr, xr, d, metric, g8, v);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + g + 4 * u;
        if (g8 == 0 && e < n) out[e] = v[u];
      }
    }
  } else {
    for (int e0 = 0; e0 < n; e0 += 4) {
      const int e = e0 + g;
      const float v = rerank_rho8(qr, X32 + (int64_t)rows[e < n ? e : 0] * d, d, metric, g8);
      if (g8 == 0 && e < n) out[e] = v;
    }
  }
}

// rerank_rho8 of U rows at once (rows x0 + u * stride, u < U; rows at or past
// e read row b instead and are ignored by the caller): the eight lanes of a
// group load all U rows' float4 elements first, then reduce each.  Rows are
// ld floats apart, ld and d multiples of 4 and X 16-byte aligned.
template <int U>
__device__ __forceinline__ void rho8_rows(const float* qr, const float* __restrict__ X, int ld,
                                          int64_t b, int64_t e, int64_t x0, int stride, int d,
                                          int metric, int g8, float (&out)[U]) {
  const float4* q4 = reinterpret_cast<const float4*>(qr);
  const float4* xr[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t x = x0 + (int64_t)u * stride;
    xr[u] = reinterpret_cast<const float4*>(X + (x < e ? x : b) * ld);
    out[u] = 0.f;
  }
  for (int i = g8; i < d / 4; i += 8) {
    const float4 qa = q4[i];
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = xr[u][i];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float t0 = qa.x - v[u].x, t1 = qa.y - v[u].y, t2 = qa.z - v[u].z, t3 = qa.w - v[u].w;
      if (metric == RBC_L2) {
        out[u] = fmaf(t0, t0, out[u]);
        out[u] = fmaf(t1, t1, out[u]);
        out[u] = fmaf(t2, t2, out[u]);
        out[u] = fmaf(t3, t3, out[u]);
      } else {
        out[u] += fabsf(t0) + fabsf(t1) + fabsf(t2) + fabsf(t3);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    float p = out[u];
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    p += __shfl_xor_sync(0xffffffffu, p, 4);
    out[u] = metric == RBC_L2 ? sqrtf(p) : p;
  }
}

// The same distance in FP64 (from the FP32 inputs), by the eight lanes of a
// group; every lane of the group returns it.  All 32 lanes of the warp must
// call it together.
__device__ __forceinline__ double rho64_8(const float* qr, const float* xr, int d, int metric,
                                          int g8) {
  double p = 0.0;
  for (int i = g8; i < d; i += 8) {
    const double t = (double)qr[i] - (double)xr[i];
    p += metric == RBC_L2 ? t * t : fabs(t);
  }
  p += __shfl_xor_sync(0xffffffffu, p, 1);
  p += __shfl_xor_sync(0xffffffffu, p, 2);
  p += __shfl_xor_sync(0xffffffffu, p, 4);
  return metric == RBC_L2 ? sqrt(p) : p;
}

// Largest low-precision score |x~|^2 - 2 q~.x~ that a point within distance
// g of q can have: (g + |q - q~| + max |x - x~|)^2 - |q~|^2 + E_f, with E_f the
// FP32 evaluation bound (d + 4) 2^-19 (|q~| + max |x~|)^2 (doubled), rounded up.
__host__ __device__ __forceinline__ float score_bound(float g, float qn, float qerr, float xerr,
                                             float xnmax, int d) {
  if (!(g < INFINITY)) return INFINITY;
  const float G = (g + qerr + xerr) * (1.0f + 4.8e-7f);
  const float span = (sqrtf(qn) + xnmax) * (1.0f + 4.8e-7f);
  // doubled FP32 evaluation bound, plus 2^-16 max|x~|^2 for a norm term that
  // enters as a bf16 (high, low) pair (error <= 2^-17 |x~|^2)
  const float ef = 2.0f * (float)(d + 4) * 1.9073486e-06f * span * span +
                   1.5258789e-05f * xnmax * xnmax;
  return (G * G * (1.0f + 4.8e-7f) - qn * (1.0f - 4.8e-7f) + ef) * (1.0f + 4.8e-7f) + 1e-30f;
}

// Largest distance a point with low-precision score s can have from q:
// sqrt(s + |q~|^2 + E_f) + |q - q~| + max |x - x~|, rounded up.
__host__ __device__ __forceinline__ float dist_upper(float s, float qn, float qerr, float xerr, float xnmax,
                                            int d) {
  if (!(s < INFINITY)) return INFINITY;
  const float span = (sqrtf(qn) + xnmax) * (1.0f + 4.8e-7f);
  const float ef = 2.0f * (float)(d + 4) * 1.9073486e-06f * span * span;
  const float t = (s + qn * (1.0f + 4.8e-7f) + ef) * (1.0f + 4.8e-7f);
  return (sqrtf(fmaxf(t, 0.0f)) * (1.0f + 4.8e-7f) + qerr + xerr) * (1.0f + 4.8e-7f);
}

// Representative-offset estimates (windowed plan with offset rows, bf16).
// The query row a = q - r and each list row y = x - r of r's list are formed
// in FP32 and rounded to bf16; with eps >= |a - a~| + |y - y~| (measured
// residuals: the query row's from its own rounding, the list's largest from
// the build, plus the FP32 subtraction's 2^-24 |a|) the exact distance
// rho = |a - y| is within eps of |a~ - y~|.  The kernel's estimate v of
// |a~ - y~|^2 (the FP32 |a~|^2 minus twice the accumulator of
// a~.y~ - |y~|^2 / 2) is within A(M) = (2 (d + 4) 2^-19 + 2^-15) (M (1 + c))^2
// of |a~ - y~|^2 for M >= |a| + |y| and c = 2^-8 (1 + 2^-7) >= the bf16
// rounding's relative size: the low-precision score's FP32 evaluation and
// norm-pair terms as in score_bound, plus the FP32 |a~|^2 and the final
// subtraction.  Hence rho <= sqrt(max(v, 0) + A) + eps and
// rho >= sqrt(max(0, v - A)) - eps.
constexpr float OFF_C = 3.9367676e-03f;  // 2^-8 (1 + 2^-7)
// M of a (query, representative) pair from rho(q, r) as stage one computed it
// (relative error below 1e-4) and the list's radius bound psi_r; explicit
// roundings, so that every kernel computes the same value from the same inputs
__host__ __device__ __forceinline__ float off_pair_m(float rho_qr, float psi_r) {
#ifdef __CUDA_ARCH__
  return __fmul_ru(__fadd_ru(__fmul_ru(rho_qr, 1.0001f), psi_r), 1.0000005f);
#else
  return (rho_qr * 1.0001f + psi_r) * 1.0000005f;
#endif
}
__host__ __device__ __forceinline__ float off_arith(float M, int d) {
  const float s = M * (1.0f + OFF_C) * (1.0f + 4.8e-7f);
  return ((float)(2 * (d + 4)) * 1.9073486e-06f + 3.0517578e-05f) * s * s * (1.0f + 4.8e-7f);
}
// Largest estimate v a point within distance g of q can have.
__host__ __device__ __forceinline__ float off_value_bound(float g, float M, float eps, int d) {
  if (!(g < INFINITY)) return INFINITY;
  const float G = (g + eps) * (1.0f + 4.8e-7f);
  return (G * G * (1.0f + 4.8e-7f) + off_arith(M, d)) * (1.0f + 4.8e-7f) + 1e-30f;
}
// Largest distance a point with estimate v can have from q.
__host__ __device__ __forceinline__ float off_dist_upper(float v, float M, float eps, int d) {
  if (!(v < INFINITY)) return INFINITY;
  const float t = (fmaxf(v, 0.0f) + off_arith(M, d)) * (1.0f + 4.8e-7f);
  return (sqrtf(t) * (1.0f + 4.8e-7f) + eps) * (1.0f + 4.8e-7f);
}

// FP32 difference-form values (rho^2 for l2, rho for l1) with relative error
// at most eps: the largest distance a value s can stand for (s >= v (1 - eps)
// for the exact value v, so v <= s (1 + 2 eps)), and the largest value a point
// within distance g can have (g^2 (1 + eps) for l2, g (1 + eps) for l1), both
// rounded up.
__host__ __device__ __forceinline__ float f32_dist_upper(float s, float eps, int metric) {
  if (!(s < INFINITY)) return INFINITY;
  const float t = fmaxf(s, 0.0f) * (1.0f + 2.0f * eps) * (1.0f + 4.8e-7f);
  return metric == RBC_L2 ? sqrtf(t) * (1.0f + 4.8e-7f) : t;
}
__host__ __device__ __forceinline__ float f32_score_bound(float g, float eps, int metric) {
  if (!(g < INFINITY)) return INFINITY;
  const float G = g * (1.0f + 4.8e-7f);
  const float v = metric == RBC_L2 ? G * G * (1.0f + 4.8e-7f) : G;
  return v * (1.0f + eps) * (1.0f + 4.8e-7f) + 1e-30f;
}

// Device-side error flags (bit mask), read back by the host after a call.
enum : uint32_t {
  DEV_ERR_TIMEOUT = 1u,      // a bounded wait gave up
  DEV_ERR_BOUNDS = 2u,       // an index check failed (access skipped)
  DEV_ERR_CAPACITY = 4u,     // a worst-case buffer bound was exceeded
};

}  // namespace rbc

// ---------------------------------------------------------------------------
// Host-side error plumbing shared by the .cu files.
// ---------------------------------------------------------------------------
namespace rbc {
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
extern thread_local long long t_launches;  // kernels launched by this thread
}  // namespace rbc

#define RBC_CUDA(call)                                                                \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess) return ::rbc::cuda_fail(_e, #call, __FILE__, __LINE__);    \
  } while (0)

#define RBC_LAUNCH_CHECK(what)                                                        \
  do {                                                                                \
    ++::rbc::t_launches;                                                              \
    cudaError_t _e = cudaGetLastError();                                              \
    if (_e != cudaSuccess) return ::rbc::cuda_fail(_e, what, __FILE__, __LINE__);     \
  } while (0)
