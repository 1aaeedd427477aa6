// Data movement and storage preparation.
//
// gather_rows: dst[i] = src[idx[i]] for FP32 rows (representatives, lists in
//   permuted order, queries in tile order).  One warp per row, float4 when the
//   row length allows it.
// to_lowp: FP32 rows -> bf16 / fp16 rows padded with zeros to `dpad` columns
//   (a multiple of 64, the tensor-core K block), plus per row the FP32 norm
//   |x~|^2 of the rounded row and an upper bound of the rounding residual
//   |x - x~| (FP32 with every operation rounded up).  The residual bounds how far any distance
//   can move under rounding (triangle inequality of the metric:
//   |rho(q~, x~) - rho(q, x)| <= |q - q~| + |x - x~|), which the exact search
//   needs to stay exact with low-precision storage.
// to_fp8: FP32 rows -> FP8 E4M3 rows padded to `dpad` (a multiple of 128) with
//   a per-row scale s (the row's max |x_i| / 448 rounded up to a power of two,
//   so x / s and s * e4m3 are exact): x~ = s * e4m3(x / s).  Norm and residual
//   as above, of the dequantised row x~.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

__global__ void gather_rows_kernel(const float* __restrict__ src, const int64_t* __restrict__ idx64,
                                   const int* __restrict__ idx32, int64_t rows, int d,
                                   float* __restrict__ dst) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const int64_t s = idx64 ? idx64[w] : (int64_t)idx32[w];
  const float* a = src + s * d;
  float* b = dst + w * d;
  if ((d & 3) == 0) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    float4* b4 = reinterpret_cast<float4*>(b);
    for (int i = lane; i < (d >> 2); i += 32) b4[i] = a4[i];
  } else {
    for (int i = lane; i < d; i += 32) b[i] = a[i];
  }
}

template <typename T>
__device__ __forceinline__ T to_lp(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_lp<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half to_lp<__half>(float v) {
  return __float2half_rn(v);
}
__device__ __forceinline__ float from_lp(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float from_lp(__half v) { return __half2float(v); }

template <typename T>
__global__ void to_lowp_kernel(const float* __restrict__ src, int64_t rows, int d, int dpad,
                               T* __restrict__ dst, float* __restrict__ norm,
                               float* __restrict__ err, unsigned* err_max_bits,
                               unsigned* norm_max_bits) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const float* a = src + w * d;
  T* b = dst + w * dpad;
  // |x - x~| as an upper bound in FP32: v - r is exact (r is v rounded to
  // fewer significant bits, so within a factor 2 of v, or 0), and every
  // square, sum and the root round upward (a nonzero square never rounds to
  // zero), so e >= the exact residual
  float nrm = 0.f, e2 = 0.f;
  for (int i = lane; i < dpad; i += 32) {
    float v = i < d ? a[i] : 0.f;
    T lv = to_lp<T>(v);
    b[i] = lv;
    float r = from_lp(lv);
    nrm = fmaf(r, r, nrm);
    const float diff = v - r;
    e2 = __fadd_ru(e2, __fmul_ru(diff, diff));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    e2 = __fadd_ru(e2, __shfl_xor_sync(0xffffffffu, e2, o));
  }
  if (lane == 0) {
    float e = __fsqrt_ru(e2);
    norm[w] = nrm;
    if (err) err[w] = e;
    // non-negative floats order like their bit patterns
    if (err_max_bits) atomicMax(err_max_bits, __float_as_uint(e));
    if (norm_max_bits) atomicMax(norm_max_bits, __float_as_uint(__fsqrt_ru(nrm)));
  }
}

// E4M3 rows with a per-row power-of-two scale.  One warp per row.
__global__ void to_fp8_kernel(const float* __restrict__ src, int64_t rows, int d, int dpad,
                              uint8_t* __restrict__ dst, float* __restrict__ norm,
                              float* __restrict__ err, float* __restrict__ scale,
                              unsigned* err_max_bits, unsigned* norm_max_bits) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const float* a = src + w * d;
  uint8_t* b = dst + w * dpad;
  float amax = 0.f;
  for (int i = lane; i < d; i += 32) amax = fmaxf(amax, fabsf(a[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  // s = 2^ceil(log2(amax / 448)): |x_i| / s <= 448, the largest finite E4M3
  // (a row whose quotient rounds below a power of two saturates at 448; the
  // residual below records that error like any other)
  int e = 0;
  const float f = frexpf(amax * (1.0f / 448.0f), &e);
  if (f == 0.5f) e -= 1;
  const float sc = amax > 0.f ? ldexpf(1.0f, e) : 1.0f;
  const float inv = 1.0f / sc;  // a power of two: exact
  float nrm = 0.f;
  double e2 = 0.0;
  for (int i = lane; i < dpad; i += 32) {
    const float v = i < d ? a[i] : 0.f;
    const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3);
    b[i] = (uint8_t)q;
    const float r = sc * __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
    nrm = fmaf(r, r, nrm);
    const double diff = (double)v - (double)r;
    e2 += diff * diff;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  }
  if (lane == 0) {
    const float er = __double2float_ru(sqrt(e2));
    norm[w] = nrm;
    scale[w] = sc;
    if (err) err[w] = er;
    if (err_max_bits) atomicMax(err_max_bits, __float_as_uint(er));
    if (norm_max_bits) atomicMax(norm_max_bits, __float_as_uint(__fsqrt_ru(nrm)));
  }
}

// Result rows i of a search over gathered queries go to output row dst[i].
__global__ void scatter_result_rows_kernel(const int64_t* __restrict__ ids,
                                           const float* __restrict__ dist,
                                           const int* __restrict__ dst, int64_t rows, int k,
                                           int64_t* __restrict__ out_ids,
                                           float* __restrict__ out_dist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * k) return;
  const int64_t r = i / k;
  const int j = (int)(i - r * k);
  const int64_t o = (int64_t)dst[r] * k + j;
  out_ids[o] = ids[i];
  out_dist[o] = dist[i];
}

// dst row i = src row idx[i] of a low-precision matrix (rows of row_bytes)
// with its norm, residual and (FP8) scale; idx[i] < 0 gives a zero row (norm
// 0, residual 0, scale 1).  One warp per row, 16-byte copies.
__global__ void gather_lp_rows_kernel(const uint4* __restrict__ src, const float* __restrict__ snorm,
                                      const float* __restrict__ serr, const int* __restrict__ idx,
                                      int64_t rows, int vec_per_row, uint4* __restrict__ dst,
                                      float* __restrict__ dnorm, float* __restrict__ derr,
                                      const float* __restrict__ sscale, float* __restrict__ dscale) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const int s = idx[w];
  for (int j = lane; j < vec_per_row; j += 32)
    dst[w * vec_per_row + j] = s >= 0 ? src[(int64_t)s * vec_per_row + j] : make_uint4(0, 0, 0, 0);
  if (lane == 0) {
    dnorm[w] = s >= 0 ? snorm[s] : 0.0f;
    derr[w] = s >= 0 ? serr[s] : 0.0f;
    if (dscale) dscale[w] = s >= 0 ? sscale[s] : 1.0f;
  }
}

__global__ void norm_block_kernel(const float* __restrict__ norm, int64_t rows, int64_t rows_out,
                                  __nv_bfloat16* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows_out;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = i < rows ? -0.5f * norm[i] : 0.0f;  // exact: a power-of-two scale
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));  // v - h exact
    __nv_bfloat16* row = dst + i * NBLOCK_COLS;
    row[0] = h;
    row[1] = l;
#pragma unroll
    for (int j = 2; j < NBLOCK_COLS; ++j) row[j] = __float2bfloat16_rn(0.0f);
  }
}

template <typename T>
__global__ void fold_norm_kernel(T* __restrict__ lp, const float* __restrict__ norm, int64_t rows,
                                 int dpad, int col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = -0.5f * norm[i];  // exact: a power-of-two scale
    const T h = to_lp<T>(v);
    const T l = to_lp<T>(v - from_lp(h));  // v - h exact
    lp[i * dpad + col] = h;
    lp[i * dpad + col + 1] = l;
  }
}

__global__ void map_rows_kernel(const int* __restrict__ rows, const int* __restrict__ n_dev, int n,
                                const int* __restrict__ qorig, int* __restrict__ out) {
  int lim = n_dev ? *n_dev : n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += gridDim.x * blockDim.x)
    out[i] = qorig ? qorig[rows[i]] : rows[i];
}

// out[r] = max of v over list r's rows (block r; 0 for an empty list).
__global__ void list_max_kernel(const float* __restrict__ v, const int* __restrict__ offsets,
                                float* __restrict__ out) {
  __shared__ float part[8];
  float m = 0.0f;
  for (int i = offsets[blockIdx.x] + threadIdx.x; i < offsets[blockIdx.x + 1]; i += blockDim.x)
    m = fmaxf(m, v[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, part[w]);
    out[blockIdx.x] = m;
  }
}

// Y[i] = X[i] - R[r] for the rows i of list r (block r), FP32.
__global__ void offset_rows_kernel(const float* __restrict__ X, const float* __restrict__ R,
                                   const int* __restrict__ offsets, int d, float* __restrict__ Y) {
  const int r = blockIdx.x;
  const int64_t b = (int64_t)offsets[r] * d, e = (int64_t)offsets[r + 1] * d;
  const float* rr = R + (int64_t)r * d;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) Y[i] = X[i] - rr[(i - b) % d];
}

}  // namespace

int launch_map_rows(const int* rows, const int* n_dev, int n, const int* qorig, int* out,
                    cudaStream_t st) {
  if (n <= 0) return RBC_OK;
  map_rows_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(rows, n_dev, n,
                                                                                  qorig, out);
  RBC_LAUNCH_CHECK("map_rows_kernel");
  return RBC_OK;
}

// |x|^2 of FP32 rows (one warp per row, FP32 partial sums) and, when asked,
// the largest |x| rounded up, as float bits (for the expansion form's bound).
__global__ void row_norms_kernel(const float* __restrict__ X, int64_t rows, int d,
                                 float* __restrict__ norm, unsigned* __restrict__ max_bits) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float* x = X + r * d;
  float s = 0.f;
  for (int i = lane; i < d; i += 32) s = fmaf(x[i], x[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    norm[r] = s;
    // sqrt rounded up, and a margin for the sum's own rounding
    if (max_bits) atomicMax(max_bits, __float_as_uint(__fsqrt_ru(s) * (1.0f + 1e-6f)));
  }
}

int launch_row_norms(const float* X, int64_t rows, int d, float* norm, unsigned* max_bits,
                     cudaStream_t st) {
  if (rows <= 0) return RBC_OK;
  const int64_t threads = rows * 32;
  row_norms_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(X, rows, d, norm, max_bits);
  RBC_LAUNCH_CHECK("row_norms_kernel");
  return RBC_OK;
}

int launch_gather_rows(const float* src, const int64_t* idx64, const int* idx32, int64_t rows,
                       int d, float* dst, cudaStream_t st) {
  if (rows <= 0) return RBC_OK;
  int64_t threads = rows * 32;
  gather_rows_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(src, idx64, idx32, rows,
                                                                       d, dst);
  RBC_LAUNCH_CHECK("gather_rows_kernel");
  return RBC_OK;
}

int launch_list_max(const float* v, const int* offsets, int n_r, float* out, cudaStream_t st) {
  if (n_r <= 0) return RBC_OK;
  list_max_kernel<<<n_r, 256, 0, st>>>(v, offsets, out);
  RBC_LAUNCH_CHECK("list_max_kernel");
  return RBC_OK;
}

int launch_offset_rows(const float* X, const float* R, const int* offsets, int n_r, int d,
                       float* Y, cudaStream_t st) {
  if (n_r <= 0) return RBC_OK;
  offset_rows_kernel<<<n_r, 256, 0, st>>>(X, R, offsets, d, Y);
  RBC_LAUNCH_CHECK("offset_rows_kernel");
  return RBC_OK;
}

int launch_to_lowp(const float* src, int64_t rows, int d, int dpad, int storage, void* dst,
                   float* norm, float* err, unsigned* err_max_bits, unsigned* norm_max_bits,
                   cudaStream_t st, float* scale) {
  if (rows <= 0) return RBC_OK;
  int64_t threads = rows * 32;
  unsigned blocks = (unsigned)((threads + 255) / 256);
  if (storage == RBC_FP8E4M3) {
    if (!scale || dpad % 128) {
      set_error("to_lowp: FP8 rows need a scale array and dpad %% 128 == 0 (dpad=%d)", dpad);
      return RBC_ERR_ARG;
    }
    to_fp8_kernel<<<blocks, 256, 0, st>>>(src, rows, d, dpad, static_cast<uint8_t*>(dst), norm,
                                          err, scale, err_max_bits, norm_max_bits);
  } else if (storage == RBC_BF16)
    to_lowp_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(
        src, rows, d, dpad, reinterpret_cast<__nv_bfloat16*>(dst), norm, err, err_max_bits,
        norm_max_bits);
  else
    to_lowp_kernel<__half><<<blocks, 256, 0, st>>>(src, rows, d, dpad,
                                                   reinterpret_cast<__half*>(dst), norm, err,
                                                   err_max_bits, norm_max_bits);
  RBC_LAUNCH_CHECK("to_lowp_kernel");
  return RBC_OK;
}

int launch_scatter_result_rows(const int64_t* ids, const float* dist, const int* dst_rows,
                               int64_t rows, int k, int64_t* out_ids, float* out_dist,
                               cudaStream_t st) {
  if (rows <= 0) return RBC_OK;
  const int64_t total = rows * k;
  scatter_result_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      ids, dist, dst_rows, rows, k, out_ids, out_dist);
  RBC_LAUNCH_CHECK("scatter_result_rows_kernel");
  return RBC_OK;
}

int launch_gather_lp_rows(const void* src, const float* snorm, const float* serr, const int* idx,
                          int64_t rows, int row_bytes, void* dst, float* dnorm, float* derr,
                          cudaStream_t st, const float* sscale, float* dscale) {
  if (rows <= 0) return RBC_OK;
  gather_lp_rows_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(
      static_cast<const uint4*>(src), snorm, serr, idx, rows, row_bytes / 16,
      static_cast<uint4*>(dst), dnorm, derr, sscale, dscale);
  RBC_LAUNCH_CHECK("gather_lp_rows_kernel");
  return RBC_OK;
}

int launch_fold_norm(void* lp, const float* norm, int64_t rows, int dpad, int col, int storage,
                     cudaStream_t st) {
  if (rows <= 0) return RBC_OK;
  if (col < 0 || col + 2 > dpad || (storage != RBC_BF16 && storage != RBC_F16)) {
    set_error("fold_norm: column %d of %d, storage %d", col, dpad, storage);
    return RBC_ERR_ARG;
  }
  const unsigned blocks = (unsigned)std::min<int64_t>((rows + 255) / 256, 148 * 16);
  if (storage == RBC_BF16)
    fold_norm_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<__nv_bfloat16*>(lp), norm,
                                                             rows, dpad, col);
  else
    fold_norm_kernel<__half><<<blocks, 256, 0, st>>>(static_cast<__half*>(lp), norm, rows, dpad,
                                                     col);
  RBC_LAUNCH_CHECK("fold_norm_kernel");
  return RBC_OK;
}

int launch_norm_block(const float* norm, int64_t rows, int64_t rows_out, void* dst,
                      cudaStream_t st) {
  if (rows_out <= 0) return RBC_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((rows_out + 255) / 256, 148 * 16);
  norm_block_kernel<<<blocks, 256, 0, st>>>(norm, rows, rows_out,
                                            static_cast<__nv_bfloat16*>(dst));
  RBC_LAUNCH_CHECK("norm_block_kernel");
  return RBC_OK;
}

}  // namespace rbc
