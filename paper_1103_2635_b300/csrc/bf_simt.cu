// FP32 CUDA-core brute-force tile kernel: BF(Q, X[segments]) fused with a
// per-query top-C (Section 3: the distance step has the structure of a
// matrix product, the comparison step is a per-query reduction).
//
// One CTA processes one work item: a tile of up to TQ = 128 query rows
// against the database rows of the item's segments, TX = 64 rows at a time.
// The query tile stays in shared memory (transposed, [d][TQ]); database rows
// are staged in 32-dimension chunks.  Each of the 256 threads accumulates an
// 8 x 4 block of distances in registers (difference form: (q - x)^2 for l2,
// |q - x| for l1), the 128 x 64 tile is written to shared memory, and two
// threads per query row merge it into their sorted register lists.  Nothing
// but the per-(query, thread) top-C lists reaches global memory.
//
// Modes: TOPC (the lists above) and STORE (write every distance to a dense
// [rows, ld] matrix; used for the representative distances of the exact
// search, Section 5.2, which must be kept).  EXP (l2 top-C only): the
// expansion |x|^2 - 2 q.x with precomputed FP32 norms instead of the
// difference form -- one FFMA per dimension instead of a subtraction and an
// FFMA; its rounding bound is absolute, (d + 4) 2^-23 (|q| + max |x|)^2, and
// the select step certifies with it (SelectArgs::exp32).
#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int TX = 64;        // database rows per inner tile
constexpr int DC = 32;        // dimensions per staged chunk
constexpr int NTHREADS = 256; // 16 x 16 threads, 8 x 4 outputs each
constexpr int QS = TQ + 4;    // padded row stride of the transposed query tile
constexpr int XS = TX + 1;    // padded row stride of the transposed database chunk
constexpr int DS = TX + 2;    // padded row stride of the distance tile

__device__ __forceinline__ void fetch_item(const TileWork& w, int item, int& q0, int& nq,
                                           int& sb, int& se, int& slot) {
  if (w.items) {
    const WorkItem it = w.items[item];
    q0 = it.q_row0;
    nq = it.nq;
    sb = it.seg_begin;
    se = it.seg_end;
    slot = it.slot;
  } else {
    // dense: item = tile * splits + split; split s covers rows
    // [s * chunk, min(n, (s + 1) * chunk)) through the implicit segment table
    int tile = item / w.dense_splits;
    int s = item - tile * w.dense_splits;
    q0 = tile * TQ;
    nq = min(TQ, (int)(w.m - (int64_t)q0));
    sb = s;
    se = s + 1;
    slot = item;
  }
}

__device__ __forceinline__ Seg get_seg(const TileWork& w, int si) {
  if (w.segs) return w.segs[si];
  int64_t b = (int64_t)si * w.dense_chunk;
  int64_t e = min(w.n, b + w.dense_chunk);
  return Seg{(int32_t)b, (int32_t)e};
}

template <int METRIC, int C, bool STORE, bool EXP = false>
__global__ void __launch_bounds__(NTHREADS, 2)
bf_simt_kernel(const float* __restrict__ Q, const float* __restrict__ X, int d, TileWork w,
               TopOut out, float* __restrict__ store, int64_t store_ld,
               const float* __restrict__ xnorm = nullptr) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int dq = (d + DC - 1) / DC * DC;  // query tile rows, padded to the chunk
  float* Qs = smem;                        // [dq][QS]
  float* Xs = Qs + dq * QS;                // [DC][XS]
  float* Ds = Xs + DC * XS;                // [TQ][DS]
  __shared__ float s_xn[TX];               // EXP: |x|^2 of the tile's rows

  const int t = threadIdx.x;
  const int tx = t & 15;
  const int ty = t >> 4;
  const int sel_row = t >> 1;
  const int sel_half = t & 1;

  int n_items = w.num_items_dev ? *w.num_items_dev : w.num_items;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    int q0, nq, sb, se, slot;
    fetch_item(w, item, q0, nq, sb, se, slot);

    __syncthreads();  // previous item's readers of Qs / Ds are done
    // ---- load the query tile, transposed and zero padded: Qs[c][r] ----
    for (int idx = t; idx < TQ * dq; idx += NTHREADS) {
      int c = idx % dq;
      int r = idx / dq;
      float v = 0.f;
      if (r < nq && c < d) v = Q[(int64_t)(q0 + r) * d + c];
      Qs[c * QS + r] = v;
    }

    TopList<C> top;
    if (!STORE) top.init();

    // STORE mode: running column of the output matrix (a dense split starts
    // at its first database row)
    int store_col = w.items ? 0 : (int)get_seg(w, sb).x_begin;
    for (int si = sb; si < se; ++si) {
      const Seg sg = get_seg(w, si);
      for (int x0 = sg.x_begin; x0 < sg.x_end; x0 += TX) {
        const int nx = min(TX, sg.x_end - x0);
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

        for (int c0 = 0; c0 < dq; c0 += DC) {
          __syncthreads();  // Xs free (and Qs complete on the first chunk)
          // stage X rows [x0, x0 + nx) x dims [c0, c0 + DC): Xs[c][r]
#pragma unroll
          for (int j = 0; j < (TX * DC) / NTHREADS; ++j) {
            int idx = t + j * NTHREADS;
            int c = idx & (DC - 1);
            int r = idx / DC;
            float v = 0.f;
            if (r < nx && c0 + c < d) v = X[(int64_t)(x0 + r) * d + c0 + c];
            Xs[c * XS + r] = v;
          }
          __syncthreads();
#pragma unroll 8
          for (int c = 0; c < DC; ++c) {
            const float4 qa = *reinterpret_cast<const float4*>(&Qs[(c0 + c) * QS + ty * 8]);
            const float4 qb = *reinterpret_cast<const float4*>(&Qs[(c0 + c) * QS + ty * 8 + 4]);
            const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
            float xv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) xv[b] = Xs[c * XS + tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                if (EXP) {
                  acc[a][b] = fmaf(qv[a], xv[b], acc[a][b]);
                } else {
                  float diff = qv[a] - xv[b];
                  if (METRIC == RBC_L2)
                    acc[a][b] = fmaf(diff, diff, acc[a][b]);
                  else
                    acc[a][b] += fabsf(diff);
                }
              }
          }
        }
        // ---- distance tile -> shared memory (columns interleaved for the
        // two selecting threads of a row) ----
        if (EXP && t < TX) s_xn[t] = t < nx ? xnorm[x0 + t] : 0.f;
        if (EXP) __syncthreads();
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int col = tx * 4 + b;
            const float v = EXP ? fmaf(-2.0f, acc[a][b], s_xn[col]) : acc[a][b];
            Ds[(ty * 8 + a) * DS + col] = (col < nx) ? v : INFINITY;
          }
        __syncthreads();
        if (STORE) {
          // write rows of the tile to the dense output (coalesced along columns)
          for (int idx = t; idx < TQ * TX; idx += NTHREADS) {
            int r = idx / TX;
            int c = idx % TX;
            if (r < nq && c < nx) {
              float v = Ds[r * DS + c];
              if (METRIC == RBC_L2) v = sqrtf(v);
              store[(int64_t)(q0 + r) * store_ld + store_col + c] = v;
            }
          }
        } else if (sel_row < nq) {
#pragma unroll 4
          for (int j = 0; j < TX / 2; ++j) {
            int col = 2 * j + sel_half;
            float v = Ds[sel_row * DS + col];
            if (v < top.worst() || v == top.worst()) {
              int id = x0 + col;
              if (top.admits(v, id)) top.insert(v, id);
            }
          }
        }
        store_col += nx;
      }
    }
    if (!STORE && sel_row < nq) {
      // partial slot layout: [slot][TQ][NSUB = 2][C]
      int64_t base = (((int64_t)slot * TQ + sel_row) * 2 + sel_half) * C;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        out.score[base + j] = top.s[j];
        out.idx[base + j] = top.s[j] == INFINITY ? -1 : top.i[j];
      }
    }
  }
}

template <int METRIC, int C, bool STORE, bool EXP = false>
int launch_one(const float* Q, const float* X, int d, const TileWork& w, const TopOut& out,
               float* store, int64_t store_ld, int grid, cudaStream_t st,
               const float* xnorm = nullptr) {
  const int dq = (d + DC - 1) / DC * DC;
  size_t smem = sizeof(float) * ((size_t)dq * QS + DC * XS + TQ * DS);
  auto kern = bf_simt_kernel<METRIC, C, STORE, EXP>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, NTHREADS, smem, st>>>(Q, X, d, w, out, store, store_ld, xnorm);
  RBC_LAUNCH_CHECK("bf_simt_kernel");
  return RBC_OK;
}

template <int METRIC>
int dispatch_c(int C, const float* Q, const float* X, int d, const TileWork& w, const TopOut& out,
               int grid, cudaStream_t st) {
  switch (C) {
    case 2: return launch_one<METRIC, 2, false>(Q, X, d, w, out, nullptr, 0, grid, st);
    case 4: return launch_one<METRIC, 4, false>(Q, X, d, w, out, nullptr, 0, grid, st);
    case 8: return launch_one<METRIC, 8, false>(Q, X, d, w, out, nullptr, 0, grid, st);
    case 16: return launch_one<METRIC, 16, false>(Q, X, d, w, out, nullptr, 0, grid, st);
    case 32: return launch_one<METRIC, 32, false>(Q, X, d, w, out, nullptr, 0, grid, st);
    default: set_error("bf_simt: unsupported list width %d", C); return RBC_ERR_UNSUPPORTED;
  }
}

// Windowed stage two on CUDA cores (FP32 storage or the l1 metric): the same
// work items as the tensor-core emission kernel -- a chunk of up to TQ
// queries that kept representative r, against a window [x_begin, x_end) of
// r's sorted list (Section 5.2 with sorted lists; the window bound holds for
// any metric by the triangle inequality).  The chunk's query rows are
// gathered into shared memory (transposed), the window streams through in
// tiles of TX rows, each thread accumulates an 8 x 4 block of FP32
// difference-form distances (squared for l2), and every (query, row) whose
// value is at most the query's threshold thr[q] is appended to q's candidate
// buffer (one atomic per hit; cand_cnt counts every emission, so a count
// above cap marks an overflow).
template <int METRIC>
__global__ void __launch_bounds__(NTHREADS, 2)
bf_simt_emit_kernel(const float* __restrict__ Q, const float* __restrict__ X, int d,
                    const EmitItem* __restrict__ items, const int* __restrict__ num_items_dev,
                    int max_items, const int* __restrict__ pair_q, int pair_stride, EmitOut out) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int dq = (d + DC - 1) / DC * DC;
  float* Qs = smem;             // [dq][QS]
  float* Xs = Qs + dq * QS;     // [DC][XS]
  __shared__ int s_q[TQ];       // query of each chunk row (-1: none)
  __shared__ float s_thr[TQ];   // its threshold
  const int t = threadIdx.x;
  const int tx = t & 15;
  const int ty = t >> 4;
  int n_items = num_items_dev ? *num_items_dev : max_items;
  if (n_items > max_items) n_items = max_items;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const EmitItem e = items[item];
    if (e.x_end <= e.x_begin) continue;  // the same for the whole CTA
    __syncthreads();  // the previous item's readers of Qs / s_q are done
    if (t < TQ) {
      const int q = t < e.nq ? pair_q[(int64_t)(e.pair_begin + t) * pair_stride] : -1;
      s_q[t] = q;
      s_thr[t] = q >= 0 ? out.thr[q] : -INFINITY;
    }
    __syncthreads();
    // the chunk's query rows, transposed and zero padded: Qs[c][r]
    for (int idx = t; idx < TQ * dq; idx += NTHREADS) {
      const int c = idx % dq;
      const int r = idx / dq;
      const int q = s_q[r];
      Qs[c * QS + r] = (q >= 0 && c < d) ? Q[(int64_t)q * d + c] : 0.f;
    }
    for (int x0 = e.x_begin; x0 < e.x_end; x0 += TX) {
      const int nx = min(TX, e.x_end - x0);
      float acc[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int c0 = 0; c0 < dq; c0 += DC) {
        __syncthreads();  // Xs free (and Qs complete on the first chunk)
#pragma unroll
        for (int j = 0; j < (TX * DC) / NTHREADS; ++j) {
          const int idx = t + j * NTHREADS;
          const int c = idx & (DC - 1);
          const int r = idx / DC;
          Xs[c * XS + r] = (r < nx && c0 + c < d) ? X[(int64_t)(x0 + r) * d + c0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < DC; ++c) {
          const float4 qa = *reinterpret_cast<const float4*>(&Qs[(c0 + c) * QS + ty * 8]);
          const float4 qb = *reinterpret_cast<const float4*>(&Qs[(c0 + c) * QS + ty * 8 + 4]);
          const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
          float xv[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) xv[b] = Xs[c * XS + tx * 4 + b];
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float diff = qv[a] - xv[b];
              if (METRIC == RBC_L2)
                acc[a][b] = fmaf(diff, diff, acc[a][b]);
              else
                acc[a][b] += fabsf(diff);
            }
        }
      }
      // emission: every value at or under its row's threshold
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int row = ty * 8 + a;
        const float th = s_thr[row];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int col = tx * 4 + b;
          if (col < nx && acc[a][b] <= th) {
            const int q = s_q[row];
            const int pos = atomicAdd(&out.cand_cnt[q], 1);
            if (pos < out.cap) {
              out.cand_score[(int64_t)q * out.cap + pos] = acc[a][b];
              out.cand_row[(int64_t)q * out.cap + pos] = x0 + col;
            }
          }
        }
      }
    }
  }
}

}  // namespace

int simt_list_width(int c_needed) {
  for (int c : {2, 4, 8, 16, 32})
    if (c >= c_needed) return c;
  return -1;
}

int launch_bf_simt_topc(const float* Q, const float* X, int d, int metric, int C,
                        const TileWork& w, const TopOut& out, int grid, cudaStream_t st) {
  if (d > SIMT_MAX_D) {
    set_error("bf_simt: d = %d exceeds %d", d, SIMT_MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  if (metric == RBC_L2) return dispatch_c<RBC_L2>(C, Q, X, d, w, out, grid, st);
  return dispatch_c<RBC_L1>(C, Q, X, d, w, out, grid, st);
}

int launch_bf_simt_topc_exp(const float* Q, const float* X, const float* xnorm, int d, int C,
                            const TileWork& w, const TopOut& out, int grid, cudaStream_t st) {
  if (d > SIMT_MAX_D) {
    set_error("bf_simt: d = %d exceeds %d", d, SIMT_MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  switch (C) {
    case 2: return launch_one<RBC_L2, 2, false, true>(Q, X, d, w, out, nullptr, 0, grid, st, xnorm);
    case 4: return launch_one<RBC_L2, 4, false, true>(Q, X, d, w, out, nullptr, 0, grid, st, xnorm);
    case 8: return launch_one<RBC_L2, 8, false, true>(Q, X, d, w, out, nullptr, 0, grid, st, xnorm);
    case 16: return launch_one<RBC_L2, 16, false, true>(Q, X, d, w, out, nullptr, 0, grid, st, xnorm);
    case 32: return launch_one<RBC_L2, 32, false, true>(Q, X, d, w, out, nullptr, 0, grid, st, xnorm);
    default: set_error("bf_simt: unsupported list width %d", C); return RBC_ERR_UNSUPPORTED;
  }
}

int launch_bf_simt_emit(const float* Q, const float* X, int d, int metric, const EmitItem* items,
                        const int* num_items_dev, int max_items, const int* pair_q,
                        int pair_stride, const EmitOut& out, int grid, cudaStream_t st) {
  if (d > SIMT_MAX_D) {
    set_error("bf_simt: d = %d exceeds %d", d, SIMT_MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  if (max_items <= 0 || grid <= 0) return RBC_OK;
  const int dq = (d + DC - 1) / DC * DC;
  const size_t smem = sizeof(float) * ((size_t)dq * QS + DC * XS);
  if (metric == RBC_L2) {
    auto kern = bf_simt_emit_kernel<RBC_L2>;
    RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, NTHREADS, smem, st>>>(Q, X, d, items, num_items_dev, max_items, pair_q,
                                       pair_stride, out);
  } else {
    auto kern = bf_simt_emit_kernel<RBC_L1>;
    RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, NTHREADS, smem, st>>>(Q, X, d, items, num_items_dev, max_items, pair_q,
                                       pair_stride, out);
  }
  RBC_LAUNCH_CHECK("bf_simt_emit_kernel");
  return RBC_OK;
}

int launch_bf_simt_store(const float* Q, const float* X, int d, int metric, const TileWork& w,
                         float* store, int64_t store_ld, int grid, cudaStream_t st) {
  if (d > SIMT_MAX_D) {
    set_error("bf_simt: d = %d exceeds %d", d, SIMT_MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  TopOut none{nullptr, nullptr};
  if (metric == RBC_L2)
    return launch_one<RBC_L2, 2, true>(Q, X, d, w, none, store, store_ld, grid, st);
  return launch_one<RBC_L1, 2, true>(Q, X, d, w, none, store, store_ld, grid, st);
}

}  // namespace rbc
