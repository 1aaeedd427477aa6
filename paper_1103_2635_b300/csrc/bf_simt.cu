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
// EXP (l2 only): the expansion |x|^2 - 2 q.x with precomputed FP32 norms
// instead of the difference form -- one FFMA per dimension instead of a
// subtraction and an FFMA; its rounding bound is absolute,
// (d + 4) 2^-23 (|q| + max |x|)^2, and the select step certifies with it
// (SelectArgs::exp32).
//
// This 8 x 4 kernel serves 32-wide lists and rows too long for the 8 x 8
// top-C kernel further down, which takes lists of up to 16.  The same file
// holds the windowed emission kernel on CUDA cores and the distance-matrix
// kernel of stage one (every distance kept), described where they are
// defined.
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

// Two terms of a distance sum, columns x0 and x1 against one query value q:
// EXP a += q x; l2 a += (q - x)^2; l1 a += |q - x|.  EXP and l2 use the
// packed two-lane FP32 instructions (fma / sub .f32x2: one issue slot for
// two terms, the same rounding as the scalar ones).
template <int METRIC, bool EXP>
__device__ __forceinline__ void two_terms(float& a0, float& a1, float x0, float x1, float q) {
  if (EXP) {
    asm("{\n\t.reg .b64 ac, xx, qq;\n\t"
        "mov.b64 ac, {%0, %1};\n\tmov.b64 xx, {%2, %3};\n\tmov.b64 qq, {%4, %4};\n\t"
        "fma.rn.f32x2 ac, xx, qq, ac;\n\tmov.b64 {%0, %1}, ac;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(x0), "f"(x1), "f"(q));
  } else if (METRIC == RBC_L2) {
    asm("{\n\t.reg .b64 ac, xx, qq, df;\n\t"
        "mov.b64 ac, {%0, %1};\n\tmov.b64 xx, {%2, %3};\n\tmov.b64 qq, {%4, %4};\n\t"
        "sub.rn.f32x2 df, qq, xx;\n\tfma.rn.f32x2 ac, df, df, ac;\n\t"
        "mov.b64 {%0, %1}, ac;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(x0), "f"(x1), "f"(q));
  } else {
    a0 += fabsf(q - x0);
    a1 += fabsf(q - x1);
  }
}

template <int METRIC, int C, bool EXP = false>
__global__ void __launch_bounds__(NTHREADS, 2)
bf_simt_kernel(const float* __restrict__ Q, const float* __restrict__ X, int d, TileWork w,
               TopOut out, const float* __restrict__ xnorm = nullptr) {
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
    top.init();
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
              for (int b = 0; b < 4; b += 2)
                two_terms<METRIC, EXP>(acc[a][b], acc[a][b + 1], xv[b], xv[b + 1], qv[a]);
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
        if (sel_row < nq) {
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
      }
    }
    if (sel_row < nq) {
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

template <int METRIC, int C, bool EXP = false>
int launch_one(const float* Q, const float* X, int d, const TileWork& w, const TopOut& out,
               int grid, cudaStream_t st, const float* xnorm = nullptr) {
  const int dq = (d + DC - 1) / DC * DC;
  size_t smem = sizeof(float) * ((size_t)dq * QS + DC * XS + TQ * DS);
  auto kern = bf_simt_kernel<METRIC, C, EXP>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, NTHREADS, smem, st>>>(Q, X, d, w, out, xnorm);
  RBC_LAUNCH_CHECK("bf_simt_kernel");
  return RBC_OK;
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
              // scalar here: the packed form measured 7% slower in this kernel
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

// 8 x 8 register-tiled kernels: the distance matrix of stage one (STORE,
// every distance kept) and the top-C pass.  A CTA computes 128 x 128 tiles:
// the query tile stays in shared memory (transposed, [d][TQ]), the database
// rows pass through in 16-dimension chunks, staged from registers that were
// loaded while the previous chunk was being used.  Each thread accumulates an
// 8 x 8 block (rows 4 ty + {0..3} and 64 + 4 ty + {0..3}, the same for columns
// with tx, so every shared-memory read is one 16-byte load per four values
// and the two query loads are broadcasts): the difference form, or (EXP) the
// product q.x for the expansion |x|^2 - 2 q.x.
constexpr int S_TX = 128;          // database rows per tile
constexpr int S_DC = 16;           // dimensions per staged chunk
constexpr int S_QS = TQ + 4;       // row stride of the transposed query tile
constexpr int S_XS = S_TX + 4;     // row stride of the transposed database chunk

// One work item: load the query tile, then every 128-row tile of the item's
// segments; on_tile(x0, nx, acc) runs after each tile's last chunk (all
// threads, acc complete; x0 the tile's first database row, nx its rows).
template <int METRIC, bool EXP, typename TileFn>
__device__ __forceinline__ void simt8_item(const float* __restrict__ Q,
                                           const float* __restrict__ X, int d, int dq,
                                           const TileWork& w, int q0, int nq, int sb, int se,
                                           float* Qs, float* Xs, TileFn&& on_tile) {
  const float4* Q4 = reinterpret_cast<const float4*>(Qs);
  const float4* X4 = reinterpret_cast<const float4*>(Xs);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int sc = t & (S_DC - 1);  // staging: dimension of this thread's values
  const int sr = t >> 4;          // staging: first row (then + 16 j)
  float xr[8];                    // the next chunk, in flight
  auto fetch = [&](int fx0, int fnx, int fc0) {
    const bool cin = fc0 + sc < d;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = sr + 16 * j;
      xr[j] = (cin && r < fnx) ? X[(int64_t)(fx0 + r) * d + fc0 + sc] : 0.f;
    }
  };
  // first non-empty segment
  int si = sb, x0 = 0, xe = 0;
  for (; si < se; ++si) {
    const Seg sg = get_seg(w, si);
    if (sg.x_end > sg.x_begin) {
      x0 = sg.x_begin;
      xe = sg.x_end;
      break;
    }
  }
  if (si < se) fetch(x0, min(S_TX, xe - x0), 0);
  __syncthreads();  // the previous item's readers of Qs are done
  for (int idx = t; idx < TQ * dq; idx += NTHREADS) {
    const int c = idx % dq;
    const int r = idx / dq;
    Qs[c * S_QS + r] = (r < nq && c < d) ? Q[(int64_t)(q0 + r) * d + c] : 0.f;
  }
  int c0 = 0;
  float acc[8][8];
  while (si < se) {
    const int nx = min(S_TX, xe - x0);
    // the chunk after this one
    int nsi = si, nx0 = x0, nxe = xe, nc0 = c0 + S_DC;
    if (nc0 >= dq) {
      nc0 = 0;
      nx0 = x0 + S_TX;
      if (nx0 >= xe) {
        for (++nsi; nsi < se; ++nsi) {
          const Seg sg = get_seg(w, nsi);
          if (sg.x_end > sg.x_begin) {
            nx0 = sg.x_begin;
            nxe = sg.x_end;
            break;
          }
        }
      }
    }
    __syncthreads();  // the previous chunk's readers of Xs are done
#pragma unroll
    for (int j = 0; j < 8; ++j) Xs[sc * S_XS + sr + 16 * j] = xr[j];
    __syncthreads();  // the chunk (and, first, the query tile) is in place
    if (nsi < se) fetch(nx0, min(S_TX, nxe - nx0), nc0);
    if (c0 == 0) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    }
#pragma unroll 4
    for (int k = 0; k < S_DC; ++k) {
      const float4 qa = Q4[(c0 + k) * (S_QS / 4) + ty];
      const float4 qb = Q4[(c0 + k) * (S_QS / 4) + 16 + ty];
      const float4 xa = X4[k * (S_XS / 4) + tx];
      const float4 xb = X4[k * (S_XS / 4) + 16 + tx];
      const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
      const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; b += 2)
          two_terms<METRIC, EXP>(acc[a][b], acc[a][b + 1], xv[b], xv[b + 1], qv[a]);
    }
    if (c0 + S_DC >= dq) on_tile(x0, nx, acc);
    si = nsi;
    x0 = nx0;
    xe = nxe;
    c0 = nc0;
  }
}

// STORE: the tile's distances, straight from registers (16-byte stores of
// four consecutive columns) to store[q][col], col running over the item's
// segments (a dense split starts at its first row).
template <int METRIC>
__global__ void __launch_bounds__(NTHREADS, 2)
bf_simt_store_kernel(const float* __restrict__ Q, const float* __restrict__ X, int d, TileWork w,
                     float* __restrict__ store, int64_t store_ld) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int dq = (d + S_DC - 1) / S_DC * S_DC;
  float* Qs = smem;            // [dq][S_QS]
  float* Xs = Qs + dq * S_QS;  // [S_DC][S_XS]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int n_items = w.num_items_dev ? *w.num_items_dev : w.num_items;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    int q0, nq, sb, se, slot;
    fetch_item(w, item, q0, nq, sb, se, slot);
    int store_col = w.items ? 0 : (int)get_seg(w, sb).x_begin;
    simt8_item<METRIC, false>(Q, X, d, dq, w, q0, nq, sb, se, Qs, Xs,
                              [&](int x0, int nx, float (&acc)[8][8]) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int row = 4 * ty + (a & 3) + (a >> 2) * 64;
        if (row >= nq) continue;
        float* orow = store + (int64_t)(q0 + row) * store_ld + store_col;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = 4 * tx + 64 * h;
          float v[4];
#pragma unroll
          for (int b = 0; b < 4; ++b)
            v[b] = METRIC == RBC_L2 ? sqrtf(acc[a][4 * h + b]) : acc[a][4 * h + b];
          if (col + 4 <= nx && (reinterpret_cast<uintptr_t>(orow + col) & 15) == 0) {
            *reinterpret_cast<float4*>(orow + col) = make_float4(v[0], v[1], v[2], v[3]);
          } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (col + b < nx) orow[col + b] = v[b];
          }
        }
      }
      store_col += nx;
    });
  }
}

// TOPC: per (query row, column parity) a list of the C best (score, id), in
// shared memory and unsorted, owned by one thread (row t / 2, parity t % 2):
// a new entry overwrites the largest, whose position the owner finds from
// the largest entry of each group of four (2-bit positions packed in one
// register); the largest entry -- the list's threshold -- is published in
// shared memory.  A
// tile goes through a half-width distance buffer in two 64-column halves:
// the threads that computed the values compare them with the thresholds and
// flag the (row, parity) lists that one of them may enter; only a flagged
// owner walks its 32 columns of the half and inserts the ones that beat its
// list.  Scores: the difference form, or (EXP) |x|^2 - 2 q.x with xnorm =
// |x|^2.  The lists go to out in the layout [slot][TQ][2][C] at the item's
// end.
constexpr int T_DH = 66;  // row stride of the half-tile buffer (owner reads conflict-free)

template <int METRIC, int C, bool EXP>
__global__ void __launch_bounds__(NTHREADS, 2)
bf_simt_top8_kernel(const float* __restrict__ Q, const float* __restrict__ X, int d, TileWork w,
                    TopOut out, const float* __restrict__ xnorm) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int dq = (d + S_DC - 1) / S_DC * S_DC;
  float* Qs = smem;                 // [dq][S_QS]
  float* Xs = Qs + dq * S_QS;       // [S_DC][S_XS]
  float* Ds = Xs + S_DC * S_XS;     // [TQ][T_DH]
  float* Ls = Ds + TQ * T_DH;       // [C][NTHREADS] list scores
  int* Li = reinterpret_cast<int*>(Ls + C * NTHREADS);  // [C][NTHREADS] list ids
  __shared__ float s_thr[NTHREADS];  // threshold of list t (row t / 2, parity t % 2)
  __shared__ int s_flag[NTHREADS];   // list t may take a value of this half
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int orow = t >> 1, osub = t & 1;
  float* ls = Ls + t;
  int* li = Li + t;
  int n_items = w.num_items_dev ? *w.num_items_dev : w.num_items;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    int q0, nq, sb, se, slot;
    fetch_item(w, item, q0, nq, sb, se, slot);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      ls[j * NTHREADS] = INFINITY;
      li[j * NTHREADS] = INT32_MAX;
    }
    float wv = INFINITY;  // the list's largest entry (score, id) ...
    int wi = INT32_MAX;
    int lpos = 0;         // ... at this position
    uint32_t gp = 0;      // 2 bits per group of four: its largest entry's position
    // (v, id) replaces the largest entry; the group's and the list's largest
    // are found again
    auto insert = [&](float v, int id) {
      ls[lpos * NTHREADS] = v;
      li[lpos * NTHREADS] = id;
      if (C < 4) {  // two entries: the larger is the other one or the new one
        const float ov = ls[(1 - lpos) * NTHREADS];
        const int oi = li[(1 - lpos) * NTHREADS];
        if (pair_lt(v, id, ov, oi)) {
          wv = ov;
          wi = oi;
          lpos = 1 - lpos;
        } else {
          wv = v;
          wi = id;
        }
        return;
      }
      const int g = lpos >> 2;
      float bv = ls[(4 * g) * NTHREADS];
      int bi = li[(4 * g) * NTHREADS], bp = 0;
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        const float cv = ls[(4 * g + u) * NTHREADS];
        const int ci = li[(4 * g + u) * NTHREADS];
        if (pair_lt(bv, bi, cv, ci)) {
          bv = cv;
          bi = ci;
          bp = u;
        }
      }
      gp = (gp & ~(3u << (2 * g))) | ((uint32_t)bp << (2 * g));
      int P = gp & 3;
      float M = ls[P * NTHREADS];
      int I = li[P * NTHREADS];
#pragma unroll
      for (int u = 1; u < C / 4; ++u) {
        const int pu = 4 * u + ((gp >> (2 * u)) & 3);
        const float cv = ls[pu * NTHREADS];
        const int ci = li[pu * NTHREADS];
        if (pair_lt(M, I, cv, ci)) {
          M = cv;
          I = ci;
          P = pu;
        }
      }
      wv = M;
      wi = I;
      lpos = P;
    };
    s_thr[t] = INFINITY;  // read by the producers after the item's first barrier
    s_flag[t] = 0;
    simt8_item<METRIC, EXP>(Q, X, d, dq, w, q0, nq, sb, se, Qs, Xs,
                            [&](int x0, int nx, float (&acc)[8][8]) {
      float xn[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int col = 4 * tx + (b & 3) + (b >> 2) * 64;
        xn[b] = (EXP && col < nx) ? xnorm[x0 + col] : 0.f;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        __syncthreads();  // the previous half's owners are done with Ds
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int row = 4 * ty + (a & 3) + (a >> 2) * 64;
          float v[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const float s = EXP ? fmaf(-2.0f, acc[a][4 * h + b], xn[4 * h + b]) : acc[a][4 * h + b];
            v[b] = (64 * h + 4 * tx + b < nx) ? s : INFINITY;
          }
          float2* dp = reinterpret_cast<float2*>(Ds + row * T_DH + 4 * tx);
          dp[0] = make_float2(v[0], v[1]);
          dp[1] = make_float2(v[2], v[3]);
          // columns 4 tx + b have parity b % 2
          const float t0 = s_thr[2 * row], t1 = s_thr[2 * row + 1];
          if (v[0] <= t0 || v[2] <= t0) s_flag[2 * row] = 1;
          if (v[1] <= t1 || v[3] <= t1) s_flag[2 * row + 1] = 1;
        }
        __syncthreads();
        if (orow < nq && s_flag[t]) {
          s_flag[t] = 0;
          const float* drow = Ds + orow * T_DH + osub;
#pragma unroll 4
          for (int j = 0; j < 32; ++j) {
            const float v = drow[2 * j];
            if (v <= wv) {
              const int id = x0 + 64 * h + 2 * j + osub;
              if (pair_lt(v, id, wv, wi)) insert(v, id);
            }
          }
          s_thr[t] = wv;
        }
      }
    });
    if (orow < nq) {
      // partial slot layout: [slot][TQ][NSUB = 2][C]
      const int64_t base = (((int64_t)slot * TQ + orow) * 2 + osub) * C;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const float v = ls[j * NTHREADS];
        out.score[base + j] = v;
        out.idx[base + j] = v == INFINITY ? -1 : li[j * NTHREADS];
      }
    }
  }
}

template <int METRIC>
int launch_store(const float* Q, const float* X, int d, const TileWork& w, float* store,
                 int64_t store_ld, int grid, cudaStream_t st) {
  const int dq = (d + S_DC - 1) / S_DC * S_DC;
  const size_t smem = sizeof(float) * ((size_t)dq * S_QS + S_DC * S_XS);
  auto kern = bf_simt_store_kernel<METRIC>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, NTHREADS, smem, st>>>(Q, X, d, w, store, store_ld);
  RBC_LAUNCH_CHECK("bf_simt_store_kernel");
  return RBC_OK;
}

size_t top8_smem(int d, int C) {
  const int dq = (d + S_DC - 1) / S_DC * S_DC;
  return sizeof(float) * ((size_t)dq * S_QS + S_DC * S_XS + TQ * T_DH) + (size_t)C * NTHREADS * 8;
}

template <int METRIC, int C, bool EXP>
int launch_top8(const float* Q, const float* X, int d, const TileWork& w, const TopOut& out,
                int grid, cudaStream_t st, const float* xnorm) {
  const size_t smem = top8_smem(d, C);
  auto kern = bf_simt_top8_kernel<METRIC, C, EXP>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, NTHREADS, smem, st>>>(Q, X, d, w, out, xnorm);
  RBC_LAUNCH_CHECK("bf_simt_top8_kernel");
  return RBC_OK;
}

// the 8 x 8 kernel for lists of up to 16 (two CTAs per SM at d = 64); the
// 8 x 4 kernel for 32-wide lists (its lists live in registers, so it keeps
// two CTAs per SM: measured 22.2 against 18.4 TFLOP/s at k = 31, d = 64) and
// wherever the 8 x 8 kernel's shared memory would not fit one CTA (227 KB)
template <int METRIC, bool EXP>
int dispatch_top8(int C, const float* Q, const float* X, int d, const TileWork& w,
                  const TopOut& out, int grid, cudaStream_t st, const float* xnorm) {
  if (C > 16 || top8_smem(d, C) > 227 * 1024) {
    switch (C) {
      case 2: return launch_one<METRIC, 2, EXP>(Q, X, d, w, out, grid, st, xnorm);
      case 4: return launch_one<METRIC, 4, EXP>(Q, X, d, w, out, grid, st, xnorm);
      case 8: return launch_one<METRIC, 8, EXP>(Q, X, d, w, out, grid, st, xnorm);
      case 16: return launch_one<METRIC, 16, EXP>(Q, X, d, w, out, grid, st, xnorm);
      case 32: return launch_one<METRIC, 32, EXP>(Q, X, d, w, out, grid, st, xnorm);
      default: set_error("bf_simt: unsupported list width %d", C); return RBC_ERR_UNSUPPORTED;
    }
  }
  switch (C) {
    case 2: return launch_top8<METRIC, 2, EXP>(Q, X, d, w, out, grid, st, xnorm);
    case 4: return launch_top8<METRIC, 4, EXP>(Q, X, d, w, out, grid, st, xnorm);
    case 8: return launch_top8<METRIC, 8, EXP>(Q, X, d, w, out, grid, st, xnorm);
    case 16: return launch_top8<METRIC, 16, EXP>(Q, X, d, w, out, grid, st, xnorm);
    default: set_error("bf_simt: unsupported list width %d", C); return RBC_ERR_UNSUPPORTED;
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
  if (metric == RBC_L2) return dispatch_top8<RBC_L2, false>(C, Q, X, d, w, out, grid, st, nullptr);
  return dispatch_top8<RBC_L1, false>(C, Q, X, d, w, out, grid, st, nullptr);
}

int launch_bf_simt_topc_exp(const float* Q, const float* X, const float* xnorm, int d, int C,
                            const TileWork& w, const TopOut& out, int grid, cudaStream_t st) {
  if (d > SIMT_MAX_D) {
    set_error("bf_simt: d = %d exceeds %d", d, SIMT_MAX_D);
    return RBC_ERR_UNSUPPORTED;
  }
  return dispatch_top8<RBC_L2, true>(C, Q, X, d, w, out, grid, st, xnorm);
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
  if (metric == RBC_L2) return launch_store<RBC_L2>(Q, X, d, w, store, store_ld, grid, st);
  return launch_store<RBC_L1>(Q, X, d, w, store, store_ld, grid, st);
}

}  // namespace rbc
