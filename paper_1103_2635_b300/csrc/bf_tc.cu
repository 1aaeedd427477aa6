// Tensor-core brute-force tile kernel (sm_103a): BF(Q, X[segments]) for the
// l2 metric, fused with a per-query top-C (Section 3: the distance step is a
// matrix product, the comparison step a per-query reduction).
//
// For l2, rho(q, x)^2 = |q|^2 - 2 q.x + |x|^2; |q|^2 does not change the
// order for a fixed query, so the kernel ranks points by the score
//     s(q, x) = |x~|^2 - 2 q~.x~
// of the low-precision (bf16 / fp16) rows q~, x~.  The products q~.x~ come
// from tcgen05.mma (kind::f16, FP32 accumulation in tensor memory); the
// score and the selection run in the epilogue, so no distance matrix is ever
// written to global memory.  Candidates are re-ranked in FP32 and certified
// afterwards (select.cu).
//
// Structure (one CTA per SM, persistent over work items):
//   warp 0     TMA producer: the 128-row query tile once per item, database
//              tiles of BN rows into an S-stage ring (128-byte swizzle, K-major),
//              and each tile's row norms (+inf past the segment end, which
//              masks those columns without a per-element test).
//   warp 1     allocates 2*BN tensor-memory columns and issues the MMAs
//              (M = 128, N = BN, K = 16 per instruction) into a double-buffered
//              accumulator.
//   warps 2-9  epilogue: warp w reads tensor-memory lanes 32*(w%4) .. +31 (one
//              query row per thread) for half of the tile's columns, forms
//              the scores two at a time (fma.f32x2), takes a running minimum
//              over each 32-column chunk (three-input min) and only when that
//              minimum beats the row's current C-th best walks the chunk and
//              inserts into a sorted register list.
// Every wait on an mbarrier is bounded; on expiry the kernel raises
// DEV_ERR_TIMEOUT, stops issuing work, waits (bounded) for its own TMA copies
// and frees its tensor memory before returning.
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace rbc {

namespace {

using namespace tc;

constexpr int NUM_THREADS = 320;   // 10 warps
constexpr int EPI_WARP0 = 2;       // first epilogue warp

struct TcParams {
  TileWork w;
  TopOut out;
  const float* xnorm;  // [rows + pad] |x~|^2, readable up to row index rows + BN
  int64_t x_rows;
  int q_rows;
  uint32_t* dev_err;
  const float* xscale;  // FP8: [rows + pad] per-row scales, readable like xnorm
  const float* qscale;  // FP8: [q_rows] per-row scales of the queries
};

__device__ __forceinline__ void item_info(const TileWork& w, int item, int& q0, int& nq, int& sb,
                                          int& se, int& slot) {
  if (w.items) {
    const WorkItem it = w.items[item];
    q0 = it.q_row0;
    nq = it.nq;
    sb = it.seg_begin;
    se = it.seg_end;
    slot = it.slot;
  } else {
    int tile = item / w.dense_splits;
    int s = item - tile * w.dense_splits;
    q0 = tile * TQ;
    nq = min(TQ, (int)(w.m - (int64_t)q0));
    sb = s;
    se = s + 1;
    slot = item;
  }
}

// K blocks the item multiplies: all KB unless the work names fewer per tile
template <int KB>
__device__ __forceinline__ int item_kb(const TileWork& w, int item) {
  if (!w.tile_kb || !w.items) return KB;
  const int v = w.tile_kb[w.items[item].tile];
  return v < 1 ? 1 : (v > KB ? KB : v);
}

__device__ __forceinline__ Seg seg_at(const TileWork& w, int si) {
  if (w.segs) return w.segs[si];
  int64_t b = (int64_t)si * w.dense_chunk;
  int64_t e = min(w.n, b + w.dense_chunk);
  return Seg{(int32_t)b, (int32_t)e};
}

// Shared-memory layout.  Database tiles start at a row index rounded down to
// a multiple of 4 so that the tile's norms (BN floats) can be fetched with
// one 16-byte-aligned bulk copy; the columns before the segment start and
// past its end are masked to +inf in the epilogue.
// Each (row, half) keeps C candidates (C = 8, 16 or 32).

template <int C, int KB, int BN, int S, int NR, bool FP8>
struct TcSmem {
  static constexpr int NBUF = (512 / BN) < 4 ? (512 / BN) : 4;  // TMEM accumulator buffers
  static_assert(NBUF * BN >= 32 && (NBUF * BN & (NBUF * BN - 1)) == 0,
                "tcgen05.alloc takes a power of two columns (>= 32)");
  static constexpr int Q_BYTES = KB * BM * 128;  // query tile, KB K-blocks of 128 bytes
  static constexpr int X_STAGE = KB * BN * 128;  // one database tile
  static constexpr int NORM_STAGE = BN * 4;
  static constexpr int NEPI_WARPS = NUM_THREADS / 32 - EPI_WARP0;
  static constexpr int OFF_Q = 0;
  static constexpr int OFF_X = OFF_Q + Q_BYTES;
  static constexpr int OFF_NORM = OFF_X + S * X_STAGE;
  // FP8: the tile's per-row scales, a ring beside the norms
  static constexpr int OFF_SCALE = OFF_NORM + NR * NORM_STAGE;
  static constexpr int NEPI_THREADS = NEPI_WARPS * 32;
  // per epilogue thread: the columns of its C list entries, entry j at [j][thread]
  static constexpr int OFF_IDS = OFF_SCALE + (FP8 ? NR * NORM_STAGE : 0);
  // per epilogue thread: one spilled 32-column chunk
  static constexpr int OFF_SCR = OFF_IDS + C * NEPI_THREADS * 4;
  // per (half, query row): the root score of that half's heap
  static constexpr int OFF_ROOT = OFF_SCR + NEPI_WARPS * 32 * 32 * 4;
  static constexpr int OFF_BAR = OFF_ROOT + 2 * BM * 4;
  // barriers: full[S], empty[S], nfull[NR], nempty[NR], tfull[NBUF], tempty[NBUF], qfull, qempty
  static constexpr int NBAR = 2 * S + 2 * NR + 2 * NBUF + 2;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;  // tmem base, abort flag
  static constexpr int BYTES = OFF_MISC + 16;
  static constexpr int ALLOC = BYTES + 1024;  // slack for 1024-byte alignment
  static_assert(ALLOC <= 232448, "shared memory budget");
};

// 10 warps: one SM sub-partition hosts three of them, so its 16K-register
// slice caps a thread at 168 registers (enforced by the launch bound).
template <int C, int KB, int BN, int S, int NRING, bool FP8>
__global__ void __launch_bounds__(NUM_THREADS, 1)
bf_tc_kernel(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap xmap,
             TcParams p, uint32_t idesc) {
  using L = TcSmem<C, KB, BN, S, NRING, FP8>;
  constexpr int KBLOCK = FP8 ? 128 : 64;  // elements per 128-byte K block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* sQ = smem + L::OFF_Q;
  uint8_t* sX = smem + L::OFF_X;
  float* sNorm = reinterpret_cast<float*>(smem + L::OFF_NORM);
  float* sScale = reinterpret_cast<float*>(smem + L::OFF_SCALE);
  int* sIds = reinterpret_cast<int*>(smem + L::OFF_IDS);
  float* sScr = reinterpret_cast<float*>(smem + L::OFF_SCR);
  float* sRoot = reinterpret_cast<float*>(smem + L::OFF_ROOT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  constexpr int NR = NRING;
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* nfull = bars + 2 * S;
  uint64_t* nempty = bars + 2 * S + NR;
  constexpr int NBUF = L::NBUF;
  uint64_t* tfull = bars + 2 * S + 2 * NR;
  uint64_t* tempty = bars + 2 * S + 2 * NR + NBUF;
  uint64_t* qfull = bars + 2 * S + 2 * NR + 2 * NBUF;
  uint64_t* qempty = bars + 2 * S + 2 * NR + 2 * NBUF + 1;
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + L::OFF_MISC);
  volatile int* sAbort = reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  constexpr int NEPI = NUM_THREADS / 32 - EPI_WARP0;  // 8 epilogue warps

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < NR; ++r) {
      mbar_init(&nfull[r], 1);
      mbar_init(&nempty[r], NEPI);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], NEPI);
    }
    mbar_init(qfull, 1);
    mbar_init(qempty, 1);
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(sTmem)),
                 "r"(NBUF * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;

  const TileWork& w = p.w;
  const int n_items = w.num_items_dev ? *w.num_items_dev : w.num_items;
  // a contiguous range of items per CTA, so that consecutive items of one
  // query tile stay on one CTA and the epilogue can carry its lists across
  // them; work whose query tiles are single items may take them strided
  // instead (neighbouring items, often of similar size, spread over CTAs)
  const int ib = w.strided ? (int)blockIdx.x : (int)((int64_t)blockIdx.x * n_items / gridDim.x);
  const int ie = w.strided ? n_items : (int)((int64_t)(blockIdx.x + 1) * n_items / gridDim.x);
  const int istep = w.strided ? (int)gridDim.x : 1;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    uint32_t it = 0, qi = 0;
    bool ok = true;
    for (int item = ib; ok && item < ie; item += istep, ++qi) {
      int q0, nq, sb, se, slot;
      item_info(w, item, q0, nq, sb, se, slot);
      if (!__all_sync(0xffffffffu, mbar_wait(qempty, (qi & 1) ^ 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
      const int kbn = item_kb<KB>(w, item);
      if (lane == 0) {
        mbar_arrive_expect_tx(qfull, kbn * BM * 128);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb)
          if (kb < kbn) tma_load_2d(sQ + kb * BM * 128, &qmap, qfull, kb * KBLOCK, q0);
      }
      for (int si = sb; ok && si < se; ++si) {
        const Seg sg = seg_at(w, si);
        for (int x = sg.x_begin & ~3; x < sg.x_end; x += BN, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          const int r = it % NR;
          const uint32_t nph = (it / NR) & 1;
          bool got = mbar_wait(&empty[s], ph ^ 1, sAbort, p.dev_err) &&
                     mbar_wait(&nempty[r], nph ^ 1, sAbort, p.dev_err);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          if (lane == 0) {
            mbar_arrive_expect_tx(&full[s], kbn * BN * 128);
#pragma unroll
            for (int kb = 0; kb < KB; ++kb)
              if (kb < kbn)
                tma_load_2d(sX + s * L::X_STAGE + kb * BN * 128, &xmap, &full[s], kb * KBLOCK, x);
            mbar_arrive_expect_tx(&nfull[r], (FP8 ? 2 : 1) * L::NORM_STAGE);
            bulk_load(sNorm + r * BN, p.xnorm + x, L::NORM_STAGE, &nfull[r]);
            if (FP8) bulk_load(sScale + r * BN, p.xscale + x, L::NORM_STAGE, &nfull[r]);
          }
          __syncwarp();
        }
      }
    }
    // drain: every issued stage must have landed before the CTA exits
    if (lane == 0) {
      for (uint32_t j = (it > (uint32_t)S ? it - S : 0); j < it; ++j)
        mbar_wait(&full[j % S], (j / S) & 1, sAbort, p.dev_err);
      for (uint32_t j = (it > (uint32_t)NR ? it - NR : 0); j < it; ++j)
        mbar_wait(&nfull[j % NR], (j / NR) & 1, sAbort, p.dev_err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    uint32_t it = 0, qi = 0;
    bool ok = true;
    for (int item = ib; ok && item < ie; item += istep, ++qi) {
      int q0, nq, sb, se, slot;
      item_info(w, item, q0, nq, sb, se, slot);
      if (!__all_sync(0xffffffffu, mbar_wait(qfull, qi & 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
      const int kbn = item_kb<KB>(w, item);
      for (int si = sb; ok && si < se; ++si) {
        const Seg sg = seg_at(w, si);
        for (int x = sg.x_begin & ~3; x < sg.x_end; x += BN, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          const int buf = it % NBUF;
          const uint32_t aph = (it / NBUF) & 1;
          bool got = mbar_wait(&full[s], ph, sAbort, p.dev_err) &&
                     mbar_wait(&tempty[buf], aph ^ 1, sAbort, p.dev_err);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t d_tmem = tmem + buf * BN;
            const uint32_t qa = smem_u32(sQ);
            const uint32_t xb = smem_u32(sX + s * L::X_STAGE);
#pragma unroll
            for (int kb = 0; kb < KB; ++kb)
#pragma unroll
              for (int k16 = 0; k16 < 4; ++k16) {
                if (kb >= kbn) continue;
                // one K step = 32 bytes (16 bf16 / fp16 or 32 e4m3 elements)
                uint64_t ad = smem_desc_sw128(qa + kb * BM * 128 + k16 * 32);
                uint64_t bd = smem_desc_sw128(xb + kb * BN * 128 + k16 * 32);
                if (FP8)
                  mma_f8(d_tmem, ad, bd, idesc, (kb | k16) != 0);
                else
                  mma_f16(d_tmem, ad, bd, idesc, (kb | k16) != 0);
              }
            mma_commit(&empty[s]);
            mma_commit(&tfull[buf]);
          }
          __syncwarp();
        }
      }
      if (lane == 0) mma_commit(qempty);
      __syncwarp();
    }
  } else {
    // ---------------- epilogue ----------------
    // Lane l of warp w owns query row 32*(w%4) + l (its TMEM lane) for one
    // half of each tile's columns.  Each thread keeps the C best scores of its
    // row so far, unsorted, in registers (their columns in shared memory), and
    // tracks the largest of them: tau, the row's threshold.  A 32-column chunk
    // whose minimum is not below tau costs only the scores and the minimum.
    // Otherwise the thread spills the chunk to its scratch row, builds the bit
    // mask of the columns below tau and, for each, overwrites the current
    // largest entry and finds the new largest with a tree of three-input
    // maxima -- short dependency chains, no memory round trips per level.
    // The two halves of a row share their thresholds: whichever half has the
    // smaller maximum holds C candidates below it, so min(max_0, max_1) bounds
    // the row's C-th best and either half may drop anything at or above it.
    const int quarter = warp & 3;
    const int half = (warp - EPI_WARP0) / 4;
    const int row = quarter * 32 + lane;
    const int et = threadIdx.x - EPI_WARP0 * 32;  // epilogue thread index
    constexpr int NT = L::NEPI_THREADS;
    int* lid = sIds + et;  // column of list entry j at lid[j * NT]
    float* scr = sScr + et * 32;
    float* my_root = sRoot + half * BM + row;
    const float* other_root = sRoot + (1 - half) * BM + row;
    constexpr int HALF = BN / 2;
    uint32_t it = 0;
    bool ok = true;
    float ls[C];               // the row's best C scores so far (unsorted)
    int lpos = 0;              // position of the largest entry of ls
    float tau_own = INFINITY;  // = ls[lpos]
    float tau = INFINITY;      // effective threshold: min(own max, other half's max)
    for (int item = ib; ok && item < ie; item += istep) {
      int q0, nq, sb, se, slot;
      item_info(w, item, q0, nq, sb, se, slot);
      int pq0 = -1, pnq, psb, pse, pslot;
      if (item - istep >= ib) item_info(w, item - istep, pq0, pnq, psb, pse, pslot);
      int nq0 = -1, nnq, nsb, nse, nslot;
      if (item + istep < ie) item_info(w, item + istep, nq0, nnq, nsb, nse, nslot);
      // FP8: score = |x~|^2 - 2 s_q s_x (a.b); cq = -2 s_q for this row
      const float cq = FP8 ? (row < nq ? -2.0f * p.qscale[q0 + row] : 0.0f) : -2.0f;
      if (pq0 != q0) {  // first item of a run of the same query tile
#pragma unroll
        for (int j = 0; j < C; ++j) {
          ls[j] = INFINITY;
          lid[j * NT] = -1;
        }
        lpos = 0;
        tau = INFINITY;
        tau_own = INFINITY;
        *my_root = INFINITY;
        // both halves have reset their maxima before either reads the other's
        asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
      }
      for (int si = sb; ok && si < se; ++si) {
        const Seg sg = seg_at(w, si);
        for (int x = sg.x_begin & ~3; x < sg.x_end; x += BN, ++it) {
          const int r = it % NR;
          const uint32_t nph = (it / NR) & 1;
          const int buf = it % NBUF;
          const uint32_t aph = (it / NBUF) & 1;
          bool got = mbar_wait(&nfull[r], nph, sAbort, p.dev_err) &&
                     mbar_wait(&tfull[buf], aph, sAbort, p.dev_err);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          tc_fence_after();
          tau = fminf(tau, *other_root);
          const float* nrm = sNorm + r * BN + half * HALF;
          const int lo = sg.x_begin - x - half * HALF;  // first valid column of this half
          const int hi = sg.x_end - x - half * HALF;    // one past the last valid column
          const bool partial = lo > 0 || hi < HALF;
          const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + buf * BN + half * HALF;
#pragma unroll 1
          for (int c0 = 0; c0 < HALF; c0 += 32) {
            float u[32];
            tmem_load_cols<32>(tbase + c0, u);
            if (c0 + 32 == HALF) {
              // the whole half is in registers: hand the accumulator back
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&tempty[buf]);
            }
            const float4* n4 = reinterpret_cast<const float4*>(nrm + c0);
            if (FP8) {
              // per-column scale: cq * s_x is a power of two times cq, exact
              const float4* s4 =
                  reinterpret_cast<const float4*>(sScale + r * BN + half * HALF + c0);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 nn = n4[j], ss = s4[j];
                u[4 * j] = fmaf(cq * ss.x, u[4 * j], nn.x);
                u[4 * j + 1] = fmaf(cq * ss.y, u[4 * j + 1], nn.y);
                u[4 * j + 2] = fmaf(cq * ss.z, u[4 * j + 2], nn.z);
                u[4 * j + 3] = fmaf(cq * ss.w, u[4 * j + 3], nn.w);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float4 nn = n4[j];
                fma2(u[4 * j], u[4 * j + 1], u[4 * j], u[4 * j + 1], -2.0f, nn.x, nn.y);
                fma2(u[4 * j + 2], u[4 * j + 3], u[4 * j + 2], u[4 * j + 3], -2.0f, nn.z, nn.w);
              }
            }
            if (partial) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                int c = c0 + j;
                if (c < lo || c >= hi) u[j] = INFINITY;
              }
            }
            const float mn = min_of32(u);
            if (mn < tau) {
              // 16-byte slots rotated by lane so that 8 lanes hit 8 bank groups
#pragma unroll
              for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4*>(scr + ((((j >> 2) ^ lane) & 7) << 2)) =
                    make_float4(u[j], u[j + 1], u[j + 2], u[j + 3]);
              uint32_t mask = hit_mask32(u, tau);
              const int cb = x + half * HALF + c0;
              const float tau_in = tau_own;
              while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const float sv = scr[((((j >> 2) ^ lane) & 7) << 2) | (j & 3)];
                if (sv < tau) {
                  // overwrite the largest entry, then find the new largest
#pragma unroll
                  for (int t = 0; t < C; ++t)
                    if (t == lpos) ls[t] = sv;
                  lid[lpos * NT] = cb + j;
                  tau_own = max_of<C>(ls);
                  lpos = __ffs(eq_mask<C>(ls, tau_own)) - 1;
                  tau = fminf(tau, tau_own);
                }
              }
              if (tau_own < tau_in) *my_root = tau_own;
            }
            __syncwarp();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&nempty[r]);
        }
      }
      const bool carry = nq0 == q0;  // the next item continues this tile's lists
      if (p.out.slot_valid && threadIdx.x == EPI_WARP0 * 32) p.out.slot_valid[slot] = carry ? 0 : 1;
      if (ok && !carry && row < nq) {
        int64_t base = (((int64_t)slot * TQ + row) * 2 + half) * C;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          p.out.score[base + j] = ls[j];
          p.out.idx[base + j] = ls[j] == INFINITY ? -1 : lid[j * NT];
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NBUF * BN)
                 : "memory");
  }
}

// ---- host side ----
// cuTensorMapEncodeTiled is taken from the driver at run time, so the library
// loads on machines without a driver (argument checks, the host sampler).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

namespace tc {

int encode_map(CUtensorMap* map, const void* base, int64_t rows, int dpad, int storage,
               int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return RBC_ERR_CUDA;
  }
  // 128-byte K blocks: 64 16-bit or 128 FP8 elements
  const int eb = lp_elem_bytes(storage);
  cuuint64_t dims[2] = {(cuuint64_t)dpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)dpad * eb};
  cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType ty = storage == RBC_BF16   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : storage == RBC_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUresult r = enc(
      map, ty,
      2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): rows=%lld dpad=%d", (int)r, (long long)rows,
              dpad);
    return RBC_ERR_CUDA;
  }
  return RBC_OK;
}

int encode_nblock_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return RBC_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)NBLOCK_COLS, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)NBLOCK_COLS * 2};
  cuuint32_t box[2] = {(cuuint32_t)NBLOCK_COLS, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (norm block) failed (%d): rows=%lld", (int)r,
              (long long)rows);
    return RBC_ERR_CUDA;
  }
  return RBC_OK;
}

}  // namespace tc

namespace {

template <int C, int KB, int BN, int S, int NR, bool FP8 = false>
int launch_tc(const LpMatrix& Qm, const LpMatrix& Xm, const TileWork& w, const TopOut& out,
              int grid, cudaStream_t st, uint32_t* dev_err) {
  using L = TcSmem<C, KB, BN, S, NR, FP8>;
  CUtensorMap qmap, xmap;
  RBC_TRY_TC(encode_map(&qmap, Qm.data, Qm.rows, Qm.dpad, Qm.storage, BM));
  RBC_TRY_TC(encode_map(&xmap, Xm.data, Xm.rows, Xm.dpad, Xm.storage, BN));
  auto kern = bf_tc_kernel<C, KB, BN, S, NR, FP8>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC));
  TcParams p{w, out, Xm.norm, Xm.rows, (int)Qm.rows, dev_err, Xm.scale, Qm.scale};
  // kind::f16: format 1 = bf16, 0 = fp16; kind::f8f6f4: format 0 = E4M3
  uint32_t idesc = idesc_f16(Qm.storage == RBC_BF16 ? 1 : 0, BM, BN);
  kern<<<grid, NUM_THREADS, L::ALLOC, st>>>(qmap, xmap, p, idesc);
  ++t_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kern);
    set_error("bf_tc_kernel<C=%d,KB=%d,BN=%d,S=%d> launch failed: %s (regs %d, max threads "
              "%d, static smem %zu, local %zu, dynamic smem %d)",
              C, KB, BN, S, cudaGetErrorString(e), fa.numRegs, fa.maxThreadsPerBlock,
              fa.sharedSizeBytes, fa.localSizeBytes, L::ALLOC);
    return RBC_ERR_CUDA;
  }
  return RBC_OK;
}

}  // namespace

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

int launch_bf_tc_topc(const LpMatrix& Qm, const LpMatrix& Xm, int C, const TileWork& w,
                      const TopOut& out, int grid, cudaStream_t st, uint32_t* dev_err) {
  if (!tc_available()) {
    set_error("tensor-core BF kernel needs an sm_103 device");
    return RBC_ERR_UNSUPPORTED;
  }
  if (Qm.dpad != Xm.dpad || Qm.storage != Xm.storage) {
    set_error("tensor-core BF: operand layouts differ");
    return RBC_ERR_ARG;
  }
  if (Qm.storage == RBC_FP8E4M3) {
    if (!Qm.scale || !Xm.scale) {
      set_error("tensor-core BF: FP8 operands need per-row scales");
      return RBC_ERR_ARG;
    }
    const int kb = Qm.dpad / 128;
    if (C == 8 && kb == 1) return launch_tc<8, 1, 256, 3, 8, true>(Qm, Xm, w, out, grid, st, dev_err);
    if (C == 8 && kb == 2) return launch_tc<8, 2, 128, 3, 8, true>(Qm, Xm, w, out, grid, st, dev_err);
    if (C == 16 && kb == 1) return launch_tc<16, 1, 256, 3, 8, true>(Qm, Xm, w, out, grid, st, dev_err);
    if (C == 16 && kb == 2) return launch_tc<16, 2, 128, 3, 8, true>(Qm, Xm, w, out, grid, st, dev_err);
    if (C == 32 && kb == 1) return launch_tc<32, 1, 256, 3, 8, true>(Qm, Xm, w, out, grid, st, dev_err);
    if (C == 32 && kb == 2) return launch_tc<32, 2, 128, 2, 8, true>(Qm, Xm, w, out, grid, st, dev_err);
    set_error("tensor-core BF: FP8 list width %d / padded dimension %d unsupported", C, Qm.dpad);
    return RBC_ERR_UNSUPPORTED;
  }
  // bf16 / fp16: the norm folded into the MMA (bf_tc_top.cu)
  return launch_bf_tc_top(Qm, Xm, C, w, out, grid, st, dev_err);
}

}  // namespace rbc
