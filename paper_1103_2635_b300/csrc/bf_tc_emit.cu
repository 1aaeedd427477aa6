// Tensor-core windowed BF with candidate emission (sm_103a), the stage two of
// the windowed exact search (Section 5.2 with sorted lists).
//
// A work item is (a chunk of up to 128 queries that all kept representative
// r, a window [x_begin, x_end) of r's sorted list).  The queries of a chunk
// are arbitrary rows of the query matrix, so they are gathered, not tiled:
// two warps copy them with 16-byte cp.async (eight lanes per row, so every
// instruction reads whole rows) into the 128-byte-swizzled K-major layout the
// MMA reads, several query stages ahead of the MMA.  A query stage also
// carries its item's window, so the MMA and epilogue warps never read the
// item list.  Database windows are contiguous rows and come by TMA as in the
// top-C kernel.
//
// Every query q carries a score threshold T(q) (window.cu): no point whose
// score |x~|^2 - 2 q~.x~ exceeds T(q) can be within g(q) of q, the bound of
// its k-th neighbour distance.  The norm term is folded into the MMA: next to
// each database tile the stage holds the tile's norm block (-|x~|^2 / 2 as a
// bf16 high and low part, 16 columns), and one extra bf16 MMA of an all-ones
// A operand against it adds -|x~|^2 / 2 to every accumulator, which then
// holds q~.x~ - |x~|^2 / 2 = -s / 2.  So the epilogue keeps no lists, loads
// no norms and does no arithmetic per score: per 32-column chunk the TMEM load
// itself returns the maximum of the raw accumulators (tcgen05.ld.red), and
// only when that reaches -T(q) / 2 does a lane walk the chunk and emit the
// qualifying (score, row) pairs: into its own slice of a hit arena (no
// atomics; a post-pass moves them to the per-query buffers; a chunk's hits
// that the slice has no room for go to the query's buffer directly, one
// atomic per chunk), or, in the
// instance for direct appends, into q's candidate buffer with one atomic per
// chunk.  When rows have two spare padding columns, the norm pair lives in
// them instead (FOLD) and no norm block or norm MMA is needed.  The
// candidates are re-ranked exactly afterwards (select.cu).
//
//   warp 0      TMA producer: database tiles of BN rows + their norm blocks
//   warp 1      tensor-memory allocation, MMA issue (M = 128, N = BN, K = 16)
//   warps 2-3   query gather (cp.async), per-row query id and threshold,
//               the item's window; the two warps take alternate items and
//               fetch their next item's ids while the copies are in flight
//   warps 4-    epilogue: TMEM lane quarter (warp % 4) x column slice; with
//               no candidate lists to keep, the warps can hold whole slices
//               (256-row tiles at d <= 64: 8 warps of 128 columns, four
//               32-column loads in flight per warp; otherwise up to 16)
// Every mbarrier wait is bounded (2 s); on expiry the kernel raises
// DEV_ERR_TIMEOUT, stops issuing work, drains its copies and frees TMEM.
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace rbc {

namespace {

using namespace tc;

constexpr int E_GATHER = 2;     // first query-gather warp
constexpr int E_NGATHER = 2;    // query-gather warps (alternate items)
constexpr int E_EPI0 = 4;       // first epilogue warp

// Epilogue parts: the tile's columns are split into NPART slices of BN/NPART
// (at least 32) columns; each (TMEM lane quarter, slice) is one warp.  256-row
// tiles of one K block (d <= 64): two slices of four chunks (eight warps;
// fewer per-tile waits and hand-offs than sixteen warps of two chunks, 2%
// faster at d = 64, 1.5% slower at d = 96, where the MMAs take longer).
template <int KB, int BN>
struct EpiShape {
  static constexpr int NPART = (BN == 256 && KB == 1) ? 2 : (BN / 32 < 4 ? BN / 32 : 4);
  static constexpr int NEPI = 4 * NPART;             // epilogue warps
  static constexpr int THREADS = 32 * (E_EPI0 + NEPI);
  static constexpr int COLS = BN / NPART;            // columns per thread per tile
  static constexpr int CHUNKS = COLS / 32;           // 32-column TMEM loads per tile
};

struct EmitParams {
  const EmitItem* items;
  const int* num_items_dev;
  int max_items;
  const int* pair_q;
  int pair_stride;      // the query of pair i is pair_q[i * pair_stride]
  const uint8_t* qlp;  // [q_rows, dpad] 16-bit rows
  int64_t q_row_bytes;
  const float* xnorm;  // [rows + pad]
  EmitOut out;
  uint32_t* dev_err;
  int fold_col;         // FOLD: the row element holding the norm pair (even)
  uint32_t fold_ones;   // FOLD: the pair (1, 1) in the storage type
  EmitOffsets off;      // OFFS: per-pair rows a~ = bf16(q - r), bounds, |a~|^2
};

template <int KB, int BN, int S, int QSTAGES>
struct EmitSmem {
  static constexpr int NBUF = (512 / BN) < 4 ? (512 / BN) : 4;  // TMEM accumulator buffers
  static_assert(NBUF * BN >= 32 && (NBUF * BN & (NBUF * BN - 1)) == 0,
                "tcgen05.alloc takes a power of two columns (>= 32)");
  static constexpr int Q_BYTES = KB * BM * 128;
  static constexpr int X_STAGE = KB * BN * 128;
  static constexpr int NB_STAGE = BN * NBLOCK_COLS * 2;          // a tile's norm block
  static constexpr int ONES_BYTES = BM * NBLOCK_COLS * 2;        // the all-ones A block
  static constexpr int OFF_Q = 0;
  static constexpr int OFF_X = OFF_Q + QSTAGES * Q_BYTES;
  static constexpr int OFF_NB = OFF_X + S * X_STAGE;
  static constexpr int OFF_ONES = OFF_NB + S * NB_STAGE;
  static constexpr int OFF_ROWQ = OFF_ONES + ONES_BYTES;        // [QSTAGES][BM] query id or -1
  static constexpr int OFF_ROWT = OFF_ROWQ + QSTAGES * BM * 4;  // [QSTAGES][BM] -T / 2
  static constexpr int OFF_ROWN = OFF_ROWT + QSTAGES * BM * 4;  // [QSTAGES][BM] OFFS: |a~|^2
  static constexpr int OFF_XWIN = OFF_ROWN + QSTAGES * BM * 4;  // [QSTAGES] item window
  static constexpr int OFF_BAR = OFF_XWIN + QSTAGES * 8;
  // full[S], empty[S], tfull[NBUF], tempty[NBUF], qfull[QS], qempty[QS]
  static constexpr int NBAR = 2 * S + 2 * NBUF + 2 * QSTAGES;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;  // tmem base, abort flag, hit count
  static constexpr int BYTES = OFF_MISC + 16;
  static constexpr int ALLOC = BYTES + 1024;  // slack for 1024-byte alignment
  static_assert(ALLOC <= 232448, "shared memory budget");
  static_assert(OFF_X % 1024 == 0 && X_STAGE % 1024 == 0, "swizzled tiles need 1024-byte alignment");
  static_assert(OFF_NB % 1024 == 0 && NB_STAGE % 1024 == 0 && OFF_ONES % 1024 == 0,
                "norm blocks need 1024-byte alignment");
  static_assert(QSTAGES % 2 == 0, "query stages alternate between two gather warps");
};

// Shared-memory descriptor of a K-major operand with 32-byte rows (16 bf16)
// and 32-byte swizzle: 8-row groups 256 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(256 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)6 << 61;                   // 32-byte swizzle
  return d;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src))
               : "memory");
}
__device__ __forceinline__ void st_shared_zero16(uint32_t dst) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0) : "memory");
}

// QSTAGES query stages (even: the two gather warps alternate over them): the
// gather of an item's rows takes a few microseconds, longer than a one-tile
// item, so several are kept in flight.
// FOLD: the database rows hold -|x~|^2 / 2 as a (high, low) pair in two of
// their zero padding columns (fold_col, fold_col + 1), and the gather sets
// those columns of every query row to 1: the data MMAs then add the norm
// themselves, and neither the norm block nor its MMA is needed.
// DIRECT: hits go straight to the per-query buffers (no hit arena); each
// instance holds only its own emission path.
// OFFS: representative offsets -- an item's query rows are the rows
// a~ = bf16(q - r) of its pairs (pair_begin + i), formed beforehand with
// their emission bounds (accumulator units) and |a~|^2; a hit's value is
// |a~|^2 - 2 acc, the estimate of |a~ - y~|^2.
template <int KB, int BN, int S, int QSTAGES, bool FOLD = false, bool DIRECT = false,
          bool OFFS = false>
__global__ void __launch_bounds__(EpiShape<KB, BN>::THREADS, 1)
bf_tc_emit_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap nbmap,
                  EmitParams p, uint32_t idesc, uint32_t idesc_norm) {
  using L = EmitSmem<KB, BN, S, QSTAGES>;
  using E = EpiShape<KB, BN>;
  constexpr int E_NEPI = E::NEPI;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* sQ = smem + L::OFF_Q;
  uint8_t* sX = smem + L::OFF_X;
  uint8_t* sNB = smem + L::OFF_NB;
  uint32_t* sOnes = reinterpret_cast<uint32_t*>(smem + L::OFF_ONES);
  int* sRowQ = reinterpret_cast<int*>(smem + L::OFF_ROWQ);
  float* sRowT = reinterpret_cast<float*>(smem + L::OFF_ROWT);
  float* sRowN = reinterpret_cast<float*>(smem + L::OFF_ROWN);
  int2* sXwin = reinterpret_cast<int2*>(smem + L::OFF_XWIN);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  constexpr int NBUF = L::NBUF;
  uint64_t* full = bars;
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + NBUF;
  uint64_t* qfull = tempty + NBUF;
  uint64_t* qempty = qfull + QSTAGES;
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + L::OFF_MISC);
  volatile int* sAbort = reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4);
  int* sHits = reinterpret_cast<int*>(smem + L::OFF_MISC + 8);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], E_NEPI);
    }
    for (int q = 0; q < QSTAGES; ++q) {
      mbar_init(&qfull[q], 32);              // every gather lane
      mbar_init(&qempty[q], 1 + E_NEPI);     // MMA commit + every epilogue warp
    }
    *sAbort = 0;
    *sHits = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  // the all-ones A block of the norm MMA (bf16 1.0 pairs; every layout of an
  // all-ones block reads the same)
  for (int i = threadIdx.x; i < L::ONES_BYTES / 4; i += blockDim.x) sOnes[i] = 0x3F803F80u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

  int n_items = p.num_items_dev ? *p.num_items_dev : p.max_items;
  if (n_items > p.max_items) n_items = p.max_items;

  if (warp == 0) {
    // ---------------- TMA producer (database windows) ----------------
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
      const EmitItem e = p.items[item];
      if (e.x_end <= e.x_begin) continue;
      for (int x = e.x_begin & ~3; x < e.x_end; x += BN, ++it) {
        const int s = it % S;
        const uint32_t ph = (it / S) & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1, sAbort, p.dev_err))) {
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[s], L::X_STAGE + (FOLD ? 0 : L::NB_STAGE));
#pragma unroll
          for (int kb = 0; kb < KB; ++kb)
            tma_load_2d(sX + s * L::X_STAGE + kb * BN * 128, &xmap, &full[s], kb * 64, x);
          if (!FOLD) tma_load_2d(sNB + s * L::NB_STAGE, &nbmap, &full[s], 0, x);
        }
        __syncwarp();
      }
    }
    if (lane == 0) {
      for (uint32_t j = (it > (uint32_t)S ? it - S : 0); j < it; ++j)
        mbar_wait(&full[j % S], (j / S) & 1, sAbort, p.dev_err);
    }
  } else if (warp >= E_GATHER && warp < E_GATHER + E_NGATHER) {
    // ---------------- query gather (warp gw takes items qi = gw mod 2) ----------------
    const uint32_t gw = warp - E_GATHER;
    // the first item at or after `it` that is this warp's: empty items are
    // skipped, q counts the non-empty ones before it
    auto seek = [&](int& it, uint32_t& q, EmitItem& ee) -> bool {
      for (; it < n_items; it += gridDim.x) {
        ee = p.items[it];
        if (ee.x_end <= ee.x_begin) continue;
        if (q % E_NGATHER == gw) return true;
        ++q;
      }
      return false;
    };
    // an item's query ids and thresholds (row lane + 32 t); OFFS: the rows'
    // bounds in accumulator units and |a~|^2, per pair
    int srcs[BM / 32];
    float thrs[BM / 32];
    float nrms[OFFS ? BM / 32 : 1];
    auto meta = [&](const EmitItem& ee) {
#pragma unroll
      for (int t = 0; t < BM / 32; ++t) {
        const int row = lane + 32 * t;
        srcs[t] = row < ee.nq ? p.pair_q[(int64_t)(ee.pair_begin + row) * p.pair_stride] : -1;
      }
      if constexpr (OFFS) {
#pragma unroll
        for (int t = 0; t < BM / 32; ++t) {
          const int64_t i = ee.pair_begin + lane + 32 * t;
          thrs[t] = srcs[t] >= 0 ? p.off.row_t[i] : INFINITY;
          nrms[t] = srcs[t] >= 0 ? p.off.row_n[i] : 0.0f;
        }
      } else {
#pragma unroll
        for (int t = 0; t < BM / 32; ++t) thrs[t] = srcs[t] >= 0 ? p.out.thr[srcs[t]] : 0.0f;
      }
    };
    int item = blockIdx.x;
    uint32_t qi = 0;
    EmitItem e;
    bool have = seek(item, qi, e);
    bool ok = true;
    if (have) meta(e);
    while (have) {
      const int qs = qi % QSTAGES;
      const uint32_t qph = (qi / QSTAGES) & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&qempty[qs], qph ^ 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
      const uint32_t qbase = smem_u32(sQ + qs * L::Q_BYTES);
#pragma unroll
      for (int t = 0; t < BM / 32; ++t) {
        const int row = lane + 32 * t;
        sRowQ[qs * BM + row] = srcs[t];
        if (OFFS) {
          sRowT[qs * BM + row] = thrs[t];
          sRowN[qs * BM + row] = nrms[t];
        } else {
          sRowT[qs * BM + row] = srcs[t] < 0 ? INFINITY : -0.5f * thrs[t];
        }
      }
      // the copies: eight consecutive lanes move the eight 16-byte chunks of
      // one 128-byte K block of a row, so one instruction reads four whole
      // rows (row 4i + lane / 8, whose id lane (4i + lane / 8) mod 32 holds)
      const int c = lane & 7;
#pragma unroll
      for (int i = 0; i < BM / 4; ++i) {
        const int row = 4 * i + (lane >> 3);
        const int src = __shfl_sync(0xffffffffu, srcs[i >> 3], (4 * i + (lane >> 3)) & 31);
        // OFFS: the row of the item's pair (query rows are per pair)
        const int64_t srow = OFFS ? (int64_t)e.pair_begin + row : (int64_t)src;
        const uint8_t* g = (OFFS ? p.off.a_rows : p.qlp) + (src >= 0 ? srow : 0) * p.q_row_bytes + c * 16;
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const uint32_t dst = qbase + kb * BM * 128 + row * 128 + ((c ^ (row & 7)) << 4);
          if (src >= 0)
            cp_async16(dst, g + kb * 128);
          else
            st_shared_zero16(dst);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (lane == 0) sXwin[qs] = make_int2(e.x_begin, e.x_end);
      // the next item's descriptor, query ids and thresholds are fetched
      // while the copies are in flight
      int item2 = item + gridDim.x;
      uint32_t qi2 = qi + 1;
      EmitItem e2;
      const bool have2 = seek(item2, qi2, e2);
      if (have2) meta(e2);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      if (FOLD) {
        // every lane's copies have landed (wait + warp barrier); then the
        // ones of the folded norm pair go into this lane's rows
        __syncwarp();
        const int kbf = p.fold_col >> 6, within = (p.fold_col & 63) * 2;
#pragma unroll
        for (int t = 0; t < BM / 32; ++t) {
          const int row = lane + 32 * t;
          const uint32_t a = qbase + kbf * BM * 128 + row * 128 +
                             ((((within >> 4) ^ (row & 7)) << 4) | (within & 15));
          asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(p.fold_ones) : "memory");
        }
      }
      // this lane's rows are in shared memory: make them visible to the
      // tensor core (async proxy), then release the stage
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&qfull[qs]);
      item = item2;
      e = e2;
      qi = qi2;
      have = have2;
    }
    // stage qi (the number of non-empty items) carries the end mark, an
    // empty window; the gather warp whose turn it is writes it
    if (ok && qi % E_NGATHER == gw) {
      const int qs = qi % QSTAGES;
      if (__all_sync(0xffffffffu, mbar_wait(&qempty[qs], ((qi / QSTAGES) & 1) ^ 1, sAbort, p.dev_err))) {
        if (lane == 0) sXwin[qs] = make_int2(0, 0);
        mbar_arrive(&qfull[qs]);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // items in query-stage order; each stage carries its window (an empty
    // window marks the end)
    uint32_t it = 0;
    bool ok = true;
    for (uint32_t qi = 0; ok; ++qi) {
      const int qs = qi % QSTAGES;
      const uint32_t qph = (qi / QSTAGES) & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&qfull[qs], qph, sAbort, p.dev_err))) break;
      const int2 xw = sXwin[qs];
      if (xw.y <= xw.x) break;
      for (int x = xw.x & ~3; x < xw.y; x += BN, ++it) {
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
          const uint32_t qa = smem_u32(sQ + qs * L::Q_BYTES);
          const uint32_t xb = smem_u32(sX + s * L::X_STAGE);
#pragma unroll
          for (int kb = 0; kb < KB; ++kb)
#pragma unroll
            for (int k16 = 0; k16 < 4; ++k16) {
              uint64_t ad = smem_desc_sw128(qa + kb * BM * 128 + k16 * 32);
              uint64_t bd = smem_desc_sw128(xb + kb * BN * 128 + k16 * 32);
              mma_f16(d_tmem, ad, bd, idesc, (kb | k16) != 0);
            }
          // + (-|x~|^2 / 2) in every row: ones x norm block (bf16, K = 16)
          if (!FOLD)
            mma_f16(d_tmem, smem_desc_sw32(smem_u32(sOnes)),
                    smem_desc_sw32(smem_u32(sNB + s * L::NB_STAGE)), idesc_norm, 1u);
          mma_commit(&empty[s]);
          mma_commit(&tfull[buf]);
        }
        __syncwarp();
      }
      if (lane == 0) mma_commit(&qempty[qs]);
      __syncwarp();
    }
  } else if (warp >= E_EPI0) {
    // ---------------- epilogue ----------------
    // Warp w reads TMEM lane quarter w % 4 (its query rows) and column slice
    // (w - E_EPI0) / 4 of each tile: all of its CHUNKS loads are issued before
    // one wait, then the accumulator is handed back and the scores formed.
    const int quarter = warp & 3;
    const int part = (warp - E_EPI0) >> 2;
    const int row = quarter * 32 + lane;
    constexpr int COLS = E::COLS;
    constexpr int CH = E::CHUNKS;
    uint32_t it = 0, qi = 0;
    bool ok = true;
    const int cap = p.out.cap;
    // hit arena: this thread's private slice (segment of its warp, split by
    // lane) and its own fill count: no atomics, no cross-lane traffic
    const int esub = p.out.arena_seg / ARENA_SUBSEG;
    const int lsub = esub / 32;
    const int ew = warp - E_EPI0;
    int4* hits = p.out.arena ? p.out.arena + (int64_t)blockIdx.x * p.out.arena_seg +
                                   (int64_t)ew * esub + (int64_t)lane * lsub
                             : nullptr;
    int nhits = 0;         // records in this thread's arena slice
    bool spilled = false;  // some chunk's hits went to the buffers directly
    for (; ok; ++qi) {
      const int qs = qi % QSTAGES;
      const uint32_t qph = (qi / QSTAGES) & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&qfull[qs], qph, sAbort, p.dev_err))) break;
      const int2 xw = sXwin[qs];
      const int myq = sRowQ[qs * BM + row];
      const float myT = sRowT[qs * BM + row];  // -T(q) / 2: emit where the accumulator reaches it
      const float myN = OFFS ? sRowN[qs * BM + row] : 0.0f;  // OFFS: |a~|^2 of the row
      __syncwarp();
      if (lane == 0) mbar_arrive(&qempty[qs]);
      if (xw.y <= xw.x) break;  // the end mark
      float* cs = p.out.cand_score + (int64_t)(myq >= 0 ? myq : 0) * cap;
      int* cr = p.out.cand_row + (int64_t)(myq >= 0 ? myq : 0) * cap;
      int* cc = p.out.cand_cnt + (myq >= 0 ? myq : 0);
      for (int x = xw.x & ~3; x < xw.y; x += BN, ++it) {
        const int buf = it % NBUF;
        const uint32_t aph = (it / NBUF) & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&tfull[buf], aph, sAbort, p.dev_err))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + buf * BN + part * COLS;
        uint32_t raw[CH][32];
        float cmax[CH];  // per chunk: the largest accumulator, from the load itself
#pragma unroll
        for (int c = 0; c < CH; ++c) tmem_ld_x32_max(tbase + c * 32, raw[c], cmax[c]);
        tmem_wait_ld();
        // every column of this slice is in registers: hand the accumulator back
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        // the common case: no row of the warp reaches its threshold anywhere
        // in the slice -- one vote instead of a test and a branch per chunk
        float cm = cmax[0];
#pragma unroll
        for (int c = 1; c < CH; ++c) cm = fmaxf(cm, cmax[c]);
        if (!__any_sync(0xffffffffu, cm >= myT)) continue;
        const int lo = xw.x - x - part * COLS;  // first valid column of the slice
        const int hi = xw.y - x - part * COLS;    // one past the last valid column
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          if (!(c * 32 < hi && c * 32 + 32 > lo)) continue;  // no window column in the chunk
          // The maximum runs over all 32 columns, including any outside the
          // window (real rows, or zero rows past the matrix end): a false
          // alarm only costs the slow path, where the in-window mask decides.
          const bool hit = cmax[c] >= myT;
          if (hit) {  // the rare path: this row has columns at or over its threshold
            const int cb = x + part * COLS + c * 32;
            const int clo = lo - c * 32, chi = hi - c * 32;
            const uint32_t below_hi = chi >= 32 ? 0xffffffffu : (chi <= 0 ? 0u : (1u << chi) - 1u);
            const uint32_t below_lo = clo >= 32 ? 0xffffffffu : (clo <= 0 ? 0u : (1u << clo) - 1u);
            const uint32_t valid = below_hi & ~below_lo;
            // the set bits of the hit mask, one by one (compact code: the
            // common path stays small in the instruction cache)
            uint32_t mask = valid & over_mask32<true>(raw[c], myT);
            if (!DIRECT && nhits + __popc(mask) <= lsub) {
              while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const float v = __uint_as_float(pick32(raw[c], j));
                hits[nhits++] = make_int4(myq, cb + j, __float_as_int(fmaf(-2.0f, v, myN)), 0);
              }
            } else {
              // direct appends (and, in the arena instance, the hits of a
              // chunk that its slice has no room for): one atomic per (lane,
              // chunk) reserves the row's slots, then the hits fill them in
              // column order
              if (!DIRECT) spilled = true;
              int pos = atomicAdd(cc, __popc(mask));
              while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const float v = __uint_as_float(pick32(raw[c], j));
                if (pos < cap) {
                  cs[pos] = fmaf(-2.0f, v, myN);
                  cr[pos] = cb + j;
                }
                ++pos;
              }
            }
          }
        }
      }
    }
    if (!DIRECT) {
      p.out.arena_cnt[(blockIdx.x * ARENA_SUBSEG + ew) * 32 + lane] = nhits;
      if (spilled) atomicOr(p.out.arena_ovf, 1);
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

template <int KB, int BN, int S, int QS, bool FOLD, bool DIRECT, bool OFFS = false>
int launch_emit(const LpMatrix& Qm, const LpMatrix& Xm, const EmitItem* items,
                const int* num_items_dev, int max_items, const int* pair_q, int pair_stride,
                const EmitOut& out, int grid, cudaStream_t st, uint32_t* dev_err, int fold_col,
                const EmitOffsets* offs = nullptr) {
  using L = EmitSmem<KB, BN, S, QS>;
  CUtensorMap xmap, nbmap;
  RBC_TRY_TC(encode_map(&xmap, Xm.data, Xm.rows, Xm.dpad, Xm.storage, BN));
  if (FOLD)
    memset(&nbmap, 0, sizeof(nbmap));  // not read: the norm is in the rows
  else
    RBC_TRY_TC(encode_nblock_map(&nbmap, Xm.nblock, Xm.rows, BN));
  auto kern = bf_tc_emit_kernel<KB, BN, S, QS, FOLD, DIRECT, OFFS>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC));
  EmitParams p{items,  num_items_dev, max_items, pair_q, pair_stride,
               static_cast<const uint8_t*>(Qm.data), (int64_t)Qm.dpad * 2, Xm.norm, out, dev_err,
               fold_col, Qm.storage == RBC_BF16 ? 0x3F803F80u : 0x3C003C00u,
               offs ? *offs : EmitOffsets{}};
  const uint32_t idesc = idesc_f16(Qm.storage == RBC_BF16 ? 1 : 0, BM, BN);
  const uint32_t idesc_norm = idesc_f16(1, BM, BN);  // the norm block is bf16 for any storage
  kern<<<grid, EpiShape<KB, BN>::THREADS, L::ALLOC, st>>>(xmap, nbmap, p, idesc, idesc_norm);
  ++t_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kern);
    set_error("bf_tc_emit_kernel<KB=%d,BN=%d,S=%d,QS=%d> launch failed: %s (regs %d, local %zu, "
              "dynamic smem %d)",
              KB, BN, S, QS, cudaGetErrorString(e), fa.numRegs, fa.localSizeBytes, L::ALLOC);
    return RBC_ERR_CUDA;
  }
  return RBC_OK;
}

}  // namespace

int launch_bf_tc_emit(const LpMatrix& Qm, const LpMatrix& Xm, const EmitItem* items,
                      const int* num_items_dev, int max_items, const int* pair_q,
                      int pair_stride, const EmitOut& out, int grid, cudaStream_t st,
                      uint32_t* dev_err, int fold_col, const EmitOffsets* offs) {
  if (!tc_available()) {
    set_error("tensor-core BF kernel needs an sm_103 device");
    return RBC_ERR_UNSUPPORTED;
  }
  if (Qm.dpad != Xm.dpad || Qm.storage != Xm.storage) {
    set_error("tensor-core BF: operand layouts differ");
    return RBC_ERR_ARG;
  }
  if (max_items <= 0) return RBC_OK;
  if (!Xm.nblock && fold_col < 0) {
    set_error("tensor-core emission: the database has no norm block");
    return RBC_ERR_ARG;
  }
  if (fold_col >= 0 && (fold_col & 1 || fold_col + 2 > Qm.dpad)) {
    set_error("tensor-core emission: folded norm column %d invalid", fold_col);
    return RBC_ERR_ARG;
  }
  if (offs && (Xm.storage != RBC_BF16 || !offs->a_rows || !offs->row_t || !offs->row_n ||
               out.arena == nullptr || (reinterpret_cast<uintptr_t>(offs->a_rows) & 15))) {
    set_error("tensor-core emission: offset rows need bf16, the per-pair rows and bounds, and "
              "the hit arena");
    return RBC_ERR_ARG;
  }
  // d <= 128: 256-row database tiles (the fewest MMA instructions per
  // column); longer rows: 64-row tiles
#define RBC_EMIT_ONE(KB, BN, S, QS, FOLD, DIRECT)                                         \
  launch_emit<KB, BN, S, QS, FOLD, DIRECT>(Qm, Xm, items, num_items_dev, max_items, pair_q,   \
                                           pair_stride, out, grid, st, dev_err, fold_col)
#define RBC_EMIT_OFFS(KB, BN, S, QS, FOLD)                                                \
  launch_emit<KB, BN, S, QS, FOLD, false, true>(Qm, Xm, items, num_items_dev, max_items, pair_q, \
                                               pair_stride, out, grid, st, dev_err, fold_col, offs)
#define RBC_EMIT(KB, BN, S, QS)                                                             \
  if (offs)                                                                                 \
    return fold_col >= 0 ? RBC_EMIT_OFFS(KB, BN, S, QS, true) : RBC_EMIT_OFFS(KB, BN, S, QS, false); \
  return direct ? (fold_col >= 0 ? RBC_EMIT_ONE(KB, BN, S, QS, true, true)                   \
                                 : RBC_EMIT_ONE(KB, BN, S, QS, false, true))                 \
                : (fold_col >= 0 ? RBC_EMIT_ONE(KB, BN, S, QS, true, false)                  \
                                 : RBC_EMIT_ONE(KB, BN, S, QS, false, false))
  const bool direct = out.arena == nullptr;
  switch (Qm.dpad / 64) {
    case 1: RBC_EMIT(1, 256, 3, 4);
    case 2: RBC_EMIT(2, 256, 2, 2);
    case 3: RBC_EMIT(3, 64, 3, 2);
    case 4: RBC_EMIT(4, 64, 2, 2);
    default: break;
  }
#undef RBC_EMIT
#undef RBC_EMIT_OFFS
#undef RBC_EMIT_ONE
  set_error("tensor-core BF: padded dimension %d unsupported", Qm.dpad);
  return RBC_ERR_UNSUPPORTED;
}

}  // namespace rbc
