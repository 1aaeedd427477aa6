// Tensor-core brute force with a fused per-query top-C, bf16 / fp16
// (sm_103a): BF(Q, X[segments]) for the l2 metric (Section 3: the distance
// step is a matrix product, the comparison step a per-query reduction).
//
// For l2, rho(q, x)^2 = |q|^2 - 2 q.x + |x|^2, and |q|^2 does not change the
// order for a fixed query, so points are ranked by the score
//     s(q, x) = |x~|^2 - 2 q~.x~
// of the stored low-precision rows q~, x~.  The norm term is folded into the
// MMA: beside each database tile the stage holds the tile's norm block
// (-|x~|^2 / 2 as a bf16 high and low part, 16 columns), and one extra bf16
// MMA of an all-ones A block against it adds -|x~|^2 / 2 to every
// accumulator, which then holds q~.x~ - |x~|^2 / 2 = -s / 2.  So the epilogue
// does no arithmetic per score: the tensor-memory load itself returns the
// largest accumulator of every 32-column chunk (tcgen05.ld.red), and a chunk
// is looked at only when that maximum beats the row's current threshold
// (the largest score in its list, halved and negated).  After the first
// tiles of an item that is rare, so the epilogue costs two TMEM loads and two
// compares per thread and tile, and the tensor pipe sets the pace.
//
// Structure (one CTA per SM, persistent over work items):
//   warp 0      TMA producer: the item's 128-row query tile (QS stages, so
//               the next item's tile can load while this one is multiplied),
//               database tiles of BN rows with their norm blocks into an
//               S-stage ring (128-byte / 32-byte swizzle, K-major)
//   warp 1      tensor-memory allocation and MMA issue (M = 128, N = BN,
//               K = 16 per instruction) into two accumulator buffers
//   warps 2-9   epilogue: warp w reads TMEM lane quarter w % 4 (one query row
//               per thread) for one half of every tile's columns, all of it
//               in one go (BN / 64 loads of 32 columns, one wait), hands the
//               buffer back and keeps the CS best (score, column) pairs of
//               its half-row: an unsorted register list (columns in shared
//               memory) whose largest entry is its threshold.  The two halves
//               of a row share their thresholds through shared memory:
//               whichever list has the smaller largest entry holds CS
//               candidates below it, so both may drop anything at or above
//               the smaller of the two (the select step's certificate bounds
//               what a full list dropped by its largest entry).
// Every wait on an mbarrier is bounded; on expiry the kernel raises
// DEV_ERR_TIMEOUT, stops issuing work, waits (bounded) for its own copies and
// frees its tensor memory before returning.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace rbc {

namespace {

using namespace tc;

constexpr int T_EPI0 = 2;  // first epilogue warp
constexpr int T_NEPI = 8;  // epilogue warps: 4 lane quarters x 2 column halves
constexpr int T_THREADS = 32 * (T_EPI0 + T_NEPI);
constexpr int T_NT = 32 * T_NEPI;  // epilogue threads

struct TopParams {
  TileWork w;
  TopOut out;
  uint32_t* dev_err;
};

// Item `item` of the work.  Paired (cluster) dense form: item = (pair of
// query tiles, split), and CTA `rank` of the cluster takes tile 2 pair + rank
// (nq <= 0 for the missing partner of an odd last tile).
template <bool MC = false>
__device__ __forceinline__ void top_item(const TileWork& w, int item, int& q0, int& nq, int& sb,
                                         int& se, int& slot, int rank = 0) {
  if (MC) {
    const int pair = item / w.dense_splits;
    const int s = item - pair * w.dense_splits;
    const int tile = 2 * pair + rank;
    q0 = tile * TQ;
    nq = (int)min((int64_t)TQ, w.m - (int64_t)q0);
    sb = s;
    se = s + 1;
    slot = tile * w.dense_splits + s;
  } else if (w.items) {
    const WorkItem it = w.items[item];
    q0 = it.q_row0;
    nq = it.nq;
    sb = it.seg_begin;
    se = it.seg_end;
    slot = it.slot;
  } else {
    const int tile = item / w.dense_splits;
    const int s = item - tile * w.dense_splits;
    q0 = tile * TQ;
    nq = min(TQ, (int)(w.m - (int64_t)q0));
    sb = s;
    se = s + 1;
    slot = item;
  }
}

template <int KB>
__device__ __forceinline__ int top_item_kb(const TileWork& w, int item) {
  if (!w.tile_kb || !w.items) return KB;
  const int v = w.tile_kb[w.items[item].tile];
  return v < 1 ? 1 : (v > KB ? KB : v);
}

__device__ __forceinline__ Seg top_seg(const TileWork& w, int si) {
  if (w.segs) return w.segs[si];
  const int64_t b = (int64_t)si * w.dense_chunk;
  const int64_t e = min(w.n, b + w.dense_chunk);
  return Seg{(int32_t)b, (int32_t)e};
}

template <int CS, int KB, int BN, int S, int QS, int PQ>
struct TopSmem {
  static constexpr int NBUF = 2;  // TMEM accumulator buffers of BN columns
  static_assert(NBUF * BN >= 32 && (NBUF * BN & (NBUF * BN - 1)) == 0,
                "tcgen05.alloc takes a power of two columns (>= 32)");
  static constexpr int QSTAGES = QS;
  static constexpr int Q_BYTES = KB * BM * 128;
  static constexpr int X_STAGE = KB * BN * 128;
  static constexpr int NB_STAGE = BN * NBLOCK_COLS * 2;
  static constexpr int ONES_BYTES = BM * NBLOCK_COLS * 2;
  static constexpr int OFF_Q = 0;
  static constexpr int OFF_X = OFF_Q + QSTAGES * Q_BYTES;
  static constexpr int OFF_NB = OFF_X + S * X_STAGE;
  static constexpr int OFF_ONES = OFF_NB + S * NB_STAGE;
  // per epilogue thread: its CS list entries (score, column), entry j at
  // [j][thread] -- only the threshold stays in registers
  static constexpr int OFF_IDS = OFF_ONES + ONES_BYTES;
  static constexpr int OFF_LS = OFF_IDS + CS * T_NT * 4;
  // per (half, query row): the largest entry of that half's list, tagged
  // with the run (first item of a query tile's run) it belongs to
  static constexpr int OFF_PQ = OFF_LS + CS * T_NT * 4;  // pending (score, column) stack
  static constexpr int OFF_ROOT = OFF_PQ + PQ * T_NT * 8;
  static constexpr int OFF_BAR = OFF_ROOT + 2 * BM * 8;
  // full[S], empty[S], tfull[NBUF], tempty[NBUF], qfull[QS], qempty[QS]
  static constexpr int NBAR = 2 * S + 2 * NBUF + 2 * QSTAGES;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;  // tmem base, abort flag
  static constexpr int BYTES = OFF_MISC + 16;
  static constexpr int ALLOC = BYTES + 1024;  // slack for 1024-byte alignment
  static_assert(ALLOC <= 232448, "shared memory budget");
  static_assert(OFF_X % 1024 == 0 && X_STAGE % 1024 == 0 && Q_BYTES % 1024 == 0,
                "swizzled tiles need 1024-byte alignment");
  static_assert(OFF_NB % 1024 == 0 && NB_STAGE % 1024 == 0 && OFF_ONES % 1024 == 0,
                "norm blocks need 1024-byte alignment");
};

// Shared-memory descriptor of a K-major operand with 32-byte rows (16 bf16)
// and 32-byte swizzle: 8-row groups 256 bytes apart.
__device__ __forceinline__ uint64_t top_desc_sw32(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(256 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)6 << 61;                   // 32-byte swizzle
  return d;
}

// Cluster helpers for the paired dense pass: the two CTAs of a cluster
// multiply different query tiles by the same database tiles, and each loads
// half of every database tile into both CTAs' shared memory (TMA multicast
// within this GPU's memory), which halves the L2 traffic per SM.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar,
                                               int c0, int c1, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}
// arrive on the same mbarrier in every CTA of `mask` when this CTA's MMAs end
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// CS: list entries per (row, column half); KB: 64-column K blocks; BN:
// database rows per tile; S: database stages; QS: query-tile stages; PQ:
// pending inserts per epilogue thread; MC: paired dense pass on a cluster of
// two CTAs sharing the database tiles by multicast.
template <int CS, int KB, int BN, int S, int QS, int PQ, bool MC>
__global__ void __launch_bounds__(T_THREADS, 1)
bf_tc_top_kernel(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap xmap,
                 const __grid_constant__ CUtensorMap nbmap, TopParams p, uint32_t idesc,
                 uint32_t idesc_norm) {
  using L = TopSmem<CS, KB, BN, S, QS, PQ>;
  constexpr int NBUF = L::NBUF;
  constexpr int NG = CS / 4;  // list groups of four entries
  static_assert(!MC || BN % 16 == 0, "paired tiles split in two halves of 8-row groups");
  const int rank = MC ? (int)cluster_rank() : 0;
  constexpr int COLS = BN / 2;     // columns per epilogue thread per tile
  constexpr int CH = COLS / 32;    // 32-column TMEM loads per thread per tile
  constexpr int RC = CH < 2 ? CH : 2;  // loads per round
  static_assert(CH >= 1 && COLS % 32 == 0, "tile too narrow for two column halves");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* sQ = smem + L::OFF_Q;
  uint8_t* sX = smem + L::OFF_X;
  uint8_t* sNB = smem + L::OFF_NB;
  uint32_t* sOnes = reinterpret_cast<uint32_t*>(smem + L::OFF_ONES);
  int* sIds = reinterpret_cast<int*>(smem + L::OFF_IDS);
  float* sLs = reinterpret_cast<float*>(smem + L::OFF_LS);
  float2* sPq = reinterpret_cast<float2*>(smem + L::OFF_PQ);
  unsigned long long* sRoot = reinterpret_cast<unsigned long long*>(smem + L::OFF_ROOT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + NBUF;
  uint64_t* qfull = tempty + NBUF;
  uint64_t* qempty = qfull + QS;
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + L::OFF_MISC);
  volatile int* sAbort = reinterpret_cast<volatile int*>(smem + L::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], MC ? 2 : 1);  // paired: both CTAs' MMAs must be done with a stage
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], T_NEPI);
    }
    for (int q = 0; q < QS; ++q) {
      mbar_init(&qfull[q], 1);
      mbar_init(&qempty[q], 1);
    }
    *sAbort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the all-ones A block of the norm MMA (bf16 1.0 pairs; every layout of an
  // all-ones block reads the same)
  for (int i = threadIdx.x; i < L::ONES_BYTES / 4; i += blockDim.x) sOnes[i] = 0x3F803F80u;
  // no half-row threshold belongs to a run yet (run tag -1)
  for (int i = threadIdx.x; i < 2 * BM; i += blockDim.x) sRoot[i] = ~0ull;
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
  // paired: the partner's barriers are initialised before any multicast
  if (MC) cluster_sync();
  const uint32_t tmem = *sTmem;

  const TileWork& w = p.w;
  const int n_items = w.num_items_dev ? *w.num_items_dev : w.num_items;
  // a contiguous range of items per CTA, so that consecutive items of one
  // query tile stay on one CTA and the epilogue carries its lists across
  // them; work whose query tiles are single items may take them strided
  // paired: the cluster's two CTAs take the same range of (pair, split) items
  const int cid = MC ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int ncta = MC ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int ib = w.strided ? cid : (int)((int64_t)cid * n_items / ncta);
  const int ie = w.strided ? n_items : (int)((int64_t)(cid + 1) * n_items / ncta);
  const int istep = w.strided ? ncta : 1;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    uint32_t it = 0, qi = 0;
    bool ok = true;
    for (int item = ib; ok && item < ie; item += istep, ++qi) {
      int q0, nq, sb, se, slot;
      top_item<MC>(w, item, q0, nq, sb, se, slot, rank);
      const int kbn = top_item_kb<KB>(w, item);
      const int qs = qi % QS;
      if (!__all_sync(0xffffffffu,
                      mbar_wait(&qempty[qs], ((qi / QS) & 1) ^ 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
      if (lane == 0) {
        mbar_arrive_expect_tx(&qfull[qs], kbn * BM * 128);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb)
          if (kb < kbn) tma_load_2d(sQ + qs * L::Q_BYTES + kb * BM * 128, &qmap, &qfull[qs], kb * 64, q0);
      }
      __syncwarp();
      for (int si = sb; ok && si < se; ++si) {
        const Seg sg = top_seg(w, si);
        for (int x = sg.x_begin; x < sg.x_end; x += BN, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1, sAbort, p.dev_err))) {
            ok = false;
            break;
          }
          if (lane == 0) {
            mbar_arrive_expect_tx(&full[s], kbn * BN * 128 + L::NB_STAGE);
            if (MC) {
              // this CTA's half of the tile (rows rank * BN / 2 ...), into both CTAs
              constexpr int HB = BN / 2;
#pragma unroll
              for (int kb = 0; kb < KB; ++kb)
                if (kb < kbn)
                  tma_load_2d_mc(sX + s * L::X_STAGE + kb * BN * 128 + rank * HB * 128, &xmap,
                                 &full[s], kb * 64, x + rank * HB, (uint16_t)3);
              tma_load_2d_mc(sNB + s * L::NB_STAGE + rank * HB * NBLOCK_COLS * 2, &nbmap, &full[s],
                             0, x + rank * HB, (uint16_t)3);
            } else {
#pragma unroll
              for (int kb = 0; kb < KB; ++kb)
                if (kb < kbn)
                  tma_load_2d(sX + s * L::X_STAGE + kb * BN * 128, &xmap, &full[s], kb * 64, x);
              tma_load_2d(sNB + s * L::NB_STAGE, &nbmap, &full[s], 0, x);
            }
          }
          __syncwarp();
        }
      }
    }
    // drain: every issued copy must have landed before the CTA exits
    if (lane == 0) {
      for (uint32_t j = (it > (uint32_t)S ? it - S : 0); j < it; ++j)
        mbar_wait(&full[j % S], (j / S) & 1, sAbort, p.dev_err);
      for (uint32_t j = (qi > (uint32_t)QS ? qi - QS : 0); j < qi; ++j)
        mbar_wait(&qfull[j % QS], (j / QS) & 1, sAbort, p.dev_err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    uint32_t it = 0, qi = 0;
    bool ok = true;
    for (int item = ib; ok && item < ie; item += istep, ++qi) {
      int q0, nq, sb, se, slot;
      top_item<MC>(w, item, q0, nq, sb, se, slot, rank);
      const int kbn = top_item_kb<KB>(w, item);
      const int qs = qi % QS;
      if (!__all_sync(0xffffffffu, mbar_wait(&qfull[qs], (qi / QS) & 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
      for (int si = sb; ok && si < se; ++si) {
        const Seg sg = top_seg(w, si);
        for (int x = sg.x_begin; x < sg.x_end; x += BN, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          const int buf = it % NBUF;
          const uint32_t aph = (it / NBUF) & 1;
          const bool got = mbar_wait(&full[s], ph, sAbort, p.dev_err) &&
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
                if (kb >= kbn) continue;
                const uint64_t ad = smem_desc_sw128(qa + kb * BM * 128 + k16 * 32);
                const uint64_t bd = smem_desc_sw128(xb + kb * BN * 128 + k16 * 32);
                mma_f16(d_tmem, ad, bd, idesc, (kb | k16) != 0);
              }
            // + (-|x~|^2 / 2) in every row: ones x norm block (bf16, K = 16)
            mma_f16(d_tmem, top_desc_sw32(smem_u32(sOnes)),
                    top_desc_sw32(smem_u32(sNB + s * L::NB_STAGE)), idesc_norm, 1u);
            if (MC)
              mma_commit_mc(&empty[s], (uint16_t)3);  // the stage is free in both CTAs
            else
              mma_commit(&empty[s]);
            mma_commit(&tfull[buf]);
          }
          __syncwarp();
        }
      }
      if (lane == 0) mma_commit(&qempty[qs]);
      __syncwarp();
    }
  } else {
    // ---------------- epilogue ----------------
    // Lane l of warp w owns query row 32 (w % 4) + l (its TMEM lane quarter)
    // in half (w - T_EPI0) / 4 of every tile.  Its list holds the CS best
    // scores seen so far, unsorted, in shared memory (the registers hold the
    // tile's accumulators), in groups of four whose maxima stay in registers;
    // the largest, tau_own, is at lpos; tau is the smaller of tau_own and the
    // other half's largest entry.  A column enters iff its score is below
    // tau; in accumulator units (acc = -s / 2) a 32-column chunk needs a look
    // iff its maximum exceeds -tau / 2.  Once the list is full, qualifying
    // columns go to a small pending stack and are inserted while the warp
    // waits for its next accumulator (the MMA of the next tile is running
    // then), so the inserts stay off the path from the MMA commit through the
    // TMEM loads to the buffer's release.
    const int quarter = warp & 3;
    const int half = (warp - T_EPI0) >> 2;
    const int row = quarter * 32 + lane;
    const int et = threadIdx.x - T_EPI0 * 32;  // epilogue thread index
    int* lid = sIds + et;                      // column of list entry j at lid[j * T_NT]
    float* lsc = sLs + et;                     // its score at lsc[j * T_NT]
    float2* pq = sPq + et;                     // pending entry j at pq[j * T_NT]
    // (run, threshold) pairs as one 64-bit word, so a reader never mixes a
    // threshold with the wrong run (the halves do not synchronise)
    volatile unsigned long long* my_root = sRoot + half * BM + row;
    const volatile unsigned long long* other_root = sRoot + (1 - half) * BM + row;
    auto root_word = [](int run, float t) {
      return ((unsigned long long)(uint32_t)run << 32) | __float_as_uint(t);
    };
    int run = -1;
    uint32_t it = 0;
    bool ok = true;
    int lpos = 0;
    float tau_own = INFINITY;  // = the list's largest entry, at lpos
    float tau = INFINITY;
    float gmax[NG];            // per group of four: its largest entry ...
    int gpos[NG];              // ... and that entry's position
    int npend = 0;
    // (sv, col) into the list if it still beats the threshold: overwrite the
    // largest entry, rescan its group, take the largest group maximum
    auto insert = [&](float sv, int col) {
      if (!(sv < tau)) return;
      lsc[lpos * T_NT] = sv;
      lid[lpos * T_NT] = col;
      const int g = lpos >> 2;
      const float v0 = lsc[(4 * g) * T_NT], v1 = lsc[(4 * g + 1) * T_NT];
      const float v2 = lsc[(4 * g + 2) * T_NT], v3 = lsc[(4 * g + 3) * T_NT];
      float m = v0;
      int mp = 4 * g;
      if (v1 > m) { m = v1; mp = 4 * g + 1; }
      if (v2 > m) { m = v2; mp = 4 * g + 2; }
      if (v3 > m) { m = v3; mp = 4 * g + 3; }
#pragma unroll
      for (int t = 0; t < NG; ++t)
        if (t == g) {
          gmax[t] = m;
          gpos[t] = mp;
        }
      float M = gmax[0];
      int P = gpos[0];
#pragma unroll
      for (int t = 1; t < NG; ++t)
        if (gmax[t] > M) {
          M = gmax[t];
          P = gpos[t];
        }
      tau_own = M;
      lpos = P;
      if (tau_own < tau) {
        tau = tau_own;
        *my_root = root_word(run, tau_own);
      }
    };
    for (int item = ib; ok && item < ie; item += istep) {
      int q0, nq, sb, se, slot;
      top_item<MC>(w, item, q0, nq, sb, se, slot, rank);
      int pq0 = -1, pnq, psb, pse, pslot;
      if (item - istep >= ib) top_item<MC>(w, item - istep, pq0, pnq, psb, pse, pslot, rank);
      int nq0 = -1, nnq, nsb, nse, nslot;
      if (item + istep < ie) top_item<MC>(w, item + istep, nq0, nnq, nsb, nse, nslot, rank);
      if (pq0 != q0) {  // the first item of a run of one query tile: empty lists
#pragma unroll
        for (int j = 0; j < CS; ++j) {
          lsc[j * T_NT] = INFINITY;
          lid[j * T_NT] = -1;
        }
#pragma unroll
        for (int t = 0; t < NG; ++t) {
          gmax[t] = INFINITY;
          gpos[t] = 4 * t;
        }
        lpos = 0;
        tau_own = INFINITY;
        tau = INFINITY;
        npend = 0;
        run = item;
        *my_root = root_word(run, INFINITY);
      }
      for (int si = sb; ok && si < se; ++si) {
        const Seg sg = top_seg(w, si);
        for (int x = sg.x_begin; x < sg.x_end; x += BN, ++it) {
          const int buf = it % NBUF;
          const uint32_t aph = (it / NBUF) & 1;
          // wait for the accumulator; while it is not there, do pending inserts
          bool got = false;
          for (;;) {
            const bool ready = mbar_try_wait(&tfull[buf], aph);
            if (__all_sync(0xffffffffu, ready)) {
              got = true;
              break;
            }
            if (__any_sync(0xffffffffu, npend > 0)) {
              if (npend > 0) {
                --npend;
                const float2 e = pq[npend * T_NT];
                insert(e.x, __float_as_int(e.y));
              }
              continue;
            }
            got = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], aph, sAbort, p.dev_err));
            break;
          }
          if (!got) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t tbase =
              tmem + ((uint32_t)(quarter * 32) << 16) + buf * BN + half * COLS;
          {
            const unsigned long long o = *other_root;
            if ((int)(o >> 32) == run) tau = fminf(tau, __uint_as_float((uint32_t)o));
          }
          const int c0 = x + half * COLS;  // database row of the half's first column
          const int lo = sg.x_begin - c0;  // first valid column of the half
          const int hi = sg.x_end - c0;    // one past the last valid column
          // the half-row in rounds of RC chunks (RC x 32 accumulators in
          // registers); the buffer goes back after the last round's loads
#pragma unroll
          for (int r0 = 0; r0 < CH; r0 += RC) {
            uint32_t raw[RC][32];
            float cmax[RC];  // per chunk: the largest accumulator, from the load itself
#pragma unroll
            for (int c = 0; c < RC; ++c) tmem_ld_x32_max(tbase + (r0 + c) * 32, raw[c], cmax[c]);
            tmem_wait_ld();
            if (r0 + RC == CH) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&tempty[buf]);
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) {
              // The maximum runs over all 32 columns, including any outside
              // the segment (rows of other segments, or zero rows past the
              // matrix end): a false alarm only costs the walk, where the
              // mask decides.
              // rows past the tile's queries (zero padding) are never written
              if (row >= nq || !(cmax[c] > -0.5f * tau)) continue;
              const int clo = lo - (r0 + c) * 32, chi = hi - (r0 + c) * 32;
              if (chi <= 0 || clo >= 32) continue;
              const uint32_t below_hi = chi >= 32 ? 0xffffffffu : (1u << chi) - 1u;
              const uint32_t below_lo = clo <= 0 ? 0u : (1u << clo) - 1u;
              uint32_t mask = below_hi & ~below_lo & over_mask32<false>(raw[c], -0.5f * tau);
              while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const float sv = -2.0f * __uint_as_float(pick32(raw[c], j));
                const int col = c0 + (r0 + c) * 32 + j;
                if (tau_own == INFINITY || npend == PQ) {
                  insert(sv, col);  // list not full yet, or the stack is
                } else if (sv < tau) {
                  pq[npend * T_NT] = make_float2(sv, __int_as_float(col));
                  ++npend;
                }
              }
            }
          }
        }
      }
      const bool carry = nq0 == q0;  // the next item continues this tile's lists
      if (p.out.slot_valid && threadIdx.x == T_EPI0 * 32 && nq > 0)
        p.out.slot_valid[slot] = carry ? 0 : 1;
      if (!carry) {
        while (npend > 0) {
          --npend;
          const float2 e = pq[npend * T_NT];
          insert(e.x, __float_as_int(e.y));
        }
      }
      if (ok && !carry && row < nq) {
        const int64_t base = (((int64_t)slot * TQ + row) * 2 + half) * CS;
#pragma unroll
        for (int j = 0; j < CS; ++j) {
          const float v = lsc[j * T_NT];
          p.out.score[base + j] = v;
          p.out.idx[base + j] = v == INFINITY ? -1 : lid[j * T_NT];
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // paired: no CTA leaves while its partner may still multicast into it or
  // arrive on its barriers (both have drained their own copies by now)
  if (MC) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NBUF * BN)
                 : "memory");
  }
}

template <int CS, int KB, int BN, int S, int QS, int PQ, bool MC>
int launch_top(const LpMatrix& Qm, const LpMatrix& Xm, const TileWork& w, const TopOut& out,
               int grid, cudaStream_t st, uint32_t* dev_err) {
  using L = TopSmem<CS, KB, BN, S, QS, PQ>;
  // paired: each CTA loads half of every database tile (and of its norm block)
  constexpr int XBOX = MC ? BN / 2 : BN;
  CUtensorMap qmap, xmap, nbmap;
  RBC_TRY_TC(encode_map(&qmap, Qm.data, Qm.rows, Qm.dpad, Qm.storage, BM));
  RBC_TRY_TC(encode_map(&xmap, Xm.data, Xm.rows, Xm.dpad, Xm.storage, XBOX));
  RBC_TRY_TC(encode_nblock_map(&nbmap, Xm.nblock, Xm.rows, XBOX));
  auto kern = bf_tc_top_kernel<CS, KB, BN, S, QS, PQ, MC>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC));
  TopParams p{w, out, dev_err};
  const uint32_t idesc = idesc_f16(Qm.storage == RBC_BF16 ? 1 : 0, BM, BN);
  const uint32_t idesc_norm = idesc_f16(1, BM, BN);  // the norm block is bf16 for any storage
  cudaError_t e;
  if (MC) {
    // items are (pair of query tiles, split); one cluster of two CTAs per
    // item range, as many clusters as fit on the GPU at once
    const int64_t tiles = (w.m + TQ - 1) / TQ;
    p.w.num_items = (int)(((tiles + 1) / 2) * w.dense_splits);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(T_THREADS);
    cfg.dynamicSmemBytes = L::ALLOC;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * ((grid + 1) / 2));
    int max_clusters = 0;
    RBC_CUDA(cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg));
    if (max_clusters < 1) {
      set_error("tensor-core BF: no cluster of two CTAs fits (%d bytes of shared memory each)",
                L::ALLOC);
      return RBC_ERR_UNSUPPORTED;
    }
    const int clusters = (int)std::min<int64_t>(max_clusters, std::max(1, p.w.num_items));
    cfg.gridDim = dim3(2 * clusters);
    e = cudaLaunchKernelEx(&cfg, kern, qmap, xmap, nbmap, p, idesc, idesc_norm);
  } else {
    kern<<<grid, T_THREADS, L::ALLOC, st>>>(qmap, xmap, nbmap, p, idesc, idesc_norm);
    e = cudaGetLastError();
  }
  ++t_launches;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kern);
    set_error("bf_tc_top_kernel<CS=%d,KB=%d,BN=%d,S=%d,MC=%d> launch failed: %s (regs %d, local "
              "%zu, dynamic smem %d)",
              CS, KB, BN, S, (int)MC, cudaGetErrorString(e), fa.numRegs, fa.localSizeBytes,
              L::ALLOC);
    return RBC_ERR_CUDA;
  }
  return RBC_OK;
}

template <int CS, int KB, int BN, int S, int QS, int PQ>
int launch_top2(const LpMatrix& Qm, const LpMatrix& Xm, const TileWork& w, const TopOut& out,
                int grid, cudaStream_t st, uint32_t* dev_err) {
  // the dense form (every query tile against the same database ranges) runs
  // paired on clusters of two; work lists run one CTA per item range
  if (!w.items && !w.segs)
    return launch_top<CS, KB, BN, S, QS, PQ, true>(Qm, Xm, w, out, grid, st, dev_err);
  return launch_top<CS, KB, BN, S, QS, PQ, false>(Qm, Xm, w, out, grid, st, dev_err);
}

template <int CS>
int dispatch_kb(const LpMatrix& Qm, const LpMatrix& Xm, const TileWork& w, const TopOut& out,
                int grid, cudaStream_t st, uint32_t* dev_err) {
  // d <= 128: 256-row database tiles (the fewest MMA instructions per
  // column); longer rows, and the widest lists, narrower tiles or fewer
  // stages so that the stages, lists and pending stacks fit in shared memory
  constexpr bool WIDE = CS > 16;
  switch (Qm.dpad / 64) {
    case 1: return launch_top2<CS, 1, 256, WIDE ? 2 : 3, 2, 8>(Qm, Xm, w, out, grid, st, dev_err);
    case 2: return launch_top2<CS, 2, WIDE ? 128 : 256, 2, 1, WIDE ? 8 : 4>(Qm, Xm, w, out, grid, st, dev_err);
    case 3: return launch_top2<CS, 3, WIDE ? 64 : 128, 2, 1, 8>(Qm, Xm, w, out, grid, st, dev_err);
    case 4: return launch_top2<CS, 4, 64, 2, 1, 8>(Qm, Xm, w, out, grid, st, dev_err);
    default: break;
  }
  set_error("tensor-core BF: padded dimension %d unsupported", Qm.dpad);
  return RBC_ERR_UNSUPPORTED;
}

}  // namespace

int launch_bf_tc_top(const LpMatrix& Qm, const LpMatrix& Xm, int cs, const TileWork& w,
                     const TopOut& out, int grid, cudaStream_t st, uint32_t* dev_err) {
  if (!Xm.nblock) {
    set_error("tensor-core BF: the database has no norm block");
    return RBC_ERR_ARG;
  }
  switch (cs) {
    case 8: return dispatch_kb<8>(Qm, Xm, w, out, grid, st, dev_err);
    case 16: return dispatch_kb<16>(Qm, Xm, w, out, grid, st, dev_err);
    case 32: return dispatch_kb<32>(Qm, Xm, w, out, grid, st, dev_err);
    default: break;
  }
  set_error("tensor-core BF: list width %d per half row unsupported (8, 16 or 32)", cs);
  return RBC_ERR_ARG;
}

}  // namespace rbc
