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
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int NUM_THREADS = 320;   // 10 warps
constexpr int EPI_WARP0 = 2;       // first epilogue warp
constexpr int BM = TQ;             // query rows per tile (MMA M)
constexpr uint64_t WAIT_NS = 2000000000ull;  // bounded waits: 2 s

#define RBC_TRY_TC(x)            \
  do {                           \
    int _r = (x);                \
    if (_r != RBC_OK) return _r; \
  } while (0)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and sets
// the CTA's abort flag and the device error word) if the wait expired or
// another role already aborted.
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                       uint32_t* dev_err) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > WAIT_NS) {
        *abort_flag = 1;
        atomicOr(dev_err, DEV_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// core groups 1024 bytes apart (SBO); start address in 16-byte units.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B both bf16 (1) or
// both fp16 (0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int ab_fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Wide tensor-memory loads: 32 lanes x N consecutive 32-bit columns, N registers
// per thread; tcgen05.wait::ld must follow before the registers are used.
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_x64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void tmem_load_cols(uint32_t taddr, float (&v)[N]) {
  uint32_t r[N];
  if constexpr (N == 64) tmem_ld_x64(taddr, r);
  else tmem_ld_x32(taddr, r);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < N; ++j) v[j] = __uint_as_float(r[j]);
}

// (d0, d1) = (a0, a1) * (b, b) + (c0, c1) as one packed FP32 instruction
__device__ __forceinline__ void fma2(float& d0, float& d1, float a0, float a1, float b, float c0,
                                     float c1) {
  uint64_t a, bb, c, d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
  asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(c0), "f"(c1));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(bb), "l"(c));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d));
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

struct TcParams {
  TileWork w;
  TopOut out;
  const float* xnorm;  // [rows + pad] |x~|^2, readable up to row index rows + BN
  int64_t x_rows;
  int q_rows;
  uint32_t* dev_err;
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

__device__ __forceinline__ Seg seg_at(const TileWork& w, int si) {
  if (w.segs) return w.segs[si];
  int64_t b = (int64_t)si * w.dense_chunk;
  int64_t e = min(w.n, b + w.dense_chunk);
  return Seg{(int32_t)b, (int32_t)e};
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory layout.  Database tiles start at a row index rounded down to
// a multiple of 4 so that the tile's norms (BN floats) can be fetched with
// one 16-byte-aligned bulk copy; the columns before the segment start and
// past its end are masked to +inf in the epilogue.
// Each (row, half) keeps C candidates (C = 8, 16 or 32).

// Minimum of 32 values as a depth-4 tree of three-input minima.
__device__ __forceinline__ float min_of32(const float (&u)[32]) {
  float a[11];
#pragma unroll
  for (int j = 0; j < 10; ++j) a[j] = min3f(u[3 * j], u[3 * j + 1], u[3 * j + 2]);
  a[10] = fminf(u[30], u[31]);
  const float b0 = min3f(a[0], a[1], a[2]), b1 = min3f(a[3], a[4], a[5]);
  const float b2 = min3f(a[6], a[7], a[8]), b3 = fminf(a[9], a[10]);
  return fminf(min3f(b0, b1, b2), b3);
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Largest of C register values (C = 8, 16 or 32): pairwise maxima, then a
// tree of three-input maxima.
template <int C>
__device__ __forceinline__ float max_of(const float (&v)[C]) {
  float m[C / 2];
#pragma unroll
  for (int j = 0; j < C / 2; ++j) m[j] = fmaxf(v[2 * j], v[2 * j + 1]);
  if constexpr (C == 8) {
    return fmaxf(max3f(m[0], m[1], m[2]), m[3]);
  } else {
    float a = max3f(m[0], m[1], m[2]);
    float b = max3f(m[3], m[4], m[5]);
    float c = fmaxf(m[6], m[7]);
#pragma unroll
    for (int j = 8; j < C / 2; j += 4) {
      a = max3f(a, m[j], m[j + 1]);
      b = max3f(b, m[j + 2], m[j + 3]);
    }
    return max3f(a, b, c);
  }
}

// Bit j set iff v[j] == x (C <= 32), OR-combined in groups of four.
template <int C>
__device__ __forceinline__ uint32_t eq_mask(const float (&v)[C], float x) {
  uint32_t g[C / 4];
#pragma unroll
  for (int q = 0; q < C / 4; ++q)
    g[q] = (v[4 * q] == x ? 1u : 0u) | (v[4 * q + 1] == x ? 2u : 0u) |
           (v[4 * q + 2] == x ? 4u : 0u) | (v[4 * q + 3] == x ? 8u : 0u);
  uint32_t m = 0;
#pragma unroll
  for (int q = 0; q < C / 4; ++q) m |= g[q] << (4 * q);
  return m;
}

// Bit j set iff u[j] < t, for a 32-column chunk.
__device__ __forceinline__ uint32_t hit_mask32(const float (&u)[32], float t) {
  uint32_t g[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    g[q] = (u[4 * q] < t ? 1u : 0u) | (u[4 * q + 1] < t ? 2u : 0u) | (u[4 * q + 2] < t ? 4u : 0u) |
           (u[4 * q + 3] < t ? 8u : 0u);
  return (g[0] | (g[1] << 4) | (g[2] << 8) | (g[3] << 12)) |
         ((g[4] | (g[5] << 4) | (g[6] << 8) | (g[7] << 12)) << 16);
}

template <int C, int KB, int BN, int S, int NR>
struct TcSmem {
  static constexpr int NBUF = (512 / BN) < 4 ? (512 / BN) : 4;  // TMEM accumulator buffers
  static constexpr int Q_BYTES = KB * BM * 128;  // query tile, KB K-blocks of 64 elements
  static constexpr int X_STAGE = KB * BN * 128;  // one database tile
  static constexpr int NORM_STAGE = BN * 4;
  static constexpr int NEPI_WARPS = NUM_THREADS / 32 - EPI_WARP0;
  static constexpr int OFF_Q = 0;
  static constexpr int OFF_X = OFF_Q + Q_BYTES;
  static constexpr int OFF_NORM = OFF_X + S * X_STAGE;
  static constexpr int NEPI_THREADS = NEPI_WARPS * 32;
  // per epilogue thread: the columns of its C list entries, entry j at [j][thread]
  static constexpr int OFF_IDS = OFF_NORM + NR * NORM_STAGE;
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
template <int C, int KB, int BN, int S, int NRING>
__global__ void __launch_bounds__(NUM_THREADS, 1)
bf_tc_kernel(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap xmap,
             TcParams p, uint32_t idesc) {
  using L = TcSmem<C, KB, BN, S, NRING>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* sQ = smem + L::OFF_Q;
  uint8_t* sX = smem + L::OFF_X;
  float* sNorm = reinterpret_cast<float*>(smem + L::OFF_NORM);
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
  // query tile stay on one CTA and the epilogue can carry its lists across them
  const int ib = (int)((int64_t)blockIdx.x * n_items / gridDim.x);
  const int ie = (int)((int64_t)(blockIdx.x + 1) * n_items / gridDim.x);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    uint32_t it = 0, qi = 0;
    bool ok = true;
    for (int item = ib; ok && item < ie; ++item, ++qi) {
      int q0, nq, sb, se, slot;
      item_info(w, item, q0, nq, sb, se, slot);
      if (!__all_sync(0xffffffffu, mbar_wait(qempty, (qi & 1) ^ 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
      if (lane == 0) {
        mbar_arrive_expect_tx(qfull, L::Q_BYTES);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) tma_load_2d(sQ + kb * BM * 128, &qmap, qfull, kb * 64, q0);
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
            mbar_arrive_expect_tx(&full[s], L::X_STAGE);
#pragma unroll
            for (int kb = 0; kb < KB; ++kb)
              tma_load_2d(sX + s * L::X_STAGE + kb * BN * 128, &xmap, &full[s], kb * 64, x);
            mbar_arrive_expect_tx(&nfull[r], L::NORM_STAGE);
            bulk_load(sNorm + r * BN, p.xnorm + x, L::NORM_STAGE, &nfull[r]);
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
    for (int item = ib; ok && item < ie; ++item, ++qi) {
      int q0, nq, sb, se, slot;
      item_info(w, item, q0, nq, sb, se, slot);
      if (!__all_sync(0xffffffffu, mbar_wait(qfull, qi & 1, sAbort, p.dev_err))) {
        ok = false;
        break;
      }
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
                uint64_t ad = smem_desc_sw128(qa + kb * BM * 128 + k16 * 32);
                uint64_t bd = smem_desc_sw128(xb + kb * BN * 128 + k16 * 32);
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
    for (int item = ib; ok && item < ie; ++item) {
      int q0, nq, sb, se, slot;
      item_info(w, item, q0, nq, sb, se, slot);
      int pq0 = -1, pnq, psb, pse, pslot;
      if (item > ib) item_info(w, item - 1, pq0, pnq, psb, pse, pslot);
      int nq0 = -1, nnq, nsb, nse, nslot;
      if (item + 1 < ie) item_info(w, item + 1, nq0, nnq, nsb, nse, nslot);
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
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float4 nn = n4[j];
              fma2(u[4 * j], u[4 * j + 1], u[4 * j], u[4 * j + 1], -2.0f, nn.x, nn.y);
              fma2(u[4 * j + 2], u[4 * j + 3], u[4 * j + 2], u[4 * j + 3], -2.0f, nn.z, nn.w);
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

int encode_map(CUtensorMap* map, const void* base, int64_t rows, int dpad, int storage,
               int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return RBC_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)dpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)dpad * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(
      map, storage == RBC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
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

template <int C, int KB, int BN, int S, int NR>
int launch_tc(const LpMatrix& Qm, const LpMatrix& Xm, const TileWork& w, const TopOut& out,
              int grid, cudaStream_t st, uint32_t* dev_err) {
  using L = TcSmem<C, KB, BN, S, NR>;
  CUtensorMap qmap, xmap;
  RBC_TRY_TC(encode_map(&qmap, Qm.data, Qm.rows, Qm.dpad, Qm.storage, BM));
  RBC_TRY_TC(encode_map(&xmap, Xm.data, Xm.rows, Xm.dpad, Xm.storage, BN));
  auto kern = bf_tc_kernel<C, KB, BN, S, NR>;
  RBC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC));
  TcParams p{w, out, Xm.norm, Xm.rows, (int)Qm.rows, dev_err};
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
  if (C == 8) {
    switch (Qm.dpad / 64) {
      case 1: return launch_tc<8, 1, 256, 4, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 2: return launch_tc<8, 2, 128, 3, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 3: return launch_tc<8, 3, 64, 3, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 4: return launch_tc<8, 4, 64, 2, 4>(Qm, Xm, w, out, grid, st, dev_err);
      default: break;
    }
  } else if (C == 16) {
    switch (Qm.dpad / 64) {
      case 1: return launch_tc<16, 1, 256, 4, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 2: return launch_tc<16, 2, 128, 3, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 3: return launch_tc<16, 3, 64, 3, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 4: return launch_tc<16, 4, 64, 2, 4>(Qm, Xm, w, out, grid, st, dev_err);
      default: break;
    }
  } else if (C == 32) {
    switch (Qm.dpad / 64) {
      case 1: return launch_tc<32, 1, 256, 4, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 2: return launch_tc<32, 2, 128, 2, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 3: return launch_tc<32, 3, 64, 3, 8>(Qm, Xm, w, out, grid, st, dev_err);
      case 4: return launch_tc<32, 4, 64, 2, 2>(Qm, Xm, w, out, grid, st, dev_err);
      default: break;
    }
  } else {
    set_error("tensor-core BF: list width %d unsupported (8, 16 or 32)", C);
    return RBC_ERR_ARG;
  }
  set_error("tensor-core BF: padded dimension %d unsupported", Qm.dpad);
  return RBC_ERR_UNSUPPORTED;
}

}  // namespace rbc
