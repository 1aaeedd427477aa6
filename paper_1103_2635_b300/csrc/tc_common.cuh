// Device helpers shared by the tensor-core kernels (sm_103a): mbarriers with
// bounded waits, TMA and bulk copies, shared-memory and instruction
// descriptors for tcgen05.mma kind::f16, tensor-memory loads, packed FP32
// arithmetic and small min / max trees.  Everything here is inline PTX.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace rbc {
namespace tc {

constexpr int BM = TQ;                       // query rows per tile (MMA M)
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

// The same with a suspend-time hint: a thread whose phase is not complete
// may sleep up to `ns` nanoseconds (it wakes when the phase completes), so
// waiting warps leave the issue slots to the working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* b, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and sets
// the CTA's abort flag and the device error word) if the wait expired or
// another role already aborted.  The first probe is inline; only a phase that
// is not complete yet pays for the call into the bounded loop.
static __device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t parity,
                                                   volatile int* abort_flag, uint32_t* dev_err) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait_sleep(b, parity, 1000)) return true;
    if ((i & 15) == 15) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > WAIT_NS) {
        *abort_flag = 1;
        atomicOr(dev_err, DEV_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                          uint32_t* dev_err) {
  if (mbar_try_wait(b, parity)) return true;
  return mbar_wait_slow(b, parity, abort_flag, dev_err);
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

// kind::f8f6f4 with E4M3 operands (instruction descriptor format 0 for both)
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
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
// The same load with a reduction: also returns the maximum of the thread's 32
// loaded values.
__device__ __forceinline__ void tmem_ld_x32_max(uint32_t taddr, uint32_t (&r)[32], float& mx) {
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, %32, [%33];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=f"(mx)
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

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

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

// r[j] for a run-time j < 32: a five-level tree of selects on the bits of j
// (a rare path's way to read one of 32 registers without local memory, in a
// few instructions of code).
__device__ __forceinline__ uint32_t pick32(const uint32_t (&r)[32], int j) {
  uint32_t a[16], b[8], c[4], d[2];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = (j & 1) ? r[2 * i + 1] : r[2 * i];
#pragma unroll
  for (int i = 0; i < 8; ++i) b[i] = (j & 2) ? a[2 * i + 1] : a[2 * i];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i] = (j & 4) ? b[2 * i + 1] : b[2 * i];
#pragma unroll
  for (int i = 0; i < 2; ++i) d[i] = (j & 8) ? c[2 * i + 1] : c[2 * i];
  return (j & 16) ? d[1] : d[0];
}

// Bit j set iff the float bits r[j] hold a value above t (GE: at least t).
template <bool GE>
__device__ __forceinline__ uint32_t over_mask32(const uint32_t (&r)[32], float t) {
  uint32_t g[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float v = __uint_as_float(r[4 * q + i]);
      m |= (GE ? v >= t : v > t) ? (1u << i) : 0u;
    }
    g[q] = m;
  }
  return (g[0] | (g[1] << 4) | (g[2] << 8) | (g[3] << 12)) |
         ((g[4] | (g[5] << 4) | (g[6] << 8) | (g[7] << 12)) << 16);
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


// 2D tensor map over a [rows, dpad] bf16 / fp16 row-major matrix: boxes of
// 64 columns x box_rows rows, 128-byte swizzle (defined in bf_tc.cu).
int encode_map(CUtensorMap* map, const void* base, int64_t rows, int dpad, int storage,
               int box_rows);
// The same for a [rows, NBLOCK_COLS] bf16 norm block: boxes of 16 columns
// (32 bytes) x box_rows rows, 32-byte swizzle.
int encode_nblock_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows);

}  // namespace tc
}  // namespace rbc
