// Merge, re-rank and certification: the comparison step of BF(Q, X)
// (Section 3) finished per query, plus the exactness machinery for the
// low-precision distance pass.
//
// One warp per query row:
//  1. merge the top-C partial lists of every work item of the row's tile
//     (each lane keeps a sorted register list of its share, then c_out rounds
//     of a warp-wide arg-min over the lane heads) -> c_out candidates, one per
//     lane, and the boundary score B of the c_out-th candidate;
//  2. re-rank: each lane recomputes its candidate's distance in FP32
//     difference form sqrt(sum (q_i - x_i)^2) (or sum |q_i - x_i|) from the
//     FP32 rows, four interleaved partial sums combined pairwise;
//  3. bitonic sort of the 32 lanes by (rho, id);
//  4. certification: every point outside the candidate set has a score >= B
//     (the c_out-th merged score, or less: the smallest maximum of a full
//     sub-list, which bounds what the tile kernels dropped); its true distance
//     is at least lower(B), a rounding-error bound of the pass that produced B.  The candidate set holds the true k nearest if
//     lower(B) > rho_(k) * (1 + eps), eps the re-rank's relative bound;
//     otherwise the row is queued for an FP32 re-search;
//  5. near-ties: if two neighbouring ranks among the first k+1 lie within the
//     FP32 bound of each other, every candidate is recomputed in FP64 and the
//     candidates re-sorted by (rho64, id);
//  6. the first k (id, rho) pairs are written at the query's original row.
#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int WARPS = 4;
constexpr float U32 = 5.9604645e-08f;  // 2^-24, unit roundoff of float

__device__ __forceinline__ bool key_lt(float a, int ia, int la, float b, int ib, int lb) {
  return a < b || (a == b && (ia < ib || (ia == ib && la < lb)));
}

// Relative error bound of the re-rank's FP32 rho (see header comment):
// each term carries <= 3u, each of the four partial sums adds (d/4 - 1)u,
// the pairwise combination 2u; halving for the square root and adding its
// rounding, (d/8 + 3)u suffices; twice that is used.
__device__ __forceinline__ float rerank_eps(int d) { return (0.25f * d + 8.0f) * U32; }

// FP32 difference-form distance with four interleaved partial sums (the
// re-rank; relative error <= (d/8 + 3) u, see rerank_eps).
__device__ __forceinline__ float rerank_rho(const float* qr, const float* xr, int d, int metric) {
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
  int i = 0;
  for (; i + 4 <= d; i += 4) {
    float t0 = qr[i] - xr[i], t1 = qr[i + 1] - xr[i + 1];
    float t2 = qr[i + 2] - xr[i + 2], t3 = qr[i + 3] - xr[i + 3];
    if (metric == RBC_L2) {
      p0 = fmaf(t0, t0, p0);
      p1 = fmaf(t1, t1, p1);
      p2 = fmaf(t2, t2, p2);
      p3 = fmaf(t3, t3, p3);
    } else {
      p0 += fabsf(t0);
      p1 += fabsf(t1);
      p2 += fabsf(t2);
      p3 += fabsf(t3);
    }
  }
  for (; i < d; ++i) {
    float t0 = qr[i] - xr[i];
    if (metric == RBC_L2) p0 = fmaf(t0, t0, p0); else p0 += fabsf(t0);
  }
  float sum = (p0 + p1) + (p2 + p3);
  return metric == RBC_L2 ? sqrtf(sum) : sum;
}

// Near-ties: if two neighbouring ranks among the first k+1 (one rank per
// lane, sorted by (rho, id)) lie within the FP32 bound of each other, every
// candidate is recomputed in FP64 and the lanes re-sorted by (rho64, id).
// Returns the ballot of tied ranks (0: nothing recomputed).
__device__ __forceinline__ unsigned fp64_ties(const float* qr, const float* X32, int ld, int d,
                                              int metric, int k, int c_out, float eps, int lane,
                                              float& rho, int& oid, int& brow) {
  float nxt = __shfl_down_sync(0xffffffffu, rho, 1);
  bool tie = lane < k && lane + 1 < c_out && rho != INFINITY && nxt != INFINITY &&
             (nxt - rho) <= eps * (nxt + rho) * 2.0f;
  unsigned tie_mask = __ballot_sync(0xffffffffu, tie);
  if (tie_mask) {
    double r64 = INFINITY;
    if (brow >= 0) {
      const float* xr = X32 + (int64_t)brow * ld;
      double s = 0.0;
      for (int i = 0; i < d; ++i) {
        double t0 = (double)qr[i] - (double)xr[i];
        s += metric == RBC_L2 ? t0 * t0 : fabs(t0);
      }
      r64 = metric == RBC_L2 ? sqrt(s) : s;
    }
    // keys are non-negative doubles, so their bit patterns order like the values
    long long key = brow >= 0 ? __double_as_longlong(r64) : LLONG_MAX;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        long long ok = __shfl_xor_sync(0xffffffffu, key, stride);
        int oi = __shfl_xor_sync(0xffffffffu, oid, stride);
        int ob = __shfl_xor_sync(0xffffffffu, brow, stride);
        bool up = (lane & size) == 0 || size == 32;
        bool lower = (lane & stride) == 0;
        bool other_less = ok < key || (ok == key && oi < oid);
        bool same = ok == key && oi == oid;
        bool take = (lower == up) ? other_less : (!other_less && !same);
        if (take) {
          key = ok;
          oid = oi;
          brow = ob;
        }
      }
    }
    rho = key == LLONG_MAX ? INFINITY : (float)__longlong_as_double(key);
  }
  return tie_mask;
}

template <int CW>
__global__ void __launch_bounds__(WARPS * 32) select_kernel(SelectArgs a) {
  __shared__ float sh_s[WARPS][32][CW + 1];
  __shared__ int sh_i[WARPS][32][CW + 1];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * WARPS + wib;
  const int64_t nrows = a.rows ? (int64_t)*a.num_rows_dev : a.m;
  if (gw >= nrows) return;
  const int row = a.rows ? a.rows[gw] : (int)gw;
  if (a.qorig && a.qorig[row] < 0) return;  // padding row of a grouped layout
  const int tile = row / TQ;
  const int r = row - tile * TQ;
  int sb, se;
  if (a.tile_slot_off) {
    sb = a.tile_slot_off[tile];
    se = a.tile_slot_off[tile + 1];
  } else {
    sb = tile * a.dense_splits;
    se = sb + a.dense_splits;
  }
  const int per_slot = a.nsub * a.C;

  // ---- 1. merge ----
  TopList<CW> lst;
  lst.init();
  const int total = (se - sb) * per_slot;
  for (int e = lane; e < total; e += 32) {
    int s = sb + e / per_slot;
    int j = e - (e / per_slot) * per_slot;
    if (a.slot_valid && !a.slot_valid[s]) continue;
    int64_t off = ((int64_t)s * TQ + r) * per_slot + j;
    int id = a.part_idx[off];
    float v = a.part_score[off];
    if (id >= 0 && lst.admits(v, id)) lst.insert(v, id);
  }
#pragma unroll
  for (int j = 0; j < CW; ++j) {
    sh_s[wib][lane][j] = lst.s[j];
    sh_i[wib][lane][j] = lst.i[j];
  }
  __syncwarp();
  int head = 0;
  float cs = INFINITY;  // this lane's candidate (rank = lane) score
  int ci = INT32_MAX;   // its database buffer row
  for (int j = 0; j < a.c_out; ++j) {
    float hv = head < CW ? sh_s[wib][lane][head] : INFINITY;
    int hi = head < CW ? sh_i[wib][lane][head] : INT32_MAX;
    float bv = hv;
    int bi = hi, bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (key_lt(ov, oi, ol, bv, bi, bl)) {
        bv = ov;
        bi = oi;
        bl = ol;
      }
    }
    if (lane == bl) ++head;
    if (lane == j) {
      cs = bv;
      ci = bi;
    }
  }
  // Every point of the searched set that is not a candidate scored at least
  // B: either it is beyond the c_out-th merged entry, or a tile kernel dropped
  // or evicted it, in which case it scored at least the final largest entry
  // of some full sub-list (thresholds only fall).  So B is the smaller of the
  // c_out-th merged score and the smallest maximum over full sub-lists.
  float bcap = INFINITY;
  for (int s = sb; s < se; ++s) {
    if (a.slot_valid && !a.slot_valid[s]) continue;
    for (int sub = 0; sub < a.nsub; ++sub) {
      const int64_t base = (((int64_t)s * TQ + r) * a.nsub + sub) * a.C;
      float v = -INFINITY;
      int valid = 0;
      for (int j = lane; j < a.C; j += 32) {
        if (a.part_idx[base + j] >= 0) {
          ++valid;
          v = fmaxf(v, a.part_score[base + j]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        valid += __shfl_xor_sync(0xffffffffu, valid, o);
      }
      if (valid == a.C) bcap = fminf(bcap, v);
    }
  }
  const float B = fminf(__shfl_sync(0xffffffffu, cs, a.c_out - 1), bcap);
  const bool valid = lane < a.c_out && ci != INT32_MAX && cs != INFINITY;

  // ---- 2. FP32 re-rank ----
  // rows are ld floats apart; the tile's own dimension (zero columns past it)
  // sets the loop length and the rounding bounds
  const int ld = a.d;
  const int d = a.tile_dim ? (int)a.tile_dim[tile] : a.d;
  const float* qr = a.Q32 + (int64_t)row * ld;
  float rho = INFINITY;
  int oid = INT32_MAX;
  if (valid) {
    rho = rerank_rho(qr, a.X32 + (int64_t)ci * ld, d, a.metric);
    oid = a.xid ? a.xid[ci] : ci;
  }
  int brow = valid ? ci : -1;  // buffer row carried through the sort

  // ---- 3. sort lanes by (rho, id) ----
  auto bitonic = [&](float& v, int& id, int& br) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, v, stride);
        int oi = __shfl_xor_sync(0xffffffffu, id, stride);
        int ob = __shfl_xor_sync(0xffffffffu, br, stride);
        bool up = (lane & size) == 0 || size == 32;
        bool lower = (lane & stride) == 0;
        bool other_less = pair_lt(ov, oi, v, id);
        bool take = (lower == up) ? other_less : (!other_less && !(ov == v && oi == id));
        if (take) {
          v = ov;
          id = oi;
          br = ob;
        }
      }
    }
  };
  bitonic(rho, oid, brow);

  // ---- 4. certification ----
  const float eps = rerank_eps(d);
  const int k = a.k;
  const float rk = __shfl_sync(0xffffffffu, rho, k - 1);
  bool certified;
  if (B == INFINITY) {
    certified = true;  // every point of the searched set is a candidate
  } else {
    float lower;
    if (!a.lp) {
      float rb = a.metric == RBC_L2 ? sqrtf(B) : B;
      lower = rb * (1.0f - a.simt_eps) * (1.0f - 4.0f * U32);
    } else {
      float qn = a.q_lpnorm[row];
      float nq = sqrtf(qn);
      const float xn = __uint_as_float(*a.x_norm_max_bits);
      float span = (nq + xn) * (1.0f + 4.0f * U32);
      // FP32 evaluation bound of |x~|^2 - 2 q~.x~ (tensor-core products are
      // exact, accumulation allowed 2^-20 relative per term): (d+4) 2^-19 span^2,
      // plus 2^-16 max|x~|^2 for a norm term that enters the accumulator as a
      // bf16 (high, low) pair (its error is at most 2^-17 |x~|^2).  FP32
      // expansion on CUDA cores: (d+1) 2^-24 span^2 for the dot product, the
      // norms and the final FMA, taken twice: (d+4) 2^-23 span^2
      float ef = a.exp32 ? (float)(d + 4) * 1.1920929e-07f * span * span
                         : (float)(d + 4) * 1.9073486e-06f * span * span + 1.5258789e-05f * xn * xn;
      float t = B + qn - ef;
      lower = (t > 0.f ? sqrtf(t) * (1.0f - 4.0f * U32) : 0.f);
      if (!a.exp32) lower -= a.q_err[row] + __uint_as_float(*a.x_err_max_bits);
      lower *= (1.0f - 8.0f * U32);
    }
    float upper = rk * (1.0f + eps) * (1.0f + 4.0f * U32);
    certified = lower > upper;
  }

  // ---- 5. near-ties among the first k+1 ranks -> FP64 ----
  const unsigned tie_mask = fp64_ties(qr, a.X32, ld, d, a.metric, a.k, a.c_out, eps, lane, rho, oid,
                                      brow);

  // ---- 6. output ----
  const int64_t orow = a.qorig ? (int64_t)a.qorig[row] : (int64_t)row;
  if (lane < k) {
    bool ok = rho != INFINITY && brow >= 0;
    a.out_ids[orow * k + lane] = ok ? (int64_t)oid : (int64_t)-1;
    a.out_dist[orow * k + lane] = ok ? rho : INFINITY;
  }
  if (lane == 0) {
    if (!certified) {
      int pos = atomicAdd(&a.counters[0], 1);
      if (a.fallback_rows) a.fallback_rows[pos] = row;
    }
    if (tie_mask) atomicAdd(&a.counters[1], 1);
    if (tie_mask & (1u << (k - 1))) atomicAdd(&a.counters[2], 1);
  }
}


// Windowed search: one warp per query.  The query's candidate buffer holds
// every point whose low-precision score passed the query's threshold, which
// includes every point within g(q) >= its k-th neighbour distance -- so the
// true k nearest are among the candidates and no certificate is needed.
//  1. s_k = the k-th smallest candidate score (k <= 16: up to 64 candidates
//     by k rounds of a warp minimum over keys held in registers, more in one
//     pass keeping each lane's 16 smallest keys; k > 16: a bitwise search
//     over the order-preserving integer keys of the scores);
//     k distinct points score <= s_k, so U = dist_upper(s_k) bounds the k-th
//     neighbour distance, and only candidates scoring <= score_bound(U) can
//     be among the k nearest;
//  2. those (normally k plus a few) are compacted into shared memory and
//     re-ranked in FP32, eight lanes per candidate row (coalesced reads,
//     partial sums of d / 8 terms, a three-level tree), then kept per lane
//     sorted by (rho, id);
//  3. c_out rounds of warp arg-min give ranks 0 .. c_out - 1, one per lane;
//     near-ties go through the FP64 step.
// A buffer that overflowed, holds fewer than k entries, or leaves more than
// RERANK_MAX survivors after step 1 sends the query to the re-search.
constexpr int RERANK_PL = 8;                    // re-ranked candidates per lane
constexpr int RERANK_MAX = 32 * RERANK_PL;

__device__ __forceinline__ unsigned score_key(float s) {
  const unsigned b = __float_as_uint(s);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_score(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The k-th smallest (k <= 16) of the n keys key(e), e < n, in one pass: each
// lane keeps the 16 smallest of its keys sorted, then k rounds of a warp
// minimum over the lists' heads (a lane holds at most k of the k smallest).
template <typename KeyFn>
__device__ __forceinline__ unsigned kth_smallest16(int n, int k, int lane, KeyFn key) {
  unsigned t[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) t[j] = 0xffffffffu;
  for (int e = lane; e < n; e += 32) {
    unsigned v = key(e);
    if (v < t[15]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const unsigned lo = min(t[j], v);
        v = max(t[j], v);
        t[j] = lo;
      }
    }
  }
  int head = 0;
  unsigned res = 0xffffffffu;
  for (int r = 0; r < k; ++r) {
    unsigned h = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j == head) h = t[j];
    unsigned mn = h;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    res = mn;
    const unsigned holders = __ballot_sync(0xffffffffu, h == mn);
    if (lane == __ffs(holders) - 1) ++head;
  }
  return res;
}

// The k-th smallest candidate score key of a query's buffer (cnt >= k).
__device__ __forceinline__ unsigned kth_score_key(const float* sc, int cnt, int k, int lane) {
  if (k <= 16) return kth_smallest16(cnt, k, lane, [&](int e) { return score_key(sc[e]); });
  unsigned kth = 0;
  for (int bit = 31; bit >= 0; --bit) {
    const unsigned t = kth | (1u << bit);
    int c = 0;
    for (int e = lane; e < cnt; e += 32) c += score_key(sc[e]) < t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (c < k) kth = t;
  }
  return kth;
}

// Band of the k-th place: the largest FP32 distance a point among the k
// nearest can have, r_k (1 + eps) / (1 - eps) rounded up (the k ranked points
// are k distinct points within r_k / (1 - eps) of the query).
__device__ __forceinline__ float kth_band(float rk, float eps) {
  return rk < INFINITY ? rk * (1.0f + eps) / (1.0f - eps) * (1.0f + 8.0f * U32) : INFINITY;
}

// Exact finish of a query whose FP32 ranks tie (within the re-rank's rounding
// band) across the k-th place: the rows of every candidate whose FP32
// distance is within kth_band -- a set that holds the true k nearest -- are
// evaluated in FP64 and ranked by (rho64, id).  They come in batches: this
// merges the batch sr[0 .. ns) (shared memory, ns <= RERANK_MAX; eight lanes
// per row evaluate it) into the sorted list best_r / best_i [0 .. nbest)
// (shared memory) by k rounds of a warp arg-min over both, and returns the
// new list length, min(k, nbest + ns).  sid / s64 are shared scratch of
// RERANK_MAX entries.  After the last batch, best[0 .. k) is the FP64 brute
// force's answer over the candidates.
__device__ int band_merge(const float* qr, const float* X32, const int* xid, int d, int metric,
                          int k, const int* sr, int ns, int* sid, double* s64, double* best_r,
                          int* best_i, int nbest, int lane) {
  for (int e0 = 0; e0 < ns; e0 += 4) {
    const int e = e0 + (lane >> 3);
    const int row = sr[e < ns ? e : 0];
    const double v = rho64_8(qr, X32 + (int64_t)row * d, d, metric, lane & 7);
    if ((lane & 7) == 0 && e < ns) s64[e] = v;
  }
  for (int e = lane; e < ns; e += 32) sid[e] = xid ? xid[sr[e]] : sr[e];
  __syncwarp();
  const int nout = min(k, nbest + ns);
  unsigned taken = 0;            // bit t: batch entry lane + 32 t already ranked
  bool btaken = lane >= nbest;   // list entry `lane` already ranked (or absent)
  double myr = INFINITY;
  int myi = INT32_MAX;
  for (int j = 0; j < nout; ++j) {
    double bv = INFINITY;
    int bi = INT32_MAX, bt = -2;
    if (!btaken) {
      bv = best_r[lane];
      bi = best_i[lane];
      bt = -1;
    }
    for (int t = 0; t < RERANK_MAX / 32; ++t) {
      const int e = lane + 32 * t;
      if (e < ns && !((taken >> t) & 1u)) {
        const double v = s64[e];
        const int id = sid[e];
        if (v < bv || (v == bv && id < bi)) {
          bv = v;
          bi = id;
          bt = t;
        }
      }
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
    if (lane == bl) {
      if (bt == -1) btaken = true;
      else if (bt >= 0) taken |= 1u << bt;
    }
    if (lane == j) {
      myr = bv;
      myi = bi;
    }
  }
  __syncwarp();
  if (lane < nout) {
    best_r[lane] = myr;
    best_i[lane] = myi;
  }
  __syncwarp();
  return nout;
}

__global__ void __launch_bounds__(WARPS * 32) select_cands_kernel(CandSelectArgs a) {
  __shared__ int stage[WARPS][RERANK_MAX];
  __shared__ float dstage[WARPS][RERANK_MAX];
  __shared__ double s64[WARPS][RERANK_MAX];
  __shared__ double best_r[WARPS][32];
  __shared__ int best_i[WARPS][32];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t wi = (int64_t)blockIdx.x * WARPS + wib;
  const int64_t nw = a.rows ? (a.nrows_dev ? (int64_t)*a.nrows_dev : (int64_t)a.nrows) : a.m;
  if (wi >= nw) return;
  const int64_t q = a.rows ? (int64_t)a.rows[wi] : wi;
  const int cnt = a.cand_cnt[q];
  const int k = a.k;
  auto to_research = [&]() {
    if (lane == 0) {
      const int pos = atomicAdd(&a.counters[0], 1);
      a.fallback_rows[pos] = (int)q;
    }
  };
  if (cnt > a.cap || cnt < k) {
    to_research();
    return;
  }
  const float* sc = a.cand_score + q * a.cap;
  const int* cr = a.cand_row + q * a.cap;
  // ---- 1. k-th smallest score ----
  unsigned kth = 0;
  if (cnt <= 64 && k <= 16) {
    unsigned k0 = lane < cnt ? score_key(sc[lane]) : 0xffffffffu;
    unsigned k1 = lane + 32 < cnt ? score_key(sc[lane + 32]) : 0xffffffffu;
    for (int r = 0; r < k; ++r) {
      unsigned mn = min(k0, k1);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      kth = mn;
      // take one copy of the minimum out: the lowest lane holding it
      const unsigned holders = __ballot_sync(0xffffffffu, k0 == mn || k1 == mn);
      if (lane == __ffs(holders) - 1) {
        if (k0 == mn)
          k0 = 0xffffffffu;
        else
          k1 = 0xffffffffu;
      }
    }
  } else {
    kth = kth_score_key(sc, cnt, k, lane);
  }
  float smax;
  if (a.f32) {
    smax = f32_score_bound(f32_dist_upper(key_score(kth), a.f32_eps, a.metric), a.f32_eps,
                           a.metric);
  } else if (a.mq_bits) {
    // representative-offset estimates: every candidate's row has M <= M_q
    // and eps <= eps_q
    const float M = __uint_as_float(a.mq_bits[q]), eps = __uint_as_float(a.eps_bits[q]);
    smax = off_value_bound(off_dist_upper(key_score(kth), M, eps, a.d), M, eps, a.d);
  } else {
    const float qn = a.q_lpnorm[q], qe = a.q_err[q];
    const float xe = __uint_as_float(*a.x_err_max_bits), xn = __uint_as_float(*a.x_norm_max_bits);
    smax = score_bound(dist_upper(key_score(kth), qn, qe, xe, xn, a.d), qn, qe, xe, xn, a.d);
  }
  // ---- 2. survivors -> shared memory ----
  int* stg = stage[wib];
  int nre = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int e0 = 0; e0 < cnt; e0 += 32) {
    const int e = e0 + lane;
    const bool pass = e < cnt && sc[e] <= smax;
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    const int pos = nre + __popc(bal & lt);
    if (pass && pos < RERANK_MAX) stg[pos] = cr[e];
    nre += __popc(bal);
  }
  if (nre > RERANK_MAX) {
    if (a.stream_rows) {
      if (lane == 0) a.stream_rows[atomicAdd(a.stream_count, 1)] = (int)q;
    } else {
      to_research();
    }
    return;
  }
  __syncwarp();
  const int d = a.d;
  const float* qr = a.Q32 + q * d;
  // FP32 distances of the survivors, four rows at a time
  float* dst = dstage[wib];
  rerank_rows<1>(qr, a.X32, d, a.metric, stg, nre, dst, lane);
  __syncwarp();
  float ls[RERANK_PL];
  int li[RERANK_PL], lr[RERANK_PL];
#pragma unroll
  for (int j = 0; j < RERANK_PL; ++j) {
    ls[j] = INFINITY;
    li[j] = INT32_MAX;
    lr[j] = -1;
  }
  for (int e = lane; e < nre; e += 32) {
    const int row = stg[e];
    float v = dst[e];
    int id = a.xid ? a.xid[row] : row;
    int rw = row;
#pragma unroll
    for (int j = 0; j < RERANK_PL; ++j) {
      const bool lt2 = pair_lt(v, id, ls[j], li[j]);
      const float ts = lt2 ? ls[j] : v;
      const int ti = lt2 ? li[j] : id;
      const int tr = lt2 ? lr[j] : rw;
      ls[j] = lt2 ? v : ls[j];
      li[j] = lt2 ? id : li[j];
      lr[j] = lt2 ? rw : lr[j];
      v = ts;
      id = ti;
      rw = tr;
    }
  }
  // ---- 3. ranks, FP64 ties, output ----
  int head = 0;
  float rho = INFINITY;
  int oid = INT32_MAX, brow = -1;
  for (int j = 0; j < a.c_out; ++j) {
    float hv = INFINITY;
    int hi = INT32_MAX, hr = -1;
#pragma unroll
    for (int t = 0; t < RERANK_PL; ++t)
      if (t == head) {
        hv = ls[t];
        hi = li[t];
        hr = lr[t];
      }
    float bv = hv;
    int bi = hi, bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (key_lt(ov, oi, ol, bv, bi, bl)) {
        bv = ov;
        bi = oi;
        bl = ol;
      }
    }
    const int br = __shfl_sync(0xffffffffu, hr, bl);
    if (lane == bl) ++head;
    if (lane == j) {
      rho = bv;
      oid = bi;
      brow = bv == INFINITY ? -1 : br;
    }
  }
  const float eps = rerank_eps(d);
  // A candidate past rank k - 1 within the band of the k-th place: the
  // lanes' ranks may miss a point of the true k nearest, so every survivor
  // in the band is decided in FP64 (compacted in place: positions only move
  // down, and each chunk is read before the ballot that places it).
  const float band = kth_band(__shfl_sync(0xffffffffu, rho, k - 1), eps);
  unsigned tie_mask;
  if (__shfl_sync(0xffffffffu, rho, k) <= band) {
    int ns = 0;
    for (int e0 = 0; e0 < nre; e0 += 32) {
      const int e = e0 + lane;
      const int row = e < nre ? stg[e] : 0;
      const bool pass = e < nre && dst[e] <= band;
      const unsigned bal = __ballot_sync(0xffffffffu, pass);
      if (pass) stg[ns + __popc(bal & lt)] = row;
      ns += __popc(bal);
    }
    __syncwarp();
    const int nb = band_merge(qr, a.X32, a.xid, d, a.metric, k, stg, ns,
                              reinterpret_cast<int*>(dst), s64[wib], best_r[wib], best_i[wib], 0,
                              lane);
    rho = lane < nb ? (float)best_r[wib][lane] : INFINITY;
    oid = lane < nb ? best_i[wib][lane] : INT32_MAX;
    brow = 0;
    tie_mask = 1u << (k - 1);
  } else {
    tie_mask = fp64_ties(qr, a.X32, d, d, a.metric, k, a.c_out, eps, lane, rho, oid, brow);
  }
  if (lane < k) {
    const bool ok = rho != INFINITY && brow >= 0;
    a.out_ids[q * k + lane] = ok ? (int64_t)oid : (int64_t)-1;
    a.out_dist[q * k + lane] = ok ? rho : INFINITY;
  }
  if (lane == 0) {
    if (tie_mask) atomicAdd(&a.counters[1], 1);
    if (tie_mask & (1u << (k - 1))) atomicAdd(&a.counters[2], 1);
  }
}

template <int CW>
int launch_cw(const SelectArgs& a, int64_t grid_rows, cudaStream_t st) {
  int64_t blocks = (grid_rows + WARPS - 1) / WARPS;
  if (blocks == 0) return RBC_OK;
  select_kernel<CW><<<(unsigned)blocks, WARPS * 32, 0, st>>>(a);
  RBC_LAUNCH_CHECK("select_kernel");
  return RBC_OK;
}

// Queries whose survivors (candidates scoring <= score_bound(U)) outnumber
// the shared-memory re-rank: one warp per query streams every survivor
// through the FP32 re-rank -- the k-th score in one pass over the buffer,
// then batches of up to 256 survivors compacted into shared memory, their
// ids fetched, their distances computed by groups of eight lanes (two rows
// per group at a time).  Each lane keeps its CW best (CW >= c_out, so the
// lanes together hold the query's c_out best for sure), then c_out rounds of
// a warp minimum rank them, then FP64 ties and the output as in select_cands.
template <int CW>
__global__ void __launch_bounds__(WARPS * 32) select_stream_kernel(CandSelectArgs a) {
  constexpr int BATCH = 256;  // survivors re-ranked together
  __shared__ int s_row[WARPS][BATCH];
  __shared__ float s_rho[WARPS][BATCH];
  __shared__ int s_id[WARPS][BATCH];
  __shared__ int s_band[WARPS][RERANK_MAX];
  __shared__ double s_b64[WARPS][RERANK_MAX];
  __shared__ double s_best_r[WARPS][32];
  __shared__ int s_best_i[WARPS][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* srow = s_row[wib];
  float* srho = s_rho[wib];
  int* sid = s_id[wib];
  int* sband = s_band[wib];
  const int64_t nw = *a.stream_count;
  const int k = a.k, d = a.d;
  const float xe = a.f32 ? 0.0f : __uint_as_float(*a.x_err_max_bits);
  const float xn = a.f32 ? 0.0f : __uint_as_float(*a.x_norm_max_bits);
  for (int64_t wi = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); wi < nw;
       wi += (int64_t)gridDim.x * WARPS) {
    const int64_t q = a.stream_rows[wi];
    const int cnt = min(a.cand_cnt[q], a.cap);
    const float* sc = a.cand_score + q * a.cap;
    const int* cr = a.cand_row + q * a.cap;
    // k-th smallest score -> survivor bound (as in select_cands)
    const unsigned kth = kth_score_key(sc, cnt, k, lane);
    float smax;
    if (a.f32) {
      smax = f32_score_bound(f32_dist_upper(key_score(kth), a.f32_eps, a.metric), a.f32_eps,
                             a.metric);
    } else if (a.mq_bits) {
      const float M = __uint_as_float(a.mq_bits[q]), eps = __uint_as_float(a.eps_bits[q]);
      smax = off_value_bound(off_dist_upper(key_score(kth), M, eps, d), M, eps, d);
    } else {
      const float qn = a.q_lpnorm[q], qe = a.q_err[q];
      smax = score_bound(dist_upper(key_score(kth), qn, qe, xe, xn, d), qn, qe, xe, xn, d);
    }
    const float* qr = a.Q32 + q * d;
    float ls[CW];
    int li[CW], lr[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) {
      ls[j] = INFINITY;
      li[j] = INT32_MAX;
      lr[j] = -1;
    }
    // survivors in batches: compacted into shared memory, FP32 distances by
    // groups of eight lanes (four rows at a time), then inserted per lane
    const unsigned lt = (1u << lane) - 1u;
    for (int b0 = 0; b0 < cnt; b0 += BATCH) {
      const int b1 = min(cnt, b0 + BATCH);
      int ns = 0;
      for (int e0 = b0; e0 < b1; e0 += 32) {
        const int e = e0 + lane;
        const bool pass = e < b1 && sc[e] <= smax;
        const unsigned bal = __ballot_sync(0xffffffffu, pass);
        if (pass) srow[ns + __popc(bal & lt)] = cr[e];
        ns += __popc(bal);
      }
      __syncwarp();
      // ids first (independent loads), then distances sixteen rows at a time
      for (int e = lane; e < ns; e += 32) sid[e] = a.xid ? a.xid[srow[e]] : srow[e];
      rerank_rows<4>(qr, a.X32, d, a.metric, srow, ns, srho, lane);
      __syncwarp();
      for (int e = lane; e < ns; e += 32) {
      const int row = srow[e];
      float v = srho[e];
      int id = sid[e];
      if (!pair_lt(v, id, ls[CW - 1], li[CW - 1])) continue;
      int rw = row;
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        const bool lt2 = pair_lt(v, id, ls[j], li[j]);
        const float ts = lt2 ? ls[j] : v;
        const int ti = lt2 ? li[j] : id;
        const int tr = lt2 ? lr[j] : rw;
        ls[j] = lt2 ? v : ls[j];
        li[j] = lt2 ? id : li[j];
        lr[j] = lt2 ? rw : lr[j];
        v = ts;
        id = ti;
        rw = tr;
      }
      }
      __syncwarp();
    }
    int head = 0;
    float rho = INFINITY;
    int oid = INT32_MAX, brow = -1;
    for (int j = 0; j < a.c_out; ++j) {
      float hv = INFINITY;
      int hi = INT32_MAX, hr = -1;
#pragma unroll
      for (int t = 0; t < CW; ++t)
        if (t == head) {
          hv = ls[t];
          hi = li[t];
          hr = lr[t];
        }
      float bv = hv;
      int bi = hi, bl = lane;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        int ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (key_lt(ov, oi, ol, bv, bi, bl)) {
          bv = ov;
          bi = oi;
          bl = ol;
        }
      }
      const int br = __shfl_sync(0xffffffffu, hr, bl);
      if (lane == bl) ++head;
      if (lane == j) {
        rho = bv;
        oid = bi;
        brow = bv == INFINITY ? -1 : br;
      }
    }
    const float eps = rerank_eps(d);
    // a candidate past rank k - 1 within the band of the k-th place: a
    // second pass over the survivors collects those in the band, batch by
    // batch, and merges them into the FP64 (rho, id) order
    const float band = kth_band(__shfl_sync(0xffffffffu, rho, k - 1), eps);
    unsigned tie_mask;
    if (__shfl_sync(0xffffffffu, rho, k) <= band) {
      int nbest = 0;
      for (int b0 = 0; b0 < cnt; b0 += BATCH) {
        const int b1 = min(cnt, b0 + BATCH);
        int nb = 0;
        for (int e0 = b0; e0 < b1; e0 += 32) {
          const int e = e0 + lane;
          const bool pass = e < b1 && sc[e] <= smax;
          const unsigned bal = __ballot_sync(0xffffffffu, pass);
          if (pass) srow[nb + __popc(bal & lt)] = cr[e];
          nb += __popc(bal);
        }
        __syncwarp();
        rerank_rows<4>(qr, a.X32, d, a.metric, srow, nb, srho, lane);
        __syncwarp();
        int ns = 0;
        for (int e0 = 0; e0 < nb; e0 += 32) {
          const int e = e0 + lane;
          const bool pass = e < nb && srho[e] <= band;
          const unsigned bal = __ballot_sync(0xffffffffu, pass);
          if (pass) sband[ns + __popc(bal & lt)] = srow[e];
          ns += __popc(bal);
        }
        __syncwarp();
        if (ns > 0)
          nbest = band_merge(qr, a.X32, a.xid, d, a.metric, k, sband, ns, sid, s_b64[wib],
                             s_best_r[wib], s_best_i[wib], nbest, lane);
      }
      rho = lane < nbest ? (float)s_best_r[wib][lane] : INFINITY;
      oid = lane < nbest ? s_best_i[wib][lane] : INT32_MAX;
      brow = 0;
      tie_mask = 1u << (k - 1);
    } else {
      tie_mask = fp64_ties(qr, a.X32, d, d, a.metric, k, a.c_out, eps, lane, rho, oid, brow);
    }
    if (lane < k) {
      const bool ok = rho != INFINITY && brow >= 0;
      a.out_ids[q * k + lane] = ok ? (int64_t)oid : (int64_t)-1;
      a.out_dist[q * k + lane] = ok ? rho : INFINITY;
    }
    if (lane == 0) {
      if (tie_mask) atomicAdd(&a.counters[1], 1);
      if (tie_mask & (1u << (k - 1))) atomicAdd(&a.counters[2], 1);
    }
  }
}

}  // namespace

int launch_select_stream(const CandSelectArgs& a, int max_rows, cudaStream_t st) {
  if (!a.stream_rows || !a.stream_count || max_rows <= 0) return RBC_OK;
  if (a.k < 1 || a.c_out < a.k || a.c_out > 32) {
    set_error("select_stream: bad k=%d c_out=%d", a.k, a.c_out);
    return RBC_ERR_ARG;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // device-side count: a grid that covers the SMs, each warp striding over rows
  const int grid = (int)std::min<int64_t>((max_rows + WARPS - 1) / WARPS, (int64_t)sms * 8);
  if (a.c_out <= 16)
    select_stream_kernel<16><<<grid, WARPS * 32, 0, st>>>(a);
  else
    select_stream_kernel<32><<<grid, WARPS * 32, 0, st>>>(a);
  RBC_LAUNCH_CHECK("select_stream_kernel");
  return RBC_OK;
}

int launch_select_cands(const CandSelectArgs& a, cudaStream_t st) {
  if (a.k < 1 || a.c_out < a.k || a.c_out > 32 || a.cap != CAND_CAP) {
    set_error("select_cands: bad k=%d c_out=%d cap=%d", a.k, a.c_out, a.cap);
    return RBC_ERR_ARG;
  }
  const int64_t nw = a.rows ? (int64_t)a.nrows : a.m;
  const int64_t blocks = (nw + WARPS - 1) / WARPS;
  if (blocks == 0) return RBC_OK;
  select_cands_kernel<<<(unsigned)blocks, WARPS * 32, 0, st>>>(a);
  RBC_LAUNCH_CHECK("select_cands_kernel");
  return RBC_OK;
}

int launch_select(const SelectArgs& a, cudaStream_t st) {
  if (a.k < 1 || a.c_out < a.k || a.c_out > 32) {
    set_error("select: bad k=%d c_out=%d", a.k, a.c_out);
    return RBC_ERR_ARG;
  }
  // with a device-side row count the grid covers the worst case (a.m rows)
  int64_t grid_rows = a.m;
  int cw = a.c_out <= 2 ? 2 : a.c_out <= 4 ? 4 : a.c_out <= 8 ? 8 : a.c_out <= 16 ? 16 : 32;
  switch (cw) {
    case 2: return launch_cw<2>(a, grid_rows, st);
    case 4: return launch_cw<4>(a, grid_rows, st);
    case 8: return launch_cw<8>(a, grid_rows, st);
    case 16: return launch_cw<16>(a, grid_rows, st);
    default: return launch_cw<32>(a, grid_rows, st);
  }
}

}  // namespace rbc
