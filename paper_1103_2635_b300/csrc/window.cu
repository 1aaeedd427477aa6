// Work generation of the windowed exact search (Section 5.2 with lists sorted
// by distance to their representative).
//
// Every query q first learns g(q), an upper bound of its k-th nearest-neighbour
// distance: the smaller of gamma_k (its k-th nearest representative, a
// database point) and the k-th distance inside the list of its nearest
// representative.  A point x of list L_r can be among q's k nearest only if
//   (1) rho(q, r) <= g + psi_r           (rule (1) of Section 5.2),
//   (2) rho(q, r) <= 2 g + gamma_1       (Lemma 1, generalised to k), and
//   (3) |rho(x, r) - rho(q, r)| <= g     (triangle inequality),
// so with L_r sorted by rho(x, r), q needs only the window of L_r between
// rho(q, r) - g and rho(q, r) + g.  All comparisons carry the FP32 rounding
// bounds of the values involved, so no needed point is ever cut.
//
// The surviving (q, r) pairs are binned by (r, bucket of rho(q, r) - g(q)),
// the lower end of the query's window -- NB buckets over [0, psi_r] for each
// r -- with a counting sort over the implicit pair list, so each r's group
// comes out ordered by the window start up to the bucket width.  Each group
// is cut into chunks of up to TQ queries: one work item per chunk, against
// the union of its queries' windows.  Ordered by window start, consecutive
// windows overlap almost entirely (ordering by rho(q, r) alone would mix
// queries of very different g and about double the union).
//
// The two pair passes (count, scatter) read D [m, n_r] in warp tiles of 32
// queries x 32 representatives through shared memory, so that a lane owns a
// query and the warp walks the representatives (a lane per representative,
// walking the queries, was measured slower: its pair writes scatter over 32
// bins).  They keep the block's bin counters in shared memory (a lane's kept
// pair takes its slot there), so global memory sees one atomic per non-empty
// (block, bin) on an array of n_r NB counters that stays in L2, and the
// pairs of one bin from one block land in consecutive slots.

#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int WT = 32;           // queries per warp tile
constexpr int WW = 8;            // warps per block of the pair passes
constexpr int RSPAN = 32;        // representatives per block (grid.y splits the rest)
constexpr int NBK = 64;          // window buckets per representative
constexpr float SLACK = 1.0f + 2.4e-7f;

__device__ __forceinline__ bool keep_pair(float d, float lo, float gh, float psi, float lemma) {
  const float dl = d * lo;
  return dl <= (gh + psi) * SLACK && dl <= lemma;
}

// g[q] = min(gamma_k (1 + rel_rep), own-list bound), both rounded up
__global__ void gbound_kernel(const float* __restrict__ own, const float* __restrict__ gk,
                              int64_t m, float rel_rep, float* __restrict__ g) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  g[q] = fminf(gk[q] * (1.0f + rel_rep) * SLACK, own[q]);
}

// Own-list bound from the tensor-core top-C lists of the grouped rows, one
// warp per row: the k best-scored candidates of the row's two sub-lists are
// k distinct points of its list, so the largest of their FP32 distances
// (rounded up by the re-rank bound) bounds the row's k-th distance.  If the
// lists hold fewer than k points the bound is infinite.
__global__ void own_kth_lp_kernel(const float* __restrict__ ps, const int* __restrict__ pi, int C,
                                  const int* __restrict__ qsrc, int64_t rows, int k,
                                  const float* __restrict__ Q32, const float* __restrict__ X32,
                                  int d, int metric, float rel, float* __restrict__ own) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const int q = qsrc[row];  // the batch query of this grouped row
  if (q < 0) return;
  const int64_t base = row * 2 * (int64_t)C;  // [slot = tile][TQ][2][C]
  // up to 2C <= 64 entries, two per lane
  float s0 = INFINITY, s1 = INFINITY;
  int c0 = -1, c1 = -1;
  if (lane < 2 * C) {
    c0 = pi[base + lane];
    s0 = c0 >= 0 ? ps[base + lane] : INFINITY;
  }
  if (lane + 32 < 2 * C) {
    c1 = pi[base + lane + 32];
    s1 = c1 >= 0 ? ps[base + lane + 32] : INFINITY;
  }
  if (s1 < s0) {  // each lane's smaller entry first
    float ts = s0;
    s0 = s1;
    s1 = ts;
    int tc = c0;
    c0 = c1;
    c1 = tc;
  }
  int mine = -1;  // lane j takes the j-th best-scored column
  for (int j = 0; j < k; ++j) {
    float bv = s0;
    int bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (ov < bv || (ov == bv && ol < bl)) {
        bv = ov;
        bl = ol;
      }
    }
    const int col = __shfl_sync(0xffffffffu, c0, bl);
    if (lane == j) mine = bv < INFINITY ? col : -1;
    if (lane == bl) {
      s0 = s1;
      c0 = c1;
      s1 = INFINITY;
      c1 = -1;
    }
  }
  // FP32 distances of the k chosen rows, four at a time by groups of eight
  // lanes (coalesced row reads); group g of round r takes lane 4r + g's row
  float rho = 0.0f;
  const bool missing = lane < k && mine < 0;
  const float* qr = Q32 + (int64_t)q * d;
  for (int r0 = 0; r0 < k; r0 += 4) {
    const int src = r0 + (lane >> 3);
    const int col = __shfl_sync(0xffffffffu, mine, src & 31);
    const float v = rerank_rho8(qr, X32 + (int64_t)(col >= 0 ? col : 0) * d, d, metric, lane & 7);
    if (src < k && col >= 0) rho = fmaxf(rho, v);
  }
  const bool any_missing = __any_sync(0xffffffffu, missing);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rho = fmaxf(rho, __shfl_xor_sync(0xffffffffu, rho, o));
  if (lane == 0) own[q] = any_missing ? INFINITY : rho * (1.0f + rel) * SLACK;
}

// One warp tile: D[q0 .. q0+31][r0 .. r0+31] -> tile[query][r] (padded).
__device__ __forceinline__ void load_tile(const float* __restrict__ D, int64_t m, int n_r,
                                          int64_t q0, int r0, float (*tile)[WT + 1], int lane) {
  const int r = r0 + lane;
#pragma unroll
  for (int j = 0; j < WT; ++j) {
    const int64_t q = q0 + j;
    tile[j][lane] = (q < m && r < n_r) ? D[q * n_r + r] : INFINITY;
  }
  __syncwarp();
}

// the binning key of a kept pair: the window's lower end rho(q, r) - g(q)
__device__ __forceinline__ float window_key(float d, float gh) { return d - gh; }

// The pair passes: block (x, y) covers queries [x * 256, +256) (one warp tile
// of 32 queries per warp) and representatives [y * RSPAN, +RSPAN).
struct PairCtx {
  int64_t q;
  bool live;
  float lo, gh, lemma;
};

__device__ __forceinline__ PairCtx pair_ctx(int64_t q0, int lane, int64_t m,
                                            const float* __restrict__ g,
                                            const float* __restrict__ g1, float rel) {
  PairCtx c;
  c.q = q0 + lane;
  c.live = c.q < m;
  c.lo = 1.0f - rel;
  c.gh = c.live ? g[c.q] : 0.0f;
  c.lemma = c.live ? (2.0f * c.gh + g1[c.q] * (1.0f + rel)) * SLACK : -1.0f;
  return c;
}

__device__ __forceinline__ int bucket_of(float key, float scale) {
  return min(NBK - 1, max(0, (int)(key * scale)));
}

// The two pair passes.  Count: the block's kept pairs per (r, bucket) bin in
// shared memory, then one global atomic per non-empty (block, bin) into
// bin_ctr, whose old value -- the block's offset within the bin -- is kept
// in blk_off (one contiguous row of n_r NB per block), and the block's kept
// count into *kept_sum.  Scatter: each bin's slots start at bin_off plus
// the block's offset, and the pairs go to those slots.  The bins of r cover the
// window starts rho(q, r) - g(q) in [0, psi_r] (every kept pair has a start
// of at most psi_r, and all starts below 0 begin the window at the list's
// first entry).  The order of the blocks' slot runs within a bin is that of
// their atomics: work items differ between runs, results do not.
template <bool SCATTER>
__global__ void __launch_bounds__(WW * 32)
wpairs_kernel(const float* __restrict__ D, int64_t m, int n_r, const float* __restrict__ g,
              const float* __restrict__ g1, const float* __restrict__ psi_plus, float rel,
              int* __restrict__ bin_ctr, const int* __restrict__ bin_off,
              int* __restrict__ blk_off, int2* __restrict__ pairs,
              unsigned long long* __restrict__ kept_sum, unsigned* __restrict__ mq_bits) {
  __shared__ float tiles[WW][WT][WT + 1];
  __shared__ int h[RSPAN * NBK];
  __shared__ float spsi[RSPAN], sscale[RSPAN];
  __shared__ int skept[WW];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.y * RSPAN, re = min(n_r, rb + RSPAN);
  const int64_t bin0 = (int64_t)rb * NBK;
  int* brow = blk_off + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (RSPAN * NBK);
  for (int i = threadIdx.x; i < RSPAN * NBK; i += blockDim.x)
    h[i] = SCATTER ? (i < (re - rb) * NBK ? bin_off[bin0 + i] + brow[i] : 0) : 0;
  for (int i = threadIdx.x; i < re - rb; i += blockDim.x) {
    const float ps = psi_plus[rb + i];
    spsi[i] = ps;
    sscale[i] = ps > 0.0f ? (float)NBK / ps : 0.0f;
  }
  __syncthreads();
  const int64_t q0 = ((int64_t)blockIdx.x * WW + wid) * WT;
  const PairCtx c = pair_ctx(q0, lane, m, g, g1, rel);
  float mq = 0.0f;  // count pass with offsets: the largest M of the lane's kept pairs
  // one pass over the warp's tiles: count, or (place) take the slots
  auto walk = [&](bool place) {
    int kept = 0;
    if (q0 >= m) return kept;
    for (int r0 = rb; r0 < re; r0 += WT) {
      load_tile(D, m, n_r, q0, r0, tiles[wid], lane);
      const int nr = min(WT, re - r0);
      for (int rr = 0; rr < nr; ++rr) {
        const int rl = r0 + rr - rb;
        const float v = tiles[wid][lane][rr];
        if (c.live && keep_pair(v, c.lo, c.gh, spsi[rl], c.lemma)) {
          int* hp = &h[rl * NBK + bucket_of(window_key(v, c.gh), sscale[rl])];
          if (place) {
            pairs[atomicAdd(hp, 1)] = make_int2((int)c.q, __float_as_int(v));
          } else {
            ++kept;
            atomicAdd(hp, 1);
            if (mq_bits) mq = fmaxf(mq, off_pair_m(v, spsi[rl]));
          }
        }
      }
      __syncwarp();
    }
    return kept;
  };
  if (SCATTER) {
    walk(true);
    return;
  }
  const int kept = walk(false);
  if (mq_bits && mq > 0.0f) atomicMax(mq_bits + c.q, __float_as_uint(mq));
  __syncthreads();
  {
    for (int i = threadIdx.x; i < (re - rb) * NBK; i += blockDim.x)
      brow[i] = h[i] ? atomicAdd(&bin_ctr[bin0 + i], h[i]) : 0;
    const int wk = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0) skept[wid] = wk;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < WW; ++w) t += (unsigned long long)skept[w];
      if (t) atomicAdd(kept_sum, t);
    }
  }
}

// per representative: chunks of TQ pairs in its group
__global__ void chunk_count_kernel(const int* __restrict__ bin_off, int nb, int n_r,
                                   int* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_r) out[r] = (bin_off[(r + 1) * nb] - bin_off[r * nb] + TQ - 1) / TQ;
}

// Warp-cooperative searches in sorted arrays: each round probes 32 evenly
// spaced positions at once and keeps the gap holding the answer, so an array
// of N entries costs about log_32(N) dependent loads.
// The two searches of a window at once: the first index with a[i] >= vlo and
// the first with a[i] > vhi, each n if none; both probes of a round are issued
// together, so the pair costs the dependent loads of one search.
__device__ __forceinline__ void warp_bounds2(const float* __restrict__ a, int n, float vlo,
                                             float vhi, int lane, int& blo, int& bhi) {
  int lo0 = 0, hi0 = n, lo1 = 0, hi1 = n;
  while (hi0 - lo0 > 32 || hi1 - lo1 > 32) {
    const int64_t len0 = hi0 - lo0, len1 = hi1 - lo1;
    const bool act0 = len0 > 32, act1 = len1 > 32;
    const int p0 = lo0 + (int)((len0 * lane) >> 5), p1 = lo1 + (int)((len1 * lane) >> 5);
    const float a0 = act0 ? a[p0] : 0.0f, a1 = act1 ? a[p1] : 0.0f;
    if (act0) {
      const int c = __popc(__ballot_sync(0xffffffffu, a0 < vlo));
      const int nlo = c == 0 ? lo0 : lo0 + (int)((len0 * (c - 1)) >> 5) + 1;
      hi0 = c == 32 ? hi0 : lo0 + (int)((len0 * c) >> 5);
      lo0 = nlo;
    }
    if (act1) {
      const int c = __popc(__ballot_sync(0xffffffffu, a1 <= vhi));
      const int nlo = c == 0 ? lo1 : lo1 + (int)((len1 * (c - 1)) >> 5) + 1;
      hi1 = c == 32 ? hi1 : lo1 + (int)((len1 * c) >> 5);
      lo1 = nlo;
    }
  }
  const int q0 = lo0 + lane, q1 = lo1 + lane;
  const float a0 = q0 < hi0 ? a[q0] : 0.0f, a1 = q1 < hi1 ? a[q1] : 0.0f;
  blo = lo0 + __popc(__ballot_sync(0xffffffffu, q0 < hi0 && a0 < vlo));
  bhi = lo1 + __popc(__ballot_sync(0xffffffffu, q1 < hi1 && a1 <= vhi));
}

// The last r in [0, n_r) with off[r] <= c (off ascending, off[0] <= c),
// probing 32 positions per round.
__device__ __forceinline__ int warp_group_of(const int* __restrict__ off, int n_r, int c,
                                             int lane) {
  int lo = 0, hi = n_r;  // the answer lies in [lo, hi)
  while (hi - lo > 32) {
    const int64_t len = hi - lo;
    const int p = lo + (int)((len * lane) >> 5);
    const int cnt = __popc(__ballot_sync(0xffffffffu, off[p] <= c));  // >= 1: off[lo] <= c
    const int nhi = cnt == 32 ? hi : lo + (int)((len * cnt) >> 5);
    lo = lo + (int)((len * (cnt - 1)) >> 5);
    hi = nhi;
  }
  const int p = lo + lane;
  const bool le = p < hi && off[p] <= c;
  return lo + __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// Warps take contiguous runs of chunks: the union of each chunk's windows,
// cut from the sorted list by a cooperative binary search.  A run finds its
// first chunk's representative by a search of chunk_off and then steps r
// forward as the run crosses representatives, so a chunk costs the loads of
// its pairs, their g, and the window search.  Statistics are summed per
// block and added once per block.
__global__ void __launch_bounds__(256)
window_items_kernel(const int* __restrict__ chunk_off, int n_r, const int* __restrict__ bin_off,
                    int nb, const int2* __restrict__ pairs,
                    const float* __restrict__ g, const int* __restrict__ offsets,
                    const float* __restrict__ xdist, float rel, float relx, int max_items,
                    EmitItem* __restrict__ items, unsigned long long* __restrict__ stats) {
  __shared__ unsigned long long part[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int total = min(chunk_off[n_r], max_items);
  const float dlo = 1.0f - rel, dup = 1.0f + rel;
  const float xlo = (1.0f - relx) * (1.0f - 2.4e-7f), xup = (1.0f + relx) * SLACK;
  unsigned long long rows_sum = 0, pairs_sum = 0;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int per = (total + nwarps - 1) / nwarps;
  const int cb = min(total, gw * per), ce = min(total, cb + per);
  int r = cb < ce ? warp_group_of(chunk_off, n_r, cb, lane) : 0;
  int r_end = cb < ce ? chunk_off[r + 1] : 0;  // first chunk past r
  for (int c = cb; c < ce; ++c) {
    while (c >= r_end) r_end = chunk_off[++r + 1];  // the run enters the next r
    const int begin = bin_off[r * nb] + (c - chunk_off[r]) * TQ;
    const int end = min(begin + TQ, bin_off[(r + 1) * nb]);
    const int ob = offsets[r], oe = offsets[r + 1];
    // the chunk's pairs (up to TQ = 4 x 32) and their g, loads issued together
    int2 pr[TQ / 32];
#pragma unroll
    for (int u = 0; u < TQ / 32; ++u) {
      const int i = begin + lane + 32 * u;
      pr[u] = i < end ? pairs[i] : make_int2(-1, 0);
    }
    float gq[TQ / 32];
#pragma unroll
    for (int u = 0; u < TQ / 32; ++u) gq[u] = pr[u].x >= 0 ? g[pr[u].x] : 0.0f;
    float wlo = INFINITY, whi = -INFINITY;
#pragma unroll
    for (int u = 0; u < TQ / 32; ++u) {
      if (pr[u].x < 0) continue;
      const float d = __int_as_float(pr[u].y);
      wlo = fminf(wlo, (d * dlo - gq[u] * SLACK) * xlo);
      whi = fmaxf(whi, (d * dup + gq[u]) * xup);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      wlo = fminf(wlo, __shfl_xor_sync(0xffffffffu, wlo, o));
      whi = fmaxf(whi, __shfl_xor_sync(0xffffffffu, whi, o));
    }
    int xb, xe;
    warp_bounds2(xdist + ob, oe - ob, wlo, whi, lane, xb, xe);
    xb += ob;
    xe += ob;
    if (lane == 0) {
      items[c] = EmitItem{begin, end - begin, xb, xe > xb ? xe : xb, r};
      if (xe > xb) {
        rows_sum += (unsigned long long)(xe - xb);
        pairs_sum += (unsigned long long)(end - begin) * (unsigned long long)(xe - xb);
      }
    }
  }
  if (lane == 0) {
    part[0][wid] = rows_sum;
    part[1][wid] = pairs_sum;
  }
  __syncthreads();
  if (threadIdx.x == 0 && stats) {
    unsigned long long a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += part[0][w];
      b += part[1][w];
    }
    if (a) atomicAdd(&stats[0], a);
    if (b) atomicAdd(&stats[1], b);
  }
}

// One warp per overflowing query: the k-th smallest of its stored scores
// (bitwise search over order-preserving keys) -> a tighter threshold.
// One block per overflowing row: the k-th smallest stored key by a radix
// select over its four bytes (a 256-bin shared histogram per byte, most
// significant first), the same key the bitwise search over all 32 bits finds.
__global__ void __launch_bounds__(256)
overflow_rethreshold_kernel(const int* __restrict__ rows, const int* __restrict__ n_dev,
                            const float* __restrict__ cand_score, int* __restrict__ cand_cnt,
                            int cap, int k, const float* __restrict__ qnorm,
                            const float* __restrict__ qerr, const unsigned* __restrict__ lp_max,
                            int d, float* __restrict__ thr, float f32_eps, int metric,
                            const unsigned* __restrict__ mq_bits,
                            const unsigned* __restrict__ eps_bits) {
  __shared__ int hist[256];
  __shared__ unsigned s_prefix;
  __shared__ int s_rank;
  const int n = *n_dev;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int q = rows[i];
    const int stored = min(cand_cnt[q], cap);
    float t = INFINITY;
    if (stored >= k) {
      const float* sc = cand_score + (int64_t)q * cap;
      unsigned prefix = 0, mask = 0;
      int rank = k;  // 1-based rank of the wanted key among those matching prefix
      for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < stored; e += blockDim.x) {
          const unsigned bits = __float_as_uint(sc[e]);
          const unsigned key = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
          if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          int cum = 0, b = 0;
          for (; b < 255 && cum + hist[b] < rank; ++b) cum += hist[b];
          s_prefix = prefix | ((unsigned)b << shift);
          s_rank = rank - cum;
        }
        __syncthreads();
        prefix = s_prefix;
        rank = s_rank;
        mask |= 255u << shift;
      }
      const unsigned res = prefix;
      const float sk = __uint_as_float((res & 0x80000000u) ? (res & 0x7fffffffu) : ~res);
      if (qnorm) {
        // stored values: low-precision scores, or offset estimates whose
        // distance bound the raw scores of the dense pass then use
        const float xe = __uint_as_float(lp_max[0]), xn = __uint_as_float(lp_max[1]);
        const float u = mq_bits ? off_dist_upper(sk, __uint_as_float(mq_bits[q]),
                                                 __uint_as_float(eps_bits[q]), d)
                                : dist_upper(sk, qnorm[q], qerr[q], xe, xn, d);
        t = score_bound(u, qnorm[q], qerr[q], xe, xn, d);
      } else {
        t = f32_score_bound(f32_dist_upper(sk, f32_eps, metric), f32_eps, metric);
      }
    }
    if (threadIdx.x == 0) {
      thr[q] = t;
      cand_cnt[q] = 0;
    }
    __syncthreads();  // the histogram is reused by the block's next row
  }
}

__global__ void dense_emit_items_kernel(const int* __restrict__ n_dev, int64_t x_rows, int xspan,
                                        int nsplit, int max_items, EmitItem* __restrict__ items,
                                        int* __restrict__ num_items) {
  const int n = *n_dev;
  const int nchunk = (n + TQ - 1) / TQ;
  const int total = min(nchunk * nsplit, max_items);
  if (blockIdx.x == 0 && threadIdx.x == 0) *num_items = total;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += gridDim.x * blockDim.x) {
    const int c = i / nsplit, sp = i - c * nsplit;
    const int64_t xb = (int64_t)sp * xspan;
    const int64_t xe = xb + xspan < x_rows ? xb + xspan : x_rows;
    items[i] = EmitItem{c * TQ, min(TQ, n - c * TQ), (int)xb, (int)xe, -1};
  }
}

// The overflowing queries of the windowed select, rows[0 .. *n): up to lim of
// them take the dense re-emission pass (*n_dense = *n); more than lim (data
// whose points tie within the rounding slack by the thousand, where a dense
// pass would overflow again) go straight on to the exact finish: *n_dense =
// 0, rest = rows, *rest_n = *n.
__global__ void overflow_split_kernel(const int* __restrict__ rows, const int* __restrict__ n_dev,
                                      int lim, int* __restrict__ n_dense, int* __restrict__ rest,
                                      int* __restrict__ rest_n) {
  const int n = *n_dev;
  const bool dense = n <= lim;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *n_dense = dense ? n : 0;
    if (!dense) *rest_n = n;
  }
  if (dense) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    rest[i] = rows[i];
}

// Hit arena -> per-query candidate buffers.
__global__ void scatter_hits_kernel(const int4* __restrict__ arena, int arena_seg,
                                    const int* __restrict__ arena_cnt, int64_t nseg,
                                    float* __restrict__ cand_score, int* __restrict__ cand_row,
                                    int* __restrict__ cand_cnt, int cap) {
  // one warp per slice, its lanes over the slice's records
  const int64_t seg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (seg >= nseg) return;
  const int n = arena_cnt[seg];
  const int4* a = arena + seg * arena_seg;
  for (int i = lane; i < n; i += 32) {
    const int4 h = a[i];
    const int pos = atomicAdd(&cand_cnt[h.x], 1);
    if (pos < cap) {
      cand_score[(int64_t)h.x * cap + pos] = __int_as_float(h.z);
      cand_row[(int64_t)h.x * cap + pos] = h.y;
    }
  }
}

// Score threshold of every query: no point within g(q) of q scores above it.
__global__ void score_threshold_kernel(const float* __restrict__ g, const float* __restrict__ qnorm,
                                       const float* __restrict__ qerr,
                                       const unsigned* __restrict__ lp_max, int d, int64_t m,
                                       float* __restrict__ thr, float f32_eps, int metric) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  thr[q] = qnorm ? score_bound(g[q], qnorm[q], qerr[q], __uint_as_float(lp_max[0]),
                               __uint_as_float(lp_max[1]), d)
                 : f32_score_bound(g[q], f32_eps, metric);
}

}  // namespace

// Warps take chunks of OP_CHUNK consecutive pairs (balanced however the
// pairs spread over the lists), eight pairs per round (a group of eight
// lanes per pair, two pairs per group, lane c holding elements
// 8 c + 64 kb .. + 7 of every 64); a pair's
// representative is the last r whose bins start at or before it, found by a
// binary search at the chunk's start and advanced from there.
constexpr int OP_CHUNK = 256;
__global__ void __launch_bounds__(256)
offset_pair_rows_kernel(const int2* __restrict__ pairs, int npairs, const int* __restrict__ bin_off,
                        int nb, int n_r, const float* __restrict__ Q32,
                        const float* __restrict__ R32, const float* __restrict__ psi,
                        const float* __restrict__ yerr, const float* __restrict__ g, int d, int dpad,
                        uint4* __restrict__ a_rows, float* __restrict__ row_t,
                        float* __restrict__ row_n, unsigned* __restrict__ eps_bits) {
  const int lane = threadIdx.x & 31, c = lane & 7;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int kbs = dpad / 64;
  for (int c0 = gw * OP_CHUNK; c0 < npairs; c0 += nw * OP_CHUNK) {
    const int c1 = min(npairs, c0 + OP_CHUNK);
    // the last r with bin_off[r nb] <= c0 (r < n_r; empty lists share starts)
    int lo = 0, hi = n_r - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bin_off[(int64_t)mid * nb] <= c0) lo = mid;
      else hi = mid - 1;
    }
    int r = lo;
    // two pairs per group and round (i and i + 4), their loads issued together
    for (int i0 = c0; i0 < c1; i0 += 8) {
      int ii[2], rr_[2];
      bool live[2];
      int2 pr[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        ii[u] = i0 + 4 * u + (lane >> 3);
        live[u] = ii[u] < c1;
        while (live[u] && r + 1 < n_r && bin_off[(int64_t)(r + 1) * nb] <= ii[u]) ++r;
        rr_[u] = r;
        pr[u] = pairs[live[u] ? ii[u] : c0];
      }
      float n2[2] = {0.0f, 0.0f}, e2[2] = {0.0f, 0.0f};
      for (int kb = 0; kb < kbs; ++kb) {
        const int j0 = kb * 64 + 8 * c;
        float4 qv[2][2], rv[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int jj = j0 < d ? j0 : 0;  // elements past d are not used
          const float* qr = Q32 + (int64_t)pr[u].x * d + jj;
          const float* rr = R32 + (int64_t)rr_[u] * d + jj;
          qv[u][0] = *reinterpret_cast<const float4*>(qr);
          qv[u][1] = *reinterpret_cast<const float4*>(qr + 4);
          rv[u][0] = *reinterpret_cast<const float4*>(rr);
          rv[u][1] = *reinterpret_cast<const float4*>(rr + 4);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          uint4 w = make_uint4(0u, 0u, 0u, 0u);
          if (j0 < d) {
            const float4 q0 = qv[u][0], q1 = qv[u][1], r0 = rv[u][0], r1 = rv[u][1];
            const float a[8] = {q0.x - r0.x, q0.y - r0.y, q0.z - r0.z, q0.w - r0.w,
                                q1.x - r1.x, q1.y - r1.y, q1.z - r1.z, q1.w - r1.w};
            uint32_t ww[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const __nv_bfloat162 bb = __floats2bfloat162_rn(a[2 * h], a[2 * h + 1]);
              ww[h] = (uint32_t)__bfloat16_as_ushort(bb.x) | ((uint32_t)__bfloat16_as_ushort(bb.y) << 16);
              const float flo = __uint_as_float(ww[h] << 16), fhi = __uint_as_float(ww[h] & 0xffff0000u);
              n2[u] = fmaf(fhi, fhi, fmaf(flo, flo, n2[u]));
              const float d0 = a[2 * h] - flo, d1 = a[2 * h + 1] - fhi;  // exact
              e2[u] = fmaf(d1, d1, fmaf(d0, d0, e2[u]));
            }
            w = make_uint4(ww[0], ww[1], ww[2], ww[3]);
          }
          if (live[u]) a_rows[((int64_t)ii[u] * dpad + kb * 64 + 8 * c) / 8] = w;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          n2[u] += __shfl_xor_sync(0xffffffffu, n2[u], o);
          e2[u] += __shfl_xor_sync(0xffffffffu, e2[u], o);
        }
        if (live[u] && c == 0) {
          const float M = off_pair_m(__int_as_float(pr[u].y), psi[rr_[u]]);
          const float ea = __fsqrt_ru(e2[u] * (1.0f + 3.0517578e-05f)) * (1.0f + 2.4e-7f);
          const float eps = (ea + yerr[rr_[u]] + 1.1920929e-07f * M) * (1.0f + 2.4e-7f);
          const float T = off_value_bound(g[pr[u].x], M, eps, d);
          row_n[ii[u]] = n2[u];
          row_t[ii[u]] = T < INFINITY ? 0.5f * (n2[u] - T) - 2.4e-7f * (n2[u] + T) - 1e-30f
                                      : -INFINITY;
          atomicMax(eps_bits + pr[u].x, __float_as_uint(eps));
        }
      }
    }
  }
}

int launch_offset_pair_rows(const int2* pairs, int npairs, const int* bin_off, int nb, int n_r,
                            const float* Q32, const float* R32, const float* psi,
                            const float* yerr, const float* g, int d, int dpad, void* a_rows,
                            float* row_t, float* row_n, unsigned* eps_bits, int sms,
                            cudaStream_t st) {
  if (npairs <= 0 || n_r <= 0) return RBC_OK;
  if (d % 8 != 0 || dpad % 64 != 0 || d > dpad) {
    set_error("offset rows: d %d must be a multiple of 8 within dpad %d", d, dpad);
    return RBC_ERR_ARG;
  }
  const int chunks = (npairs + OP_CHUNK - 1) / OP_CHUNK;
  const int grid = std::max(1, std::min((chunks + 7) / 8, sms * 8));
  offset_pair_rows_kernel<<<grid, 256, 0, st>>>(pairs, npairs, bin_off, nb, n_r, Q32, R32, psi,
                                                yerr, g, d, dpad, static_cast<uint4*>(a_rows),
                                                row_t, row_n, eps_bits);
  RBC_LAUNCH_CHECK("offset_pair_rows_kernel");
  return RBC_OK;
}

int launch_gbound(const float* own, const float* gk, int64_t m, float rel_rep, float* g,
                  cudaStream_t st) {
  if (m <= 0) return RBC_OK;
  gbound_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(own, gk, m, rel_rep, g);
  RBC_LAUNCH_CHECK("gbound_kernel");
  return RBC_OK;
}

int launch_own_kth_lp(const float* ps, const int* pi, int C, const int* qsrc, int64_t rows,
                      int k, const float* Q32, const float* X32, int d, int metric, float rel,
                      float* own, cudaStream_t st) {
  if (rows <= 0) return RBC_OK;
  own_kth_lp_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(
      ps, pi, C, qsrc, rows, k, Q32, X32, d, metric, rel, own);
  RBC_LAUNCH_CHECK("own_kth_lp_kernel");
  return RBC_OK;
}

int64_t window_pair_blocks(int64_t m) { return (m + WW * WT - 1) / (WW * WT); }

int launch_window_pairs_count(const float* D, int64_t m, int n_r, const float* g,
                              const float* g1, const float* psi_plus, float rel, int* totals,
                              int* bin_off, int* blk_off, unsigned long long* kept_sum,
                              cudaStream_t st, int* scan_scratch, unsigned* mq_bits) {
  const int64_t nbins = (int64_t)n_r * NBK;
  const int64_t qblocks = window_pair_blocks(m);
  RBC_CUDA(cudaMemsetAsync(totals, 0, nbins * sizeof(int), st));
  if (qblocks > 0) {
    const dim3 grid((unsigned)qblocks, (n_r + RSPAN - 1) / RSPAN);
    wpairs_kernel<false><<<grid, WW * 32, 0, st>>>(D, m, n_r, g, g1, psi_plus, rel, totals,
                                                   nullptr, blk_off, nullptr, kept_sum, mq_bits);
    RBC_LAUNCH_CHECK("wpairs_kernel");
  }
  return launch_exclusive_scan(totals, (int)nbins, bin_off, st, scan_scratch);
}

int64_t window_block_offsets(int64_t m, int n_r) {
  return window_pair_blocks(m) * ((n_r + RSPAN - 1) / RSPAN) * RSPAN * NBK;
}

int launch_window_pairs_scatter(const float* D, int64_t m, int n_r, const float* g,
                                const float* g1, const float* psi_plus, float rel,
                                const int* bin_off, int* blk_off, int2* pairs, cudaStream_t st) {
  const int64_t qblocks = window_pair_blocks(m);
  if (qblocks == 0) return RBC_OK;
  const dim3 grid((unsigned)qblocks, (n_r + RSPAN - 1) / RSPAN);
  wpairs_kernel<true><<<grid, WW * 32, 0, st>>>(D, m, n_r, g, g1, psi_plus, rel, nullptr,
                                                bin_off, blk_off, pairs, nullptr, nullptr);
  RBC_LAUNCH_CHECK("wpairs_kernel");
  return RBC_OK;
}

int window_buckets() { return NBK; }

int launch_window_items(const int* bin_off, int nb, int n_r, const int2* pairs,
                        const float* g, const int* offsets,
                        const float* xdist, float rel, float relx, int* chunk_counts,
                        int* chunk_off, int max_items, EmitItem* items,
                        unsigned long long* stats, cudaStream_t st) {
  chunk_count_kernel<<<(n_r + 255) / 256, 256, 0, st>>>(bin_off, nb, n_r, chunk_counts);
  RBC_LAUNCH_CHECK("chunk_count_kernel");
  int rc = launch_exclusive_scan(chunk_counts, n_r, chunk_off, st);
  if (rc != RBC_OK) return rc;
  if (max_items <= 0) return RBC_OK;
  const int64_t want = ((int64_t)max_items * 32 + 255) / 256;
  window_items_kernel<<<(unsigned)std::min<int64_t>(want, 148 * 16), 256, 0, st>>>(
      chunk_off, n_r, bin_off, nb, pairs, g, offsets, xdist, rel, relx, max_items, items,
      stats);
  RBC_LAUNCH_CHECK("window_items_kernel");
  return RBC_OK;
}

int launch_score_threshold(const float* g, const float* qnorm, const float* qerr,
                           const unsigned* lp_max, int d, int64_t m, float* thr,
                           cudaStream_t st, float f32_eps, int metric) {
  if (m <= 0) return RBC_OK;
  score_threshold_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(g, qnorm, qerr, lp_max, d,
                                                                      m, thr, f32_eps, metric);
  RBC_LAUNCH_CHECK("score_threshold_kernel");
  return RBC_OK;
}

int launch_overflow_rethreshold(const int* rows, const int* n_dev, int64_t max_rows,
                                const float* cand_score, int* cand_cnt, int cap, int k,
                                const float* qnorm, const float* qerr, const unsigned* lp_max,
                                int d, float* thr, cudaStream_t st, float f32_eps, int metric,
                                const unsigned* mq_bits, const unsigned* eps_bits) {
  if (max_rows <= 0) return RBC_OK;
  overflow_rethreshold_kernel<<<(unsigned)std::min<int64_t>(max_rows, 148 * 4), 256, 0, st>>>(
      rows, n_dev, cand_score, cand_cnt, cap, k, qnorm, qerr, lp_max, d, thr, f32_eps, metric,
      mq_bits, eps_bits);
  RBC_LAUNCH_CHECK("overflow_rethreshold_kernel");
  return RBC_OK;
}

int launch_dense_emit_items(const int* n_dev, int64_t x_rows, int xspan, int max_items,
                            EmitItem* items, int* num_items, cudaStream_t st) {
  const int nsplit = (int)((x_rows + xspan - 1) / xspan);
  dense_emit_items_kernel<<<64, 256, 0, st>>>(n_dev, x_rows, xspan, nsplit, max_items, items,
                                              num_items);
  RBC_LAUNCH_CHECK("dense_emit_items_kernel");
  return RBC_OK;
}

int launch_overflow_split(const int* rows, const int* n_dev, int max_rows, int lim, int* n_dense,
                          int* rest, int* rest_n, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(64, ((int64_t)max_rows + 255) / 256 + 1);
  overflow_split_kernel<<<blocks, 256, 0, st>>>(rows, n_dev, lim, n_dense, rest, rest_n);
  RBC_LAUNCH_CHECK("overflow_split_kernel");
  return RBC_OK;
}

int launch_scatter_hits(const int4* arena, int arena_seg, const int* arena_cnt, int nseg,
                        float* cand_score, int* cand_row, int* cand_cnt, int cap,
                        cudaStream_t st) {
  if (nseg <= 0) return RBC_OK;
  scatter_hits_kernel<<<(unsigned)((nseg * 32 + 255) / 256), 256, 0, st>>>(
      arena, arena_seg, arena_cnt, nseg, cand_score, cand_row, cand_cnt, cap);
  RBC_LAUNCH_CHECK("scatter_hits_kernel");
  return RBC_OK;
}

}  // namespace rbc
