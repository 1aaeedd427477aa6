// Index construction and exact-search bookkeeping around the BF calls.
//
// * counting sort   -- forms the ownership lists L_r (Sections 4, 5.2): a
//                      stable counting sort of the points by owner, so each
//                      list is one contiguous run of the permuted database.
// * list radii      -- psi_r = max_{x in L_r} rho(x, r) (Section 4).
// * row stats       -- gamma_1 and gamma_k of every query from its retained
//                      representative distances (Section 5.2).
// * prune           -- the two pruning rules of Section 5.2 (rule (1) with
//                      gamma_k, Lemma 1 generalised to 2 gamma_k + gamma_1),
//                      evaluated with rounding slack so that no surviving
//                      representative is dropped; per query tile the union
//                      of survivors is kept as a bitmask.
// * workgen         -- cuts each tile's union of lists into work items for
//                      the stage-two BF kernel.
#include "common.cuh"
#include "kernels.cuh"

namespace rbc {

namespace {

constexpr int CS_CHUNK = 512;  // keys per counting-sort block

__global__ void cs_hist_kernel(const int64_t* __restrict__ key, int64_t n, int nbins,
                               int* __restrict__ counts) {
  extern __shared__ int h[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * CS_CHUNK;
  for (int i = threadIdx.x; i < CS_CHUNK; i += blockDim.x) {
    int64_t j = base + i;
    if (j < n) atomicAdd(&h[(int)key[j]], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    counts[(int64_t)blockIdx.x * nbins + b] = h[b];
}

// per bin (one warp, lanes over 32 blocks at a time): exclusive prefix over
// blocks in place; totals[bin] = sum
__global__ void cs_colscan_kernel(int* __restrict__ counts, int nblocks, int nbins,
                                  int* __restrict__ totals) {
  const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nbins) return;
  int carry = 0;
  for (int k0 = 0; k0 < nblocks; k0 += 32) {
    const int k = k0 + lane;
    const int64_t o = (int64_t)k * nbins + b;
    const int v = k < nblocks ? counts[o] : 0;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (k < nblocks) counts[o] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) totals[b] = carry;
}

// single block exclusive scan of n ints: out[i] = sum_{j<i} in[j], out[n] = total
__global__ void exclusive_scan_kernel(const int* __restrict__ in, int n, int* __restrict__ out) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    int warp_off = wid ? warp_sums[wid - 1] : 0;
    if (i < n) out[i] = carry + warp_off + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// Two-level exclusive scan for long arrays: per tile of SCAN_TILE elements a
// sum, a scan of the sums (the single-block kernel), then each tile scanned
// from its offset.  out[n] = total.
constexpr int SCAN_TILE = 4096;
__global__ void scan_tile_sums_kernel(const int* __restrict__ in, int n, int* __restrict__ sums) {
  __shared__ int part[32];
  const int base = blockIdx.x * SCAN_TILE;
  int s = 0;
  for (int i = base + threadIdx.x; i < min(n, base + SCAN_TILE); i += blockDim.x) s += in[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < (int)(blockDim.x >> 5) ? part[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}
__global__ void scan_tiles_kernel(const int* __restrict__ in, int n, const int* __restrict__ off,
                                  int* __restrict__ out) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  const int base = blockIdx.x * SCAN_TILE;
  const int end = min(n, base + SCAN_TILE);
  if (threadIdx.x == 0) carry = off[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b0 = base; b0 < end; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const int v = i < end ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const int warp_off = wid ? warp_sums[wid - 1] : 0;
    if (i < end) out[i] = carry + warp_off + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = off[gridDim.x];
}

// one warp per block walks its chunk in order; equal keys within a group of
// 32 are ranked by lane, so the scatter is stable
__global__ void cs_scatter_kernel(const int64_t* __restrict__ key, int64_t n, int nbins,
                                  const int* __restrict__ counts, const int* __restrict__ offsets,
                                  int* __restrict__ perm) {
  extern __shared__ int run[];
  const int lane = threadIdx.x;
  for (int b = lane; b < nbins; b += 32)
    run[b] = offsets[b] + counts[(int64_t)blockIdx.x * nbins + b];
  __syncwarp();
  int64_t base = (int64_t)blockIdx.x * CS_CHUNK;
  for (int g = 0; g < CS_CHUNK; g += 32) {
    int64_t j = base + g + lane;
    bool act = j < n;
    unsigned active = __ballot_sync(0xffffffffu, act);
    if (!active) break;
    int kv = act ? (int)key[j] : -1 - lane;  // inactive lanes get unique dummy keys
    unsigned same = __match_any_sync(0xffffffffu, kv);
    int rank = __popc(same & ((1u << lane) - 1u));
    int pos = act ? run[kv] + rank : 0;
    __syncwarp();
    if (act) {
      perm[pos] = (int)j;
      if (rank == 0) run[kv] += __popc(same);
    }
    __syncwarp();
  }
}

__global__ void list_radii_kernel(const float* __restrict__ dist_by_id, const int* __restrict__ perm,
                                  const int* __restrict__ offsets, int n_r, float rel,
                                  float* __restrict__ psi_plus) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_r) return;
  float mx = 0.f;
  for (int p = offsets[w] + lane; p < offsets[w + 1]; p += 32) mx = fmaxf(mx, dist_by_id[perm[p]]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) psi_plus[w] = mx * (1.0f + rel);
}

// One warp per query row of D (distances >= 0, so their bit patterns order
// like their values): gamma_1 and the nearest column by a warp arg-min
// (ties to the smaller column); gamma_k, the k-th smallest value.  Rows of up
// to 2048 values are held in registers, 32 or 64 per lane, and gamma_k is found in
// two short selections: T = the k-th smallest of the 32 lane minima bounds
// gamma_k from above (k lanes hold a value <= T), the values <= T (normally
// a few more than k) are compacted one per lane, and k rounds of a warp
// minimum over them give gamma_k exactly.  Rows with more than 32 values <= T,
// and longer rows, use a bitwise search for the k-th smallest bit pattern.
template <int VPL>  // values per lane held in registers (0: none)
__global__ void row_stats_kernel(const float* __restrict__ D, int64_t m, int n_r, int k,
                                 float* __restrict__ g1, float* __restrict__ gk,
                                 int64_t* __restrict__ nearest) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const float* row = D + w * n_r;
  constexpr bool CACHED = VPL > 0;
  unsigned vals[CACHED ? VPL : 1];
  float bv = INFINITY;
  int bi = INT32_MAX;
  if (CACHED) {
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
      const int c = lane + 32 * j;
      const float v = c < n_r ? row[c] : INFINITY;
      vals[j] = __float_as_uint(v);
      if (v < bv) {
        bv = v;
        bi = c;
      }
    }
  } else {
    for (int c = lane; c < n_r; c += 32) {
      const float v = row[c];
      if (v < bv) {
        bv = v;
        bi = c;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov < bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  float kth = INFINITY;
  bool done = false;
  if constexpr (CACHED) {
  if (k <= n_r && k <= 32) {
    // the k-th smallest of {vals[j] ... } by k rounds of a warp minimum over
    // one value per lane (x); the lane holding the minimum drops it
    auto kth_of_lanes = [&](unsigned x) {
      unsigned res = 0xffffffffu;
      for (int r = 0; r < k; ++r) {
        unsigned mn = x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        res = mn;
        const unsigned holders = __ballot_sync(0xffffffffu, x == mn);
        if (lane == __ffs(holders) - 1) x = 0xffffffffu;
      }
      return res;
    };
    unsigned lmin = vals[0];
#pragma unroll
    for (int j = 1; j < VPL; ++j) lmin = min(lmin, vals[j]);
    const unsigned T = kth_of_lanes(lmin);
    int c = 0;
#pragma unroll
    for (int j = 0; j < VPL; ++j) c += vals[j] <= T;
    int pre = c;  // inclusive prefix over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += t;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    if (total <= 32) {
      __shared__ unsigned cand[8][32];  // one slot row per warp of the block
      unsigned* cw = cand[(threadIdx.x >> 5) & 7];
      int pos = pre - c;
#pragma unroll
      for (int j = 0; j < VPL; ++j)
        if (vals[j] <= T) cw[pos++] = vals[j];
      __syncwarp();
      const unsigned x = lane < total ? cw[lane] : 0xffffffffu;
      kth = __uint_as_float(kth_of_lanes(x));
      done = true;
    }
  }
  }
  if (!done && k <= n_r) {
    unsigned res = 0;
    for (int bit = 31; bit >= 0; --bit) {
      const unsigned t = res | (1u << bit);
      int cnt = 0;
      if (CACHED) {
#pragma unroll
        for (int j = 0; j < VPL; ++j) cnt += vals[j] < t;
      } else {
        for (int c = lane; c < n_r; c += 32) cnt += __float_as_uint(row[c]) < t;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      if (cnt < k) res = t;
    }
    kth = __uint_as_float(res);
  }
  if (lane == 0) {
    g1[w] = bv;
    gk[w] = kth;
    nearest[w] = bi;
  }
}

constexpr int PRUNE_WARPS = 8;

__global__ void __launch_bounds__(PRUNE_WARPS * 32)
prune_kernel(const float* __restrict__ D, const int* __restrict__ qperm, int64_t m, int n_r,
             const float* __restrict__ g1, const float* __restrict__ gk,
             const float* __restrict__ psi_plus, const int* __restrict__ offsets, float rel,
             uint32_t* __restrict__ tile_mask, int64_t* __restrict__ tile_points,
             int* __restrict__ q_kept) {
  extern __shared__ uint32_t mask[];
  const int words = (n_r + 31) / 32;
  const int tile = blockIdx.x;
  for (int i = threadIdx.x; i < words; i += blockDim.x) mask[i] = 0;
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float up = 1.0f + rel, lo = 1.0f - rel, slack = 1.0f + 2.4e-7f;
  for (int r = wid; r < TQ; r += PRUNE_WARPS) {
    int64_t pos = (int64_t)tile * TQ + r;
    if (pos >= m) break;
    int q = qperm ? qperm[pos] : (int)pos;
    float gkh = gk[q] * up, g1h = g1[q] * up;
    float lemma = (2.0f * gkh + g1h) * slack;
    const float* row = D + (int64_t)q * n_r;
    int kept = 0;
    for (int c0 = 0; c0 < n_r; c0 += 32) {
      int c = c0 + lane;
      bool keep = false;
      if (c < n_r) {
        float dl = row[c] * lo;
        keep = dl <= (gkh + psi_plus[c]) * slack && dl <= lemma;
      }
      unsigned bits = __ballot_sync(0xffffffffu, keep);
      kept += __popc(bits);
      if (lane == 0 && bits) atomicOr(&mask[c0 >> 5], bits);
    }
    if (lane == 0 && q_kept) q_kept[q] = kept;
  }
  __syncthreads();
  // tile point count = sum of kept list sizes
  long long pts = 0;
  for (int r = threadIdx.x; r < n_r; r += blockDim.x)
    if (mask[r >> 5] & (1u << (r & 31))) pts += offsets[r + 1] - offsets[r];
  for (int o = 16; o > 0; o >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o);
  __shared__ long long part[PRUNE_WARPS];
  if (lane == 0) part[wid] = pts;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int i = 0; i < PRUNE_WARPS; ++i) s += part[i];
    tile_points[tile] = s;
  }
  for (int i = threadIdx.x; i < words; i += blockDim.x)
    tile_mask[(int64_t)tile * words + i] = mask[i];
}

__global__ void item_count_kernel(const int64_t* __restrict__ tile_points, int tiles, int W,
                                  int* __restrict__ counts) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < tiles) counts[t] = (int)((tile_points[t] + W - 1) / W);
}

// one thread per tile: walk the kept representatives in order, merge adjacent
// lists into runs, cut runs so that every item holds at most W points
__global__ void workgen_kernel(const uint32_t* __restrict__ tile_mask, const int* __restrict__ offsets,
                               int n_r, int64_t m, int W, int item_cap, int seg_cap,
                               const int* __restrict__ tile_item_off, WorkItem* __restrict__ items,
                               Seg* __restrict__ segs, uint32_t* dev_err) {
  const int tiles = (int)((m + TQ - 1) / TQ);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tiles) return;
  const int words = (n_r + 31) / 32;
  const uint32_t* mk = tile_mask + (int64_t)t * words;
  const int q0 = t * TQ;
  const int nq = (int)min((int64_t)TQ, m - q0);
  int item = tile_item_off[t];
  const int item_end = tile_item_off[t + 1];
  if (item_end - item > item_cap) {
    atomicOr(dev_err, DEV_ERR_CAPACITY);
    return;
  }
  const int seg0 = t * seg_cap;
  int seg = seg0;
  int acc = 0;          // points in the open item
  int item_seg0 = seg;  // first segment of the open item
  auto close_item = [&]() {
    if (item < item_end) items[item] = WorkItem{q0, nq, item_seg0, seg, item, t};
    ++item;
    item_seg0 = seg;
    acc = 0;
  };
  for (int r = 0; r < n_r; ++r) {
    if (!(mk[r >> 5] & (1u << (r & 31)))) continue;
    int b = offsets[r], e = offsets[r + 1];
    while (b < e) {
      int take = min(e - b, W - acc);
      if (seg > item_seg0 && segs[seg - 1].x_end == b) {
        segs[seg - 1].x_end = b + take;  // extend the previous run
      } else {
        if (seg - seg0 >= seg_cap) {
          atomicOr(dev_err, DEV_ERR_CAPACITY);
          return;
        }
        segs[seg++] = Seg{b, b + take};
      }
      acc += take;
      b += take;
      if (acc == W) close_item();
    }
  }
  if (acc > 0) close_item();
}

__global__ void sum_i32_kernel(const int* __restrict__ v, int64_t n, unsigned long long* out) {
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void sum_i64_kernel(const int64_t* __restrict__ v, int64_t n, unsigned long long* out) {
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void sum_pairs_kernel(const int64_t* __restrict__ tpts, int64_t m,
                                 unsigned long long* out) {
  const int64_t tiles = (m + TQ - 1) / TQ;
  unsigned long long s = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles;
       t += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)tpts[t] * (unsigned long long)min((int64_t)TQ, m - t * TQ);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void add_ints_kernel(int* __restrict__ dst, const int* __restrict__ src, int n) {
  int i = threadIdx.x;
  if (i < n) dst[i] += src[i];
}

// ---- lists ordered by distance to their representative ----
__global__ void iota_kernel(int* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int)i;
}

// key[j] = 8-bit digit of the float bit pattern of val[cur[j]] (values >= 0,
// so bit patterns order like the values)
__global__ void digit_key_kernel(const float* __restrict__ val, const int* __restrict__ cur,
                                 int64_t n, int shift, int64_t* __restrict__ key) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    key[j] = (__float_as_uint(val[cur[j]]) >> shift) & 255u;
}

__global__ void owner_key_kernel(const int64_t* __restrict__ owner, const int* __restrict__ cur,
                                 int64_t n, int64_t* __restrict__ key) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    key[j] = owner[cur[j]];
}

// out[pos] = cur[perm[pos]]
__global__ void compose_kernel(const int* __restrict__ cur, const int* __restrict__ perm,
                               int64_t n, int* __restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = cur[perm[j]];
}

__global__ void gather_f32_kernel(const float* __restrict__ val, const int* __restrict__ idx,
                                  int64_t n, float* __restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = val[idx[j]];
}

}  // namespace

int exclusive_scan_scratch_ints(int n) { return 2 * ((n + SCAN_TILE - 1) / SCAN_TILE) + 2; }

int launch_exclusive_scan(const int* in, int n, int* out, cudaStream_t st, int* scratch) {
  if (!scratch || n <= 2 * SCAN_TILE) {
    exclusive_scan_kernel<<<1, 1024, 0, st>>>(in, n, out);
    RBC_LAUNCH_CHECK("exclusive_scan_kernel");
    return RBC_OK;
  }
  const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  int* sums = scratch;
  int* off = scratch + nb + 1;
  scan_tile_sums_kernel<<<nb, 1024, 0, st>>>(in, n, sums);
  RBC_LAUNCH_CHECK("scan_tile_sums_kernel");
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(sums, nb, off);
  RBC_LAUNCH_CHECK("exclusive_scan_kernel");
  scan_tiles_kernel<<<nb, 1024, 0, st>>>(in, n, off, out);
  RBC_LAUNCH_CHECK("scan_tiles_kernel");
  return RBC_OK;
}

__global__ void or_flags_kernel(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src) {
  if (threadIdx.x == 0 && *src) atomicOr(dst, *src);
}

int launch_or_flags(uint32_t* dst, const uint32_t* src, cudaStream_t st) {
  or_flags_kernel<<<1, 32, 0, st>>>(dst, src);
  RBC_LAUNCH_CHECK("or_flags_kernel");
  return RBC_OK;
}

int launch_add_ints(int* dst, const int* src, int n, cudaStream_t st) {
  add_ints_kernel<<<1, 32, 0, st>>>(dst, src, n);
  RBC_LAUNCH_CHECK("add_ints_kernel");
  return RBC_OK;
}

int launch_sum_pairs(const int64_t* tile_points, int64_t m, unsigned long long* out,
                     cudaStream_t st) {
  if (m <= 0) return RBC_OK;
  sum_pairs_kernel<<<16, 256, 0, st>>>(tile_points, m, out);
  RBC_LAUNCH_CHECK("sum_pairs_kernel");
  return RBC_OK;
}

int64_t counting_sort_scratch_ints(int64_t n, int nbins) {
  int64_t blocks = (n + CS_CHUNK - 1) / CS_CHUNK;
  return blocks * nbins + nbins + 1;
}

int launch_counting_sort(const int64_t* key, int64_t n, int nbins, int* perm, int* offsets,
                         int* scratch, cudaStream_t st) {
  if (nbins > 12000) {
    set_error("counting sort: %d bins exceed the shared-memory histogram", nbins);
    return RBC_ERR_UNSUPPORTED;
  }
  int blocks = (int)((n + CS_CHUNK - 1) / CS_CHUNK);
  int* counts = scratch;
  int* totals = scratch + (int64_t)blocks * nbins;
  if (blocks > 0) {
    cs_hist_kernel<<<blocks, 256, nbins * sizeof(int), st>>>(key, n, nbins, counts);
    RBC_LAUNCH_CHECK("cs_hist_kernel");
    cs_colscan_kernel<<<(unsigned)(((int64_t)nbins * 32 + 255) / 256), 256, 0, st>>>(
        counts, blocks, nbins, totals);
    RBC_LAUNCH_CHECK("cs_colscan_kernel");
  } else {
    RBC_CUDA(cudaMemsetAsync(totals, 0, nbins * sizeof(int), st));
  }
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(totals, nbins, offsets);
  RBC_LAUNCH_CHECK("exclusive_scan_kernel");
  if (blocks > 0) {
    cs_scatter_kernel<<<blocks, 32, nbins * sizeof(int), st>>>(key, n, nbins, counts, offsets,
                                                                perm);
    RBC_LAUNCH_CHECK("cs_scatter_kernel");
  }
  return RBC_OK;
}

int64_t sort_lists_scratch_ints(int64_t n, int n_r) {
  // three permutations, 64-bit keys (8-byte aligned), counting-sort scratch,
  // digit offsets
  return 5 * n + 2 + counting_sort_scratch_ints(n, n_r > 256 ? n_r : 256) + 257;
}

int launch_sort_lists(const int64_t* owner, const float* dist, int64_t n, int n_r, int* members,
                      int* offsets, float* xdist, int* scratch, cudaStream_t st) {
  if (n <= 0) return RBC_OK;
  int* cur = scratch;
  int* tmp = scratch + n;
  int* perm = scratch + 2 * n;
  // the keys start at an even int offset: 8-byte aligned for any n
  const int64_t key_off = (3 * n + 1) & ~(int64_t)1;
  int64_t* key = reinterpret_cast<int64_t*>(scratch + key_off);
  int* cs = scratch + key_off + 2 * n;
  int* digit_off = cs + counting_sort_scratch_ints(n, n_r > 256 ? n_r : 256);
  const unsigned g = (unsigned)((n + 255) / 256 < 148 * 16 ? (n + 255) / 256 : 148 * 16);
  iota_kernel<<<g, 256, 0, st>>>(cur, n);
  RBC_LAUNCH_CHECK("iota_kernel");
  // least significant digit first; every pass is stable, so equal distances
  // keep ascending ids
  for (int shift = 0; shift < 32; shift += 8) {
    digit_key_kernel<<<g, 256, 0, st>>>(dist, cur, n, shift, key);
    RBC_LAUNCH_CHECK("digit_key_kernel");
    int rc = launch_counting_sort(key, n, 256, perm, digit_off, cs, st);
    if (rc != RBC_OK) return rc;
    compose_kernel<<<g, 256, 0, st>>>(cur, perm, n, tmp);
    RBC_LAUNCH_CHECK("compose_kernel");
    int* t = cur;
    cur = tmp;
    tmp = t;
  }
  // finally by owner (stable): lists in owner order, each by (distance, id)
  owner_key_kernel<<<g, 256, 0, st>>>(owner, cur, n, key);
  RBC_LAUNCH_CHECK("owner_key_kernel");
  int rc = launch_counting_sort(key, n, n_r, perm, offsets, cs, st);
  if (rc != RBC_OK) return rc;
  compose_kernel<<<g, 256, 0, st>>>(cur, perm, n, members);
  RBC_LAUNCH_CHECK("compose_kernel");
  gather_f32_kernel<<<g, 256, 0, st>>>(dist, members, n, xdist);
  RBC_LAUNCH_CHECK("gather_f32_kernel");
  return RBC_OK;
}

int launch_list_radii(const float* dist_by_id, const int* perm, const int* offsets, int n_r,
                      float rel, float* psi_plus, cudaStream_t st) {
  list_radii_kernel<<<(n_r * 32 + 255) / 256, 256, 0, st>>>(dist_by_id, perm, offsets, n_r, rel,
                                                           psi_plus);
  RBC_LAUNCH_CHECK("list_radii_kernel");
  return RBC_OK;
}

int launch_row_stats(const float* D, int64_t m, int n_r, int k, float* g1, float* gk,
                     int64_t* nearest, cudaStream_t st) {
  if (m <= 0) return RBC_OK;
  const unsigned blocks = (unsigned)((m * 32 + 255) / 256);
  if (n_r <= 1024)
    row_stats_kernel<32><<<blocks, 256, 0, st>>>(D, m, n_r, k, g1, gk, nearest);
  else if (n_r <= 2048)
    row_stats_kernel<64><<<blocks, 256, 0, st>>>(D, m, n_r, k, g1, gk, nearest);
  else
    row_stats_kernel<0><<<blocks, 256, 0, st>>>(D, m, n_r, k, g1, gk, nearest);
  RBC_LAUNCH_CHECK("row_stats_kernel");
  return RBC_OK;
}

int launch_prune(const float* D, const int* qperm, int64_t m, int n_r, const float* g1,
                 const float* gk, const float* psi_plus, const int* offsets, float rel,
                 uint32_t* tile_mask, int64_t* tile_points, int* q_kept, cudaStream_t st) {
  int tiles = (int)((m + TQ - 1) / TQ);
  if (tiles == 0) return RBC_OK;
  int words = (n_r + 31) / 32;
  prune_kernel<<<tiles, PRUNE_WARPS * 32, words * sizeof(uint32_t), st>>>(
      D, qperm, m, n_r, g1, gk, psi_plus, offsets, rel, tile_mask, tile_points, q_kept);
  RBC_LAUNCH_CHECK("prune_kernel");
  return RBC_OK;
}

int launch_item_offsets(const int64_t* tile_points, int tiles, int W, int* counts_scratch,
                        int* tile_item_off, cudaStream_t st) {
  if (tiles == 0) return RBC_OK;
  item_count_kernel<<<(tiles + 255) / 256, 256, 0, st>>>(tile_points, tiles, W, counts_scratch);
  RBC_LAUNCH_CHECK("item_count_kernel");
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(counts_scratch, tiles, tile_item_off);
  RBC_LAUNCH_CHECK("exclusive_scan_kernel");
  return RBC_OK;
}

int launch_workgen_items(const uint32_t* tile_mask, const int* offsets, int n_r, int64_t m, int W,
                         int item_cap_per_tile, int seg_cap_per_tile, const int* tile_item_off,
                         WorkItem* items, Seg* segs, uint32_t* dev_err, cudaStream_t st) {
  int tiles = (int)((m + TQ - 1) / TQ);
  if (tiles == 0) return RBC_OK;
  workgen_kernel<<<(tiles + 127) / 128, 128, 0, st>>>(tile_mask, offsets, n_r, m, W,
                                                       item_cap_per_tile, seg_cap_per_tile,
                                                       tile_item_off, items, segs, dev_err);
  RBC_LAUNCH_CHECK("workgen_kernel");
  return RBC_OK;
}

int launch_sum_i32(const int* v, int64_t n, unsigned long long* out, cudaStream_t st) {
  if (n <= 0) return RBC_OK;
  sum_i32_kernel<<<64, 256, 0, st>>>(v, n, out);
  RBC_LAUNCH_CHECK("sum_i32_kernel");
  return RBC_OK;
}

int launch_sum_i64(const int64_t* v, int64_t n, unsigned long long* out, cudaStream_t st) {
  if (n <= 0) return RBC_OK;
  sum_i64_kernel<<<64, 256, 0, st>>>(v, n, out);
  RBC_LAUNCH_CHECK("sum_i64_kernel");
  return RBC_OK;
}

}  // namespace rbc
