// Launch interfaces shared by the host orchestration and the kernel files.
#pragma once

#include "common.cuh"

namespace rbc {

constexpr int MAX_D = 256;       // largest supported dimension
constexpr int SIMT_MAX_D = 256;  // FP32 tile kernel limit (query tile in shared memory)
constexpr int MAX_C = 32;        // largest candidate list per query

// Where a tile kernel finds its work.  items == nullptr selects the dense
// form: item = tile * dense_splits + split, query rows [tile*TQ, +TQ) of an
// m-row buffer against database rows [split*dense_chunk, +dense_chunk) of n.
struct TileWork {
  const WorkItem* items;
  const int* num_items_dev;  // list form: device-side item count (or nullptr)
  int num_items;             // dense form / host-known count
  const Seg* segs;           // list form: segment table
  int64_t m;
  int64_t n;
  int dense_splits;
  int64_t dense_chunk;
  // optional (tensor-core kernels, list form): K blocks of 64 columns that
  // item tile t multiplies (the rest of its rows are zero); nullptr = all
  const int8_t* tile_kb = nullptr;
  // tensor-core top-C kernel: every query tile is one item, so CTAs may take
  // items strided (balances runs of large items) instead of in ranges
  bool strided = false;
};

// Per-(slot, query row, sub-list) top-C output of a tile kernel.
struct TopOut {
  float* score;
  int* idx;
  int* slot_valid;  // optional: 0 marks a slot whose list was carried into a later slot
};

int simt_list_width(int c_needed);
int launch_bf_simt_topc(const float* Q, const float* X, int d, int metric, int C,
                        const TileWork& w, const TopOut& out, int grid, cudaStream_t st);
int launch_bf_simt_store(const float* Q, const float* X, int d, int metric, const TileWork& w,
                         float* store, int64_t store_ld, int grid, cudaStream_t st);
// l2 top-C in the expansion form |x|^2 - 2 q.x (one FFMA per dimension), with
// the rows' FP32 squared norms xnorm: scores for the select step's
// expansion-form certificate (SelectArgs::exp32)
int launch_bf_simt_topc_exp(const float* Q, const float* X, const float* xnorm, int d, int C,
                            const TileWork& w, const TopOut& out, int grid, cudaStream_t st);

// ---- low-precision (tensor-core) path ----
struct LpMatrix {
  const void* data;  // [rows, dpad] bf16 / f16 / e4m3, row-major, rows 16-byte aligned
  const float* norm; // [rows] |x~|^2 in FP32
  int64_t rows;
  int dpad;          // elements per row: multiple of 64 (16-bit) or 128 (FP8)
  int storage;       // RBC_BF16 / RBC_F16 / RBC_FP8E4M3
  const void* nblock = nullptr;  // optional [rows, 16] bf16: -|x~|^2 / 2 as (high, low, 0 ...)
  const float* scale = nullptr;  // FP8: [rows] power-of-two scale, x~ = scale * e4m3 row
};

// bytes per stored element of a low-precision row
inline int lp_elem_bytes(int storage) { return storage == RBC_FP8E4M3 ? 1 : 2; }

// columns of a norm block row, and the rows past the end that stay readable
constexpr int NBLOCK_COLS = 16;

bool tc_available();
// Tensor-core BF fused with a per-query top-C: per (slot, query row) two
// sub-lists (column halves) of C entries.  FP8 runs bf_tc.cu; bf16 / fp16 run
// bf_tc_top.cu, which needs Xm.nblock.
int launch_bf_tc_topc(const LpMatrix& Qm, const LpMatrix& Xm, int C, const TileWork& w,
                      const TopOut& out, int grid, cudaStream_t st, uint32_t* dev_err);
// the bf16 / fp16 pass itself: cs entries per (row, column half)
int launch_bf_tc_top(const LpMatrix& Qm, const LpMatrix& Xm, int cs, const TileWork& w,
                     const TopOut& out, int grid, cudaStream_t st, uint32_t* dev_err);

// ---- windowed stage two: per (representative, query chunk) work items ----
// Queries pair_q[pair_begin .. pair_begin + nq) (rows of the query buffer)
// against database rows [x_begin, x_end) of the list-ordered matrix.
struct EmitItem {
  int32_t pair_begin;
  int32_t nq;
  int32_t x_begin;
  int32_t x_end;
  int32_t rep;  // the representative whose list holds the window (-1: any rows)
};

// Candidate emission: every (query, row) pair whose score is <= thr[query]
// is appended to the query's candidate buffer (score, list-ordered row);
// cand_cnt counts every emission, so a count above cap marks an overflow.
struct EmitOut {
  const float* thr;  // [m] score threshold per query
  float* cand_score; // [m, cap]
  int* cand_row;     // [m, cap]
  int* cand_cnt;     // [m]
  int cap;
  // Optional hit arena: CTA b owns arena[b * arena_seg, +arena_seg), split
  // into ARENA_SUBSEG equal parts, one per epilogue warp, and each of those
  // into 32 lane slices; a thread appends (query, row, score bits, 0) records
  // to its slice with a count kept in a register (no atomics), writes the
  // count to arena_cnt[(b * ARENA_SUBSEG + warp) * 32 + lane] and sets
  // *arena_ovf if its slice overflowed (the hits past a full slice are
  // appended to the per-query buffers directly); launch_scatter_hits then
  // fills the per-query buffers.  arena == nullptr: append to them directly.
  int4* arena = nullptr;
  int arena_seg = 0;
  int* arena_cnt = nullptr;
  int* arena_ovf = nullptr;
};
constexpr int ARENA_SUBSEG = 16;  // arena parts per CTA (at least its epilogue warps)
// per-query buffers from the hit arena of an emission pass: `nseg` slices of
// arena_seg records each, counts in arena_cnt[slice]
int launch_scatter_hits(const int4* arena, int arena_seg, const int* arena_cnt, int nseg,
                        float* cand_score, int* cand_row, int* cand_cnt, int cap,
                        cudaStream_t st);
// overflowing rows[0 .. *n_dev) (at most max_rows): *n_dense = *n_dev if it
// is at most lim (they take the dense re-emission pass), else 0, with the
// rows copied to rest and *rest_n = *n_dev (they go to the exact finish)
int launch_overflow_split(const int* rows, const int* n_dev, int max_rows, int lim, int* n_dense,
                          int* rest, int* rest_n, cudaStream_t st);
// the query of an item's row i is pair_q[(pair_begin + i) * pair_stride].
// fold_col >= 0: the database rows carry -|x~|^2 / 2 as a (high, low) pair
// in padding columns fold_col, fold_col + 1 (launch_fold_norm), so no norm
// block or norm MMA is used.
// Representative-offset rows (bf16): Xm holds y~ = bf16(x - r) per list
// row; the query rows of an item are the rows a_rows[pair_begin + i] (one
// per kept pair, launch_offset_pair_rows) with their emission bounds in
// accumulator units row_t and |a~|^2 row_n; a hit's value is the estimate
// |a~|^2 - 2 acc of |a~ - y~|^2.
struct EmitOffsets {
  const uint8_t* a_rows = nullptr;  // [pairs, dpad] bf16, 16-byte aligned
  const float* row_t = nullptr;     // [pairs]
  const float* row_n = nullptr;     // [pairs]
};
int launch_bf_tc_emit(const LpMatrix& Qm, const LpMatrix& Xm, const EmitItem* items,
                      const int* num_items_dev, int max_items, const int* pair_q,
                      int pair_stride, const EmitOut& out, int grid, cudaStream_t st,
                      uint32_t* dev_err, int fold_col = -1, const EmitOffsets* offs = nullptr);

// The same windowed stage two on CUDA cores (FP32 rows, l2 or l1): every
// (query, window row) whose FP32 difference-form value (rho^2 for l2, rho
// for l1) is at most thr[query] is appended to the query's buffer.
int launch_bf_simt_emit(const float* Q, const float* X, int d, int metric, const EmitItem* items,
                        const int* num_items_dev, int max_items, const int* pair_q,
                        int pair_stride, const EmitOut& out, int grid, cudaStream_t st);

// ---- merge + re-rank + certification ----
struct SelectArgs {
  const float* part_score;
  const int* part_idx;
  const int* slot_valid;     // optional: slots with 0 hold no list
  int C;       // entries per sub-list
  int nsub;    // sub-lists per (slot, row)
  const int* tile_slot_off;  // list form: slots of tile t are [off[t], off[t+1])
  int dense_splits;          // dense form: slots of tile t are [t*splits, (t+1)*splits)
  const int* rows;           // optional: buffer rows to process (fallback); else 0..m-1
  const int* num_rows_dev;   // with `rows`: device-side count
  int64_t m;                 // number of query rows (buffer rows) when rows == nullptr
  const float* Q32;          // [m, d] buffer queries FP32
  int d;
  int metric;
  const int* qorig;          // buffer row -> original query index (nullptr = identity;
                             // rows mapped to -1 are padding and skipped)
  const float* X32;          // database buffer rows FP32
  const int* xid;            // buffer row -> original id (nullptr = identity)
  int lp;                    // 1: scores are |x~|^2 - 2 q~.x~ (low precision)
  const float* q_lpnorm;     // [m] |q~|^2 (lp)
  const float* q_err;        // [m] |q - q~| rounded up (lp)
  const unsigned* x_err_max_bits;   // max |x - x~| rounded up, float bits (lp)
  const unsigned* x_norm_max_bits;  // max |x~| rounded up, float bits (lp)
  float simt_eps;            // FP32 path: relative bound of the tile kernel's rho
  int k;
  int c_out;
  int64_t* out_ids;
  float* out_dist;
  int* fallback_rows;        // uncertified rows are appended here (lp)
  int* counters;             // [0] uncertified, [1] fp64 ties, [2] boundary ties
  // optional: per tile (row / TQ) the number of leading columns that can be
  // nonzero (rows of Q32 / X32 stay d apart); sets the re-rank length and its
  // rounding bounds
  const int16_t* tile_dim = nullptr;
  // lp with FP32 expansion-form scores (|x|^2 - 2 q.x on CUDA cores): no
  // rounding residuals (q_err / x_err_max_bits unused), FP32 evaluation bound
  // (d + 4) 2^-23 (|q| + max |x|)^2, q_lpnorm = |q|^2, x_norm_max_bits = max |x|
  int exp32 = 0;
};
int launch_select(const SelectArgs& a, cudaStream_t st);


// Exact finish of uncertified rows (band.cu): for each buffer row rows[i],
// i < *nrows_dev, every point of the row's database range whose FP32
// distance lies within the rounding band of the row's current k-th distance
// (read from out_dist at the row's output row) is evaluated in FP64, and the
// row's output is overwritten with the k smallest (rho64, id).
struct BandArgs {
  const int* rows;
  const int* nrows_dev;
  const float* Q32;          // buffer queries, rows ld floats apart
  const int* qorig;          // buffer row -> output row (nullptr: identity; < 0: skip)
  const float* X32;          // database rows, ld floats apart
  const int* xid;            // row -> database id (nullptr: identity)
  int64_t n;                 // database rows (default range [0, n))
  // optional per-row range, grouped layout: g = tile_grp[row / TQ] ->
  // [grp_base[g], grp_base[g] + grp_len[g])
  const int* tile_grp;
  const int64_t* grp_base;
  const int64_t* grp_len;
  // optional per-row range, one-shot layout: r = tile_list[row / TQ] ->
  // [list_off[r], list_off[r + 1]), or [r list_len, (r + 1) list_len)
  const int* tile_list;
  const int* list_off;
  int list_len;
  int d;                     // columns evaluated
  int ld;                    // row stride of Q32 and X32 (>= d)
  int k;                     // <= 32
  int metric;
  float eps;                 // relative bound of the FP32 re-rank that wrote out_dist
  int64_t* out_ids;
  float* out_dist;
  // optional, per buffer row: an upper bound of the row's true k-th
  // neighbour distance, used instead of the k-th distance in out_dist (rows
  // for which no select step wrote k points)
  const float* kth_bound = nullptr;
  // optional scratch of band_split_scratch_entries() (rho64, id) entries: the
  // first rows of the launch are then scanned in chunks by several CTAs
  double* split_r = nullptr;
  int* split_i = nullptr;
};
int64_t band_split_scratch_entries();
// grid over at most max_rows rows (the count itself is read on the device)
int launch_band(const BandArgs& a, int max_rows, cudaStream_t st);

// rbc_last_stats after bf_search_noalloc: queries / pairs from the host, the
// certification counters read from counters_dev (static scratch) on demand
void stats_publish_static(const int* counters_dev, int64_t queries, int64_t pairs,
                          cudaStream_t st);

// Candidate buffers of the windowed search -> exact k-NN per query.
constexpr int CAND_CAP = 8192;  // candidates per query
struct CandSelectArgs {
  const float* cand_score;  // [m, cap]
  const int* cand_row;      // [m, cap] list-ordered database rows
  const int* cand_cnt;      // [m] emissions (may exceed cap: overflow)
  int cap;
  int64_t m;
  const int* rows;      // optional: the queries to finish; else 0 .. m-1
  const int* nrows_dev; // with rows: device-side count (else nrows)
  int nrows;            // with rows: the count, or the bound of *nrows_dev
  const float* Q32;  // [m, d] queries FP32
  int d;
  int metric;
  const float* q_lpnorm;            // [m] |q~|^2
  const float* q_err;               // [m] |q - q~| rounded up
  const unsigned* x_err_max_bits;   // max |x - x~| rounded up (float bits)
  const unsigned* x_norm_max_bits;  // max |x~| rounded up (float bits)
  const float* X32;  // list-ordered rows FP32
  const int* xid;    // row -> original id
  int k;
  int c_out;
  int64_t* out_ids;  // [m, k]
  float* out_dist;
  int* fallback_rows;  // queries sent to the FP32 re-search are appended here
  int* counters;       // [0] such queries, [1] fp64 ties, [2] boundary ties
  // optional: queries with more survivors than the shared-memory re-rank
  // holds are appended here (count in *stream_count) for launch_select_stream
  // instead of going to the re-search
  int* stream_rows = nullptr;
  int* stream_count = nullptr;
  // representative-offset values (launch_bf_tc_emit with offsets): [m] M and
  // eps of each query as float bits; the survivor bound comes from
  // off_dist_upper
  const unsigned* mq_bits = nullptr;
  const unsigned* eps_bits = nullptr;
  // FP32 candidates (CUDA-core emission): scores are FP32 difference-form
  // values with relative error <= f32_eps; the low-precision fields are unused
  int f32 = 0;
  float f32_eps = 0.0f;
};
int launch_select_cands(const CandSelectArgs& a, cudaStream_t st);
// The queries a.stream_rows[0 .. *a.stream_count) of a launch_select_cands:
// every survivor re-ranked in FP32 in a stream (one warp per query, k + 1
// best kept per lane), FP64 ties, output.  max_rows bounds the count.
int launch_select_stream(const CandSelectArgs& a, int max_rows, cudaStream_t st);


// ---- windowed exact search (window.cu) ----
// g[q] = min(gk[q] (1 + rel_rep) rounded up, own[q]): an upper bound of q's
// k-th nearest-neighbour distance
int launch_gbound(const float* own, const float* gk, int64_t m, float rel_rep, float* g,
                  cudaStream_t st);
// Own-list bound of every grouped query row from the tensor-core top-C lists
// ([tile][TQ][2][C] unsorted low-precision scores and list-ordered rows,
// C <= 32): own[qsrc[row]] = the largest FP32 distance of the row's k
// best-scored rows, rounded up by rel (INF if fewer than k); Q32 holds the
// batch queries, qsrc maps grouped rows to them (-1: padding)
int launch_own_kth_lp(const float* ps, const int* pi, int C, const int* qsrc, int64_t rows,
                      int k, const float* Q32, const float* X32, int d, int metric, float rel,
                      float* own, cudaStream_t st);
// Kept (q, r) pairs binned by (r, bucket of the window start rho(q, r) - g(q)),
// window_buckets() per r over [0, psi_r]: totals [n_r nb] (pairs per bin),
// bin_off [n_r nb + 1] (their exclusive prefix), blk_off
// [window_block_offsets(m, n_r)] (each pass block's offset within each bin),
// *kept_sum += the kept pairs; then the pairs themselves, each bin's run
// from bin_off: pairs[i] = (query, rho(q, r) as float bits).
int window_buckets();
int64_t window_pair_blocks(int64_t m);
int64_t window_block_offsets(int64_t m, int n_r);
// (mq_bits != nullptr: also mq_bits[q] = max over q's kept pairs of
// off_pair_m(rho(q, r), psi_r) as float bits; mq_bits zeroed by the caller)
// Representative offsets of the kept pairs [0, npairs) (binned as by the
// scatter pass, bins of r in bin_off[r nb .. (r + 1) nb]): for pair
// i = (q, rho(q, r)),
// a_rows[i] = bf16(fl(q - r)) ([dpad] columns, zero padded), row_n[i] =
// |a~|^2, row_t[i] = 0.5 (|a~|^2 - T) lowered by a few units in the last
// place with T = off_value_bound(g(q), M, eps, d), M = off_pair_m(rho, psi_r),
// eps = |fl(q - r) - a~| (measured) + yerr[r] + 2^-23 M; eps_bits[q] (zeroed
// by the caller) = the largest eps of q's pairs.  d % 8 == 0, Q32 and R32
// 16-byte aligned.
int launch_offset_pair_rows(const int2* pairs, int npairs, const int* bin_off, int nb, int n_r,
                            const float* Q32, const float* R32, const float* psi,
                            const float* yerr, const float* g, int d, int dpad, void* a_rows,
                            float* row_t, float* row_n, unsigned* eps_bits, int sms,
                            cudaStream_t st);
int launch_window_pairs_count(const float* D, int64_t m, int n_r, const float* g,
                              const float* g1, const float* psi_plus, float rel, int* totals,
                              int* bin_off, int* blk_off, unsigned long long* kept_sum,
                              cudaStream_t st, int* scan_scratch = nullptr,
                              unsigned* mq_bits = nullptr);
int launch_window_pairs_scatter(const float* D, int64_t m, int n_r, const float* g,
                                const float* g1, const float* psi_plus, float rel,
                                const int* bin_off, int* blk_off, int2* pairs, cudaStream_t st);
// chunks of TQ pairs per representative -> items (the chunk's window in the
// sorted list); stats[0] += window rows, stats[1] += query x row pairs
int launch_window_items(const int* bin_off, int nb, int n_r, const int2* pairs,
                        const float* g, const int* offsets,
                        const float* xdist, float rel, float relx, int* chunk_counts,
                        int* chunk_off, int max_items, EmitItem* items,
                        unsigned long long* stats, cudaStream_t st);
// Second pass for queries whose candidate buffer overflowed (rows[i], i < n):
// threshold = score_bound(dist_upper(k-th smallest stored score)), which k
// stored candidates already meet, and the buffer count reset to zero; then
// items over the whole list storage (chunks of TQ of these queries x row
// spans of xspan) for the emission kernel.
// (the number of rows is read from n_dev on the device; at most max_rows)
// (qnorm == nullptr: FP32 difference-form scores, bounds from f32_eps / metric)
// (mq_bits != nullptr: the stored values are representative-offset
// estimates, bounded with mq_bits[q] as M and eps_bits[q] as eps)
int launch_overflow_rethreshold(const int* rows, const int* n_dev, int64_t max_rows,
                                const float* cand_score, int* cand_cnt, int cap, int k,
                                const float* qnorm, const float* qerr, const unsigned* lp_max,
                                int d, float* thr, cudaStream_t st, float f32_eps = 0.0f,
                                int metric = RBC_L2, const unsigned* mq_bits = nullptr,
                                const unsigned* eps_bits = nullptr);
int launch_dense_emit_items(const int* n_dev, int64_t x_rows, int xspan, int max_items,
                            EmitItem* items, int* num_items, cudaStream_t st);
// (qnorm == nullptr: thr = f32_score_bound(g, f32_eps, metric))
int launch_score_threshold(const float* g, const float* qnorm, const float* qerr,
                           const unsigned* lp_max, int d, int64_t m, float* thr,
                           cudaStream_t st, float f32_eps = 0.0f, int metric = RBC_L2);

// ---- one-shot RBC (oneshot.cu) ----
// candidate capacity per representative for a list of s points
int oneshot_candidate_cap(int s);
// per row r < reps of D [reps, ld] (distances to n points): the s-th smallest
// value t and every column with D <= t (1 + 3 eps) -> cand[r][0 .. cand_cnt[r])
int launch_oneshot_select(const float* D, int64_t ld, int64_t n, int reps, int s, float eps,
                          int cap, int* cand, int* cand_cnt, uint32_t* dev_err, cudaStream_t st);
// FP64 distances of the candidates of representatives r0 .. r0 + reps - 1,
// sorted by (rho, id): the first s ids -> members[r][0 .. s), psi[r] = the
// s-th distance rounded to float; DEV_ERR_BOUNDS when a representative had
// fewer than s candidates (non-finite distances)
int launch_oneshot_refine(const float* X, const float* R, int d, int metric, int s, int cap,
                          const int* cand, const int* cand_cnt, int r0, int reps, int* members,
                          float* psi, uint32_t* dev_err, cudaStream_t st);
// queries grouped by representative (qperm, qoff from a counting sort), each
// group padded to a multiple of TQ rows: pad_off [n_r + 1], per padded row
// the source row (qsrc_pad) and the output row (qout_pad, through `orig` when
// given), -1 on padding, and per tile its representative
int launch_oneshot_layout(const int* qoff, int n_r, const int* qperm, const int* orig,
                          int* counts_scratch, int* pad_off, int* qsrc_pad, int* qout_pad,
                          int* tile_rep, cudaStream_t st);
// one work item per padded tile: its rows against list r = [r s, (r + 1) s),
// or [list_off[r], list_off[r + 1]) when list_off is given; adds each tile's
// list length to *points_sum when given
int launch_oneshot_items(const int* pad_off, int n_r, const int* tile_rep, const int* qoff, int s,
                         const int* list_off, WorkItem* items, Seg* segs, int* num_items,
                         int max_tiles, unsigned long long* points_sum, cudaStream_t st);
// out[i] = Q[src[i]] (zero row where src[i] < 0), i < rows
int launch_gather_padded(const float* Q, const int* src, int64_t rows, int d, float* out,
                         cudaStream_t st);
// rows[i] (i < n) of a padded layout -> rep64[i] = tile_rep[rows[i] / TQ],
// out_row[i] = qout_pad[rows[i]]
int launch_oneshot_fallback_map(const int* rows, int n, const int* tile_rep, const int* qout_pad,
                                int64_t* rep64, int* out_row, cudaStream_t st);

}  // namespace rbc

namespace rbc {

// ---- data movement and preparation (prep.cu) ----
int launch_gather_rows(const float* src, const int64_t* idx64, const int* idx32, int64_t rows,
                       int d, float* dst, cudaStream_t st);
// Y rows = X rows of list r minus R row r, for every list r (lists
// [offsets[r], offsets[r + 1]) of the list-ordered rows), FP32
int launch_offset_rows(const float* X, const float* R, const int* offsets, int n_r, int d,
                       float* Y, cudaStream_t st);
// out[r] = the largest v[i] over list r's rows [offsets[r], offsets[r + 1])
int launch_list_max(const float* v, const int* offsets, int n_r, float* out, cudaStream_t st);
// FP32 rows -> low-precision rows [rows, dpad] (zero padded), |x~|^2, |x - x~|
// (FP64, rounded up); global maxima of |x - x~| and |x~| as float bits.
int launch_to_lowp(const float* src, int64_t rows, int d, int dpad, int storage, void* dst,
                   float* norm, float* err, unsigned* err_max_bits, unsigned* norm_max_bits,
                   cudaStream_t st, float* scale = nullptr);  // scale: [rows], FP8 only
// dst row i = src row idx[i] of a bf16 / fp16 [*, dpad] matrix plus its norm
// and residual; idx[i] < 0 gives a zero row
int launch_gather_lp_rows(const void* src, const float* snorm, const float* serr, const int* idx,
                          int64_t rows, int row_bytes, void* dst, float* dnorm, float* derr,
                          cudaStream_t st, const float* sscale = nullptr, float* dscale = nullptr);
// -|x~[i]|^2 / 2 as a (high, low) pair of the storage type (bf16 / fp16)
// written into columns col, col + 1 of each row (zero padding until then):
// a query row with 1 in those columns then picks the norm term up in its
// ordinary MMA, and one with 0 there (every other use) is unaffected
int launch_fold_norm(void* lp, const float* norm, int64_t rows, int dpad, int col, int storage,
                     cudaStream_t st);
// Norm block of a low-precision matrix: row i = (h, l, 0, ..., 0) in bf16
// with h = bf16(-norm[i] / 2), l = bf16(-norm[i] / 2 - h), so that an MMA of
// an all-ones row against it adds -|x~|^2 / 2 to every accumulator of column
// i (to about 2^-17 relative).  rows_out >= rows; rows past `rows` are zero.
int launch_norm_block(const float* norm, int64_t rows, int64_t rows_out, void* dst,
                      cudaStream_t st);
// |x|^2 of FP32 rows [rows, d]; max_bits (optional): the largest |x| rounded up
int launch_row_norms(const float* X, int64_t rows, int d, float* norm, unsigned* max_bits,
                     cudaStream_t st);
// out[i] = qorig ? qorig[rows[i]] : rows[i], for i < *n_dev (or n when n_dev is null)
int launch_map_rows(const int* rows, const int* n_dev, int n, const int* qorig, int* out,
                    cudaStream_t st);
// out_ids / out_dist row dst_rows[i] = row i of ids / dist ([rows, k])
int launch_scatter_result_rows(const int64_t* ids, const float* dist, const int* dst_rows,
                               int64_t rows, int k, int64_t* out_ids, float* out_dist,
                               cudaStream_t st);

// ---- index construction / exact-search helpers (rbc_kernels.cu) ----
// counting sort of `key[i]` in [0, nbins): stable positions.  perm[pos] = i,
// offsets[nbins + 1].  `scratch` needs counting_sort_scratch_ints() ints.
int64_t counting_sort_scratch_ints(int64_t n, int nbins);
int launch_counting_sort(const int64_t* key, int64_t n, int nbins, int* perm, int* offsets,
                         int* scratch, cudaStream_t st);
// Lists ordered by distance: members[pos] = the point ids sorted by
// (owner, dist, id), offsets[n_r + 1] the list starts, xdist[pos] =
// dist[members[pos]] (dist >= 0).  Scratch: sort_lists_scratch_ints() ints.
int64_t sort_lists_scratch_ints(int64_t n, int n_r);
int launch_sort_lists(const int64_t* owner, const float* dist, int64_t n, int n_r, int* members,
                      int* offsets, float* xdist, int* scratch, cudaStream_t st);
// psi_plus[r] = max over list r of dist[perm[pos]] * (1 + rel) (0 if empty)
int launch_list_radii(const float* dist_by_id, const int* perm, const int* offsets, int n_r,
                      float rel, float* psi_plus, cudaStream_t st);
// Per query of D [m, n_r]: gamma_1, gamma_k (k-th smallest), nearest ordinal.
int launch_row_stats(const float* D, int64_t m, int n_r, int k, float* g1, float* gk,
                     int64_t* nearest, cudaStream_t st);
// Exact-search pruning per query tile (tile t = positions [t*TQ, +TQ)):
// representative r is kept for query q iff
//   D_lo(q,r) <= gk_hi(q) + psi_plus[r]  and  D_lo(q,r) <= 2 gk_hi(q) + g1_hi(q)
// with D_lo = D (1 - rel) and gamma_hi = gamma (1 + rel).  Writes the tile's
// union bitmask [tiles][words], the tile's point count (sum of kept list
// sizes) and per-query kept counts.
int launch_prune(const float* D, const int* qperm, int64_t m, int n_r, const float* g1,
                 const float* gk, const float* psi_plus, const int* offsets, float rel,
                 uint32_t* tile_mask, int64_t* tile_points, int* q_kept, cudaStream_t st);
// Work generation: item counts per tile (ceil(points / W)) and their
// exclusive scan -> tile_item_off [tiles + 1] (last entry = total items).
int launch_item_offsets(const int64_t* tile_points, int tiles, int W, int* counts_scratch,
                        int* tile_item_off, cudaStream_t st);
// Each tile's kept lists (merged where adjacent) cut into items of at most W
// points; segments of tile t live at [t * seg_cap_per_tile, ...).
int launch_workgen_items(const uint32_t* tile_mask, const int* offsets, int n_r, int64_t m, int W,
                         int item_cap_per_tile, int seg_cap_per_tile, const int* tile_item_off,
                         WorkItem* items, Seg* segs, uint32_t* dev_err, cudaStream_t st);
// reduce helpers for statistics
int launch_sum_i32(const int* v, int64_t n, unsigned long long* out, cudaStream_t st);
int launch_sum_i64(const int64_t* v, int64_t n, unsigned long long* out, cudaStream_t st);
// out[0 .. n] = exclusive prefix sums of in[0 .. n) and the total; with a
// scratch of exclusive_scan_scratch_ints(n) ints long arrays scan on many blocks
int exclusive_scan_scratch_ints(int n);
int launch_exclusive_scan(const int* in, int n, int* out, cudaStream_t st, int* scratch = nullptr);
// dst[i] += src[i] for i < n (n <= 32)
int launch_add_ints(int* dst, const int* src, int n, cudaStream_t st);
// *dst |= *src (device error flags)
int launch_or_flags(uint32_t* dst, const uint32_t* src, cudaStream_t st);
// sum over query tiles of (tile rows) x (tile union points)
int launch_sum_pairs(const int64_t* tile_points, int64_t m, unsigned long long* out,
                     cudaStream_t st);


}  // namespace rbc
