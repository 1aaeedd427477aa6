/*
 * rbc.h -- C ABI of the B300 Random Ball Cover library (librbc.so).
 *
 * Exact and one-shot nearest-neighbour search with the Random Ball Cover of
 * Cayton, "Accelerating Nearest Neighbor Search on Manycore Systems": every
 * search and build step is a call of the brute-force primitive BF(Q, X)
 * (Section 3), run by hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Pointers.  Every array argument may be a DEVICE pointer (cudaMalloc /
 *   torch CUDA tensor on the current device) or a HOST pointer (pageable or
 *   pinned).  The library inspects each pointer; host inputs are copied to the
 *   device and host outputs are filled by a device-to-host copy, inside the
 *   call, on the given stream -- except that the windowed exact search copies
 *   host query rows of batches of 8,192 rows or more in row chunks on a
 *   library-owned stream (one per calling thread and device), ordered against
 *   the given stream by events, so that each chunk's first steps start as
 *   soon as its rows have landed.  Arrays are dense row-major: X [n, d],
 *   Q [m, d] float32; out_ids [m, k] int64; out_dist [m, k] float32.
 * Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   With device outputs the call is asynchronous: results are valid once the
 *   stream has drained.  With host outputs the call returns after they are
 *   written.  Calls synchronise the stream internally when the amount of
 *   stage-two work must be read back (exact search) -- see rbc_search.
 * Results.  Row i of out_ids / out_dist holds the k nearest database points
 *   of query i in increasing (rho, id) order: equal distances are ordered by
 *   the smaller database id.  out_dist holds rho itself (Euclidean distance,
 *   not its square, for RBC_L2; the l1 sum for RBC_L1).  When k exceeds the
 *   number of points the tail holds id -1 and distance +inf.
 * Exactness.  Low-precision storage (RBC_BF16 / RBC_F16 / RBC_FP8E4M3) is used for the
 *   tensor-core distance pass only; candidates are re-ranked in FP32
 *   difference form, the candidate set is certified with a rounding-error
 *   bound, queries that fail certification are re-searched in FP32, and
 *   near-ties are decided in FP64.  On every FP32 path (RBC_F32, RBC_L1, the
 *   re-search itself) a query whose candidate set still fails the
 *   certificate -- more points than the set holds within the FP32 rounding
 *   bound of its k-th distance -- is finished by an FP64 pass over every
 *   point within that band of its database range.  Results are those of an
 *   FP64 brute force, up to ties closer than its own rounding.
 * Errors.  Every int-returning call returns RBC_OK (0) or a negative code;
 *   rbc_last_error() then returns a message for the calling thread.  On error
 *   no output is guaranteed.  Inputs containing NaN or Inf are undefined.
 * Threads.  Different indexes may be used from different threads.  One index
 *   may be searched concurrently from several threads on different streams
 *   (the index is read-only after build; each call owns its workspace).
 */
#ifndef RBC_H_
#define RBC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define RBC_OK 0
#define RBC_ERR_ARG (-1)         /* invalid argument (sizes, k, n_r, null pointer) */
#define RBC_ERR_OOM (-2)         /* device allocation failed */
#define RBC_ERR_CUDA (-3)        /* a CUDA runtime call or kernel failed */
#define RBC_ERR_TIMEOUT (-4)     /* a bounded device-side wait expired */
#define RBC_ERR_UNSUPPORTED (-5) /* combination not supported (e.g. d > 256) */

/* ---- enumerations ---- */
typedef enum {
  RBC_L2 = 0, /* Euclidean distance (Section 7: used for every experiment) */
  RBC_L1 = 1  /* sum of absolute differences (Section 6, lattice example) */
} rbc_metric;

typedef enum {
  RBC_EXACT = 0,  /* exact search: lists are a partition, Section 5.2 */
  RBC_ONESHOT = 1 /* one-shot search: lists are the s-NN of each rep, Section 5.1 */
} rbc_mode;

typedef enum {
  RBC_F32 = 0,     /* FP32 CUDA-core distance kernels throughout */
  RBC_BF16 = 1,    /* bf16 tensor-core pass (L2), FP32 re-rank, FP64 ties */
  RBC_F16 = 2,     /* fp16 tensor-core pass (L2), FP32 re-rank, FP64 ties */
  RBC_FP8E4M3 = 3  /* FP8 E4M3 with a per-vector scale (the vector's max |x_i| / 448
                      rounded up to a power of two), tcgen05 kind::f8f6f4 pass with
                      FP32 accumulation (L2), FP32 re-rank, FP64 ties; the residual
                      |x - x~| of the scaled dequantisation enters the certification.
                      Exact search uses the tile-union plan.  Rows are padded to a
                      multiple of 128 elements. */
} rbc_storage;

/* Stage two of the exact search with bf16 / fp16 storage (L2).
 *   RBC_PLAN_WINDOW: every query first bounds its k-th neighbour distance by
 *     g = min(gamma_k, the k-th distance inside its nearest representative's
 *     list); each surviving list is sorted by rho(x, r), so a query scans only
 *     the window rho(q, r) - g <= rho(x, r) <= rho(q, r) + g of it (triangle
 *     inequality).  Queries are grouped per representative, ordered by
 *     rho(q, r) and cut into chunks of 128; the tensor-core pass emits every
 *     point whose score can be within g, and the candidates are re-ranked.
 *   RBC_PLAN_TILE_UNION: tiles of 128 queries ordered by nearest
 *     representative search the union of their surviving lists, keeping a
 *     top-c list per query, then re-rank and certify.
 *   RBC_PLAN_WINDOW_OFFSET: the windowed plan on offsets from the
 *     representative (bf16 storage, d a multiple of 8; otherwise the same as
 *     RBC_PLAN_WINDOW): the build also stores every list row as
 *     y~ = bf16(x - r) of its representative r, and each (query chunk,
 *     window of r's list) multiplies a~ = bf16(q - r) by those rows.  The
 *     rounding then scales with |q - r| + |x - r| instead of |q| + |x|, so
 *     far fewer points fall in the band a candidate must be re-ranked for
 *     (data far from the origin, tight clusters).  Uses n x dpad more bf16
 *     of device memory, and per batch one bf16 row per kept (query, list)
 *     pair, sized by reading the pair count back (so a search on this plan
 *     cannot be recorded into a CUDA graph).
 * FP32 and L1 searches run the windowed plan on CUDA cores (the tile-union
 * plan when asked for). */
typedef enum {
  RBC_PLAN_WINDOW = 0,
  RBC_PLAN_TILE_UNION = 1,
  RBC_PLAN_WINDOW_OFFSET = 2
} rbc_plan;

typedef struct rbc_index rbc_index; /* opaque; owned by the library */

/* Build options.  Zero-initialised (or rbc_default_opts) means: seed 0,
 * RBC_EXACT, RBC_F32, default re-rank width, sampled representatives. */
typedef struct {
  uint64_t seed;          /* seed of the representative sampler */
  int32_t mode;           /* rbc_mode */
  int32_t storage;        /* rbc_storage used by the search and the build */
  int32_t rerank_c;       /* candidates per query kept by the low-precision
                             pass before re-ranking; 0 = automatic */
  int32_t plan;           /* exact-search stage two: RBC_PLAN_WINDOW (0),
                             RBC_PLAN_TILE_UNION (1) or
                             RBC_PLAN_WINDOW_OFFSET (2) */
  const int64_t* rep_ids; /* optional HOST array of n_r distinct ids in
                             [0, n), ascending; NULL = sample them */
} rbc_opts;

void rbc_default_opts(rbc_opts* opts);

/*
 * rbc_sample_reps -- the representative set R (Section 4).
 *   The paper selects each point independently with probability n_r / n; this
 *   library draws exactly n_r distinct ids uniformly without replacement: a
 *   partial Fisher-Yates shuffle of [0, n) whose swap positions come from
 *   SplitMix64(seed) (Steele, Lea & Flood 2014) with rejection of the top
 *   2^64 mod (n - i) values, and returns them sorted ascending.  Host-only
 *   (no device work).  out: HOST array of n_r int64.
 *   Errors: RBC_ERR_ARG if n < 1, n_r < 1, n_r > n or out is NULL.
 */
int rbc_sample_reps(int64_t n, int32_t n_r, uint64_t seed, int64_t* out);

/*
 * rbc_build -- build a Random Ball Cover over X (Sections 4 and 5).
 *   X [n, d] float32 (device or host).  n_r representatives are sampled with
 *   rbc_sample_reps(n, n_r, opts->seed) unless opts->rep_ids is given.
 *   Exact mode: BF(X, R) assigns every point to its nearest representative
 *   (ties to the smaller id), each representative's list L_r is the set of
 *   points it owns and psi_r = max over L_r of rho(x, r).  `s` is ignored.
 *   One-shot mode: BF(R, X) with k = s gives each L_r = the s nearest points
 *   of r in (rho, id) order and psi_r = the s-th distance; lists are stored
 *   back to back (offsets r * s, n_r * s < 2^31 entries).  The FP32 distances
 *   are screened per representative by an exact radix select of the s-th
 *   smallest; every point within the FP32 rounding bound of it is recomputed
 *   in FP64 and sorted, so the lists are those of FP64 arithmetic.
 *   The index keeps its own copies (FP32 rows in list order, the
 *   low-precision copy, norms, rounding residuals, radii); X may be freed
 *   after the call returns and the stream has drained.
 *   out: receives the new index; free with rbc_free.
 *   Errors: RBC_ERR_ARG if n < 1, d < 1, n_r < 1, n_r > n, n >= 2^31,
 *   one-shot with s < 1 or s > n, bad enum, or NULL X/out;
 *   RBC_ERR_UNSUPPORTED if d > 256, if one-shot n_r * s >= 2^31, or if more
 *   than 16384 points of a one-shot list tie within FP32 rounding of its
 *   s-th distance; RBC_ERR_OOM; RBC_ERR_CUDA.
 */
int rbc_build(const float* X, int64_t n, int32_t d, int32_t n_r, int32_t s, int32_t metric,
              const rbc_opts* opts, void* stream, rbc_index** out);

/*
 * rbc_search -- k nearest neighbours of every query (Section 5).
 *   Exact mode (Section 5.2, generalised to k): stage one is BF(Q, R) keeping
 *   every distance; gamma_1 / gamma_k are the distances to the nearest / k-th
 *   nearest representative; representative r survives iff
 *   rho(q, r) <= gamma_k + psi_r and rho(q, r) <= 2 gamma_k + gamma_1 (both
 *   evaluated with certified rounding bounds); stage two is BF over the union
 *   of the surviving lists.  Queries are processed in tiles of nearby queries
 *   (ordered by nearest representative) and each tile searches the union of
 *   its queries' surviving lists -- a superset, so results are unchanged.
 *   One-shot mode (Section 5.1): BF(q, R) picks the nearest representative r
 *   (ties to the smaller id) and BF(q, X[L_r]) gives the answer; requires
 *   k <= s.  Queries are grouped by representative and each group padded to
 *   whole 128-query tiles, so every tile searches exactly one list.
 *   Q [m, d] float32; out_ids [m, k] int64; out_dist [m, k] float32 (device
 *   or host).  m may be 0 (no work).
 *   Host read-backs: the tile-union plan and one-shot mode read back small
 *   counters (stage-two work sizes) and so synchronise `stream`.  The
 *   windowed plan decides its overflow passes on the device and reads back
 *   once per batch of queries, at its end: the count of rows left for the
 *   FP32 exact search (rows with more points tying within rounding than a
 *   candidate buffer holds) and the device error flags.
 *   Stream capture (windowed plan only): called while `stream` is being
 *   captured into a CUDA graph, rbc_search reads nothing back and
 *   synchronises nothing, so the graph replays the whole search.  Rows left
 *   after the overflow pass are then finished on the device by the FP64
 *   band pass over the whole database (exact, slow only when thousands of
 *   points tie); device error flags (a bounded wait that expired) are
 *   recorded in the index and reported by rbc_search_check.  Requirements:
 *   Q and the outputs in device memory, rbc_set_timing off, and one call
 *   with the same batch shape made on this thread before the capture (it
 *   sets up the kernels' attributes and the pinned statistics block).
 *   Workspace is then taken from the graph's own memory (stream-ordered
 *   allocation nodes) instead of the library's pool.
 *   Errors: RBC_ERR_ARG if idx/Q/outputs NULL, m < 0, k < 1, k > n,
 *   one-shot with k > s, or host memory under capture; RBC_ERR_UNSUPPORTED
 *   under capture with a plan other than RBC_PLAN_WINDOW or with timing
 *   on; RBC_ERR_OOM; RBC_ERR_CUDA; RBC_ERR_TIMEOUT.
 */
int rbc_search(const rbc_index* idx, const float* Q, int64_t m, int32_t k, int64_t* out_ids,
               float* out_dist, void* stream);

/*
 * rbc_search_check -- waits for `stream`, then reports and clears the device
 *   error flags that searches recorded under stream capture left in the
 *   index (each bounded wait of the tensor-core kernels gives up after
 *   2 s and sets a flag instead of hanging).  RBC_OK when none is set.
 *   No counterpart in the paper (error reporting of replayed graphs).
 *   Errors: RBC_ERR_ARG if idx is NULL; RBC_ERR_TIMEOUT or RBC_ERR_CUDA for
 *   recorded flags; RBC_ERR_CUDA.
 */
int rbc_search_check(const rbc_index* idx, void* stream);

/*
 * rbc_search_workspace -- upper bound of the device workspace (bytes
 *   requested from the library's workspace pool) that one rbc_search(idx, Q,
 *   m, k, ...) call holds at any time: the sum of every request the search may
 *   make, with each data-dependent size at its maximum (every candidate list
 *   at full width, every query falling back to the FP32 re-search) and host
 *   I/O copies included.  A call over more queries than one internal batch
 *   (131,072, or 2^28 / n_r for the windowed plan) holds one batch's
 *   workspace at a time, so the bound stops growing there except for the
 *   I/O copies.  Host only; no device work.  rbc_last_stats reports the
 *   measured peak of a call (workspace_bytes).  Used for admission by memory
 *   in the serving engine (rbc_server_*).  No counterpart in the paper.
 *   Errors: RBC_ERR_ARG on NULL idx / bytes, m < 0 or k < 1.
 */
int rbc_search_workspace(const rbc_index* idx, int64_t m, int32_t k, int64_t* bytes);

/*
 * bf_search -- the brute-force primitive BF(Q, X) (Section 3): all m x n
 *   distances fused with a per-query top-k; no distance matrix is stored.
 *   storage RBC_F32: FP32 CUDA-core kernel.  RBC_BF16 / RBC_F16 with RBC_L2:
 *   tcgen05 tensor-core pass over the expansion |x|^2 - 2 q.x, then the FP32
 *   re-rank / certification / FP64 tie steps described above.  RBC_L1 always
 *   runs in FP32 on CUDA cores.
 *   Errors: RBC_ERR_ARG (m < 0, n < 1, d < 1, k < 1, n >= 2^31, bad enum,
 *   NULL pointers); RBC_ERR_UNSUPPORTED (d > 256); RBC_ERR_OOM; RBC_ERR_CUDA.
 */
int bf_search(const float* Q, int64_t m, const float* X, int64_t n, int32_t d, int32_t k,
              int32_t metric, int32_t storage, int64_t* out_ids, float* out_dist, void* stream);

/*
 * bf_search_noalloc -- BF(Q, X) like bf_search with storage RBC_F32, for
 *   callers that cannot allocate device memory (for example a serving engine
 *   that has reserved the device memory budget for its own pool, or a
 *   latency-critical path where an allocation, which may synchronise the
 *   device or fail under memory pressure, is not acceptable).  The paper has
 *   no counterpart: this is a deployment variant of the brute-force search.
 *   It makes no allocation: its scratch is one static device array of 32 MiB
 *   inside the library, held by every GPU that loads the library until the
 *   process exits.  Q, X, out_ids and out_dist must be DEVICE pointers on the
 *   current device (host buffers, or buffers of another GPU, are rejected with
 *   RBC_ERR_ARG).  Limit: the per-query candidate lists of all ceil(m / 128)
 *   query tiles plus one int per query (rows to finish exactly, rounded up to
 *   256 bytes) must fit in the array after a 256-byte head, i.e.
 *   ceil(m / 128) * 128 * 2 * C * 8 + ceil(4 m / 256) * 256 <= 32 MiB - 256
 *   with C the smallest of 2, 4, 8, 16, 32 that is >= k + 1: m <= 931,968
 *   for k = 1, 493,440 for k = 2-3, 254,080 for k = 4-7, 129,024 for
 *   k = 8-15, 65,024 for k = 16-31.  A larger m returns RBC_ERR_UNSUPPORTED
 *   with the limit in the message.  Queries whose candidate set fails the
 *   FP32 certificate are finished exactly in the same call (the FP64 band
 *   pass, working in the same scratch), as in bf_search; rbc_last_stats
 *   then reports them (uncertified), read from the scratch on demand, so
 *   call it before the next bf_search_noalloc on that device.  The first call
 *   on a device looks up the array's device address (cudaGetSymbolAddress,
 *   once per device, with that device current) and keeps it for the life of
 *   the process: make that first call before any stream capture, and do not
 *   use the library across a cudaDeviceReset.  All calls share the array:
 *   calls that overlap on the GPU race and must be serialised by the caller.
 *   Results and errors otherwise as bf_search.
 */
int bf_search_noalloc(const float* Q, int64_t m, const float* X, int64_t n, int32_t d, int32_t k,
                      int32_t metric, int64_t* out_ids, float* out_dist, void* stream);

/* Index description. */
typedef struct {
  int64_t n;
  int32_t d;
  int32_t n_r;
  int32_t s;
  int32_t metric;
  int32_t mode;
  int32_t storage;
  int64_t list_entries;  /* total entries over all lists (n in exact mode) */
  int64_t device_bytes;  /* device memory held by the index */
  int32_t device;        /* CUDA device the index was built on */
} rbc_index_desc;

/* rbc_index_info -- fills *out.  Errors: RBC_ERR_ARG on NULL. */
int rbc_index_info(const rbc_index* idx, rbc_index_desc* out);

/*
 * rbc_index_export -- copies the built structure to HOST arrays (each may be
 *   NULL to skip it): reps [n_r] representative ids (ascending);
 *   offsets [n_r + 1] start of each list in `members`; members
 *   [list_entries] database ids, list by list, each list ordered by
 *   (rho(x, r), id) (exact mode: rho as computed in FP32 by the build;
 *   one-shot: in FP64); psi [n_r] radii as float32
 *   (exact mode: an upper bound of max_{x in L_r} rho(x, r) within the FP32
 *   rounding bound; one-shot: the FP64 s-th distance rounded to float).
 *   Synchronises the index's build stream.  Errors: RBC_ERR_ARG, RBC_ERR_CUDA.
 */
int rbc_index_export(const rbc_index* idx, int64_t* reps, int64_t* offsets, int64_t* members,
                     float* psi);

/* Statistics of the most recent rbc_search / bf_search on this thread. */
typedef struct {
  int64_t queries;
  int64_t kept_reps;         /* sum over queries of surviving representatives
                                (one-shot: one per query) */
  int64_t tile_points;       /* sum over query tiles of the points in the tile's
                                union of surviving lists (one-shot: padded
                                tiles x s) */
  int64_t stage2_items;      /* stage-two work-item capacity launched */
  int64_t uncertified;       /* queries whose candidate set failed certification:
                                re-searched in FP32 (low-precision pass), or
                                finished by the FP64 band pass (FP32 paths) */
  int64_t fp64_ties;         /* queries whose order needed the FP64 tie step */
  int64_t boundary_ties;     /* queries with an FP32 near-tie at the k-th place */
  int64_t pairs;             /* (query, point) distances of the main BF pass:
                                dense BF m*n; exact search sum over tiles of
                                tile rows x union points; one-shot m*s */
  int64_t kernel_launches;   /* CUDA kernels this call launched */
  double stage1_ms;          /* device time per phase, filled only while
                                rbc_set_timing(1) is in effect: preparation and */
  double stage2_ms;          /*   stage one / the main BF distance kernel / */
  double select_ms;          /*   merge + re-rank + certification / */
  double fallback_ms;        /*   FP32 re-search of uncertified queries */
  int64_t candidates;        /* windowed search: points emitted by the tensor-core
                                pass for the exact re-rank (summed over queries) */
  int64_t workspace_bytes;   /* rbc_search: peak device workspace the call held
                                (bytes requested from the workspace pool) */
} rbc_search_stats;

/* rbc_last_stats -- statistics of this thread's last search call (host only;
 * waits for that call's stream). */
int rbc_last_stats(rbc_search_stats* out);

/* rbc_set_timing -- on != 0: later searches on this thread record CUDA events
 * around their phases (one extra stream synchronisation per call) so that
 * rbc_last_stats reports per-phase device times.  Off by default.  Returns
 * the previous setting. */
int rbc_set_timing(int on);

/*
 * rbc_trim_workspace -- returns the search workspace cached for the current
 *   device to the driver.  Search calls take their scratch (distance rows,
 *   work items, candidate buffers: a few GB for large batches) from a
 *   library-owned stream-ordered pool that keeps freed memory mapped for the
 *   next call; this call synchronises the device and releases all of it.
 *   Errors: RBC_ERR_CUDA.  No counterpart in the paper (memory management).
 */
int rbc_trim_workspace(void);

/* ---------------------------------------------------------------------------
 * Serving engine: continuous batching over a resident index.  No counterpart
 * in the paper, whose experiments search each data set's queries as one
 * batch (Section 7); this is the request loop a deployment puts around
 * rbc_search.
 *
 * A server owns `workers` worker threads, each with its own CUDA stream and
 * resident device buffers for one merged batch (max_batch queries).  A free
 * worker takes the requests waiting at the head of the queue, in arrival
 * order, as many as fit within max_batch queries, shrinking the batch until
 * its workspace bound (rbc_search_workspace with the batch's largest k)
 * fits the HBM budget left by the batches already in flight -- or waits for
 * memory to be released.  It copies the requests' queries into its batch
 * buffer, runs one rbc_search over the batch, and copies each request's
 * first k columns into that request's own output buffers.  Batches of
 * different workers run concurrently on the device.  Each query's result
 * depends only on that query, so a request gets the same answer alone and
 * in any mix.
 * ------------------------------------------------------------------------- */
typedef struct rbc_server rbc_server; /* opaque; owned by the library */

typedef struct {
  int32_t workers;    /* batches in flight at once (threads + streams); 0 = 2; <= 16 */
  int32_t max_batch;  /* queries per merged batch and per request; 0 = 16384 */
  int32_t k_max;      /* largest k a request may ask for; 0 = 10; <= 31 */
  int32_t reserved;   /* must be 0 */
  int64_t hbm_budget; /* device bytes the in-flight batches' search workspace
                         may take (sum of their rbc_search_workspace bounds);
                         0 = half the free device memory at creation */
} rbc_server_opts;

/* What happened to one request (times from a steady clock, nanoseconds). */
typedef struct {
  int64_t t_submit_ns;    /* rbc_server_submit */
  int64_t t_start_ns;     /* its batch was admitted */
  int64_t t_done_ns;      /* its results were in its host buffers */
  int64_t batch;          /* sequence number of the batch that served it (-1: m = 0) */
  int64_t batch_queries;  /* queries in that batch */
  int32_t batch_requests; /* requests in that batch */
  int32_t status;         /* RBC_OK or the search's error code */
} rbc_request_info;

/* Aggregate over the requests collected since creation or the last reset. */
typedef struct {
  int64_t requests, queries, batches;
  double p50_ms, p99_ms, mean_ms, max_ms; /* latency: submit -> results on the host */
  double queue_p50_ms, queue_p99_ms;      /* submit -> batch admitted */
  double wall_s;                          /* first submit -> last completion */
  double queries_per_s;                   /* queries / wall_s */
  double mean_batch_queries;
  int64_t peak_reserved_bytes;            /* largest workspace bound held at once */
  int64_t hbm_budget;
  int32_t max_in_flight;                  /* most batches on the device at once */
  int32_t workers;
} rbc_serving_stats;

/*
 * rbc_server_create -- starts a server over `idx`, which must stay alive and
 *   unchanged until rbc_server_destroy.  opts may be NULL (defaults above).
 *   Errors: RBC_ERR_ARG (NULL, workers > 16, max_batch > 2^24, k_max > 31,
 *   k_max > n, one-shot k_max > s), RBC_ERR_CUDA / RBC_ERR_OOM (streams,
 *   buffers).
 */
int rbc_server_create(const rbc_index* idx, const rbc_server_opts* opts, rbc_server** out);

/*
 * rbc_server_submit -- queues a request of m queries Q [m, d] float32 and
 *   returns at once with its ticket.  out_ids [m, k] int64 and out_dist
 *   [m, k] float32 receive the results as rbc_search would (host or device
 *   pointers; pinned host memory gives asynchronous copies).  Q and the
 *   outputs must stay valid until rbc_server_wait reports the request done.
 *   Errors: RBC_ERR_ARG (NULL, m < 0, m > max_batch, k outside [1, k_max],
 *   server stopping); RBC_ERR_OOM if the workspace bound of a batch of this
 *   request alone exceeds the HBM budget (it could never be admitted).
 */
int rbc_server_submit(rbc_server* s, const float* Q, int64_t m, int32_t k, int64_t* out_ids,
                      float* out_dist, uint64_t* ticket);

/*
 * rbc_server_wait -- waits until request `ticket` is done (timeout_us < 0:
 *   no limit), fills *info (may be NULL) and releases the ticket.  Returns
 *   the request's status (the error of the batch's search, message in
 *   rbc_last_error), or RBC_ERR_TIMEOUT if still running after timeout_us
 *   (the ticket stays valid), or RBC_ERR_ARG for an unknown ticket.
 */
int rbc_server_wait(rbc_server* s, uint64_t ticket, int64_t timeout_us, rbc_request_info* info);

/* rbc_server_stats -- fills *out; reset != 0 then starts a new window. */
int rbc_server_stats(rbc_server* s, int32_t reset, rbc_serving_stats* out);

/* rbc_server_destroy -- finishes every queued request, stops the workers and
 * frees the server (not the index).  No other call on `s` may be running. */
void rbc_server_destroy(rbc_server* s);

/*
 * rbc_plan_batch -- the admission rule of the server's workers, exposed for
 *   tests with a linear workspace model: of n queued requests (m[i] queries,
 *   k[i] neighbours, in arrival order) a batch takes the first c, the largest
 *   c whose queries sum to at most max_batch and whose bound
 *   fixed_bytes + queries * (bytes_per_query + max k * bytes_per_query_k)
 *   is at most mem_left.  Returns c (0: nothing fits).  Host only.
 *   Errors: RBC_ERR_ARG (n < 0, NULL arrays, max_batch < 1).
 */
int rbc_plan_batch(const int64_t* m, const int32_t* k, int32_t n, int64_t max_batch,
                   int64_t mem_left, int64_t fixed_bytes, int64_t bytes_per_query,
                   int64_t bytes_per_query_k);

/* ---------------------------------------------------------------------------
 * Grouped multi-index search.  No counterpart in the paper, which searches
 * one database at a time (Sections 5, 7): a group holds many independent
 * exact indexes (one per tenant, shard, category ...) and searches a batch
 * of queries for every one of them together.  The indexes' rows, lists,
 * representatives and radii are concatenated into one resident layout (rows
 * zero-padded to the widest dimension, which changes no distance), and every
 * step of the exact search runs once for all indexes: stage one against each
 * query's own representatives, pruning and work generation per 128-query tile
 * of one index, ONE persistent tensor-core launch over the work items of all
 * indexes, one merge / re-rank / certification launch, and an exact finish
 * over the query's own index (the FP64 band pass) for uncertified queries.
 * No count is read back to the host inside the search, so each batch shape
 * (the per-index query counts and k) is captured once as a CUDA graph and
 * replayed.
 * Results equal those of rbc_search on each index alone.
 * ------------------------------------------------------------------------- */
typedef struct rbc_group rbc_group; /* opaque; owned by the library */

typedef struct {
  int64_t indexes, rows, representatives;
  int32_t dim;               /* common (padded) row length */
  int32_t work_item_points;  /* stage-two work-item size of the last search */
  int64_t queries;           /* queries of the last search */
  int64_t tiles, work_items; /* its 128-query tiles and stage-two work items */
  int64_t uncertified;       /* its queries finished by the FP64 band pass */
  int64_t fp64_ties;         /* its queries whose order needed FP64 */
  int64_t graph_replays;     /* launches of the batch shape's CUDA graph */
  uint32_t device_errors;    /* device error flags of the last search (0 = none) */
} rbc_grouped_stats;

/*
 * rbc_group_create -- copies `count` built indexes into a new group (the
 *   indexes may be freed afterwards).  Every index must be exact-mode L2 with
 *   the same bf16 or fp16 storage, on the same device, d <= 256; the group's
 *   rows and representatives must each number < 2^31.  Synchronises `stream`.
 *   Errors: RBC_ERR_ARG (NULL, count < 1, mismatched storage / device),
 *   RBC_ERR_UNSUPPORTED (mode, metric, FP32 / FP8 storage, sizes), RBC_ERR_OOM.
 */
int rbc_group_create(const rbc_index* const* indexes, int32_t count, void* stream,
                     rbc_group** out);

/*
 * rbc_group_search -- k nearest neighbours of every query of every index.
 *   m [count]: HOST array, queries per index (0 allowed).  Q: the queries
 *   packed index after index, index i's m[i] rows of its own d_i floats
 *   (sum m_i d_i floats, host or device).  out_ids / out_dist: [sum m_i, k]
 *   in the same order, ids within each query's own index (host or device).
 *   The first search of a batch shape builds its workspace and CUDA graph;
 *   later searches of the same shape replay the graph (inputs and outputs are
 *   copied through the group's buffers).  Synchronises `stream` once (device
 *   error flags).  Errors: RBC_ERR_ARG (NULL, m out of range, k outside
 *   [1, 31], k above an index's size), RBC_ERR_OOM, RBC_ERR_CUDA,
 *   RBC_ERR_TIMEOUT.
 */
int rbc_group_search(rbc_group* g, const float* Q, const int64_t* m, int32_t k, int64_t* out_ids,
                     float* out_dist, void* stream);

/*
 * rbc_group_search_split -- rbc_group_search with the queries of each index
 *   in a buffer of its own: Q is a HOST array of `count` pointers, Q[i] index
 *   i's m[i] rows of d_i floats (host or device; may be NULL when m[i] = 0).
 *   Each is copied to its place in the group's input buffer, so queries held
 *   per index need no packing on the host.  Outputs, synchronisation and
 *   errors as rbc_group_search (RBC_ERR_ARG also for a NULL Q or Q[i]).
 */
int rbc_group_search_split(rbc_group* g, const float* const* Q, const int64_t* m, int32_t k,
                           int64_t* out_ids, float* out_dist, void* stream);

/*
 * rbc_group_tune -- autotuner: times the search of this batch (3 graph
 *   replays each, CUDA events) for stage-two work-item sizes of 1024 to
 *   32768 points and keeps the fastest for later searches; *chosen (may be
 *   NULL) receives it.  Errors as rbc_group_search.
 */
int rbc_group_tune(rbc_group* g, const float* Q, const int64_t* m, int32_t k, void* stream,
                   int32_t* chosen);

/* rbc_group_stats -- fills *out (reads the last search's device counters). */
int rbc_group_stats(rbc_group* g, rbc_grouped_stats* out);

/* rbc_group_free -- waits for the device and releases the group. NULL ok. */
void rbc_group_free(rbc_group* g);

/* rbc_free -- releases the index (waits for its outstanding work). NULL ok. */
void rbc_free(rbc_index* idx);

/* rbc_last_error -- message of the last failing call on this thread ("" if none). */
const char* rbc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RBC_H_ */
