/*
 * aidw.h - C ABI of the GB300 (sm_103a) AIDW interpolation library.
 *
 * Adaptive inverse distance weighting with an even-grid kNN search, after
 * Mei, Xu & Xu, "Improving GPU-accelerated Adaptive IDW Interpolation
 * Algorithm Using Fast kNN Search" (arXiv 1601.05904).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Point sets are structure-of-arrays float32 (x[], y[], z[]), the layout
 *    of the paper's Sec. 4.2.1.  "Data points" are the samples with known z;
 *    "queries" are the interpolated points.
 *  - Every array argument is a DEVICE pointer owned by the caller unless the
 *    comment says otherwise.  The library never frees caller memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream).  A function that must read a device result back says
 *    so; every other function only enqueues work.
 *  - Arguments are validated on the host before any CUDA call; a rejected
 *    call enqueues nothing.  Errors the device finds (non-finite input
 *    coordinates, an expired bounded wait) are latched in the grid and
 *    returned by aidw_grid_status() and aidw_grid_destroy().
 *  - The library owns grid handles and per-call scratch, which it takes in
 *    stream order on `stream` from a memory pool of its own (one per device)
 *    and returns the same way; freed blocks stay in that pool for reuse
 *    until the process exits.
 */
#ifndef AIDW_H_
#define AIDW_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so that callers need no CUDA header. */
typedef struct CUstream_st *aidw_stream_t;

typedef enum {
    AIDW_OK = 0,
    AIDW_ERR_INVALID_ARG = 1, /* null pointer, negative size, bad parameter    */
    AIDW_ERR_K_RANGE = 2,     /* k < 1, k > 32 or k > number of data points    */
    AIDW_ERR_NONFINITE = 3,   /* a NaN or Inf coordinate or value was found    */
    AIDW_ERR_OOM = 4,         /* a device allocation failed                    */
    AIDW_ERR_CUDA = 5,        /* any other CUDA runtime error                  */
    AIDW_ERR_TIMEOUT = 6      /* a bounded device-side wait expired            */
} aidw_status;

/* Arithmetic of the kNN and weighting stages.
 *  AIDW_FP32_COMP  float32 distances, power by exp2(alpha*log2) on the SFU,
 *                  compensated float32 sums, float64 final divide; alpha
 *                  from a compensated float32 sum of float32 square roots
 *                  (Eq. 3) and Eq. 4-6 in float32.  Outputs are float32.
 *  AIDW_FP64_PLAIN float64 distances, pow(), plain float64 sums.  Outputs
 *                  are float64. */
typedef enum { AIDW_FP32_COMP = 0, AIDW_FP64_PLAIN = 1 } aidw_precision;

#define AIDW_MAX_K 32

/* Parameters of the method.  aidw_params_default() fills the defaults.
 *  k           neighbours for r_obs (Eq. 3); 1 <= k <= 32 and k <= n_data.
 *  alpha[5]    the five distance-decay levels of Eq. 6 (finite, > 0).  The
 *              paper gives no values; the default is {1, 2, 3, 4, 5}.
 *  r_min/r_max bounds of the membership of Eq. 5 (paper: 0.0 and 2.0);
 *              0 <= r_min < r_max.
 *  area        A of Eq. 2; <= 0 selects the area of the data bounding box.
 *  cell_scale  grid cell width = cell_scale * r_exp (the paper's width is
 *              r_exp itself, Sec. 4.1.1, i.e. cell_scale = 1); <= 0 lets
 *              the library choose.
 *  precision   an aidw_precision value. */
typedef struct {
    int k;
    double alpha[5];
    double r_min;
    double r_max;
    double area;
    double cell_scale;
    int precision;
} aidw_params;

void aidw_params_default(aidw_params *p);

/* Static description of a built grid (host copy). */
typedef struct {
    int64_t n_data;
    int64_t n_col;      /* nCol = (int)((maxX - minX + cw) / cw), Sec. 4.1.1 */
    int64_t n_row;
    int64_t n_cells;    /* n_col * n_row */
    double min_x, min_y, max_x, max_y; /* bounding box of the data points */
    double area;        /* A used for r_exp */
    double r_exp;       /* Eq. 2 with n = n_data */
    double cell_width;  /* cw */
    double cell_scale;  /* the scale the grid was built with */
} aidw_grid_info;

/* Opaque grid over a set of data points; owns its device buffers. */
typedef struct aidw_grid aidw_grid;

/* Builds the even grid of Sec. 3.2.1-3.2.3 / 4.1.1-4.1.3: bounding box,
 * cell width (Eq. 2), nCol/nRow, a cell index per point, and a stable
 * counting sort that stores the points in cell order with the (head, count)
 * pair of every cell (Fig. 3).  x, y, z: [n_data] device float32; they are
 * copied into the grid and may be freed once the stream reaches this call.
 * Reads the device result back once (stream-synchronous) to report
 * non-finite input as AIDW_ERR_NONFINITE.  On success *out owns the grid.
 * Uses p->area and p->cell_scale; the other fields are ignored here. */
aidw_status aidw_grid_build(const float *x, const float *y, const float *z, int64_t n_data,
                            const aidw_params *p, aidw_stream_t stream, aidw_grid **out);

/* Synchronises the device (work on any stream may still read the grid),
 * frees the grid and returns its latched device status (AIDW_OK if none). */
aidw_status aidw_grid_destroy(aidw_grid *g);

/* The grid's dimensions (a host copy taken when the build returned; no
 * device access). */
aidw_status aidw_grid_get_info(const aidw_grid *g, aidw_grid_info *info);

/* Copies the grid's cell heads and cell-ordered permutation into caller
 * device buffers: cell_start [n_cells + 1] (head of cell c; count of c is
 * cell_start[c+1] - cell_start[c]) and perm [n_data] (original index of the
 * point stored at each position; stable within a cell).  Either may be NULL. */
aidw_status aidw_grid_export(const aidw_grid *g, int64_t *cell_start, int32_t *perm,
                             aidw_stream_t stream);

/* Synchronises the device (calls on any stream may latch errors in the
 * grid) and returns then clears the latched device-side error (non-finite
 * query coordinates, expired waits). */
aidw_status aidw_grid_status(aidw_grid *g);

/* Exact k nearest neighbours of each query by the grid search of
 * Sec. 3.2.4 / 4.1.4: locate the query's cell, visit rings of cells
 * outwards, keep the k best squared distances (Sec. 4.1.4's remark on
 * avoiding square roots) in a register top-k, and stop once the nearest
 * cell outside the visited block is farther than the k-th distance (an
 * exact rule in place of the paper's "one extra level", which can miss
 * neighbours).  Distances are float32 (Euclidean, from float32 squared
 * distances).  Ties are ordered by original index.
 *  qx, qy    [n_query] device float32
 *  out_idx   [n_query * k] int32 original indices, row-major by query,
 *            increasing distance; or NULL
 *  out_dist  [n_query * k] float32 distances; or NULL
 *  out_robs  [n_query] float32 r_obs of Eq. 3; or NULL
 * A query with a NaN/Inf coordinate gets idx -1, NaN distances and latches
 * AIDW_ERR_NONFINITE in the grid. */
aidw_status aidw_knn(const aidw_grid *g, const float *qx, const float *qy, int64_t n_query,
                     int k, int32_t *out_idx, float *out_dist, float *out_robs,
                     aidw_stream_t stream);

/* AIDW prediction of every query: kNN (above), then per query r_exp
 * (Eq. 2), R (Eq. 4), mu (Eq. 5) and alpha (Eq. 6), then Eq. 1 summed over
 * ALL data points of the grid.  A query at distance 0 from data points
 * returns the mean z of those points (the limit of Eq. 1).  If a bounded
 * wait of the weighting stage expires (aidw_grid_status then reports
 * AIDW_ERR_TIMEOUT), every prediction of the call is NaN.
 *  out_z      [n_query] predictions: float32 for AIDW_FP32_COMP, float64
 *             for AIDW_FP64_PLAIN
 *  out_alpha  [n_query] alpha of each query, same element type; or NULL
 * p->area (when > 0) overrides the area the grid was built with. */
aidw_status aidw_interpolate(const aidw_grid *g, const float *qx, const float *qy,
                             int64_t n_query, const aidw_params *p, void *out_z,
                             void *out_alpha, aidw_stream_t stream);

/* End to end from HOST memory: the path of aidw_grid_build + aidw_interpolate
 * for a caller whose arrays live on the host.  x, y, z [n_data] and qx, qy
 * [n_query] are host float32 arrays (pageable or pinned; pinned ones copy
 * asynchronously at full link speed); out_z (and out_alpha, if not NULL)
 * [n_query] are host arrays of float32 (AIDW_FP32_COMP) or float64
 * (AIDW_FP64_PLAIN).  The call copies the inputs to the current device,
 * builds the grid, interpolates, copies the results back and waits for
 * `stream`; device memory comes from the library's pool and is returned
 * before the call ends.  Returns the first error, including a device error
 * latched during the call (as aidw_grid_status). */
aidw_status aidw_interpolate_host(const float *x, const float *y, const float *z, int64_t n_data,
                                  const float *qx, const float *qy, int64_t n_query,
                                  const aidw_params *p, void *out_z, void *out_alpha,
                                  aidw_stream_t stream);

/* ---- query sharding over several GPUs --------------------------------------
 * Every query is computed independently given all data points (the
 * one-thread-per-query decomposition of Sec. 4.2), so one query set splits
 * over G GPUs with no exchange on the data path: each GPU (one process per
 * GPU) builds its own grid from a replica of the data points, interpolates
 * one contiguous slice of the queries, and writes that slice of the output.
 * No counterpart in the paper, which runs on one GPU. */

/* The slice [*begin, *end) of a query set of n_query queries that shard
 * `shard` of `n_shards` takes: contiguous slices in shard order whose sizes
 * differ by at most one (the first n_query % n_shards shards take one query
 * more).  Host only: no CUDA call.  AIDW_ERR_INVALID_ARG for a null output,
 * n_query < 0, n_shards < 1 or shard outside [0, n_shards). */
aidw_status aidw_shard_range(int64_t n_query, int shard, int n_shards, int64_t *begin,
                             int64_t *end);

/* One shard of a query-sharded interpolation: aidw_interpolate of the
 * queries [begin, end) = aidw_shard_range(n_query, shard, n_shards) on the
 * current device, against grid g (built on this device from the full data
 * set).  qx, qy are the FULL query arrays [n_query] and out_z (out_alpha, if
 * not NULL) full-length output arrays [n_query] of the precision's element
 * type, all device memory on this device; only elements [begin, end) of the
 * outputs are written.  The shards of all GPUs together write every output
 * element exactly once; bringing the slices together (if one process needs
 * them all) is the caller's.  Per-query results equal those of
 * aidw_interpolate on the whole set to rounding (the all-points sums of
 * Eq. 1 may be grouped differently).  Errors as aidw_interpolate, plus
 * AIDW_ERR_INVALID_ARG for a bad shard. */
aidw_status aidw_interpolate_shard(const aidw_grid *g, const float *qx, const float *qy,
                                   int64_t n_query, int shard, int n_shards,
                                   const aidw_params *p, void *out_z, void *out_alpha,
                                   aidw_stream_t stream);

/* ---- batched interpolation ------------------------------------------------
 * Many independent AIDW problems ("jobs"), each with its own data points,
 * queries and k, computed together: the method of the functions above
 * applied to every job (the paper runs one problem at a time; batching is a
 * throughput form of the same computation).  Every step of the path is one
 * launch over all jobs, the all-points weighting (Eq. 1) is a single
 * persistent launch whose work units span all jobs, and the launch sequence
 * is captured once into a CUDA graph that each run replays.
 *
 * A job: x, y, z [n_data] and qx, qy [n_query] device float32 (caller-owned);
 * out_z [n_query] device array of float32 (AIDW_FP32_COMP) or float64
 * (AIDW_FP64_PLAIN); k <= 0 takes params->k.  n_data >= 1, 1 <= k <= 32,
 * k <= n_data; n_query may be 0. */
typedef struct {
    const float *x, *y, *z;
    int64_t n_data;
    const float *qx, *qy;
    int64_t n_query;
    int k;
    void *out_z;
} aidw_job;

/* Opaque plan: the job shapes, one pooled device allocation for every job's
 * grid, kNN records and partial sums, the device job table and the graph. */
typedef struct aidw_batch_plan aidw_batch_plan;

/* Creates a plan for jobs with these shapes (only n_data, n_query and k are
 * read).  Allocates the pool (cudaMalloc) and a pinned staging table. */
aidw_status aidw_batch_plan_create(const aidw_job *jobs, int n_jobs, const aidw_params *p,
                                   aidw_batch_plan **out);

/* Runs the plan on jobs of the plan's shapes (pointers may differ from run
 * to run): uploads the job table from pinned memory and launches the graph
 * on `stream` (captured at the first run).  Asynchronous; the inputs must
 * stay valid and unchanged until the stream reaches the end of the run. */
aidw_status aidw_batch_run(aidw_batch_plan *plan, const aidw_job *jobs, aidw_stream_t stream);

/* Jobs are grouped by top-k width class: the kNN of a job runs in the
 * launch of the smallest class whose register slots (8, 16, 24, 32) hold
 * its k.  Each class has its own cell-width scale (of its jobs' grids) and
 * kNN block size; the defaults are the single-grid choices (scale 2 up to
 * k = 16, 3 above; 128-thread blocks).  The classes' kNN launches run one
 * after another (AIDW_BATCH_BRANCHES=1 runs them as parallel branches). */
#define AIDW_BATCH_CLASSES 4

/* Autotuner: times the grid build + kNN of all jobs (two runs per candidate,
 * the second counted) and descends class by class: for every class with
 * queries, the cell-width scales {1, 1.5, 2, 3, 4} (unless params->cell_scale
 * fixed it), then the kNN block sizes {warp per query, 64, 128, 256},
 * keeping whatever lowers the total.  Discards the captured graph.
 * Synchronous.  *best_ms (may be NULL) receives the best build+kNN time.
 * The result is cached in the process under a key of the precision, the
 * GPU's SM count, a fixed scale and the histogram of the jobs' shapes (log2
 * buckets of n_data and n_query, and k); aidw_batch_plan_create applies a
 * cached tuning to a plan with the same key.  With the environment variable
 * AIDW_TUNE_CACHE=<file> entries are also loaded from and appended to that
 * file, one JSON object per line ({"key", "cell_scale": [4],
 * "knn_threads": [4], "build_knn_ms"}). */
aidw_status aidw_batch_plan_tune(aidw_batch_plan *plan, const aidw_job *jobs,
                                 aidw_stream_t stream, double *best_ms);

/* The plan's size and the choices of its largest class (by queries):
 * cell-width scale, kNN block size (0: warp per query), sum over jobs of
 * n_data * n_query, pool bytes.  Any output may be NULL. */
aidw_status aidw_batch_plan_get(const aidw_batch_plan *plan, double *cell_scale,
                                int *knn_threads, int64_t *total_pairs, int64_t *pool_bytes);

/* Per class (arrays of AIDW_BATCH_CLASSES): register slots, cell-width
 * scale, kNN block size and queries of the class; *source: 0 defaults,
 * 1 measured by aidw_batch_plan_tune, 2 taken from the tuning cache when
 * the plan was created.  Any output may be NULL.  Host only. */
aidw_status aidw_batch_plan_get_classes(const aidw_batch_plan *plan, int *kmax,
                                        double *cell_scale, int *knn_threads, int64_t *queries,
                                        int *source);

/* Synchronises the device and returns then clears the device-side errors of
 * the last runs (any job). */
aidw_status aidw_batch_plan_status(aidw_batch_plan *plan);

aidw_status aidw_batch_plan_destroy(aidw_batch_plan *plan);

/* One-shot: create a plan, run it, wait, check the device status, destroy. */
aidw_status aidw_batch(const aidw_job *jobs, int n_jobs, const aidw_params *p,
                       aidw_stream_t stream);

/* ---- interpolation without device allocation ------------------------------
 * No counterpart in the paper; this is a library service.  Some callers
 * cannot let a library allocate device memory: an application that reserves
 * the GPU's memory up front and hands out slices from its own pool, or a
 * latency-critical loop where cudaMalloc/cudaFree (which may synchronise the
 * device, or fail under memory pressure halfway through a pipeline) is not
 * acceptable.  aidw_interpolate_noalloc gives the predictions (and alphas)
 * of aidw_interpolate, but keeps its per-call scratch (the per-query kNN
 * records and the partial sums of the weighting stage) in one fixed-size
 * array inside the library's device image, so the call performs no
 * allocation of any kind.  The caller still passes the grid, the queries
 * and the outputs.
 *  - It runs the kNN and weighting kernels of aidw_interpolate but not the
 *    pass that first orders the queries by grid cell (its temporaries would
 *    need memory): the kNN takes the queries in input order, which gives
 *    the same results and is slower on clustered data.
 *  - n_query must not exceed AIDW_NOALLOC_MAX_QUERIES; larger calls return
 *    AIDW_ERR_INVALID_ARG and enqueue nothing.
 *  - The scratch array (AIDW_NOALLOC_SCRATCH_BYTES) lives in every GPU that
 *    loads the library until the process exits.
 *  - The first call on a device looks up the array's device address (host
 *    set-up); make that first call before any stream capture.  A first call
 *    on a stream that is being captured returns AIDW_ERR_INVALID_ARG and
 *    enqueues nothing.
 *  - If a weighting wait expires (aidw_grid_status then reports
 *    AIDW_ERR_TIMEOUT), every prediction of that call is NaN, as in
 *    aidw_interpolate: no sum left in the shared array by an earlier call
 *    reaches the output.
 *  - Every call on a device shares the one array: calls that can overlap on
 *    the GPU (different streams, no ordering between them) race on it.
 *    Calls ordered on one stream are safe.  Nothing in the array needs to
 *    start at zero; each call overwrites what it reads.
 *  - The grid must belong to the current device. */
#define AIDW_NOALLOC_MAX_QUERIES 65536
#define AIDW_NOALLOC_SCRATCH_BYTES (8u << 20)
aidw_status aidw_interpolate_noalloc(const aidw_grid *g, const float *qx, const float *qy,
                                     int64_t n_query, const aidw_params *p, void *out_z,
                                     void *out_alpha, aidw_stream_t stream);

/* The kNN of the authors' earlier GPU AIDW, which the paper improves on
 * (Sec. 3.1): one thread per query scans every data point and keeps its k
 * best distances in a sorted list (insertion with neighbour swaps), with the
 * data points staged through shared memory in tiles.  O(n_query * n_data).
 * Same outputs, float32 distance and (distance, index) order as aidw_knn, so
 * the two return identical results; kept as the baseline that measures the
 * grid search's gain (the paper's Table 3 comparison). */
aidw_status aidw_knn_bruteforce(const aidw_grid *g, const float *qx, const float *qy,
                                int64_t n_query, int k, int32_t *out_idx, float *out_dist,
                                float *out_robs, aidw_stream_t stream);

/* The grid kNN with the paper's own stop rule (Sec. 3.2.4, Step 2 and the
 * remark on Fig. 4): the level of cell expanding is the first L whose block
 * of (2L+1)^2 cells (clipped to the grid) holds at least k points, and the
 * search covers one level more, L+1; the result is the k nearest of the
 * points in that block.  This is not always the exact kNN (a point just
 * outside the widened block can be nearer than the k-th point inside it);
 * aidw_knn is exact.  Kept to measure how often the paper's rule misses.
 * Same arguments, outputs, float32 distances, (distance, index) order and
 * error behaviour as aidw_knn; distances are never below aidw_knn's. */
aidw_status aidw_knn_paper_rule(const aidw_grid *g, const float *qx, const float *qy,
                                int64_t n_query, int k, int32_t *out_idx, float *out_dist,
                                float *out_robs, aidw_stream_t stream);

/* Local AIDW: alpha exactly as aidw_interpolate (Eq. 2-6 from the k nearest
 * neighbours), but the weighted average of Eq. 1 taken over those k
 * neighbours only (n = k in Eq. 1's "data points used in interpolating")
 * instead of all data points.  O(n_query * k) after the kNN search; one
 * kernel, no scratch.  Coincident neighbours give their mean z.  Outputs as
 * aidw_interpolate (float32 or float64 by p->precision). */
aidw_status aidw_interpolate_local(const aidw_grid *g, const float *qx, const float *qy,
                                   int64_t n_query, const aidw_params *p, void *out_z,
                                   void *out_alpha, aidw_stream_t stream);

/* Caps the device memory the library holds at once from its pool (grids and
 * per-call scratch, not batch plans): a call that would pass the cap fails
 * with AIDW_ERR_OOM before any work.  bytes = 0 removes the cap.  *held (may
 * be NULL) receives the bytes held now.  A library service with no
 * counterpart in the paper (memory budgets, and testing the OOM path without
 * exhausting the GPU). */
aidw_status aidw_set_memory_limit(int64_t bytes, int64_t *held);

/* Test hook for the device-side timeout path (no counterpart in the paper).
 * Every wait of the weighting kernel for a shared-memory data tile is
 * bounded: at most 2000 tries, each suspending for up to ~1 ms.  After this
 * call the next weighting launch (aidw_interpolate, the no-alloc form or a
 * batch run; a launch being captured into a graph leaves the hook for the
 * next one) leaves the copy of one data tile unissued and bounds its waits
 * at `tries` (1..2000) tries, so the CTA that needs that tile gives up: it
 * latches AIDW_ERR_TIMEOUT, sets the launch's failure flag, waits (bounded)
 * for its own copies in flight and returns.  The GPU stays usable; every
 * prediction of that launch is NaN (the finalize step reads the flag);
 * aidw_grid_status (or aidw_batch_plan_status) reports the timeout. */
aidw_status aidw_test_expire_next_wait(int tries);

/* Short English name of a status code (static storage). */
const char *aidw_status_string(aidw_status s);

/* ---- stage timing ---------------------------------------------------------
 * When enabled, every call records CUDA events around each stage it
 * launches on its stream.  aidw_profile_read() waits for those events, adds
 * the elapsed milliseconds and launch counts per stage into ms[] and
 * launches[] (each AIDW_STAGE_COUNT long), then clears the record. */
typedef enum {
    AIDW_STAGE_GRID_BUILD = 0, /* bounding box .. cell-ordered points      */
    AIDW_STAGE_KNN = 1,        /* grid kNN + alpha                         */
    AIDW_STAGE_WEIGHT = 2,     /* all-points weighting (Eq. 1), stream-K   */
    AIDW_STAGE_FINALIZE = 3,   /* combine partial sums, divide             */
    AIDW_STAGE_BATCH = 4,      /* one aidw_batch_run (whole graph)         */
    AIDW_STAGE_COUNT = 5
} aidw_stage;

aidw_status aidw_profile_enable(int on);
aidw_status aidw_profile_read(double *ms, int64_t *launches);

/* Measures, on the current device, the sustained per-SM per-clock rate of
 * the three pipes the weighting stage uses: SFU log2 (lg2.approx), SFU exp2
 * (ex2.approx) and packed float32 FMA (lanes of fma.f32x2).  One CTA per SM
 * runs independent chains of each instruction for ~1 ms; rates come from
 * clock64(), so they do not depend on the clock speed.  Synchronous.
 * Measurement helper with no counterpart in the paper: the benchmark uses it
 * as the denominator of the weighting kernel's roofline. */
aidw_status aidw_probe_pipe_rates(double *lg2_per_sm_clk, double *ex2_per_sm_clk,
                                  double *ffma2_lanes_per_sm_clk);

/* Measures, on the current device, the rate (query/data pairs per SM per
 * clock) that the float32 weighting kernel's inner loop reaches when it runs
 * alone: the same compiled loop (default split: 2 of 8 exp2 on the FMA
 * pipe, 4 queries per thread, 256 threads) over a shared-memory tile filled
 * once, with no bulk copies, waits or barriers, ctas_per_sm (2: the kernel's
 * 128-register form; 3: an 80-register form) CTAs on every SM for ~1 ms,
 * timed with clock64() (independent of the clock speed).  The kernel's own
 * rate divided by this one tells how much its data pipeline and scheduling
 * lose against what its instruction mix allows.  Synchronous; allocates a
 * few KB of device memory for the duration of the call.  Returns
 * AIDW_ERR_INVALID_ARG for another ctas_per_sm or a NULL output, and
 * AIDW_ERR_CUDA if that many CTAs do not fit on an SM.  Measurement helper
 * with no counterpart in the paper. */
aidw_status aidw_probe_weight_loop(int ctas_per_sm, double *pairs_per_sm_clk);

/* Index checks of the bounds-checked build of this library
 * (libaidw_checked.so, built with -DAIDW_BOUNDS_CHECK; no GPU memory checker
 * can run here).  In that build the kernels test the indices they compute
 * (cells of points and queries, cell heads, scatter and fix-up
 * destinations, ring segments of the kNN, the source range of every
 * weighting tile copy, the partial-sum slots of the weighting and its
 * finalize) against the sizes of the arrays they index; a failed
 * test skips the access and is counted.  This call waits for the device,
 * then reports: *checked_build 1 in the checked build, 0 in the normal one
 * (whose kernels carry no checks); *violations the number of failed tests
 * since the library was loaded; *first the first one as (site << 48 |
 * index), or all ones if none.  Any pointer may be NULL.  Measurement and
 * test helper with no counterpart in the paper. */
aidw_status aidw_bounds_report(int *checked_build, uint64_t *violations, uint64_t *first);

/* Test hook of the index checks: one GPU thread evaluates the check of the
 * checked build on `index` against [0, n) (the test accesses no memory) and
 * writes 1 (in range) or 0 to *in_range (may be NULL).  In the checked build
 * a value out of range is recorded like a kernel's failed check (site 12);
 * in the normal build the check is the constant true.  Synchronous. */
aidw_status aidw_test_bounds_check(int64_t index, int64_t n, int *in_range);

/* Instruction mix of the float32 weighting loop (AIDW_FP32_COMP) that this
 * library launches, for roofline accounting (no counterpart in the paper).
 * Every (query, data point) pair needs one log2 and one exp2; of every
 * *products pairs of two consecutive inner steps of the loop, *poly_exp2
 * take the exp2 and *poly_lg2 the log2 from float32 polynomials on the FMA
 * pipe instead of the SFU.  fma_lanes[3] receives the FMA-pipe lane operations per pair of
 * the base loop, of one exp2 polynomial and of one log2 polynomial;
 * instr[3] the instructions per pair of the same three parts, not counting
 * the SFU instructions, loads and loop control (a packed two-lane
 * instruction counts as half an instruction per pair).  Any pointer may be
 * NULL.  Host only: no CUDA call. */
aidw_status aidw_weight_mix(int *products, int *poly_exp2, int *poly_lg2, double *fma_lanes,
                            double *instr);

#ifdef __cplusplus
}
#endif

#endif /* AIDW_H_ */
