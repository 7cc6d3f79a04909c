// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "aidw.h"
#include "bounds.cuh"

namespace aidw {

// ---------------------------------------------------------------------------
// Device-side description of a built grid (one per grid, in device memory).
// ---------------------------------------------------------------------------
struct GridDev {
    // bounding box as order-preserving integer encodings of float32 (written
    // by the last block of the bounding-box reduction)
    int enc_min_x, enc_min_y, enc_max_x, enc_max_y;
    double min_x, min_y, max_x, max_y;
    double area;        // A of Eq. 2
    double r_exp;       // Eq. 2
    double cw;          // cell width
    long long n_col, n_row, n_cells;
    // float32 forms for the cell-index fast path and the stop-test bounds:
    // min_x/min_y exactly (they are float32 values), 1/cw rounded to
    // nearest, cw rounded down and up
    float min_x_f, min_y_f, inv_cw_f, cw_rd, cw_ru, pad_f;
    long long n_data;
    int status;         // latched AIDW error bits (see StatusBit)
    int pad_;
};

enum StatusBit : int {
    kStatusNonfiniteData = 1,
    kStatusNonfiniteQuery = 2,
    kStatusTimeout = 4,
    kStatusCapacity = 8,
};

// Cell-ordered data point: x, y, z and the original index (bit pattern in w).
// 16 bytes so a tile of them is one bulk (TMA) copy.
struct __align__(16) Point { float x, y, z; int idx; };

// Points per tile of the weighting layout: the grid also stores its points
// as tiles of kWeightTile {-x[], -y[], z[]} float32 arrays (structure of
// arrays inside a tile, negated coordinates so that q + (-p) == q - p), which
// the weighting kernel streams into shared memory one tile per bulk copy.
constexpr int kWeightTile = 2048;

// Per-query result of the kNN stage consumed by the weighting stage.
struct QRec {
    double alpha;  // Eq. 6
    double hit_z;  // mean z of the data points at distance 0 (if any)
    float d1sq;    // smallest squared distance (float32 path)
    int n_hit;     // number of data points at distance 0
};

}  // namespace aidw

// Host-side grid handle (the opaque aidw_grid of the C ABI).
struct aidw_grid {
    void *block;                 // the one pool allocation holding the buffers below
    aidw::GridDev *dev;          // device struct
    aidw::Point *pts;            // [n_pad] cell-ordered points, padded
    int *cell_start;             // [cap + 1] head of each cell (int32), then the
                                 // build's scan records (grid_cell_start_ints)
    int *perm;                   // [n_data] original index at each position
    float *wt;                   // [n_wtiles][3][kWeightTile] weighting tiles
    float *zorig;                // [n_data] z in the caller's order (local AIDW)
    long long n_wtiles;          // ceil(n_data / kWeightTile)
    long long n_data;
    long long n_pad;             // n_data rounded up (padding points at +inf)
    long long cap_cells;         // capacity of cell_start minus one
    double cell_scale;
    double area_param;
    aidw::GridDev host_copy;     // the device record as it was when the build returned
    int device;
};

namespace aidw {

// Names the host-side span of a library call or stage for profilers (an
// NVTX range, e.g. `ncu --nvtx --nvtx-include "aidw_interpolate/"`); a no-op
// unless such a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---- launch helpers (defined in api.cu) -----------------------------------
aidw_status cuda_status(cudaError_t e);
// Stream-ordered device allocation from the library's own memory pool on the
// current device (freed memory stays in the pool for reuse).
cudaError_t lib_alloc(void **p, size_t bytes, cudaStream_t s);
void lib_free(void *p, cudaStream_t s);
// Stage timing: begin returns a handle (-1 when timing is off); end records
// the closing event and the number of kernels the stage launched.
int profile_begin(cudaStream_t s);
void profile_end(int handle, cudaStream_t s, int stage, int launches);

// ---- stages (defined in grid_build.cu, knn.cu, weight.cu) ------------------
long long grid_cells_capacity(long long n, double c);
// Ints to allocate for a grid's cell_start array of capacity cap (the cell
// heads plus the build's scan records and tickets).
long long grid_cell_start_ints(long long cap);
aidw_status grid_build_launch(aidw_grid *g, const float *x, const float *y, const float *z,
                              cudaStream_t s);

// Parameters of Eq. 4-6 passed by value to the kNN kernel.
struct AlphaParams {
    double level[5];
    double r_min, r_max;
    double area_override;  // > 0 replaces the grid's area in Eq. 2
    // float32 copies for the float32 path's Eq. 4-6 (pi / R_max as printed)
    float level_f[5];
    float r_min_f, r_max_f, pi_over_rmax_f, area_override_f;
};

// One kNN job: a grid, its queries and where the results go.  Batched
// launches index a device array of these by flat query number (q_base).
struct KnnJob {
    const GridDev *g;
    const Point *pts;
    const int *start;
    const float *qx, *qy;
    QRec *recs;
    int *out_idx;
    float *out_dist;
    float *out_robs;
    void *out_alpha;
    const float *zorig;  // z by original index (local AIDW)
    void *out_zlocal;    // local AIDW prediction (Eq. 1 over the k nearest); or null
    const int *order;    // queries in grid-cell order (thread i takes order[i]); or null
    long long nq;
    long long q_base;
    int k;
    int stop_rule;  // kStopExact, or kStopPaperLevel (the paper's rule, Sec. 3.2.4)
};

// Stop rules of the ring search.
constexpr int kStopExact = 0;       // stop once no unvisited cell can hold a nearer point
constexpr int kStopPaperLevel = 1;  // first level whose block holds k points, plus one

// One weighting job.  Units of all jobs are numbered job after job
// (unit_base), and so are their query tiles (tile_base) and queries (q_base).
struct WJob {
    const float *wt;   // weighting tiles (float32 path)
    const Point *pts;  // AoS points (float64 path)
    const float *qx, *qy;
    const QRec *recs;
    void *out_z;
    long long n_data, n_pad;
    long long D, T;    // data units (pieces of weighting tiles), query tiles
    int piece_shift;   // a data unit is 1/2^piece_shift of a weighting tile
                       // (float32 path; 0 on the float64 path)
    long long nq;
    long long unit_base, tile_base, q_base;
};

// kNN (+ alpha): fills recs (if not null) and the optional public outputs;
// out_zlocal (if not null) receives the local AIDW prediction.  sort allows
// visiting the queries in grid-cell order (takes pool memory).
aidw_status knn_launch(const aidw_grid *g, const float *qx, const float *qy, long long n_query,
                       int k, bool fp64, const AlphaParams &ap, QRec *recs, int *out_idx,
                       float *out_dist, float *out_robs, void *out_alpha, cudaStream_t s,
                       void *out_zlocal = nullptr, bool sort = true,
                       int stop_rule = kStopExact);

// Brute-force kNN over all data points of the grid (the paper's original
// per-thread algorithm, kept as a baseline).
aidw_status knn_launch_brute(const aidw_grid *g, const float *qx, const float *qy,
                             long long n_query, int k, int *out_idx, float *out_dist,
                             float *out_robs, cudaStream_t s);

// Batched kNN over jobs[0, n_jobs) (device array) whose k all need at most
// kmax (8, 16, 24 or 32) slots; total_q is the sum of their query counts.
// threads: block size of the thread-per-query kernel, or 0 for the
// warp-per-query kernel.
int knn_default_threads(int k);
aidw_status knn_launch_batch(const KnnJob *jobs, int n_jobs, long long total_q, int kmax,
                             bool fp64, const AlphaParams &ap, int threads, cudaStream_t s);

// Data tiles per job of the weighting stage and query tiles per job.
long long weight_data_tiles(long long n_data, long long n_pad, bool fp64);
long long weight_query_tile(bool fp64);
// Persistent CTAs the weighting kernel runs with on `device`.
int weight_resident_ctas(int device, bool fp64);

// Batched weighting + finalize over jobs[0, n_jobs) (device array), total_u
// units and total_q queries; part holds (total tiles + G) * query-tile
// partial records; bounds (device, G + 1 entries, strictly increasing from
// 0 to total_u; or null for equal unit counts) is the first unit of each
// CTA's share; fail is one int of device memory for the launch's failure
// flag (zeroed by the launch; a CTA whose wait expires sets it and the
// finalize then writes NaN).
aidw_status weight_launch_batch(const WJob *jobs, int n_jobs, long long total_u,
                                long long total_q, bool fp64, void *part, long long G,
                                const long long *bounds, int *status, int *fail, int device,
                                cudaStream_t s, long long n_slots);
// Points of data tile d that the weighting kernel processes for a job of
// n_data points (n_pad padded): the cost of one unit.
long long weight_unit_points(long long n_data, long long n_pad, long long d, bool fp64);
size_t weight_partial_bytes(bool fp64);  // bytes of one query tile's partials
// Instruction mix of the float32 weighting loop (see aidw_weight_mix).
void weight_mix(int *products, int *poly_exp2, int *poly_lg2, double *fma_lanes, double *instr);
// Test hook: the next weighting launch leaves one data-tile copy unissued and
// bounds its waits at `tries` tries, so a wait expires.
void weight_expire_next_wait(int tries);

// Weighting (stream-K over all data points) + finalize.  Allocates its
// partial-sum scratch with cudaMallocAsync on s.
aidw_status weight_launch(const aidw_grid *g, const float *qx, const float *qy,
                          long long n_query, bool fp64, const QRec *recs, void *out_z,
                          cudaStream_t s);

// Same computation as weight_launch, with the partial sums and the launch's
// failure flag (the last 256 bytes) in caller-given device memory
// (scratch_bytes long) instead of an allocation; the number of persistent
// CTAs is reduced if needed so that the partials fit.  Returns
// AIDW_ERR_INVALID_ARG if not even one CTA's partials fit.
aidw_status weight_launch_scratch(const aidw_grid *g, const float *qx, const float *qy,
                                  long long n_query, bool fp64, const QRec *recs, void *out_z,
                                  void *scratch, size_t scratch_bytes, cudaStream_t s);

namespace api_detail {
// Argument checks and Eq. 4-6 parameters shared by the entry points (api.cu).
aidw_status check_params(const aidw_params *p, bool need_k);
AlphaParams alpha_params(const aidw_params *p);
}  // namespace api_detail

}  // namespace aidw
