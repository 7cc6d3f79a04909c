// Batched AIDW: many independent interpolation jobs (each its own data
// points, queries and k) in one pass.
//
// A plan fixes the job shapes (n_data, n_query, k per job) and carves one
// pooled device allocation into every job's grid arrays, kNN records and the
// weighting partial sums.  Each step of the path is one launch over all jobs:
// the grid-build kernels (the single-grid build's five: bounding box with the
// dimensions from its last block, keys, single-pass scan, scatter, fix-up
// with padding; each job has its own tickets and scan records) map blocks
// to jobs through per-job block prefixes,
// the kNN kernels (one per top-k width class) map queries to jobs, and the
// weighting stage is a single persistent stream-K launch over the units of
// all jobs, so jobs of very different sizes share the GPU evenly.  The launch
// sequence is captured once into a CUDA graph; each run uploads the job
// table (the caller's pointers) and replays the graph.  The cell width scale
// and the kNN block size can be chosen by a measuring autotuner.
#include <string.h>

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "aidw_device.cuh"
#include "aidw_internal.cuh"
#include "grid_device.cuh"

namespace aidw {
namespace {

using namespace gridk;

// Everything the batched build kernels need about one job.
struct BJob {
    const float *x, *y, *z;
    GridDev *g;
    Point *pts;
    int *start;
    int *perm;
    float *wt;
    int *key, *rank;
    Point *tmp;  // points in cell order, unstable within a cell
    float *bpart;                      // bounding-box records, 5 per block
    // zeroed at the start of every run, after the cell heads in the start
    // region: the scan's chunk records and the tickets (bounding box, scan)
    unsigned long long *flags;
    int *tickets;
    long long n, n_pad, n_wpad, cap;
    long long nchunks;      // scan chunks of start[0, cap]
    long long bbox_blocks;  // blocks of the bounding-box reduction
    long long blk_pt, blk_bbox, blk_scan, blk_fp;  // first block in each launch
    double cell_scale, area_param;
    // queries, sorted by grid cell before the kNN (see knn.cu); qflags and
    // qticket follow the counts in the query-count region
    const float *qx, *qy;
    long long m;
    int *qcount, *qkey, *qrank, *qorder;
    unsigned long long *qflags;
    int *qticket;
    long long blk_q;
};

// Job whose first block (field F of the table) is the largest <= b.
template <long long BJob::*F>
__device__ __forceinline__ int job_of_block(const BJob *__restrict__ jobs, int n_jobs, long long b)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].*F <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) k_b_bbox_dims(const BJob *__restrict__ jobs,
                                                          int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_bbox>(jobs, n_jobs, blockIdx.x)];
    bbox_dims_block(J.x, J.y, J.z, J.n, J.bpart, J.tickets, J.g, J.cell_scale, J.area_param, J.cap,
                    blockIdx.x - J.blk_bbox, J.bbox_blocks);
}

__global__ void __launch_bounds__(kThreads) k_b_keys(const BJob *__restrict__ jobs, int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_pt>(jobs, n_jobs, blockIdx.x)];
    const long long i = (blockIdx.x - J.blk_pt) * kThreads + threadIdx.x;
    if (i >= J.n || grid_failed(J.g)) return;
    key_one(i, J.x, J.y, J.g, J.start, J.key, J.rank);
}

// One chunk of one job's single-pass scan; the chunk comes from the job's
// own ticket, so a block waits only on earlier chunks of its job.
__global__ void __launch_bounds__(kThreads) k_b_scan(const BJob *__restrict__ jobs, int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_scan>(jobs, n_jobs, blockIdx.x)];
    scan_lookback_block(J.start, J.cap + 1, J.flags, J.tickets + 1, &J.g->status);
}

__global__ void __launch_bounds__(kThreads) k_b_scatter(const BJob *__restrict__ jobs, int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_pt>(jobs, n_jobs, blockIdx.x)];
    const long long i = (blockIdx.x - J.blk_pt) * kThreads + threadIdx.x;
    if (i >= J.n || grid_failed(J.g)) return;
    scatter_point(i, J.x, J.y, J.z, J.start, J.key, J.rank, J.tmp, J.g, J.n);
}

__global__ void __launch_bounds__(kThreads) k_b_fixup_pad(const BJob *__restrict__ jobs,
                                                          int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_fp>(jobs, n_jobs, blockIdx.x)];
    const long long s = (blockIdx.x - J.blk_fp) * kThreads + threadIdx.x;
    if (s < J.n) {
        if (!grid_failed(J.g)) fixup_one(s, J.g, J.start, J.tmp, J.pts, J.perm, J.wt, J.n);
    } else if (s < (J.n_pad > J.n_wpad ? J.n_pad : J.n_wpad)) {
        pad_one(s, J.n_pad, J.n_wpad, J.pts, J.wt);
    }
}

// ---- queries of every job in grid-cell order (as the single-grid kNN) ----
__global__ void __launch_bounds__(kThreads) k_b_qkeys(const BJob *__restrict__ jobs, int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_q>(jobs, n_jobs, blockIdx.x)];
    const long long i = (blockIdx.x - J.blk_q) * kThreads + threadIdx.x;
    if (i >= J.m || grid_failed(J.g)) return;
    float x = J.qx[i], y = J.qy[i];
    if (!isfinite(x) || !isfinite(y)) x = y = 0.0f;  // flagged by the kNN kernel
    key_one_xy(i, x, y, J.g, J.qcount, J.qkey, J.qrank);
}

__global__ void __launch_bounds__(kThreads) k_b_qscan(const BJob *__restrict__ jobs, int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_scan>(jobs, n_jobs, blockIdx.x)];
    scan_lookback_block(J.qcount, J.cap + 1, J.qflags, J.qticket, &J.g->status);
}

__global__ void __launch_bounds__(kThreads) k_b_qscatter(const BJob *__restrict__ jobs, int n_jobs)
{
    const BJob &J = jobs[job_of_block<&BJob::blk_q>(jobs, n_jobs, blockIdx.x)];
    const long long i = (blockIdx.x - J.blk_q) * kThreads + threadIdx.x;
    if (i >= J.m || grid_failed(J.g)) return;
    scatter_one(i, J.qcount, J.qkey, J.qrank, J.qorder, J.m);
}

__global__ void k_b_status(const BJob *__restrict__ jobs, int n_jobs, int *status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_jobs) {
        const int s = jobs[j].g->status;
        if (s) atomicOr(status, s);
    }
}

constexpr double kTuneScales[] = {1.0, 1.5, 2.0, 3.0, 4.0};
constexpr int kTuneThreads[] = {0, 64, 128, 256};  // 0: warp per query
constexpr double kMinScale = 1.0;

// Top-k width classes: a job's kNN runs in the launch of the smallest class
// whose register slots hold its k.
constexpr int kClasses = AIDW_BATCH_CLASSES;
constexpr int kClassKmax[kClasses] = {8, 16, 24, 32};
inline int class_of(int k)
{
    for (int c = 0; c < kClasses; ++c)
        if (k <= kClassKmax[c]) return c;
    return kClasses - 1;
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }
inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

}  // namespace
}  // namespace aidw

using namespace aidw;

struct aidw_batch_plan {
    int n_jobs = 0;
    int device = 0;
    bool fp64 = false;
    bool tuned_scale = false;   // cell scale chosen by the caller
    aidw_params params;
    AlphaParams ap;
    // per top-k class: cell-width scale of its jobs' grids and kNN block size
    double class_scale[kClasses] = {};
    int class_threads[kClasses] = {};
    int tuned = 0;  // 0: defaults, 1: measured by the tuner, 2: from the tuning cache
    std::vector<long long> n, m;
    std::vector<int> k, jclass;

    // per-job layout (host copies of the device tables without caller pointers)
    std::vector<BJob> bj;
    std::vector<KnnJob> kj;   // ordered by top-k class
    std::vector<WJob> wj;
    std::vector<int> korder;  // job index of each kj entry
    int kclass_begin[kClasses + 1] = {};
    long long kclass_q[kClasses] = {};
    long long total_pt_blocks = 0, total_bbox_blocks = 0, total_chunks = 0, total_fp_blocks = 0;
    long long total_q_blocks = 0;
    int *qcount_pool = nullptr;
    long long total_u = 0, total_q = 0, total_tiles = 0, G = 1;
    long long start_ints = 0;

    unsigned char *pool = nullptr;
    size_t pool_bytes = 0;
    int *start_pool = nullptr;
    BJob *d_bj = nullptr;
    KnnJob *d_kj = nullptr;
    WJob *d_wj = nullptr;
    GridDev *d_grids = nullptr;
    int *d_status = nullptr;
    void *d_part = nullptr;
    long long *d_bounds = nullptr;  // [G + 1] cost-balanced stream-K shares

    unsigned char *h_stage = nullptr;  // pinned copy of the three tables
    size_t stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;

    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the kNN launches of the classes run as parallel branches (side streams
    // forked from and joined back to the launching stream)
    cudaStream_t side[kClasses] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kClasses] = {};
};

namespace {

// Whether the per-class kNN launches run one after another on the launching
// stream (default) or as parallel branches forked from it
// (AIDW_BATCH_BRANCHES=1).  On the 512-job workload the branches shorten
// build + kNN on a plain stream (27.4 -> 24.1 ms) but lengthen the replayed
// graph's step (662.1 -> 663.7 ms, two runs each on one GB300), so the
// graph keeps the serial form.
bool batch_knn_branches()
{
    static const bool on = [] {
        const char *e = getenv("AIDW_BATCH_BRANCHES");
        return e && atoi(e) != 0;
    }();
    return on;
}

// Recomputes the cell-width dependent part of the layout (caps, chunks).
void layout_cells(aidw_batch_plan *P)
{
    long long blk_scan = 0;
    for (int j = 0; j < P->n_jobs; ++j) {
        BJob &b = P->bj[j];
        b.cell_scale = P->class_scale[P->jclass[j]];
        b.cap = grid_cells_capacity(b.n, b.cell_scale);
        b.nchunks = cdiv(b.cap + 1, kScanChunk);
        b.blk_scan = blk_scan;
        blk_scan += b.nchunks;
    }
    P->total_chunks = blk_scan;
}

// Fills the caller's pointers into the staged tables and uploads them.
aidw_status upload_tables(aidw_batch_plan *P, const aidw_job *jobs, cudaStream_t s)
{
    if (P->stage_pending) {
        const cudaError_t e = cudaEventSynchronize(P->stage_done);
        if (e != cudaSuccess) return cuda_status(e);
        P->stage_pending = false;
    }
    BJob *hb = reinterpret_cast<BJob *>(P->h_stage);
    KnnJob *hk = reinterpret_cast<KnnJob *>(P->h_stage + sizeof(BJob) * P->n_jobs);
    WJob *hw = reinterpret_cast<WJob *>(P->h_stage + (sizeof(BJob) + sizeof(KnnJob)) * P->n_jobs);
    for (int j = 0; j < P->n_jobs; ++j) {
        hb[j] = P->bj[j];
        hb[j].x = jobs[j].x;
        hb[j].y = jobs[j].y;
        hb[j].z = jobs[j].z;
        hb[j].qx = jobs[j].qx;
        hb[j].qy = jobs[j].qy;
        hw[j] = P->wj[j];
        hw[j].qx = jobs[j].qx;
        hw[j].qy = jobs[j].qy;
        hw[j].out_z = jobs[j].out_z;
    }
    for (int i = 0; i < P->n_jobs; ++i) {
        const int j = P->korder[i];
        hk[i] = P->kj[i];
        hk[i].qx = jobs[j].qx;
        hk[i].qy = jobs[j].qy;
    }
    cudaError_t e = cudaMemcpyAsync(P->d_bj, P->h_stage, P->stage_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(P->stage_done, s);
    if (e != cudaSuccess) return cuda_status(e);
    P->stage_pending = true;
    return AIDW_OK;
}

// Enqueues the whole path on s (used for capture and for tuning).
aidw_status enqueue(aidw_batch_plan *P, cudaStream_t s, bool knn_only)
{
    const int J = P->n_jobs;
    const unsigned jb = (unsigned)cdiv(J, 128);
    // cell counts, scan records and tickets of every job start at zero
    cudaMemsetAsync(P->start_pool, 0, sizeof(int) * (size_t)P->start_ints, s);
    k_b_bbox_dims<<<(unsigned)P->total_bbox_blocks, kThreads, 0, s>>>(P->d_bj, J);
    k_b_keys<<<(unsigned)P->total_pt_blocks, kThreads, 0, s>>>(P->d_bj, J);
    k_b_scan<<<(unsigned)P->total_chunks, kThreads, 0, s>>>(P->d_bj, J);
    k_b_scatter<<<(unsigned)P->total_pt_blocks, kThreads, 0, s>>>(P->d_bj, J);
    k_b_fixup_pad<<<(unsigned)P->total_fp_blocks, kThreads, 0, s>>>(P->d_bj, J);
    if (P->total_q_blocks > 0) {
        cudaMemsetAsync(P->qcount_pool, 0, sizeof(int) * (size_t)P->start_ints, s);
        k_b_qkeys<<<(unsigned)P->total_q_blocks, kThreads, 0, s>>>(P->d_bj, J);
        k_b_qscan<<<(unsigned)P->total_chunks, kThreads, 0, s>>>(P->d_bj, J);
        k_b_qscatter<<<(unsigned)P->total_q_blocks, kThreads, 0, s>>>(P->d_bj, J);
    }
    aidw_status st = cuda_status(cudaGetLastError());
    // one kNN launch per class, one after another on s; optionally
    // (batch_knn_branches) all but the first with queries run on side streams
    // forked from s after the build and joined back before the weighting
    bool forked = false;
    int first = -1;
    for (int c = 0; c < kClasses && st == AIDW_OK; ++c) {
        const int b = P->kclass_begin[c], e = P->kclass_begin[c + 1];
        if (e == b) continue;
        cudaStream_t cs = s;
        if (first < 0 || !batch_knn_branches()) {
            first = c;
        } else {
            if (!forked) {
                st = cuda_status(cudaEventRecord(P->fork, s));
                forked = true;
            }
            if (st == AIDW_OK) st = cuda_status(cudaStreamWaitEvent(P->side[c], P->fork, 0));
            cs = P->side[c];
        }
        if (st == AIDW_OK)
            st = knn_launch_batch(P->d_kj + b, e - b, P->kclass_q[c], kClassKmax[c], P->fp64,
                                  P->ap, P->class_threads[c], cs);
        if (st == AIDW_OK && cs != s) {
            st = cuda_status(cudaEventRecord(P->join[c], cs));
            if (st == AIDW_OK) st = cuda_status(cudaStreamWaitEvent(s, P->join[c], 0));
        }
    }
    if (st != AIDW_OK || knn_only) return st;
    st = weight_launch_batch(P->d_wj, J, P->total_u, P->total_q, P->fp64, P->d_part, P->G,
                             P->d_bounds, P->d_status, P->d_status + 1, P->device, s,
                             P->total_tiles + P->G);
    if (st != AIDW_OK) return st;
    k_b_status<<<jb, 128, 0, s>>>(P->d_bj, J, P->d_status);
    return cuda_status(cudaGetLastError());
}

aidw_status capture(aidw_batch_plan *P)
{
    NvtxRange nvtx_("graph capture");
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e);
    const aidw_status st = enqueue(P, P->cap_stream, false);
    e = cudaStreamEndCapture(P->cap_stream, &graph);
    if (st != AIDW_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphInstantiate(&P->exec, graph, 0);
    cudaGraphDestroy(graph);
    return cuda_status(e);
}

aidw_status check_jobs(const aidw_batch_plan *P, const aidw_job *jobs, int n_jobs)
{
    if (!jobs || n_jobs != P->n_jobs) return AIDW_ERR_INVALID_ARG;
    for (int j = 0; j < n_jobs; ++j) {
        const aidw_job &J = jobs[j];
        const int k = J.k > 0 ? J.k : P->params.k;
        if (J.n_data != P->n[j] || J.n_query != P->m[j] || k != P->k[j]) return AIDW_ERR_INVALID_ARG;
        if (!J.x || !J.y || !J.z) return AIDW_ERR_INVALID_ARG;
        if (J.n_query > 0 && (!J.qx || !J.qy || !J.out_z)) return AIDW_ERR_INVALID_ARG;
    }
    return AIDW_OK;
}

// ---- tuning cache ---------------------------------------------------------------
// The tuner's choices are kept per process, keyed by what they depend on: the
// precision, the GPU's SM count, a cell scale fixed by the caller, and the
// histogram of the jobs' shapes (log2 buckets of n and m, and k).  A plan
// created for jobs with a cached key starts with that tuning.  With
// AIDW_TUNE_CACHE=<file> the entries are also read from and appended to that
// file, one JSON object per line:
//   {"key": "...", "cell_scale": [s8, s16, s24, s32],
//    "knn_threads": [t8, t16, t24, t32], "build_knn_ms": ms}
// so later processes reuse them (a later line for the same key wins).
struct TuneVal {
    double scale[kClasses];
    int threads[kClasses];
    double ms;
};
std::mutex g_cache_mu;
std::map<std::string, TuneVal> g_cache;
bool g_cache_loaded = false;

std::string tune_key(const aidw_batch_plan *P)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
    std::map<std::tuple<int, int, int>, int> hist;
    for (int j = 0; j < P->n_jobs; ++j) {
        const int bn = (int)ceil(log2((double)P->n[j]));
        const int bm = P->m[j] > 0 ? (int)ceil(log2((double)P->m[j])) : -1;
        ++hist[std::make_tuple(bn, bm, P->k[j])];
    }
    std::string key = "v1 fp64=" + std::to_string(P->fp64 ? 1 : 0) + " sms=" + std::to_string(sms) +
                      " scale=" + std::to_string(P->tuned_scale ? P->params.cell_scale : 0.0);
    for (const auto &h : hist)
        key += " " + std::to_string(std::get<0>(h.first)) + "/" + std::to_string(std::get<1>(h.first)) +
               "/" + std::to_string(std::get<2>(h.first)) + "x" + std::to_string(h.second);
    return key;
}

void cache_load_file()
{
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const char *path = getenv("AIDW_TUNE_CACHE");
    if (!path || !*path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        // the fixed shape written by cache_store; anything else is skipped
        const std::string k0 = "{\"key\": \"";
        if (line.compare(0, k0.size(), k0) != 0) continue;
        const size_t kend = line.find('"', k0.size());
        if (kend == std::string::npos) continue;
        TuneVal v;
        const int got = sscanf(line.c_str() + kend,
                               "\", \"cell_scale\": [%lf, %lf, %lf, %lf], "
                               "\"knn_threads\": [%d, %d, %d, %d], \"build_knn_ms\": %lf}",
                               &v.scale[0], &v.scale[1], &v.scale[2], &v.scale[3],
                               &v.threads[0], &v.threads[1], &v.threads[2], &v.threads[3], &v.ms);
        if (got == 9) g_cache[line.substr(k0.size(), kend - k0.size())] = v;
    }
}

bool cache_lookup(aidw_batch_plan *P)
{
    const std::string key = tune_key(P);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache_load_file();
    const auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    for (int c = 0; c < kClasses; ++c) {
        P->class_scale[c] = it->second.scale[c];
        P->class_threads[c] = it->second.threads[c];
    }
    return true;
}

void cache_store(const aidw_batch_plan *P, double ms)
{
    const std::string key = tune_key(P);
    TuneVal v;
    for (int c = 0; c < kClasses; ++c) {
        v.scale[c] = P->class_scale[c];
        v.threads[c] = P->class_threads[c];
    }
    v.ms = ms;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache_load_file();
    g_cache[key] = v;
    const char *path = getenv("AIDW_TUNE_CACHE");
    if (!path || !*path) return;
    char buf[256];
    snprintf(buf, sizeof buf,
             "\", \"cell_scale\": [%.17g, %.17g, %.17g, %.17g], \"knn_threads\": [%d, %d, %d, %d], "
             "\"build_knn_ms\": %.6g}\n",
             v.scale[0], v.scale[1], v.scale[2], v.scale[3], v.threads[0], v.threads[1],
             v.threads[2], v.threads[3], v.ms);
    std::ofstream f(path, std::ios::app);
    f << "{\"key\": \"" << key << buf;
}

// Cost-balanced stream-K shares of the weighting launch.  The units of all
// jobs, in launch order, are split into G contiguous shares of about equal
// cost, where a unit costs the points it processes (its data tile, part-filled
// at a job's edge) plus a fixed overhead, and the first unit of a query-tile
// row (a new segment: job look-up, query loads) a little more.  Equal unit
// counts left the CTAs whose shares hold many small jobs' part-filled tiles
// idle at the end (measured on the 512-job workload: per-SM active cycles,
// max / mean 1.0074).  Shares are kept non-empty (strictly increasing
// boundaries), which the partial-sum slots (tile + CTA) rely on.
void stream_k_bounds(const aidw_batch_plan *P, std::vector<long long> &b)
{
    constexpr double kUnitCost = 16.0, kSegmentCost = 16.0;  // in points
    const long long G = P->G, U = P->total_u;
    b.assign((size_t)G + 1, 0);
    b[(size_t)G] = U;
    if (U <= G) {
        for (long long k = 0; k < G; ++k) b[(size_t)k] = std::min(k, U);
        return;
    }
    const int J = P->n_jobs;
    std::vector<double> row(J, 0.0);
    double total = 0.0;
    for (int j = 0; j < J; ++j) {
        const WJob &w = P->wj[j];
        double r = kSegmentCost;
        for (long long d = 0; d < w.D; ++d)
            r += (double)weight_unit_points(w.n_data, w.n_pad, d, P->fp64) + kUnitCost;
        row[j] = r;
        total += (double)w.T * r;
    }
    long long k = 1;
    double base = 0.0;
    for (int j = 0; j < J && k < G; ++j) {
        const WJob &w = P->wj[j];
        const double jc = (double)w.T * row[j];
        while (k < G && base + jc >= (double)k * total / (double)G) {
            const double x = (double)k * total / (double)G - base;
            long long t = std::min<long long>(w.T - 1, (long long)(x / row[j]));
            double rem = x - (double)t * row[j] - kSegmentCost;
            long long d = 0;
            while (d < w.D - 1) {
                const double c = (double)weight_unit_points(w.n_data, w.n_pad, d, P->fp64) + kUnitCost;
                if (rem < c) break;
                rem -= c;
                ++d;
            }
            b[(size_t)k] = w.unit_base + t * w.D + d;
            ++k;
        }
        base += jc;
    }
    for (; k < G; ++k) b[(size_t)k] = U;
    for (long long i = 1; i < G; ++i) b[(size_t)i] = std::max(b[(size_t)i], b[(size_t)i - 1] + 1);
    for (long long i = G - 1; i >= 1; --i) b[(size_t)i] = std::min(b[(size_t)i], b[(size_t)i + 1] - 1);
}

void free_plan(aidw_batch_plan *P)
{
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    for (int c = 0; c < kClasses; ++c) {
        if (P->side[c]) cudaStreamDestroy(P->side[c]);
        if (P->join[c]) cudaEventDestroy(P->join[c]);
    }
    if (P->fork) cudaEventDestroy(P->fork);
    if (P->stage_done) cudaEventDestroy(P->stage_done);
    if (P->h_stage) cudaFreeHost(P->h_stage);
    if (P->pool) cudaFree(P->pool);
    delete P;
}

}  // namespace

extern "C" {

aidw_status aidw_batch_plan_create(const aidw_job *jobs, int n_jobs, const aidw_params *p,
                                   aidw_batch_plan **out)
{
    NvtxRange nvtx_("aidw_batch_plan_create");
    if (!out) return AIDW_ERR_INVALID_ARG;
    *out = nullptr;
    if (!jobs || n_jobs < 1 || n_jobs > (1 << 20)) return AIDW_ERR_INVALID_ARG;
    aidw_status st = api_detail::check_params(p, false);
    if (st != AIDW_OK) return st;
    for (int j = 0; j < n_jobs; ++j) {
        const long long n = jobs[j].n_data, m = jobs[j].n_query;
        const int k = jobs[j].k > 0 ? jobs[j].k : p->k;
        if (n < 1 || n > 0x7fffffffLL - 1024 || m < 0 || m > 0x7fffffffLL) return AIDW_ERR_INVALID_ARG;
        if (k < 1 || k > AIDW_MAX_K || k > n) return AIDW_ERR_K_RANGE;
    }
    aidw_batch_plan *P = new (std::nothrow) aidw_batch_plan();
    if (!P) return AIDW_ERR_OOM;
    P->n_jobs = n_jobs;
    P->params = *p;
    P->ap = api_detail::alpha_params(p);
    P->fp64 = p->precision == AIDW_FP64_PLAIN;
    P->tuned_scale = p->cell_scale > 0.0;
    // defaults as the single-grid path (scale 2 up to k = 16, 3 above); the
    // tuner may change them
    for (int c = 0; c < kClasses; ++c) {
        P->class_scale[c] = p->cell_scale > 0.0 ? p->cell_scale : (kClassKmax[c] <= 16 ? 2.0 : 3.0);
        P->class_threads[c] = knn_default_threads(kClassKmax[c]);
    }
    cudaGetDevice(&P->device);
    P->n.resize(n_jobs);
    P->m.resize(n_jobs);
    P->k.resize(n_jobs);
    P->jclass.resize(n_jobs);
    P->bj.assign(n_jobs, BJob());
    P->wj.assign(n_jobs, WJob());
    for (int j = 0; j < n_jobs; ++j) {
        P->n[j] = jobs[j].n_data;
        P->m[j] = jobs[j].n_query;
        P->k[j] = jobs[j].k > 0 ? jobs[j].k : p->k;
        P->jclass[j] = class_of(P->k[j]);
    }

    // ---- sizes and block prefixes ----
    const long long qt = weight_query_tile(P->fp64);
    long long blk_pt = 0, blk_bbox = 0, blk_fp = 0, ubase = 0, tbase = 0, qbase = 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    // the start region is sized for the smallest scale the tuner may pick
    const double scale_for_cap = P->tuned_scale ? p->cell_scale : kMinScale;
    std::vector<size_t> o_pts(n_jobs), o_wt(n_jobs), o_start(n_jobs), o_perm(n_jobs),
        o_key(n_jobs), o_rank(n_jobs), o_tmp(n_jobs), o_bpart(n_jobs), o_rec(n_jobs),
        o_qkey(n_jobs), o_qrank(n_jobs), o_qorder(n_jobs);
    // inside each job's share of the start (and query-count) region, in ints:
    // the cell heads, then the scan records, then the tickets
    std::vector<long long> flags_off(n_jobs), tick_off(n_jobs);
    long long blk_q = 0;
    const size_t o_grids = take(sizeof(GridDev) * (size_t)n_jobs);
    long long start_ints = 0;
    for (int j = 0; j < n_jobs; ++j) {
        BJob &b = P->bj[j];
        memset(&b, 0, sizeof(b));
        b.n = P->n[j];
        b.n_pad = cdiv(b.n, 32) * 32;
        const long long nwt = cdiv(b.n, kWeightTile);
        b.n_wpad = nwt * kWeightTile;
        b.area_param = p->area > 0.0 ? p->area : 0.0;
        b.bbox_blocks = std::min<long long>(cdiv(b.n, kThreads), 64);
        b.blk_pt = blk_pt;
        blk_pt += cdiv(b.n, kThreads);
        b.blk_bbox = blk_bbox;
        blk_bbox += b.bbox_blocks;
        b.blk_fp = blk_fp;  // fix-up of the n points and the padding after them
        blk_fp += cdiv(std::max(b.n, std::max(b.n_pad, b.n_wpad)), kThreads);
        const long long cap_max = grid_cells_capacity(b.n, scale_for_cap);
        o_pts[j] = take(sizeof(Point) * (size_t)b.n_pad);
        o_wt[j] = take(sizeof(float) * 3 * (size_t)b.n_wpad);
        o_perm[j] = take(sizeof(int) * (size_t)b.n);
        o_key[j] = take(sizeof(int) * (size_t)b.n);
        o_rank[j] = take(sizeof(int) * (size_t)b.n);
        o_tmp[j] = take(sizeof(Point) * (size_t)b.n);
        o_bpart[j] = take(sizeof(float) * 5 * (size_t)b.bbox_blocks);
        o_rec[j] = take(sizeof(QRec) * (size_t)std::max<long long>(P->m[j], 1));
        const size_t mq = (size_t)std::max<long long>(P->m[j], 1);
        o_qkey[j] = take(sizeof(int) * mq);
        o_qrank[j] = take(sizeof(int) * mq);
        o_qorder[j] = take(sizeof(int) * mq);
        b.m = P->m[j];
        b.blk_q = blk_q;
        blk_q += cdiv(b.m, kThreads);
        o_start[j] = (size_t)start_ints;  // in ints, inside the start region
        flags_off[j] = (cap_max + 2) / 2 * 2;
        tick_off[j] = flags_off[j] + 2 * cdiv(cap_max + 1, kScanChunk);
        start_ints += (tick_off[j] + 4 + 63) / 64 * 64;

        WJob &w = P->wj[j];
        memset(&w, 0, sizeof(w));
        w.n_data = b.n;
        w.n_pad = b.n_pad;
        w.D = weight_data_tiles(b.n, b.n_pad, P->fp64);
        w.nq = P->m[j];
        w.T = cdiv(w.nq, qt);
        w.unit_base = ubase;
        w.tile_base = tbase;
        w.q_base = qbase;
        ubase += w.T * w.D;
        tbase += w.T;
        qbase += w.nq;
    }
    P->total_pt_blocks = blk_pt;
    P->total_bbox_blocks = blk_bbox;
    P->total_fp_blocks = blk_fp;
    P->total_q_blocks = blk_q;
    P->total_u = ubase;
    P->total_tiles = tbase;
    P->total_q = qbase;
    P->start_ints = start_ints;
    P->G = std::max<long long>(1, std::min<long long>(weight_resident_ctas(P->device, P->fp64),
                                                      std::max<long long>(ubase, 1)));
    const size_t o_startreg = take(sizeof(int) * (size_t)start_ints);
    const size_t o_qcountreg = take(sizeof(int) * (size_t)start_ints);
    const size_t o_part = take(weight_partial_bytes(P->fp64) * (size_t)(P->total_tiles + P->G));
    const size_t o_bounds = take(sizeof(long long) * (size_t)(P->G + 1));
    const size_t o_tables = take((sizeof(BJob) + sizeof(KnnJob) + sizeof(WJob)) * (size_t)n_jobs);
    const size_t o_status = take(2 * sizeof(int));  // latched status, launch failure flag
    P->pool_bytes = off;

    cudaError_t e = cudaMalloc((void **)&P->pool, P->pool_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&P->h_stage,
                                             (sizeof(BJob) + sizeof(KnnJob) + sizeof(WJob)) * (size_t)n_jobs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->stage_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
    for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
        e = cudaStreamCreateWithFlags(&P->side[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join[c], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(P);
        return e == cudaErrorMemoryAllocation ? AIDW_ERR_OOM : AIDW_ERR_CUDA;
    }
    unsigned char *base = P->pool;
    P->d_grids = reinterpret_cast<GridDev *>(base + o_grids);
    P->start_pool = reinterpret_cast<int *>(base + o_startreg);
    P->qcount_pool = reinterpret_cast<int *>(base + o_qcountreg);
    P->d_part = base + o_part;
    P->d_bounds = reinterpret_cast<long long *>(base + o_bounds);
    P->d_bj = reinterpret_cast<BJob *>(base + o_tables);
    P->d_kj = reinterpret_cast<KnnJob *>(base + o_tables + sizeof(BJob) * n_jobs);
    P->d_wj = reinterpret_cast<WJob *>(base + o_tables + (sizeof(BJob) + sizeof(KnnJob)) * n_jobs);
    P->d_status = reinterpret_cast<int *>(base + o_status);
    P->stage_bytes = (sizeof(BJob) + sizeof(KnnJob) + sizeof(WJob)) * (size_t)n_jobs;
    for (int j = 0; j < n_jobs; ++j) {
        BJob &b = P->bj[j];
        b.g = P->d_grids + j;
        b.pts = reinterpret_cast<Point *>(base + o_pts[j]);
        b.wt = reinterpret_cast<float *>(base + o_wt[j]);
        b.perm = reinterpret_cast<int *>(base + o_perm[j]);
        b.key = reinterpret_cast<int *>(base + o_key[j]);
        b.rank = reinterpret_cast<int *>(base + o_rank[j]);
        b.tmp = reinterpret_cast<Point *>(base + o_tmp[j]);
        b.bpart = reinterpret_cast<float *>(base + o_bpart[j]);
        b.start = P->start_pool + o_start[j];
        b.flags = reinterpret_cast<unsigned long long *>(b.start + flags_off[j]);
        b.tickets = b.start + tick_off[j];
        b.qcount = P->qcount_pool + o_start[j];
        b.qflags = reinterpret_cast<unsigned long long *>(b.qcount + flags_off[j]);
        b.qticket = b.qcount + tick_off[j];
        b.qkey = reinterpret_cast<int *>(base + o_qkey[j]);
        b.qrank = reinterpret_cast<int *>(base + o_qrank[j]);
        b.qorder = reinterpret_cast<int *>(base + o_qorder[j]);
        WJob &w = P->wj[j];
        w.wt = b.wt;
        w.pts = b.pts;
        w.recs = reinterpret_cast<QRec *>(base + o_rec[j]);
    }
    layout_cells(P);

    // kNN table ordered by top-k class (8, 16, 24, 32 slots)
    P->korder.clear();
    P->kj.clear();
    for (int c = 0; c < kClasses; ++c) {
        P->kclass_begin[c] = (int)P->korder.size();
        long long qb = 0;
        for (int j = 0; j < n_jobs; ++j) {
            if (P->jclass[j] != c || P->m[j] == 0) continue;
            KnnJob kj;
            memset(&kj, 0, sizeof(kj));
            kj.g = P->bj[j].g;
            kj.pts = P->bj[j].pts;
            kj.start = P->bj[j].start;
            kj.recs = const_cast<QRec *>(P->wj[j].recs);
            kj.order = P->bj[j].qorder;
            kj.nq = P->m[j];
            kj.q_base = qb;
            kj.k = P->k[j];
            qb += P->m[j];
            P->kj.push_back(kj);
            P->korder.push_back(j);
        }
        P->kclass_q[c] = qb;
    }
    P->kclass_begin[kClasses] = (int)P->korder.size();
    // jobs without queries still need a kNN table slot for the upload layout
    while ((int)P->kj.size() < n_jobs) {
        KnnJob kj;
        memset(&kj, 0, sizeof(kj));
        P->kj.push_back(kj);
        P->korder.push_back(0);
    }
    {
        std::vector<long long> bounds;
        stream_k_bounds(P, bounds);
        e = cudaMemcpy(P->d_bounds, bounds.data(), sizeof(long long) * bounds.size(),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_plan(P);
            return AIDW_ERR_CUDA;
        }
    }
    // a tuning measured earlier for jobs of the same shapes
    if (cache_lookup(P)) {
        P->tuned = 2;
        layout_cells(P);
    }
    // warm the weighting kernel's attributes before any capture
    weight_resident_ctas(P->device, P->fp64);
    *out = P;
    return AIDW_OK;
}

aidw_status aidw_batch_run(aidw_batch_plan *plan, const aidw_job *jobs, aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_batch_run");
    if (!plan) return AIDW_ERR_INVALID_ARG;
    aidw_status st = check_jobs(plan, jobs, jobs ? plan->n_jobs : 0);
    if (st != AIDW_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!plan->exec) {
        st = capture(plan);
        if (st != AIDW_OK) return st;
    }
    st = upload_tables(plan, jobs, s);
    if (st != AIDW_OK) return st;
    const int prof = profile_begin(s);
    st = cuda_status(cudaGraphLaunch(plan->exec, s));
    profile_end(prof, s, AIDW_STAGE_BATCH, 1);
    return st;
}

aidw_status aidw_batch_plan_tune(aidw_batch_plan *plan, const aidw_job *jobs,
                                 aidw_stream_t stream, double *best_ms)
{
    NvtxRange nvtx_("aidw_batch_plan_tune");
    if (!plan) return AIDW_ERR_INVALID_ARG;
    aidw_status st = check_jobs(plan, jobs, jobs ? plan->n_jobs : 0);
    if (st != AIDW_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double old_scale[kClasses];
    int old_threads[kClasses];
    for (int c = 0; c < kClasses; ++c) {
        old_scale[c] = plan->class_scale[c];
        old_threads[c] = plan->class_threads[c];
    }
    // grid build + kNN of all jobs with the current choices (second of two runs)
    auto measure = [&](double *ms_out) -> aidw_status {
        layout_cells(plan);
        aidw_status r = upload_tables(plan, jobs, s);
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && r == AIDW_OK; ++rep) {
            cudaEventRecord(a, s);
            r = enqueue(plan, s, true);
            cudaEventRecord(b, s);
            if (cudaEventSynchronize(b) != cudaSuccess) r = AIDW_ERR_CUDA;
            cudaEventElapsedTime(&ms, a, b);
        }
        *ms_out = ms;
        return r;
    };
    // coordinate descent over the top-k classes: for each class that has
    // queries, the cell scale of its jobs' grids (unless the caller fixed
    // it), then the kNN block size, keeping whatever lowers the total
    double best = 0.0;
    st = measure(&best);
    for (int c = 0; c < kClasses && st == AIDW_OK; ++c) {
        if (plan->kclass_begin[c + 1] == plan->kclass_begin[c]) continue;
        if (!plan->tuned_scale) {
            const double keep = plan->class_scale[c];
            double bsc = keep;
            for (double sc : kTuneScales) {
                if (sc == keep) continue;
                plan->class_scale[c] = sc;
                double ms = 0.0;
                st = measure(&ms);
                if (st != AIDW_OK) break;
                if (ms < best) {
                    best = ms;
                    bsc = sc;
                }
            }
            plan->class_scale[c] = bsc;
        }
        const int keep_t = plan->class_threads[c];
        int bth = keep_t;
        for (int th : kTuneThreads) {
            if (th == keep_t || st != AIDW_OK) continue;
            plan->class_threads[c] = th;
            double ms = 0.0;
            st = measure(&ms);
            if (st != AIDW_OK) break;
            if (ms < best) {
                best = ms;
                bth = th;
            }
        }
        plan->class_threads[c] = bth;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != AIDW_OK) {
        for (int c = 0; c < kClasses; ++c) {
            plan->class_scale[c] = old_scale[c];
            plan->class_threads[c] = old_threads[c];
        }
    } else {
        plan->tuned = 1;
        cache_store(plan, best);
    }
    layout_cells(plan);
    if (plan->exec) {
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
    }
    if (best_ms) *best_ms = best;
    return st;
}

// The class holding most queries (what aidw_batch_plan_get reports).
static int main_class(const aidw_batch_plan *plan)
{
    int best = 0;
    for (int c = 1; c < kClasses; ++c)
        if (plan->kclass_q[c] > plan->kclass_q[best]) best = c;
    return best;
}

aidw_status aidw_batch_plan_get(const aidw_batch_plan *plan, double *cell_scale,
                                int *knn_threads, int64_t *total_pairs, int64_t *pool_bytes)
{
    if (!plan) return AIDW_ERR_INVALID_ARG;
    const int c = main_class(plan);
    if (cell_scale) *cell_scale = plan->class_scale[c];
    if (knn_threads) *knn_threads = plan->class_threads[c];
    if (total_pairs) {
        long long t = 0;
        for (int j = 0; j < plan->n_jobs; ++j) t += plan->n[j] * plan->m[j];
        *total_pairs = t;
    }
    if (pool_bytes) *pool_bytes = (int64_t)plan->pool_bytes;
    return AIDW_OK;
}

aidw_status aidw_batch_plan_get_classes(const aidw_batch_plan *plan, int *kmax,
                                        double *cell_scale, int *knn_threads, int64_t *queries,
                                        int *source)
{
    if (!plan) return AIDW_ERR_INVALID_ARG;
    for (int c = 0; c < kClasses; ++c) {
        if (kmax) kmax[c] = kClassKmax[c];
        if (cell_scale) cell_scale[c] = plan->class_scale[c];
        if (knn_threads) knn_threads[c] = plan->class_threads[c];
        if (queries) queries[c] = plan->kclass_q[c];
    }
    if (source) *source = plan->tuned;
    return AIDW_OK;
}

aidw_status aidw_batch_plan_status(aidw_batch_plan *plan)
{
    if (!plan) return AIDW_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    const int zero = 0;
    cudaMemcpy(plan->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (status & kStatusTimeout) return AIDW_ERR_TIMEOUT;
    if (status & (kStatusNonfiniteData | kStatusNonfiniteQuery)) return AIDW_ERR_NONFINITE;
    if (status & kStatusCapacity) return AIDW_ERR_INVALID_ARG;
    return AIDW_OK;
}

aidw_status aidw_batch_plan_destroy(aidw_batch_plan *plan)
{
    if (!plan) return AIDW_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    free_plan(plan);
    return AIDW_OK;
}

aidw_status aidw_batch(const aidw_job *jobs, int n_jobs, const aidw_params *p,
                       aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_batch");
    aidw_batch_plan *plan = nullptr;
    aidw_status st = aidw_batch_plan_create(jobs, n_jobs, p, &plan);
    if (st != AIDW_OK) return st;
    st = aidw_batch_run(plan, jobs, stream);
    if (st == AIDW_OK) st = cuda_status(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    if (st == AIDW_OK) st = aidw_batch_plan_status(plan);
    aidw_batch_plan_destroy(plan);
    return st;
}

}  // extern "C"
