// C ABI entry points (include/aidw.h): argument checks, grid ownership,
// per-call scratch and stage timing.  All arithmetic happens in the kernels
// of grid_build.cu, knn.cu and weight.cu.
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "aidw_internal.cuh"

namespace aidw {

namespace bounds {
// Readers of the index-check records of every translation unit (registered
// at load time by the checked build; empty in the normal build).
static std::mutex g_readers_mu;
static std::vector<Reader> &readers()
{
    static std::vector<Reader> v;
    return v;
}
bool add_reader(Reader r)
{
    std::lock_guard<std::mutex> lk(g_readers_mu);
    readers().push_back(r);
    return true;
}
}  // namespace bounds

aidw_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return AIDW_OK;
    if (e == cudaErrorMemoryAllocation) return AIDW_ERR_OOM;
    return AIDW_ERR_CUDA;
}

// ---- memory pool ---------------------------------------------------------------
// One stream-ordered pool per device, private to the library, that keeps
// freed blocks (release threshold unbounded): grids and per-call scratch
// come from it, so repeated builds and calls reuse memory without a
// cudaMalloc (which can synchronise the device) after the first use.
namespace api_detail {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaMemPool_t pool_for(int device)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (device < 0 || device >= 64) return nullptr;
    if (!g_pools[device]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[device] = pool;
    }
    return g_pools[device];
}
}  // namespace api_detail

// Optional cap on the bytes the library holds from its pool at once (0: no
// cap); allocations past it fail with cudaErrorMemoryAllocation (reported as
// AIDW_ERR_OOM) without touching the device.
namespace api_detail {
std::mutex g_cap_mu;
size_t g_cap_bytes = 0;
size_t g_held_bytes = 0;
std::unordered_map<void *, size_t> g_sizes;
}  // namespace api_detail

cudaError_t lib_alloc(void **p, size_t bytes, cudaStream_t s)
{
    using namespace api_detail;
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    {
        std::lock_guard<std::mutex> lk(g_cap_mu);
        if (g_cap_bytes && g_held_bytes + bytes > g_cap_bytes) return cudaErrorMemoryAllocation;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = pool_for(device);
    e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lk(g_cap_mu);
    g_sizes[*p] = bytes;
    g_held_bytes += bytes;
    return e;
}

void lib_free(void *p, cudaStream_t s)
{
    using namespace api_detail;
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_cap_mu);
        auto it = g_sizes.find(p);
        if (it != g_sizes.end()) {
            g_held_bytes -= it->second;
            g_sizes.erase(it);
        }
    }
    cudaFreeAsync(p, s);
}

// ---- stage timing ------------------------------------------------------------
namespace api_detail {

struct ProfRec {
    cudaEvent_t a, b;
    int stage;
    int launches;
    bool closed;
};

std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;

cudaEvent_t take_event()
{
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace api_detail
using namespace api_detail;

int profile_begin(cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return -1;  // no timing events inside a graph capture
    }
    ProfRec r;
    r.a = take_event();
    r.b = take_event();
    r.stage = -1;
    r.launches = 0;
    r.closed = false;
    cudaEventRecord(r.a, s);
    g_prof.push_back(r);
    return (int)g_prof.size() - 1;
}

void profile_end(int handle, cudaStream_t s, int stage, int launches)
{
    if (handle < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (handle >= (int)g_prof.size()) return;
    ProfRec &r = g_prof[handle];
    cudaEventRecord(r.b, s);
    r.stage = stage;
    r.launches = launches;
    r.closed = true;
}

}  // namespace aidw

using namespace aidw;
using namespace aidw::api_detail;

namespace aidw {
namespace api_detail {

constexpr long long kMaxPoints = 0x7fffffffLL - 64;  // int32 indices + padding

bool finite(double v) { return isfinite(v) != 0; }

aidw_status check_params(const aidw_params *p, bool need_k)
{
    if (!p) return AIDW_ERR_INVALID_ARG;
    for (int i = 0; i < 5; ++i)
        if (!finite(p->alpha[i]) || !(p->alpha[i] > 0.0)) return AIDW_ERR_INVALID_ARG;
    if (!finite(p->r_min) || !finite(p->r_max) || !(p->r_max > 0.0) || !(p->r_min >= 0.0) ||
        !(p->r_min < p->r_max))
        return AIDW_ERR_INVALID_ARG;
    if (!finite(p->area) || !finite(p->cell_scale)) return AIDW_ERR_INVALID_ARG;
    if (p->cell_scale > 0.0 && (p->cell_scale < 1.0 / 64.0 || p->cell_scale > 64.0))
        return AIDW_ERR_INVALID_ARG;
    if (p->precision != AIDW_FP32_COMP && p->precision != AIDW_FP64_PLAIN)
        return AIDW_ERR_INVALID_ARG;
    if (need_k && (p->k < 1 || p->k > AIDW_MAX_K)) return AIDW_ERR_K_RANGE;
    return AIDW_OK;
}

// Cell width scale used when the caller passes cell_scale <= 0.  Grid build
// + kNN on GB300, n = m = 1M, ms at scales 1 / 1.5 / 2 / 3:
//   k = 10 uniform 2.11 / 1.79 / 1.73 / 1.63, clustered 4.05 / 2.66 / 2.31 / 2.35
//   k = 32 uniform 7.89 / 6.10 / 5.36 / 4.93, clustered 18.2 / 11.7 / 8.66 / 6.90
// Wider cells than the paper's (scale 1) mean fewer, longer contiguous runs
// of points per ring, which costs less than the extra distances they add.
double auto_cell_scale(int k)
{
    return k <= 16 ? 2.0 : 3.0;
}

AlphaParams alpha_params(const aidw_params *p)
{
    AlphaParams ap;
    for (int i = 0; i < 5; ++i) ap.level[i] = p->alpha[i];
    ap.r_min = p->r_min;
    ap.r_max = p->r_max;
    ap.area_override = p->area > 0.0 ? p->area : 0.0;
    for (int i = 0; i < 5; ++i) ap.level_f[i] = (float)p->alpha[i];
    ap.r_min_f = (float)p->r_min;
    ap.r_max_f = (float)p->r_max;
    ap.pi_over_rmax_f = (float)(3.141592653589793 / p->r_max);
    ap.area_override_f = (float)ap.area_override;
    return ap;
}

__global__ void k_widen(const int *__restrict__ a, long long n, int64_t *__restrict__ b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int64_t)a[i];
}

}  // namespace api_detail
}  // namespace aidw

extern "C" {

void aidw_params_default(aidw_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->k = 10;
    for (int i = 0; i < 5; ++i) p->alpha[i] = (double)(i + 1);
    p->r_min = 0.0;
    p->r_max = 2.0;
    p->area = 0.0;
    p->cell_scale = 0.0;
    p->precision = AIDW_FP32_COMP;
}

const char *aidw_status_string(aidw_status s)
{
    switch (s) {
    case AIDW_OK: return "ok";
    case AIDW_ERR_INVALID_ARG: return "invalid argument";
    case AIDW_ERR_K_RANGE: return "k out of range (1..32 and <= number of data points)";
    case AIDW_ERR_NONFINITE: return "non-finite coordinate or value";
    case AIDW_ERR_OOM: return "device allocation failed";
    case AIDW_ERR_CUDA: return "CUDA error";
    case AIDW_ERR_TIMEOUT: return "bounded device wait expired";
    }
    return "unknown status";
}

aidw_status aidw_grid_build(const float *x, const float *y, const float *z, int64_t n_data,
                            const aidw_params *p, aidw_stream_t stream, aidw_grid **out)
{
    NvtxRange nvtx_("aidw_grid_build");
    if (!out) return AIDW_ERR_INVALID_ARG;
    *out = nullptr;
    if (!x || !y || !z || n_data < 1 || n_data > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    const aidw_status ps = check_params(p, false);
    if (ps != AIDW_OK) return ps;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    aidw_grid *g = new (std::nothrow) aidw_grid();
    if (!g) return AIDW_ERR_OOM;
    memset(g, 0, sizeof(*g));
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return AIDW_ERR_CUDA;
    }
    g->n_data = n_data;
    g->n_pad = (n_data + 31) / 32 * 32;
    g->cell_scale = p->cell_scale > 0.0 ? p->cell_scale : auto_cell_scale(p->k);
    g->area_param = p->area > 0.0 ? p->area : 0.0;
    g->cap_cells = grid_cells_capacity(n_data, g->cell_scale);

    // every buffer of the grid in one pool allocation (256-byte aligned parts)
    g->n_wtiles = (n_data + kWeightTile - 1) / kWeightTile;
    size_t off = 0;
    const auto part = [&off](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_dev = part(sizeof(GridDev));
    const size_t o_pts = part(sizeof(Point) * (size_t)g->n_pad);
    const size_t o_start = part(sizeof(int) * (size_t)grid_cell_start_ints(g->cap_cells));
    const size_t o_perm = part(sizeof(int) * (size_t)n_data);
    const size_t o_wt = part(sizeof(float) * 3 * kWeightTile * (size_t)g->n_wtiles);
    const size_t o_zorig = part(sizeof(float) * (size_t)n_data);
    cudaError_t e = lib_alloc(&g->block, off, s);
    if (e == cudaSuccess) {
        unsigned char *base = static_cast<unsigned char *>(g->block);
        g->dev = reinterpret_cast<GridDev *>(base + o_dev);
        g->pts = reinterpret_cast<Point *>(base + o_pts);
        g->cell_start = reinterpret_cast<int *>(base + o_start);
        g->perm = reinterpret_cast<int *>(base + o_perm);
        g->wt = reinterpret_cast<float *>(base + o_wt);
        g->zorig = reinterpret_cast<float *>(base + o_zorig);
        e = cudaMemcpyAsync(g->zorig, z, sizeof(float) * (size_t)n_data, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        aidw_grid_destroy(g);
        return e == cudaErrorMemoryAllocation ? AIDW_ERR_OOM : AIDW_ERR_CUDA;
    }
    aidw_status st = grid_build_launch(g, x, y, z, s);
    if (st == AIDW_OK) {
        // one stream-ordered read of the device record (dimensions, status)
        st = cuda_status(cudaMemcpyAsync(&g->host_copy, g->dev, sizeof(GridDev),
                                         cudaMemcpyDeviceToHost, s));
        if (st == AIDW_OK) st = cuda_status(cudaStreamSynchronize(s));
    }
    if (st == AIDW_OK) {
        const int status = g->host_copy.status;
        if (st == AIDW_OK && (status & kStatusNonfiniteData)) st = AIDW_ERR_NONFINITE;
        if (st == AIDW_OK && (status & kStatusCapacity)) st = AIDW_ERR_INVALID_ARG;
        if (st == AIDW_OK && (status & kStatusTimeout)) st = AIDW_ERR_TIMEOUT;
    }
    if (st != AIDW_OK) {
        aidw_grid_destroy(g);
        return st;
    }
    *out = g;
    return AIDW_OK;
}

aidw_status aidw_grid_status(aidw_grid *g)
{
    if (!g) return AIDW_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_status(e);
    int status = 0;
    e = cudaMemcpy(&status, &g->dev->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    const int zero = 0;
    cudaMemcpy(&g->dev->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (status & kStatusTimeout) return AIDW_ERR_TIMEOUT;
    if (status & (kStatusNonfiniteData | kStatusNonfiniteQuery)) return AIDW_ERR_NONFINITE;
    if (status & kStatusCapacity) return AIDW_ERR_INVALID_ARG;
    return AIDW_OK;
}

aidw_status aidw_grid_destroy(aidw_grid *g)
{
    if (!g) return AIDW_ERR_INVALID_ARG;
    aidw_status st = AIDW_OK;
    if (g->dev) {
        // drain all work that may still read the grid, then report its status
        // as aidw_grid_status would (the record dies with the grid: no reset)
        cudaError_t e = cudaDeviceSynchronize();
        int status = 0;
        if (e == cudaSuccess)
            e = cudaMemcpy(&status, &g->dev->status, sizeof(int), cudaMemcpyDeviceToHost);
        st = e != cudaSuccess                                          ? cuda_status(e)
             : (status & kStatusTimeout)                               ? AIDW_ERR_TIMEOUT
             : (status & (kStatusNonfiniteData | kStatusNonfiniteQuery)) ? AIDW_ERR_NONFINITE
             : (status & kStatusCapacity)                              ? AIDW_ERR_INVALID_ARG
                                                                       : AIDW_OK;
    }
    // the device is idle (drained above); return the buffers to the pool
    lib_free(g->block, nullptr);
    delete g;
    return st;
}

aidw_status aidw_grid_get_info(const aidw_grid *g, aidw_grid_info *info)
{
    if (!g || !info) return AIDW_ERR_INVALID_ARG;
    const GridDev &d = g->host_copy;  // dimensions are fixed once the build returns
    info->n_data = d.n_data;
    info->n_col = d.n_col;
    info->n_row = d.n_row;
    info->n_cells = d.n_cells;
    info->min_x = d.min_x;
    info->min_y = d.min_y;
    info->max_x = d.max_x;
    info->max_y = d.max_y;
    info->area = d.area;
    info->r_exp = d.r_exp;
    info->cell_width = d.cw;
    info->cell_scale = g->cell_scale;
    return AIDW_OK;
}


aidw_status aidw_grid_export(const aidw_grid *g, int64_t *cell_start, int32_t *perm,
                             aidw_stream_t stream)
{
    if (!g) return AIDW_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cell_start) {
        aidw_grid_info info;
        const aidw_status st = aidw_grid_get_info(g, &info);
        if (st != AIDW_OK) return st;
        const long long n = info.n_cells + 1;
        k_widen<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->cell_start, n, cell_start);
    }
    if (perm)
        cudaMemcpyAsync(perm, g->perm, sizeof(int32_t) * (size_t)g->n_data,
                        cudaMemcpyDeviceToDevice, s);
    return cuda_status(cudaGetLastError());
}

aidw_status aidw_knn(const aidw_grid *g, const float *qx, const float *qy, int64_t n_query,
                     int k, int32_t *out_idx, float *out_dist, float *out_robs,
                     aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_knn");
    if (!g || n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    if (k < 1 || k > AIDW_MAX_K || k > g->n_data) return AIDW_ERR_K_RANGE;
    if (n_query == 0) return AIDW_OK;
    if (!qx || !qy) return AIDW_ERR_INVALID_ARG;
    aidw_params p;
    aidw_params_default(&p);
    return knn_launch(g, qx, qy, n_query, k, false, alpha_params(&p), nullptr, out_idx, out_dist,
                      out_robs, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

aidw_status aidw_interpolate(const aidw_grid *g, const float *qx, const float *qy,
                             int64_t n_query, const aidw_params *p, void *out_z,
                             void *out_alpha, aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_interpolate");
    if (!g || n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    const aidw_status ps = check_params(p, true);
    if (ps != AIDW_OK) return ps;
    if (p->k > g->n_data) return AIDW_ERR_K_RANGE;
    if (n_query == 0) return AIDW_OK;
    if (!qx || !qy || !out_z) return AIDW_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = p->precision == AIDW_FP64_PLAIN;
    QRec *recs = nullptr;
    if (lib_alloc((void **)&recs, sizeof(QRec) * (size_t)n_query, s) != cudaSuccess)
        return AIDW_ERR_OOM;
    aidw_status st = knn_launch(g, qx, qy, n_query, p->k, fp64, alpha_params(p), recs, nullptr,
                                nullptr, nullptr, out_alpha, s);
    if (st == AIDW_OK) st = weight_launch(g, qx, qy, n_query, fp64, recs, out_z, s);
    lib_free(recs, s);
    return st;
}

aidw_status aidw_knn_bruteforce(const aidw_grid *g, const float *qx, const float *qy,
                                int64_t n_query, int k, int32_t *out_idx, float *out_dist,
                                float *out_robs, aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_knn_bruteforce");
    if (!g || n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    if (k < 1 || k > AIDW_MAX_K || k > g->n_data) return AIDW_ERR_K_RANGE;
    if (n_query == 0) return AIDW_OK;
    if (!qx || !qy) return AIDW_ERR_INVALID_ARG;
    return knn_launch_brute(g, qx, qy, n_query, k, out_idx, out_dist, out_robs,
                            reinterpret_cast<cudaStream_t>(stream));
}

aidw_status aidw_knn_paper_rule(const aidw_grid *g, const float *qx, const float *qy,
                                int64_t n_query, int k, int32_t *out_idx, float *out_dist,
                                float *out_robs, aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_knn_paper_rule");
    if (!g || n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    if (k < 1 || k > AIDW_MAX_K || k > g->n_data) return AIDW_ERR_K_RANGE;
    if (n_query == 0) return AIDW_OK;
    if (!qx || !qy) return AIDW_ERR_INVALID_ARG;
    aidw_params p;
    aidw_params_default(&p);
    return knn_launch(g, qx, qy, n_query, k, false, alpha_params(&p), nullptr, out_idx, out_dist,
                      out_robs, nullptr, reinterpret_cast<cudaStream_t>(stream), nullptr, true,
                      kStopPaperLevel);
}

aidw_status aidw_interpolate_local(const aidw_grid *g, const float *qx, const float *qy,
                                   int64_t n_query, const aidw_params *p, void *out_z,
                                   void *out_alpha, aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_interpolate_local");
    if (!g || n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    const aidw_status ps = check_params(p, true);
    if (ps != AIDW_OK) return ps;
    if (p->k > g->n_data) return AIDW_ERR_K_RANGE;
    if (n_query == 0) return AIDW_OK;
    if (!qx || !qy || !out_z) return AIDW_ERR_INVALID_ARG;
    return knn_launch(g, qx, qy, n_query, p->k, p->precision == AIDW_FP64_PLAIN,
                      alpha_params(p), nullptr, nullptr, nullptr, nullptr, out_alpha,
                      reinterpret_cast<cudaStream_t>(stream), out_z);
}

aidw_status aidw_interpolate_host(const float *x, const float *y, const float *z, int64_t n_data,
                                  const float *qx, const float *qy, int64_t n_query,
                                  const aidw_params *p, void *out_z, void *out_alpha,
                                  aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_interpolate_host");
    if (!x || !y || !z || n_data < 1 || n_data > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    if (n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    aidw_status st = check_params(p, true);
    if (st != AIDW_OK) return st;
    if (p->k > n_data) return AIDW_ERR_K_RANGE;
    if (n_query > 0 && (!qx || !qy || !out_z)) return AIDW_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)n_data, m = (size_t)n_query;
    const size_t es = p->precision == AIDW_FP64_PLAIN ? sizeof(double) : sizeof(float);
    // one pool block: inputs (x, y, z, qx, qy), then the outputs 8-byte aligned
    const size_t in_bytes = sizeof(float) * (3 * n + 2 * m);
    const size_t out_off = (in_bytes + 255) / 256 * 256;
    const size_t out_bytes = es * m * (out_alpha ? 2 : 1);
    unsigned char *d = nullptr;
    if (lib_alloc((void **)&d, out_off + out_bytes, s) != cudaSuccess) return AIDW_ERR_OOM;
    float *dx = reinterpret_cast<float *>(d), *dy = dx + n, *dz = dy + n, *dqx = dz + n,
          *dqy = dqx + m;
    void *dout = d + out_off;
    void *dalpha = out_alpha ? d + out_off + es * m : nullptr;
    cudaError_t e = cudaMemcpyAsync(dx, x, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dz, z, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && m)
        e = cudaMemcpyAsync(dqx, qx, sizeof(float) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && m)
        e = cudaMemcpyAsync(dqy, qy, sizeof(float) * m, cudaMemcpyHostToDevice, s);
    st = cuda_status(e);
    aidw_grid *g = nullptr;
    if (st == AIDW_OK) st = aidw_grid_build(dx, dy, dz, n_data, p, stream, &g);
    if (st == AIDW_OK && m) st = aidw_interpolate(g, dqx, dqy, n_query, p, dout, dalpha, stream);
    if (st == AIDW_OK && m)
        st = cuda_status(cudaMemcpyAsync(out_z, dout, es * m, cudaMemcpyDeviceToHost, s));
    if (st == AIDW_OK && m && out_alpha)
        st = cuda_status(cudaMemcpyAsync(out_alpha, dalpha, es * m, cudaMemcpyDeviceToHost, s));
    if (st == AIDW_OK) st = cuda_status(cudaStreamSynchronize(s));
    if (g) {
        const aidw_status gs = aidw_grid_destroy(g);  // latched device errors of the call
        if (st == AIDW_OK) st = gs;
    }
    lib_free(d, s);
    return st;
}

aidw_status aidw_shard_range(int64_t n_query, int shard, int n_shards, int64_t *begin,
                             int64_t *end)
{
    if (!begin || !end || n_query < 0 || n_shards < 1 || shard < 0 || shard >= n_shards)
        return AIDW_ERR_INVALID_ARG;
    // the first n_query % n_shards shards take one query more
    const int64_t q = n_query / n_shards, r = n_query % n_shards;
    *begin = (int64_t)shard * q + (shard < r ? shard : r);
    *end = *begin + q + (shard < r ? 1 : 0);
    return AIDW_OK;
}

aidw_status aidw_interpolate_shard(const aidw_grid *g, const float *qx, const float *qy,
                                   int64_t n_query, int shard, int n_shards,
                                   const aidw_params *p, void *out_z, void *out_alpha,
                                   aidw_stream_t stream)
{
    NvtxRange nvtx_("aidw_interpolate_shard");
    if (!g || n_query < 0 || n_query > kMaxPoints) return AIDW_ERR_INVALID_ARG;
    int64_t b = 0, e = 0;
    aidw_status st = aidw_shard_range(n_query, shard, n_shards, &b, &e);
    if (st != AIDW_OK) return st;
    st = check_params(p, true);
    if (st != AIDW_OK) return st;
    if (p->k > g->n_data) return AIDW_ERR_K_RANGE;
    if (e == b) return AIDW_OK;
    if (!qx || !qy || !out_z) return AIDW_ERR_INVALID_ARG;
    const size_t es = p->precision == AIDW_FP64_PLAIN ? sizeof(double) : sizeof(float);
    void *oz = static_cast<unsigned char *>(out_z) + es * (size_t)b;
    void *oa = out_alpha ? static_cast<unsigned char *>(out_alpha) + es * (size_t)b : nullptr;
    return aidw_interpolate(g, qx + b, qy + b, e - b, p, oz, oa, stream);
}

aidw_status aidw_set_memory_limit(int64_t bytes, int64_t *held)
{
    if (bytes < 0) return AIDW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_cap_mu);
    g_cap_bytes = (size_t)bytes;
    if (held) *held = (int64_t)g_held_bytes;
    return AIDW_OK;
}

aidw_status aidw_test_expire_next_wait(int tries)
{
    if (tries < 1 || tries > 2000) return AIDW_ERR_INVALID_ARG;
    weight_expire_next_wait(tries);
    return AIDW_OK;
}

aidw_status aidw_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return AIDW_OK;
}

aidw_status aidw_profile_read(double *ms, int64_t *launches)
{
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof);
    }
    aidw_status st = AIDW_OK;
    for (const ProfRec &r : recs) {
        if (r.closed && r.stage >= 0 && r.stage < AIDW_STAGE_COUNT) {
            cudaError_t e = cudaEventSynchronize(r.b);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
            if (e != cudaSuccess) {
                st = cuda_status(e);
            } else {
                if (ms) ms[r.stage] += (double)t;
                if (launches) launches[r.stage] += r.launches;
            }
        }
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const ProfRec &r : recs) {
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    return st;
}

aidw_status aidw_bounds_report(int *checked_build, uint64_t *violations, uint64_t *first)
{
    using namespace aidw::bounds;
    std::vector<Reader> rs;
    {
        std::lock_guard<std::mutex> lk(g_readers_mu);
        rs = readers();
    }
    if (checked_build) *checked_build = rs.empty() ? 0 : 1;
    unsigned long long total = 0, f = ~0ull;
    if (!rs.empty() && cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return AIDW_ERR_CUDA;
    }
    for (Reader r : rs) {
        unsigned long long c = 0, fi = ~0ull;
        r(&c, &fi);
        total += c;
        if (f == ~0ull) f = fi;
    }
    if (violations) *violations = total;
    if (first) *first = f;
    return AIDW_OK;
}

}  // extern "C"
