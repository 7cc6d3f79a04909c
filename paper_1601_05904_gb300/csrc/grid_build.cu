// Even-grid build (Sec. 3.2.1-3.2.3, 4.1.1-4.1.3 of arXiv 1601.05904).
//
// The paper builds the grid with Thrust: minmax_element for the bounding
// box, a key kernel, sort_by_key, then reduce_by_key / unique_by_key for the
// count and head of every cell (Fig. 3).  Here the same result comes from a
// counting sort in five plain kernels and one memset, all on the caller's
// stream and without a host round trip (the cell-array capacity is a
// function of n alone):
//
//   memset        cell counts, scan records and tickets to zero
//   k_bbox_dims   min/max of x and y (and a non-finite check of x, y, z);
//                 the last block computes A, r_exp (Eq. 2), the cell
//                 width, nCol and nRow and writes the grid record
//   k_keys        cell of each point + histogram (atomic) -> rank in cell
//   k_scan        exclusive scan of the histogram = head of each cell
//                 (single pass, decoupled look-back)
//   k_scatter     point index to head + rank (unstable within a cell)
//   k_fixup_pad   stable order within each cell + write the cell-ordered
//                 float4 points {x, y, z, index}; padding points at +inf
//                 after the last one
//
// All kernels are memory-bound; each reads or writes its arrays once with
// coalesced accesses except the scatter/fixup steps, whose targets are
// random by nature.
#include <algorithm>

#include "aidw_device.cuh"
#include "aidw_internal.cuh"
#include "grid_device.cuh"

namespace aidw {

namespace {

using namespace gridk;

__global__ void __launch_bounds__(kThreads) k_bbox_dims(const float *__restrict__ x,
                                                        const float *__restrict__ y,
                                                        const float *__restrict__ z, long long n,
                                                        float *__restrict__ part, int *ticket,
                                                        GridDev *g, double cell_scale,
                                                        double area_param, long long cap)
{
    bbox_dims_block(x, y, z, n, part, ticket, g, cell_scale, area_param, cap, blockIdx.x,
                    gridDim.x);
}

__global__ void __launch_bounds__(kThreads) k_keys(const float *__restrict__ x,
                                                   const float *__restrict__ y, long long n,
                                                   const GridDev *__restrict__ g,
                                                   int *__restrict__ count, int *__restrict__ key,
                                                   int *__restrict__ rank)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || grid_failed(g)) return;
    key_one(i, x, y, g, count, key, rank);
}

__global__ void __launch_bounds__(kThreads) k_scan(int *__restrict__ a, long long len,
                                                   unsigned long long *flags, int *ticket,
                                                   GridDev *g)
{
    scan_lookback_block(a, len, flags, ticket, &g->status);
}

__global__ void __launch_bounds__(kThreads) k_scatter(const float *__restrict__ x,
                                                      const float *__restrict__ y,
                                                      const float *__restrict__ z, long long n,
                                                      const GridDev *__restrict__ g,
                                                      const int *__restrict__ start,
                                                      const int *__restrict__ key,
                                                      const int *__restrict__ rank,
                                                      Point *__restrict__ tmp)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || grid_failed(g)) return;
    scatter_point(i, x, y, z, start, key, rank, tmp, g, n);
}

__global__ void __launch_bounds__(kThreads) k_fixup_pad(long long n, long long pad_hi,
                                                        long long n_pad, long long n_wpad,
                                                        const GridDev *__restrict__ g,
                                                        const int *__restrict__ start,
                                                        const Point *__restrict__ tmp,
                                                        Point *__restrict__ pts,
                                                        int *__restrict__ perm,
                                                        float *__restrict__ wt)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) {
        if (!grid_failed(g)) fixup_one(s, g, start, tmp, pts, perm, wt, n);
    } else if (s < pad_hi) {
        pad_one(s, n_pad, n_wpad, pts, wt);
    }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Capacity bound on the number of cells: 4n/c^2 cells cover the data box at
// width c*r_exp when A is the box area; the second term allows elongated
// boxes (perimeter cells).
long long grid_cells_capacity(long long n, double c)
{
    return (long long)(4.0 * (double)n / (c * c) + 16.0 * sqrt((double)n) / c) + 16;
}

// Ints of the grid's cell_start allocation: the cap + 1 cell heads, then
// (8-byte aligned) the single-pass scan's records (one 64-bit record per
// scan chunk) and two tickets, all zeroed at the start of every build.
long long grid_cell_start_ints(long long cap)
{
    const long long nb = (cap + 1 + kScanChunk - 1) / kScanChunk;
    return (cap + 2) / 2 * 2 + 2 * nb + 4;
}

aidw_status grid_build_launch(aidw_grid *g, const float *x, const float *y, const float *z,
                              cudaStream_t s)
{
    NvtxRange nvtx_("grid build");
    const long long n = g->n_data;
    const long long cap = g->cap_cells;
    const long long scan_len = cap + 1;
    const long long nb = (scan_len + kScanChunk - 1) / kScanChunk;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, g->device);
    const unsigned bb = (unsigned)std::min<long long>(blocks_for(n, kThreads),
                                                      (long long)dev_sms * 4);
    int *key = nullptr, *rank = nullptr;
    Point *tmp = nullptr;
    float *bpart = nullptr;
    cudaError_t e = lib_alloc((void **)&key, sizeof(int) * n, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&rank, sizeof(int) * n, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&tmp, sizeof(Point) * n, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&bpart, sizeof(float) * 5 * bb, s);
    if (e != cudaSuccess) {
        lib_free(key, s);
        lib_free(rank, s);
        lib_free(tmp, s);
        return AIDW_ERR_OOM;
    }
    // cell_start holds the counts, then (8-byte aligned) the scan records and
    // the two tickets
    int *start = g->cell_start;
    const long long rec_off = (scan_len + 1) / 2 * 2;
    unsigned long long *flags = reinterpret_cast<unsigned long long *>(start + rec_off);
    int *tickets = start + rec_off + 2 * nb;
    const int prof = profile_begin(s);
    int nl = 0;
    cudaMemsetAsync(start, 0, sizeof(int) * (size_t)grid_cell_start_ints(cap), s);
    k_bbox_dims<<<bb, kThreads, 0, s>>>(x, y, z, n, bpart, tickets, g->dev, g->cell_scale,
                                        g->area_param, cap);
    k_keys<<<blocks_for(n, kThreads), kThreads, 0, s>>>(x, y, n, g->dev, start, key, rank);
    k_scan<<<(unsigned)nb, kThreads, 0, s>>>(start, scan_len, flags, tickets + 1, g->dev);
    k_scatter<<<blocks_for(n, kThreads), kThreads, 0, s>>>(x, y, z, n, g->dev, start, key, rank,
                                                           tmp);
    const long long n_wpad = g->n_wtiles * kWeightTile;
    const long long pad_hi = std::max(std::max(g->n_pad, n_wpad), n);
    k_fixup_pad<<<blocks_for(pad_hi, kThreads), kThreads, 0, s>>>(
        n, pad_hi, g->n_pad, n_wpad, g->dev, start, tmp, g->pts, g->perm, g->wt);
    nl += 5;
    lib_free(key, s);
    lib_free(rank, s);
    lib_free(tmp, s);
    lib_free(bpart, s);
    profile_end(prof, s, AIDW_STAGE_GRID_BUILD, nl);
    return cuda_status(cudaGetLastError());
}

}  // namespace aidw
