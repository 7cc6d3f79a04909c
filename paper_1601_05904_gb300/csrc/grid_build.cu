// Even-grid build (Sec. 3.2.1-3.2.3, 4.1.1-4.1.3 of arXiv 1601.05904).
//
// The paper builds the grid with Thrust: minmax_element for the bounding
// box, a key kernel, sort_by_key, then reduce_by_key / unique_by_key for the
// count and head of every cell (Fig. 3).  Here the same result comes from a
// counting sort in plain kernels, all on the caller's stream and without a
// host round trip (the cell-array capacity is a function of n alone):
//
//   k_grid_init   reset the device grid record
//   k_bbox        min/max of x and y (and a non-finite check of x, y, z)
//   k_dims        A, r_exp (Eq. 2), cell width, nCol, nRow
//   k_keys        cell of each point + histogram (atomic) -> rank in cell
//   k_scan_*      exclusive scan of the histogram = head of each cell
//   k_scatter     point index to head + rank (unstable within a cell)
//   k_fixup       stable order within each cell + write the cell-ordered
//                 float4 points {x, y, z, index}
//   k_pad         padding points at +inf after the last one
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

__global__ void k_grid_init(GridDev *g, long long n) { grid_init(g, n); }

__global__ void __launch_bounds__(kThreads) k_bbox(const float *__restrict__ x,
                                                   const float *__restrict__ y,
                                                   const float *__restrict__ z, long long n,
                                                   GridDev *g)
{
    bbox_block(x, y, z, (long long)blockIdx.x * blockDim.x + threadIdx.x, n,
               (long long)gridDim.x * blockDim.x, g);
}

__global__ void k_dims(GridDev *g, double cell_scale, double area_param, long long cap)
{
    grid_dims(g, cell_scale, area_param, cap);
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

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int *__restrict__ a, long long len,
                                                          int *__restrict__ block_sum)
{
    scan_reduce_chunk(a, len, blockIdx.x, block_sum + blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_scan_sums(int *block_sum, int nb)
{
    scan_sums(block_sum, nb);
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(int *__restrict__ a, long long len,
                                                         const int *__restrict__ block_sum)
{
    scan_apply_chunk(a, len, blockIdx.x, block_sum[blockIdx.x]);
}

__global__ void __launch_bounds__(kThreads) k_scatter(long long n, const GridDev *__restrict__ g,
                                                      const int *__restrict__ start,
                                                      const int *__restrict__ key,
                                                      const int *__restrict__ rank,
                                                      int *__restrict__ tmp)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || grid_failed(g)) return;
    scatter_one(i, start, key, rank, tmp);
}

__global__ void __launch_bounds__(kThreads) k_fixup(const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    const float *__restrict__ z, long long n,
                                                    const GridDev *__restrict__ g,
                                                    const int *__restrict__ start,
                                                    const int *__restrict__ key,
                                                    const int *__restrict__ tmp,
                                                    Point *__restrict__ pts, int *__restrict__ perm,
                                                    float *__restrict__ wt)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || grid_failed(g)) return;
    fixup_one(s, x, y, z, start, key, tmp, pts, perm, wt);
}

__global__ void k_pad(Point *pts, long long n, long long n_pad, float *wt, long long n_wpad)
{
    const long long i = n + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    pad_one(i, n_pad, n_wpad, pts, wt);
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

aidw_status grid_build_launch(aidw_grid *g, const float *x, const float *y, const float *z,
                              cudaStream_t s)
{
    const long long n = g->n_data;
    const long long cap = g->cap_cells;
    int *key = nullptr, *rank = nullptr, *tmp = nullptr, *bsum = nullptr;
    const long long scan_len = cap + 1;
    const long long nb = (scan_len + kScanChunk - 1) / kScanChunk;
    cudaError_t e = lib_alloc((void **)&key, sizeof(int) * n, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&rank, sizeof(int) * n, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&tmp, sizeof(int) * n, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&bsum, sizeof(int) * nb, s);
    if (e != cudaSuccess) {
        lib_free(key, s);
        lib_free(rank, s);
        lib_free(tmp, s);
        return AIDW_ERR_OOM;
    }
    int *start = g->cell_start;
    const int prof = profile_begin(s);
    int nl = 0;
    k_grid_init<<<1, 1, 0, s>>>(g->dev, n);
    ++nl;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, g->device);
    const unsigned bb = (unsigned)std::min<long long>(blocks_for(n, kThreads),
                                                      (long long)dev_sms * 4);
    k_bbox<<<bb, kThreads, 0, s>>>(x, y, z, n, g->dev);
    ++nl;
    k_dims<<<1, 1, 0, s>>>(g->dev, g->cell_scale, g->area_param, cap);
    ++nl;
    cudaMemsetAsync(start, 0, sizeof(int) * scan_len, s);
    k_keys<<<blocks_for(n, kThreads), kThreads, 0, s>>>(x, y, n, g->dev, start, key, rank);
    ++nl;
    k_scan_reduce<<<(unsigned)nb, kThreads, 0, s>>>(start, scan_len, bsum);
    k_scan_sums<<<1, kThreads, 0, s>>>(bsum, (int)nb);
    k_scan_apply<<<(unsigned)nb, kThreads, 0, s>>>(start, scan_len, bsum);
    nl += 3;
    k_scatter<<<blocks_for(n, kThreads), kThreads, 0, s>>>(n, g->dev, start, key, rank, tmp);
    k_fixup<<<blocks_for(n, kThreads), kThreads, 0, s>>>(x, y, z, n, g->dev, start, key, tmp,
                                                         g->pts, g->perm, g->wt);
    nl += 2;
    const long long n_wpad = g->n_wtiles * kWeightTile;
    const long long pad_hi = std::max(g->n_pad, n_wpad);
    if (pad_hi > n) {
        k_pad<<<blocks_for(pad_hi - n, kThreads), kThreads, 0, s>>>(g->pts, n, g->n_pad, g->wt,
                                                                    n_wpad);
        ++nl;
    }
    lib_free(key, s);
    lib_free(rank, s);
    lib_free(tmp, s);
    lib_free(bsum, s);
    profile_end(prof, s, AIDW_STAGE_GRID_BUILD, nl);
    return cuda_status(cudaGetLastError());
}

}  // namespace aidw
