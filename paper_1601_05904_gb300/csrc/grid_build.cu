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
#include <float.h>
#include <math.h>

#include <algorithm>

#include "aidw_device.cuh"
#include "aidw_internal.cuh"

namespace aidw {

namespace {

constexpr int kThreads = 256;
constexpr int kScanItems = 16;                       // per thread
constexpr int kScanChunk = kThreads * kScanItems;    // per block

__device__ __forceinline__ int enc_float(float f)
{
    const int b = __float_as_int(f);
    return b >= 0 ? b : (b ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float dec_float(int e)
{
    return __int_as_float(e >= 0 ? e : (e ^ 0x7FFFFFFF));
}

__global__ void k_grid_init(GridDev *g, long long n)
{
    g->enc_min_x = 0x7FFFFFFF;
    g->enc_min_y = 0x7FFFFFFF;
    g->enc_max_x = (int)0x80000000;
    g->enc_max_y = (int)0x80000000;
    g->n_data = n;
    g->status = 0;
}

__global__ void __launch_bounds__(kThreads) k_bbox(const float *__restrict__ x,
                                                   const float *__restrict__ y,
                                                   const float *__restrict__ z, long long n,
                                                   GridDev *g)
{
    float mnx = FLT_MAX, mny = FLT_MAX, mxx = -FLT_MAX, mxy = -FLT_MAX;
    int bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float xi = __ldg(x + i), yi = __ldg(y + i), zi = __ldg(z + i);
        if (!isfinite(xi) || !isfinite(yi) || !isfinite(zi)) {
            bad = 1;
            continue;
        }
        mnx = fminf(mnx, xi);
        mxx = fmaxf(mxx, xi);
        mny = fminf(mny, yi);
        mxy = fmaxf(mxy, yi);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    bad = __any_sync(0xffffffffu, bad);
    __shared__ float s[4][kThreads / 32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s[0][w] = mnx;
        s[1][w] = mxx;
        s[2][w] = mny;
        s[3][w] = mxy;
        if (bad) sbad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThreads / 32; ++i) {
            mnx = fminf(mnx, s[0][i]);
            mxx = fmaxf(mxx, s[1][i]);
            mny = fminf(mny, s[2][i]);
            mxy = fmaxf(mxy, s[3][i]);
        }
        atomicMin(&g->enc_min_x, enc_float(mnx));
        atomicMax(&g->enc_max_x, enc_float(mxx));
        atomicMin(&g->enc_min_y, enc_float(mny));
        atomicMax(&g->enc_max_y, enc_float(mxy));
        if (sbad) atomicOr(&g->status, kStatusNonfiniteData);
    }
}

// Grid dimensions (one thread).  cap is the capacity of the cell arrays:
// if the box's aspect ratio or an explicit area would need more cells, the
// width is doubled until it fits (the kNN result does not depend on it).
__global__ void k_dims(GridDev *g, double cell_scale, double area_param, long long cap)
{
    if (g->status & kStatusNonfiniteData) return;
    const double minx = (double)dec_float(g->enc_min_x), maxx = (double)dec_float(g->enc_max_x);
    const double miny = (double)dec_float(g->enc_min_y), maxy = (double)dec_float(g->enc_max_y);
    const double W = maxx - minx, H = maxy - miny;
    const double n = (double)g->n_data;
    const double area = area_param > 0.0 ? area_param : W * H;
    const double r_exp = (area > 0.0) ? 1.0 / (2.0 * sqrt(n / area)) : 0.0;  // Eq. 2
    double cw = cell_scale * r_exp;
    if (!(cw > 0.0)) {
        const double side = W > H ? W : H;
        cw = side > 0.0 ? cell_scale * side / (2.0 * n) : 1.0;
    }
    for (int it = 0; it < 2100; ++it) {
        const double nc = floor((W + cw) / cw), nr = floor((H + cw) / cw);
        if (nc * nr <= (double)cap) break;
        cw = cw * 2.0;
    }
    g->min_x = minx;
    g->min_y = miny;
    g->max_x = maxx;
    g->max_y = maxy;
    g->area = area;
    g->r_exp = r_exp;
    g->cw = cw;
    g->n_col = (long long)((W + cw) / cw);
    g->n_row = (long long)((H + cw) / cw);
    g->n_cells = g->n_col * g->n_row;
    if (g->n_cells > cap) atomicOr(&g->status, kStatusCapacity);
}

__global__ void __launch_bounds__(kThreads) k_keys(const float *__restrict__ x,
                                                   const float *__restrict__ y, long long n,
                                                   const GridDev *__restrict__ g,
                                                   int *__restrict__ count, int *__restrict__ key,
                                                   int *__restrict__ rank)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (g->status & (kStatusNonfiniteData | kStatusCapacity))) return;
    const double minx = g->min_x, miny = g->min_y, cw = g->cw;
    const long long nc = g->n_col, nr = g->n_row;
    long long col = (long long)floor(((double)x[i] - minx) / cw);
    long long row = (long long)floor(((double)y[i] - miny) / cw);
    col = col < 0 ? 0 : (col > nc - 1 ? nc - 1 : col);
    row = row < 0 ? 0 : (row > nr - 1 ? nr - 1 : row);
    const int c = (int)(row * nc + col);
    key[i] = c;
    rank[i] = atomicAdd(count + c, 1);
}

// --- exclusive scan of count[0, len) in place (reduce, scan sums, apply) ---

__device__ __forceinline__ int block_exclusive_scan(int v, int &total)
{
    __shared__ int warp_tot[kThreads / 32];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += t;
    }
    if (l == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = l < kThreads / 32 ? warp_tot[l] : 0;
        int ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, ti, o);
            if (l >= o) ti += u;
        }
        if (l < kThreads / 32) warp_tot[l] = ti - t;  // exclusive warp offsets
        if (l == kThreads / 32 - 1) total = ti;
    }
    __syncthreads();
    const int r = warp_tot[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int *__restrict__ a, long long len,
                                                          int *__restrict__ block_sum)
{
    const long long base = (long long)blockIdx.x * kScanChunk;
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long i = base + (long long)j * kThreads + threadIdx.x;
        if (i < len) s += a[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < kThreads / 32; ++i) t += ws[i];
        block_sum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_scan_sums(int *block_sum, int nb)
{
    __shared__ int carry;
    __shared__ int tot;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kThreads) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? block_sum[i] : 0;
        const int ex = block_exclusive_scan(v, tot);
        if (i < nb) block_sum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

// Each thread owns kScanItems consecutive elements of the block's chunk.
__global__ void __launch_bounds__(kThreads) k_scan_apply(int *__restrict__ a, long long len,
                                                         const int *__restrict__ block_sum)
{
    __shared__ int tot;
    const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < len) ? a[base + j] : 0;
        s += v[j];
    }
    int run = block_sum[blockIdx.x] + block_exclusive_scan(s, tot);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < len) a[base + j] = run;
        run += v[j];
    }
}

__global__ void __launch_bounds__(kThreads) k_scatter(long long n, const GridDev *__restrict__ g,
                                                      const int *__restrict__ start,
                                                      const int *__restrict__ key,
                                                      const int *__restrict__ rank,
                                                      int *__restrict__ tmp)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (g->status & (kStatusNonfiniteData | kStatusCapacity))) return;
    tmp[start[key[i]] + rank[i]] = (int)i;
}

// Position s holds some point i of cell c = key[i]; its stable place is the
// head of c plus the number of indices smaller than i in c's segment.
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
    if (s >= n || (g->status & (kStatusNonfiniteData | kStatusCapacity))) return;
    const int i = tmp[s];
    const int c = key[i];
    const int a = start[c], b = start[c + 1];
    int r = 0;
    for (int t = a; t < b; ++t) r += (tmp[t] < i);
    Point p;
    p.x = x[i];
    p.y = y[i];
    p.z = z[i];
    p.idx = i;
    pts[a + r] = p;
    perm[a + r] = i;
    const long long pos = a + r;
    float *tile = wt + (pos / kWeightTile) * (3 * kWeightTile) + pos % kWeightTile;
    tile[0] = -p.x;
    tile[kWeightTile] = -p.y;
    tile[2 * kWeightTile] = p.z;
}

// Padding after the last point: +inf coordinates, whose weight is exactly 0
// (d^2 = inf, log2 = inf, exp2(-inf) = 0), in both layouts.
__global__ void k_pad(Point *pts, long long n, long long n_pad, float *wt, long long n_wpad)
{
    const long long i = n + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float inf = __int_as_float(0x7f800000);
    if (i < n_pad) {
        Point p;
        p.x = inf;
        p.y = inf;
        p.z = 0.0f;
        p.idx = -1;
        pts[i] = p;
    }
    if (i < n_wpad) {
        float *tile = wt + (i / kWeightTile) * (3 * kWeightTile) + i % kWeightTile;
        tile[0] = -inf;
        tile[kWeightTile] = -inf;
        tile[2 * kWeightTile] = 0.0f;
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

aidw_status grid_build_launch(aidw_grid *g, const float *x, const float *y, const float *z,
                              cudaStream_t s)
{
    const long long n = g->n_data;
    const long long cap = g->cap_cells;
    int *key = nullptr, *rank = nullptr, *tmp = nullptr, *bsum = nullptr;
    const long long scan_len = cap + 1;
    const long long nb = (scan_len + kScanChunk - 1) / kScanChunk;
    cudaError_t e = cudaMallocAsync((void **)&key, sizeof(int) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&rank, sizeof(int) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tmp, sizeof(int) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&bsum, sizeof(int) * nb, s);
    if (e != cudaSuccess) {
        if (key) cudaFreeAsync(key, s);
        if (rank) cudaFreeAsync(rank, s);
        if (tmp) cudaFreeAsync(tmp, s);
        cudaGetLastError();
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
    cudaFreeAsync(key, s);
    cudaFreeAsync(rank, s);
    cudaFreeAsync(tmp, s);
    cudaFreeAsync(bsum, s);
    profile_end(prof, s, AIDW_STAGE_GRID_BUILD, nl);
    return cuda_status(cudaGetLastError());
}

}  // namespace aidw
