/*
 * Plain FP64 CPU oracle for Adaptive IDW (AIDW) interpolation with kNN
 * (Mei, Xu & Xu, "Improving GPU-accelerated Adaptive IDW Interpolation
 * Algorithm Using Fast kNN Search", arXiv 1601.05904).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA library is checked against.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is computed in double precision from float32 inputs promoted
 * to double.  Nothing here is blocked, fused or reordered beyond what the
 * definitions state; each query is computed serially and independently, so
 * the optional OpenMP loop over queries does not change any result.
 *
 * Functions and the passages they follow:
 *   oracle_r_exp        Eq. 2  (expected nearest-neighbour distance)
 *   oracle_r_obs        Eq. 3  (observed mean kNN distance)
 *   oracle_mu           Eq. 5  (cosine fuzzy membership of R = Eq. 4)
 *   oracle_alpha        Eq. 6  (triangular membership -> power alpha)
 *   oracle_knn          Sec. 2.3 brute-force kNN: every distance, full sort,
 *                       first k; ties ordered by the original index
 *   oracle_aidw         Sec. 2.2 steps 1-3 then Eq. 1 over all data points
 *   oracle_aidw_local   the same with Eq. 1 over the k nearest points only
 *   oracle_grid_dims /
 *   oracle_grid_fill    Sec. 3.2.1-3.2.3 / 4.1.1-4.1.3 even grid: bounding
 *                       box, cell width from Eq. 2, nCol/nRow, cell index
 *                       per point, points ordered by cell (stable), and the
 *                       (head, count) pair of every cell.
 *   oracle_knn_paper_rule  Sec. 3.2.4 grid kNN with the paper's own stop
 *                       rule (first level holding k points, plus one level),
 *                       which is not always exact; kept to measure that.
 *
 * Readings of the paper that this oracle fixes (the paper is silent or
 * garbled there):
 *   - Eq. 1 sums over ALL data points; kNN only feeds alpha (Sec. 3.3, 4.2).
 *   - n in Eq. 2 is the number of data points; A is the area of the data
 *     bounding box unless the caller passes an explicit area.
 *   - A query at distance exactly 0 from one or more data points returns the
 *     mean z of those points (the limit of Eq. 1 as d -> 0).
 *   - R = 0 when r_obs = 0; R = +inf when r_exp = 0 < r_obs.
 *   - Eq. 6 overlapping interval ends: the first matching interval is used.
 *   - kNN ties: lexicographic (squared distance, original index).
 *   - Cell index: col = floor((x - minX) / cw) clamped to [0, nCol - 1]
 *     (the printed cast binds before the division, a typo), and
 *     nCol = (int)((maxX - minX + cw) / cw) as printed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------- */
/* Eq. 2: r_exp = 1 / (2 sqrt(n / A)).  Zero when the area is zero.        */
/* ---------------------------------------------------------------------- */
double oracle_r_exp(int64_t n, double area)
{
    if (!(area > 0.0) || n <= 0) return 0.0;
    return 1.0 / (2.0 * sqrt((double)n / area));
}

/* Eq. 3: r_obs = (1/k) sum_{i<=k} d_i. */
double oracle_r_obs(const double *d, int k)
{
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += d[i];
    return s / (double)k;
}

/* Eq. 4: R = r_obs / r_exp, with the two degenerate cases fixed above. */
double oracle_R(double r_obs, double r_exp)
{
    if (r_obs == 0.0) return 0.0;
    if (r_exp == 0.0) return INFINITY;
    return r_obs / r_exp;
}

/* Eq. 5: cosine membership, printed with pi / R_max. */
double oracle_mu(double R, double r_min, double r_max)
{
    if (R <= r_min) return 0.0;
    if (R >= r_max) return 1.0;
    return 0.5 - 0.5 * cos((M_PI / r_max) * (R - r_min));
}

/* Eq. 6: triangular membership from mu to the five alpha levels. */
double oracle_alpha(double mu, const double a[5])
{
    if (mu <= 0.1) return a[0];
    if (mu <= 0.3) return a[0] * (1.0 - 5.0 * (mu - 0.1)) + 5.0 * a[1] * (mu - 0.1);
    if (mu <= 0.5) return 5.0 * a[2] * (mu - 0.3) + a[1] * (1.0 - 5.0 * (mu - 0.3));
    if (mu <= 0.7) return a[2] * (1.0 - 5.0 * (mu - 0.5)) + 5.0 * a[3] * (mu - 0.5);
    if (mu <= 0.9) return 5.0 * a[4] * (mu - 0.7) + a[3] * (1.0 - 5.0 * (mu - 0.7));
    return a[4];
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.3 brute-force kNN.                                              */
/* ---------------------------------------------------------------------- */
typedef struct {
    double d2;
    int64_t idx;
} oracle_pair;

static int oracle_pair_cmp(const void *pa, const void *pb)
{
    const oracle_pair *a = (const oracle_pair *)pa;
    const oracle_pair *b = (const oracle_pair *)pb;
    if (a->d2 < b->d2) return -1;
    if (a->d2 > b->d2) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

/* Step 1: every squared distance; step 2: sort all of them; step 3: the
 * first k in increasing order.  buf holds n pairs. */
static void oracle_knn_one(const float *x, const float *y, int64_t n,
                           double qx, double qy, int k, oracle_pair *buf,
                           int32_t *out_idx, double *out_d)
{
    for (int64_t i = 0; i < n; ++i) {
        double dx = qx - (double)x[i];
        double dy = qy - (double)y[i];
        buf[i].d2 = dx * dx + dy * dy;
        buf[i].idx = i;
    }
    qsort(buf, (size_t)n, sizeof(oracle_pair), oracle_pair_cmp);
    for (int j = 0; j < k; ++j) {
        out_idx[j] = (int32_t)buf[j].idx;
        out_d[j] = sqrt(buf[j].d2);
    }
}

/* 1 when the query loops run in parallel (compiled with OpenMP), else 0. */
int oracle_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out_idx, out_d: [m * k], row-major by query. */
void oracle_knn(const float *x, const float *y, int64_t n,
                const float *qx, const float *qy, int64_t m, int k,
                int32_t *out_idx, double *out_d, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        oracle_pair *buf = (oracle_pair *)malloc((size_t)n * sizeof(oracle_pair));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t q = 0; q < m; ++q)
            oracle_knn_one(x, y, n, (double)qx[q], (double)qy[q], k, buf,
                           out_idx + q * k, out_d + q * k);
        free(buf);
    }
    (void)nthreads;
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.2 + Eq. 1: the full AIDW prediction for each query.             */
/* ---------------------------------------------------------------------- */
/* Outputs (each [m], any may be NULL except out_z):
 *   out_z      prediction (Eq. 1 with the adaptive alpha)
 *   out_alpha  alpha of Eq. 6
 *   out_robs   r_obs of Eq. 3
 *   out_scale  S_q = sum w |z| / sum w, the scale of Eq. 1's cancellation
 *              (mean |z| of the coincident points for an exact hit)
 * area <= 0 selects the area of the data bounding box. */
void oracle_aidw(const float *x, const float *y, const float *z, int64_t n,
                 const float *qx, const float *qy, int64_t m, int k,
                 const double alpha_levels[5], double r_min, double r_max,
                 double area, double *out_z, double *out_alpha,
                 double *out_robs, double *out_scale, int nthreads)
{
    if (!(area > 0.0)) {
        double minx = x[0], maxx = x[0], miny = y[0], maxy = y[0];
        for (int64_t i = 1; i < n; ++i) {
            if (x[i] < minx) minx = x[i];
            if (x[i] > maxx) maxx = x[i];
            if (y[i] < miny) miny = y[i];
            if (y[i] > maxy) maxy = y[i];
        }
        area = (maxx - minx) * (maxy - miny);
    }
    const double r_exp = oracle_r_exp(n, area);

#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        oracle_pair *buf = (oracle_pair *)malloc((size_t)n * sizeof(oracle_pair));
        int32_t *nn_idx = (int32_t *)malloc((size_t)k * sizeof(int32_t));
        double *nn_d = (double *)malloc((size_t)k * sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t q = 0; q < m; ++q) {
            const double px = (double)qx[q], py = (double)qy[q];
            /* Step 1 of Sec. 2.2: kNN, r_obs (Eq. 3), R (Eq. 4). */
            oracle_knn_one(x, y, n, px, py, k, buf, nn_idx, nn_d);
            const double r_obs = oracle_r_obs(nn_d, k);
            const double R = oracle_R(r_obs, r_exp);
            /* Step 2: mu (Eq. 5).  Step 3: alpha (Eq. 6). */
            const double mu = oracle_mu(R, r_min, r_max);
            const double a = oracle_alpha(mu, alpha_levels);

            /* Eq. 1 over all n data points. */
            int64_t nhit = 0;
            double hit_z = 0.0, hit_abs = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if ((double)x[i] == px && (double)y[i] == py) {
                    ++nhit;
                    hit_z += (double)z[i];
                    hit_abs += fabs((double)z[i]);
                }
            }
            double zq, sq;
            if (nhit > 0) {
                zq = hit_z / (double)nhit;
                sq = hit_abs / (double)nhit;
            } else {
                double sw = 0.0, swz = 0.0, swa = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    const double dx = px - (double)x[i];
                    const double dy = py - (double)y[i];
                    const double d = sqrt(dx * dx + dy * dy);
                    const double w = pow(d, -a);
                    sw += w;
                    swz += w * (double)z[i];
                    swa += w * fabs((double)z[i]);
                }
                zq = swz / sw;
                sq = swa / sw;
            }
            out_z[q] = zq;
            if (out_alpha) out_alpha[q] = a;
            if (out_robs) out_robs[q] = r_obs;
            if (out_scale) out_scale[q] = sq;
        }
        free(nn_d);
        free(nn_idx);
        free(buf);
    }
    (void)nthreads;
}

/* ---------------------------------------------------------------------- */
/* Local AIDW: Eq. 1 with n = k, the k nearest data points only.           */
/* ---------------------------------------------------------------------- */
/* Eq. 1 reads "n is the total number of data points used in interpolating";
 * this variant uses the k nearest points of Sec. 2.3's brute force (ties by
 * index) both for alpha (Eq. 2-6, unchanged) and for the weighted average.
 * Coincident points among those k give their mean z. */
void oracle_aidw_local(const float *x, const float *y, const float *z, int64_t n,
                       const float *qx, const float *qy, int64_t m, int k,
                       const double alpha_levels[5], double r_min, double r_max,
                       double area, double *out_z, double *out_alpha, double *out_scale,
                       int nthreads)
{
    if (!(area > 0.0)) {
        double minx = x[0], maxx = x[0], miny = y[0], maxy = y[0];
        for (int64_t i = 1; i < n; ++i) {
            if (x[i] < minx) minx = x[i];
            if (x[i] > maxx) maxx = x[i];
            if (y[i] < miny) miny = y[i];
            if (y[i] > maxy) maxy = y[i];
        }
        area = (maxx - minx) * (maxy - miny);
    }
    const double r_exp = oracle_r_exp(n, area);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        oracle_pair *buf = (oracle_pair *)malloc((size_t)n * sizeof(oracle_pair));
        int32_t *nn_idx = (int32_t *)malloc((size_t)k * sizeof(int32_t));
        double *nn_d = (double *)malloc((size_t)k * sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t q = 0; q < m; ++q) {
            oracle_knn_one(x, y, n, (double)qx[q], (double)qy[q], k, buf, nn_idx, nn_d);
            const double R = oracle_R(oracle_r_obs(nn_d, k), r_exp);
            const double a = oracle_alpha(oracle_mu(R, r_min, r_max), alpha_levels);
            int nhit = 0;
            double hz = 0.0, ha = 0.0, sw = 0.0, swz = 0.0, swa = 0.0;
            for (int j = 0; j < k; ++j) {
                const double zj = (double)z[nn_idx[j]];
                if (nn_d[j] == 0.0) {
                    ++nhit;
                    hz += zj;
                    ha += fabs(zj);
                } else {
                    const double w = pow(nn_d[j], -a);
                    sw += w;
                    swz += w * zj;
                    swa += w * fabs(zj);
                }
            }
            out_z[q] = nhit ? hz / nhit : swz / sw;
            if (out_alpha) out_alpha[q] = a;
            if (out_scale) out_scale[q] = nhit ? ha / nhit : swa / sw;
        }
        free(nn_d);
        free(nn_idx);
        free(buf);
    }
    (void)nthreads;
}

/* ---------------------------------------------------------------------- */
/* Even grid (Sec. 3.2.1-3.2.3, 4.1.1-4.1.3).                             */
/* ---------------------------------------------------------------------- */
/* info layout (doubles):
 *   [0] minX [1] minY [2] maxX [3] maxY [4] area used for Eq. 2
 *   [5] r_exp [6] cell width cw [7] nCol [8] nRow
 *
 * Cell width: cw = cell_scale * r_exp (the paper uses cell_scale = 1).
 * When the data box has zero area r_exp is 0; cw then falls back to the
 * one-dimensional spacing c * max(W, H) / (2 n), or 1 when all points
 * coincide.  The number of cells
 * is bounded by cap = 4 n / c^2 + 16 sqrt(n) / c + 16 (c = cell_scale); if
 * the box's aspect ratio or an explicit area pushes nCol * nRow past cap,
 * cw is doubled until it fits.  A positive cw_override replaces all of this.
 */
static int64_t oracle_grid_ncells_cap(int64_t n, double c)
{
    return (int64_t)(4.0 * (double)n / (c * c) + 16.0 * sqrt((double)n) / c) + 16;
}

void oracle_grid_dims(const float *x, const float *y, int64_t n,
                      double cell_scale, double area, double cw_override,
                      double *info)
{
    double minx = x[0], maxx = x[0], miny = y[0], maxy = y[0];
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < minx) minx = x[i];
        if (x[i] > maxx) maxx = x[i];
        if (y[i] < miny) miny = y[i];
        if (y[i] > maxy) maxy = y[i];
    }
    const double W = maxx - minx, H = maxy - miny;
    if (!(area > 0.0)) area = W * H;
    const double r_exp = oracle_r_exp(n, area);
    double cw;
    if (cw_override > 0.0) {
        cw = cw_override;
    } else {
        cw = cell_scale * r_exp;
        if (!(cw > 0.0)) {
            const double side = W > H ? W : H;
            cw = side > 0.0 ? cell_scale * side / (2.0 * (double)n) : 1.0;
        }
        const int64_t cap = oracle_grid_ncells_cap(n, cell_scale);
        for (;;) {
            const double ncol = floor((W + cw) / cw);
            const double nrow = floor((H + cw) / cw);
            if (ncol * nrow <= (double)cap) break;
            cw = cw * 2.0;
        }
    }
    info[0] = minx;
    info[1] = miny;
    info[2] = maxx;
    info[3] = maxy;
    info[4] = area;
    info[5] = r_exp;
    info[6] = cw;
    info[7] = (double)(int64_t)((W + cw) / cw);
    info[8] = (double)(int64_t)((H + cw) / cw);
}

/* Given info from oracle_grid_dims:
 *   out_key[n]              cell index row * nCol + col of each point
 *   out_cell_start[nCells+1] head of each cell's segment; the last entry is n
 *                            (count of cell c = start[c+1] - start[c])
 *   out_perm[n]             original indices in cell order, stable by index */
void oracle_grid_fill(const float *x, const float *y, int64_t n,
                      const double *info, int64_t *out_key,
                      int64_t *out_cell_start, int64_t *out_perm)
{
    const double minx = info[0], miny = info[1], cw = info[6];
    const int64_t ncol = (int64_t)info[7], nrow = (int64_t)info[8];
    const int64_t ncells = ncol * nrow;
    for (int64_t i = 0; i < n; ++i) {
        int64_t col = (int64_t)floor(((double)x[i] - minx) / cw);
        int64_t row = (int64_t)floor(((double)y[i] - miny) / cw);
        if (col < 0) col = 0;
        if (col > ncol - 1) col = ncol - 1;
        if (row < 0) row = 0;
        if (row > nrow - 1) row = nrow - 1;
        out_key[i] = row * ncol + col;
    }
    /* segmented count (reduce by key) and head (exclusive scan) */
    for (int64_t c = 0; c <= ncells; ++c) out_cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) out_cell_start[out_key[i] + 1] += 1;
    for (int64_t c = 0; c < ncells; ++c) out_cell_start[c + 1] += out_cell_start[c];
    /* stable placement in index order */
    int64_t *fill = (int64_t *)malloc((size_t)ncells * sizeof(int64_t));
    for (int64_t c = 0; c < ncells; ++c) fill[c] = out_cell_start[c];
    for (int64_t i = 0; i < n; ++i) out_perm[fill[out_key[i]]++] = i;
    free(fill);
}

/* ---------------------------------------------------------------------- */
/* Sec. 3.2.4 grid kNN with the paper's level rule.                        */
/* ---------------------------------------------------------------------- */
/* Number of points in the block of cells of level L around (col, row):
 * columns col-L .. col+L and rows row-L .. row+L, clipped to the grid. */
static int64_t oracle_block_count(const int64_t *cell_start, int64_t ncol, int64_t nrow,
                                  int64_t col, int64_t row, int64_t L)
{
    const int64_t c0 = col - L < 0 ? 0 : col - L;
    const int64_t c1 = col + L > ncol - 1 ? ncol - 1 : col + L;
    const int64_t r0 = row - L < 0 ? 0 : row - L;
    const int64_t r1 = row + L > nrow - 1 ? nrow - 1 : row + L;
    int64_t cnt = 0;
    for (int64_t r = r0; r <= r1; ++r)
        cnt += cell_start[r * ncol + c1 + 1] - cell_start[r * ncol + c0];
    return cnt;
}

/* The kNN search of Sec. 3.2.4 as the paper states it, on the grid of
 * oracle_grid_dims / oracle_grid_fill (info, cell_start, perm):
 *   Step 1  locate the query's cell (same floor-and-clamp as the points);
 *   Step 2  the level of cell expanding: the smallest L whose block of
 *           (2L+1)^2 cells holds at least k points, then one level more
 *           (the remark on Fig. 4);
 *   Step 3  the k nearest of the points in that block (every squared
 *           distance, full sort by (d^2, original index), first k).
 * The candidate set is a subset of all points, so the result can miss true
 * neighbours; out_d[j] >= the exact j-th distance for every j.
 * k fixes the level; the first k_out >= k candidates of the block are
 * written (index -1 and +inf beyond the block's point count), so a caller
 * can see the gap after the k-th.
 * out_idx: [m * k_out] original indices; out_d: [m * k_out] distances. */
void oracle_knn_paper_rule(const float *x, const float *y, int64_t n, const double *info,
                           const int64_t *cell_start, const int64_t *perm,
                           const float *qx, const float *qy, int64_t m, int k, int k_out,
                           int32_t *out_idx, double *out_d, int nthreads)
{
    const double minx = info[0], miny = info[1], cw = info[6];
    const int64_t ncol = (int64_t)info[7], nrow = (int64_t)info[8];
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        oracle_pair *buf = (oracle_pair *)malloc((size_t)n * sizeof(oracle_pair));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t q = 0; q < m; ++q) {
            const double px = (double)qx[q], py = (double)qy[q];
            int64_t col = (int64_t)floor((px - minx) / cw);
            int64_t row = (int64_t)floor((py - miny) / cw);
            if (col < 0) col = 0;
            if (col > ncol - 1) col = ncol - 1;
            if (row < 0) row = 0;
            if (row > nrow - 1) row = nrow - 1;
            int64_t L = 0;
            while (oracle_block_count(cell_start, ncol, nrow, col, row, L) < k) ++L;
            L += 1;
            const int64_t c0 = col - L < 0 ? 0 : col - L;
            const int64_t c1 = col + L > ncol - 1 ? ncol - 1 : col + L;
            const int64_t r0 = row - L < 0 ? 0 : row - L;
            const int64_t r1 = row + L > nrow - 1 ? nrow - 1 : row + L;
            int64_t cnt = 0;
            for (int64_t r = r0; r <= r1; ++r)
                for (int64_t s = cell_start[r * ncol + c0]; s < cell_start[r * ncol + c1 + 1];
                     ++s) {
                    const int64_t i = perm[s];
                    const double dx = px - (double)x[i];
                    const double dy = py - (double)y[i];
                    buf[cnt].d2 = dx * dx + dy * dy;
                    buf[cnt].idx = i;
                    ++cnt;
                }
            qsort(buf, (size_t)cnt, sizeof(oracle_pair), oracle_pair_cmp);
            for (int j = 0; j < k_out; ++j) {
                out_idx[q * k_out + j] = j < cnt ? (int32_t)buf[j].idx : -1;
                out_d[q * k_out + j] = j < cnt ? sqrt(buf[j].d2) : INFINITY;
            }
        }
        free(buf);
    }
    (void)nthreads;
}
