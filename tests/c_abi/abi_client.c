/* A plain C client of the library: reads float32 inputs from a directory,
 * runs the grid build, kNN, interpolation (both precisions), the local form,
 * a two-job batch and the end-to-end call from host arrays through
 * include/aidw.h with device memory from the CUDA runtime, and writes the
 * outputs next to the inputs.  Used by
 * tests/test_gpu_c_abi.py; no Python or torch is involved in the calls. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "aidw.h"

static float *read_f32(const char *dir, const char *name, int64_t n)
{
    char path[1024];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE *f = fopen(path, "rb");
    if (!f) return NULL;
    float *h = (float *)malloc(sizeof(float) * (size_t)n);
    size_t got = fread(h, sizeof(float), (size_t)n, f);
    fclose(f);
    if ((int64_t)got != n) {
        free(h);
        return NULL;
    }
    return h;
}

static int write_bytes(const char *dir, const char *name, const void *p, size_t bytes)
{
    char path[1024];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE *f = fopen(path, "wb");
    if (!f) return 1;
    fwrite(p, 1, bytes, f);
    fclose(f);
    return 0;
}

static void *to_dev(const void *h, size_t bytes)
{
    void *d = NULL;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return NULL;
    cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
    return d;
}

static int fetch(const char *dir, const char *name, const void *d, size_t bytes)
{
    void *h = malloc(bytes);
    cudaMemcpy(h, d, bytes, cudaMemcpyDeviceToHost);
    const int r = write_bytes(dir, name, h, bytes);
    free(h);
    return r;
}

#define CHECK(call)                                                                    \
    do {                                                                               \
        aidw_status st_ = (call);                                                      \
        if (st_ != AIDW_OK) {                                                          \
            fprintf(stderr, "%s failed: %s\n", #call, aidw_status_string(st_));        \
            return 2;                                                                  \
        }                                                                              \
    } while (0)

int main(int argc, char **argv)
{
    if (argc != 5) {
        fprintf(stderr, "usage: %s dir n m k\n", argv[0]);
        return 1;
    }
    const char *dir = argv[1];
    const int64_t n = atoll(argv[2]), m = atoll(argv[3]);
    const int k = atoi(argv[4]);
    float *hx = read_f32(dir, "x.bin", n), *hy = read_f32(dir, "y.bin", n);
    float *hz = read_f32(dir, "z.bin", n);
    float *hqx = read_f32(dir, "qx.bin", m), *hqy = read_f32(dir, "qy.bin", m);
    if (!hx || !hy || !hz || !hqx || !hqy) {
        fprintf(stderr, "missing input\n");
        return 1;
    }
    float *x = (float *)to_dev(hx, 4 * (size_t)n), *y = (float *)to_dev(hy, 4 * (size_t)n);
    float *z = (float *)to_dev(hz, 4 * (size_t)n);
    float *qx = (float *)to_dev(hqx, 4 * (size_t)m), *qy = (float *)to_dev(hqy, 4 * (size_t)m);
    float *z32 = NULL, *a32 = NULL, *zl = NULL, *dist = NULL, *robs = NULL, *zb0 = NULL,
          *zb1 = NULL;
    double *z64 = NULL;
    int32_t *idx = NULL;
    cudaMalloc((void **)&z32, 4 * (size_t)m);
    cudaMalloc((void **)&a32, 4 * (size_t)m);
    cudaMalloc((void **)&zl, 4 * (size_t)m);
    cudaMalloc((void **)&z64, 8 * (size_t)m);
    cudaMalloc((void **)&idx, 4 * (size_t)m * k);
    cudaMalloc((void **)&dist, 4 * (size_t)m * k);
    cudaMalloc((void **)&robs, 4 * (size_t)m);
    cudaMalloc((void **)&zb0, 4 * (size_t)m);
    cudaMalloc((void **)&zb1, 4 * (size_t)m);

    aidw_params p;
    aidw_params_default(&p);
    p.k = k;
    aidw_grid *g = NULL;
    CHECK(aidw_grid_build(x, y, z, n, &p, NULL, &g));
    aidw_grid_info info;
    CHECK(aidw_grid_get_info(g, &info));
    CHECK(aidw_knn(g, qx, qy, m, k, idx, dist, robs, NULL));
    CHECK(aidw_interpolate(g, qx, qy, m, &p, z32, a32, NULL));
    CHECK(aidw_interpolate_local(g, qx, qy, m, &p, zl, NULL, NULL));
    p.precision = AIDW_FP64_PLAIN;
    CHECK(aidw_interpolate(g, qx, qy, m, &p, z64, NULL, NULL));
    p.precision = AIDW_FP32_COMP;
    CHECK(aidw_grid_status(g));
    CHECK(aidw_grid_destroy(g));

    /* the same problem twice as a two-job batch (the second with k = 4) */
    aidw_job jobs[2];
    memset(jobs, 0, sizeof jobs);
    for (int j = 0; j < 2; ++j) {
        jobs[j].x = x;
        jobs[j].y = y;
        jobs[j].z = z;
        jobs[j].n_data = n;
        jobs[j].qx = qx;
        jobs[j].qy = qy;
        jobs[j].n_query = m;
    }
    jobs[0].k = k;
    jobs[0].out_z = zb0;
    jobs[1].k = 4;
    jobs[1].out_z = zb1;
    CHECK(aidw_batch(jobs, 2, &p, NULL));
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;

    /* end to end from the host arrays */
    float *hz32 = (float *)malloc(4 * (size_t)m), *ha32 = (float *)malloc(4 * (size_t)m);
    CHECK(aidw_interpolate_host(hx, hy, hz, n, hqx, hqy, m, &p, hz32, ha32, NULL));

    int rc = 0;
    rc |= fetch(dir, "z32.bin", z32, 4 * (size_t)m);
    rc |= fetch(dir, "alpha32.bin", a32, 4 * (size_t)m);
    rc |= fetch(dir, "zlocal.bin", zl, 4 * (size_t)m);
    rc |= fetch(dir, "z64.bin", z64, 8 * (size_t)m);
    rc |= fetch(dir, "idx.bin", idx, 4 * (size_t)m * k);
    rc |= fetch(dir, "dist.bin", dist, 4 * (size_t)m * k);
    rc |= fetch(dir, "robs.bin", robs, 4 * (size_t)m);
    rc |= fetch(dir, "zbatch0.bin", zb0, 4 * (size_t)m);
    rc |= fetch(dir, "zbatch1.bin", zb1, 4 * (size_t)m);
    rc |= write_bytes(dir, "zhost.bin", hz32, 4 * (size_t)m);
    rc |= write_bytes(dir, "alphahost.bin", ha32, 4 * (size_t)m);
    printf("ok n_col=%lld n_row=%lld cell_width=%.9g\n", (long long)info.n_col,
           (long long)info.n_row, info.cell_width);
    return rc;
}
