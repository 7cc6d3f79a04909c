// aidw_interpolate_noalloc: the AIDW prediction of aidw_interpolate with its
// per-call scratch in a fixed array of the library's device image instead of
// an allocation, for callers that cannot let the library allocate (see
// include/aidw.h).  The kNN and weighting kernels are the ones
// aidw_interpolate launches; the query cell-ordering pass that
// aidw_interpolate runs first (from 4096 queries) is left out, because its
// temporaries would need an allocation.
#include <mutex>

#include "aidw_internal.cuh"

namespace {

// Scratch: [kNN records (24 B per query), rounded up to 256 B][partial sums].
// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[AIDW_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (the current device).  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up once per device with cudaGetSymbolAddress.  That look-up is host
// set-up (it may load the library's device code), which must not happen
// while `s` is being captured into a graph: such a first call is refused.
aidw_status scratch_address(int device, cudaStream_t s, void **out)
{
    if (device < 0 || device >= kMaxDevices) return AIDW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[device]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
            cudaGetLastError();
            return AIDW_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) return AIDW_ERR_INVALID_ARG;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return AIDW_ERR_CUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return AIDW_OK;
}

}  // namespace

extern "C" aidw_status aidw_interpolate_noalloc(const aidw_grid *g, const float *qx,
                                                const float *qy, int64_t n_query,
                                                const aidw_params *p, void *out_z,
                                                void *out_alpha, aidw_stream_t stream)
{
    using namespace aidw;
    NvtxRange nvtx_("aidw_interpolate_noalloc");
    if (!g || n_query < 0 || n_query > AIDW_NOALLOC_MAX_QUERIES) return AIDW_ERR_INVALID_ARG;
    const aidw_status ps = api_detail::check_params(p, true);
    if (ps != AIDW_OK) return ps;
    if (p->k > g->n_data) return AIDW_ERR_K_RANGE;
    if (n_query == 0) return AIDW_OK;
    if (!qx || !qy || !out_z) return AIDW_ERR_INVALID_ARG;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return AIDW_ERR_CUDA;
    }
    if (device != g->device) return AIDW_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *base = nullptr;
    aidw_status st = scratch_address(device, s, &base);
    if (st != AIDW_OK) return st;

    const size_t rec_bytes = (sizeof(QRec) * (size_t)n_query + 255) / 256 * 256;
    QRec *recs = static_cast<QRec *>(base);
    void *part = static_cast<unsigned char *>(base) + rec_bytes;
    const size_t part_bytes = (size_t)AIDW_NOALLOC_SCRATCH_BYTES - rec_bytes;

    const bool fp64 = p->precision == AIDW_FP64_PLAIN;
    // sort = false: the pass that visits the queries in grid-cell order needs
    // pool memory, so the kNN takes the queries in input order (same results,
    // slower on clustered data)
    st = knn_launch(g, qx, qy, n_query, p->k, fp64, api_detail::alpha_params(p), recs, nullptr,
                    nullptr, nullptr, out_alpha, s, nullptr, false);
    if (st == AIDW_OK)
        st = weight_launch_scratch(g, qx, qy, n_query, fp64, recs, out_z, part, part_bytes, s);
    return st;
}
