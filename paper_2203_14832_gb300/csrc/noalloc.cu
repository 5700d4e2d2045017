// nnca_matvec_noalloc: the H^2 product for one right-hand side without any
// device allocation.
//
// nnca_matvec allocates its workspace (the vector in tree order, the multipole
// and local coefficients) with cudaMalloc on its first call. Some callers
// cannot allocate at that point: code that runs under a fixed device-memory
// budget already handed to its own allocator, or latency-critical loops that
// cannot accept cudaMalloc's implicit device synchronisation. This entry point
// takes its workspace from one file-scope device array of NNCA_NOALLOC_BYTES
// instead. The array is part of the library's device image: every GPU that
// loads the library holds it until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (host code may not use the symbol itself as a device
// pointer), so make that first call before any stream capture. All calls, on
// any stream, share the array and it keeps the last call's contents: the
// coefficients that must start at zero are cleared by every call, and calls
// whose work overlaps on the GPU race on the array.
#include <mutex>

#include "nnca_internal.cuh"

namespace {

constexpr size_t kScratchBytes = NNCA_NOALLOC_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mutex;
void *g_scratch_ptr[256] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
nnca_status scratch_address(void **out, std::string &err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        err = "nnca_matvec_noalloc: no current CUDA device";
        return NNCA_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            err = std::string("nnca_matvec_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return NNCA_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NNCA_OK;
}

}  // namespace

extern "C" nnca_status nnca_matvec_noalloc(nnca_handle hh, const void *x, void *y, int64_t ld, int dtype,
                                           int precision, void *stream) {
    nnca::Handle *h = static_cast<nnca::Handle *>(hh);
    if (!h) return NNCA_ERR_INVALID_ARG;
    if (h->pq) {
        h->last_error = "nnca_matvec_noalloc: P != Q handles take nnca_matvec";
        return NNCA_ERR_UNSUPPORTED;
    }
    if (!x || !y || ld < h->n || (dtype != NNCA_F64 && dtype != NNCA_F32) ||
        (precision != NNCA_PREC_FP64 && precision != NNCA_PREC_FP32)) {
        h->last_error = "nnca_matvec_noalloc: invalid x, y, ld, dtype or precision";
        return NNCA_ERR_INVALID_ARG;
    }
    if (!nnca::is_device_ptr(x) || !nnca::is_device_ptr(y)) {
        h->last_error = "nnca_matvec_noalloc: x and y must be device memory";
        return NNCA_ERR_INVALID_ARG;
    }
    if (h->profile) {
        h->last_error = "nnca_matvec_noalloc: turn profiling off first (it creates events)";
        return NNCA_ERR_INVALID_ARG;
    }
    // the workspace of one right-hand side: x in tree order (double and float),
    // w and u (double), w (float)
    const size_t need = (size_t)(h->n + 2 * h->npiv) * sizeof(double) + (size_t)(h->n + h->npiv) * sizeof(float) + 256;
    if (need > kScratchBytes) {
        h->last_error = "nnca_matvec_noalloc: the problem needs " + std::to_string(need) +
                        " bytes of workspace, more than the fixed " + std::to_string(kScratchBytes) +
                        " (12 * n + 20 * pivots + 256 bytes)";
        return NNCA_ERR_INVALID_ARG;
    }
    void *scratch = nullptr;
    std::string err;
    nnca_status st = scratch_address(&scratch, err);
    if (st != NNCA_OK) {
        h->last_error = err;
        return st;
    }
    // run the ordinary product on the fixed array: the workspace check in the
    // product finds a workspace of one right-hand side and allocates nothing
    void *saved_ws = h->ws;
    const size_t saved_bytes = h->ws_bytes;
    const int64_t saved_nrhs = h->ws_nrhs;
    h->ws = scratch;
    h->ws_bytes = kScratchBytes;
    h->ws_nrhs = 1;
    h->no_alloc = true;   // paths that would allocate their tables take their allocation-free form
    st = NNCA_OK;
    try {
        h->stream = (cudaStream_t)stream;
        nnca::matvec(h, x, y, 1, ld, dtype, precision);
        h->stats.launches_per_product = h->launches;
    } catch (const nnca::Error &e) {
        h->last_error = e.what();
        st = e.status;
    } catch (const std::exception &e) {
        h->last_error = e.what();
        st = NNCA_ERR_INTERNAL;
    }
    h->ws = saved_ws;
    h->ws_bytes = saved_bytes;
    h->ws_nrhs = saved_nrhs;
    h->no_alloc = false;
    return st;
}
