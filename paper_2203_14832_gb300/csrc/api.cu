// C ABI of the NNCA library: argument checks, handle lifecycle, statistics,
// export of internal arrays, and the host-buffer product. Every entry point
// catches the library's internal errors and returns a status code.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>

#include "nnca_internal.cuh"

namespace nnca {

static thread_local std::string g_last_error;

void *dev_alloc(Handle *h, size_t bytes) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(NNCA_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    h->allocs.push_back(p);
    h->stats.device_bytes += (int64_t)bytes;
    return p;
}

void dev_free(Handle *h, void *p) {
    for (auto &q : h->allocs)
        if (q == p) {
            cudaFree(q);
            q = nullptr;
        }
}

unsigned read_status(Handle *h) {
    unsigned v = 0;
    NNCA_CUDA(cudaMemcpyAsync(&v, h->dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    NNCA_CUDA(cudaStreamSynchronize(h->stream));
    return v;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void prof_mark(Handle *h, int slot) {
    (void)slot;
    if (!h->profile) return;
    cudaEvent_t e;
    if (h->event_pool.empty()) {
        NNCA_CUDA(cudaEventCreate(&e));
    } else {
        e = h->event_pool.back();
        h->event_pool.pop_back();
    }
    NNCA_CUDA(cudaEventRecord(e, h->stream));
    h->prof_events.push_back(e);
}

namespace {

// Fold pending profiling events (6 per product) into the pass timings.
void prof_flush(Handle *h) {
    const size_t groups = h->prof_events.size() / 6;
    for (size_t g = 0; g < groups; ++g) {
        cudaEvent_t *e = &h->prof_events[g * 6];
        NNCA_CUDA(cudaEventSynchronize(e[5]));
        for (int k = 0; k < 5; ++k) {
            float ms = 0.f;
            NNCA_CUDA(cudaEventElapsedTime(&ms, e[k], e[k + 1]));
            h->stats.pass_ms[k] += ms;
        }
        float tot = 0.f;
        NNCA_CUDA(cudaEventElapsedTime(&tot, e[0], e[5]));
        h->stats.pass_ms[5] += tot;
        h->stats.pass_calls += 1;
    }
    for (cudaEvent_t e : h->prof_events) h->event_pool.push_back(e);
    h->prof_events.clear();
}

nnca_status fail(Handle *h, nnca_status s, const std::string &msg) {
    if (h) h->last_error = msg;
    g_last_error = msg;
    return s;
}

void free_all(Handle *h) {
    cudaDeviceSynchronize();
    cudaGetLastError();
    release_cross_plans(h->uid);
    for (cudaEvent_t e : h->prof_events) cudaEventDestroy(e);
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    h->prof_events.clear();
    h->event_pool.clear();
    for (void *p : h->allocs)
        if (p) cudaFree(p);
    h->allocs.clear();
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace nnca

using namespace nnca;

extern "C" {

const char *nnca_status_string(nnca_status s) {
    switch (s) {
    case NNCA_OK: return "ok";
    case NNCA_ERR_INVALID_ARG: return "invalid argument";
    case NNCA_ERR_OOM: return "out of device memory";
    case NNCA_ERR_CUDA: return "CUDA error";
    case NNCA_ERR_UNSUPPORTED: return "unsupported";
    case NNCA_ERR_TIMEOUT: return "timeout";
    case NNCA_ERR_INTERNAL: return "internal error";
    default: return "unknown status";
    }
}

const char *nnca_last_error(nnca_handle h) {
    if (h) return h->last_error.c_str();
    return g_last_error.c_str();
}

nnca_status nnca_build(const nnca_config *cfg, const double *P, int64_t nP, const double *Q, int64_t nQ, int layout,
                       void *stream, nnca_handle *out) {
    if (out) *out = nullptr;
    if (!cfg || !P || !out) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: NULL cfg, P or out");
    if (cfg->d < 1 || cfg->d > 4) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: d must be 1..4");
    if (cfg->leaf_size < 1) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: leaf_size must be >= 1");
    if (cfg->eta2_num < 1 || cfg->eta2_den < 1) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: eta^2 must be > 0");
    if (!(cfg->aca_tol > 0.0) || !std::isfinite(cfg->aca_tol))
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: aca_tol must be finite and > 0");
    if (cfg->kernel < NNCA_K_LOG || cfg->kernel > NNCA_K_POLY2)
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: unknown kernel");
    if ((cfg->kernel == NNCA_K_GAUSS || cfg->kernel == NNCA_K_MATERN || cfg->kernel == NNCA_K_PAPER_I ||
         cfg->kernel == NNCA_K_PAPER_II) && !(cfg->kparam[1] > 0.0))
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: kparam[1] (h or a) must be > 0");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(cfg->kparam[k])) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: non-finite kparam");
    if (nP < 1 || nP >= (1ll << 31)) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: need 1 <= nP < 2^31");
    if (layout != NNCA_LAYOUT_AOS && layout != NNCA_LAYOUT_SOA)
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: unknown layout");
    if (cfg->symmetric != 1)
        return fail(nullptr, NNCA_ERR_UNSUPPORTED, "nnca_build: only the symmetric form (P = Q, symmetric K) is built");
    if (cfg->m2l_form != NNCA_M2L_AUTO && cfg->m2l_form != NNCA_M2L_FULL)
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: unknown m2l_form");
    if (cfg->m2l_item_targets != 0 && (cfg->m2l_item_targets < 32 || cfg->m2l_item_targets > 256))
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: m2l_item_targets must be 0 or 32..256");
    const bool pq = Q && (Q != P || nQ != nP);
    if (pq && (nQ < 1 || nP + nQ >= (1ll << 31)))
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: need 1 <= nQ and nP + nQ < 2^31");
    if (!is_device_ptr(P) || (pq && !is_device_ptr(Q)))
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_build: P and Q must be device memory");

    static std::atomic<uint64_t> next_uid{1};
    nnca_handle_s *h = new nnca_handle_s();
    h->uid = next_uid++;
    const auto t0 = std::chrono::steady_clock::now();
    try {
        h->cfg = *cfg;
        h->d = cfg->d;
        h->n = nP;
        h->stream = (cudaStream_t)stream;
        h->kp.kind = cfg->kernel;
        h->kp.d = cfg->d;
        h->kp.s = cfg->kparam[0];
        h->kp.h = cfg->kparam[1];
        h->kp.diag = cfg->kparam[2];
        h->kp.sf = (float)cfg->kparam[0];
        if (cfg->kernel == NNCA_K_GAUSS)
            h->kp.hf = (float)(-1.4426950408889634 / (2.0 * cfg->kparam[1] * cfg->kparam[1]));
        else
            h->kp.hf = (float)cfg->kparam[1];
        h->dev_status = dalloc<unsigned>(h, 1);
        NNCA_CUDA(cudaMemsetAsync(h->dev_status, 0, sizeof(unsigned), h->stream));
        if (pq) {
            // the union [P; Q] in the caller's layout, kept only for the tree build
            h->pq = true;
            h->n_rows = nP;
            h->n_cols = nQ;
            h->n = nP + nQ;
            const int64_t n = h->n, d = cfg->d;
            double *U = nullptr;
            NNCA_CUDA(cudaMalloc(&U, sizeof(double) * n * d));
            if (layout == NNCA_LAYOUT_AOS) {
                NNCA_CUDA(cudaMemcpyAsync(U, P, sizeof(double) * nP * d, cudaMemcpyDeviceToDevice, h->stream));
                NNCA_CUDA(cudaMemcpyAsync(U + nP * d, Q, sizeof(double) * nQ * d, cudaMemcpyDeviceToDevice, h->stream));
            } else {
                for (int64_t k = 0; k < d; ++k) {
                    NNCA_CUDA(cudaMemcpyAsync(U + k * n, P + k * nP, sizeof(double) * nP, cudaMemcpyDeviceToDevice,
                                              h->stream));
                    NNCA_CUDA(cudaMemcpyAsync(U + k * n + nP, Q + k * nQ, sizeof(double) * nQ,
                                              cudaMemcpyDeviceToDevice, h->stream));
                }
            }
            try {
                build_tree(h, U, layout);
            } catch (...) {
                cudaStreamSynchronize(h->stream);
                cudaFree(U);
                throw;
            }
            NNCA_CUDA(cudaStreamSynchronize(h->stream));
            NNCA_CUDA(cudaFree(U));
        } else {
            build_tree(h, P, layout);
        }
        NNCA_REQUIRE(!(read_status(h) & DEV_BAD_INDEX), NNCA_ERR_INVALID_ARG, "nnca_build: non-finite coordinates");
        h->stats.build_ms[0] = ms_since(t0);
        auto t1 = std::chrono::steady_clock::now();
        build_lists(h);
        h->stats.build_ms[1] = ms_since(t1);
        t1 = std::chrono::steady_clock::now();
        build_pivots(h);
        h->stats.build_ms[2] = ms_since(t1);
        t1 = std::chrono::steady_clock::now();
        build_finish(h);
        h->stats.build_ms[4] = ms_since(t1);
        const unsigned st = read_status(h);
        NNCA_REQUIRE(!(st & DEV_ZERO_PIVOT), NNCA_ERR_INTERNAL, "nnca_build: exactly singular pivot block");
        NNCA_REQUIRE(!(st & ~DEV_POOL_EXHAUSTED), NNCA_ERR_INTERNAL, "nnca_build: device consistency check failed");
        // statistics
        nnca_stats &S = h->stats;
        S.d = h->d;
        S.lmax = h->lmax;
        S.kappa = h->kappa;
        S.lmin = h->lmin;
        S.n = h->n;
        S.ncell = h->ncell;
        for (int l = 0; l <= h->kappa && l < 64; ++l) S.ncell_level[l] = h->level_base[l + 1] - h->level_base[l];
        S.n_il = h->n_il;
        S.n_nb = h->n_nb;
        S.n_pivots = h->npiv;
        S.op_entries = h->nop;
        int64_t mr = 0;
        for (int64_t c = 0; c < h->ncell; ++c) mr = std::max<int64_t>(mr, h->h_piv_off[c + 1] - h->h_piv_off[c]);
        S.max_rank = mr;
        std::vector<int32_t> pt(h->ncell);
        NNCA_CUDA(cudaMemcpy(pt.data(), h->passthru, h->ncell * sizeof(int32_t), cudaMemcpyDeviceToHost));
        S.n_passthru = 0;
        for (int32_t v : pt) S.n_passthru += v;
        S.build_ms[5] = ms_since(t0);
    } catch (const Error &e) {
        const nnca_status s = e.status;
        fail(h, s, e.what());
        free_all(h);
        delete h;
        return s;
    } catch (const std::exception &e) {
        fail(h, NNCA_ERR_INTERNAL, e.what());
        free_all(h);
        delete h;
        return NNCA_ERR_INTERNAL;
    }
    *out = h;
    return NNCA_OK;
}

namespace {
// P != Q: y (rows of n_rows at pitch ld) = the P rows of the product of the union
// matrix with [0; x] (x: rows of n_cols at pitch ld). kind: the copies' direction
// for x and y (device or host buffers).
void pq_matvec(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld, int dtype, int precision, bool host) {
    cudaStream_t s = h->stream;
    const size_t es = dtype == NNCA_F64 ? 8 : 4;
    const int64_t n = h->n, np = h->n_rows, nq = h->n_cols;
    const size_t need = 2 * (size_t)n * nrhs * es;
    if (h->pq_buf_bytes < need) {
        if (h->pq_buf) dev_free(h, h->pq_buf);
        h->pq_buf = nullptr;
        h->pq_buf = dev_alloc(h, need);
        h->pq_buf_bytes = need;
    }
    char *xb = (char *)h->pq_buf;
    char *yb = xb + (size_t)n * nrhs * es;
    NNCA_CUDA(cudaMemset2DAsync(xb, n * es, 0, np * es, nrhs, s));
    NNCA_CUDA(cudaMemcpy2DAsync(xb + np * es, n * es, x, ld * es, nq * es, nrhs,
                                host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    matvec(h, xb, yb, nrhs, n, dtype, precision);
    NNCA_CUDA(cudaMemcpy2DAsync(y, ld * es, yb, n * es, np * es, nrhs,
                                host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
}
}  // namespace

nnca_status nnca_matvec(nnca_handle h, const void *x, void *y, int64_t nrhs, int64_t ld, int dtype, int precision,
                        void *stream) {
    if (!h) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec: NULL handle");
    if (!x || !y) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec: NULL x or y");
    if (nrhs < 1) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec: nrhs must be >= 1");
    if (ld < (h->pq ? std::max(h->n_rows, h->n_cols) : h->n))
        return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec: ld must be >= n (>= max(nP, nQ) for P != Q)");
    if (dtype != NNCA_F64 && dtype != NNCA_F32) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec: unknown dtype");
    if (precision < NNCA_PREC_FP64 || precision > NNCA_PREC_BF16)
        return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec: unknown precision");
    if (!is_device_ptr(x) || !is_device_ptr(y))
        return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec: x and y must be device memory");
    try {
        h->stream = (cudaStream_t)stream;
        if (h->pq) pq_matvec(h, x, y, nrhs, ld, dtype, precision, false);
        else matvec(h, x, y, nrhs, ld, dtype, precision);
        h->stats.launches_per_product = h->launches;
    } catch (const Error &e) {
        return fail(h, e.status, e.what());
    } catch (const std::exception &e) {
        return fail(h, NNCA_ERR_INTERNAL, e.what());
    }
    return NNCA_OK;
}

namespace {

// Worker streams of nnca_matvec_batch, per device, created once and kept.
constexpr int kBatchStreams = 16;
struct BatchPool {
    cudaStream_t s[kBatchStreams] = {};
    cudaEvent_t fork = nullptr, join[kBatchStreams] = {};
    bool ready = false;
};
std::mutex g_batch_mutex;
BatchPool g_batch_pool[64];

BatchPool &batch_pool() {
    int dev = 0;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_REQUIRE(dev >= 0 && dev < 64, NNCA_ERR_UNSUPPORTED, "nnca_matvec_batch: device index above 63");
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    BatchPool &P = g_batch_pool[dev];
    if (!P.ready) {
        for (int i = 0; i < kBatchStreams; ++i) {
            NNCA_CUDA(cudaStreamCreateWithFlags(&P.s[i], cudaStreamNonBlocking));
            NNCA_CUDA(cudaEventCreateWithFlags(&P.join[i], cudaEventDisableTiming));
        }
        NNCA_CUDA(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
        P.ready = true;
    }
    return P;
}

}  // namespace

nnca_status nnca_matvec_batch(const nnca_handle *hs, int count, const void *const *x, void *const *y,
                              const int64_t *ld, int64_t nrhs, int dtype, int precision, void *stream) {
    if (!hs || !x || !y || !ld) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec_batch: NULL array");
    if (count < 1 || count > 4096) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec_batch: count must be 1..4096");
    if (nrhs < 1) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec_batch: nrhs must be >= 1");
    if (dtype != NNCA_F64 && dtype != NNCA_F32) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec_batch: unknown dtype");
    if (precision < NNCA_PREC_FP64 || precision > NNCA_PREC_BF16)
        return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec_batch: unknown precision");
    std::set<const void *> seen;
    for (int k = 0; k < count; ++k) {
        const std::string at = "nnca_matvec_batch: product " + std::to_string(k) + ": ";
        if (!hs[k]) return fail(nullptr, NNCA_ERR_INVALID_ARG, at + "NULL handle");
        if (!seen.insert(hs[k]).second) return fail(nullptr, NNCA_ERR_INVALID_ARG, at + "handle repeated");
        if (!x[k] || !y[k]) return fail(nullptr, NNCA_ERR_INVALID_ARG, at + "NULL x or y");
        if (hs[k]->pq) return fail(nullptr, NNCA_ERR_UNSUPPORTED, at + "P != Q handles take nnca_matvec");
        if (ld[k] < hs[k]->n) return fail(nullptr, NNCA_ERR_INVALID_ARG, at + "ld below n");
        if (!is_device_ptr(x[k]) || !is_device_ptr(y[k]))
            return fail(nullptr, NNCA_ERR_INVALID_ARG, at + "x and y must be device memory");
    }
    int k = 0;
    try {
        BatchPool &P = batch_pool();
        const cudaStream_t s = (cudaStream_t)stream;
        const int nw = std::min(count, kBatchStreams);
        if (precision == NNCA_PREC_FP32 &&
            matvec_batch_fp32(reinterpret_cast<Handle *const *>(hs), count, x, y, ld, nrhs, dtype, s, P.s, nw, P.fork,
                              P.join)) {
            for (k = 0; k < count; ++k) hs[k]->stats.launches_per_product = hs[k]->launches;
            return NNCA_OK;
        }
        NNCA_CUDA(cudaEventRecord(P.fork, s));
        for (int i = 0; i < nw; ++i) NNCA_CUDA(cudaStreamWaitEvent(P.s[i], P.fork, 0));
        for (k = 0; k < count; ++k) {
            Handle *h = hs[k];
            h->stream = P.s[k % nw];
            matvec(h, x[k], y[k], nrhs, ld[k], dtype, precision);
            h->stats.launches_per_product = h->launches;
        }
        for (int i = 0; i < nw; ++i) {
            NNCA_CUDA(cudaEventRecord(P.join[i], P.s[i]));
            NNCA_CUDA(cudaStreamWaitEvent(s, P.join[i], 0));
        }
    } catch (const Error &e) {
        return fail(k < count ? hs[k] : nullptr, e.status, "nnca_matvec_batch: product " + std::to_string(k) + ": " + e.what());
    } catch (const std::exception &e) {
        return fail(nullptr, NNCA_ERR_INTERNAL, e.what());
    }
    return NNCA_OK;
}

nnca_status nnca_matvec_host(nnca_handle h, const void *x_host, void *y_host, int64_t nrhs, int64_t ld, int dtype,
                             int precision, void *stream) {
    if (!h) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_matvec_host: NULL handle");
    if (!x_host || !y_host) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec_host: NULL x or y");
    if (nrhs < 1 || ld < (h->pq ? std::max(h->n_rows, h->n_cols) : h->n))
        return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec_host: bad nrhs or ld");
    if (dtype != NNCA_F64 && dtype != NNCA_F32) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec_host: unknown dtype");
    if (precision < NNCA_PREC_FP64 || precision > NNCA_PREC_BF16)
        return fail(h, NNCA_ERR_INVALID_ARG, "nnca_matvec_host: unknown precision");
    try {
        cudaStream_t s = (cudaStream_t)stream;
        h->stream = s;
        if (h->pq) {
            pq_matvec(h, x_host, y_host, nrhs, ld, dtype, precision, true);
            NNCA_CUDA(cudaStreamSynchronize(s));
            NNCA_REQUIRE(!(read_status(h) & (DEV_WAIT_TIMEOUT | DEV_BAD_INDEX)), NNCA_ERR_INTERNAL,
                         "nnca_matvec_host: a device-side check of the product failed");
            return NNCA_OK;
        }
        const size_t es = dtype == NNCA_F64 ? 8 : 4;
        const size_t need = 2 * (size_t)h->n * nrhs * es;
        if (h->host_stage_bytes < need) {
            if (h->host_stage) dev_free(h, h->host_stage);
            h->host_stage = dev_alloc(h, need);
            h->host_stage_bytes = need;
        }
        char *xd = (char *)h->host_stage;
        char *yd = xd + (size_t)h->n * nrhs * es;
        NNCA_CUDA(cudaMemcpy2DAsync(xd, h->n * es, x_host, ld * es, h->n * es, nrhs, cudaMemcpyHostToDevice, s));
        matvec(h, xd, yd, nrhs, h->n, dtype, precision);
        NNCA_CUDA(cudaMemcpy2DAsync(y_host, ld * es, yd, h->n * es, h->n * es, nrhs, cudaMemcpyDeviceToHost, s));
        NNCA_CUDA(cudaStreamSynchronize(s));
        NNCA_REQUIRE(!(read_status(h) & (DEV_WAIT_TIMEOUT | DEV_BAD_INDEX)), NNCA_ERR_INTERNAL,
                     "nnca_matvec_host: a device-side check of the product failed");
    } catch (const Error &e) {
        return fail(h, e.status, e.what());
    } catch (const std::exception &e) {
        return fail(h, NNCA_ERR_INTERNAL, e.what());
    }
    return NNCA_OK;
}

nnca_status nnca_gradient(nnca_handle h, const double *x, const double *g, int64_t nrhs, int64_t ld, double *grad_p,
                          double *grad_h, void *stream) {
    if (!h) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_gradient: NULL handle");
    if (h->pq) return fail(h, NNCA_ERR_UNSUPPORTED, "nnca_gradient: the gradient is built for P = Q");
    if (!x || !g || !grad_p) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_gradient: NULL x, g or grad_p");
    if (nrhs < 1 || ld < h->n) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_gradient: bad nrhs or ld");
    if (!is_device_ptr(x) || !is_device_ptr(g) || !is_device_ptr(grad_p) || (grad_h && !is_device_ptr(grad_h)))
        return fail(h, NNCA_ERR_INVALID_ARG, "nnca_gradient: x, g, grad_p and grad_h must be device memory");
    try {
        h->stream = (cudaStream_t)stream;
        gradient(h, x, g, nrhs, ld, grad_p, grad_h);
        NNCA_REQUIRE(!(read_status(h) & DEV_ZERO_PIVOT), NNCA_ERR_INTERNAL, "nnca_gradient: singular pivot block");
    } catch (const Error &e) {
        return fail(h, e.status, e.what());
    } catch (const std::exception &e) {
        return fail(h, NNCA_ERR_INTERNAL, e.what());
    }
    return NNCA_OK;
}

nnca_status nnca_set_wait_test(int64_t wait_limit_clocks, unsigned extra_tx_bytes) {
    try {
        set_wait_test(wait_limit_clocks, extra_tx_bytes);
        set_wait_test_tc(wait_limit_clocks, extra_tx_bytes);
    } catch (const Error &e) {
        return fail(nullptr, e.status, e.what());
    }
    return NNCA_OK;
}

void nnca_destroy(nnca_handle h) {
    if (!h) return;
    free_all(h);
    delete h;
}

nnca_status nnca_get_stats(nnca_handle h, nnca_stats *out) {
    if (!h || !out) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_get_stats: NULL argument");
    try {
        prof_flush(h);
        h->stats.device_status = read_status(h);
    } catch (const Error &e) {
        return fail(h, e.status, e.what());
    }
    *out = h->stats;
    return NNCA_OK;
}

nnca_status nnca_set_profiling(nnca_handle h, int on) {
    if (!h) return fail(nullptr, NNCA_ERR_INVALID_ARG, "nnca_set_profiling: NULL handle");
    try {
        prof_flush(h);
    } catch (const Error &e) {
        return fail(h, e.status, e.what());
    }
    if (on) {
        for (double &v : h->stats.pass_ms) v = 0.0;
        h->stats.pass_calls = 0;
    }
    h->profile = on != 0;
    return NNCA_OK;
}

nnca_status nnca_export(nnca_handle h, int what, void *buf, int64_t cap, int64_t *bytes) {
    if (!h || !bytes) return fail(h, NNCA_ERR_INVALID_ARG, "nnca_export: NULL argument");
    const int64_t nc = h->ncell, n = h->n, np = h->npiv;
    const void *src = nullptr;
    int64_t count = 0;
    int kind = 0;   // 0: int32 -> int64, 1: int64, 2: uint64, 3: double, 4: host int64
    std::vector<int64_t> host64;
    switch (what) {
    case NNCA_EXPORT_PERM: src = h->perm; count = n; kind = 0; break;
    case NNCA_EXPORT_KEYS: src = h->keys; count = n; kind = 2; break;
    case NNCA_EXPORT_LEVEL_BASE: host64 = h->level_base; count = (int64_t)host64.size(); kind = 4; break;
    case NNCA_EXPORT_CKEY: src = h->ckey; count = nc; kind = 2; break;
    case NNCA_EXPORT_CBEG: src = h->cbeg; count = nc; kind = 0; break;
    case NNCA_EXPORT_CEND: src = h->cend; count = nc; kind = 0; break;
    case NNCA_EXPORT_CPAR: src = h->cpar; count = nc; kind = 0; break;
    case NNCA_EXPORT_CCH_BEG: src = h->cch_beg; count = nc; kind = 0; break;
    case NNCA_EXPORT_CCH_END: src = h->cch_end; count = nc; kind = 0; break;
    case NNCA_EXPORT_NB_OFF: src = h->nb_off; count = nc + 1; kind = 0; break;
    case NNCA_EXPORT_NB_IDX: src = h->nb_idx; count = h->n_nb; kind = 0; break;
    case NNCA_EXPORT_IL_OFF: src = h->il_off; count = nc + 1; kind = 0; break;
    case NNCA_EXPORT_IL_IDX: src = h->il_idx; count = h->n_il; kind = 0; break;
    case NNCA_EXPORT_PIV_OFF: src = h->piv_off; count = nc + 1; kind = 0; break;
    case NNCA_EXPORT_PIV_ROW: src = h->piv_row; count = np; kind = 0; break;
    case NNCA_EXPORT_PIV_COL: src = h->piv_col; count = np; kind = 0; break;
    case NNCA_EXPORT_PASSTHRU: src = h->passthru; count = nc; kind = 0; break;
    case NNCA_EXPORT_CAND_OFF: src = h->cand_off; count = nc + 1; kind = 1; break;
    case NNCA_EXPORT_OP_OFF: src = h->op_off; count = nc + 1; kind = 1; break;
    case NNCA_EXPORT_OP: src = h->op; count = h->nop; kind = 3; break;
    default: return fail(h, NNCA_ERR_INVALID_ARG, "nnca_export: unknown array");
    }
    *bytes = count * 8;
    if (!buf) return NNCA_OK;
    try {
        const int64_t ncopy = std::min<int64_t>(count, cap / 8);
        if (ncopy <= 0) return NNCA_OK;
        if (kind == 4) {
            std::memcpy(buf, host64.data(), ncopy * 8);
        } else if (kind == 0) {
            std::vector<int32_t> tmp(ncopy);
            NNCA_CUDA(cudaMemcpy(tmp.data(), src, ncopy * 4, cudaMemcpyDeviceToHost));
            int64_t *o = (int64_t *)buf;
            for (int64_t i = 0; i < ncopy; ++i) o[i] = tmp[i];
        } else {
            NNCA_CUDA(cudaMemcpy(buf, src, ncopy * 8, cudaMemcpyDeviceToHost));
        }
    } catch (const Error &e) {
        return fail(h, e.status, e.what());
    }
    return NNCA_OK;
}

}  // extern "C"
