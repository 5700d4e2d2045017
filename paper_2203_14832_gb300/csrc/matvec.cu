// The H^2 matrix-vector product on the GPU (Sec. 4, steps 2-5).
//
//   P2M   w^{B,o} = U_B^T x^B                       leaves            (V_B = U_B)
//   M2M   w^{B,o} = sum_c C_{B_c B}^T w^{B_c,o}     levels kappa-1 .. lmin
//   M2L   u^{B,i} = sum_{B' in IL(B)} S_{B B'} w^{B',o},  S_{B B'} = K(p_{t^{B,i}}, p_{t^{B',i}})
//         evaluated on the fly over the pivot pairs (Sec. 3 step 2), all levels in one launch
//   L2L   u^{B_c,i} += C_{B_c B} u^{B,i}            levels lmin+1 .. kappa
//   L2P   y^B = U_B u^{B,i}, fused with
//   P2P   y^B += sum_{B' in N(B)} A_{t^B s^{B'}} x^{B'} evaluated on the fly (Sec. 3 step 3)
//
// Two arithmetic forms share the structure:
//   FP64: everything in double;
//   FP32: the kernel evaluations (M2L over pivot pairs, P2P over point pairs,
//         which are all but a few percent of the work) in float. Coordinates
//         are stored relative to the centre of their cell; a source cell is
//         moved into the target cell's frame by the FP64 centre difference
//         rounded once, so a distance is formed from numbers of the size of the
//         neighbourhood, not of the domain. Each target sums at most 32 sources
//         in float, then adds that partial into a compensated (two-sum) total.
//         The bases and translations (P2M, M2M, L2L, L2P: interpolation
//         operators with large entries of both signs) and the coefficient
//         vectors stay FP64.
// The scale s of the kernel multiplies each sum once at the end.
//
// Vectors in tree order are right-hand-side major: x_t[r * N + i].
#include <algorithm>

#include "nnca_internal.cuh"

namespace nnca {

namespace {

// f(r^2) with K = s f(r); FP32 and FP64 forms, one instantiation per kernel.
template <int KIND> struct KF;
template <> struct KF<NNCA_K_INV_R> {
    static __device__ __forceinline__ float f32(const KParams &, float r2) { return r2 > 0.f ? rsqrtf(r2) : 0.f; }
    static __device__ __forceinline__ float f32_far(const KParams &, float r2) { return rsqrtf(r2); }
    static __device__ __forceinline__ double f64(const KParams &, double r2) { return r2 > 0.0 ? rsqrt(r2) : 0.0; }
};
template <> struct KF<NNCA_K_LOG> {
    static __device__ __forceinline__ float f32(const KParams &, float r2) { return r2 > 0.f ? 0.5f * __logf(r2) : 0.f; }
    static __device__ __forceinline__ float f32_far(const KParams &, float r2) { return 0.5f * __logf(r2); }
    static __device__ __forceinline__ double f64(const KParams &, double r2) { return r2 > 0.0 ? 0.5 * log(r2) : 0.0; }
};
template <> struct KF<NNCA_K_GAUSS> {
    // exp(-r^2 / (2 h^2)) = 2^(r^2 * c), c = -log2(e) / (2 h^2) precomputed in kp.hf
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) { return exp2f(r2 * kp.hf); }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return exp2f(r2 * kp.hf); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) { return exp(-r2 / (2.0 * kp.h * kp.h)); }
};
template <> struct KF<NNCA_K_MATERN> {
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) { return __expf(-sqrtf(r2) / (float)kp.h); }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return f32(kp, r2); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) { return exp(-sqrt(r2) / kp.h); }
};
template <> struct KF<NNCA_K_PAPER_I> {
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) {
        if (!(r2 > 0.f)) return 0.f;
        const float a = (float)kp.h, r = sqrtf(r2);
        return r < a ? (r * (logf(r) - 1.f)) / (a * (logf(a) - 1.f)) : logf(r) / logf(a);
    }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return f32(kp, r2); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) {
        if (!(r2 > 0.0)) return 0.0;
        const double a = kp.h, r = sqrt(r2);
        return r < a ? (r * (log(r) - 1.0)) / (a * (log(a) - 1.0)) : log(r) / log(a);
    }
};
template <> struct KF<NNCA_K_PAPER_II> {
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) {
        const float a = (float)kp.h, r = sqrtf(r2);
        return r < a ? r / a : a / r;
    }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return f32(kp, r2); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) {
        const double a = kp.h, r = sqrt(r2);
        return r < a ? r / a : a / r;
    }
};

// compensated accumulation: (s, c) += v
__device__ __forceinline__ void two_sum_add(float &s, float &c, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (v - bp);
    s = t;
    c += err;
}

unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ---- permutation into tree order --------------------------------------------
template <class TI>
__global__ void k_perm_in(const TI *x, int64_t ld, int64_t N, int64_t nrhs, const int32_t *perm, double *xt,
                          float *xt32) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / N, i = e - r * N;
        const double v = (double)x[r * ld + perm[i]];
        xt[e] = v;
        if (xt32) xt32[e] = (float)v;
    }
}

// ---- P2M / M2M: w_B[b] = sum_a op_B[a][b] * src[a] (one warp per cell) -------
template <class T, int NR>
__global__ void k_upward(int64_t b0, int64_t b1, int leaf, const int32_t *cbeg, const int32_t *cend,
                         const int32_t *cch_beg, const int32_t *cch_end, const int32_t *piv_off, const int64_t *op_off,
                         const T *op, const T *xt, int64_t N, T *w, int64_t npiv) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t B = b0 + warp; B < b1; B += nw) {
        const int64_t r = piv_off[B + 1] - piv_off[B];
        if (r == 0) continue;
        const T *src;
        int64_t m, ld;
        if (leaf) {
            src = xt + cbeg[B];
            m = cend[B] - cbeg[B];
            ld = N;
        } else {
            src = w + piv_off[cch_beg[B]];
            m = piv_off[cch_end[B]] - piv_off[cch_beg[B]];
            ld = npiv;
        }
        const T *A = op + op_off[B];
        for (int64_t b = lane; b < r; b += 32) {
            T acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = 0;
            for (int64_t a = 0; a < m; ++a) {
                const T c = A[a * r + b];
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[q] += c * src[q * ld + a];
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) w[q * npiv + piv_off[B] + b] = acc[q];
        }
    }
}

// ---- L2L: u_B[a] += sum_b op_P[row0 + a][b] * u_P[b] (one warp per cell) ----
template <class T, int NR>
__global__ void k_l2l(int64_t b0, int64_t b1, const int32_t *cpar, const int32_t *cch_beg, const int32_t *piv_off,
                      const int64_t *op_off, const T *op, T *u, int64_t npiv) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t B = b0 + warp; B < b1; B += nw) {
        const int64_t P = cpar[B];
        const int64_t rB = piv_off[B + 1] - piv_off[B], rP = piv_off[P + 1] - piv_off[P];
        if (rB == 0 || rP == 0) continue;
        const int64_t row0 = piv_off[B] - piv_off[cch_beg[P]];
        const T *C = op + op_off[P] + row0 * rP;
        const T *uP = u + piv_off[P];
        for (int64_t a = lane; a < rB; a += 32) {
            T acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = 0;
            for (int64_t b = 0; b < rP; ++b) {
                const T c = C[a * rP + b];
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[q] += c * uP[q * npiv + b];
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) u[q * npiv + piv_off[B] + a] += acc[q];
        }
    }
}

// ---- M2L, FP64: one warp per target cell, source pivots staged per warp ------
constexpr int MV_WARPS = 4;

template <int KIND, int NR>
__global__ void __launch_bounds__(32 * MV_WARPS) k_m2l_f64(KParams kp, int d, const int32_t *tgt, int64_t ntgt,
                                                          const int32_t *il_off, const int32_t *il_idx,
                                                          const int32_t *piv_off, const double *pv, int64_t npiv,
                                                          const double *w, double *u) {
    __shared__ double sx[MV_WARPS][4][32];
    __shared__ double sw[MV_WARPS][NR][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp = blockIdx.x * (int64_t)MV_WARPS + wl;
    const int64_t nw = (int64_t)gridDim.x * MV_WARPS;
    for (int64_t t = warp; t < ntgt; t += nw) {
        const int64_t X = tgt[t];
        const int64_t p0 = piv_off[X], rX = piv_off[X + 1] - p0;
        for (int64_t a0 = 0; a0 < rX; a0 += 32) {
            const int64_t a = a0 + lane;
            const bool act = a < rX;
            double xa[4] = {0, 0, 0, 0};
            if (act)
                for (int k = 0; k < d; ++k) xa[k] = pv[(int64_t)k * npiv + p0 + a];
            double acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = 0.0;
            for (int32_t e = il_off[X]; e < il_off[X + 1]; ++e) {
                const int64_t Y = il_idx[e];
                const int64_t q0 = piv_off[Y], rY = piv_off[Y + 1] - q0;
                for (int64_t b0 = 0; b0 < rY; b0 += 32) {
                    const int64_t nb = min((int64_t)32, rY - b0);
                    __syncwarp();
                    if (lane < nb) {
                        for (int k = 0; k < d; ++k) sx[wl][k][lane] = pv[(int64_t)k * npiv + q0 + b0 + lane];
#pragma unroll
                        for (int q = 0; q < NR; ++q) sw[wl][q][lane] = w[q * npiv + q0 + b0 + lane];
                    }
                    __syncwarp();
                    for (int j = 0; j < nb; ++j) {
                        double r2 = 0.0;
                        for (int k = 0; k < d; ++k) {
                            const double t2 = sx[wl][k][j] - xa[k];
                            r2 = fma(t2, t2, r2);
                        }
                        const double f = KF<KIND>::f64(kp, r2);
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] = fma(f, sw[wl][q][j], acc[q]);
                    }
                }
            }
            if (act)
#pragma unroll
                for (int q = 0; q < NR; ++q) u[q * npiv + p0 + a] = kp.s * acc[q];
        }
    }
}

// ---- M2L, FP32 evaluation -----------------------------------------------------
template <int KIND, int NR>
__global__ void __launch_bounds__(32 * MV_WARPS) k_m2l_f32(KParams kp, int d, const int32_t *tgt, int64_t ntgt,
                                                          const int32_t *il_off, const int32_t *il_idx,
                                                          const int32_t *piv_off, const float *pv, int64_t npiv,
                                                          const double *ccen, int64_t ncell, const double *w,
                                                          double *u) {
    __shared__ float4 sx[MV_WARPS][32];
    __shared__ float sw[MV_WARPS][NR][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp = blockIdx.x * (int64_t)MV_WARPS + wl;
    const int64_t nw = (int64_t)gridDim.x * MV_WARPS;
    for (int64_t t = warp; t < ntgt; t += nw) {
        const int64_t X = tgt[t];
        const int64_t p0 = piv_off[X], rX = piv_off[X + 1] - p0;
        double cX[3] = {0, 0, 0};
        for (int k = 0; k < d && k < 3; ++k) cX[k] = ccen[(int64_t)k * ncell + X];
        for (int64_t a0 = 0; a0 < rX; a0 += 32) {
            const int64_t a = a0 + lane;
            const bool act = a < rX;
            float xa[3] = {0.f, 0.f, 0.f};
            if (act)
                for (int k = 0; k < d && k < 3; ++k) xa[k] = pv[(int64_t)k * npiv + p0 + a];
            float s[NR], c[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) { s[q] = 0.f; c[q] = 0.f; }
            for (int32_t e = il_off[X]; e < il_off[X + 1]; ++e) {
                const int64_t Y = il_idx[e];
                const int64_t q0 = piv_off[Y], rY = piv_off[Y + 1] - q0;
                float sh[3] = {0.f, 0.f, 0.f};
                for (int k = 0; k < d && k < 3; ++k) sh[k] = (float)(ccen[(int64_t)k * ncell + Y] - cX[k]);
                for (int64_t b0 = 0; b0 < rY; b0 += 32) {
                    const int64_t nb = min((int64_t)32, rY - b0);
                    __syncwarp();
                    if (lane < nb) {
                        const int64_t p = q0 + b0 + lane;
                        float4 v;
                        v.x = d > 0 ? pv[p] + sh[0] : 0.f;
                        v.y = d > 1 ? pv[npiv + p] + sh[1] : 0.f;
                        v.z = d > 2 ? pv[2 * npiv + p] + sh[2] : 0.f;
                        v.w = 0.f;
                        sx[wl][lane] = v;
#pragma unroll
                        for (int q = 0; q < NR; ++q) sw[wl][q][lane] = (float)w[q * npiv + p];
                    }
                    __syncwarp();
                    float part[NR];
#pragma unroll
                    for (int q = 0; q < NR; ++q) part[q] = 0.f;
#pragma unroll 4
                    for (int j = 0; j < nb; ++j) {
                        const float4 v = sx[wl][j];
                        const float dx = v.x - xa[0], dy = v.y - xa[1], dz = v.z - xa[2];
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        const float f = KF<KIND>::f32_far(kp, r2);
#pragma unroll
                        for (int q = 0; q < NR; ++q) part[q] = fmaf(f, sw[wl][q][j], part[q]);
                    }
#pragma unroll
                    for (int q = 0; q < NR; ++q) two_sum_add(s[q], c[q], part[q]);
                }
            }
            if (act)
#pragma unroll
                for (int q = 0; q < NR; ++q) u[q * npiv + p0 + a] = kp.s * ((double)s[q] + (double)c[q]);
        }
    }
}

// ---- leaves: L2P + P2P, FP64 -------------------------------------------------
template <int KIND, int NR, class TO>
__global__ void __launch_bounds__(32 * MV_WARPS) k_leaf_f64(KParams kp, int d, const int32_t *leaves, int64_t nleaf,
                                                           const int32_t *cbeg, const int32_t *cend,
                                                           const int32_t *nb_off, const int32_t *nb_idx,
                                                           const int32_t *piv_off, const int64_t *op_off,
                                                           const double *op, const double *u, int64_t npiv,
                                                           const double *xs, int64_t N, const double *xt,
                                                           const int32_t *perm, TO *y, int64_t ld) {
    __shared__ double sx[MV_WARPS][4][32];
    __shared__ double sw[MV_WARPS][NR][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp = blockIdx.x * (int64_t)MV_WARPS + wl;
    const int64_t nw = (int64_t)gridDim.x * MV_WARPS;
    const double k0 = KF<KIND>::f64(kp, 0.0);
    for (int64_t t = warp; t < nleaf; t += nw) {
        const int64_t B = leaves[t];
        const int64_t i0 = cbeg[B], nB = cend[B] - i0;
        const int64_t r = piv_off[B + 1] - piv_off[B];
        const double *U = op + op_off[B];
        for (int64_t a0 = 0; a0 < nB; a0 += 32) {
            const int64_t a = a0 + lane;
            const bool act = a < nB;
            double xa[4] = {0, 0, 0, 0};
            if (act)
                for (int k = 0; k < d; ++k) xa[k] = xs[(int64_t)k * N + i0 + a];
            double far[NR], acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) { far[q] = 0.0; acc[q] = 0.0; }
            if (act)
                for (int64_t b = 0; b < r; ++b) {
                    const double c = U[a * r + b];
#pragma unroll
                    for (int q = 0; q < NR; ++q) far[q] = fma(c, u[q * npiv + piv_off[B] + b], far[q]);
                }
            for (int32_t e = nb_off[B]; e < nb_off[B + 1]; ++e) {
                const int64_t Y = nb_idx[e];
                const int64_t j0 = cbeg[Y], nY = cend[Y] - j0;
                for (int64_t b0 = 0; b0 < nY; b0 += 32) {
                    const int64_t nb = min((int64_t)32, nY - b0);
                    __syncwarp();
                    if (lane < nb) {
                        for (int k = 0; k < d; ++k) sx[wl][k][lane] = xs[(int64_t)k * N + j0 + b0 + lane];
#pragma unroll
                        for (int q = 0; q < NR; ++q) sw[wl][q][lane] = xt[q * N + j0 + b0 + lane];
                    }
                    __syncwarp();
                    for (int j = 0; j < nb; ++j) {
                        double r2 = 0.0;
                        for (int k = 0; k < d; ++k) {
                            const double t2 = sx[wl][k][j] - xa[k];
                            r2 = fma(t2, t2, r2);
                        }
                        const double f = KF<KIND>::f64(kp, r2);
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] = fma(f, sw[wl][q][j], acc[q]);
                    }
                }
            }
            if (act) {
                const int64_t dst = perm[i0 + a];
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    // the pair (i, i) was evaluated as K(0); the diagonal takes the configured value
                    const double near = kp.s * acc[q] + (kp.diag - kp.s * k0) * xt[q * N + i0 + a];
                    y[q * ld + dst] = (TO)(far[q] + near);
                }
            }
        }
    }
}

// ---- leaves: L2P (FP64) + P2P (FP32 evaluation) ---------------------------------
template <int KIND, int NR, class TO>
__global__ void __launch_bounds__(32 * MV_WARPS) k_leaf_f32(KParams kp, int d, const int32_t *leaves, int64_t nleaf,
                                                           const int32_t *cbeg, const int32_t *cend,
                                                           const int32_t *nb_off, const int32_t *nb_idx,
                                                           const int32_t *piv_off, const int64_t *op_off,
                                                           const double *op, const double *u, int64_t npiv,
                                                           const float *xs32, int64_t N, const double *ccen,
                                                           int64_t ncell, const float *xt32, const int32_t *perm, TO *y,
                                                           int64_t ld) {
    __shared__ float4 sx[MV_WARPS][32];
    __shared__ float sw[MV_WARPS][NR][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp = blockIdx.x * (int64_t)MV_WARPS + wl;
    const int64_t nw = (int64_t)gridDim.x * MV_WARPS;
    const float k0 = KF<KIND>::f32(kp, 0.f);
    for (int64_t t = warp; t < nleaf; t += nw) {
        const int64_t B = leaves[t];
        const int64_t i0 = cbeg[B], nB = cend[B] - i0;
        const int64_t r = piv_off[B + 1] - piv_off[B];
        const double *U = op + op_off[B];
        double cB[3] = {0, 0, 0};
        for (int k = 0; k < d && k < 3; ++k) cB[k] = ccen[(int64_t)k * ncell + B];
        for (int64_t a0 = 0; a0 < nB; a0 += 32) {
            const int64_t a = a0 + lane;
            const bool act = a < nB;
            float xa[3] = {0.f, 0.f, 0.f};
            if (act)
                for (int k = 0; k < d && k < 3; ++k) xa[k] = xs32[(int64_t)k * N + i0 + a];
            double far[NR];
            float s[NR], c[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) { far[q] = 0.0; s[q] = 0.f; c[q] = 0.f; }
            if (act)
                for (int64_t b = 0; b < r; ++b) {
                    const double cc = U[a * r + b];
#pragma unroll
                    for (int q = 0; q < NR; ++q) far[q] = fma(cc, u[q * npiv + piv_off[B] + b], far[q]);
                }
            for (int32_t e = nb_off[B]; e < nb_off[B + 1]; ++e) {
                const int64_t Y = nb_idx[e];
                const int64_t j0 = cbeg[Y], nY = cend[Y] - j0;
                float sh[3] = {0.f, 0.f, 0.f};
                for (int k = 0; k < d && k < 3; ++k) sh[k] = (float)(ccen[(int64_t)k * ncell + Y] - cB[k]);
                for (int64_t b0 = 0; b0 < nY; b0 += 32) {
                    const int64_t nb = min((int64_t)32, nY - b0);
                    __syncwarp();
                    if (lane < nb) {
                        const int64_t p = j0 + b0 + lane;
                        float4 v;
                        v.x = d > 0 ? xs32[p] + sh[0] : 0.f;
                        v.y = d > 1 ? xs32[N + p] + sh[1] : 0.f;
                        v.z = d > 2 ? xs32[2 * N + p] + sh[2] : 0.f;
                        v.w = 0.f;
                        sx[wl][lane] = v;
#pragma unroll
                        for (int q = 0; q < NR; ++q) sw[wl][q][lane] = xt32[q * N + p];
                    }
                    __syncwarp();
                    float part[NR];
#pragma unroll
                    for (int q = 0; q < NR; ++q) part[q] = 0.f;
#pragma unroll 4
                    for (int j = 0; j < nb; ++j) {
                        const float4 v = sx[wl][j];
                        const float dx = v.x - xa[0], dy = v.y - xa[1], dz = v.z - xa[2];
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        const float f = KF<KIND>::f32(kp, r2);
#pragma unroll
                        for (int q = 0; q < NR; ++q) part[q] = fmaf(f, sw[wl][q][j], part[q]);
                    }
#pragma unroll
                    for (int q = 0; q < NR; ++q) two_sum_add(s[q], c[q], part[q]);
                }
            }
            if (act) {
                const int64_t dst = perm[i0 + a];
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    // the pair (i, i) was evaluated as K(0); the diagonal takes the configured value
                    const double near = kp.s * ((double)s[q] + (double)c[q]) +
                                        (kp.diag - kp.s * (double)k0) * (double)xt32[q * N + i0 + a];
                    y[q * ld + dst] = (TO)(far[q] + near);
                }
            }
        }
    }
}

// ---- non-radial kernels (FP64 only): point-based evaluation -----------------
template <int NR>
__global__ void k_m2l_generic(KParams kp, int d, const int32_t *tgt, int64_t ntgt, const int32_t *il_off,
                              const int32_t *il_idx, const int32_t *piv_off, const double *pv, int64_t npiv,
                              const double *w, double *u) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < ntgt; t += nw) {
        const int64_t X = tgt[t];
        const int64_t p0 = piv_off[X], rX = piv_off[X + 1] - p0;
        for (int64_t a = lane; a < rX; a += 32) {
            double xa[4], xb[4], acc[NR];
            for (int k = 0; k < d; ++k) xa[k] = pv[(int64_t)k * npiv + p0 + a];
            for (int q = 0; q < NR; ++q) acc[q] = 0.0;
            for (int32_t e = il_off[X]; e < il_off[X + 1]; ++e) {
                const int64_t Y = il_idx[e];
                for (int64_t b = piv_off[Y]; b < piv_off[Y + 1]; ++b) {
                    for (int k = 0; k < d; ++k) xb[k] = pv[(int64_t)k * npiv + b];
                    const double f = kern_exact(kp, xa, xb);
                    for (int q = 0; q < NR; ++q) acc[q] = fma(f, w[q * npiv + b], acc[q]);
                }
            }
            for (int q = 0; q < NR; ++q) u[q * npiv + p0 + a] = acc[q];
        }
    }
}

template <int NR, class TO>
__global__ void k_leaf_generic(KParams kp, int d, const int32_t *leaves, int64_t nleaf, const int32_t *cbeg,
                               const int32_t *cend, const int32_t *nb_off, const int32_t *nb_idx,
                               const int32_t *piv_off, const int64_t *op_off, const double *op, const double *u,
                               int64_t npiv, const double *xs, int64_t N, const double *xt, const int32_t *perm, TO *y,
                               int64_t ld) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < nleaf; t += nw) {
        const int64_t B = leaves[t];
        const int64_t i0 = cbeg[B], nB = cend[B] - i0, r = piv_off[B + 1] - piv_off[B];
        const double *U = op + op_off[B];
        for (int64_t a = lane; a < nB; a += 32) {
            double xa[4], xb[4], acc[NR];
            for (int k = 0; k < d; ++k) xa[k] = xs[(int64_t)k * N + i0 + a];
            for (int q = 0; q < NR; ++q) acc[q] = 0.0;
            for (int64_t b = 0; b < r; ++b)
                for (int q = 0; q < NR; ++q) acc[q] = fma(U[a * r + b], u[q * npiv + piv_off[B] + b], acc[q]);
            for (int32_t e = nb_off[B]; e < nb_off[B + 1]; ++e) {
                const int64_t Y = nb_idx[e];
                for (int64_t j = cbeg[Y]; j < cend[Y]; ++j) {
                    double f;
                    if (j == i0 + a) {
                        f = kp.diag;
                    } else {
                        for (int k = 0; k < d; ++k) xb[k] = xs[(int64_t)k * N + j];
                        f = kern_exact(kp, xa, xb);
                    }
                    for (int q = 0; q < NR; ++q) acc[q] = fma(f, xt[q * N + j], acc[q]);
                }
            }
            const int64_t dst = perm[i0 + a];
            for (int q = 0; q < NR; ++q) y[q * ld + dst] = (TO)acc[q];
        }
    }
}

// ---- launch helpers ----------------------------------------------------------
void ensure_workspace(Handle *h, int64_t nrhs) {
    if (h->ws && h->ws_nrhs >= nrhs) return;
    if (h->ws) {
        dev_free(h, h->ws);
        h->ws = nullptr;
    }
    // x in tree order (FP64 and FP32 copies), w and u (FP64)
    const size_t bytes = (size_t)nrhs * ((h->n + 2 * h->npiv) * sizeof(double) + h->n * sizeof(float)) + 256;
    h->ws = dev_alloc(h, bytes);
    h->ws_bytes = bytes;
    h->ws_nrhs = nrhs;
}

// One group of NR right-hand sides. FP32 == true selects FP32 kernel evaluations.
template <bool FP32, int NR, int KIND, class TO>
void run_chunk(Handle *h, const void *x, void *y, int64_t ld, int64_t r0) {
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv, nc = h->ncell;
    double *xt = (double *)h->ws;
    double *w = xt + NR * N;
    double *u = w + NR * npiv;
    float *xt32 = FP32 ? (float *)(u + NR * npiv) : nullptr;
    const TO *xin = (const TO *)x + r0 * ld;
    TO *yout = (TO *)y + r0 * ld;
    prof_mark(h, 0);
    k_perm_in<TO><<<grid_for(N * NR, 256), 256, 0, s>>>(xin, ld, N, NR, h->perm, xt, xt32);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
    prof_mark(h, 1);
    const double *op = h->op;
    if (npiv > 0) NNCA_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * NR * npiv, s));
    if (h->lmin <= h->kappa && npiv > 0) {
        const int64_t lb = h->level_base[h->kappa], le = h->level_base[h->kappa + 1];
        k_upward<double, NR><<<grid_for((le - lb) * 32, 128), 128, 0, s>>>(lb, le, 1, h->cbeg, h->cend, h->cch_beg,
                                                                           h->cch_end, h->piv_off, h->op_off, op, xt,
                                                                           N, w, npiv);
        NNCA_LAUNCH_CHECK();
        ++h->launches;
        for (int l = h->kappa - 1; l >= h->lmin; --l) {
            const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1];
            ++h->launches;
            k_upward<double, NR><<<grid_for((b1 - b0) * 32, 128), 128, 0, s>>>(b0, b1, 0, h->cbeg, h->cend,
                                                                               h->cch_beg, h->cch_end, h->piv_off,
                                                                               h->op_off, op, xt, N, w, npiv);
            NNCA_LAUNCH_CHECK();
        }
        prof_mark(h, 2);
        if (h->n_m2l_tgt > 0) {
            ++h->launches;
            const unsigned g = grid_for(h->n_m2l_tgt, MV_WARPS, 152 * 16);
            if (!kernel_is_radial(h->kp.kind)) {
                k_m2l_generic<NR><<<grid_for(h->n_m2l_tgt * 32, 128), 128, 0, s>>>(
                    h->kp, h->d, h->m2l_tgt, h->n_m2l_tgt, h->il_off, h->il_idx, h->piv_off, h->pv64, npiv, w, u);
            } else if (FP32) {
                k_m2l_f32<KIND, NR><<<g, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->m2l_tgt, h->n_m2l_tgt, h->il_off,
                                                                h->il_idx, h->piv_off, h->pv32, npiv, h->ccen, nc, w,
                                                                u);
            } else {
                k_m2l_f64<KIND, NR><<<g, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->m2l_tgt, h->n_m2l_tgt, h->il_off,
                                                                h->il_idx, h->piv_off, h->pv64, npiv, w, u);
            }
            NNCA_LAUNCH_CHECK();
        }
        prof_mark(h, 3);
        for (int l = h->lmin + 1; l <= h->kappa; ++l) {
            const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1];
            ++h->launches;
            k_l2l<double, NR><<<grid_for((b1 - b0) * 32, 128), 128, 0, s>>>(b0, b1, h->cpar, h->cch_beg, h->piv_off,
                                                                            h->op_off, op, u, npiv);
            NNCA_LAUNCH_CHECK();
        }
    }
    else {
        prof_mark(h, 2);
        prof_mark(h, 3);
    }
    prof_mark(h, 4);
    ++h->launches;
    const unsigned gl = grid_for(h->nleaf, MV_WARPS, 152 * 16);
    if (!kernel_is_radial(h->kp.kind)) {
        k_leaf_generic<NR, TO><<<grid_for(h->nleaf * 32, 128), 128, 0, s>>>(
            h->kp, h->d, h->leaf_order, h->nleaf, h->cbeg, h->cend, h->nb_off, h->nb_idx, h->piv_off, h->op_off, op, u,
            npiv, h->xs, N, xt, h->perm, yout, ld);
    } else if (FP32) {
        k_leaf_f32<KIND, NR, TO><<<gl, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->leaf_order, h->nleaf, h->cbeg, h->cend,
                                                              h->nb_off, h->nb_idx, h->piv_off, h->op_off, op, u, npiv,
                                                              h->xs32, N, h->ccen, nc, xt32, h->perm, yout, ld);
    } else {
        k_leaf_f64<KIND, NR, TO><<<gl, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->leaf_order, h->nleaf, h->cbeg, h->cend,
                                                              h->nb_off, h->nb_idx, h->piv_off, h->op_off, op, u, npiv,
                                                              h->xs, N, xt, h->perm, yout, ld);
    }
    NNCA_LAUNCH_CHECK();
    prof_mark(h, 5);
}

template <bool FP32, int KIND, class TO>
void run_all(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld) {
    int64_t r0 = 0;
    while (r0 < nrhs) {
        if (nrhs - r0 >= 4) {
            run_chunk<FP32, 4, KIND, TO>(h, x, y, ld, r0);
            r0 += 4;
        } else {
            run_chunk<FP32, 1, KIND, TO>(h, x, y, ld, r0);
            r0 += 1;
        }
    }
}

template <bool FP32, class TO>
void dispatch_kind(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld) {
    switch (h->kp.kind) {
    case NNCA_K_INV_R: run_all<FP32, NNCA_K_INV_R, TO>(h, x, y, nrhs, ld); break;
    case NNCA_K_LOG: run_all<FP32, NNCA_K_LOG, TO>(h, x, y, nrhs, ld); break;
    case NNCA_K_GAUSS: run_all<FP32, NNCA_K_GAUSS, TO>(h, x, y, nrhs, ld); break;
    case NNCA_K_MATERN: run_all<FP32, NNCA_K_MATERN, TO>(h, x, y, nrhs, ld); break;
    case NNCA_K_PAPER_I: run_all<FP32, NNCA_K_PAPER_I, TO>(h, x, y, nrhs, ld); break;
    case NNCA_K_PAPER_II: run_all<FP32, NNCA_K_PAPER_II, TO>(h, x, y, nrhs, ld); break;
    default: run_all<false, NNCA_K_INV_R, TO>(h, x, y, nrhs, ld); break;   // non-radial: generic FP64 path
    }
}

}  // namespace

void matvec(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld, int dtype, int precision) {
    const bool radial = kernel_is_radial(h->kp.kind);
    NNCA_REQUIRE(radial || precision == NNCA_PREC_FP64, NNCA_ERR_UNSUPPORTED,
                 "non-radial kernels support only the FP64 product");
    NNCA_REQUIRE(h->d <= 3 || precision == NNCA_PREC_FP64, NNCA_ERR_UNSUPPORTED,
                 "the FP32 product supports d <= 3");
    ensure_workspace(h, std::min<int64_t>(nrhs, 4));
    h->launches = 0;
    if (precision == NNCA_PREC_FP32) {
        if (dtype == NNCA_F64) dispatch_kind<true, double>(h, x, y, nrhs, ld);
        else dispatch_kind<true, float>(h, x, y, nrhs, ld);
    } else {
        if (dtype == NNCA_F64) dispatch_kind<false, double>(h, x, y, nrhs, ld);
        else dispatch_kind<false, float>(h, x, y, nrhs, ld);
    }
}

}  // namespace nnca
