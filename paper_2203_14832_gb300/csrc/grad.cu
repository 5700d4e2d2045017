// Gradient of L = g^T A~ x with respect to the points and the kernel parameter h,
// with every index set of the build held (the pivots fixed).
//
// A~ is the H^2 matrix of the handle: near blocks K(p_X, p_Y), Y in N(X) (Sec. 3
// step 3), and far blocks U_X S_XY U_Y^T, Y in IL(X) (Sec. 3 step 2), with the
// nested bases of Sec. 2.3.1: X_B = A_{t~ sigma} (A_{tau sigma})^{-1} per cell
// (Eqs. 11 and 14). Reverse mode through the product of Sec. 4:
//   1. the FP64 product of x and of g gives the multipoles w(x), w(g) of every
//      cell and the local coefficients u(x), u(g) after L2L; u(g) is dL/dw(x)
//      and u(x) is dL/dw(g) (A~ is symmetric under V_B = U_B);
//   2. near field: dL/dp_i += sum_j grad_a K(p_i, p_j) (g_i x_j + x_i g_j);
//   3. interaction lists: a pivot a of cell B at point i gets
//      sum_{Y in IL(B)} sum_b grad_a K(p_i, p_{t^{Y,i}_b}) (w_B(g)_a w_Y(x)_b + w_B(x)_a w_Y(g)_b);
//   4. bases: dL/dX_B = z(x) u_B(g)^T + z(g) u_B(x)^T (z the vector X_B
//      multiplies in the upward pass), and dX = (dA_{t~ sigma} - X dA_{tau sigma})
//      A_{tau sigma}^{-1}, so the entries of A_{t~ sigma} take the adjoint
//      H = z(x) a^T + z(g) b^T with A_{tau sigma} a = u_B(g), A_{tau sigma} b = u_B(x),
//      and the entries of A_{tau sigma} take -X^T H = -(w_B(x) a^T + w_B(g) b^T);
//      an entry K(p_i, p_j) passes its adjoint times grad_a K to p_i and times
//      -grad_a K to p_j.
// dK/dh in place of grad_a K gives dL/dh. Everything is FP64; contributions to a
// point from several cells are added with atomics (the order of those FP64 adds
// is not fixed). Diagonal entries (a fixed value) and distinct points at r = 0
// carry no derivative.
#include <algorithm>

#include "nnca_internal.cuh"

namespace nnca {

namespace {

// K = s f(r): grad_a K(a, b) = dk.g * (a - b) and dK/dh = dk.h
struct KDer {
    double g, h;
};
__device__ __forceinline__ KDer kder(const KParams &kp, double r2) {
    KDer o{0.0, 0.0};
    switch (kp.kind) {
    case NNCA_K_INV_R:   // f = 1/r, f'/r = -1/r^3
        if (r2 > 0.0) {
            const double r = sqrt(r2);
            o.g = -kp.s / (r2 * r);
        }
        break;
    case NNCA_K_LOG:     // f = log r, f'/r = 1/r^2
        if (r2 > 0.0) o.g = kp.s / r2;
        break;
    case NNCA_K_GAUSS: { // f = exp(-r^2 / (2 h^2)), f'/r = -f / h^2, df/dh = r^2 f / h^3
        const double f = exp(-r2 / (2.0 * kp.h * kp.h));
        o.g = -kp.s * f / (kp.h * kp.h);
        o.h = kp.s * r2 * f / (kp.h * kp.h * kp.h);
        break;
    }
    case NNCA_K_MATERN: { // f = exp(-r / h), f'/r = -f / (h r), df/dh = r f / h^2
        const double r = sqrt(r2);
        const double f = exp(-r / kp.h);
        if (r > 0.0) o.g = -kp.s * f / (kp.h * r);
        o.h = kp.s * r * f / (kp.h * kp.h);
        break;
    }
    default: break;
    }
    return o;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int GW = 4;   // warps per block of the near and interaction kernels

// 2. near field, one warp per leaf, a lane per target; gs = grad in sorted order [n][d]
__global__ void __launch_bounds__(32 * GW) k_grad_near(KParams kp, int d, int64_t l0, int64_t l1, const int32_t *cbeg,
                                                       const int32_t *cend, const int32_t *nb_off,
                                                       const int32_t *nb_idx, const double *xs, int64_t N,
                                                       const double *vx, const double *vg, double *gs, double *dh) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * GW;
    double dha = 0.0;
    for (int64_t B = l0 + blockIdx.x * (int64_t)GW + (threadIdx.x >> 5); B < l1; B += nw) {
        const int64_t i0 = cbeg[B], nB = cend[B] - i0;
        for (int64_t a0 = 0; a0 < nB; a0 += 32) {
            const int64_t i = i0 + a0 + lane;
            const bool act = a0 + lane < nB;
            double p[4] = {0, 0, 0, 0}, acc[4] = {0, 0, 0, 0};
            double xi = 0.0, gi = 0.0;
            if (act) {
                for (int k = 0; k < d; ++k) p[k] = xs[(int64_t)k * N + i];
                xi = vx[i];
                gi = vg[i];
            }
            for (int32_t e = nb_off[B]; e < nb_off[B + 1]; ++e) {
                const int64_t Y = nb_idx[e];
                for (int64_t j = cbeg[Y]; j < cend[Y]; ++j) {
                    if (!act || j == i) continue;
                    double dv[4] = {0, 0, 0, 0}, r2 = 0.0;
                    for (int k = 0; k < d; ++k) {
                        dv[k] = p[k] - xs[(int64_t)k * N + j];
                        r2 = fma(dv[k], dv[k], r2);
                    }
                    const KDer q = kder(kp, r2);
                    const double xj = vx[j], gj = vg[j];
                    const double c = q.g * (gi * xj + xi * gj);
                    for (int k = 0; k < d; ++k) acc[k] = fma(c, dv[k], acc[k]);
                    dha = fma(gi * xj, q.h, dha);
                }
            }
            if (act)
                for (int k = 0; k < d; ++k) gs[i * d + k] += acc[k];
        }
    }
    dha = warp_sum(dha);
    if (lane == 0 && dha != 0.0) atomicAdd(dh, dha);
}

// 3. interaction lists, one warp per cell with a non-empty list, a lane per pivot
__global__ void __launch_bounds__(32 * GW) k_grad_il(KParams kp, int d, const int32_t *tgt, int64_t ntgt,
                                                     const int32_t *il_off, const int32_t *il_idx,
                                                     const int32_t *piv_off, const int32_t *piv_row, const double *pv,
                                                     int64_t npiv, const double *wx, const double *wg, double *gs,
                                                     double *dh) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * GW;
    double dha = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)GW + (threadIdx.x >> 5); t < ntgt; t += nw) {
        const int64_t X = tgt[t];
        const int64_t q0 = piv_off[X], r = piv_off[X + 1] - q0;
        for (int64_t a0 = 0; a0 < r; a0 += 32) {
            const int64_t a = q0 + a0 + lane;
            const bool act = a0 + lane < r;
            double p[4] = {0, 0, 0, 0}, acc[4] = {0, 0, 0, 0};
            double wxa = 0.0, wga = 0.0;
            if (act) {
                for (int k = 0; k < d; ++k) p[k] = pv[(int64_t)k * npiv + a];
                wxa = wx[a];
                wga = wg[a];
            }
            for (int32_t e = il_off[X]; e < il_off[X + 1]; ++e) {
                const int64_t Y = il_idx[e];
                for (int64_t b = piv_off[Y]; b < piv_off[Y + 1]; ++b) {
                    if (!act) continue;
                    double dv[4] = {0, 0, 0, 0}, r2 = 0.0;
                    for (int k = 0; k < d; ++k) {
                        dv[k] = p[k] - pv[(int64_t)k * npiv + b];
                        r2 = fma(dv[k], dv[k], r2);
                    }
                    const KDer q = kder(kp, r2);
                    const double c = q.g * (wga * wx[b] + wxa * wg[b]);
                    for (int k = 0; k < d; ++k) acc[k] = fma(c, dv[k], acc[k]);
                    dha = fma(wga * wx[b], q.h, dha);
                }
            }
            if (act)
                for (int k = 0; k < d; ++k) atomicAdd(&gs[(int64_t)piv_row[a] * d + k], acc[k]);
        }
    }
    dha = warp_sum(dha);
    if (lane == 0 && dha != 0.0) atomicAdd(dh, dha);
}

// 4. bases, one block per cell: LU of A_{tau sigma} (partial pivoting), the two
// solves, then the adjoints of the entries of A_{t~ sigma} and A_{tau sigma}
constexpr int GB = 128;

struct BasisArgs {
    KParams kp;
    int d;
    int64_t N, npiv;
    const int32_t *cells;        // cells with a basis to differentiate
    int64_t ncells;
    int kappa_first;             // first global id of the leaf level
    const int32_t *cbeg, *cend, *cch_beg, *cch_end, *piv_off, *piv_row, *piv_col;
    const double *xs, *xt;       // sorted coordinates [d][N]; x and g in tree order [2][N]
    const double *w, *u;         // [2][npiv]: x's and g's multipoles and local coefficients
    const int64_t *lu_off;       // r * r per cell
    double *lu;
    int32_t *ipiv;               // r per cell (at piv_off)
    double *sol;                 // 2 r per cell (at 2 piv_off): a then b
    double *gs, *dh;
    unsigned *status;
};

__device__ __forceinline__ void load3(const double *xs, int64_t N, int d, int64_t i, double *p) {
    for (int k = 0; k < d; ++k) p[k] = xs[(int64_t)k * N + i];
}

__global__ void __launch_bounds__(GB) k_grad_basis(BasisArgs A) {
    __shared__ double red[GB / 32];
    __shared__ long long redi[GB / 32];
    __shared__ double sh_dh[GB / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int d = A.d;
    double dha = 0.0;
    for (int64_t ci = blockIdx.x; ci < A.ncells; ci += gridDim.x) {
        const int64_t X = A.cells[ci];
        const int64_t q0 = A.piv_off[X], r = A.piv_off[X + 1] - q0;
        const bool leaf = X >= A.kappa_first;
        // candidate rows: the leaf's points, or the children's pivots (contiguous)
        const int64_t c0 = leaf ? A.cbeg[X] : A.piv_off[A.cch_beg[X]];
        const int64_t m = leaf ? A.cend[X] - A.cbeg[X] : A.piv_off[A.cch_end[X]] - c0;
        double *L = A.lu + A.lu_off[ci];
        int32_t *ip = A.ipiv + q0;
        double *sa = A.sol + 2 * q0, *sb = sa + r;
        // M(a, b) = K(p_{tau_a}, p_{sigma_b}); right-hand sides u(g) and u(x)
        for (int64_t e = t; e < r * r; e += GB) {
            const int64_t a = e / r, b = e % r;
            double p[4], q[4];
            load3(A.xs, A.N, d, A.piv_row[q0 + a], p);
            load3(A.xs, A.N, d, A.piv_col[q0 + b], q);
            L[e] = kern_exact(A.kp, p, q);
        }
        for (int64_t a = t; a < r; a += GB) {
            sa[a] = A.u[A.npiv + q0 + a];
            sb[a] = A.u[q0 + a];
        }
        __syncthreads();
        // LU with partial pivoting, right-looking; the row swaps applied to both solves
        for (int64_t c = 0; c < r; ++c) {
            double bv = -1.0;
            long long bi = -1;
            for (int64_t a = c + t; a < r; a += GB)
                if (fabs(L[a * r + c]) > bv) { bv = fabs(L[a * r + c]); bi = a; }
            for (int o = 16; o; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
                const long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (i2 >= 0 && (bi < 0 || v2 > bv || (v2 == bv && i2 < bi))) { bv = v2; bi = i2; }
            }
            if (lane == 0) { red[wid] = bv; redi[wid] = bi; }
            __syncthreads();
            if (t == 0) {
                for (int w = 1; w < GB / 32; ++w)
                    if (redi[w] >= 0 && (redi[0] < 0 || red[w] > red[0] || (red[w] == red[0] && redi[w] < redi[0]))) {
                        red[0] = red[w];
                        redi[0] = redi[w];
                    }
                ip[c] = (int32_t)redi[0];
                if (!(red[0] > 0.0)) atomicOr(A.status, DEV_ZERO_PIVOT);
            }
            __syncthreads();
            const int64_t p = ip[c];
            if (p != c) {
                for (int64_t j = t; j < r; j += GB) {
                    const double tmp = L[c * r + j];
                    L[c * r + j] = L[p * r + j];
                    L[p * r + j] = tmp;
                }
                if (t == 0) {
                    double tmp = sa[c]; sa[c] = sa[p]; sa[p] = tmp;
                    tmp = sb[c]; sb[c] = sb[p]; sb[p] = tmp;
                }
            }
            __syncthreads();
            const double piv = L[c * r + c];
            for (int64_t a = c + 1 + t; a < r; a += GB) L[a * r + c] = piv != 0.0 ? L[a * r + c] / piv : 0.0;
            __syncthreads();
            const int64_t wdt = r - c - 1;
            for (int64_t e = t; e < wdt * wdt; e += GB) {
                const int64_t a = c + 1 + e / wdt, j = c + 1 + e % wdt;
                L[a * r + j] = fma(-L[a * r + c], L[c * r + j], L[a * r + j]);
            }
            for (int64_t a = c + 1 + t; a < r; a += GB) {
                sa[a] = fma(-L[a * r + c], sa[c], sa[a]);
                sb[a] = fma(-L[a * r + c], sb[c], sb[a]);
            }
            __syncthreads();
        }
        // back substitution (one thread: r is at most a few hundred)
        if (t == 0)
            for (int64_t a = r - 1; a >= 0; --a) {
                double va = sa[a], vb = sb[a];
                for (int64_t j = a + 1; j < r; ++j) {
                    va = fma(-L[a * r + j], sa[j], va);
                    vb = fma(-L[a * r + j], sb[j], vb);
                }
                const double piv = L[a * r + a];
                sa[a] = piv != 0.0 ? va / piv : 0.0;
                sb[a] = piv != 0.0 ? vb / piv : 0.0;
            }
        __syncthreads();
        // z(x), z(g) of candidate row i: the leaf's x and g, or the children's multipoles
        auto zx = [&](int64_t i) { return leaf ? A.xt[c0 + i] : A.w[c0 + i]; };
        auto zg = [&](int64_t i) { return leaf ? A.xt[A.N + c0 + i] : A.w[A.npiv + c0 + i]; };
        auto rowpt = [&](int64_t i) { return leaf ? (int64_t)(c0 + i) : (int64_t)A.piv_row[c0 + i]; };
        // entries of A_{t~ sigma}: adjoint z(x)_i a_b + z(g)_i b_b (rows, then columns)
        for (int64_t i = t; i < m; i += GB) {
            double p[4], acc[4] = {0, 0, 0, 0};
            const int64_t pi = rowpt(i);
            load3(A.xs, A.N, d, pi, p);
            const double zxi = zx(i), zgi = zg(i);
            for (int64_t b = 0; b < r; ++b) {
                double q[4], dv[4], r2 = 0.0;
                load3(A.xs, A.N, d, A.piv_col[q0 + b], q);
                for (int k = 0; k < d; ++k) { dv[k] = p[k] - q[k]; r2 = fma(dv[k], dv[k], r2); }
                const KDer kd = kder(A.kp, r2);
                const double adj = zxi * sa[b] + zgi * sb[b];
                for (int k = 0; k < d; ++k) acc[k] = fma(adj * kd.g, dv[k], acc[k]);
                dha = fma(adj, kd.h, dha);
            }
            for (int k = 0; k < d; ++k) atomicAdd(&A.gs[pi * d + k], acc[k]);
        }
        for (int64_t b = t; b < r; b += GB) {
            double q[4], acc[4] = {0, 0, 0, 0};
            const int64_t pb = A.piv_col[q0 + b];
            load3(A.xs, A.N, d, pb, q);
            for (int64_t i = 0; i < m; ++i) {
                double p[4], dv[4], r2 = 0.0;
                load3(A.xs, A.N, d, rowpt(i), p);
                for (int k = 0; k < d; ++k) { dv[k] = p[k] - q[k]; r2 = fma(dv[k], dv[k], r2); }
                const KDer kd = kder(A.kp, r2);
                const double adj = zx(i) * sa[b] + zg(i) * sb[b];
                for (int k = 0; k < d; ++k) acc[k] = fma(-adj * kd.g, dv[k], acc[k]);
            }
            // entries of A_{tau sigma}: adjoint -(w(x)_a a_b + w(g)_a b_b)
            for (int64_t a = 0; a < r; ++a) {
                double p[4], dv[4], r2 = 0.0;
                const int64_t pa = A.piv_row[q0 + a];
                load3(A.xs, A.N, d, pa, p);
                for (int k = 0; k < d; ++k) { dv[k] = p[k] - q[k]; r2 = fma(dv[k], dv[k], r2); }
                const KDer kd = kder(A.kp, r2);
                const double mb = -(A.w[q0 + a] * sa[b] + A.w[A.npiv + q0 + a] * sb[b]);
                for (int k = 0; k < d; ++k) acc[k] = fma(-mb * kd.g, dv[k], acc[k]);
                double g3[4];
                for (int k = 0; k < d; ++k) g3[k] = mb * kd.g * dv[k];
                for (int k = 0; k < d; ++k) atomicAdd(&A.gs[pa * d + k], g3[k]);
                dha = fma(mb, kd.h, dha);
            }
            for (int k = 0; k < d; ++k) atomicAdd(&A.gs[pb * d + k], acc[k]);
        }
        __syncthreads();
    }
    dha = warp_sum(dha);
    if (lane == 0) sh_dh[wid] = dha;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < GB / 32; ++w) s += sh_dh[w];
        if (s != 0.0) atomicAdd(A.dh, s);
    }
}

// the gradient in the caller's order, n x d row-major
__global__ void k_grad_out(int64_t n, int d, const int32_t *perm, const double *gs, double *out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d, k = e - i * d;
        out[(int64_t)perm[i] * d + k] = gs[e];
    }
}

// x and g of one right-hand side into the first two of four columns (caller order)
__global__ void k_grad_stage(int64_t n, const double *x, const double *g, double *X4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        X4[i] = x[i];
        X4[n + i] = g[i];
        X4[2 * n + i] = 0.0;
        X4[3 * n + i] = 0.0;
    }
}

unsigned gridn(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

}  // namespace

void gradient(Handle *h, const double *x, const double *g, int64_t nrhs, int64_t ld, double *grad_p, double *grad_h) {
    const int kind = h->kp.kind;
    NNCA_REQUIRE(kind == NNCA_K_INV_R || kind == NNCA_K_LOG || kind == NNCA_K_GAUSS || kind == NNCA_K_MATERN,
                 NNCA_ERR_UNSUPPORTED, "nnca_gradient: the log, 1/r, Gaussian and Matern kernels only");
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv, d = h->d;
    Scratch scr;
    double *X4 = scr.get<double>(4 * N), *Y4 = scr.get<double>(4 * N);
    double *gs = scr.get<double>(N * d), *dh = scr.get<double>(1);
    NNCA_CUDA(cudaMemsetAsync(gs, 0, sizeof(double) * N * d, s));
    NNCA_CUDA(cudaMemsetAsync(dh, 0, sizeof(double), s));
    // bases with a derivative: levels lmin .. kappa, not pass-through, rank > 0
    std::vector<int32_t> hcells;
    std::vector<int32_t> pt(h->ncell);
    NNCA_CUDA(cudaMemcpy(pt.data(), h->passthru, h->ncell * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int64_t> hlu(1, 0);
    if (h->lmin <= h->kappa)
        for (int64_t c = h->level_base[h->lmin]; c < h->level_base[h->kappa + 1]; ++c) {
            const int64_t r = h->h_piv_off[c + 1] - h->h_piv_off[c];
            if (pt[c] || r == 0) continue;
            hcells.push_back((int32_t)c);
            hlu.push_back(hlu.back() + r * r);
        }
    const int64_t nbc = (int64_t)hcells.size();
    int32_t *cells = scr.get<int32_t>(nbc);
    int64_t *lu_off = scr.get<int64_t>(nbc + 1);
    if (nbc) {
        NNCA_CUDA(cudaMemcpyAsync(cells, hcells.data(), nbc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        NNCA_CUDA(cudaMemcpyAsync(lu_off, hlu.data(), (nbc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    double *lu = scr.get<double>(hlu.back());
    int32_t *ipiv = scr.get<int32_t>(npiv);
    double *sol = scr.get<double>(2 * npiv);
    for (int64_t r = 0; r < nrhs; ++r) {
        k_grad_stage<<<gridn(N, 256), 256, 0, s>>>(N, x + r * ld, g + r * ld, X4);
        NNCA_LAUNCH_CHECK();
        // FP64 product of x and g: the workspace then holds x, g in tree order and
        // their multipoles and local coefficients (a pass of four right-hand sides)
        matvec(h, X4, Y4, 4, N, NNCA_F64, NNCA_PREC_FP64);
        const double *xt = (const double *)h->ws;
        const double *w = xt + 4 * N;
        const double *u = w + 4 * npiv;
        const int64_t lb = h->level_base[h->kappa], le = h->level_base[h->kappa + 1];
        k_grad_near<<<gridn((le - lb) * 32, 32 * GW), 32 * GW, 0, s>>>(h->kp, (int)d, lb, le, h->cbeg, h->cend,
                                                                       h->nb_off, h->nb_idx, h->xs, N, xt, xt + N, gs,
                                                                       dh);
        NNCA_LAUNCH_CHECK();
        if (h->n_m2l_tgt > 0 && npiv > 0) {
            k_grad_il<<<gridn(h->n_m2l_tgt * 32, 32 * GW), 32 * GW, 0, s>>>(h->kp, (int)d, h->m2l_tgt, h->n_m2l_tgt,
                                                                            h->il_off, h->il_idx, h->piv_off,
                                                                            h->piv_row, h->pv64, npiv, w, w + npiv, gs,
                                                                            dh);
            NNCA_LAUNCH_CHECK();
        }
        if (nbc > 0) {
            BasisArgs A{};
            A.kp = h->kp;
            A.d = (int)d;
            A.N = N;
            A.npiv = npiv;
            A.cells = cells;
            A.ncells = nbc;
            A.kappa_first = (int)h->level_base[h->kappa];
            A.cbeg = h->cbeg;
            A.cend = h->cend;
            A.cch_beg = h->cch_beg;
            A.cch_end = h->cch_end;
            A.piv_off = h->piv_off;
            A.piv_row = h->piv_row;
            A.piv_col = h->piv_col;
            A.xs = h->xs;
            A.xt = xt;
            A.w = w;
            A.u = u;
            A.lu_off = lu_off;
            A.lu = lu;
            A.ipiv = ipiv;
            A.sol = sol;
            A.gs = gs;
            A.dh = dh;
            A.status = h->dev_status;
            k_grad_basis<<<(unsigned)std::min<int64_t>(nbc, 152 * 8), GB, 0, s>>>(A);
            NNCA_LAUNCH_CHECK();
        }
    }
    k_grad_out<<<gridn(N * d, 256), 256, 0, s>>>(N, (int)d, h->perm, gs, grad_p);
    NNCA_LAUNCH_CHECK();
    if (grad_h) NNCA_CUDA(cudaMemcpyAsync(grad_h, dh, sizeof(double), cudaMemcpyDeviceToDevice, s));
    // the scratch is freed on return: finish the work that uses it first
    NNCA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace nnca
