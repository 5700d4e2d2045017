// Bottom-up pivot identification and bases on the GPU (Sec. 2.3).
//
// For each level from the leaves up (Sec. 2.3.2, "reverse level-order"):
//  1. candidate sets (Eqs. 15-18, symmetric shortcut of Sec. 5):
//       leaf      t~ = t^B,                      s~ = U_{B' in IL(B)} s^{B'}
//       non-leaf  t~ = U_{children c} t^{c,i},   s~ = U_{B' in IL(B)} U_{B'' in C(B')} t^{B'',i}
//     in ascending cell order, each child's pivots in selection order;
//  2. partially pivoted ACA (Sec. 2.2.1, Eqs. 3-4) on A_{t~ s~} with the
//     kernel evaluated on the fly: one CTA per cell, FP64, the ACA arithmetic
//     written as the same sequence of IEEE operations as its definition (every
//     multiply-add fused, every dot product and norm reduced in the canonical
//     order: element j into partial j mod 256 in ascending j, then the
//     partials folded p[t] += p[t + o] for o = 128 ... 1), so the pivots are
//     reproducible bit for bit;
//  3. bases (Sec. 2.3.1, Eqs. 11 and 14, Remark of Sec. 2.3.2):
//       X = A_{t~ sigma} (A_{tau sigma})^{-1}   (|t~| x r, row-major)
//     by LU with partial pivoting of (A_{tau sigma})^T and one forward and
//     back substitution per candidate row; rows of X at the pivots are the
//     identity by definition and are set exactly.
// A cell whose far-field candidates cannot determine its basis passes all its
// candidates up with an identity basis: no candidates at all, or an ACA that
// used up every candidate column without meeting its stopping rule while rows
// remain (rank = |s~| < |t~|: the cross says nothing about the rows it did not
// pick, which the ancestors' far field needs). The ACA reading (start row, tie breaks, the cross that meets
// the stopping rule is not kept) is the one stated in the library header.
//
// ACA scratch (the residual row, the crosses u_l and v_l) comes from one pool
// per level; a cell that finds the pool exhausted gives up and is re-run in a
// later launch with an empty pool, so results never depend on the pool size.
#include <algorithm>

#include "nnca_internal.cuh"

namespace nnca {

namespace {

constexpr int ACA_T = 256;      // threads per cell; also the number of canonical partials
constexpr int MAXK = 1024;      // largest rank a cell may reach
constexpr int DOT_CHUNK = 4;    // dot products folded together

unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

// ---- candidate sets -------------------------------------------------------
struct LevelPivots {              // compact pivots of one level (local cell index)
    int64_t *off = nullptr;       // [cnt + 1]
    int32_t *row = nullptr;       // point positions t^{B,i}
    int32_t *col = nullptr;       // point positions s^{B,i} (-1 for pass-through)
    int32_t *rank = nullptr;      // [cnt]
    int32_t *pass = nullptr;      // [cnt]
    int64_t total = 0;
};

__global__ void k_cand_sizes(int64_t b0, int64_t b1, int leaf, const int32_t *cbeg, const int32_t *cend,
                             const int32_t *cch_beg, const int32_t *cch_end, const int32_t *il_off,
                             const int32_t *il_idx, const int32_t *crank, int64_t cb0, int64_t *msz, int64_t *nsz) {
    for (int64_t X = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; X < b1; X += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = 0, n = 0;
        if (leaf) {
            m = cend[X] - cbeg[X];
            for (int32_t q = il_off[X]; q < il_off[X + 1]; ++q) {
                int32_t Y = il_idx[q];
                n += cend[Y] - cbeg[Y];
            }
        } else {
            for (int32_t c = cch_beg[X]; c < cch_end[X]; ++c) m += crank[c - cb0];
            for (int32_t q = il_off[X]; q < il_off[X + 1]; ++q) {
                int32_t Y = il_idx[q];
                for (int32_t Z = cch_beg[Y]; Z < cch_end[Y]; ++Z) n += crank[Z - cb0];
            }
        }
        msz[X - b0] = m;
        nsz[X - b0] = n;
    }
}

// one warp per cell
__global__ void k_cand_gather(int64_t b0, int64_t b1, int leaf, const int32_t *cbeg, const int32_t *cend,
                              const int32_t *cch_beg, const int32_t *cch_end, const int32_t *il_off,
                              const int32_t *il_idx, const int64_t *cpoff, const int32_t *cprow, int64_t cb0,
                              const int64_t *row_off, const int64_t *col_off, int32_t *rows, int32_t *cols) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t X = b0 + warp; X < b1; X += nwarps) {
        const int64_t x = X - b0;
        int32_t *R = rows + row_off[x];
        int32_t *Cc = cols + col_off[x];
        int64_t o = 0;
        if (leaf) {
            for (int32_t t = cbeg[X] + lane; t < cend[X]; t += 32) R[t - cbeg[X]] = t;
            for (int32_t q = il_off[X]; q < il_off[X + 1]; ++q) {
                int32_t Y = il_idx[q];
                int32_t len = cend[Y] - cbeg[Y];
                for (int32_t t = lane; t < len; t += 32) Cc[o + t] = cbeg[Y] + t;
                o += len;
            }
        } else {
            for (int32_t c = cch_beg[X]; c < cch_end[X]; ++c) {
                int64_t p0 = cpoff[c - cb0], len = cpoff[c - cb0 + 1] - p0;
                for (int64_t t = lane; t < len; t += 32) R[o + t] = cprow[p0 + t];
                o += len;
            }
            o = 0;
            for (int32_t q = il_off[X]; q < il_off[X + 1]; ++q) {
                int32_t Y = il_idx[q];
                for (int32_t Z = cch_beg[Y]; Z < cch_end[Y]; ++Z) {
                    int64_t p0 = cpoff[Z - cb0], len = cpoff[Z - cb0 + 1] - p0;
                    for (int64_t t = lane; t < len; t += 32) Cc[o + t] = cprow[p0 + t];
                    o += len;
                }
            }
        }
    }
}

// ---- ACA ------------------------------------------------------------------
struct AcaArgs {
    KParams kp;
    int d;
    int64_t N;
    const double *xs;             // [d][N]
    double eps;
    const int64_t *row_off, *col_off, *cap_off;
    const int32_t *rows, *cols;
    int32_t *rank, *prow, *pcol;  // outputs (local indices; capacity cap per cell)
    int32_t *pass;                // output: 1 for a pass-through cell
    const int32_t *work;
    int nwork;
    int *work_ctr;
    int32_t *retry;
    int *retry_ctr;
    double *pool;
    unsigned long long pool_size;
    unsigned long long *pool_top;
    unsigned *status;
};

__device__ __forceinline__ void load_point(const double *xs, int64_t N, int d, int64_t i, double *p) {
    for (int k = 0; k < d; ++k) p[k] = xs[(int64_t)k * N + i];
}

// (value, index) maximum over the block, ties to the smaller index; idx -1 = none.
__device__ void block_argmax(double &v, int64_t &idx, double *sv, long long *si) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        long long i2 = __shfl_xor_sync(0xffffffffu, (long long)idx, o);
        if (i2 >= 0 && (idx < 0 || v2 > v || (v2 == v && i2 < idx))) { v = v2; idx = i2; }
    }
    if (lane == 0) { sv[wid] = v; si[wid] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0];
        long long bi = si[0];
        for (int w = 1; w < ACA_T / 32; ++w)
            if (si[w] >= 0 && (bi < 0 || sv[w] > bv || (sv[w] == bv && si[w] < bi))) { bv = sv[w]; bi = si[w]; }
        sv[0] = bv;
        si[0] = bi;
    }
    __syncthreads();
    v = sv[0];
    idx = si[0];
    __syncthreads();
}

// Fold the partials part[c][0..ACA_T) of nc dot products in the canonical
// order; results in part[c][0].
__device__ void fold_partials(double (*part)[ACA_T], int nc) {
    for (int o = ACA_T / 2; o >= 1; o >>= 1) {
        __syncthreads();
        if ((int)threadIdx.x < o)
            for (int c = 0; c < nc; ++c) part[c][threadIdx.x] = __dadd_rn(part[c][threadIdx.x], part[c][threadIdx.x + o]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(ACA_T) k_aca(AcaArgs A) {
    __shared__ double sv_l[MAXK];          // u_l(i) for the residual row, then v_l(j*)
    __shared__ double dvv[MAXK];           // v_l . v_k
    __shared__ double duu[MAXK];           // u_l . u_k
    __shared__ long long vtab[MAXK];       // pool offset of cross l: v_l (n) then u_l (m)
    __shared__ double part[DOT_CHUNK][ACA_T];
    __shared__ double redv[ACA_T / 32];
    __shared__ long long redi[ACA_T / 32];
    __shared__ double xi[4], yj[4];
    __shared__ int s_work;
    __shared__ long long s_off;
    __shared__ int s_ctl;                  // 0 continue, 1 done, 2 retry
    const int t = threadIdx.x;
    const int d = A.d;
    const int64_t N = A.N;

    for (;;) {
        if (t == 0) s_work = atomicAdd(A.work_ctr, 1);
        __syncthreads();
        const int w = s_work;
        __syncthreads();
        if (w >= A.nwork) return;
        const int64_t x = A.work[w];
        const int64_t m = A.row_off[x + 1] - A.row_off[x];
        const int64_t n = A.col_off[x + 1] - A.col_off[x];
        const int32_t *rows = A.rows + A.row_off[x];
        const int32_t *cols = A.cols + A.col_off[x];
        int32_t *prow = A.prow + A.cap_off[x];
        int32_t *pcol = A.pcol + A.cap_off[x];
        if (n == 0 || m == 0) {
            // no far-field candidates: pass-through (all rows), or an empty cell
            if (n == 0)
                for (int64_t i = t; i < m; i += ACA_T) { prow[i] = (int32_t)i; pcol[i] = -1; }
            if (t == 0) {
                A.rank[x] = (n == 0) ? (int32_t)m : 0;
                A.pass[x] = (n == 0) ? 1 : 0;
            }
            continue;
        }
        const int64_t kmax = m < n ? m : n;
        // per-cell scratch: residual row r (n), used-column bits, used-row bytes
        const unsigned long long words = (unsigned long long)n + (n + 63) / 64 + (m + 7) / 8;
        if (t == 0) {
            unsigned long long off = atomicAdd(A.pool_top, words);
            s_off = (off + words <= A.pool_size) ? (long long)off : -1;
        }
        __syncthreads();
        if (s_off < 0) {
            if (t == 0) A.retry[atomicAdd(A.retry_ctr, 1)] = (int32_t)x;
            __syncthreads();
            continue;
        }
        double *r = A.pool + s_off;
        unsigned long long *ucol = (unsigned long long *)(r + n);
        unsigned char *urow = (unsigned char *)(ucol + (n + 63) / 64);
        for (int64_t q = t; q < (n + 63) / 64; q += ACA_T) ucol[q] = 0ull;
        for (int64_t q = t; q < m; q += ACA_T) urow[q] = 0;
        int64_t k = 0, i = 0;
        double frob2 = 0.0;
        if (t == 0) s_ctl = 0;
        __syncthreads();

        for (;;) {
            // --- residual of row i: r_j = A(i, j) - sum_l u_l(i) v_l(j) -------------
            for (int64_t l = t; l < k; l += ACA_T) sv_l[l] = A.pool[vtab[l] + n + i];
            if (t < d) xi[t] = A.xs[(int64_t)t * N + rows[i]];
            __syncthreads();
            double best = -1.0, amax = 0.0;
            int64_t bj = -1;
            for (int64_t j0 = t; j0 < n; j0 += 4 * ACA_T) {
                double s[4];
                int64_t jj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    jj[u] = j0 + (int64_t)u * ACA_T;
                    if (jj[u] < n) {
                        double y[4];
                        load_point(A.xs, N, d, cols[jj[u]], y);
                        s[u] = kern_exact(A.kp, xi, y);
                        amax = fmax(amax, fabs(s[u]));
                    } else {
                        s[u] = 0.0;
                    }
                }
                for (int64_t l = 0; l < k; ++l) {
                    const double a = -sv_l[l];
                    const double *Vl = A.pool + vtab[l];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (jj[u] < n) s[u] = __fma_rn(a, Vl[jj[u]], s[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jj[u] < n) {
                        r[jj[u]] = s[u];
                        const bool used = (ucol[jj[u] >> 6] >> (jj[u] & 63)) & 1ull;
                        if (!used && fabs(s[u]) > best) { best = fabs(s[u]); bj = jj[u]; }
                    }
                }
            }
            block_argmax(best, bj, redv, redi);
            int64_t aidx = 0;
            block_argmax(amax, aidx, redv, redi);   // the row's largest entry (a maximum: order-free)
            if (bj < 0 || best <= ldexp(amax, -44)) {
                // the row carries nothing new (its residual is 0 or at round-off level, as
                // for a point at the same location as a pivot): mark it used and take the
                // smallest unused row
                if (t == 0) urow[i] = 1;
                __syncthreads();
                int64_t ni = -1;
                for (int64_t q = t; q < m; q += ACA_T)
                    if (!urow[q]) { ni = q; break; }
                // smallest index: use argmax on -index
                double key = ni >= 0 ? -(double)ni : -1.0;
                int64_t kidx = ni;
                block_argmax(key, kidx, redv, redi);
                if (kidx < 0) break;
                i = kidx;
                continue;
            }
            const int64_t jp = bj;
            if (k >= MAXK) {
                if (t == 0) atomicOr(A.status, DEV_LIST_OVERFLOW);
                break;
            }
            // --- new cross: v = r / r_{j*}, u(i') = A(i', j*) - sum_l v_l(j*) u_l(i') ----
            const unsigned long long need = (unsigned long long)n + (unsigned long long)m;
            if (t == 0) {
                unsigned long long off = atomicAdd(A.pool_top, need);
                s_off = (off + need <= A.pool_size) ? (long long)off : -1;
                if (s_off >= 0) vtab[k] = s_off;
            }
            __syncthreads();
            if (s_off < 0) {
                if (t == 0) { A.retry[atomicAdd(A.retry_ctr, 1)] = (int32_t)x; s_ctl = 2; }
                __syncthreads();
                break;
            }
            double *Vk = A.pool + vtab[k];
            double *Uk = Vk + n;
            const double inv = __ddiv_rn(1.0, r[jp]);
            for (int64_t j = t; j < n; j += ACA_T) Vk[j] = __dmul_rn(r[j], inv);
            // v_l . v_k for l < k, and |v_k|^2 (as l = k), canonical order
            for (int64_t c0 = 0; c0 <= k; c0 += DOT_CHUNK) {
                double acc[DOT_CHUNK];
#pragma unroll
                for (int c = 0; c < DOT_CHUNK; ++c) acc[c] = 0.0;
                for (int64_t j = t; j < n; j += ACA_T) {
                    const double v = Vk[j];
#pragma unroll
                    for (int c = 0; c < DOT_CHUNK; ++c)
                        if (c0 + c <= k) acc[c] = __fma_rn(A.pool[vtab[c0 + c] + j], v, acc[c]);
                }
#pragma unroll
                for (int c = 0; c < DOT_CHUNK; ++c) part[c][t] = acc[c];
                fold_partials(part, DOT_CHUNK);
                if (t == 0)
                    for (int c = 0; c < DOT_CHUNK && c0 + c <= k; ++c) dvv[c0 + c] = part[c][0];
                __syncthreads();
            }
            // u column
            for (int64_t l = t; l < k; l += ACA_T) sv_l[l] = A.pool[vtab[l] + jp];
            if (t < d) yj[t] = A.xs[(int64_t)t * N + cols[jp]];
            __syncthreads();
            for (int64_t q = t; q < m; q += ACA_T) {
                double xq[4];
                load_point(A.xs, N, d, rows[q], xq);
                double s = kern_exact(A.kp, xq, yj);
                for (int64_t l = 0; l < k; ++l) s = __fma_rn(-sv_l[l], A.pool[vtab[l] + n + q], s);
                Uk[q] = s;
            }
            __syncthreads();
            for (int64_t c0 = 0; c0 <= k; c0 += DOT_CHUNK) {
                double acc[DOT_CHUNK];
#pragma unroll
                for (int c = 0; c < DOT_CHUNK; ++c) acc[c] = 0.0;
                for (int64_t q = t; q < m; q += ACA_T) {
                    const double u = Uk[q];
#pragma unroll
                    for (int c = 0; c < DOT_CHUNK; ++c)
                        if (c0 + c <= k) acc[c] = __fma_rn(A.pool[vtab[c0 + c] + n + q], u, acc[c]);
                }
#pragma unroll
                for (int c = 0; c < DOT_CHUNK; ++c) part[c][t] = acc[c];
                fold_partials(part, DOT_CHUNK);
                if (t == 0)
                    for (int c = 0; c < DOT_CHUNK && c0 + c <= k; ++c) duu[c0 + c] = part[c][0];
                __syncthreads();
            }
            // Frobenius norm with the new cross, stopping rule (the cross that meets it is not kept)
            if (t == 0) {
                double cross = 0.0;
                for (int64_t l = 0; l < k; ++l) cross = __fma_rn(duu[l], dvv[l], cross);
                const double nu2 = duu[k], nv2 = dvv[k];
                double f2 = __dadd_rn(frob2, __dmul_rn(2.0, cross));
                f2 = __dadd_rn(f2, __dmul_rn(nu2, nv2));
                const bool stop = __dmul_rn(__dsqrt_rn(nu2), __dsqrt_rn(nv2)) <= __dmul_rn(A.eps, __dsqrt_rn(f2));
                if (stop) {
                    s_ctl = 1;
                } else {
                    urow[i] = 1;
                    ucol[jp >> 6] |= 1ull << (jp & 63);
                    prow[k] = (int32_t)i;
                    pcol[k] = (int32_t)jp;
                    redv[0] = f2;   // broadcast the new norm
                    s_ctl = 0;
                }
            }
            __syncthreads();
            if (s_ctl == 1) break;
            frob2 = redv[0];
            ++k;
            __syncthreads();
            if (k == kmax) break;
            // next row: argmax over unused rows of |u_k|
            double bv = -1.0;
            int64_t bi = -1;
            for (int64_t q = t; q < m; q += ACA_T)
                if (!urow[q] && fabs(Uk[q]) > bv) { bv = fabs(Uk[q]); bi = q; }
            block_argmax(bv, bi, redv, redi);
            if (bi < 0) break;
            i = bi;
        }
        __syncthreads();
        if (s_ctl != 2) {
            // every column used without meeting the stopping rule, rows left: pass-through
            const bool pass = k == n && k < m;
            if (pass)
                for (int64_t q = t; q < m; q += ACA_T) { prow[q] = (int32_t)q; pcol[q] = -1; }
            if (t == 0) {
                A.rank[x] = pass ? (int32_t)m : (int32_t)k;
                A.pass[x] = pass ? 1 : 0;
            }
        }
        __syncthreads();
    }
}

// ---- bases by LU of the pivot block ---------------------------------------
struct TransferArgs {
    KParams kp;
    int d;
    int64_t N;
    const double *xs;
    const int64_t *row_off;      // candidate rows per cell
    const int32_t *rows;
    const int64_t *piv_off;      // compact pivots
    const int32_t *prow_pt, *pcol_pt;   // point positions
    const int32_t *prow_loc;     // local row index of each pivot (into the candidate rows)
    const int32_t *pass;
    const int64_t *op_off;
    double *op;
    const int64_t *lu_off;       // r*r scratch per cell
    double *lu;
    int32_t *ipiv;               // r per cell (at piv_off)
    unsigned *status;
};

__global__ void __launch_bounds__(256) k_transfer(TransferArgs T, int64_t cnt) {
    __shared__ double redv[8];
    __shared__ long long redi[8];
    const int t = threadIdx.x;
    for (int64_t x = blockIdx.x; x < cnt; x += gridDim.x) {
        const int64_t m = T.row_off[x + 1] - T.row_off[x];
        const int64_t r = T.piv_off[x + 1] - T.piv_off[x];
        double *op = T.op + T.op_off[x];
        if (T.pass[x]) {
            for (int64_t e = t; e < m * m; e += 256) op[e] = (e / m == e % m) ? 1.0 : 0.0;
            continue;
        }
        if (r == 0) continue;
        const int32_t *tau = T.prow_pt + T.piv_off[x];
        const int32_t *sig = T.pcol_pt + T.piv_off[x];
        const int32_t *rows = T.rows + T.row_off[x];
        double *L = T.lu + T.lu_off[x];
        int32_t *ip = T.ipiv + T.piv_off[x];
        // L = M^T, M(a, b) = A(tau_a, sigma_b):  L(a, c) = K(x_{tau_c}, x_{sigma_a})
        for (int64_t e = t; e < r * r; e += 256) {
            const int64_t a = e / r, c = e % r;
            double p[4], q[4];
            load_point(T.xs, T.N, T.d, tau[c], p);
            load_point(T.xs, T.N, T.d, sig[a], q);
            L[e] = kern_exact(T.kp, p, q);
        }
        __syncthreads();
        for (int64_t c = 0; c < r; ++c) {
            double bv = -1.0;
            int64_t bi = -1;
            for (int64_t a = c + t; a < r; a += 256)
                if (fabs(L[a * r + c]) > bv) { bv = fabs(L[a * r + c]); bi = a; }
            block_argmax(bv, bi, redv, redi);
            const int64_t p = bi;
            if (t == 0) {
                ip[c] = (int32_t)p;
                if (L[p * r + c] == 0.0) atomicOr(T.status, DEV_ZERO_PIVOT);
            }
            if (p != c)
                for (int64_t j = t; j < r; j += 256) {
                    double tmp = L[c * r + j];
                    L[c * r + j] = L[p * r + j];
                    L[p * r + j] = tmp;
                }
            __syncthreads();
            const double piv = L[c * r + c];
            for (int64_t a = c + 1 + t; a < r; a += 256) L[a * r + c] = __ddiv_rn(L[a * r + c], piv);
            __syncthreads();
            const int64_t w = r - c - 1;
            for (int64_t e = t; e < w * w; e += 256) {
                const int64_t a = c + 1 + e / w, j = c + 1 + e % w;
                L[a * r + j] = __fma_rn(-L[a * r + c], L[c * r + j], L[a * r + j]);
            }
            __syncthreads();
        }
        // one candidate row per thread: b = A(t~_row, sigma), swaps, forward, back
        for (int64_t row = t; row < m; row += 256) {
            double *b = op + row * r;
            double p[4], q[4];
            load_point(T.xs, T.N, T.d, rows[row], p);
            for (int64_t a = 0; a < r; ++a) {
                load_point(T.xs, T.N, T.d, sig[a], q);
                b[a] = kern_exact(T.kp, p, q);
            }
            for (int64_t c = 0; c < r; ++c) {
                const int64_t pc = ip[c];
                if (pc != c) { double tmp = b[c]; b[c] = b[pc]; b[pc] = tmp; }
            }
            for (int64_t a = 0; a < r; ++a) {
                double s = b[a];
                for (int64_t j = 0; j < a; ++j) s = __fma_rn(-L[a * r + j], b[j], s);
                b[a] = s;
            }
            for (int64_t a = r - 1; a >= 0; --a) {
                double s = b[a];
                for (int64_t j = a + 1; j < r; ++j) s = __fma_rn(-L[a * r + j], b[j], s);
                b[a] = __ddiv_rn(s, L[a * r + a]);
            }
        }
        __syncthreads();
        // rows at the pivots are the identity
        const int32_t *loc = T.prow_loc + T.piv_off[x];
        for (int64_t e = t; e < r * r; e += 256) {
            const int64_t a = e / r, c = e % r;
            op[(int64_t)loc[a] * r + c] = (a == c) ? 1.0 : 0.0;
        }
        __syncthreads();
    }
}

// compact per-cell ACA outputs (capacity layout) into the level's pivot CSR
__global__ void k_compact_pivots(int64_t cnt, const int64_t *cap_off, const int32_t *rank, const int64_t *poff,
                                 const int64_t *row_off, const int64_t *col_off, const int32_t *rows,
                                 const int32_t *cols, const int32_t *prow_loc_cap, const int32_t *pcol_loc_cap,
                                 int32_t *prow_pt, int32_t *pcol_pt, int32_t *prow_loc) {
    for (int64_t x = blockIdx.x; x < cnt; x += gridDim.x) {
        const int64_t r = rank[x];
        for (int64_t a = threadIdx.x; a < r; a += blockDim.x) {
            const int32_t li = prow_loc_cap[cap_off[x] + a];
            const int32_t lj = pcol_loc_cap[cap_off[x] + a];
            prow_loc[poff[x] + a] = li;
            prow_pt[poff[x] + a] = rows[row_off[x] + li];
            pcol_pt[poff[x] + a] = lj >= 0 ? cols[col_off[x] + lj] : -1;
        }
    }
}

__global__ void k_ranks_i64(int64_t cnt, const int32_t *rank, int64_t *out) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x)
        out[x] = rank[x];
}

__global__ void k_sizes_prod(int64_t cnt, const int64_t *a_off, const int32_t *rank, const int32_t *pass, int64_t *out,
                             int square) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = a_off[x + 1] - a_off[x];
        const int64_t r = rank[x];
        out[x] = square ? (pass[x] ? 0 : r * r) : m * r;
    }
}

__global__ void k_cap_sizes(int64_t cnt, const int64_t *msz, const int64_t *nsz, int64_t *cap, int32_t *pass) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = msz[x], n = nsz[x];
        (void)n;
        cap[x] = m;        // a pass-through cell keeps all m candidate rows
        pass[x] = 0;       // set by the ACA
    }
}

__global__ void k_iota(int32_t *a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

}  // namespace

// Per-level outputs kept until build_finish assembles the global arrays.
struct LevelOut {
    int64_t cnt = 0;
    int64_t *row_off = nullptr;     // candidate rows (cnt + 1)
    int32_t *rows = nullptr;
    int64_t *piv_off = nullptr;     // (cnt + 1)
    int32_t *prow_pt = nullptr, *pcol_pt = nullptr;
    int32_t *pass = nullptr, *rank = nullptr;
    int64_t *op_off = nullptr;      // (cnt + 1)
    double *op = nullptr;
    int64_t npiv = 0, nrows = 0, nop = 0;
};

void build_pivots_impl(Handle *h, std::vector<LevelOut> &lv, Scratch &keep) {
    cudaStream_t s = h->stream;
    const int kappa = h->kappa;
    lv.assign(kappa + 1, LevelOut{});
    size_t free_b = 0, total_b = 0;
    NNCA_CUDA(cudaMemGetInfo(&free_b, &total_b));
    int dev = 0, nsm = 152;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int aca_per_sm = 1;
    NNCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&aca_per_sm, k_aca, ACA_T, 0));
    aca_per_sm = std::max(1, aca_per_sm);

    for (int l = kappa; l >= h->lmin; --l) {
        Scratch scr;
        const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1], cnt = b1 - b0;
        const int leaf = (l == kappa);
        LevelOut &L = lv[l];
        L.cnt = cnt;
        const LevelOut *C = leaf ? nullptr : &lv[l + 1];
        const int64_t cb0 = leaf ? 0 : h->level_base[l + 1];
        int64_t *msz = scr.get<int64_t>(cnt + 1), *nsz = scr.get<int64_t>(cnt + 1);
        k_cand_sizes<<<grid_for(cnt, 128), 128, 0, s>>>(b0, b1, leaf, h->cbeg, h->cend, h->cch_beg, h->cch_end,
                                                        h->il_off, h->il_idx, leaf ? nullptr : C->rank, cb0, msz, nsz);
        NNCA_LAUNCH_CHECK();
        int64_t *cap = scr.get<int64_t>(cnt + 1);
        L.pass = (int32_t *)keep.get<int32_t>(cnt);
        L.rank = (int32_t *)keep.get<int32_t>(cnt);
        k_cap_sizes<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, msz, nsz, cap, L.pass);
        NNCA_LAUNCH_CHECK();
        L.row_off = keep.get<int64_t>(cnt + 1);
        NNCA_CUDA(cudaMemcpyAsync(L.row_off, msz, cnt * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        NNCA_CUDA(cudaMemsetAsync(L.row_off + cnt, 0, sizeof(int64_t), s));
        L.nrows = scan_total_i64(L.row_off, L.row_off, cnt + 1, s, scr);
        int64_t *col_off = scr.get<int64_t>(cnt + 1);
        NNCA_CUDA(cudaMemcpyAsync(col_off, nsz, cnt * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        NNCA_CUDA(cudaMemsetAsync(col_off + cnt, 0, sizeof(int64_t), s));
        const int64_t ncols = scan_total_i64(col_off, col_off, cnt + 1, s, scr);
        NNCA_CUDA(cudaMemsetAsync(cap + cnt, 0, sizeof(int64_t), s));
        const int64_t ncap = scan_total_i64(cap, cap, cnt + 1, s, scr);
        NNCA_REQUIRE(L.nrows < (1ll << 31) && ncols < (1ll << 40), NNCA_ERR_UNSUPPORTED, "candidate sets too large");
        L.rows = keep.get<int32_t>(L.nrows);
        int32_t *cols = scr.get<int32_t>(ncols);
        k_cand_gather<<<grid_for(cnt * 32, 256), 256, 0, s>>>(b0, b1, leaf, h->cbeg, h->cend, h->cch_beg, h->cch_end,
                                                              h->il_off, h->il_idx, leaf ? nullptr : C->piv_off,
                                                              leaf ? nullptr : C->prow_pt, cb0, L.row_off, col_off,
                                                              L.rows, cols);
        NNCA_LAUNCH_CHECK();

        // ACA with a scratch pool; cells that find the pool exhausted are re-run
        int32_t *prow_cap = scr.get<int32_t>(ncap), *pcol_cap = scr.get<int32_t>(ncap);
        int32_t *work = scr.get<int32_t>(cnt), *retry = scr.get<int32_t>(cnt);
        int *ctrs = scr.get<int>(2);
        unsigned long long *ptop = scr.get<unsigned long long>(1);
        k_iota<<<grid_for(cnt, 256), 256, 0, s>>>(work, cnt);
        NNCA_LAUNCH_CHECK();
        NNCA_CUDA(cudaStreamSynchronize(s));
        NNCA_CUDA(cudaMemGetInfo(&free_b, &total_b));
        // pool: the worst case of every cell if that fits, else most of free memory
        std::vector<int64_t> hm(cnt), hn(cnt);
        NNCA_CUDA(cudaMemcpy(hm.data(), msz, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost));
        NNCA_CUDA(cudaMemcpy(hn.data(), nsz, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost));
        unsigned long long worst = 0, biggest = 0;
        for (int64_t x = 0; x < cnt; ++x) {
            if (hn[x] == 0 || hm[x] == 0) continue;
            unsigned long long kx = (unsigned long long)std::min(hm[x], hn[x]);
            unsigned long long need = hn[x] + (hn[x] + 63) / 64 + (hm[x] + 7) / 8 + (kx + 1) * (hn[x] + hm[x]);
            worst += need;
            biggest = std::max(biggest, need);
        }
        unsigned long long avail = (unsigned long long)(free_b * 0.7) / sizeof(double);
        unsigned long long pool_words = std::max<unsigned long long>(std::min(worst, avail), 1);
        NNCA_REQUIRE(biggest <= pool_words || worst == 0, NNCA_ERR_OOM, "one cell's ACA scratch exceeds device memory");
        double *pool = scr.get<double>(pool_words);
        int nwork = (int)cnt;
        int rounds = 0;
        while (nwork > 0) {
            NNCA_CUDA(cudaMemsetAsync(ctrs, 0, 2 * sizeof(int), s));
            NNCA_CUDA(cudaMemsetAsync(ptop, 0, sizeof(unsigned long long), s));
            AcaArgs A{};
            A.kp = h->kp;
            A.d = h->d;
            A.N = h->n;
            A.xs = h->xs;
            A.eps = h->cfg.aca_tol;
            A.row_off = L.row_off;
            A.col_off = col_off;
            A.cap_off = cap;
            A.rows = L.rows;
            A.cols = cols;
            A.rank = L.rank;
            A.prow = prow_cap;
            A.pcol = pcol_cap;
            A.pass = L.pass;
            A.work = work;
            A.nwork = nwork;
            A.work_ctr = ctrs;
            A.retry = retry;
            A.retry_ctr = ctrs + 1;
            A.pool = pool;
            A.pool_size = pool_words;
            A.pool_top = ptop;
            A.status = h->dev_status;
            const unsigned grid = (unsigned)std::min<int64_t>(nwork, (int64_t)nsm * aca_per_sm);
            k_aca<<<grid, ACA_T, 0, s>>>(A);
            NNCA_LAUNCH_CHECK();
            int nretry = 0;
            NNCA_CUDA(cudaMemcpyAsync(&nretry, ctrs + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
            NNCA_CUDA(cudaStreamSynchronize(s));
            NNCA_REQUIRE(nretry < nwork, NNCA_ERR_OOM, "ACA scratch pool too small for one cell");
            if (nretry > 0) {
                h->stats.aca_retries += nretry;
                NNCA_CUDA(cudaMemcpyAsync(work, retry, nretry * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            }
            nwork = nretry;
            ++rounds;
        }
        const unsigned st = read_status(h);
        NNCA_REQUIRE(!(st & DEV_LIST_OVERFLOW), NNCA_ERR_UNSUPPORTED, "a cell's rank exceeds the supported maximum");

        // compact pivots
        L.piv_off = keep.get<int64_t>(cnt + 1);
        k_ranks_i64<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, L.rank, L.piv_off);
        NNCA_LAUNCH_CHECK();
        NNCA_CUDA(cudaMemsetAsync(L.piv_off + cnt, 0, sizeof(int64_t), s));
        L.npiv = scan_total_i64(L.piv_off, L.piv_off, cnt + 1, s, scr);
        L.prow_pt = keep.get<int32_t>(L.npiv);
        L.pcol_pt = keep.get<int32_t>(L.npiv);
        int32_t *prow_loc = scr.get<int32_t>(L.npiv);
        k_compact_pivots<<<grid_for(cnt * 64, 64), 64, 0, s>>>(cnt, cap, L.rank, L.piv_off, L.row_off, col_off, L.rows,
                                                               cols, prow_cap, pcol_cap, L.prow_pt, L.pcol_pt, prow_loc);
        NNCA_LAUNCH_CHECK();

        // bases
        L.op_off = keep.get<int64_t>(cnt + 1);
        k_sizes_prod<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, L.row_off, L.rank, L.pass, L.op_off, 0);
        NNCA_LAUNCH_CHECK();
        NNCA_CUDA(cudaMemsetAsync(L.op_off + cnt, 0, sizeof(int64_t), s));
        L.nop = scan_total_i64(L.op_off, L.op_off, cnt + 1, s, scr);
        L.op = keep.get<double>(L.nop);
        int64_t *lu_off = scr.get<int64_t>(cnt + 1);
        k_sizes_prod<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, L.row_off, L.rank, L.pass, lu_off, 1);
        NNCA_LAUNCH_CHECK();
        NNCA_CUDA(cudaMemsetAsync(lu_off + cnt, 0, sizeof(int64_t), s));
        const int64_t nlu = scan_total_i64(lu_off, lu_off, cnt + 1, s, scr);
        scr.release(pool);
        TransferArgs T{};
        T.kp = h->kp;
        T.d = h->d;
        T.N = h->n;
        T.xs = h->xs;
        T.row_off = L.row_off;
        T.rows = L.rows;
        T.piv_off = L.piv_off;
        T.prow_pt = L.prow_pt;
        T.pcol_pt = L.pcol_pt;
        T.prow_loc = prow_loc;
        T.pass = L.pass;
        T.op_off = L.op_off;
        T.op = L.op;
        T.lu_off = lu_off;
        T.lu = scr.get<double>(nlu);
        T.ipiv = scr.get<int32_t>(L.npiv);
        T.status = h->dev_status;
        k_transfer<<<(unsigned)std::min<int64_t>(cnt, (int64_t)nsm * 8), 256, 0, s>>>(T, cnt);
        NNCA_LAUNCH_CHECK();
        NNCA_CUDA(cudaStreamSynchronize(s));
    }
}


namespace {

__global__ void k_level_scatter_i32(int64_t cnt, int64_t b0, const int32_t *src, int32_t *dst) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x)
        dst[b0 + x] = src[x];
}

__global__ void k_level_scatter_off(int64_t cnt, int64_t b0, int64_t base, const int64_t *src, int64_t *dst) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x <= cnt; x += (int64_t)gridDim.x * blockDim.x)
        dst[b0 + x] = base + src[x];
}

__global__ void k_fill_off(int64_t from, int64_t to, int64_t v, int64_t *dst) {
    for (int64_t x = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < to; x += (int64_t)gridDim.x * blockDim.x)
        dst[x] = v;
}

__global__ void k_off_to_i32(int64_t n, const int64_t *src, int32_t *dst) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        dst[x] = (int32_t)src[x];
}

// cell centres: corner + (coord + 0.5) * side / 2^l, in FP64 and as a float hi/lo pair
__global__ void k_centres(int64_t b0, int64_t b1, int l, int d, int64_t ncell, const int32_t *ccoord, double c0,
                          double c1, double c2, double c3, double side, double *ccen, float *chi, float *clo) {
    const double corner[4] = {c0, c1, c2, c3};
    const double w = ldexp(side, -l);
    for (int64_t c = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < b1; c += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < d; ++k) {
            const double v = corner[k] + ((double)ccoord[(int64_t)k * ncell + c] + 0.5) * w;
            const float hi = (float)v;
            ccen[(int64_t)k * ncell + c] = v;
            chi[(int64_t)k * ncell + c] = hi;
            clo[(int64_t)k * ncell + c] = (float)(v - (double)hi);
        }
}

// pivot coordinates (FP64) and relative to their cell's centre (FP32)
__global__ void k_pivot_coords(int64_t b0, int64_t b1, int d, int64_t N, int64_t ncell, int64_t npiv,
                               const int32_t *piv_off, const int32_t *piv_row, const double *xs, const double *ccen,
                               double *pv64, float *pv32) {
    for (int64_t c = b0 + blockIdx.x; c < b1; c += gridDim.x)
        for (int64_t p = piv_off[c] + threadIdx.x; p < piv_off[c + 1]; p += blockDim.x)
            for (int k = 0; k < d; ++k) {
                const double v = xs[(int64_t)k * N + piv_row[p]];
                pv64[(int64_t)k * npiv + p] = v;
                pv32[(int64_t)k * npiv + p] = (float)(v - ccen[(int64_t)k * ncell + c]);
            }
}

// leaf of every point, and coordinates relative to the leaf centre (FP32)
__global__ void k_leaf_coords(int64_t b0, int64_t b1, int d, int64_t N, int64_t ncell, const int32_t *cbeg,
                              const int32_t *cend, const double *xs, const double *ccen, int32_t *leaf_of, float *xs32) {
    for (int64_t c = b0 + blockIdx.x; c < b1; c += gridDim.x)
        for (int64_t i = cbeg[c] + threadIdx.x; i < cend[c]; i += blockDim.x) {
            leaf_of[i] = (int32_t)c;
            for (int k = 0; k < d; ++k)
                xs32[(int64_t)k * N + i] = (float)(xs[(int64_t)k * N + i] - ccen[(int64_t)k * ncell + c]);
        }
}

// packed data of the FP32 product
__global__ void k_pack_cells(int64_t nc, int d, const int32_t *piv_off, const double *ccen, int2 *prange, float4 *chi,
                             float4 *clo) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        prange[c] = make_int2(piv_off[c], piv_off[c + 1] - piv_off[c]);
        float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < d && k < 3; ++k) {
            const double v = ccen[(int64_t)k * nc + c];
            h[k] = (float)v;
            l[k] = (float)(v - (double)h[k]);
        }
        chi[c] = make_float4(h[0], h[1], h[2], 0.f);
        clo[c] = make_float4(l[0], l[1], l[2], 0.f);
    }
}

__global__ void k_pack_points(int64_t n, int64_t npiv, int d, const double *xs, const float *pv32, float4 *xh,
                              float4 *xl, float4 *pv4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n || i < npiv; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) {
            float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
            for (int k = 0; k < d && k < 3; ++k) {
                const double v = xs[(int64_t)k * n + i];
                h[k] = (float)v;
                l[k] = (float)(v - (double)h[k]);
            }
            xh[i] = make_float4(h[0], h[1], h[2], 0.f);
            xl[i] = make_float4(l[0], l[1], l[2], 0.f);
        }
        if (i < npiv) {
            float p[3] = {0.f, 0.f, 0.f};
            for (int k = 0; k < d && k < 3; ++k) p[k] = pv32[(int64_t)k * npiv + i];
            pv4[i] = make_float4(p[0], p[1], p[2], 0.f);
        }
    }
}

// Sources of every cell for the FP32 M2L, in pairs [x0 x1 y0 y1][z0 z1 w0 w1]
// relative to the centre of the cell's PARENT (so that sibling cells share a
// frame and consecutive siblings can be evaluated as one segment; the FP64
// difference rounded once); padding sources far away; weights 0 (each product
// writes its own). One warp per cell; the root has no sources in the M2L.
__global__ void k_pack_sources(int64_t nc, int d, int64_t npiv, const int2 *prange, const int32_t *spk_off,
                               const int32_t *cpar, const double *pv64, const double *ccen, float4 *spk) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < nc; c += nw) {
        const int2 pr = prange[c];
        const int64_t q0 = spk_off[c], nq = spk_off[c + 1] - q0;
        const int64_t Q = c > 0 ? cpar[c] : 0;
        for (int64_t q = lane; q < nq; q += 32) {
            float a[2][3];
            for (int e = 0; e < 2; ++e)
                for (int k = 0; k < 3; ++k)
                    a[e][k] = 2 * q + e < pr.y
                                  ? (k < d ? (float)(pv64[(int64_t)k * npiv + pr.x + 2 * q + e] - ccen[(int64_t)k * nc + Q])
                                           : 0.f)
                                  : FAR_AWAY;
            spk[2 * (q0 + q)] = make_float4(a[0][0], a[1][0], a[0][1], a[1][1]);
            spk[2 * (q0 + q) + 1] = make_float4(a[0][2], a[1][2], 0.f, 0.f);
        }
    }
}

// Staging plan of the FP32 M2L for parent P (Table 1): the children Y of N(P)
// with sources, each with the mask of P's children that admit it (the test of
// the list construction, so the mask bit of child X is set exactly when Y is
// in IL(X)), cut greedily into rounds of at most M2L_STAGE_RECS records and
// M2L_STAGE_CAP padded sources. Consecutive siblings (one parent Q, adjacent
// cell ids, so adjacent packed sources) with the same mask share one record
// and the shift c_Q - c_P. PASS 0 counts the records, PASS 1 writes them.
// cap: padded sources per round. sym: only neighbours Q > P (admissibility and
// the neighbour relation are symmetric, so every admissible pair of cells
// under two different parents appears in exactly one plan; siblings are never
// admissible, so Q = P adds nothing).
template <int PASS>
__global__ void k_m2l_plan(int64_t np, const int32_t *parents, int d, int num, int den, const int32_t *ccoord,
                           int64_t ncell, const int32_t *cch_beg, const int32_t *cch_end, const int32_t *nb_off,
                           const int32_t *nb_idx, const int2 *prange, const int32_t *spk_off, const double *ccen,
                           int cap, int sym, const int64_t *rec_off, int64_t *rec_cnt, int4 *rec, float4 *rec_sh) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const int P = parents[i];
        const int cb = cch_beg[P], nch = cch_end[P] - cb;
        int4 *out = PASS ? rec + rec_off[i] : nullptr;
        int64_t n = 0, first = 0;
        int used = 0, nr = 0, last_y = -2, last_mask = -1, last_q = -1;
        for (int q = nb_off[P]; q < nb_off[P + 1]; ++q) {
            const int Q = nb_idx[q];
            if (sym && Q <= P) continue;
            for (int y = cch_beg[Q]; y < cch_end[Q]; ++y) {
                const int rank = prange[y].y;
                if (rank == 0) continue;
                int mask = 0;
                for (int c = 0; c < nch; ++c) {
                    int64_t g2 = 0;
                    for (int k = 0; k < d; ++k) {
                        int64_t t = (int64_t)ccoord[(int64_t)k * ncell + y] - ccoord[(int64_t)k * ncell + cb + c];
                        if (t < 0) t = -t;
                        t -= 1;
                        if (t < 0) t = 0;
                        g2 += t * t;
                    }
                    if ((int64_t)d * den <= (int64_t)num * g2) mask |= 1 << c;
                }
                if (!mask) continue;
                const int npad = m2l_padded(rank);
                if (nr > 0 && Q == last_q && y == last_y + 1 && mask == last_mask && used + npad <= cap) {
                    // the next sibling with the same mask extends the last record
                    if (PASS) out[n - 1].z += (npad >> 1) << 11;
                    used += npad;
                    last_y = y;
                    continue;
                }
                if (nr == M2L_STAGE_RECS || used + npad > cap) {
                    if (PASS) out[first].w = nr;
                    first = n;
                    used = 0;
                    nr = 0;
                }
                if (PASS) {
                    out[n] = make_int4(y, spk_off[y], (used >> 1) | ((npad >> 1) << 11) | (mask << 22), 0);
                    // c_Q - c_P for the parent Q of y, the FP64 difference rounded once
                    float sh[3] = {0.f, 0.f, 0.f};
                    for (int k = 0; k < d && k < 3; ++k) sh[k] = (float)(ccen[(int64_t)k * ncell + Q] - ccen[(int64_t)k * ncell + P]);
                    rec_sh[rec_off[i] + n] = make_float4(sh[0], sh[1], sh[2], 0.f);
                }
                used += npad;
                ++nr;
                ++n;
                last_y = y;
                last_mask = mask;
                last_q = Q;
            }
        }
        if (PASS && nr > 0) out[first].w = nr;
        if (!PASS) rec_cnt[i] = n;
    }
}

// Points of every leaf for the FP32 near field, in pairs
// [xh0 xh1 yh0 yh1][zh0 zh1 w0 w1][xl0 xl1 yl0 yl1][zl0 zl1 0 0]; padding points
// far away with weight 0; weights 0 (each product writes its own). One warp per leaf.
__global__ void k_pack_near(int64_t l0, int64_t l1, int d, int64_t N, const int32_t *cbeg, const int32_t *cend,
                            const int32_t *ppk_off, const float4 *xh4, const float4 *xl4, const float *xs32, float4 *ppk,
                            float4 *ppl) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = l0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); c < l1; c += nw) {
        const int64_t i0 = cbeg[c], n = cend[c] - i0;
        const int64_t q0 = ppk_off[c], nq = ppk_off[c + 1] - q0;
        for (int64_t q = lane; q < nq; q += 32) {
            const float4 farh = make_float4(FAR_AWAY, FAR_AWAY, FAR_AWAY, 0.f), zero = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 h0 = 2 * q < n ? xh4[i0 + 2 * q] : farh, h1 = 2 * q + 1 < n ? xh4[i0 + 2 * q + 1] : farh;
            const float4 o0 = 2 * q < n ? xl4[i0 + 2 * q] : zero, o1 = 2 * q + 1 < n ? xl4[i0 + 2 * q + 1] : zero;
            float4 *dst = ppk + 4 * (q0 + q);
            dst[0] = make_float4(h0.x, h1.x, h0.y, h1.y);
            dst[1] = make_float4(h0.z, h1.z, 0.f, 0.f);
            dst[2] = make_float4(o0.x, o1.x, o0.y, o1.y);
            dst[3] = make_float4(o0.z, o1.z, 0.f, 0.f);
            // relative to the leaf centre (the FP64 difference rounded once)
            float a[2][3];
            for (int e = 0; e < 2; ++e)
                for (int k = 0; k < 3; ++k)
                    a[e][k] = 2 * q + e < n ? (k < d ? xs32[(int64_t)k * N + i0 + 2 * q + e] : 0.f) : FAR_AWAY;
            float4 *dl = ppl + 2 * (q0 + q);
            dl[0] = make_float4(a[0][0], a[1][0], a[0][1], a[1][1]);
            dl[1] = make_float4(a[0][2], a[1][2], 0.f, 0.f);
        }
    }
}

// Staging plan of the FP32 near field for leaf X: the leaves Y of N(X) (Table 1),
// with flags for X itself and for leaves adjacent to X (integer offset at most 1
// in every coordinate: their points can be arbitrarily close to X's and travel
// as hi/lo pairs, 64 bytes per point pair; the others travel in their leaf's
// frame, 32 bytes), cut greedily into rounds of at most NEAR_RECS cells and
// NEAR_UNITS 16-byte units. PASS 0 counts the records, PASS 1 writes them.
template <int PASS>
__global__ void k_near_plan(int64_t l0, int64_t l1, int d, const int32_t *ccoord, int64_t ncell,
                            const int32_t *nb_off, const int32_t *nb_idx, const int32_t *ppk_off,
                            const int64_t *rec_off, int64_t *rec_cnt, int4 *rec) {
    for (int64_t X = l0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; X < l1; X += (int64_t)gridDim.x * blockDim.x) {
        int4 *out = PASS ? rec + rec_off[X - l0] : nullptr;
        int64_t n = 0, first = 0;
        int used = 0, nr = 0;
        for (int q = nb_off[X]; q < nb_off[X + 1]; ++q) {
            const int Y = nb_idx[q];
            const int np = ppk_off[Y + 1] - ppk_off[Y];
            if (np == 0) continue;
            int adj = 1;
            for (int k = 0; k < d; ++k) {
                const int t = ccoord[(int64_t)k * ncell + X] - ccoord[(int64_t)k * ncell + Y];
                if (t > 1 || t < -1) adj = 0;
            }
            const int units = np * (adj ? 4 : 2);
            if (nr == NEAR_RECS || used + units > NEAR_UNITS) {
                if (PASS) out[first].w = nr;
                first = n;
                used = 0;
                nr = 0;
            }
            if (PASS) out[n] = make_int4(Y, ppk_off[Y], used | (np << 11) | ((Y == X ? 1 : 0) << 22) | (adj << 23), 0);
            used += units;
            ++nr;
            ++n;
        }
        if (PASS && nr > 0) out[first].w = nr;
        if (!PASS) rec_cnt[X - l0] = n;
    }
}

// work counts: m2l pairs per target cell, p2p pairs per leaf
__global__ void k_work_counts(int64_t b0, int64_t b1, int64_t leaf0, const int32_t *il_off, const int32_t *il_idx,
                              const int32_t *nb_off, const int32_t *nb_idx, const int32_t *piv_off,
                              const int32_t *cbeg, const int32_t *cend, int64_t *m2l_w, int64_t *p2p_w,
                              unsigned long long *tot) {
    for (int64_t c = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < b1; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = piv_off[c + 1] - piv_off[c], s = 0;
        for (int32_t q = il_off[c]; q < il_off[c + 1]; ++q) s += piv_off[il_idx[q] + 1] - piv_off[il_idx[q]];
        m2l_w[c] = r * s;
        atomicAdd(&tot[0], (unsigned long long)(r * s));
        if (c >= leaf0) {
            int64_t nb = cend[c] - cbeg[c], t = 0;
            for (int32_t q = nb_off[c]; q < nb_off[c + 1]; ++q) t += cend[nb_idx[q]] - cbeg[nb_idx[q]];
            p2p_w[c - leaf0] = nb * t;
            atomicAdd(&tot[1], (unsigned long long)(nb * t));
        }
    }
}

}  // namespace

void build_pivots(Handle *h) {
    cudaStream_t s = h->stream;
    Scratch keep;
    std::vector<LevelOut> lv;
    build_pivots_impl(h, lv, keep);
    const int kappa = h->kappa;
    const int64_t nc = h->ncell;
    Scratch scr;

    // global CSR of pivots, candidates and operators (levels above lmin hold nothing)
    int64_t *poff = scr.get<int64_t>(nc + 1);
    h->cand_off = dalloc<int64_t>(h, nc + 1);
    h->op_off = dalloc<int64_t>(h, nc + 1);
    h->passthru = dalloc<int32_t>(h, nc);
    NNCA_CUDA(cudaMemsetAsync(h->passthru, 0, nc * sizeof(int32_t), s));
    int64_t npiv = 0, nrows = 0, nop = 0;
    for (int l = 0; l <= kappa; ++l) {
        const int64_t b0 = h->level_base[l], cnt = h->level_base[l + 1] - b0;
        if (l < h->lmin) {
            k_fill_off<<<grid_for(cnt + 1, 256), 256, 0, s>>>(b0, b0 + cnt + 1, npiv, poff);
            k_fill_off<<<grid_for(cnt + 1, 256), 256, 0, s>>>(b0, b0 + cnt + 1, nrows, h->cand_off);
            k_fill_off<<<grid_for(cnt + 1, 256), 256, 0, s>>>(b0, b0 + cnt + 1, nop, h->op_off);
            NNCA_LAUNCH_CHECK();
            continue;
        }
        const LevelOut &L = lv[l];
        k_level_scatter_off<<<grid_for(cnt + 1, 256), 256, 0, s>>>(cnt, b0, npiv, L.piv_off, poff);
        k_level_scatter_off<<<grid_for(cnt + 1, 256), 256, 0, s>>>(cnt, b0, nrows, L.row_off, h->cand_off);
        k_level_scatter_off<<<grid_for(cnt + 1, 256), 256, 0, s>>>(cnt, b0, nop, L.op_off, h->op_off);
        k_level_scatter_i32<<<grid_for(cnt, 256), 256, 0, s>>>(cnt, b0, L.pass, h->passthru);
        NNCA_LAUNCH_CHECK();
        npiv += L.npiv;
        nrows += L.nrows;
        nop += L.nop;
    }
    NNCA_REQUIRE(npiv < (1ll << 31), NNCA_ERR_UNSUPPORTED, "more than 2^31 pivots");
    h->npiv = npiv;
    h->nop = nop;
    h->piv_off = dalloc<int32_t>(h, nc + 1);
    k_off_to_i32<<<grid_for(nc + 1, 256), 256, 0, s>>>(nc + 1, poff, h->piv_off);
    NNCA_LAUNCH_CHECK();
    h->piv_row = dalloc<int32_t>(h, npiv);
    h->piv_col = dalloc<int32_t>(h, npiv);
    h->op = dalloc<double>(h, nop);
    int64_t ep = 0, eo = 0;
    for (int l = h->lmin; l <= kappa; ++l) {
        const LevelOut &L = lv[l];
        if (L.npiv) {
            NNCA_CUDA(cudaMemcpyAsync(h->piv_row + ep, L.prow_pt, L.npiv * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            NNCA_CUDA(cudaMemcpyAsync(h->piv_col + ep, L.pcol_pt, L.npiv * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        }
        if (L.nop) NNCA_CUDA(cudaMemcpyAsync(h->op + eo, L.op, L.nop * sizeof(double), cudaMemcpyDeviceToDevice, s));
        ep += L.npiv;
        eo += L.nop;
    }
    h->h_piv_off.resize(nc + 1);
    NNCA_CUDA(cudaMemcpyAsync(h->h_piv_off.data(), h->piv_off, (nc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaStreamSynchronize(s));
}

void build_finish(Handle *h) {
    cudaStream_t s = h->stream;
    Scratch scr;
    const int d = h->d, kappa = h->kappa;
    const int64_t nc = h->ncell, N = h->n;
    h->ccen = dalloc<double>(h, (size_t)nc * d);
    h->ccen_hi = dalloc<float>(h, (size_t)nc * d);
    h->ccen_lo = dalloc<float>(h, (size_t)nc * d);
    double cr[4] = {0, 0, 0, 0};
    for (int k = 0; k < d; ++k) cr[k] = h->corner[k];
    for (int l = 0; l <= kappa; ++l) {
        const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1];
        k_centres<<<grid_for(b1 - b0, 256), 256, 0, s>>>(b0, b1, l, d, nc, h->ccoord, cr[0], cr[1], cr[2], cr[3], h->side,
                                                         h->ccen, h->ccen_hi, h->ccen_lo);
        NNCA_LAUNCH_CHECK();
    }
    h->pv64 = dalloc<double>(h, (size_t)h->npiv * d);
    h->pv32 = dalloc<float>(h, (size_t)h->npiv * d);
    if (h->npiv) {
        k_pivot_coords<<<(unsigned)std::min<int64_t>(nc, 152 * 64), 64, 0, s>>>(0, nc, d, N, nc, h->npiv, h->piv_off,
                                                                               h->piv_row, h->xs, h->ccen, h->pv64,
                                                                               h->pv32);
        NNCA_LAUNCH_CHECK();
    }
    const int64_t leaf0 = h->level_base[kappa], leaf1 = h->level_base[kappa + 1];
    h->nleaf = leaf1 - leaf0;
    h->leaf_of = dalloc<int32_t>(h, N);
    h->xs32 = dalloc<float>(h, (size_t)N * d);
    k_leaf_coords<<<(unsigned)std::min<int64_t>(h->nleaf, 152 * 64), 64, 0, s>>>(leaf0, leaf1, d, N, nc, h->cbeg,
                                                                                 h->cend, h->xs, h->ccen, h->leaf_of,
                                                                                 h->xs32);
    NNCA_LAUNCH_CHECK();

    // work lists, heaviest first: M2L target cells and leaves for the near field
    int64_t *m2l_w = scr.get<int64_t>(nc), *p2p_w = scr.get<int64_t>(h->nleaf);
    unsigned long long *tot = scr.get<unsigned long long>(2);
    NNCA_CUDA(cudaMemsetAsync(tot, 0, 2 * sizeof(unsigned long long), s));
    k_work_counts<<<grid_for(nc, 128), 128, 0, s>>>(0, nc, leaf0, h->il_off, h->il_idx, h->nb_off, h->nb_idx,
                                                    h->piv_off, h->cbeg, h->cend, m2l_w, p2p_w, tot);
    NNCA_LAUNCH_CHECK();
    std::vector<int64_t> hw(nc), hp(h->nleaf);
    unsigned long long ht[2];
    NNCA_CUDA(cudaMemcpyAsync(hw.data(), m2l_w, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaMemcpyAsync(hp.data(), p2p_w, h->nleaf * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaMemcpyAsync(ht, tot, sizeof(ht), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> tg;
    for (int64_t c = 0; c < nc; ++c)
        if (hw[c] > 0) tg.push_back((int32_t)c);
    std::stable_sort(tg.begin(), tg.end(), [&](int32_t a, int32_t b) { return hw[a] > hw[b]; });
    h->n_m2l_tgt = (int64_t)tg.size();
    h->m2l_tgt = dalloc<int32_t>(h, tg.size());
    if (!tg.empty())
        NNCA_CUDA(cudaMemcpyAsync(h->m2l_tgt, tg.data(), tg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    std::vector<int32_t> lo(h->nleaf);
    for (int64_t c = 0; c < h->nleaf; ++c) lo[c] = (int32_t)(leaf0 + c);
    std::stable_sort(lo.begin(), lo.end(), [&](int32_t a, int32_t b) { return hp[a - leaf0] > hp[b - leaf0]; });
    h->leaf_order = dalloc<int32_t>(h, lo.size());
    NNCA_CUDA(cudaMemcpyAsync(h->leaf_order, lo.data(), lo.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    h->stats.m2l_pairs = (int64_t)ht[0];
    h->stats.p2p_pairs = (int64_t)ht[1];

    // FP32 product: packed arrays and work items. Near field: a leaf's targets
    // form items of 32; the remainder c < 32 gets S = 2^s lanes per target
    // (c * S <= 32, S <= 16), which split its sources. Items are ordered
    // heaviest first.
    h->prange = dalloc<int2>(h, nc);
    h->chi4 = dalloc<float4>(h, nc);
    h->clo4 = dalloc<float4>(h, nc);
    h->xh4 = dalloc<float4>(h, N);
    h->xl4 = dalloc<float4>(h, N);
    h->pv4 = dalloc<float4>(h, h->npiv);
    k_pack_cells<<<grid_for(nc, 256), 256, 0, s>>>(nc, d, h->piv_off, h->ccen, h->prange, h->chi4, h->clo4);
    NNCA_LAUNCH_CHECK();
    k_pack_points<<<grid_for(std::max<int64_t>(N, h->npiv), 256), 256, 0, s>>>(N, h->npiv, d, h->xs, h->pv32, h->xh4,
                                                                                h->xl4, h->pv4);
    NNCA_LAUNCH_CHECK();
    std::vector<int32_t> hpo(h->h_piv_off);
    std::vector<int32_t> hcb(nc), hce(nc);
    NNCA_CUDA(cudaMemcpy(hcb.data(), h->cbeg, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
    NNCA_CUDA(cudaMemcpy(hce.data(), h->cend, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
    auto make_items = [&](const std::vector<int32_t> &cells, const std::vector<int64_t> &count,
                          const std::vector<int64_t> &weight, int2 **dst, int *ndst) {
        std::vector<std::pair<int64_t, int2>> lists[5];
        for (size_t k = 0; k < cells.size(); ++k) {
            const int64_t cnt = count[k];
            NNCA_REQUIRE(cnt < 65536, NNCA_ERR_UNSUPPORTED, "a cell with 65536 or more targets");
            int64_t a0 = 0;
            for (; a0 + 32 <= cnt; a0 += 32) lists[0].push_back({weight[k], make_int2(cells[k], (int)(a0 | (32 << 16)))});
            const int64_t rem = cnt - a0;
            if (rem > 0) {
                int ls = 0;
                while (ls < 4 && rem * (2 << ls) <= 32) ++ls;
                lists[ls].push_back({weight[k] >> ls, make_int2(cells[k], (int)(a0 | (rem << 16)))});
            }
        }
        for (int ls = 0; ls < 5; ++ls) {
            std::stable_sort(lists[ls].begin(), lists[ls].end(),
                             [](const std::pair<int64_t, int2> &x, const std::pair<int64_t, int2> &y) { return x.first > y.first; });
            std::vector<int2> v;
            for (auto &p : lists[ls]) v.push_back(p.second);
            ndst[ls] = (int)v.size();
            dst[ls] = dalloc<int2>(h, v.size());
            if (!v.empty())
                NNCA_CUDA(cudaMemcpy(dst[ls], v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice));
        }
    };
    {
        // FP32 M2L sources, packed per cell
        std::vector<int32_t> hso(nc + 1, 0);
        int64_t npairs = 0;
        h->m2l_fp32_unsupported = nullptr;
        for (int64_t c = 0; c < nc; ++c) {
            if (hpo[c + 1] - hpo[c] > M2L_STAGE_CAP)
                h->m2l_fp32_unsupported = "the FP32 product supports ranks up to 512 (use FP64)";
            npairs += m2l_padded(hpo[c + 1] - hpo[c]) / 2;
            NNCA_REQUIRE(npairs < (1ll << 30), NNCA_ERR_UNSUPPORTED, "too many pivots for the FP32 M2L");
            hso[c + 1] = (int32_t)npairs;
        }
        h->n_spk_pairs = npairs;
        h->spk_off = dalloc<int32_t>(h, nc + 1);
        NNCA_CUDA(cudaMemcpy(h->spk_off, hso.data(), (nc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
        h->spk = dalloc<float4>(h, 2 * (size_t)npairs);
        h->spw = dalloc<float4>(h, (M2L_RHS / 2) * (size_t)npairs);
        NNCA_CUDA(cudaMemsetAsync(h->spw, 0, (M2L_RHS / 2) * (size_t)npairs * sizeof(float4), s));
        k_pack_sources<<<grid_for(nc * 32, 256), 256, 0, s>>>(nc, d, h->npiv, h->prange, h->spk_off, h->cpar, h->pv64,
                                                              h->ccen, h->spk);
        NNCA_LAUNCH_CHECK();

        // M2L items: the targets of one parent's children (their pivots are
        // contiguous) in items of M2L_GROUP_TARGETS and a remainder; one staging
        // plan per parent
        std::vector<int32_t> hchb(nc), hche(nc);
        NNCA_CUDA(cudaMemcpy(hchb.data(), h->cch_beg, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
        NNCA_CUDA(cudaMemcpy(hche.data(), h->cch_end, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
        struct Group { int64_t weight; int parent_slot, t0, nt; };
        const int item_targets = h->cfg.m2l_item_targets > 0 ? h->cfg.m2l_item_targets : M2L_GROUP_TARGETS;
        std::vector<Group> groups;
        std::vector<int32_t> parents;
        const int64_t pl0 = h->lmin >= 1 ? h->level_base[h->lmin - 1] : 0;
        const int64_t pl1 = h->level_base[kappa];
        for (int64_t P = pl0; P < pl1 && h->lmin <= kappa; ++P) {
            const int32_t c0 = hchb[P], c1 = hche[P];
            if (c1 <= c0) continue;
            int64_t work = 0;
            for (int32_t c = c0; c < c1; ++c) work += hw[c];
            const int64_t T = hpo[c1] - hpo[c0];
            if (work == 0 || T == 0) continue;
            if (T >= 65536) {
                h->m2l_fp32_unsupported = "the FP32 product supports up to 65535 pivots per group of siblings (use FP64)";
                continue;
            }
            const int slot = (int)parents.size();
            parents.push_back((int32_t)P);
            for (int64_t t0 = 0; t0 < T; t0 += item_targets) {
                const int64_t t1 = std::min<int64_t>(T, t0 + item_targets);
                groups.push_back({work * (t1 - t0) / T, slot, (int)t0, (int)(t1 - t0)});
            }
        }
        std::stable_sort(groups.begin(), groups.end(), [](const Group &x, const Group &y) { return x.weight > y.weight; });
        const int64_t np = (int64_t)parents.size();
        int32_t *dpar = np > 0 ? scr.get<int32_t>(np) : nullptr;
        if (np > 0) NNCA_CUDA(cudaMemcpy(dpar, parents.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
        // staging plans of all parents (cap sources per round; sym: neighbours Q > P only)
        auto build_plan = [&](int cap, int sym, int4 *&plan, float4 *&plan_sh, int64_t &nplan,
                              std::vector<int64_t> &roff) {
            roff.assign(np + 1, 0);
            nplan = 0;
            int64_t *dcnt = scr.get<int64_t>(np), *doff = scr.get<int64_t>(np);
            k_m2l_plan<0><<<grid_for(np, 128), 128, 0, s>>>(np, dpar, d, h->cfg.eta2_num, h->cfg.eta2_den, h->ccoord, nc,
                                                           h->cch_beg, h->cch_end, h->nb_off, h->nb_idx, h->prange,
                                                           h->spk_off, h->ccen, cap, sym, nullptr, dcnt, nullptr, nullptr);
            NNCA_LAUNCH_CHECK();
            std::vector<int64_t> hcnt(np);
            NNCA_CUDA(cudaMemcpy(hcnt.data(), dcnt, np * sizeof(int64_t), cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < np; ++i) roff[i + 1] = roff[i] + hcnt[i];
            NNCA_REQUIRE(roff[np] < (1ll << 31), NNCA_ERR_UNSUPPORTED, "FP32 M2L plan exceeds 2^31 records");
            nplan = roff[np];
            plan = dalloc<int4>(h, roff[np]);
            plan_sh = dalloc<float4>(h, roff[np]);
            NNCA_CUDA(cudaMemcpy(doff, roff.data(), np * sizeof(int64_t), cudaMemcpyHostToDevice));
            k_m2l_plan<1><<<grid_for(np, 128), 128, 0, s>>>(np, dpar, d, h->cfg.eta2_num, h->cfg.eta2_den, h->ccoord, nc,
                                                           h->cch_beg, h->cch_end, h->nb_off, h->nb_idx, h->prange,
                                                           h->spk_off, h->ccen, cap, sym, doff, nullptr, plan, plan_sh);
            NNCA_LAUNCH_CHECK();
        };
        // Items, heaviest first. An item whose pairs (targets x staged sources)
        // exceed a share of the whole that one block of a full wave would carry
        // (total / (4 * 5 * SMs)) is cut at staging-round boundaries into pieces of
        // about equal work, so that no single block holds the launch's tail.
        int dev = 0, nsm = 152;
        NNCA_CUDA(cudaGetDevice(&dev));
        NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        struct Round { int k, n; int64_t src; };
        struct ItemSet {
            std::vector<int4> items;
            std::vector<int64_t> weight;   // pairs (targets x staged sources) of each item
            std::vector<int> part;
            std::vector<int4> splits;
            int nparts = 0;
        };
        auto make_items = [&](const int4 *plan, int64_t nplan, const std::vector<int64_t> &roff, bool skip_empty,
                              std::vector<int4> &hplan, ItemSet &out) {
            hplan.assign(nplan, make_int4(0, 0, 0, 0));
            if (nplan) NNCA_CUDA(cudaMemcpy(hplan.data(), plan, nplan * sizeof(int4), cudaMemcpyDeviceToHost));
            std::vector<std::vector<Round>> rounds(np);
            for (int64_t i = 0; i < np && nplan; ++i)
                for (int64_t k = roff[i]; k < roff[i + 1];) {
                    const int nrec = hplan[k].w;
                    NNCA_REQUIRE(nrec >= 1 && k + nrec <= roff[i + 1], NNCA_ERR_INTERNAL, "malformed M2L staging plan");
                    int64_t src = 0;
                    for (int e = 0; e < nrec; ++e) src += 2 * ((hplan[k + e].z >> 11) & 0x7ff);
                    rounds[i].push_back({(int)k, nrec, src});
                    k += nrec;
                }
            int64_t total = 0;
            for (auto &g : groups)
                for (auto &r : rounds[g.parent_slot]) total += (int64_t)g.nt * r.src;
            const int64_t wmax = std::max<int64_t>(1, total / ((int64_t)nsm * 5 * 4));
            struct Piece { int64_t weight; int4 item; int part; };
            std::vector<Piece> pieces;
            for (auto &g : groups) {
                const int P = parents[g.parent_slot];
                const auto &R = rounds[g.parent_slot];
                if (skip_empty && R.empty()) continue;
                int64_t wsum = 0;
                for (auto &r : R) wsum += (int64_t)g.nt * r.src;
                const int64_t want = std::min<int64_t>((int64_t)R.size(), std::max<int64_t>(1, (wsum + wmax - 1) / wmax));
                if (want <= 1) {
                    pieces.push_back({wsum, make_int4(P, g.t0 | (g.nt << 16), (int)roff[g.parent_slot],
                                                      (int)(roff[g.parent_slot + 1] - roff[g.parent_slot])), -1});
                    continue;
                }
                const int first = out.nparts;
                int64_t acc = 0, cut = 0;
                size_t r0 = 0;
                for (size_t r = 0; r < R.size(); ++r) {
                    acc += (int64_t)g.nt * R[r].src;
                    const bool last = r + 1 == R.size();
                    if (last || acc * want >= (cut + 1) * wsum) {
                        const int k0 = R[r0].k, k1 = R[r].k + R[r].n;
                        int64_t wp = 0;
                        for (size_t q = r0; q <= r; ++q) wp += (int64_t)g.nt * R[q].src;
                        pieces.push_back({wp, make_int4(P, g.t0 | (g.nt << 16), k0, k1 - k0), out.nparts++});
                        r0 = r + 1;
                        ++cut;
                    }
                }
                out.splits.push_back(make_int4((int)(hpo[hchb[P]] + g.t0), g.nt, first, out.nparts - first));
            }
            std::stable_sort(pieces.begin(), pieces.end(),
                             [](const Piece &x, const Piece &y) { return x.weight > y.weight; });
            for (auto &p : pieces) {
                out.items.push_back(p.item);
                out.weight.push_back(p.weight);
                out.part.push_back(p.part);
            }
        };
        std::vector<int64_t> roff;
        std::vector<int4> hplan;
        ItemSet full;
        h->n_m2l_plan = 0;
        if (np > 0 && !h->m2l_fp32_unsupported) {
            build_plan(M2L_STAGE_CAP, 0, h->m2l_plan, h->m2l_plan_sh, h->n_m2l_plan, roff);
            make_items(h->m2l_plan, h->n_m2l_plan, roff, false, hplan, full);
        }
        h->n_m2l_groups = (int)full.items.size();
        h->h_m2l_weight = full.weight;
        h->m2l_groups = dalloc<int4>(h, full.items.size());
        h->m2l_item_part = dalloc<int>(h, full.part.size());
        h->m2l_next = dalloc<int>(h, 1);
        if (!full.items.empty()) {
            NNCA_CUDA(cudaMemcpy(h->m2l_groups, full.items.data(), full.items.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice));
            NNCA_CUDA(cudaMemcpy(h->m2l_item_part, full.part.data(), full.part.size() * sizeof(int),
                                 cudaMemcpyHostToDevice));
        }
        // tensor-core M2L items: at most 64 targets of one parent's children, each
        // over the parent's whole full-form plan, heaviest first
        if (np > 0 && !h->m2l_fp32_unsupported) {
            std::vector<std::pair<int64_t, int4>> tci;
            for (int64_t i = 0; i < np; ++i) {
                const int P = parents[i];
                const int64_t T = hpo[hche[P]] - hpo[hchb[P]];
                const int64_t k0 = roff[i], nk = roff[i + 1] - roff[i];
                if (nk == 0 || T == 0) continue;
                int64_t src = 0;
                for (int64_t k = k0; k < k0 + nk; ++k) src += 2 * ((hplan[k].z >> 11) & 0x7ff);
                for (int64_t t0 = 0; t0 < T; t0 += 64) {
                    const int nt = (int)std::min<int64_t>(64, T - t0);
                    tci.push_back({(int64_t)nt * src, make_int4(P, (int)t0 | (nt << 16), (int)k0, (int)nk)});
                }
            }
            std::stable_sort(tci.begin(), tci.end(),
                             [](const std::pair<int64_t, int4> &a, const std::pair<int64_t, int4> &b) {
                                 return a.first > b.first;
                             });
            std::vector<int4> tcv(tci.size());
            for (size_t i = 0; i < tci.size(); ++i) tcv[i] = tci[i].second;
            h->n_tc_items = (int)tcv.size();
            h->tc_items = dalloc<int4>(h, tcv.size());
            if (!tcv.empty())
                NNCA_CUDA(cudaMemcpy(h->tc_items, tcv.data(), tcv.size() * sizeof(int4), cudaMemcpyHostToDevice));
        }
        h->n_m2l_split = (int)full.splits.size();
        h->m2l_split = dalloc<int4>(h, full.splits.size());
        h->m2l_parts = dalloc<double>(h, (size_t)std::max(full.nparts, 1) * M2L_GROUP_TARGETS * M2L_RHS);
        if (!full.splits.empty())
            NNCA_CUDA(cudaMemcpy(h->m2l_split, full.splits.data(), full.splits.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice));

        // The symmetric form (one right-hand side): a plan over neighbours Q > P,
        // the column slots of every item in staging order, and per cell the slots
        // of its pivots' column sums, in item order.
        int64_t maxr = 0;
        for (int64_t c = 0; c < nc; ++c) maxr = std::max<int64_t>(maxr, hpo[c + 1] - hpo[c]);
        h->stats.m2l_evals = h->stats.m2l_pairs;
        if (np > 0 && !h->m2l_fp32_unsupported && maxr <= M2L_SYM_CAP && h->cfg.symmetric &&
            h->cfg.m2l_form == NNCA_M2L_AUTO) {
            std::vector<int64_t> sroff;
            std::vector<int4> splan;
            ItemSet sym;
            build_plan(M2L_SYM_CAP, 1, h->sym_plan, h->sym_plan_sh, h->n_sym_plan, sroff);
            make_items(h->sym_plan, h->n_sym_plan, sroff, true, splan, sym);
            {
                // the pair loop's form (see m2l_sym_pairs): unrolled when the staged
                // records hold at least a chunk of source pairs on average
                int64_t pairs = 0;
                for (const int4 &r : splan) pairs += (r.z >> 11) & 0x7ff;
                h->sym_unroll = !splan.empty() && pairs >= (int64_t)M2L_CHUNK_PAIRS * (int64_t)splan.size();
            }
            std::vector<int> icol(sym.items.size());
            std::vector<std::vector<int32_t>> per_cell(nc);
            int64_t ncol = 0;
            for (size_t it = 0; it < sym.items.size(); ++it) {
                const int4 item = sym.items[it];
                icol[it] = (int)ncol;
                for (int64_t k = item.z; k < (int64_t)item.z + item.w;) {
                    const int nrec = splan[k].w;
                    int64_t rsrc = 0;
                    for (int e = 0; e < nrec; ++e) {
                        const int4 r = splan[k + e];
                        const int64_t pairs = (r.z >> 11) & 0x7ff, slot = ncol + 2 * (int64_t)(r.z & 0x7ff);
                        // the record's cells: consecutive siblings with contiguous packed sources
                        int64_t pq = r.y;
                        for (int32_t y = r.x; pq < r.y + pairs; ++y) {
                            NNCA_REQUIRE(y < nc && hso[y] == pq, NNCA_ERR_INTERNAL, "malformed symmetric M2L plan");
                            if (hpo[y + 1] > hpo[y]) per_cell[y].push_back((int32_t)(slot + 2 * (pq - r.y)));
                            pq = hso[y + 1];
                        }
                        rsrc += 2 * pairs;
                    }
                    ncol += rsrc;
                    NNCA_REQUIRE(ncol < (1ll << 31), NNCA_ERR_UNSUPPORTED, "symmetric M2L exceeds 2^31 column slots");
                    k += nrec;
                }
            }
            std::vector<int32_t> eoff(nc + 1, 0), ent;
            std::vector<int2> tasks;
            for (int64_t c = 0; c < nc; ++c) {
                eoff[c + 1] = eoff[c] + (int32_t)per_cell[c].size();
                ent.insert(ent.end(), per_cell[c].begin(), per_cell[c].end());
                if (!per_cell[c].empty())
                    for (int64_t j0 = 0; j0 < hpo[c + 1] - hpo[c]; j0 += 32) tasks.push_back(make_int2((int)c, (int)j0));
            }
            h->n_sym_items = (int)sym.items.size();
            h->sym_items = dalloc<int4>(h, sym.items.size());
            h->sym_item_part = dalloc<int>(h, sym.part.size());
            h->sym_item_col = dalloc<int>(h, icol.size());
            h->n_sym_split = (int)sym.splits.size();
            h->sym_split = dalloc<int4>(h, sym.splits.size());
            h->sym_parts = dalloc<double>(h, (size_t)std::max(sym.nparts, 1) * M2L_GROUP_TARGETS);
            h->n_sym_col = ncol;
            h->sym_col = dalloc<float>(h, (size_t)ncol);
            h->sym_ent_off = dalloc<int32_t>(h, nc + 1);
            h->sym_ent = dalloc<int32_t>(h, ent.size());
            h->n_sym_tasks = (int)tasks.size();
            h->sym_tasks = dalloc<int2>(h, tasks.size());
            if (!sym.items.empty()) {
                NNCA_CUDA(cudaMemcpy(h->sym_items, sym.items.data(), sym.items.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice));
                NNCA_CUDA(cudaMemcpy(h->sym_item_part, sym.part.data(), sym.part.size() * sizeof(int),
                                     cudaMemcpyHostToDevice));
                NNCA_CUDA(cudaMemcpy(h->sym_item_col, icol.data(), icol.size() * sizeof(int), cudaMemcpyHostToDevice));
            }
            if (!sym.splits.empty())
                NNCA_CUDA(cudaMemcpy(h->sym_split, sym.splits.data(), sym.splits.size() * sizeof(int4),
                                     cudaMemcpyHostToDevice));
            NNCA_CUDA(cudaMemcpy(h->sym_ent_off, eoff.data(), (nc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
            if (!ent.empty())
                NNCA_CUDA(cudaMemcpy(h->sym_ent, ent.data(), ent.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            if (!tasks.empty())
                NNCA_CUDA(cudaMemcpy(h->sym_tasks, tasks.data(), tasks.size() * sizeof(int2), cudaMemcpyHostToDevice));
            h->stats.m2l_evals = h->stats.m2l_pairs / 2;
        }
        NNCA_CUDA(cudaStreamSynchronize(s));
    }
    {
        // FP32 near field: packed point pairs, per-leaf plans and items
        std::vector<int32_t> hpk(nc + 1, 0);
        int64_t npairs = 0, maxpts = 0;
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t pts = c >= leaf0 ? hce[c] - hcb[c] : 0;
            maxpts = std::max(maxpts, pts);
            npairs += m2l_padded((int)pts) / 2;
            NNCA_REQUIRE(npairs < (1ll << 30), NNCA_ERR_UNSUPPORTED, "too many points for the FP32 near field");
            hpk[c + 1] = (int32_t)npairs;
        }
        h->near_packed = maxpts <= 2 * NEAR_CAP;
        if (h->near_packed) {
            h->ppk_off = dalloc<int32_t>(h, nc + 1);
            NNCA_CUDA(cudaMemcpy(h->ppk_off, hpk.data(), (nc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
            h->ppk = dalloc<float4>(h, 4 * (size_t)npairs);
            h->ppl = dalloc<float4>(h, 2 * (size_t)npairs);
            k_pack_near<<<grid_for(h->nleaf * 32, 256), 256, 0, s>>>(leaf0, leaf1, d, N, h->cbeg, h->cend, h->ppk_off,
                                                                     h->xh4, h->xl4, h->xs32, h->ppk, h->ppl);
            NNCA_LAUNCH_CHECK();
            int64_t *dcnt = scr.get<int64_t>(h->nleaf), *doff = scr.get<int64_t>(h->nleaf);
            k_near_plan<0><<<grid_for(h->nleaf, 128), 128, 0, s>>>(leaf0, leaf1, d, h->ccoord, nc, h->nb_off, h->nb_idx,
                                                                   h->ppk_off, nullptr, dcnt, nullptr);
            NNCA_LAUNCH_CHECK();
            std::vector<int64_t> hcnt(h->nleaf), roff(h->nleaf + 1, 0);
            NNCA_CUDA(cudaMemcpy(hcnt.data(), dcnt, h->nleaf * sizeof(int64_t), cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < h->nleaf; ++i) roff[i + 1] = roff[i] + hcnt[i];
            NNCA_REQUIRE(roff[h->nleaf] < (1ll << 31), NNCA_ERR_UNSUPPORTED, "near-field plan exceeds 2^31 records");
            h->n_near_plan = roff[h->nleaf];
            h->near_plan = dalloc<int4>(h, roff[h->nleaf]);
            NNCA_CUDA(cudaMemcpy(doff, roff.data(), h->nleaf * sizeof(int64_t), cudaMemcpyHostToDevice));
            k_near_plan<1><<<grid_for(h->nleaf, 128), 128, 0, s>>>(leaf0, leaf1, d, h->ccoord, nc, h->nb_off, h->nb_idx,
                                                                   h->ppk_off, doff, nullptr, h->near_plan);
            NNCA_LAUNCH_CHECK();
            // items: one leaf each; its c targets sit TPL (2 or 3) per lane on
            // L = ceil(c / TPL) lanes, and G = floor(32 / L) groups of L lanes
            // split the source pairs. The TPL with the fewer idle target slots per
            // unit of work (c G / (32 TPL) largest) wins. Heaviest first.
            std::vector<std::pair<int64_t, int4>> its[2];
            for (int64_t c = leaf0; c < leaf1; ++c) {
                const int64_t nb = hce[c] - hcb[c];
                if (nb == 0) continue;
                int best = 0, bestG = 1;
                double beste = -1.0;
                for (int t = 2; t <= 3; ++t) {
                    const int64_t L = (nb + t - 1) / t;
                    if (L > 32) continue;
                    const int G = (int)std::min<int64_t>(16, 32 / L);
                    const double e = (double)nb * G / (32.0 * t);
                    if (e > beste + 1e-12) {
                        beste = e;
                        best = t;
                        bestG = G;
                    }
                }
                NNCA_REQUIRE(best >= 2, NNCA_ERR_INTERNAL, "near-field layout: a leaf larger than 96 points");
                its[best - 2].push_back({hp[c - leaf0],
                                         make_int4((int)c, (int)(nb << 16) | (bestG << 24), (int)roff[c - leaf0],
                                                   (int)(roff[c - leaf0 + 1] - roff[c - leaf0]))});
            }
            for (int t = 0; t < 2; ++t) {
                std::stable_sort(its[t].begin(), its[t].end(),
                                 [](const std::pair<int64_t, int4> &x, const std::pair<int64_t, int4> &y) { return x.first > y.first; });
                std::vector<int4> v;
                for (auto &p : its[t]) v.push_back(p.second);
                h->n_near_items[t] = (int)v.size();
                h->near_items[t] = dalloc<int4>(h, v.size());
                if (!v.empty())
                    NNCA_CUDA(cudaMemcpy(h->near_items[t], v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice));
            }
            h->near_next = dalloc<int>(h, 3);
            // items of the four-right-hand-side kernel: two targets per lane, leaves of
            // more than 64 points in pieces of at most 64 targets
            std::vector<std::pair<int64_t, int4>> it4;
            for (int64_t c = leaf0; c < leaf1; ++c) {
                const int64_t nb = hce[c] - hcb[c];
                const int64_t pieces = (nb + 63) / 64;
                for (int64_t p = 0; p < pieces; ++p) {
                    const int64_t f = nb * p / pieces, cnt = nb * (p + 1) / pieces - f;
                    const int64_t L = (cnt + 1) / 2;
                    const int G = (int)std::min<int64_t>(16, 32 / L);
                    it4.push_back({hp[c - leaf0] * cnt / std::max<int64_t>(nb, 1),
                                   make_int4((int)c, (int)f | (int)(cnt << 16) | (G << 24), (int)roff[c - leaf0],
                                             (int)(roff[c - leaf0 + 1] - roff[c - leaf0]))});
                }
            }
            std::stable_sort(it4.begin(), it4.end(),
                             [](const std::pair<int64_t, int4> &x, const std::pair<int64_t, int4> &y) { return x.first > y.first; });
            std::vector<int4> v4;
            for (auto &p : it4) v4.push_back(p.second);
            h->n_near_items4 = (int)v4.size();
            h->near_items4 = dalloc<int4>(h, v4.size());
            if (!v4.empty())
                NNCA_CUDA(cudaMemcpy(h->near_items4, v4.data(), v4.size() * sizeof(int4), cudaMemcpyHostToDevice));
            h->near_pairs = npairs;
            h->pw4 = dalloc<float4>(h, 2 * (size_t)npairs);
            NNCA_CUDA(cudaMemsetAsync(h->pw4, 0, 2 * (size_t)npairs * sizeof(float4), s));
        }
    }
    {
        std::vector<int32_t> cells;
        std::vector<int64_t> count, weight;
        for (int64_t c = leaf0; c < leaf1; ++c) {
            const int64_t nb = hce[c] - hcb[c];
            cells.push_back((int32_t)c);
            count.push_back(nb);
            weight.push_back(hp[c - leaf0] / std::max<int64_t>(nb, 1));
        }
        make_items(cells, count, weight, h->leaf_items, h->n_leaf_items);
    }
    NNCA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace nnca
