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
#include <map>
#include <mutex>

#include "nnca_internal.cuh"

namespace nnca {

namespace {

#include "dev_common.cuh"

unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ---- permutation into tree order --------------------------------------------
// FP32 product (one right-hand side): also the float weight slot of each point
// in the packed near-field pairs, hi/lo and local (leaf Y, local index j: pair
// ppk_off[Y] + j/2)
template <class TI>
__global__ void k_perm_in(const TI *x, int64_t ld, int64_t N, int64_t nrhs, const int32_t *perm, double *xt,
                          float *xt32, float *ppk_w, float *ppl_w, const int32_t *leaf_of, const int32_t *cbeg,
                          const int32_t *ppk_off) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / N, i = e - r * N;
        const double v = (double)x[r * ld + perm[i]];
        xt[e] = v;
        if (xt32) xt32[e] = (float)v;
        if (ppk_w) {
            const int Y = leaf_of[i];
            const int64_t j = i - cbeg[Y];
            ppk_w[((int64_t)ppk_off[Y] + (j >> 1)) * 16 + 6 + (j & 1)] = (float)v;
            ppl_w[((int64_t)ppk_off[Y] + (j >> 1)) * 8 + 6 + (j & 1)] = (float)v;
        }
    }
}

// FP32 product, one right-hand side of a multi-RHS pass: its float weights into
// the packed near-field pairs (hi/lo and local)
__global__ void k_near_weights(int64_t N, const double *xt, float *ppk_w, float *ppl_w, const int32_t *leaf_of,
                               const int32_t *cbeg, const int32_t *ppk_off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int Y = leaf_of[i];
        const int64_t j = i - cbeg[Y];
        const float v = (float)xt[i];
        ppk_w[((int64_t)ppk_off[Y] + (j >> 1)) * 16 + 6 + (j & 1)] = v;
        ppl_w[((int64_t)ppk_off[Y] + (j >> 1)) * 8 + 6 + (j & 1)] = v;
    }
}

// ---- P2M / M2M and L2L: batched small products with the FP64 operators --------
// The operators of the upper levels are few and large (hundreds of rows), those
// of the leaves many and small, so a team of TW warps serves one cell and each
// lane keeps UP_BATCH independent loads of the operator in flight. The vector
// the operator multiplies is staged in shared memory in chunks of UP_CHUNK.
constexpr int UP_THREADS = 256;
constexpr int UP_BATCH = 8;
constexpr int UP_CHUNK = 512;

// w_B[b] = sum_a op_B[a][b] src[a]; op_B is m x r, row-major (m: the points of a
// leaf or the pivots of the children). The TW warps of a team split the rows;
// the lanes take 32 columns at a time (coalesced row segments). blockIdx.y
// selects a group of NR right-hand sides (xt and w advanced by NR rows per
// group), so one launch serves every group of a pass.
template <class T, int NR, int TW>
__global__ void __launch_bounds__(UP_THREADS) k_upward(int64_t b0, int64_t b1, int leaf, const int32_t *cbeg,
                                                      const int32_t *cend, const int32_t *cch_beg,
                                                      const int32_t *cch_end, const int32_t *piv_off,
                                                      const int64_t *op_off, const T *op, const T *xt, int64_t N,
                                                      T *w, int64_t npiv, float *spk_w, const int32_t *spk_off,
                                                      float *spw = nullptr, int64_t spw_stride = 0) {
    xt += (int64_t)blockIdx.y * NR * N;
    w += (int64_t)blockIdx.y * NR * npiv;
    if (spw) spw += (int64_t)blockIdx.y * spw_stride;
    constexpr int TEAMS = UP_THREADS / (32 * TW);
    // rows staged per chunk (halved for eight right-hand sides: the static shared memory)
    constexpr int CH = (TW == 1 ? 64 : UP_CHUNK) / (NR > 4 ? 2 : 1);
    __shared__ T sv[TEAMS][NR][CH];
    __shared__ T part[TEAMS][TW][NR][32];
    const int lane = threadIdx.x & 31, tw = (threadIdx.x >> 5) % TW, team = threadIdx.x / (32 * TW);
    const int tt = threadIdx.x % (32 * TW);   // thread within the team
    for (int64_t B0 = b0 + (int64_t)blockIdx.x * TEAMS; B0 < b1; B0 += (int64_t)gridDim.x * TEAMS) {
        const int64_t B = B0 + team;
        const bool live = B < b1;
        int64_t r = 0, m = 0, ld = 0;
        const T *src = nullptr;
        if (live) {
            r = piv_off[B + 1] - piv_off[B];
            if (leaf) {
                src = xt + cbeg[B];
                m = cend[B] - cbeg[B];
                ld = N;
            } else {
                src = w + piv_off[cch_beg[B]];
                m = piv_off[cch_end[B]] - piv_off[cch_beg[B]];
                ld = npiv;
            }
        }
        const T *A = live ? op + op_off[B] : nullptr;
        // the loops below run the same trip counts in every team of the block
        int64_t mmax = m, rmax = r;
        if (TEAMS > 1) {
            __shared__ int64_t mr[TEAMS][2];
            if (tt == 0) {
                mr[team][0] = m;
                mr[team][1] = r;
            }
            __syncthreads();
            for (int k = 0; k < TEAMS; ++k) {
                mmax = mr[k][0] > mmax ? mr[k][0] : mmax;
                rmax = mr[k][1] > rmax ? mr[k][1] : rmax;
            }
        }
        for (int64_t c0 = 0; c0 < rmax; c0 += 32) {
            const int64_t b = c0 + lane;
            T acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = 0;
            for (int64_t a0 = 0; a0 < mmax; a0 += CH) {
                const int64_t na = m - a0 < CH ? (m - a0 > 0 ? m - a0 : 0) : CH;
                __syncthreads();
                for (int64_t i = tt; i < na; i += 32 * TW)
#pragma unroll
                    for (int q = 0; q < NR; ++q) sv[team][q][i] = src[q * ld + a0 + i];
                __syncthreads();
                if (b < r) {
                    int64_t a = tw;
                    for (; a + (UP_BATCH - 1) * TW < na; a += UP_BATCH * TW) {
                        T c[UP_BATCH];
#pragma unroll
                        for (int k = 0; k < UP_BATCH; ++k) c[k] = A[(a0 + a + k * TW) * r + b];
#pragma unroll
                        for (int k = 0; k < UP_BATCH; ++k)
#pragma unroll
                            for (int q = 0; q < NR; ++q) acc[q] += c[k] * sv[team][q][a + k * TW];
                    }
                    for (; a < na; a += TW)
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] += A[(a0 + a) * r + b] * sv[team][q][a];
                }
            }
            if (TW > 1) {
#pragma unroll
                for (int q = 0; q < NR; ++q) part[team][tw][q][lane] = acc[q];
                __syncthreads();
                if (tw == 0)
#pragma unroll
                    for (int q = 0; q < NR; ++q) {
                        T v = part[team][0][q][lane];
#pragma unroll
                        for (int k = 1; k < TW; ++k) v += part[team][k][q][lane];
                        acc[q] = v;
                    }
            }
            if (tw == 0 && b < r) {
#pragma unroll
                for (int q = 0; q < NR; ++q) w[q * npiv + piv_off[B] + b] = acc[q];
                // FP32 product: the weight slot of pivot b in the packed sources
                if (spk_w) spk_w[((int64_t)spk_off[B] + (b >> 1)) * 8 + 6 + (b & 1)] = (float)acc[0];
                // FP32 product with M2L_RHS right-hand sides: the packed weights of each
                if (spw && NR == M2L_RHS)
#pragma unroll
                    for (int q = 0; q < NR; ++q)
                        spw[((int64_t)spk_off[B] + (b >> 1)) * (2 * M2L_RHS) + (q >> 1) * 4 + (q & 1) * 2 + (b & 1)] =
                            (float)acc[q];
            }
        }
    }
}

// u_{B_c} += C_{B_c P} u_P for the children of P: P's transfer C is m x r_P,
// row-major, one row per pivot of P's children (in order). A block serves one
// parent; its warps take rows 32 at a time, one row per lane, with u_P staged
// in shared memory and UP_BATCH operator loads in flight per lane. blockIdx.y
// selects a group of NR right-hand sides (u advanced by NR rows per group).
template <class T, int NR>
__global__ void __launch_bounds__(UP_THREADS) k_l2l(int64_t p0, int64_t p1, const int32_t *cch_beg,
                                                   const int32_t *cch_end, const int32_t *piv_off,
                                                   const int64_t *op_off, const T *op, T *u, int64_t npiv) {
    u += (int64_t)blockIdx.y * NR * npiv;
    __shared__ T su[NR][UP_CHUNK];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    constexpr int W = UP_THREADS / 32;
    for (int64_t P = p0 + blockIdx.x; P < p1; P += gridDim.x) {
        const int64_t rP = piv_off[P + 1] - piv_off[P];
        if (rP == 0 || cch_end[P] <= cch_beg[P]) continue;
        const int64_t row0 = piv_off[cch_beg[P]], m = piv_off[cch_end[P]] - row0;
        const T *C = op + op_off[P];
        for (int64_t a0 = 0; a0 < m; a0 += 32 * W) {
            const int64_t a = a0 + wl * 32 + lane;
            T acc[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = 0;
            for (int64_t c0 = 0; c0 < rP; c0 += UP_CHUNK) {
                const int64_t nc = rP - c0 < UP_CHUNK ? rP - c0 : UP_CHUNK;
                __syncthreads();
                for (int64_t i = threadIdx.x; i < nc; i += UP_THREADS)
#pragma unroll
                    for (int q = 0; q < NR; ++q) su[q][i] = u[q * npiv + piv_off[P] + c0 + i];
                __syncthreads();
                if (a < m) {
                    const T *row = C + a * rP + c0;
                    int64_t b = 0;
                    for (; b + UP_BATCH <= nc; b += UP_BATCH) {
                        T c[UP_BATCH];
#pragma unroll
                        for (int k = 0; k < UP_BATCH; ++k) c[k] = row[b + k];
#pragma unroll
                        for (int k = 0; k < UP_BATCH; ++k)
#pragma unroll
                            for (int q = 0; q < NR; ++q) acc[q] += c[k] * su[q][b + k];
                    }
                    for (; b < nc; ++b)
#pragma unroll
                        for (int q = 0; q < NR; ++q) acc[q] += row[b] * su[q][b];
                }
            }
            if (a < m)
#pragma unroll
                for (int q = 0; q < NR; ++q) u[q * npiv + row0 + a] += acc[q];
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

// FP64 M2L of one right-hand side in the symmetric form: f(|p - q|) = f(|q - p|)
// and Y in IL(X) exactly when X in IL(Y), so the warp of cell X evaluates only
// the entries Y > X of its list, each value feeding the row sum of its target
// a in X and the column sum of its source b in Y. The column sums of entry
// (X, Y) go to slots slot[e] .. + r_Y (accumulated over X's chunks of 32
// targets in order); k_m2l_f64_gather then adds, for every cell, the slots of
// its entries Y < X in list order. Every order is fixed.
template <int KIND>
__global__ void __launch_bounds__(32 * MV_WARPS) k_m2l_f64_sym(KParams kp, int d, const int32_t *tgt, int64_t ntgt,
                                                              const int32_t *il_off, const int32_t *il_idx,
                                                              const int64_t *slot_of, const int32_t *piv_off,
                                                              const double *pv, int64_t npiv, const double *w,
                                                              double *u, double *slots) {
    __shared__ double sx[MV_WARPS][4][32];
    __shared__ double sw[MV_WARPS][32];
    __shared__ double cs[MV_WARPS][32][33];   // column values of a chunk: [source][target lane], padded
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
            const double wa = act ? w[p0 + a] : 0.0;
            double acc = 0.0;
            for (int32_t e = il_off[X]; e < il_off[X + 1]; ++e) {
                const int64_t Y = il_idx[e];
                if (Y <= X) continue;
                double *col = slots + slot_of[e];
                const int64_t q0 = piv_off[Y], rY = piv_off[Y + 1] - q0;
                for (int64_t b0 = 0; b0 < rY; b0 += 32) {
                    const int64_t nb = min((int64_t)32, rY - b0);
                    __syncwarp();
                    if (lane < nb) {
                        for (int k = 0; k < d; ++k) sx[wl][k][lane] = pv[(int64_t)k * npiv + q0 + b0 + lane];
                        sw[wl][lane] = w[q0 + b0 + lane];
                    }
                    __syncwarp();
                    for (int j = 0; j < nb; ++j) {
                        double r2 = 0.0;
                        for (int k = 0; k < d; ++k) {
                            const double t2 = sx[wl][k][j] - xa[k];
                            r2 = fma(t2, t2, r2);
                        }
                        const double f = act ? KF<KIND>::f64(kp, r2) : 0.0;
                        acc = fma(f, sw[wl][j], acc);
                        cs[wl][j][lane] = f * wa;
                    }
                    __syncwarp();
                    // lane j sums column j over the targets, in lane order
                    if (lane < nb) {
                        double c = 0.0;
                        for (int l = 0; l < 32; ++l) c += cs[wl][lane][l];
                        col[b0 + lane] = a0 == 0 ? kp.s * c : col[b0 + lane] + kp.s * c;
                    }
                }
            }
            if (act) u[p0 + a] = kp.s * acc;
        }
    }
}

// u(X) += the column slots of X's entries Y < X, in list order
__global__ void __launch_bounds__(32 * MV_WARPS) k_m2l_f64_gather(const int32_t *tgt, int64_t ntgt,
                                                                 const int32_t *il_off, const int32_t *il_idx,
                                                                 const int64_t *slot_of, const int32_t *piv_off,
                                                                 const double *slots, double *u) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < ntgt; t += nw) {
        const int64_t X = tgt[t];
        const int64_t p0 = piv_off[X], rX = piv_off[X + 1] - p0;
        for (int64_t a = lane; a < rX; a += 32) {
            double v = u[p0 + a];
            for (int32_t e = il_off[X]; e < il_off[X + 1]; ++e)
                if (il_idx[e] < X) v += slots[slot_of[e] + a];
            u[p0 + a] = v;
        }
    }
}

// ---- FP32 source streaming -----------------------------------------------------
// A warp streams the sources of its source cells through a 64-entry ring in
// shared memory and evaluates them in full chunks of 32. Sources are stored in
// pairs, [x0 x1 y0 y1][z0 z1 w0 w1] (and, for the near field, the low parts
// [xl0 xl1 yl0 yl1][zl0 zl1 - -]), so one 128-bit load yields two packed
// operands. Only the last chunk of a work item is padded, with far-away
// sources of weight 0. A work item is up to 32/S targets of one cell; each
// target is served by S lanes that split every chunk's sources between them.
constexpr int RING = 64;

// LO: near field, low parts of the coordinates in slots 2-3.
template <bool LO> struct Ring2 {
    float4 v[RING / 2][LO ? 4 : 2];
};

template <int KIND, int LOGS, bool SAFE, bool LO>
struct Stream2 {
    static constexpr int S = 1 << LOGS;
    Ring2<LO> &R;
    int fill = 0, done = 0;
    const int s;             // this lane's slice
    f2 tx, ty, tz, txl, tyl, tzl;
    float sum = 0.f, comp = 0.f;
    __device__ Stream2(Ring2<LO> &r, int slice, float x, float y, float z, float xl, float yl, float zl)
        : R(r), s(slice) {
        tx = f2_pack(x, x);
        ty = f2_pack(y, y);
        tz = f2_pack(z, z);
        txl = f2_pack(xl, xl);
        tyl = f2_pack(yl, yl);
        tzl = f2_pack(zl, zl);
    }
    __device__ __forceinline__ void eval_chunk(const KParams &kp) {
        const int base = (done & (RING - 1)) >> 1;   // source-pair index of the chunk
        // four short partial chains per lane (two sources each), combined pairwise
        f2 acc[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
        for (int i = 0; i < 16 / S; ++i) {
            const int q = base + s + S * i;
            const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(&R.v[q][0]);
            const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(&R.v[q][1]);
            f2 dx = f2_sub(A.x, tx), dy = f2_sub(A.y, ty), dz = f2_sub(B.x, tz);
            if (LO) {
                const ulonglong2 C = *reinterpret_cast<const ulonglong2 *>(&R.v[q][2]);
                const ulonglong2 D = *reinterpret_cast<const ulonglong2 *>(&R.v[q][3]);
                dx = f2_add(dx, f2_sub(C.x, txl));
                dy = f2_add(dy, f2_sub(C.y, tyl));
                dz = f2_add(dz, f2_sub(D.x, tzl));
            }
            f2 r2 = f2_mul(dx, dx);
            r2 = f2_fma(dy, dy, r2);
            r2 = f2_fma(dz, dz, r2);
            acc[i & 3] = f2_fma(KF2<KIND, SAFE>::eval(kp, r2), B.y, acc[i & 3]);
        }
        const float2 a = f2_unpack(f2_add(f2_add(acc[0], acc[1]), f2_add(acc[2], acc[3])));
        two_sum_add(sum, comp, a.x + a.y);
    }
    __device__ __forceinline__ void flush_full(const KParams &kp) {
        if (fill - done >= 32) {
            __syncwarp();
            eval_chunk(kp);
            done += 32;
        }
    }
    // lanes < n push one source each
    __device__ __forceinline__ void push(const KParams &kp, int lane, int n, float x, float y, float z, float w,
                                         float xl, float yl, float zl) {
        __syncwarp();
        if (lane < n) {
            const int pos = (fill + lane) & (RING - 1);
            float *p = reinterpret_cast<float *>(&R.v[pos >> 1][0]);
            const int h = pos & 1;
            p[0 + h] = x;
            p[2 + h] = y;
            p[4 + h] = z;
            p[6 + h] = w;
            if (LO) {
                p[8 + h] = xl;
                p[10 + h] = yl;
                p[12 + h] = zl;
            }
        }
        fill += n;
        flush_full(kp);
    }
    __device__ __forceinline__ void finish(const KParams &kp, int lane) {
        if (fill > done) push(kp, lane, done + 32 - fill, FAR_AWAY, FAR_AWAY, FAR_AWAY, 0.f, 0.f, 0.f, 0.f);
    }
    // combine the S slices of every target (lanes t*S .. t*S + S-1) into the first
    __device__ __forceinline__ double result() {
#pragma unroll
        for (int o = 1; o < S; o <<= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, sum, o);
            const float co = __shfl_xor_sync(0xffffffffu, comp, o);
            two_sum_add(sum, comp, so);
            comp += co;
        }
        return (double)sum + (double)comp;
    }
};

// Work item: cell, first target, number of targets, log2 of the slices.
__device__ __forceinline__ void unpack_item(int2 it, int &cell, int &a0, int &c) {
    cell = it.x;
    a0 = it.y & 0xffff;
    c = (it.y >> 16) & 0xff;
}

// ---- M2L, FP32 evaluation: one thread block per group of sibling cells -------------
// The children X of one parent P draw their interaction lists from one set, the
// children of N(P): IL(X) is its part that is admissible for X (Table 1). A
// block serves up to M2L_GROUP_TARGETS targets (pivots) of P's children, two
// consecutive ones per lane, in their order (so a warp spans few children).
// P's staging plan lists the children of N(P) with sources, each with the
// mask of P's children that admit it, in rounds. One warp stages a round with
// one bulk asynchronous copy (TMA) per cell from the packed sources into one of
// M2L_STAGE_BUFS shared buffers, tracked by a "full" mbarrier, up to
// M2L_STAGE_AHEAD rounds ahead of its own evaluation; the warps release each
// buffer on its "empty" mbarrier, so a warp may run a round behind the others
// without stalling the staging. Blocks take items from a counter, heaviest
// first. A
// warp evaluates a staged cell when it is admissible for the child of one of
// its targets: the targets move into the cell's frame (c_Y - c_P subtracted
// once per cell), sum the cell in float, and add the partial into their
// compensated total only when their own child admits the cell. Every wait is
// bounded (about 2^31 clocks); one that runs out sets DEV_WAIT_TIMEOUT.
constexpr int M2L_GROUP_THREADS = 32 * M2L_GROUP_WARPS;

constexpr int M2L_STAGE_AHEAD = M2L_STAGE_BUFS - 2;
constexpr int M2L_FOLD = 8;   // couples of source pairs per lane between folds into the compensated totals
static_assert(2 * M2L_FOLD == M2L_CHUNK_PAIRS, "chunk size shared with the build's choice of the pair loop");
constexpr int M2L_FOLD_RHS = 4;   // the same with M2L_RHS right-hand sides (one chain per right-hand side)

struct M2lGroupSmem {
    float4 src[M2L_STAGE_BUFS][M2L_STAGE_CAP / 2][2];   // staged source pairs
    int hdr[M2L_STAGE_BUFS][M2L_STAGE_RECS];            // staging slot | pairs << 11 | child mask << 22
    float4 sh[M2L_STAGE_BUFS][M2L_STAGE_RECS];          // centre of the cell minus centre of P
    int nrec[M2L_STAGE_BUFS];
    unsigned long long full[M2L_STAGE_BUFS], empty[M2L_STAGE_BUFS];   // mbarriers
    int2 ch_range[8];                                   // pivots of P's children
    int item;
    int abort;
};

// The symmetric form's block state: staging buffers like k_m2l_group's (rounds of
// at most M2L_SYM_CAP sources), each warp's column sums of the rounds in flight,
// a per-warp transpose buffer for the column sums of one chunk, and per buffer
// the round's first column slot, its sources and the warps done with it. Three
// staging buffers (one round of lookahead): with 1/r the block then fits five
// times per SM (96 registers per thread, 43 KB of shared memory).
constexpr int M2L_SYM_BUFS = 3;
constexpr int M2L_SYM_AHEAD = M2L_SYM_BUFS - 2;
constexpr int M2L_SYM_COLBUF = 32 * (2 * M2L_FOLD + 1);   // float2 per warp: L rows of 2 M2L_FOLD G + 1, L G <= 32
struct M2lSymSmem {
    float4 src[M2L_SYM_BUFS][M2L_SYM_CAP / 2][2];
    float colw[M2L_SYM_BUFS][M2L_GROUP_WARPS][M2L_SYM_CAP];
    float2 colbuf[M2L_GROUP_WARPS][M2L_SYM_COLBUF];
    int hdr[M2L_SYM_BUFS][M2L_STAGE_RECS];
    float4 sh[M2L_SYM_BUFS][M2L_STAGE_RECS];
    int nrec[M2L_SYM_BUFS], rbase[M2L_SYM_BUFS], rsrc[M2L_SYM_BUFS], cnt[M2L_SYM_BUFS];
    unsigned long long full[M2L_SYM_BUFS], empty[M2L_SYM_BUFS];
    int2 ch_range[8];
    int item;
    int abort;
    int scol;   // next column slot of the item (staging warp)
};

// what the staging warp records about a round besides its records
__device__ __forceinline__ void stage_note(M2lGroupSmem &, int, unsigned) {}
__device__ __forceinline__ void stage_note(M2lSymSmem &S, int b, unsigned bytes) {
    if ((threadIdx.x & 31) == 0) {
        const int n = (int)(bytes / 16u);   // 32 bytes per source pair
        S.rbase[b] = S.scol;
        S.rsrc[b] = n;
        S.scol += n;
    }
}

// The staging warp's copy of the plan records of the next round: lane i holds
// record k + i and its shift (loaded one round ahead, so staging never waits).
struct StageCursor {
    int k = 0;
    int4 r = make_int4(0, 0, 0, 0);
    float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
};

__device__ __forceinline__ void stage_load(StageCursor &c, const int4 *plan, const float4 *plan_sh, int k, int kend) {
    const int lane = threadIdx.x & 31;
    c.k = k;
    if (k + lane < kend) {
        c.r = plan[k + lane];
        c.sh = plan_sh[k + lane];
    }
}

// Staging warp: stage the round held by the cursor into buffer b, for its use-th use
// (after the warps have released its previous use), then load the records of
// the round after it. Returns the first record of that round, or kend after a
// timed-out wait or a malformed record.
template <class SM>
__device__ __forceinline__ int m2l_stage(SM &S, int b, unsigned use, StageCursor &cur, const int4 *plan,
                                         const float4 *plan_sh, int kend, const float4 *spk, unsigned *status) {
    const int lane = threadIdx.x & 31;
    if (use > 0 && !mbar_wait_warp(&S.empty[b], (use - 1) & 1)) {
        if (lane == 0) {
            atomicOr(status, DEV_WAIT_TIMEOUT);
            *(volatile int *)&S.abort = 1;
        }
        return kend;
    }
    const int k = cur.k;
    const int nrec = __shfl_sync(0xffffffffu, cur.r.w, 0);   // cells in this round (first record)
    if (nrec < 1 || nrec > M2L_STAGE_RECS || k + nrec > kend) {   // a malformed plan: stop, never spin
        if (lane == 0) {
            atomicOr(status, DEV_BAD_INDEX);
            *(volatile int *)&S.abort = 1;
        }
        return kend;
    }
    unsigned bytes = 0;
    const int4 r = cur.r;
    // every record's slots must lie inside the buffer
    constexpr int cap_pairs = (int)(sizeof(S.src[0]) / (2 * sizeof(float4)));
    const bool bad = lane < nrec && (r.z & 0x7ff) + ((r.z >> 11) & 0x7ff) > cap_pairs;
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) {
            atomicOr(status, DEV_BAD_INDEX);
            *(volatile int *)&S.abort = 1;
        }
        return kend;
    }
    if (lane < nrec) {
        S.hdr[b][lane] = r.z;
        S.sh[b][lane] = cur.sh;
        bytes = (unsigned)((r.z >> 11) & 0x7ff) * 32u;
    }
    const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
    if (lane == 0) S.nrec[b] = nrec;
    stage_note(S, b, total);
    __syncwarp();
    if (lane == 0) mbar_arrive_tx(&S.full[b], total + g_stage_extra_tx);
    __syncwarp();
    if (lane < nrec) bulk_g2s(&S.src[b][r.z & 0x7ff][0], spk + 2 * (int64_t)r.y, bytes, &S.full[b]);
    if (k + nrec < kend) stage_load(cur, plan, plan_sh, k + nrec, kend);
    return k + nrec;
}

// one target of a lane: child slot (31: none), pivot, coordinates in P's frame, sum
struct GroupTarget {
    int c = 31;
    int g = 0;
    f2 tx = 0ull, ty = 0ull, tz = 0ull;   // (t, t) packed
    float sum = 0.f, comp = 0.f;
};

__device__ __forceinline__ void group_target(GroupTarget &T, bool act, int g, int nch, int cb, const int2 *ch_range,
                                             const float4 *pv4, const float4 *chi, const float4 *clo, float4 hP,
                                             float4 lP) {
    T.g = g;
    if (!act) return;
    int c = 0;
    for (int k = 1; k < nch; ++k)
        if (ch_range[k].x <= g) c = k;
    T.c = c;
    const int X = cb + c;
    const float4 v = pv4[g], hX = chi[X], lX = clo[X];
    const float tx = v.x + ((hX.x - hP.x) + (lX.x - lP.x));
    const float ty = v.y + ((hX.y - hP.y) + (lX.y - lP.y));
    const float tz = v.z + ((hX.z - hP.z) + (lX.z - lP.z));
    T.tx = f2_pack(tx, tx);
    T.ty = f2_pack(ty, ty);
    T.tz = f2_pack(tz, tz);
}

// acc += f(|s - t|^2) w over a packed pair of sources
template <int KIND>
__device__ __forceinline__ f2 group_pair(const KParams &kp, const ulonglong2 &A, const ulonglong2 &B, f2 tx, f2 ty,
                                         f2 tz, f2 acc) {
    const f2 dx = f2_sub(A.x, tx), dy = f2_sub(A.y, ty), dz = f2_sub(B.x, tz);
    f2 r2 = f2_mul(dx, dx);
    r2 = f2_fma(dy, dy, r2);
    r2 = f2_fma(dz, dz, r2);
    return f2_fma(KF2<KIND, false>::eval(kp, r2), B.y, acc);
}

// f(|s - t|^2) of a packed pair of sources
template <int KIND>
__device__ __forceinline__ f2 group_f(const KParams &kp, const ulonglong2 &A, const ulonglong2 &B, f2 tx, f2 ty, f2 tz) {
    const f2 dx = f2_sub(A.x, tx), dy = f2_sub(A.y, ty), dz = f2_sub(B.x, tz);
    f2 r2 = f2_mul(dx, dx);
    r2 = f2_fma(dy, dy, r2);
    r2 = f2_fma(dz, dz, r2);
    return KF2<KIND, false>::eval(kp, r2);
}

// the source pairs q0, q0 + step, ... below q1 (pairs taken two at a time) of one
// staged cell against two targets. FULL (the whole warp, step 2): at most
// M2L_FOLD steps (one chunk), unrolled with a warp-uniform exit; otherwise
// (lane groups splitting the pairs of small items) a counted loop, which keeps
// the kernel's code small for the clustered inputs that run that path most.
template <int KIND, int FULL>
__device__ __forceinline__ void m2l_cell_pairs(const KParams &kp, const float4 (*src)[2], int q0, int q1, f2 xa, f2 ya,
                                               f2 za, f2 xb, f2 yb, f2 zb, f2 &a0, f2 &a1, f2 &b0, f2 &b1,
                                               int step = 2) {
    auto body = [&](int q) {
        const ulonglong2 A0 = *reinterpret_cast<const ulonglong2 *>(&src[q][0]);
        const ulonglong2 B0 = *reinterpret_cast<const ulonglong2 *>(&src[q][1]);
        const ulonglong2 A1 = *reinterpret_cast<const ulonglong2 *>(&src[q + 1][0]);
        const ulonglong2 B1 = *reinterpret_cast<const ulonglong2 *>(&src[q + 1][1]);
        a0 = group_pair<KIND>(kp, A0, B0, xa, ya, za, a0);
        b0 = group_pair<KIND>(kp, A0, B0, xb, yb, zb, b0);
        a1 = group_pair<KIND>(kp, A1, B1, xa, ya, za, a1);
        b1 = group_pair<KIND>(kp, A1, B1, xb, yb, zb, b1);
    };
    if (FULL) {
#pragma unroll
        for (int k = 0; k < M2L_FOLD; ++k) {
            if (q0 + 2 * k >= q1) break;
            body(q0 + 2 * k);
        }
    } else {
        for (int q = q0; q < q1; q += step) body(q);
    }
}

template <int KIND>
__global__ void __launch_bounds__(M2L_GROUP_THREADS) k_m2l_group(KParams kp, const int4 *items, int nitems,
                                                               int *next_item, const int4 *plan,
                                                               const float4 *plan_sh,
                                                               const int32_t *cch_beg, const int32_t *cch_end,
                                                               const int2 *prange, const float4 *pv4,
                                                               const float4 *chi, const float4 *clo,
                                                               const float4 *spk, const int *item_part,
                                                               double *parts, double *u, unsigned *status) {
    __shared__ __align__(128) M2lGroupSmem S;
    const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < M2L_STAGE_BUFS; ++b) {
            mbar_init(&S.full[b], 1);
            mbar_init(&S.empty[b], M2L_GROUP_WARPS);
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the staging warp: spread over the blocks so that every SM sub-partition
    // (which holds the same warp index of each block) carries a share of it
    const int pw = blockIdx.x % M2L_GROUP_WARPS;
    unsigned R = 0, Rp = 0;   // rounds consumed by every warp; rounds staged (warp pw)
    for (;;) {
        __syncthreads();   // the previous item is done with the shared state
        if (tid == 0) S.item = atomicAdd(next_item, 1);
        __syncthreads();
        const int it = S.item;
        if (it >= nitems || *(volatile int *)&S.abort) break;
        const int4 item = items[it];
        const int part = item_part[it];   // -1: the whole item, else the slot of its partial sums
        const int P = item.x, t0 = item.y & 0xffff, nt = item.y >> 16, kend = item.z + item.w;
        const int cb = cch_beg[P], nch = cch_end[P] - cb;
        if (tid < nch) S.ch_range[tid] = prange[cb + tid];
        __syncthreads();
        const float4 hP = chi[P], lP = clo[P];
        int kprod = item.z, kcons = item.z;
        StageCursor cur;
        if (wl == pw && kprod < kend) stage_load(cur, plan, plan_sh, kprod, kend);
        // this warp's cw targets sit two per lane on L lanes; in a partial warp
        // G groups of L lanes split the source pairs of every cell
        const int wt = m2l_warp_targets(nt);
        const int wj0 = t0 + wl * wt, jend = t0 + nt;
        const int cw = min(wt, max(0, jend - wj0));
        const int L = cw > 0 ? (cw + 1) / 2 : 32;
        const int G = min(16, 32 / L);
        const int grp = lane / L, ti = lane - grp * L;
        const bool live = grp < G;
        const int j = wj0 + 2 * ti;
        const int g = S.ch_range[0].x + j;
        GroupTarget Ta, Tb;
        group_target(Ta, live && j < jend, g, nch, cb, S.ch_range, pv4, chi, clo, hP, lP);
        group_target(Tb, live && j + 1 < jend, g + 1, nch, cb, S.ch_range, pv4, chi, clo, hP, lP);
        const unsigned omask =
            __reduce_or_sync(0xffffffffu, (Ta.c < 31 ? 1u << Ta.c : 0u) | (Tb.c < 31 ? 1u << Tb.c : 0u));
        while (kcons < kend) {
            // warp pw keeps up to M2L_STAGE_AHEAD rounds staged beyond the one it evaluates
            if (wl == pw)
                while (kprod < kend && Rp <= R + M2L_STAGE_AHEAD) {
                    kprod = m2l_stage(S, Rp % M2L_STAGE_BUFS, Rp / M2L_STAGE_BUFS, cur, plan, plan_sh, kend, spk,
                                      status);
                    ++Rp;
                }
            const int b = R % M2L_STAGE_BUFS;
            if (!mbar_wait_warp(&S.full[b], (R / M2L_STAGE_BUFS) & 1)) {
                if (lane == 0) {
                    atomicOr(status, DEV_WAIT_TIMEOUT);
                    *(volatile int *)&S.abort = 1;
                }
                break;
            }
            const int nrec = S.nrec[b];
            if (nrec < 1) break;   // unreachable with a well-formed plan
            if (omask && live) {
                for (int i = 0; i < nrec; ++i) {
                    const int hw = S.hdr[b][i];
                    const unsigned m = ((unsigned)hw >> 22) & omask;
                    if (!m) continue;
                    const float4 sh = S.sh[b][i];
                    const f2 SX = f2_pack(sh.x, sh.x), SY = f2_pack(sh.y, sh.y), SZ = f2_pack(sh.z, sh.z);
                    const f2 xa = f2_sub(Ta.tx, SX), ya = f2_sub(Ta.ty, SY), za = f2_sub(Ta.tz, SZ);
                    const f2 xb = f2_sub(Tb.tx, SX), yb = f2_sub(Tb.ty, SY), zb = f2_sub(Tb.tz, SZ);
                    const int q0 = hw & 0x7ff, q1 = q0 + ((hw >> 11) & 0x7ff);
                    const bool ona = (m >> Ta.c) & 1u, onb = (m >> Tb.c) & 1u;
                    // a segment (one cell or a run of siblings) in chunks of M2L_FOLD couples of
                    // pairs per lane, each chunk folded into the compensated totals
                    const int span = 2 * M2L_FOLD * G;
                    for (int c0 = q0; c0 < q1; c0 += span) {
                        const int c1 = min(q1, c0 + span);
                        f2 a0 = 0ull, a1 = 0ull, b0 = 0ull, b1 = 0ull;
                        if (G == 1)
                            m2l_cell_pairs<KIND, 1>(kp, S.src[b], c0, c1, xa, ya, za, xb, yb, zb, a0, a1, b0, b1);
                        else
                            m2l_cell_pairs<KIND, 0>(kp, S.src[b], c0 + 2 * grp, c1, xa, ya, za, xb, yb, zb, a0, a1, b0,
                                                    b1, 2 * G);
                        const float2 pa = f2_unpack(f2_add(a0, a1)), pb = f2_unpack(f2_add(b0, b1));
                        if (ona) two_sum_add(Ta.sum, Ta.comp, pa.x + pa.y);
                        if (onb) two_sum_add(Tb.sum, Tb.comp, pb.x + pb.y);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[b]);
            ++R;
            kcons += nrec;
        }
        // the groups summed disjoint source pairs of the same targets: combine into group 0
        for (int gg = 1; gg < G; ++gg) {
            const int srcl = min(ti + gg * L, 31);
            const float sa = __shfl_sync(0xffffffffu, Ta.sum, srcl), ca = __shfl_sync(0xffffffffu, Ta.comp, srcl);
            const float sb = __shfl_sync(0xffffffffu, Tb.sum, srcl), cb2 = __shfl_sync(0xffffffffu, Tb.comp, srcl);
            if (grp == 0) {
                two_sum_add(Ta.sum, Ta.comp, sa);
                Ta.comp += ca;
                two_sum_add(Tb.sum, Tb.comp, sb);
                Tb.comp += cb2;
            }
        }
        if (grp == 0) {
            const int gb = S.ch_range[0].x + t0;   // pivot of the item's first target
            double *dst = part < 0 ? u + gb : parts + (int64_t)part * M2L_GROUP_TARGETS;
            if (Ta.c < 31) dst[Ta.g - gb] = kp.s * ((double)Ta.sum + (double)Ta.comp);
            if (Tb.c < 31) dst[Tb.g - gb] = kp.s * ((double)Tb.sum + (double)Tb.comp);
        }
    }
    // after a timed-out wait: let copies still in flight land before the block exits
    if (wl == pw && lane == 0)
        for (unsigned r = R; r < Rp; ++r) mbar_wait(&S.full[r % M2L_STAGE_BUFS], (r / M2L_STAGE_BUFS) & 1);
}

// ---- leaves: L2P (FP64) + P2P (FP32 evaluation on hi/lo coordinates) ------------
// Points carry absolute coordinates as float pairs x = hi + lo. The difference
// (hi_j - hi_i) + (lo_j - lo_i) is exact in its first term whenever the points
// are close (Sterbenz), so close pairs keep full relative accuracy.
template <int KIND, int LOGS, class TO>
__global__ void __launch_bounds__(32 * MV_WARPS) k_leaf_f32(KParams kp, const int2 *items, int nitems,
                                                           const int32_t *cbeg, const int32_t *cend,
                                                           const int32_t *nb_off, const int32_t *nb_idx,
                                                           const int32_t *piv_off, const int64_t *op_off,
                                                           const double *op, const double *u, const float4 *xh4,
                                                           const float4 *xl4, const float *xt32, const double *xt64,
                                                           const int32_t *perm, TO *y) {
    __shared__ __align__(16) Ring2<true> ring[MV_WARPS];
    constexpr int S = 1 << LOGS;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int t = lane >> LOGS, s = lane & (S - 1);
    const float k0 = KF<KIND>::f32(kp, 0.f);
    for (int it = blockIdx.x * MV_WARPS + wl; it < nitems; it += gridDim.x * MV_WARPS) {
        int B, a0, c;
        unpack_item(items[it], B, a0, c);
        const int i0 = cbeg[B], nB = cend[B] - i0;
        const bool act = t < c;
        const int i = i0 + a0 + t;
        const float4 th = act ? xh4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 tl = act ? xl4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        // neighbours other than B: distinct cells, r > 0 for every pair
        Stream2<KIND, LOGS, false, true> st(ring[wl], s, th.x, th.y, th.z, tl.x, tl.y, tl.z);
        const int e1 = nb_off[B + 1];
        for (int e0 = nb_off[B]; e0 < e1; e0 += 32) {
            const int ne = min(32, e1 - e0);
            int jb = 0, jn = 0;   // point range of the neighbour (empty for B itself)
            if (lane < ne) {
                const int Y = nb_idx[e0 + lane];
                if (Y != B) {
                    jb = cbeg[Y];
                    jn = cend[Y] - jb;
                }
            }
            int k = 0, b0 = 0;
            int j0 = __shfl_sync(0xffffffffu, jb, 0), nY = __shfl_sync(0xffffffffu, jn, 0);
            int n = min(32, nY);
            float4 vh = make_float4(0.f, 0.f, 0.f, 0.f), vl = vh;
            float wv = 0.f;
            if (lane < n) {
                vh = xh4[j0 + lane];
                vl = xl4[j0 + lane];
                wv = xt32[j0 + lane];
            }
            while (k < ne) {
                int k2 = k, b2 = b0 + 32;
                int j2 = j0, n2tot = nY;
                if (b2 >= nY) {
                    k2 = k + 1;
                    b2 = 0;
                    j2 = k2 < ne ? __shfl_sync(0xffffffffu, jb, k2) : 0;
                    n2tot = k2 < ne ? __shfl_sync(0xffffffffu, jn, k2) : 0;
                }
                const int n2 = k2 < ne ? max(0, min(32, n2tot - b2)) : 0;
                float4 vh2 = make_float4(0.f, 0.f, 0.f, 0.f), vl2 = vh2;
                float w2 = 0.f;
                if (lane < n2) {
                    vh2 = xh4[j2 + b2 + lane];
                    vl2 = xl4[j2 + b2 + lane];
                    w2 = xt32[j2 + b2 + lane];
                }
                if (n > 0) st.push(kp, lane, n, vh.x, vh.y, vh.z, wv, vl.x, vl.y, vl.z);
                k = k2;
                b0 = b2;
                j0 = j2;
                nY = n2tot;
                n = n2;
                vh = vh2;
                vl = vl2;
                wv = w2;
            }
        }
        st.finish(kp, lane);
        double near = st.result();
        // the leaf itself: pairs with r = 0 (the diagonal, coincident points) are guarded
        Stream2<KIND, LOGS, true, true> self(ring[wl], s, th.x, th.y, th.z, tl.x, tl.y, tl.z);
        for (int b0 = 0; b0 < nB; b0 += 32) {
            const int n = min(32, nB - b0);
            float4 vh = make_float4(0.f, 0.f, 0.f, 0.f), vl = vh;
            float wv = 0.f;
            if (lane < n) {
                vh = xh4[i0 + b0 + lane];
                vl = xl4[i0 + b0 + lane];
                wv = xt32[i0 + b0 + lane];
            }
            self.push(kp, lane, n, vh.x, vh.y, vh.z, wv, vl.x, vl.y, vl.z);
        }
        self.finish(kp, lane);
        near += self.result();
        if (act && s == 0) {
            // L2P in FP64
            const int r = piv_off[B + 1] - piv_off[B];
            const double *U = op + op_off[B] + (int64_t)(a0 + t) * r;
            const double *uB = u + piv_off[B];
            double far = 0.0;
            for (int b = 0; b < r; ++b) far = fma(U[b], uB[b], far);
            // the pair (i, i) was evaluated as K(0); the diagonal takes the configured value
            const double yv = far + kp.s * near + (kp.diag - kp.s * (double)k0) * xt64[i];
            y[perm[i]] = (TO)yv;
        }
    }
}

// ---- leaves: L2P (FP64) + P2P (FP32), one warp per leaf ------------------------------
// A warp serves the c targets of one leaf: TPL consecutive targets per lane on
// L = ceil(c / TPL) lanes, and G = floor(32 / L) groups of L lanes that split
// the source pairs of every cell (the layout is chosen per leaf at build time
// to leave few target slots idle). The points of N(B) arrive by bulk
// asynchronous copies (TMA), one per cell, into NEAR_BUFS buffers of the warp,
// each tracked by its own mbarrier; the warp stages up to two rounds ahead of
// its evaluation, so no other warp takes part. Leaves adjacent to B (offset at
// most 1 in every coordinate) hold points that can come arbitrarily close to
// B's: they travel as absolute hi/lo pairs and every difference is formed as
// (hi_s - hi_t) + (lo_s - lo_t). The other leaves of N(B) are at least one leaf
// away: they travel relative to their own centre c_Y, and each target moves
// into that frame once per cell, t - c_Y = (hi_t - hi_c) + (lo_t - lo_c). Each
// cell is summed in float and added into a compensated total; pairs of B with
// itself are guarded against r = 0 (the diagonal takes the configured value
// afterwards).
// The near-field kernels do their packed arithmetic on float2 values with the
// compiler's f32x2 builtins instead of the 64-bit inline-PTX form the M2L
// kernels use: measured on the 1M-point 1/r product, the near pass takes 1.41
// instead of 1.52 ms this way, while the M2L kernels are faster in the other
// form (5.11 against 5.29 ms). The names shadow the outer ones inside this
// namespace.
namespace nf {
typedef float2 f2;
struct __align__(16) f2x2 {
    f2 x, y;
};
#define F2Z make_float2(0.f, 0.f)
__device__ __forceinline__ f2 f2_pack(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ float2 f2_unpack(f2 a) { return a; }
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2x2 ld2(const float4 *p) {
    const float4 v = *p;
    return f2x2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ f2x2 ldg2(const float4 *p) {
    const float4 v = __ldg(p);
    return f2x2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
// f(r^2) of a packed pair (SAFE: r^2 = 0 gives the singular kernels' 0)
template <int KIND, bool SAFE> struct KF2 {
    static __device__ __forceinline__ f2 eval(const KParams &kp, f2 r2) {
        return make_float2(SAFE ? KF<KIND>::f32(kp, r2.x) : KF<KIND>::f32_far(kp, r2.x),
                           SAFE ? KF<KIND>::f32(kp, r2.y) : KF<KIND>::f32_far(kp, r2.y));
    }
};
template <bool SAFE> struct KF2<NNCA_K_INV_R, SAFE> {
    static __device__ __forceinline__ f2 eval(const KParams &, f2 r2) {
        f2 f = make_float2(mufu_rsqrt(r2.x), mufu_rsqrt(r2.y));
#if NNCA_RSQRT_NEWTON
        const f2 h = f2_mul(r2, f);
        const f2 e = f2_fma(h, f, make_float2(-1.f, -1.f));
        f = f2_fma(f2_mul(f, make_float2(-0.5f, -0.5f)), e, f);
#endif
        if (SAFE) {
            f.x = r2.x > 0.f ? f.x : 0.f;
            f.y = r2.y > 0.f ? f.y : 0.f;
        }
        return f;
    }
};
// f(|s - t|^2) of a packed pair of sources A = (x0 x1 | y0 y1), B = (z0 z1 | w0 w1)
template <int KIND>
__device__ __forceinline__ f2 near_group_f(const KParams &kp, const f2x2 &A, const f2x2 &B, f2 tx, f2 ty, f2 tz) {
    const f2 dx = f2_sub(A.x, tx), dy = f2_sub(A.y, ty), dz = f2_sub(B.x, tz);
    f2 r2 = f2_mul(dx, dx);
    r2 = f2_fma(dy, dy, r2);
    r2 = f2_fma(dz, dz, r2);
    return KF2<KIND, false>::eval(kp, r2);
}
// acc += f(|s - t|^2) w over the same pair
template <int KIND>
__device__ __forceinline__ f2 near_group_pair(const KParams &kp, const f2x2 &A, const f2x2 &B, f2 tx, f2 ty, f2 tz,
                                              f2 acc) {
    return f2_fma(near_group_f<KIND>(kp, A, B, tx, ty, tz), B.y, acc);
}

struct NearWarpSmem {
    float4 u[NEAR_BUFS][NEAR_UNITS];      // staged points: hi/lo pairs (4 units) or local pairs (2 units)
    int hdr[NEAR_BUFS][NEAR_RECS];        // slot | pairs << 11 | own leaf << 22 | adjacent << 23
    float4 ch[NEAR_BUFS][NEAR_RECS];      // centre of the cell as float hi
    float4 cl[NEAR_BUFS][NEAR_RECS];      // and lo
    int nrec[NEAR_BUFS];
    unsigned long long full[NEAR_BUFS];   // mbarriers
};

struct NearTarget {
    bool act = false;
    int i = 0;   // sorted position
    f2 xh = F2Z, yh = F2Z, zh = F2Z, xl = F2Z, yl = F2Z, zl = F2Z;   // (t, t) packed
    float sum = 0.f, comp = 0.f;
};

__device__ __forceinline__ void near_target(NearTarget &T, bool act, int i, const float4 *xh4, const float4 *xl4) {
    T.act = act;
    T.i = i;
    if (!act) return;
    const float4 h = xh4[i], l = xl4[i];
    T.xh = f2_pack(h.x, h.x);
    T.yh = f2_pack(h.y, h.y);
    T.zh = f2_pack(h.z, h.z);
    T.xl = f2_pack(l.x, l.x);
    T.yl = f2_pack(l.y, l.y);
    T.zl = f2_pack(l.z, l.z);
}

// acc += f(|s - t|^2) w over a packed pair of sources; (hi_s - hi_t) + (lo_s - lo_t) per coordinate
template <int KIND, bool SAFE>
__device__ __forceinline__ f2 near_pair(const KParams &kp, const f2x2 &A, const f2x2 &B,
                                        const f2x2 &C, const f2x2 &D, const NearTarget &T, f2 acc) {
    const f2 dx = f2_add(f2_sub(A.x, T.xh), f2_sub(C.x, T.xl));
    const f2 dy = f2_add(f2_sub(A.y, T.yh), f2_sub(C.y, T.yl));
    const f2 dz = f2_add(f2_sub(B.x, T.zh), f2_sub(D.x, T.zl));
    f2 r2 = f2_mul(dx, dx);
    r2 = f2_fma(dy, dy, r2);
    r2 = f2_fma(dz, dz, r2);
    return f2_fma(KF2<KIND, SAFE>::eval(kp, r2), B.y, acc);
}

// The staging warp's copy of the next round's plan records (lane i: record k + i)
// and of the records' cell centres, loaded one round ahead.
struct NearCursor {
    int4 r = make_int4(0, 0, 0, 0);
    float4 ch = make_float4(0.f, 0.f, 0.f, 0.f), cl = make_float4(0.f, 0.f, 0.f, 0.f);
};

__device__ __forceinline__ void near_load(NearCursor &c, const int4 *plan, const float4 *chi, const float4 *clo, int k,
                                          int kend) {
    const int lane = threadIdx.x & 31;
    if (k + lane < kend) {
        c.r = plan[k + lane];
        c.ch = chi[c.r.x];
        c.cl = clo[c.r.x];
    }
}

// Stage the round held by the cursor into buffer b.
__device__ __forceinline__ int near_stage(NearWarpSmem &W, int b, const NearCursor &c, int k, int kend,
                                          const float4 *ppk, const float4 *ppl, unsigned *status) {
    const int lane = threadIdx.x & 31;
    const int nrec = __shfl_sync(0xffffffffu, c.r.w, 0);
    if (nrec < 1 || nrec > NEAR_RECS || k + nrec > kend) {   // a malformed plan: stop, never spin
        if (lane == 0) atomicOr(status, DEV_BAD_INDEX);
        return -1;
    }
    unsigned bytes = 0;
    const float4 *src = nullptr;
    if (lane < nrec) {
        const int adj = (c.r.z >> 23) & 1, np = (c.r.z >> 11) & 0x7ff;
        W.hdr[b][lane] = c.r.z;
        W.ch[b][lane] = c.ch;
        W.cl[b][lane] = c.cl;
        bytes = (unsigned)np * (adj ? 64u : 32u);
        src = adj ? ppk + 4 * (int64_t)c.r.y : ppl + 2 * (int64_t)c.r.y;
    }
    const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
    if (lane == 0) W.nrec[b] = nrec;
    // the buffer's previous contents were read by this warp's generic loads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive_tx(&W.full[b], total + g_stage_extra_tx);
    __syncwarp();
    if (lane < nrec) bulk_g2s(&W.u[b][c.r.z & 0x7ff], src, bytes, &W.full[b]);
    return k + nrec;
}

// an adjacent cell (hi/lo pairs at P[4 q]): this lane's group takes pairs g, g + G, ...
// (blocks of eight steps unrolled with a warp-uniform exit; the two chains take
// alternate pairs)
template <int KIND, int TPL, bool SAFE>
__device__ __forceinline__ void near_cell(const KParams &kp, const float4 *P, int np, int g, int G,
                                          NearTarget (&T)[TPL]) {
    f2 acc[TPL][2];
#pragma unroll
    for (int k = 0; k < TPL; ++k) acc[k][0] = acc[k][1] = F2Z;
    for (int q0 = g; q0 < np; q0 += 8 * G) {
        int q = q0;
#pragma unroll
        for (int s = 0; s < 8; ++s, q += G) {
            if (q >= np) break;
            const f2x2 A = ld2(&P[4 * q]);
            const f2x2 B = ld2(&P[4 * q + 1]);
            const f2x2 C = ld2(&P[4 * q + 2]);
            const f2x2 D = ld2(&P[4 * q + 3]);
#pragma unroll
            for (int k = 0; k < TPL; ++k) acc[k][s & 1] = near_pair<KIND, SAFE>(kp, A, B, C, D, T[k], acc[k][s & 1]);
        }
    }
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
        const float2 p = f2_unpack(f2_add(acc[k][0], acc[k][1]));
        two_sum_add(T[k].sum, T[k].comp, p.x + p.y);
    }
}

// a leaf at least one leaf away (pairs relative to its centre at P[2 q]): the
// targets move into its frame once, then one packed difference per coordinate
template <int KIND, int TPL>
__device__ __forceinline__ void near_cell_far(const KParams &kp, const float4 *P, int np, int g, int G, float4 ch,
                                              float4 cl, NearTarget (&T)[TPL]) {
    f2 tx[TPL], ty[TPL], tz[TPL], acc[TPL][2];
    {
        const f2 hx = f2_pack(ch.x, ch.x), hy = f2_pack(ch.y, ch.y), hz = f2_pack(ch.z, ch.z);
        const f2 lx = f2_pack(cl.x, cl.x), ly = f2_pack(cl.y, cl.y), lz = f2_pack(cl.z, cl.z);
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            tx[k] = f2_add(f2_sub(T[k].xh, hx), f2_sub(T[k].xl, lx));
            ty[k] = f2_add(f2_sub(T[k].yh, hy), f2_sub(T[k].yl, ly));
            tz[k] = f2_add(f2_sub(T[k].zh, hz), f2_sub(T[k].zl, lz));
            acc[k][0] = acc[k][1] = F2Z;
        }
    }
    for (int q0 = g; q0 < np; q0 += 8 * G) {
        int q = q0;
#pragma unroll
        for (int s = 0; s < 8; ++s, q += G) {
            if (q >= np) break;
            const f2x2 A = ld2(&P[2 * q]);
            const f2x2 B = ld2(&P[2 * q + 1]);
#pragma unroll
            for (int k = 0; k < TPL; ++k) acc[k][s & 1] = near_group_pair<KIND>(kp, A, B, tx[k], ty[k], tz[k], acc[k][s & 1]);
        }
    }
#pragma unroll
    for (int k = 0; k < TPL; ++k) {
        const float2 p = f2_unpack(f2_add(acc[k][0], acc[k][1]));
        two_sum_add(T[k].sum, T[k].comp, p.x + p.y);
    }
}

template <int KIND, int TPL, class TO>
__global__ void __launch_bounds__(32 * NEAR_WARPS) k_near_group(KParams kp, const int4 *items, int nitems,
                                                               int *next_item, const int4 *plan, const int32_t *cbeg,
                                                               const int32_t *piv_off, const int64_t *op_off,
                                                               const double *op, const double *u, const float4 *xh4,
                                                               const float4 *xl4, const float4 *chi, const float4 *clo,
                                                               const float4 *ppk, const float4 *ppl,
                                                               const double *xt64, const int32_t *perm, TO *y,
                                                               unsigned *status) {
    __shared__ __align__(128) NearWarpSmem Sm[NEAR_WARPS];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    NearWarpSmem &W = Sm[wl];
    if (lane == 0) {
        for (int b = 0; b < NEAR_BUFS; ++b) mbar_init(&W.full[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const float k0 = KF<KIND>::f32(kp, 0.f);
    unsigned R = 0, Rp = 0;   // rounds consumed, rounds staged
    bool failed = false;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(next_item, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems || failed) break;
        const int4 item = items[it];
        const int B = item.x, c = (item.y >> 16) & 0xff, G = (item.y >> 24) & 0x1f, kend = item.z + item.w;
        const int L = (c + TPL - 1) / TPL;
        const int g = lane / L, ti = lane - g * L;   // group, lane within the group
        const bool live = g < G;
        const int i0 = cbeg[B];
        NearTarget T[TPL];
#pragma unroll
        for (int k = 0; k < TPL; ++k) near_target(T[k], live && ti * TPL + k < c, i0 + ti * TPL + k, xh4, xl4);
        int kprod = item.z, kcons = item.z;
        NearCursor cur;
        near_load(cur, plan, chi, clo, kprod, kend);
        while (kcons < kend) {
            // stage up to two rounds beyond the one evaluated (the third buffer is free)
            while (kprod < kend && Rp <= R + NEAR_BUFS - 2) {
                const int kn = near_stage(W, Rp % NEAR_BUFS, cur, kprod, kend, ppk, ppl, status);
                if (kn < 0) {
                    kprod = kend;
                    failed = true;
                    break;
                }
                kprod = kn;
                ++Rp;
                near_load(cur, plan, chi, clo, kprod, kend);
            }
            if (failed) break;
            const int b = R % NEAR_BUFS;
            if (!mbar_wait_warp(&W.full[b], (R / NEAR_BUFS) & 1)) {
                if (lane == 0) atomicOr(status, DEV_WAIT_TIMEOUT);
                failed = true;
                break;
            }
            const int nrec = W.nrec[b];
            if (live)
                for (int e = 0; e < nrec; ++e) {
                    const int hw = W.hdr[b][e];
                    const float4 *P = &W.u[b][hw & 0x7ff];
                    const int np = (hw >> 11) & 0x7ff;
                    if (!((hw >> 23) & 1)) near_cell_far<KIND, TPL>(kp, P, np, g, G, W.ch[b][e], W.cl[b][e], T);
                    else if ((hw >> 22) & 1) near_cell<KIND, TPL, true>(kp, P, np, g, G, T);
                    else near_cell<KIND, TPL, false>(kp, P, np, g, G, T);
                }
            __syncwarp();
            ++R;
            kcons += nrec;
        }
        if (failed) break;
        // the groups summed disjoint source pairs of the same targets: combine into group 0
        for (int gg = 1; gg < G; ++gg) {
            const int srcl = min(ti + gg * L, 31);
#pragma unroll
            for (int k = 0; k < TPL; ++k) {
                const float so = __shfl_sync(0xffffffffu, T[k].sum, srcl);
                const float co = __shfl_sync(0xffffffffu, T[k].comp, srcl);
                if (g == 0) {
                    two_sum_add(T[k].sum, T[k].comp, so);
                    T[k].comp += co;
                }
            }
        }
        if (g == 0) {
            // L2P in FP64, then the diagonal: the pair (i, i) was evaluated as K(0)
            const int r = piv_off[B + 1] - piv_off[B];
            const double *uB = u + piv_off[B];
#pragma unroll
            for (int k = 0; k < TPL; ++k) {
                if (!T[k].act) continue;
                const double *Urow = op + op_off[B] + (int64_t)(T[k].i - i0) * r;
                double far = 0.0;
                for (int bb = 0; bb < r; ++bb) far = fma(Urow[bb], uB[bb], far);
                const double near = (double)T[k].sum + (double)T[k].comp;
                const double yv = far + kp.s * near + (kp.diag - kp.s * (double)k0) * xt64[T[k].i];
                y[perm[T[k].i]] = (TO)yv;
            }
        }
    }
    // after a failure: let copies still in flight land before the warp exits
    if (lane == 0)
        for (unsigned r = R; r < Rp; ++r) mbar_wait(&W.full[r % NEAR_BUFS], (r / NEAR_BUFS) & 1);
}

// ---- near field of M2L_RHS right-hand sides at once (FP32) -----------------------
// The same staging and pair arithmetic as k_near_group with two targets per lane;
// each kernel value feeds the four right-hand sides' accumulators, whose source
// weights come from pw4 (two float4 per point pair, L2-resident) beside the
// staged coordinates. L2P of the four and the diagonal term follow in the warp.
template <int NR> struct NearTarget4 {
    bool act = false;
    int i = 0;
    f2 xh = F2Z, yh = F2Z, zh = F2Z, xl = F2Z, yl = F2Z, zl = F2Z;
    float sum[NR] = {}, comp[NR] = {};
};

template <int NR>
__device__ __forceinline__ void near_target4(NearTarget4<NR> &T, bool act, int i, const float4 *xh4,
                                             const float4 *xl4) {
    T.act = act;
    T.i = i;
    if (!act) return;
    const float4 h = xh4[i], l = xl4[i];
    T.xh = f2_pack(h.x, h.x);
    T.yh = f2_pack(h.y, h.y);
    T.zh = f2_pack(h.z, h.z);
    T.xl = f2_pack(l.x, l.x);
    T.yl = f2_pack(l.y, l.y);
    T.zl = f2_pack(l.z, l.z);
}

// fold a cell's partial sums (acc[k][r]) into the compensated totals
template <int NR>
__device__ __forceinline__ void near4_fold(NearTarget4<NR> (&T)[2], f2 (&acc)[2][NR]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float2 p = f2_unpack(acc[k][r]);
            two_sum_add(T[k].sum[r], T[k].comp[r], p.x + p.y);
        }
}

// an adjacent cell (hi/lo pairs at P[4 q], weights of pair q at W[NR / 2 q]):
// this lane's group takes pairs g, g + G, ...
template <int KIND, bool SAFE, int NR>
__device__ __forceinline__ void near4_cell(const KParams &kp, const float4 *P, const float4 *W, int np, int g, int G,
                                           NearTarget4<NR> (&T)[2]) {
    f2 acc[2][NR];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[k][r] = F2Z;
    for (int q = g; q < np; q += G) {
        const f2x2 A = ld2(&P[4 * q]);
        const f2x2 B = ld2(&P[4 * q + 1]);
        const f2x2 C = ld2(&P[4 * q + 2]);
        const f2x2 D = ld2(&P[4 * q + 3]);
        f2x2 wv[NR / 2];
#pragma unroll
        for (int r2 = 0; r2 < NR / 2; ++r2) wv[r2] = ldg2(&W[(NR / 2) * q + r2]);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const f2 dx = f2_add(f2_sub(A.x, T[k].xh), f2_sub(C.x, T[k].xl));
            const f2 dy = f2_add(f2_sub(A.y, T[k].yh), f2_sub(C.y, T[k].yl));
            const f2 dz = f2_add(f2_sub(B.x, T[k].zh), f2_sub(D.x, T[k].zl));
            f2 r2 = f2_mul(dx, dx);
            r2 = f2_fma(dy, dy, r2);
            r2 = f2_fma(dz, dz, r2);
            const f2 f = KF2<KIND, SAFE>::eval(kp, r2);
#pragma unroll
            for (int r2 = 0; r2 < NR / 2; ++r2) {
                acc[k][2 * r2] = f2_fma(f, wv[r2].x, acc[k][2 * r2]);
                acc[k][2 * r2 + 1] = f2_fma(f, wv[r2].y, acc[k][2 * r2 + 1]);
            }
        }
    }
    near4_fold(T, acc);
}

// a leaf at least one leaf away (pairs relative to its centre at P[2 q])
template <int KIND, int NR>
__device__ __forceinline__ void near4_cell_far(const KParams &kp, const float4 *P, const float4 *W, int np, int g,
                                               int G, float4 ch, float4 cl, NearTarget4<NR> (&T)[2]) {
    f2 tx[2], ty[2], tz[2], acc[2][NR];
    {
        const f2 hx = f2_pack(ch.x, ch.x), hy = f2_pack(ch.y, ch.y), hz = f2_pack(ch.z, ch.z);
        const f2 lx = f2_pack(cl.x, cl.x), ly = f2_pack(cl.y, cl.y), lz = f2_pack(cl.z, cl.z);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            tx[k] = f2_add(f2_sub(T[k].xh, hx), f2_sub(T[k].xl, lx));
            ty[k] = f2_add(f2_sub(T[k].yh, hy), f2_sub(T[k].yl, ly));
            tz[k] = f2_add(f2_sub(T[k].zh, hz), f2_sub(T[k].zl, lz));
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[k][r] = F2Z;
        }
    }
    for (int q = g; q < np; q += G) {
        const f2x2 A = ld2(&P[2 * q]);
        const f2x2 B = ld2(&P[2 * q + 1]);
        f2x2 wv[NR / 2];
#pragma unroll
        for (int r2 = 0; r2 < NR / 2; ++r2) wv[r2] = ldg2(&W[(NR / 2) * q + r2]);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const f2 f = near_group_f<KIND>(kp, A, B, tx[k], ty[k], tz[k]);
#pragma unroll
            for (int r2 = 0; r2 < NR / 2; ++r2) {
                acc[k][2 * r2] = f2_fma(f, wv[r2].x, acc[k][2 * r2]);
                acc[k][2 * r2 + 1] = f2_fma(f, wv[r2].y, acc[k][2 * r2 + 1]);
            }
        }
    }
    near4_fold(T, acc);
}

// items: (leaf, first target | targets << 16 | groups << 24, first record, records);
// u, xt64: NR rows of npiv and N; y: NR rows of ld; pw: NR / 2 float4 of weights
// per point pair (k_near_weights4<NR>)
template <int KIND, class TO, int NR>
__global__ void __launch_bounds__(32 * NEAR_WARPS) k_near_rhs(KParams kp, const int4 *items, int nitems,
                                                             int *next_item, const int4 *plan, const int32_t *cbeg,
                                                             const int32_t *piv_off, const int64_t *op_off,
                                                             const double *op, const double *u, int64_t npiv,
                                                             const float4 *xh4, const float4 *xl4, const float4 *chi,
                                                             const float4 *clo, const float4 *ppk, const float4 *ppl,
                                                             const float4 *pw4, const double *xt64, int64_t N,
                                                             const int32_t *perm, TO *y, int64_t ld, unsigned *status) {
    __shared__ __align__(128) NearWarpSmem Sm[NEAR_WARPS];
    __shared__ int pq[NEAR_WARPS][NEAR_BUFS][NEAR_RECS];   // first global pair of each staged record
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    NearWarpSmem &W = Sm[wl];
    if (lane == 0) {
        for (int b = 0; b < NEAR_BUFS; ++b) mbar_init(&W.full[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const float k0 = KF<KIND>::f32(kp, 0.f);
    unsigned R = 0, Rp = 0;
    bool failed = false;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(next_item, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems || failed) break;
        const int4 item = items[it];
        const int B = item.x, f0 = item.y & 0xffff, c = (item.y >> 16) & 0xff, G = (item.y >> 24) & 0x1f;
        const int kend = item.z + item.w;
        const int L = (c + 1) / 2;
        const int g = lane / L, ti = lane - g * L;
        const bool live = g < G;
        const int i0 = cbeg[B] + f0;
        NearTarget4<NR> T[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) near_target4(T[k], live && ti * 2 + k < c, i0 + ti * 2 + k, xh4, xl4);
        int kprod = item.z, kcons = item.z;
        NearCursor cur;
        near_load(cur, plan, chi, clo, kprod, kend);
        while (kcons < kend) {
            while (kprod < kend && Rp <= R + NEAR_BUFS - 2) {
                const int b = Rp % NEAR_BUFS;
                if (lane < NEAR_RECS) pq[wl][b][lane] = cur.r.y;
                const int kn = near_stage(W, b, cur, kprod, kend, ppk, ppl, status);
                if (kn < 0) {
                    kprod = kend;
                    failed = true;
                    break;
                }
                kprod = kn;
                ++Rp;
                near_load(cur, plan, chi, clo, kprod, kend);
            }
            if (failed) break;
            const int b = R % NEAR_BUFS;
            if (!mbar_wait_warp(&W.full[b], (R / NEAR_BUFS) & 1)) {
                if (lane == 0) atomicOr(status, DEV_WAIT_TIMEOUT);
                failed = true;
                break;
            }
            const int nrec = W.nrec[b];
            if (live)
                for (int e = 0; e < nrec; ++e) {
                    const int hw = W.hdr[b][e];
                    const float4 *P = &W.u[b][hw & 0x7ff];
                    const float4 *Wt = pw4 + (NR / 2) * (int64_t)pq[wl][b][e];
                    const int np = (hw >> 11) & 0x7ff;
                    if (!((hw >> 23) & 1)) near4_cell_far<KIND, NR>(kp, P, Wt, np, g, G, W.ch[b][e], W.cl[b][e], T);
                    else if ((hw >> 22) & 1) near4_cell<KIND, true, NR>(kp, P, Wt, np, g, G, T);
                    else near4_cell<KIND, false, NR>(kp, P, Wt, np, g, G, T);
                }
            __syncwarp();
            ++R;
            kcons += nrec;
        }
        if (failed) break;
        for (int gg = 1; gg < G; ++gg) {
            const int srcl = min(ti + gg * L, 31);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float so = __shfl_sync(0xffffffffu, T[k].sum[r], srcl);
                    const float co = __shfl_sync(0xffffffffu, T[k].comp[r], srcl);
                    if (g == 0) {
                        two_sum_add(T[k].sum[r], T[k].comp[r], so);
                        T[k].comp[r] += co;
                    }
                }
        }
        if (g == 0) {
            // L2P of the NR in FP64 (one pass over the row of U_B), then the diagonal
            const int rk = piv_off[B + 1] - piv_off[B];
            const int64_t ub = piv_off[B];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!T[k].act) continue;
                const double *Urow = op + op_off[B] + (int64_t)(T[k].i - cbeg[B]) * rk;
                double far[NR] = {};
                for (int bb = 0; bb < rk; ++bb) {
                    const double ue = Urow[bb];
#pragma unroll
                    for (int r = 0; r < NR; ++r) far[r] = fma(ue, u[r * npiv + ub + bb], far[r]);
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const double near = (double)T[k].sum[r] + (double)T[k].comp[r];
                    const double yv =
                        far[r] + kp.s * near + (kp.diag - kp.s * (double)k0) * xt64[r * N + T[k].i];
                    y[r * ld + perm[T[k].i]] = (TO)yv;
                }
            }
        }
    }
    if (lane == 0)
        for (unsigned r = R; r < Rp; ++r) mbar_wait(&W.full[r % NEAR_BUFS], (r / NEAR_BUFS) & 1);
}

}  // namespace nf
using nf::k_near_group;
using nf::k_near_rhs;
#undef F2Z

// the NR right-hand sides' FP32 weights of every leaf point into pw: per point
// pair q, NR / 2 float4 [w(2q, r) w(2q+1, r) w(2q, r+1) w(2q+1, r+1)], r even
template <int NR>
__global__ void k_near_weights4(int64_t N, const double *xt, float *pw4, const int32_t *leaf_of, const int32_t *cbeg,
                                const int32_t *ppk_off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int B = leaf_of[i];
        const int64_t j = i - cbeg[B];
        const int64_t q = (int64_t)ppk_off[B] + (j >> 1);
#pragma unroll
        for (int r = 0; r < NR; ++r) pw4[2 * NR * q + (r >> 1) * 4 + (r & 1) * 2 + (j & 1)] = (float)xt[r * N + i];
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
// ---- M2L, FP32 evaluation, M2L_RHS right-hand sides per pass ---------------------------
// The same staging and evaluation as k_m2l_group; every round also brings the
// cells' weights of the M2L_RHS right-hand sides (a second bulk copy per record),
// and each kernel value f(|s - t|) feeds M2L_RHS accumulators, so the geometry
// and the MUFU work of a pair serve all of them.
struct M2lRhsSmem {
    float4 src[M2L_STAGE_BUFS][M2L_STAGE_CAP / 2][2];             // source pairs (coordinates)
    float4 wt[M2L_STAGE_BUFS][M2L_STAGE_CAP / 2][M2L_RHS / 2];    // their weights, two right-hand sides per float4
    int hdr[M2L_STAGE_BUFS][M2L_STAGE_RECS];
    float4 sh[M2L_STAGE_BUFS][M2L_STAGE_RECS];
    int nrec[M2L_STAGE_BUFS];
    unsigned long long full[M2L_STAGE_BUFS], empty[M2L_STAGE_BUFS];
    int2 ch_range[8];
    int item;
    int abort;
};

__device__ __forceinline__ int m2l_stage_rhs(M2lRhsSmem &S, int b, unsigned use, StageCursor &cur, const int4 *plan,
                                             const float4 *plan_sh, int kend, const float4 *spk, const float4 *spw,
                                             unsigned *status) {
    const int lane = threadIdx.x & 31;
    if (use > 0 && !mbar_wait_warp(&S.empty[b], (use - 1) & 1)) {
        if (lane == 0) {
            atomicOr(status, DEV_WAIT_TIMEOUT);
            *(volatile int *)&S.abort = 1;
        }
        return kend;
    }
    const int k = cur.k;
    const int nrec = __shfl_sync(0xffffffffu, cur.r.w, 0);
    if (nrec < 1 || nrec > M2L_STAGE_RECS || k + nrec > kend) {   // a malformed plan: stop, never spin
        if (lane == 0) {
            atomicOr(status, DEV_BAD_INDEX);
            *(volatile int *)&S.abort = 1;
        }
        return kend;
    }
    unsigned bytes = 0;
    const int4 r = cur.r;
    const unsigned np = (unsigned)((r.z >> 11) & 0x7ff);
    if (lane < nrec) {
        S.hdr[b][lane] = r.z;
        S.sh[b][lane] = cur.sh;
        bytes = np * 32u + np * (unsigned)(16 * (M2L_RHS / 2));
    }
    const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
    if (lane == 0) S.nrec[b] = nrec;
    __syncwarp();
    if (lane == 0) mbar_arrive_tx(&S.full[b], total + g_stage_extra_tx);
    __syncwarp();
    if (lane < nrec) {
        bulk_g2s(&S.src[b][r.z & 0x7ff][0], spk + 2 * (int64_t)r.y, np * 32u, &S.full[b]);
        bulk_g2s(&S.wt[b][r.z & 0x7ff][0], spw + (M2L_RHS / 2) * (int64_t)r.y, np * (unsigned)(16 * (M2L_RHS / 2)),
                 &S.full[b]);
    }
    if (k + nrec < kend) stage_load(cur, plan, plan_sh, k + nrec, kend);
    return k + nrec;
}


// The arguments of one problem of the four-RHS FP32 M2L. A launch serves the
// problems of a table, passed by value as a __grid_constant__ parameter (no
// device memory to fill, and captured as it is by a CUDA graph): items come from
// one counter over a cross-problem list of (problem, item) pairs, heaviest
// first, or, without such a list, from the first problem's own items.
struct M2lRhsArgs {
    KParams kp;
    const int4 *items;
    const int4 *plan;
    const float4 *plan_sh;
    const int32_t *cch_beg, *cch_end;
    const int2 *prange;
    const float4 *pv4, *chi, *clo, *spk, *spw;
    const int *item_part;
    double *parts, *u;
    int64_t npiv;
    unsigned *status;
};
template <int NT> struct M2lRhsTable {
    M2lRhsArgs a[NT];
};
constexpr int M2L_MULTI_MAX = 48;   // problems of one cross-problem launch (the table is a kernel parameter)

template <int KIND, int NT>
__global__ void __launch_bounds__(M2L_GROUP_THREADS) k_m2l_group_rhs(const __grid_constant__ M2lRhsTable<NT> tab,
                                                                   const int2 *gitems, int nitems, int *next_item) {
    extern __shared__ __align__(128) unsigned char m2l_rhs_smem[];
    M2lRhsSmem &S = *reinterpret_cast<M2lRhsSmem *>(m2l_rhs_smem);
    const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < M2L_STAGE_BUFS; ++b) {
            mbar_init(&S.full[b], 1);
            mbar_init(&S.empty[b], M2L_GROUP_WARPS);
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int pw = blockIdx.x % M2L_GROUP_WARPS;
    unsigned R = 0, Rp = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) S.item = atomicAdd(next_item, 1);
        __syncthreads();
        const int gi = S.item;
        if (gi >= nitems || *(volatile int *)&S.abort) break;
        int pidx = 0, it = gi;
        if (gitems) {
            const int2 e = gitems[gi];
            pidx = e.x;
            it = e.y;
        }
        const M2lRhsArgs &A = tab.a[pidx];
        const KParams &kp = A.kp;
        const int4 *plan = A.plan;
        const float4 *plan_sh = A.plan_sh, *pv4 = A.pv4, *chi = A.chi, *clo = A.clo, *spk = A.spk, *spw = A.spw;
        const int32_t *cch_beg = A.cch_beg, *cch_end = A.cch_end;
        const int2 *prange = A.prange;
        double *parts = A.parts, *u = A.u;
        const int64_t npiv = A.npiv;
        unsigned *status = A.status;
        const int4 item = A.items[it];
        const int part = A.item_part[it];
        const int P = item.x, t0 = item.y & 0xffff, nt = item.y >> 16, kend = item.z + item.w;
        const int cb = cch_beg[P], nch = cch_end[P] - cb;
        if (tid < nch) S.ch_range[tid] = prange[cb + tid];
        __syncthreads();
        const float4 hP = chi[P], lP = clo[P];
        int kprod = item.z, kcons = item.z;
        StageCursor cur;
        if (wl == pw && kprod < kend) stage_load(cur, plan, plan_sh, kprod, kend);
        const int wt = m2l_warp_targets(nt);
        const int wj0 = t0 + wl * wt, jend = t0 + nt;
        const int cw = min(wt, max(0, jend - wj0));
        const int L = cw > 0 ? (cw + 1) / 2 : 32;
        const int G = min(16, 32 / L);
        const int grp = lane / L, ti = lane - grp * L;
        const bool live = grp < G;
        const int j = wj0 + 2 * ti;
        const int g = S.ch_range[0].x + j;
        GroupTarget Ta, Tb;
        group_target(Ta, live && j < jend, g, nch, cb, S.ch_range, pv4, chi, clo, hP, lP);
        group_target(Tb, live && j + 1 < jend, g + 1, nch, cb, S.ch_range, pv4, chi, clo, hP, lP);
        float sa[M2L_RHS], ca[M2L_RHS], sb[M2L_RHS], cbm[M2L_RHS];
#pragma unroll
        for (int r = 0; r < M2L_RHS; ++r) sa[r] = ca[r] = sb[r] = cbm[r] = 0.f;
        const unsigned omask =
            __reduce_or_sync(0xffffffffu, (Ta.c < 31 ? 1u << Ta.c : 0u) | (Tb.c < 31 ? 1u << Tb.c : 0u));
        while (kcons < kend) {
            if (wl == pw)
                while (kprod < kend && Rp <= R + M2L_STAGE_AHEAD) {
                    kprod = m2l_stage_rhs(S, Rp % M2L_STAGE_BUFS, Rp / M2L_STAGE_BUFS, cur, plan, plan_sh, kend, spk,
                                          spw, status);
                    ++Rp;
                }
            const int b = R % M2L_STAGE_BUFS;
            if (!mbar_wait_warp(&S.full[b], (R / M2L_STAGE_BUFS) & 1)) {
                if (lane == 0) {
                    atomicOr(status, DEV_WAIT_TIMEOUT);
                    *(volatile int *)&S.abort = 1;
                }
                break;
            }
            const int nrec = S.nrec[b];
            if (nrec < 1) break;   // unreachable with a well-formed plan
            if (omask && live) {
                for (int i = 0; i < nrec; ++i) {
                    const int hw = S.hdr[b][i];
                    const unsigned m = ((unsigned)hw >> 22) & omask;
                    if (!m) continue;
                    const float4 sh = S.sh[b][i];
                    const f2 SX = f2_pack(sh.x, sh.x), SY = f2_pack(sh.y, sh.y), SZ = f2_pack(sh.z, sh.z);
                    const f2 xa = f2_sub(Ta.tx, SX), ya = f2_sub(Ta.ty, SY), za = f2_sub(Ta.tz, SZ);
                    const f2 xb = f2_sub(Tb.tx, SX), yb = f2_sub(Tb.ty, SY), zb = f2_sub(Tb.tz, SZ);
                    const int q0 = hw & 0x7ff, q1 = q0 + ((hw >> 11) & 0x7ff);
                    const bool ona = (m >> Ta.c) & 1u, onb = (m >> Tb.c) & 1u;
                    const int span = 2 * M2L_FOLD_RHS * G;
                    for (int c0 = q0; c0 < q1; c0 += span) {
                        const int c1 = min(q1, c0 + span);
                        f2 aa[M2L_RHS], ab[M2L_RHS];
#pragma unroll
                        for (int r = 0; r < M2L_RHS; ++r) aa[r] = ab[r] = 0ull;
                        // at most M2L_FOLD_RHS steps: unrolled with a warp-uniform exit
                        int q = c0 + (G == 1 ? 0 : 2 * grp);
#pragma unroll
                        for (int k = 0; k < M2L_FOLD_RHS; ++k, q += 2 * G) {
                            if (q >= c1) break;
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(&S.src[b][q + h2][0]);
                                const ulonglong2 B = *reinterpret_cast<const ulonglong2 *>(&S.src[b][q + h2][1]);
                                const f2 fa = group_f<KIND>(kp, A, B, xa, ya, za);
                                const f2 fb = group_f<KIND>(kp, A, B, xb, yb, zb);
#pragma unroll
                                for (int r2 = 0; r2 < M2L_RHS / 2; ++r2) {
                                    const ulonglong2 W = *reinterpret_cast<const ulonglong2 *>(&S.wt[b][q + h2][r2]);
                                    aa[2 * r2] = f2_fma(fa, W.x, aa[2 * r2]);
                                    aa[2 * r2 + 1] = f2_fma(fa, W.y, aa[2 * r2 + 1]);
                                    ab[2 * r2] = f2_fma(fb, W.x, ab[2 * r2]);
                                    ab[2 * r2 + 1] = f2_fma(fb, W.y, ab[2 * r2 + 1]);
                                }
                            }
                        }
#pragma unroll
                        for (int r = 0; r < M2L_RHS; ++r) {
                            const float2 pa = f2_unpack(aa[r]), pb = f2_unpack(ab[r]);
                            if (ona) two_sum_add(sa[r], ca[r], pa.x + pa.y);
                            if (onb) two_sum_add(sb[r], cbm[r], pb.x + pb.y);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[b]);
            ++R;
            kcons += nrec;
        }
        // the groups summed disjoint source pairs of the same targets: combine into group 0
        for (int gg = 1; gg < G; ++gg) {
            const int srcl = min(ti + gg * L, 31);
#pragma unroll
            for (int r = 0; r < M2L_RHS; ++r) {
                const float x1 = __shfl_sync(0xffffffffu, sa[r], srcl), y1 = __shfl_sync(0xffffffffu, ca[r], srcl);
                const float x2 = __shfl_sync(0xffffffffu, sb[r], srcl), y2 = __shfl_sync(0xffffffffu, cbm[r], srcl);
                if (grp == 0) {
                    two_sum_add(sa[r], ca[r], x1);
                    ca[r] += y1;
                    two_sum_add(sb[r], cbm[r], x2);
                    cbm[r] += y2;
                }
            }
        }
        if (grp == 0) {
            const int gb = S.ch_range[0].x + t0;
#pragma unroll
            for (int r = 0; r < M2L_RHS; ++r) {
                double *dst = part < 0 ? u + r * npiv + gb : parts + ((int64_t)part * M2L_RHS + r) * M2L_GROUP_TARGETS;
                if (Ta.c < 31) dst[Ta.g - gb] = kp.s * ((double)sa[r] + (double)ca[r]);
                if (Tb.c < 31) dst[Tb.g - gb] = kp.s * ((double)sb[r] + (double)cbm[r]);
            }
        }
    }
    if (wl == pw && lane == 0)
        for (unsigned r = R; r < Rp; ++r) mbar_wait(&S.full[r % M2L_STAGE_BUFS], (r / M2L_STAGE_BUFS) & 1);
}

// ---- M2L, FP32, symmetric form (one right-hand side) ------------------------------
// f(|s - t|) = f(|t - s|), and Y is in IL(X) exactly when X is in IL(Y)
// (admissibility and the neighbour relation are symmetric). So the plan of
// parent P lists only the children of its neighbours Q > P, and every kernel
// value a block evaluates serves twice: in the row sum u_X(t) += f w_Y(s), as in
// k_m2l_group, and in the column sum u_Y(s) += f w_X(t). Column sums of one
// chunk of sources (M2L_FOLD couples of pairs per lane) go through a per-warp
// transpose buffer and are summed over the warp's targets in a fixed order;
// the last warp to finish a round adds the four warps' sums (warp order) and
// writes them to the item's column slots; k_m2l_cols adds each cell's slots
// into u in a fixed order. The result is deterministic.

// the source pairs q0, q0 + step, ... below q1 (two at a time) of one staged
// segment against two targets: row sums into a*, b*; the column values
// f_a w_a + f_b w_b of each source pair into crow[q]. FULL (the whole warp,
// step 2) with UNR: a chunk takes at most M2L_FOLD steps, and the loop is
// unrolled that far with a warp-uniform exit; otherwise a counted loop. The
// unrolled form is faster on trees with long staged records (M2L of the
// 1M-point 1/r workload 5.39 -> 5.15 ms) and slower on trees of tiny cells
// (262k-point Chebyshev grid 12.8 -> 16.5 ms; unrolling the lane-group path of
// small items as well took it to 21.4 ms), so the build picks UNR per handle.
template <int KIND, int FULL, int UNR = 1>
__device__ __forceinline__ void m2l_sym_pairs(const KParams &kp, const float4 (*src)[2], int q0, int q1, f2 xa, f2 ya,
                                              f2 za, f2 xb, f2 yb, f2 zb, f2 WA, f2 WB, f2 *crow, f2 &a0, f2 &a1,
                                              f2 &b0, f2 &b1, int step = 2) {
    auto body = [&](int q) {
        const ulonglong2 A0 = *reinterpret_cast<const ulonglong2 *>(&src[q][0]);
        const ulonglong2 B0 = *reinterpret_cast<const ulonglong2 *>(&src[q][1]);
        const ulonglong2 A1 = *reinterpret_cast<const ulonglong2 *>(&src[q + 1][0]);
        const ulonglong2 B1 = *reinterpret_cast<const ulonglong2 *>(&src[q + 1][1]);
        const f2 fa0 = group_f<KIND>(kp, A0, B0, xa, ya, za), fb0 = group_f<KIND>(kp, A0, B0, xb, yb, zb);
        const f2 fa1 = group_f<KIND>(kp, A1, B1, xa, ya, za), fb1 = group_f<KIND>(kp, A1, B1, xb, yb, zb);
        a0 = f2_fma(fa0, B0.y, a0);
        b0 = f2_fma(fb0, B0.y, b0);
        a1 = f2_fma(fa1, B1.y, a1);
        b1 = f2_fma(fb1, B1.y, b1);
        crow[q] = f2_fma(fb0, WB, f2_mul(fa0, WA));
        crow[q + 1] = f2_fma(fb1, WB, f2_mul(fa1, WA));
    };
    if (FULL && !UNR) {
        for (int q = q0; q < q1; q += 2) body(q);
    } else if (FULL) {
#pragma unroll
        for (int k = 0; k < M2L_FOLD; ++k) {
            if (q0 + 2 * k >= q1) break;
            body(q0 + 2 * k);
        }
    } else {
        for (int q = q0; q < q1; q += step) body(q);
    }
}

// Column sums of one chunk: the transpose buffer holds, per target lane t < L
// (row t, stride rs), the column values of the chunk's np2 source pairs. Lane
// (h, p) sums pair p over one half of the rows, in row order; the halves are
// added (half 0 + half 1) and written as the pair's two column sums. LL > 0:
// L = LL rows with G = 32 / LL groups (row stride 16 G + 1), unrolled.
template <int LL>
__device__ __forceinline__ void m2l_sym_columns(const f2 *cbuf, int rs, int L, int np2, int lane, f2 *out) {
    const int h = lane >> 4, pl = lane & 15;
    for (int pb = 0; pb < np2; pb += 16) {
        const int p = pb + pl;
        f2 s0 = 0ull, s1 = 0ull;
        if (p < np2) {
            if (LL > 0) {
                constexpr int RS = LL > 0 ? 2 * M2L_FOLD * (32 / (LL > 0 ? LL : 1)) + 1 : 1;
                constexpr int HR = LL > 1 ? LL / 2 : 1;   // rows per half
                if (LL > 1 || h == 0) {
                    const f2 *c = cbuf + h * HR * RS + p;
#pragma unroll
                    for (int k = 0; k < HR; k += 2) {
                        s0 = f2_add(s0, c[k * RS]);
                        if (k + 1 < HR) s1 = f2_add(s1, c[(k + 1) * RS]);
                    }
                }
            } else {
                const int hl = (L + 1) >> 1, r0 = h ? hl : 0, r1 = h ? L : hl;
                for (int r = r0; r < r1; ++r) s0 = f2_add(s0, cbuf[r * rs + p]);
            }
        }
        const f2 mine = f2_add(s0, s1);
        const f2 other = __shfl_xor_sync(0xffffffffu, mine, 16);
        if (h == 0 && p < np2) out[p] = f2_add(mine, other);
    }
}

__device__ __forceinline__ void m2l_sym_columns_any(const f2 *cbuf, int rs, int L, int G, int np2, int lane, f2 *out) {
    if (L * G == 32) {
        switch (L) {
        case 32: m2l_sym_columns<32>(cbuf, rs, L, np2, lane, out); return;
        case 16: m2l_sym_columns<16>(cbuf, rs, L, np2, lane, out); return;
        case 8: m2l_sym_columns<8>(cbuf, rs, L, np2, lane, out); return;
        case 4: m2l_sym_columns<4>(cbuf, rs, L, np2, lane, out); return;
        default: break;
        }
    }
    m2l_sym_columns<0>(cbuf, rs, L, np2, lane, out);
}

template <int KIND, int UNR>
__global__ void __launch_bounds__(M2L_GROUP_THREADS, KIND == NNCA_K_INV_R ? 5 : 4) k_m2l_sym(KParams kp, const int4 *items, int nitems,
                                                             int *next_item, const int4 *plan, const float4 *plan_sh,
                                                             const int32_t *cch_beg, const int32_t *cch_end,
                                                             const int2 *prange, const float4 *pv4, const float4 *chi,
                                                             const float4 *clo, const float4 *spk, const double *w,
                                                             const int *item_part, const int *item_col, double *parts,
                                                             double *u, float *col, unsigned *status) {
    extern __shared__ __align__(128) unsigned char sym_smem[];
    M2lSymSmem &S = *reinterpret_cast<M2lSymSmem *>(sym_smem);
    const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < M2L_SYM_BUFS; ++b) {
            mbar_init(&S.full[b], 1);
            mbar_init(&S.empty[b], M2L_GROUP_WARPS);
            S.cnt[b] = 0;
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int pw = blockIdx.x % M2L_GROUP_WARPS;
    unsigned R = 0, Rp = 0;
    f2 *cbuf = reinterpret_cast<f2 *>(S.colbuf[wl]);
    for (;;) {
        __syncthreads();
        if (tid == 0) S.item = atomicAdd(next_item, 1);
        __syncthreads();
        const int it = S.item;
        if (it >= nitems || *(volatile int *)&S.abort) break;
        const int4 item = items[it];
        const int part = item_part[it];
        const int P = item.x, t0 = item.y & 0xffff, nt = item.y >> 16, kend = item.z + item.w;
        const int cb = cch_beg[P], nch = cch_end[P] - cb;
        if (tid < nch) S.ch_range[tid] = prange[cb + tid];
        if (tid == 0) S.scol = item_col[it];
        __syncthreads();
        const float4 hP = chi[P], lP = clo[P];
        int kprod = item.z, kcons = item.z;
        StageCursor cur;
        if (wl == pw && kprod < kend) stage_load(cur, plan, plan_sh, kprod, kend);
        const int wt = m2l_warp_targets(nt);
        const int wj0 = t0 + wl * wt, jend = t0 + nt;
        const int cw = min(wt, max(0, jend - wj0));
        const int L = cw > 0 ? (cw + 1) / 2 : 32;
        const int G = min(16, 32 / L);
        const int grp = lane / L, ti = lane - grp * L;
        const bool live = grp < G;
        const int j = wj0 + 2 * ti;
        const int g = S.ch_range[0].x + j;
        GroupTarget Ta, Tb;
        group_target(Ta, live && j < jend, g, nch, cb, S.ch_range, pv4, chi, clo, hP, lP);
        group_target(Tb, live && j + 1 < jend, g + 1, nch, cb, S.ch_range, pv4, chi, clo, hP, lP);
        const float wa = Ta.c < 31 ? (float)w[Ta.g] : 0.f, wb = Tb.c < 31 ? (float)w[Tb.g] : 0.f;
        const unsigned omask =
            __reduce_or_sync(0xffffffffu, (Ta.c < 31 ? 1u << Ta.c : 0u) | (Tb.c < 31 ? 1u << Tb.c : 0u));
        const int span = 2 * M2L_FOLD * G, rs = span + 1;   // chunk (source pairs) and transpose row length
        while (kcons < kend) {
            if (wl == pw)
                while (kprod < kend && Rp <= R + M2L_SYM_AHEAD) {
                    kprod = m2l_stage(S, Rp % M2L_SYM_BUFS, Rp / M2L_SYM_BUFS, cur, plan, plan_sh, kend, spk,
                                      status);
                    ++Rp;
                }
            const int b = R % M2L_SYM_BUFS;
            if (!mbar_wait_warp(&S.full[b], (R / M2L_SYM_BUFS) & 1)) {
                if (lane == 0) {
                    atomicOr(status, DEV_WAIT_TIMEOUT);
                    *(volatile int *)&S.abort = 1;
                }
                break;
            }
            const int nrec = S.nrec[b];
            if (nrec < 1) break;   // unreachable with a well-formed plan
            float *cwb = S.colw[b][wl];
            for (int i = 0; i < nrec; ++i) {
                const int hw = S.hdr[b][i];
                const unsigned m = ((unsigned)hw >> 22) & omask;
                const int q0 = hw & 0x7ff, q1 = q0 + ((hw >> 11) & 0x7ff);
                if (!m) {   // no target of this warp sees the segment: its column sums here are 0
                    for (int e = 2 * q0 + lane; e < 2 * q1; e += 32) cwb[e] = 0.f;
                    continue;
                }
                const float4 sh = S.sh[b][i];
                const f2 SX = f2_pack(sh.x, sh.x), SY = f2_pack(sh.y, sh.y), SZ = f2_pack(sh.z, sh.z);
                const f2 xa = f2_sub(Ta.tx, SX), ya = f2_sub(Ta.ty, SY), za = f2_sub(Ta.tz, SZ);
                const f2 xb = f2_sub(Tb.tx, SX), yb = f2_sub(Tb.ty, SY), zb = f2_sub(Tb.tz, SZ);
                const bool ona = (m >> Ta.c) & 1u, onb = (m >> Tb.c) & 1u;
                const float ea = ona ? wa : 0.f, eb = onb ? wb : 0.f;
                const f2 WA = f2_pack(ea, ea), WB = f2_pack(eb, eb);
                for (int c0 = q0; c0 < q1; c0 += span) {
                    const int c1 = min(q1, c0 + span);
                    if (live) {
                        f2 a0 = 0ull, a1 = 0ull, b0 = 0ull, b1 = 0ull;
                        f2 *crow = cbuf + ti * rs - c0;
                        if (G == 1)
                            m2l_sym_pairs<KIND, 1, UNR>(kp, S.src[b], c0, c1, xa, ya, za, xb, yb, zb, WA, WB, crow, a0, a1, b0,
                                                   b1);
                        else
                            m2l_sym_pairs<KIND, 0>(kp, S.src[b], c0 + 2 * grp, c1, xa, ya, za, xb, yb, zb, WA, WB, crow,
                                                   a0, a1, b0, b1, 2 * G);
                        const float2 pa = f2_unpack(f2_add(a0, a1)), pb = f2_unpack(f2_add(b0, b1));
                        if (ona) two_sum_add(Ta.sum, Ta.comp, pa.x + pa.y);
                        if (onb) two_sum_add(Tb.sum, Tb.comp, pb.x + pb.y);
                    }
                    __syncwarp();
                    m2l_sym_columns_any(cbuf, rs, L, G, c1 - c0, lane, reinterpret_cast<f2 *>(cwb) + c0);
                    __syncwarp();
                }
            }
            // this warp's column sums of the round are in colw[b][wl]; the last
            // warp to get here adds the four in warp order and writes the slots
            __threadfence_block();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&S.cnt[b], 1) == M2L_GROUP_WARPS - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence_block();
                const int ns = min(S.rsrc[b], M2L_SYM_CAP);
                float *dst = col + S.rbase[b];
                for (int e = lane; e < ns; e += 32)
                    dst[e] = (S.colw[b][0][e] + S.colw[b][1][e]) + (S.colw[b][2][e] + S.colw[b][3][e]);
                __syncwarp();
                if (lane == 0) S.cnt[b] = 0;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.empty[b]);
            ++R;
            kcons += nrec;
        }
        for (int gg = 1; gg < G; ++gg) {
            const int srcl = min(ti + gg * L, 31);
            const float sa = __shfl_sync(0xffffffffu, Ta.sum, srcl), ca = __shfl_sync(0xffffffffu, Ta.comp, srcl);
            const float sb = __shfl_sync(0xffffffffu, Tb.sum, srcl), cb2 = __shfl_sync(0xffffffffu, Tb.comp, srcl);
            if (grp == 0) {
                two_sum_add(Ta.sum, Ta.comp, sa);
                Ta.comp += ca;
                two_sum_add(Tb.sum, Tb.comp, sb);
                Tb.comp += cb2;
            }
        }
        if (grp == 0) {
            const int gb = S.ch_range[0].x + t0;
            double *dst = part < 0 ? u + gb : parts + (int64_t)part * M2L_GROUP_TARGETS;
            if (Ta.c < 31) dst[Ta.g - gb] = kp.s * ((double)Ta.sum + (double)Ta.comp);
            if (Tb.c < 31) dst[Tb.g - gb] = kp.s * ((double)Tb.sum + (double)Tb.comp);
        }
    }
    if (wl == pw && lane == 0)
        for (unsigned r = R; r < Rp; ++r) mbar_wait(&S.full[r % M2L_SYM_BUFS], (r / M2L_SYM_BUFS) & 1);
}

// column sums of the symmetric M2L: u(Y) += s * (Y's slots, in their fixed order).
// One warp per task (cell Y, first pivot j0): lane j0 + l sums its column over
// Y's slots, reading 32 slot offsets at a time and issuing the 32 slot loads
// before adding them; the sums are compensated float sums (two-sum), so no
// FP64 arithmetic sits in the loop
__global__ void k_m2l_cols(const int2 *tasks, int ntasks, const int32_t *ent_off, const int32_t *ent,
                           const int2 *prange, const float *col, double s, double *u) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < ntasks; i += nw) {
        const int2 tk = tasks[i];
        const int Y = tk.x;
        const int2 pr = prange[Y];
        const int e0 = ent_off[Y], e1 = ent_off[Y + 1];
        const int jj = tk.y + lane;
        const bool on = jj < pr.y;
        float sum = 0.f, comp = 0.f;
        for (int eb = e0; eb < e1; eb += 32) {
            const int n = min(32, e1 - eb);
            const int my = lane < n ? ent[eb + lane] : 0;
            float f[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int sl = __shfl_sync(0xffffffffu, my, q);
                f[q] = on && q < n ? col[sl + jj] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) two_sum_add(sum, comp, f[q]);   // a 0 leaves (sum, comp) unchanged
        }
        if (on) u[pr.x + jj] += s * ((double)sum + (double)comp);
    }
}

// u of the targets of a split item: the sum of its pieces' partial sums, in piece order
// (nr right-hand sides: slot s holds nr consecutive rows of M2L_GROUP_TARGETS)
__global__ void k_m2l_combine(const int4 *split, int nsplit, const double *parts, double *u, int nr, int64_t npiv) {
    for (int i = blockIdx.x; i < nsplit; i += gridDim.x) {
        const int4 sp = split[i];   // first pivot, targets, first slot, pieces
        for (int e = threadIdx.x; e < sp.y * nr; e += blockDim.x) {
            const int r = e / sp.y, j = e - r * sp.y;
            double v = 0.0;
            for (int p = 0; p < sp.w; ++p) v += parts[((int64_t)(sp.z + p) * nr + r) * M2L_GROUP_TARGETS + j];
            u[r * npiv + sp.x + j] = v;
        }
    }
}

template <int KIND>
void launch_m2l_f32(Handle *h, double *u) {
    if (!h->n_m2l_groups) return;
    int dev = 0, nsm = 152, per_sm = 1;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    NNCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_m2l_group<KIND>, M2L_GROUP_THREADS, 0));
    const unsigned g = (unsigned)std::min<int64_t>(h->n_m2l_groups, (int64_t)nsm * std::max(1, per_sm));
    NNCA_CUDA(cudaMemsetAsync(h->m2l_next, 0, sizeof(int), h->stream));
    k_m2l_group<KIND><<<g, M2L_GROUP_THREADS, 0, h->stream>>>(h->kp, h->m2l_groups, h->n_m2l_groups, h->m2l_next,
                                                             h->m2l_plan, h->m2l_plan_sh, h->cch_beg, h->cch_end, h->prange, h->pv4,
                                                             h->chi4, h->clo4, h->spk, h->m2l_item_part, h->m2l_parts, u,
                                                             h->dev_status);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
    if (h->n_m2l_split) {
        k_m2l_combine<<<(unsigned)std::min(h->n_m2l_split, 152 * 16), 256, 0, h->stream>>>(h->m2l_split, h->n_m2l_split,
                                                                                          h->m2l_parts, u, 1, h->npiv);
        NNCA_LAUNCH_CHECK();
        ++h->launches;
    }
}

// the symmetric form: rows by k_m2l_sym (and the split pieces' combine), then
// the column sums of every cell
template <int KIND, int UNR>
void launch_m2l_sym_kernel(Handle *h, const double *w, double *u) {
    const int smem = (int)sizeof(M2lSymSmem);
    NNCA_CUDA(cudaFuncSetAttribute(k_m2l_sym<KIND, UNR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int dev = 0, nsm = 152, per_sm = 1;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    NNCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_m2l_sym<KIND, UNR>, M2L_GROUP_THREADS, smem));
    const unsigned g = (unsigned)std::min<int64_t>(h->n_sym_items, (int64_t)nsm * std::max(1, per_sm));
    NNCA_CUDA(cudaMemsetAsync(h->m2l_next, 0, sizeof(int), h->stream));
    k_m2l_sym<KIND, UNR><<<g, M2L_GROUP_THREADS, smem, h->stream>>>(
        h->kp, h->sym_items, h->n_sym_items, h->m2l_next, h->sym_plan, h->sym_plan_sh, h->cch_beg, h->cch_end,
        h->prange, h->pv4, h->chi4, h->clo4, h->spk, w, h->sym_item_part, h->sym_item_col, h->sym_parts, u,
        h->sym_col, h->dev_status);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
}

template <int KIND>
void launch_m2l_sym(Handle *h, const double *w, double *u) {
    if (h->n_sym_items) {
        if (h->sym_unroll) launch_m2l_sym_kernel<KIND, 1>(h, w, u);
        else launch_m2l_sym_kernel<KIND, 0>(h, w, u);
    }
    if (h->n_sym_split) {
        k_m2l_combine<<<(unsigned)std::min(h->n_sym_split, 152 * 16), 256, 0, h->stream>>>(h->sym_split, h->n_sym_split,
                                                                                          h->sym_parts, u, 1, h->npiv);
        NNCA_LAUNCH_CHECK();
        ++h->launches;
    }
    if (h->n_sym_tasks) {
        k_m2l_cols<<<grid_for((int64_t)h->n_sym_tasks * 32, 256), 256, 0, h->stream>>>(
            h->sym_tasks, h->n_sym_tasks, h->sym_ent_off, h->sym_ent, h->prange, h->sym_col, h->kp.s, u);
        NNCA_LAUNCH_CHECK();
        ++h->launches;
    }
}

// M2L_RHS right-hand sides at once (u: M2L_RHS rows of npiv)
M2lRhsArgs m2l_rhs_args(Handle *h, double *u) {
    M2lRhsArgs A{};
    A.kp = h->kp;
    A.items = h->m2l_groups;
    A.plan = h->m2l_plan;
    A.plan_sh = h->m2l_plan_sh;
    A.cch_beg = h->cch_beg;
    A.cch_end = h->cch_end;
    A.prange = h->prange;
    A.pv4 = h->pv4;
    A.chi = h->chi4;
    A.clo = h->clo4;
    A.spk = h->spk;
    A.spw = h->spw;
    A.item_part = h->m2l_item_part;
    A.parts = h->m2l_parts;
    A.u = u;
    A.npiv = h->npiv;
    A.status = h->dev_status;
    return A;
}

// one launch of the four-RHS FP32 M2L over a table of problems (gitems: the
// cross-problem (problem, item) list, or null for the first problem's items)
template <int KIND, int NT>
void launch_m2l_rhs_table(const M2lRhsTable<NT> &tab, const int2 *gitems, int nitems, int *next, cudaStream_t s) {
    const int smem = (int)sizeof(M2lRhsSmem);
    NNCA_CUDA(cudaFuncSetAttribute(k_m2l_group_rhs<KIND, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int dev = 0, nsm = 152, per_sm = 1;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    NNCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_m2l_group_rhs<KIND, NT>, M2L_GROUP_THREADS, smem));
    const unsigned g = (unsigned)std::min<int64_t>(nitems, (int64_t)nsm * std::max(1, per_sm));
    NNCA_CUDA(cudaMemsetAsync(next, 0, sizeof(int), s));
    k_m2l_group_rhs<KIND, NT><<<g, M2L_GROUP_THREADS, smem, s>>>(tab, gitems, nitems, next);
    NNCA_LAUNCH_CHECK();
}

void m2l_rhs_combine(Handle *h, double *u) {
    if (!h->n_m2l_split) return;
    k_m2l_combine<<<(unsigned)std::min(h->n_m2l_split, 152 * 16), 256, 0, h->stream>>>(h->m2l_split, h->n_m2l_split,
                                                                                       h->m2l_parts, u, M2L_RHS,
                                                                                       h->npiv);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
}

template <int KIND>
void launch_m2l_f32_rhs(Handle *h, double *u, const float4 *spw = nullptr) {
    if (!h->n_m2l_groups) return;
    M2lRhsTable<1> tab;
    tab.a[0] = m2l_rhs_args(h, u);
    if (spw) tab.a[0].spw = spw;   // the packed weights of this group (else the handle's one-group buffer)
    launch_m2l_rhs_table<KIND, 1>(tab, nullptr, h->n_m2l_groups, h->m2l_next, h->stream);
    ++h->launches;
    m2l_rhs_combine(h, u);
}

template <int KIND, class TO>
void launch_leaf_f32(Handle *h, const double *op, const double *u, const float *xt32, const double *xt64, TO *y) {
    if (h->near_packed) {
        int dev = 0, nsm = 152;
        NNCA_CUDA(cudaGetDevice(&dev));
        NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        NNCA_CUDA(cudaMemsetAsync(h->near_next, 0, 2 * sizeof(int), h->stream));
        for (int t = 0; t < 2; ++t) {
            const int n = h->n_near_items[t];
            if (!n) continue;
            int per_sm = 1;
#define NNCA_NEAR(TPL)                                                                                                 \
    do {                                                                                                               \
        NNCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_near_group<KIND, TPL, TO>, 32 * NEAR_WARPS, 0)); \
        const int64_t warps = (int64_t)nsm * std::max(1, per_sm) * NEAR_WARPS;                                         \
        const unsigned g = (unsigned)((std::min<int64_t>(n, warps) + NEAR_WARPS - 1) / NEAR_WARPS);                    \
        k_near_group<KIND, TPL, TO><<<g, 32 * NEAR_WARPS, 0, h->stream>>>(                                             \
            h->kp, h->near_items[t], n, h->near_next + t, h->near_plan, h->cbeg, h->piv_off, h->op_off, op, u, h->xh4, \
            h->xl4, h->chi4, h->clo4, h->ppk, h->ppl, xt64, h->perm, y, h->dev_status);                                \
    } while (0)
            if (t == 0) NNCA_NEAR(2);
            else NNCA_NEAR(3);
#undef NNCA_NEAR
            NNCA_LAUNCH_CHECK();
            ++h->launches;
        }
        return;
    }
    for (int ls = 0; ls < 5; ++ls) {
        const int n = h->n_leaf_items[ls];
        if (!n) continue;
        const unsigned g = grid_for(n, MV_WARPS, 152 * 16);
#define NNCA_LEAF(LS)                                                                                                  \
    k_leaf_f32<KIND, LS, TO><<<g, 32 * MV_WARPS, 0, h->stream>>>(h->kp, h->leaf_items[ls], n, h->cbeg, h->cend,         \
                                                                 h->nb_off, h->nb_idx, h->piv_off, h->op_off, op, u,    \
                                                                 h->xh4, h->xl4, xt32, xt64, h->perm, y)
        switch (ls) {
        case 0: NNCA_LEAF(0); break;
        case 1: NNCA_LEAF(1); break;
        case 2: NNCA_LEAF(2); break;
        case 3: NNCA_LEAF(3); break;
        default: NNCA_LEAF(4); break;
        }
#undef NNCA_LEAF
        NNCA_LAUNCH_CHECK();
        ++h->launches;
    }
}

// the near field of NR right-hand sides (u, xt64: NR rows; y: rows of ld): their
// weights into pw (NR / 2 float4 per point pair), then one pass over the leaves
template <int KIND, class TO, int NR>
void launch_near_rhs(Handle *h, const double *op, const double *u, const double *xt64, TO *y, int64_t ld, float4 *pw) {
    NNCA_REQUIRE(pw != nullptr, NNCA_ERR_INTERNAL, "near-field weights of this group size not allocated");
    const int64_t N = h->n;
    k_near_weights4<NR><<<grid_for(N, 256), 256, 0, h->stream>>>(N, xt64, reinterpret_cast<float *>(pw), h->leaf_of,
                                                                 h->cbeg, h->ppk_off);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
    int dev = 0, nsm = 152, per_sm = 1;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    NNCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_near_rhs<KIND, TO, NR>, 32 * NEAR_WARPS, 0));
    const int n = h->n_near_items4;
    const int64_t warps = (int64_t)nsm * std::max(1, per_sm) * NEAR_WARPS;
    const unsigned g = (unsigned)((std::min<int64_t>(n, warps) + NEAR_WARPS - 1) / NEAR_WARPS);
    NNCA_CUDA(cudaMemsetAsync(h->near_next + 2, 0, sizeof(int), h->stream));
    k_near_rhs<KIND, TO, NR><<<g, 32 * NEAR_WARPS, 0, h->stream>>>(
        h->kp, h->near_items4, n, h->near_next + 2, h->near_plan, h->cbeg, h->piv_off, h->op_off, op, u, h->npiv,
        h->xh4, h->xl4, h->chi4, h->clo4, h->ppk, h->ppl, pw, xt64, h->n, h->perm, y, ld, h->dev_status);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
}

// The slot tables of the symmetric FP64 M2L (built on the first FP64 product of
// one right-hand side): per interaction-list entry e = (X, Y) with Y > X its
// column slots' first index, and for an entry with Y < X the first slot of its
// partner (Y, X); the slots themselves (one double per column of every entry
// Y > X).
void ensure_f64_sym(Handle *h) {
    if (h->f64_slot_of || h->n_il == 0) return;
    const int64_t nc = h->ncell, nil = h->n_il;
    std::vector<int32_t> off(nc + 1), idx(nil);
    NNCA_CUDA(cudaMemcpy(off.data(), h->il_off, (nc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    NNCA_CUDA(cudaMemcpy(idx.data(), h->il_idx, nil * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int64_t> slot(nil, -1);
    int64_t total = 0;
    for (int64_t X = 0; X < nc; ++X)
        for (int32_t e = off[X]; e < off[X + 1]; ++e) {
            const int32_t Y = idx[e];
            if (Y > X) {
                slot[e] = total;
                total += h->h_piv_off[Y + 1] - h->h_piv_off[Y];
            }
        }
    for (int64_t X = 0; X < nc; ++X)
        for (int32_t e = off[X]; e < off[X + 1]; ++e) {
            const int32_t Y = idx[e];
            if (Y >= X) continue;
            // the partner entry (Y, X) in Y's list (lists are in ascending cell order)
            const int32_t *b = idx.data() + off[Y], *eend = idx.data() + off[Y + 1];
            const int32_t *f = std::lower_bound(b, eend, (int32_t)X);
            NNCA_REQUIRE(f != eend && *f == X, NNCA_ERR_INTERNAL, "interaction lists are not symmetric");
            slot[e] = slot[off[Y] + (f - b)];
        }
    h->f64_slot_of = dalloc<int64_t>(h, nil);
    NNCA_CUDA(cudaMemcpy(h->f64_slot_of, slot.data(), nil * sizeof(int64_t), cudaMemcpyHostToDevice));
    h->f64_slots = dalloc<double>(h, std::max<int64_t>(total, 1));
}

void ensure_workspace(Handle *h, int64_t nrhs) {
    if (h->ws && h->ws_nrhs >= nrhs) return;
    if (h->ws) {
        dev_free(h, h->ws);
        h->ws = nullptr;
    }
    // x in tree order (FP64 and FP32 copies), w (FP64 and FP32) and u (FP64)
    const size_t bytes = (size_t)nrhs * ((h->n + 2 * h->npiv) * sizeof(double) + (h->n + h->npiv) * sizeof(float)) + 256;
    h->ws = dev_alloc(h, bytes);
    h->ws_bytes = bytes;
    h->ws_nrhs = nrhs;
}

// The passes of one group of NR right-hand sides (vectors right-hand-side major,
// NR rows of N or npiv).

// a14: x (caller order) into tree order (FP64 and, for the FP32 form, FP32);
// near_w: the float weights of the packed near-field pairs too (one right-hand side)
template <int NR, class TO>
void pass_perm(Handle *h, const TO *xin, int64_t ld, double *xt, float *xt32, bool near_w) {
    float *ppk_w = near_w ? reinterpret_cast<float *>(h->ppk) : nullptr;
    float *ppl_w = ppk_w ? reinterpret_cast<float *>(h->ppl) : nullptr;
    k_perm_in<TO><<<grid_for(h->n * NR, 256), 256, 0, h->stream>>>(xin, ld, h->n, NR, h->perm, xt, xt32, ppk_w, ppl_w,
                                                                 h->leaf_of, h->cbeg, h->ppk_off);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
}

// a8, a9: P2M on the leaves, then M2M level by level (FP64 operators); spk_w,
// spw: the float weights of the FP32 M2L's packed sources (one or M2L_RHS
// right-hand sides), or null
// groups: consecutive groups of NR right-hand sides served by the same launches
// (spk_w only with one group; the packed weights spw of group g at spw + g spw_stride)
template <int NR>
void pass_up(Handle *h, const double *xt, double *w, float *spk_w, float *spw, int groups = 1,
             int64_t spw_stride = 0) {
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv;
    const double *op = h->op;
    const int64_t lb = h->level_base[h->kappa], le = h->level_base[h->kappa + 1];
    NNCA_REQUIRE(groups >= 1 && (groups == 1 || (!spk_w && (!spw || spw_stride > 0))), NNCA_ERR_INTERNAL,
                 "pass_up: bad group count");
    k_upward<double, NR, 1><<<dim3(grid_for(le - lb, UP_THREADS / 32), groups), UP_THREADS, 0, s>>>(
        lb, le, 1, h->cbeg, h->cend, h->cch_beg, h->cch_end, h->piv_off, h->op_off, op, xt, N, w, npiv, spk_w,
        h->spk_off, spw, spw_stride);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
    for (int l = h->kappa - 1; l >= h->lmin; --l) {
        const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1];
        ++h->launches;
        k_upward<double, NR, UP_THREADS / 32><<<dim3(grid_for(b1 - b0, 1), groups), UP_THREADS, 0, s>>>(
            b0, b1, 0, h->cbeg, h->cend, h->cch_beg, h->cch_end, h->piv_off, h->op_off, op, xt, N, w, npiv, spk_w,
            h->spk_off, spw, spw_stride);
        NNCA_LAUNCH_CHECK();
    }
}

// a11: L2L, parents at level l - 1 push down to their children at level l
template <int NR>
void pass_l2l(Handle *h, double *u, int groups = 1) {
    for (int l = h->lmin + 1; l <= h->kappa; ++l) {
        const int64_t p0 = h->level_base[l - 1], p1 = h->level_base[l];
        ++h->launches;
        k_l2l<double, NR><<<dim3(grid_for(p1 - p0, 1), groups), UP_THREADS, 0, h->stream>>>(p0, p1, h->cch_beg, h->cch_end,
                                                                              h->piv_off, h->op_off, h->op, u,
                                                                              h->npiv);
        NNCA_LAUNCH_CHECK();
    }
}

// a12, a13: L2P fused with P2P, output in caller order
template <bool FP32, int NR, int KIND, class TO>
void pass_near(Handle *h, const double *u, const double *xt, const float *xt32, TO *yout, int64_t ld) {
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv;
    const double *op = h->op;
    if (!(FP32 && kernel_is_radial(h->kp.kind))) ++h->launches;
    const unsigned gl = grid_for(h->nleaf, MV_WARPS, 152 * 16);
    if (!kernel_is_radial(h->kp.kind)) {
        k_leaf_generic<NR, TO><<<grid_for(h->nleaf * 32, 128), 128, 0, s>>>(
            h->kp, h->d, h->leaf_order, h->nleaf, h->cbeg, h->cend, h->nb_off, h->nb_idx, h->piv_off, h->op_off, op, u,
            npiv, h->xs, N, xt, h->perm, yout, ld);
    } else if (FP32 && NR == 1) {
        launch_leaf_f32<KIND, TO>(h, op, u, xt32, xt, yout);
    } else if (FP32 && NR == M2L_RHS && h->near_packed && h->n_near_items4) {
        // the near field of the four right-hand sides in one pass
        launch_near_rhs<KIND, TO, M2L_RHS>(h, op, u, xt, yout, ld, h->pw4);
    } else if (FP32 && NR == 2 * M2L_RHS && h->near_packed && h->n_near_items4 && h->pw8) {
        // eight in one pass (tensor-core forms): each kernel value serves eight
        launch_near_rhs<KIND, TO, 2 * M2L_RHS>(h, op, u, xt, yout, ld, h->pw8);
    } else if (FP32) {
        // the near field one right-hand side at a time
        for (int r = 0; r < NR; ++r) {
            if (h->near_packed) {
                k_near_weights<<<grid_for(N, 256), 256, 0, s>>>(N, xt + r * N, reinterpret_cast<float *>(h->ppk),
                                                                reinterpret_cast<float *>(h->ppl), h->leaf_of, h->cbeg,
                                                                h->ppk_off);
                NNCA_LAUNCH_CHECK();
                ++h->launches;
            }
            launch_leaf_f32<KIND, TO>(h, op, u + r * npiv, xt32 + r * N, xt + r * N, yout + r * ld);
        }
    } else {
        k_leaf_f64<KIND, NR, TO><<<gl, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->leaf_order, h->nleaf, h->cbeg, h->cend,
                                                              h->nb_off, h->nb_idx, h->piv_off, h->op_off, op, u, npiv,
                                                              h->xs, N, xt, h->perm, yout, ld);
    }
    NNCA_LAUNCH_CHECK();
}

// One group of NR right-hand sides. FP32 == true selects FP32 kernel evaluations.
template <bool FP32, int NR, int KIND, class TO>
void run_chunk(Handle *h, const void *x, void *y, int64_t ld, int64_t r0) {
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv;
    double *xt = (double *)h->ws;
    double *w = xt + NR * N;
    double *u = w + NR * npiv;
    float *xt32 = FP32 ? (float *)(u + NR * npiv) : nullptr;
    // FP32: the weights go straight into the packed M2L sources (one right-hand
    // side) or into the packed weights of an M2L_RHS pass
    const bool f32 = FP32 && kernel_is_radial(h->kp.kind);
    float *spk_w = f32 && NR == 1 ? reinterpret_cast<float *>(h->spk) : nullptr;
    float *spw = f32 && NR == M2L_RHS ? reinterpret_cast<float *>(h->spw) : nullptr;
    const TO *xin = (const TO *)x + r0 * ld;
    TO *yout = (TO *)y + r0 * ld;
    prof_mark(h, 0);
    pass_perm<NR, TO>(h, xin, ld, xt, xt32, f32 && NR == 1 && h->near_packed);
    prof_mark(h, 1);
    if (npiv > 0) NNCA_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * NR * npiv, s));
    if (h->lmin <= h->kappa && npiv > 0) {
        pass_up<NR>(h, xt, w, spk_w, spw);
        prof_mark(h, 2);
        if (h->n_m2l_tgt > 0) {
            const unsigned g = grid_for(h->n_m2l_tgt, MV_WARPS, 152 * 16);
            if (!(FP32 && kernel_is_radial(h->kp.kind))) ++h->launches;
            if (!kernel_is_radial(h->kp.kind)) {
                k_m2l_generic<NR><<<grid_for(h->n_m2l_tgt * 32, 128), 128, 0, s>>>(
                    h->kp, h->d, h->m2l_tgt, h->n_m2l_tgt, h->il_off, h->il_idx, h->piv_off, h->pv64, npiv, w, u);
            } else if (FP32 && NR == 1 && h->sym_items) {
                launch_m2l_sym<KIND>(h, w, u);
            } else if (FP32 && NR == 1) {
                launch_m2l_f32<KIND>(h, u);
            } else if (FP32 && NR == M2L_RHS) {
                launch_m2l_f32_rhs<KIND>(h, u);
            } else if (NR == 1 && (h->f64_slot_of || !h->no_alloc)) {
                // FP64, one right-hand side: each admissible pair of cells evaluated once
                ensure_f64_sym(h);
                k_m2l_f64_sym<KIND><<<g, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->m2l_tgt, h->n_m2l_tgt, h->il_off,
                                                               h->il_idx, h->f64_slot_of, h->piv_off, h->pv64, npiv,
                                                               w, u, h->f64_slots);
                NNCA_LAUNCH_CHECK();
                k_m2l_f64_gather<<<g, 32 * MV_WARPS, 0, s>>>(h->m2l_tgt, h->n_m2l_tgt, h->il_off, h->il_idx,
                                                             h->f64_slot_of, h->piv_off, h->f64_slots, u);
                ++h->launches;
            } else {
                k_m2l_f64<KIND, NR><<<g, 32 * MV_WARPS, 0, s>>>(h->kp, h->d, h->m2l_tgt, h->n_m2l_tgt, h->il_off,
                                                                h->il_idx, h->piv_off, h->pv64, npiv, w, u);
            }
            NNCA_LAUNCH_CHECK();
        }
        prof_mark(h, 3);
        pass_l2l<NR>(h, u);
    } else {
        prof_mark(h, 2);
        prof_mark(h, 3);
    }
    prof_mark(h, 4);
    pass_near<FP32, NR, KIND, TO>(h, u, xt, xt32, yout, ld);
    prof_mark(h, 5);
}

// The tensor-core forms: passes of up to tc_rhs_per_pass() right-hand sides.
// Per pass: the permutation and the upward pass for all of its right-hand
// sides (groups of eight, FP64 operators: each operator load serves eight),
// one tensor-core M2L for all of them, then L2L (groups of eight) and the near
// field (the FP32 kernels, groups of M2L_RHS).
template <int KIND, class TO>
void run_tc(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld, int mode) {
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv;
    const int RW = tc_rhs_per_pass();
    double *xt = (double *)h->tc_ws;
    double *w = xt + (size_t)RW * N;
    double *u = w + (size_t)RW * npiv;
    float *xt32 = (float *)(u + (size_t)RW * npiv);
    float *tcws = xt32 + (size_t)RW * N;
    for (int64_t p0 = 0; p0 < nrhs; p0 += RW) {
        const int nr = (int)std::min<int64_t>(RW, nrhs - p0);
        const TO *xin = (const TO *)x + p0 * ld;
        TO *yout = (TO *)y + p0 * ld;
        prof_mark(h, 0);
        for (int r = 0; r < nr;) {
            if (nr - r >= M2L_RHS) {
                pass_perm<M2L_RHS, TO>(h, xin + r * ld, ld, xt + r * N, xt32 + r * N, false);
                r += M2L_RHS;
            } else {
                pass_perm<1, TO>(h, xin + r * ld, ld, xt + r * N, xt32 + r * N, false);
                r += 1;
            }
        }
        prof_mark(h, 1);
        const bool far = h->lmin <= h->kappa && npiv > 0;
        if (far) {
            for (int r = 0; r < nr;) {
                if (nr - r >= 2 * M2L_RHS) {
                    const int ng = (nr - r) / (2 * M2L_RHS);   // every group of eight in the same launches
                    pass_up<2 * M2L_RHS>(h, xt + r * N, w + r * npiv, nullptr, nullptr, ng);
                    r += ng * 2 * M2L_RHS;
                } else if (nr - r >= M2L_RHS) {
                    pass_up<M2L_RHS>(h, xt + r * N, w + r * npiv, nullptr, nullptr);
                    r += M2L_RHS;
                } else {
                    pass_up<1>(h, xt + r * N, w + r * npiv, nullptr, nullptr);
                    r += 1;
                }
            }
        }
        prof_mark(h, 2);
        if (far) m2l_tensor(h, mode, nr, w, u, tcws);
        else if (npiv > 0) NNCA_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * nr * npiv, s));
        prof_mark(h, 3);
        if (far)
            for (int r = 0; r < nr;) {
                if (nr - r >= 2 * M2L_RHS) {
                    const int ng = (nr - r) / (2 * M2L_RHS);
                    pass_l2l<2 * M2L_RHS>(h, u + r * npiv, ng);
                    r += ng * 2 * M2L_RHS;
                } else if (nr - r >= M2L_RHS) {
                    pass_l2l<M2L_RHS>(h, u + r * npiv);
                    r += M2L_RHS;
                } else {
                    pass_l2l<1>(h, u + r * npiv);
                    r += 1;
                }
            }
        prof_mark(h, 4);
        for (int r = 0; r < nr;) {
            if (nr - r >= 2 * M2L_RHS && h->pw8) {
                pass_near<true, 2 * M2L_RHS, KIND, TO>(h, u + r * npiv, xt + r * N, xt32 + r * N, yout + r * ld, ld);
                r += 2 * M2L_RHS;
            } else if (nr - r >= M2L_RHS) {
                pass_near<true, M2L_RHS, KIND, TO>(h, u + r * npiv, xt + r * N, xt32 + r * N, yout + r * ld, ld);
                r += M2L_RHS;
            } else {
                // one right-hand side: the near-field weights from its tree-order copy
                if (h->near_packed) {
                    k_near_weights<<<grid_for(N, 256), 256, 0, s>>>(N, xt + r * N, reinterpret_cast<float *>(h->ppk),
                                                                    reinterpret_cast<float *>(h->ppl), h->leaf_of,
                                                                    h->cbeg, h->ppk_off);
                    NNCA_LAUNCH_CHECK();
                    ++h->launches;
                }
                pass_near<true, 1, KIND, TO>(h, u + r * npiv, xt + r * N, xt32 + r * N, yout + r * ld, ld);
                r += 1;
            }
        }
        prof_mark(h, 5);
    }
}

void ensure_tc_workspace(Handle *h) {
    const size_t RW = (size_t)tc_rhs_per_pass();
    const size_t bytes = RW * ((size_t)h->n + 2 * (size_t)h->npiv) * sizeof(double) + RW * (size_t)h->n * sizeof(float) +
                         tc_workspace_floats(h) * sizeof(float) + 256;
    if (h->tc_ws && h->tc_ws_bytes >= bytes) return;
    if (h->tc_ws) dev_free(h, h->tc_ws);
    h->tc_ws = nullptr;
    h->tc_ws = dev_alloc(h, bytes);
    h->tc_ws_bytes = bytes;
    // the packed weights' padding must read as zero: clear once
    NNCA_CUDA(cudaMemsetAsync(h->tc_ws, 0, bytes, h->stream));
    if (!h->pw8 && h->near_packed && h->n_near_items4) {
        h->pw8 = dalloc<float4>(h, 4 * (size_t)h->near_pairs);
        NNCA_CUDA(cudaMemsetAsync(h->pw8, 0, 4 * (size_t)h->near_pairs * sizeof(float4), h->stream));
    }
}

// The FP32 form with ng groups of M2L_RHS right-hand sides (r0 .. r0 + 4 ng - 1):
// the permutation, P2M/M2M and L2L of every group in the same launches (grid y
// over the groups: the upper levels' few cells fill the GPU and each launch
// serves all groups), the M2L one launch per group (its packed weights per group
// in spw_multi), the near field in passes of eight right-hand sides where two
// groups remain.
template <int KIND, class TO>
void run_quads(Handle *h, const void *x, void *y, int64_t ld, int64_t r0, int ng) {
    cudaStream_t s = h->stream;
    const int64_t N = h->n, npiv = h->npiv, nrt = (int64_t)ng * M2L_RHS;
    double *xt = (double *)h->ws;
    double *w = xt + nrt * N;
    double *u = w + nrt * npiv;
    float *xt32 = (float *)(u + nrt * npiv);
    const TO *xin = (const TO *)x + r0 * ld;
    TO *yout = (TO *)y + r0 * ld;
    const int64_t sstride = 2 * M2L_RHS * h->n_spk_pairs;   // floats of one group's packed M2L weights
    float *spw = reinterpret_cast<float *>(h->spw_multi);
    prof_mark(h, 0);
    for (int g = 0; g < ng; ++g)
        pass_perm<M2L_RHS, TO>(h, xin + g * M2L_RHS * ld, ld, xt + g * M2L_RHS * N, xt32 + g * M2L_RHS * N, false);
    prof_mark(h, 1);
    if (npiv > 0) NNCA_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * nrt * npiv, s));
    const bool far = h->lmin <= h->kappa && npiv > 0;
    if (far) pass_up<M2L_RHS>(h, xt, w, nullptr, spw, ng, sstride);
    prof_mark(h, 2);
    if (far && h->n_m2l_tgt > 0)
        for (int g = 0; g < ng; ++g)
            launch_m2l_f32_rhs<KIND>(h, u + g * M2L_RHS * npiv, reinterpret_cast<const float4 *>(spw + g * sstride));
    prof_mark(h, 3);
    if (far) pass_l2l<M2L_RHS>(h, u, ng);
    prof_mark(h, 4);
    for (int g = 0; g < ng;) {
        const int64_t o = (int64_t)g * M2L_RHS;
        if (ng - g >= 2 && h->pw8) {
            pass_near<true, 2 * M2L_RHS, KIND, TO>(h, u + o * npiv, xt + o * N, xt32 + o * N, yout + o * ld, ld);
            g += 2;
        } else {
            pass_near<true, M2L_RHS, KIND, TO>(h, u + o * npiv, xt + o * N, xt32 + o * N, yout + o * ld, ld);
            g += 1;
        }
    }
    prof_mark(h, 5);
}

// buffers of the grouped FP32 passes: workspace rows, one set of packed M2L
// weights per group, and the near field's weights of eight right-hand sides
void ensure_quads(Handle *h, int ng) {
    ensure_workspace(h, (int64_t)ng * M2L_RHS);
    if (!h->spw_multi || h->spw_multi_groups < ng) {
        if (h->spw_multi) dev_free(h, h->spw_multi);
        h->spw_multi = nullptr;
        const size_t n4 = (size_t)ng * (M2L_RHS / 2) * (size_t)h->n_spk_pairs;
        h->spw_multi = dalloc<float4>(h, std::max<size_t>(n4, 1));
        // the padding sources' weights must read as zero
        NNCA_CUDA(cudaMemsetAsync(h->spw_multi, 0, std::max<size_t>(n4, 1) * sizeof(float4), h->stream));
        h->spw_multi_groups = ng;
    }
    if (!h->pw8 && h->near_packed && h->n_near_items4) {
        h->pw8 = dalloc<float4>(h, 4 * (size_t)h->near_pairs);
        NNCA_CUDA(cudaMemsetAsync(h->pw8, 0, 4 * (size_t)h->near_pairs * sizeof(float4), h->stream));
    }
}

constexpr int QUAD_GROUPS = 16;   // groups of M2L_RHS per grouped FP32 pass (64 right-hand sides)

template <bool FP32, int KIND, class TO>
void run_all(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld) {
    int64_t r0 = 0;
    if (FP32 && kernel_is_radial(h->kp.kind) && nrhs >= 2 * M2L_RHS && !h->no_alloc) {
        ensure_quads(h, (int)std::min<int64_t>(QUAD_GROUPS, nrhs / M2L_RHS));
        while (nrhs - r0 >= 2 * M2L_RHS) {
            const int ng = (int)std::min<int64_t>(QUAD_GROUPS, (nrhs - r0) / M2L_RHS);
            run_quads<KIND, TO>(h, x, y, ld, r0, ng);
            r0 += (int64_t)ng * M2L_RHS;
        }
    }
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

void set_wait_test(int64_t wait_limit_clocks, unsigned extra_tx_bytes) {
    const long long lim = wait_limit_clocks > 0 ? (long long)wait_limit_clocks : (1ll << 31);
    NNCA_CUDA(cudaMemcpyToSymbol(g_wait_limit, &lim, sizeof(lim)));
    NNCA_CUDA(cudaMemcpyToSymbol(g_stage_extra_tx, &extra_tx_bytes, sizeof(extra_tx_bytes)));
    NNCA_CUDA(cudaDeviceSynchronize());
}

// ---- batched products of independent problems (FP32 form) -------------------------
// Cross-problem item lists of the four-RHS M2L, one per kernel family and group
// of at most M2L_MULTI_MAX problems: (problem in the group, item) pairs, heaviest
// first over all the group's problems. Built on the first call with a set of
// handles and kept (a CUDA graph of the batched product refers to them).
struct CrossList {
    int kind = 0;
    std::vector<int> members;   // indices into the call's handle array
    int2 *gitems = nullptr;
    int nitems = 0;
    int *next = nullptr;
};
struct CrossPlan {
    std::vector<CrossList> lists;
};
std::mutex g_cross_mutex;
std::map<std::vector<uint64_t>, CrossPlan> g_cross_plans;

CrossPlan &cross_plan(Handle *const *hs, int count) {
    std::vector<uint64_t> key;
    for (int k = 0; k < count; ++k) {
        key.push_back(hs[k]->uid);
        key.push_back((uint64_t)(uintptr_t)hs[k]);
    }
    std::lock_guard<std::mutex> lock(g_cross_mutex);
    auto it = g_cross_plans.find(key);
    if (it != g_cross_plans.end()) return it->second;
    CrossPlan plan;
    std::map<int, std::vector<int>> by_kind;
    for (int k = 0; k < count; ++k)
        if (hs[k]->n_m2l_groups > 0) by_kind[hs[k]->kp.kind].push_back(k);
    for (auto &kv : by_kind)
        for (size_t g0 = 0; g0 < kv.second.size(); g0 += M2L_MULTI_MAX) {
            CrossList L;
            L.kind = kv.first;
            L.members.assign(kv.second.begin() + g0,
                             kv.second.begin() + std::min(kv.second.size(), g0 + (size_t)M2L_MULTI_MAX));
            std::vector<std::pair<int64_t, int2>> all;
            for (size_t m = 0; m < L.members.size(); ++m) {
                const Handle *h = hs[L.members[m]];
                for (int i = 0; i < h->n_m2l_groups; ++i)
                    all.push_back({i < (int)h->h_m2l_weight.size() ? h->h_m2l_weight[i] : 0, make_int2((int)m, i)});
            }
            std::stable_sort(all.begin(), all.end(), [](const std::pair<int64_t, int2> &a,
                                                        const std::pair<int64_t, int2> &b) { return a.first > b.first; });
            std::vector<int2> gi(all.size());
            for (size_t i = 0; i < all.size(); ++i) gi[i] = all[i].second;
            L.nitems = (int)gi.size();
            NNCA_CUDA(cudaMalloc(&L.gitems, sizeof(int2) * std::max<size_t>(1, gi.size())));
            NNCA_CUDA(cudaMalloc(&L.next, sizeof(int)));
            if (!gi.empty())
                NNCA_CUDA(cudaMemcpy(L.gitems, gi.data(), gi.size() * sizeof(int2), cudaMemcpyHostToDevice));
            plan.lists.push_back(L);
        }
    return g_cross_plans.emplace(key, std::move(plan)).first->second;
}

void release_cross_plans(uint64_t uid) {
    std::lock_guard<std::mutex> lock(g_cross_mutex);
    for (auto it = g_cross_plans.begin(); it != g_cross_plans.end();) {
        bool member = false;
        for (size_t i = 0; i < it->first.size(); i += 2) member |= it->first[i] == uid;
        if (!member) { ++it; continue; }
        for (CrossList &L : it->second.lists) {
            cudaFree(L.gitems);
            cudaFree(L.next);
        }
        it = g_cross_plans.erase(it);
    }
}

template <int KIND>
void launch_cross(Handle *const *hs, const CrossList &L, double *const *u, const float4 *const *spw, cudaStream_t s) {
    M2lRhsTable<M2L_MULTI_MAX> tab;
    for (size_t m = 0; m < L.members.size(); ++m) {
        tab.a[m] = m2l_rhs_args(hs[L.members[m]], u[L.members[m]]);
        tab.a[m].spw = spw[L.members[m]];
    }
    launch_m2l_rhs_table<KIND, M2L_MULTI_MAX>(tab, L.gitems, L.nitems, L.next, s);
}

template <class TO>
void near8_kind(Handle *h, const double *u, const double *xt, const float *xt32, TO *yout, int64_t ld) {
    switch (h->kp.kind) {
    case NNCA_K_INV_R: pass_near<true, 2 * M2L_RHS, NNCA_K_INV_R, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_LOG: pass_near<true, 2 * M2L_RHS, NNCA_K_LOG, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_GAUSS: pass_near<true, 2 * M2L_RHS, NNCA_K_GAUSS, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_MATERN: pass_near<true, 2 * M2L_RHS, NNCA_K_MATERN, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_PAPER_I: pass_near<true, 2 * M2L_RHS, NNCA_K_PAPER_I, TO>(h, u, xt, xt32, yout, ld); break;
    default: pass_near<true, 2 * M2L_RHS, NNCA_K_PAPER_II, TO>(h, u, xt, xt32, yout, ld); break;
    }
}

template <class TO>
void near4_kind(Handle *h, const double *u, const double *xt, const float *xt32, TO *yout, int64_t ld) {
    switch (h->kp.kind) {
    case NNCA_K_INV_R: pass_near<true, M2L_RHS, NNCA_K_INV_R, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_LOG: pass_near<true, M2L_RHS, NNCA_K_LOG, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_GAUSS: pass_near<true, M2L_RHS, NNCA_K_GAUSS, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_MATERN: pass_near<true, M2L_RHS, NNCA_K_MATERN, TO>(h, u, xt, xt32, yout, ld); break;
    case NNCA_K_PAPER_I: pass_near<true, M2L_RHS, NNCA_K_PAPER_I, TO>(h, u, xt, xt32, yout, ld); break;
    default: pass_near<true, M2L_RHS, NNCA_K_PAPER_II, TO>(h, u, xt, xt32, yout, ld); break;
    }
}

template <class TO>
void batch_fp32(Handle *const *hs, int count, const void *const *x, void *const *y, const int64_t *ld, int64_t nrhs,
                cudaStream_t s, cudaStream_t *wk, int nw, cudaEvent_t fork, cudaEvent_t *join) {
    auto fork_all = [&]() {
        NNCA_CUDA(cudaEventRecord(fork, s));
        for (int i = 0; i < nw; ++i) NNCA_CUDA(cudaStreamWaitEvent(wk[i], fork, 0));
    };
    auto join_all = [&]() {
        for (int i = 0; i < nw; ++i) {
            NNCA_CUDA(cudaEventRecord(join[i], wk[i]));
            NNCA_CUDA(cudaStreamWaitEvent(s, join[i], 0));
        }
    };
    // eight or more right-hand sides: passes of up to QUAD_GROUPS groups of four,
    // with P2M/M2M and L2L of all groups in the same launches, the near field in
    // groups of eight (as in the single product)
    const int ngq = (int)std::min<int64_t>(QUAD_GROUPS, nrhs / M2L_RHS);
    const bool grouped = ngq >= 2;
    for (int k = 0; k < count; ++k) {
        if (grouped) ensure_quads(hs[k], ngq);
        else ensure_workspace(hs[k], std::min<int64_t>(nrhs, 4));
        hs[k]->launches = 0;
    }
    CrossPlan &plan = cross_plan(hs, count);
    std::vector<double *> uptr(count), ug(count);
    std::vector<const float4 *> spwg(count);
    int64_t r0 = 0;
    while (r0 < nrhs) {
        if (nrhs - r0 < M2L_RHS) {
            // a last right-hand side: the products of one right-hand side, problem by problem
            fork_all();
            for (int k = 0; k < count; ++k) {
                Handle *h = hs[k];
                h->stream = wk[k % nw];
                switch (h->kp.kind) {
                case NNCA_K_INV_R: run_chunk<true, 1, NNCA_K_INV_R, TO>(h, x[k], y[k], ld[k], r0); break;
                case NNCA_K_LOG: run_chunk<true, 1, NNCA_K_LOG, TO>(h, x[k], y[k], ld[k], r0); break;
                case NNCA_K_GAUSS: run_chunk<true, 1, NNCA_K_GAUSS, TO>(h, x[k], y[k], ld[k], r0); break;
                case NNCA_K_MATERN: run_chunk<true, 1, NNCA_K_MATERN, TO>(h, x[k], y[k], ld[k], r0); break;
                case NNCA_K_PAPER_I: run_chunk<true, 1, NNCA_K_PAPER_I, TO>(h, x[k], y[k], ld[k], r0); break;
                default: run_chunk<true, 1, NNCA_K_PAPER_II, TO>(h, x[k], y[k], ld[k], r0); break;
                }
            }
            join_all();
            r0 += 1;
            continue;
        }
        const int ng = grouped && nrhs - r0 >= 2 * M2L_RHS ? (int)std::min<int64_t>(ngq, (nrhs - r0) / M2L_RHS) : 1;
        const int64_t nrt = (int64_t)ng * M2L_RHS;
        // permutation, P2M and M2M of every problem
        fork_all();
        for (int k = 0; k < count; ++k) {
            Handle *h = hs[k];
            h->stream = wk[k % nw];
            const int64_t N = h->n, npiv = h->npiv;
            double *xt = (double *)h->ws, *w = xt + nrt * N, *u = w + nrt * npiv;
            float *xt32 = (float *)(u + nrt * npiv);
            uptr[k] = u;
            const TO *xin = (const TO *)x[k] + r0 * ld[k];
            for (int g = 0; g < ng; ++g)
                pass_perm<M2L_RHS, TO>(h, xin + g * M2L_RHS * ld[k], ld[k], xt + g * M2L_RHS * N, xt32 + g * M2L_RHS * N,
                                       false);
            if (npiv > 0) NNCA_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * nrt * npiv, h->stream));
            if (h->lmin <= h->kappa && npiv > 0) {
                if (ng > 1)
                    pass_up<M2L_RHS>(h, xt, w, nullptr, reinterpret_cast<float *>(h->spw_multi), ng,
                                     2 * M2L_RHS * h->n_spk_pairs);
                else
                    pass_up<M2L_RHS>(h, xt, w, nullptr, reinterpret_cast<float *>(h->spw));
            }
        }
        join_all();
        // the M2L of all problems, group by group: one launch per kernel family over
        // the cross-problem list, then the split pieces' combine of that group
        for (int g = 0; g < ng; ++g) {
            for (int k = 0; k < count; ++k) {
                ug[k] = uptr[k] + (int64_t)g * M2L_RHS * hs[k]->npiv;
                spwg[k] = ng > 1 ? hs[k]->spw_multi + (size_t)g * (M2L_RHS / 2) * (size_t)hs[k]->n_spk_pairs : hs[k]->spw;
            }
            for (const CrossList &L : plan.lists) {
                switch (L.kind) {
                case NNCA_K_INV_R: launch_cross<NNCA_K_INV_R>(hs, L, ug.data(), spwg.data(), s); break;
                case NNCA_K_LOG: launch_cross<NNCA_K_LOG>(hs, L, ug.data(), spwg.data(), s); break;
                case NNCA_K_GAUSS: launch_cross<NNCA_K_GAUSS>(hs, L, ug.data(), spwg.data(), s); break;
                case NNCA_K_MATERN: launch_cross<NNCA_K_MATERN>(hs, L, ug.data(), spwg.data(), s); break;
                case NNCA_K_PAPER_I: launch_cross<NNCA_K_PAPER_I>(hs, L, ug.data(), spwg.data(), s); break;
                default: launch_cross<NNCA_K_PAPER_II>(hs, L, ug.data(), spwg.data(), s); break;
                }
                ++hs[L.members[0]]->launches;
            }
            for (int k = 0; k < count; ++k) {
                Handle *h = hs[k];
                if (h->lmin <= h->kappa && h->npiv > 0) {
                    h->stream = s;
                    m2l_rhs_combine(h, ug[k]);
                }
            }
        }
        // L2L and the near field of every problem
        fork_all();
        for (int k = 0; k < count; ++k) {
            Handle *h = hs[k];
            h->stream = wk[k % nw];
            const int64_t N = h->n, npiv = h->npiv;
            double *xt = (double *)h->ws, *u = uptr[k];
            float *xt32 = (float *)(u + nrt * npiv);
            TO *yout = (TO *)y[k] + r0 * ld[k];
            if (h->lmin <= h->kappa && npiv > 0) pass_l2l<M2L_RHS>(h, u, ng);
            for (int g = 0; g < ng;) {
                const int64_t o = (int64_t)g * M2L_RHS;
                if (ng - g >= 2 && h->pw8) {
                    near8_kind<TO>(h, u + o * npiv, xt + o * N, xt32 + o * N, yout + o * ld[k], ld[k]);
                    g += 2;
                } else {
                    near4_kind<TO>(h, u + o * npiv, xt + o * N, xt32 + o * N, yout + o * ld[k], ld[k]);
                    g += 1;
                }
            }
        }
        join_all();
        r0 += nrt;
    }
}

template <class TO>
void dispatch_tc(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld, int mode) {
    switch (h->kp.kind) {
    case NNCA_K_INV_R: run_tc<NNCA_K_INV_R, TO>(h, x, y, nrhs, ld, mode); break;
    case NNCA_K_LOG: run_tc<NNCA_K_LOG, TO>(h, x, y, nrhs, ld, mode); break;
    case NNCA_K_GAUSS: run_tc<NNCA_K_GAUSS, TO>(h, x, y, nrhs, ld, mode); break;
    case NNCA_K_MATERN: run_tc<NNCA_K_MATERN, TO>(h, x, y, nrhs, ld, mode); break;
    case NNCA_K_PAPER_I: run_tc<NNCA_K_PAPER_I, TO>(h, x, y, nrhs, ld, mode); break;
    case NNCA_K_PAPER_II: run_tc<NNCA_K_PAPER_II, TO>(h, x, y, nrhs, ld, mode); break;
    default: NNCA_REQUIRE(false, NNCA_ERR_UNSUPPORTED, "the tensor-core forms need a radial kernel");
    }
}

bool matvec_batch_fp32(Handle *const *hs, int count, const void *const *x, void *const *y, const int64_t *ld,
                       int64_t nrhs, int dtype, cudaStream_t s, cudaStream_t *workers, int nworkers, cudaEvent_t fork,
                       cudaEvent_t *join) {
    if (nrhs < M2L_RHS) return false;
    for (int k = 0; k < count; ++k) {
        const Handle *h = hs[k];
        if (!kernel_is_radial(h->kp.kind) || h->d > 3 || h->m2l_fp32_unsupported) return false;
    }
    if (dtype == NNCA_F64) batch_fp32<double>(hs, count, x, y, ld, nrhs, s, workers, nworkers, fork, join);
    else batch_fp32<float>(hs, count, x, y, ld, nrhs, s, workers, nworkers, fork, join);
    return true;
}

void matvec(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld, int dtype, int precision) {
    const bool radial = kernel_is_radial(h->kp.kind);
    NNCA_REQUIRE(radial || precision == NNCA_PREC_FP64, NNCA_ERR_UNSUPPORTED,
                 "non-radial kernels support only the FP64 product");
    NNCA_REQUIRE(h->d <= 3 || precision == NNCA_PREC_FP64, NNCA_ERR_UNSUPPORTED,
                 "the FP32 product supports d <= 3");
    NNCA_REQUIRE(!h->m2l_fp32_unsupported || precision == NNCA_PREC_FP64, NNCA_ERR_UNSUPPORTED,
                 h->m2l_fp32_unsupported ? h->m2l_fp32_unsupported : "");
    const bool tc = precision == NNCA_PREC_TF32X3 || precision == NNCA_PREC_TF32 || precision == NNCA_PREC_BF16;
    if (tc) {
        ensure_tc_workspace(h);
        h->launches = 0;
        if (dtype == NNCA_F64) dispatch_tc<double>(h, x, y, nrhs, ld, precision);
        else dispatch_tc<float>(h, x, y, nrhs, ld, precision);
        return;
    }
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
