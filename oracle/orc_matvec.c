/*
 * H^2 matrix-vector product and dense product (oracle; test infrastructure
 * only).
 *
 * H^2 representation (Sec. 3): the bases and translations of every cell, the
 * couplings S_{X,Y} = A_{t^{X,i} s^{Y,o}} for Y in IL(X) (with the symmetric
 * shortcut s^{Y,o} = t^{Y,i}), and the near blocks A_{t^X s^Y} for leaves X
 * and Y in N(X). orc_assemble stores them (form 1); form 0 evaluates the same
 * entries on the fly instead. Both run the same loops in the same order.
 *
 * H^2 product u = A w (Sec. 4, steps 2-5), with the symmetric shortcut
 * V_B = U_B, T_{B B_c} = C_{B_c B}^T:
 *   2. upward pass:  leaf w^{B,o} = U_B^T w^B;
 *                    non-leaf w^{B,o} = sum_c C_{B_c B}^T w^{B_c,o}, levels
 *                    kappa-1 down to the first level with pivots;
 *   3. transverse:   u^{B,i} = sum_{B' in IL(B)} S_{B B'} w^{B',o}, all levels;
 *   4. downward:     u^{B_c,i} += C_{B_c B} u^{B,i}, levels top-down;
 *                    leaf u^B = U_B u^{B,i};
 *   5. near field:   u^B += sum_{B' in N(B)} A_{t^B s^{B'}} w^{B'}.
 * The paper writes the M2M step with T^T_{B B'}; with T_{B B_c} of Eq. 14
 * (r_B x r_{B_c}) the product that has the right shape, and that equals
 * V_B^T w^B through the nested form of V_B, is T_{B B_c} w^{B_c,o}. Every
 * sum runs in ascending index order.
 *
 * Dense product (Eq. 19): y_i = sum_j K(p_i, p_j) x_j with the diagonal value
 * for j == i, summed in ascending j.
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#include "orc_internal.h"

int orc_assemble(orc_h2 *h) {
    const long nil = h->il_off[h->ncell], nnb = h->nb_off[h->ncell];
    free(h->s_off); free(h->s_blk); free(h->near_off); free(h->near_blk);
    h->s_off = (long *)calloc((size_t)nil + 1, sizeof(long));
    h->near_off = (long *)calloc((size_t)nnb + 1, sizeof(long));
    for (long X = 0; X < h->ncell; ++X) {
        long rX = h->piv_off[X + 1] - h->piv_off[X];
        for (long q = h->il_off[X]; q < h->il_off[X + 1]; ++q) {
            long Y = h->il_idx[q];
            h->s_off[q + 1] = rX * (h->piv_off[Y + 1] - h->piv_off[Y]);
        }
        long nX = h->cend[X] - h->cbeg[X];
        int leaf = (orc_level_of(h, X) == h->kappa);
        for (long q = h->nb_off[X]; q < h->nb_off[X + 1]; ++q) {
            long Y = h->nb_idx[q];
            h->near_off[q + 1] = leaf ? nX * (h->cend[Y] - h->cbeg[Y]) : 0;
        }
    }
    for (long q = 0; q < nil; ++q) h->s_off[q + 1] += h->s_off[q];
    for (long q = 0; q < nnb; ++q) h->near_off[q + 1] += h->near_off[q];
    h->s_blk = (double *)malloc(sizeof(double) * (size_t)(h->s_off[nil] > 0 ? h->s_off[nil] : 1));
    h->near_blk = (double *)malloc(sizeof(double) * (size_t)(h->near_off[nnb] > 0 ? h->near_off[nnb] : 1));
    for (long X = 0; X < h->ncell; ++X) {
        const long *tX = h->piv_row + h->piv_off[X];
        long rX = h->piv_off[X + 1] - h->piv_off[X];
        for (long q = h->il_off[X]; q < h->il_off[X + 1]; ++q) {
            long Y = h->il_idx[q];
            const long *tY = h->piv_row + h->piv_off[Y];
            long rY = h->piv_off[Y + 1] - h->piv_off[Y];
            double *S = h->s_blk + h->s_off[q];
            for (long a = 0; a < rX; ++a)
                for (long b = 0; b < rY; ++b) S[a * rY + b] = orc_entry(h, tX[a], tY[b]);
        }
        if (orc_level_of(h, X) != h->kappa) continue;
        for (long q = h->nb_off[X]; q < h->nb_off[X + 1]; ++q) {
            long Y = h->nb_idx[q];
            long nY = h->cend[Y] - h->cbeg[Y];
            double *Nb = h->near_blk + h->near_off[q];
            for (long a = h->cbeg[X]; a < h->cend[X]; ++a)
                for (long b = h->cbeg[Y]; b < h->cend[Y]; ++b)
                    Nb[(a - h->cbeg[X]) * nY + (b - h->cbeg[Y])] = orc_entry(h, a, b);
        }
    }
    return 0;
}

int orc_h2_matvec(const orc_h2 *h, const double *x, double *y, long nrhs, long ld, int form, int nthreads) {
    /* nthreads > 0: that many threads; each output is summed by one thread in a
     * fixed order, so the result does not depend on it */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
    if (form < 0 || form > 2 || (form == 1 && !h->s_blk)) return -1;
    const long n = h->n, nc = h->ncell, npiv = h->piv_off[nc];
    double *xs = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *ys = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)(npiv > 0 ? npiv : 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)(npiv > 0 ? npiv : 1));
    for (long rhs = 0; rhs < nrhs; ++rhs) {
        /* step 1 (ordering): the vector in tree order */
        for (long i = 0; i < n; ++i) xs[i] = x[rhs * ld + h->perm[i]];
        for (long t = 0; t < npiv; ++t) { w[t] = 0.0; u[t] = 0.0; }
        /* step 2: upward pass */
        for (int l = h->kappa; l >= h->lmin; --l) {
            #pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
            for (long B = h->level_base[l]; B < h->level_base[l + 1]; ++B) {
                const long r = h->piv_off[B + 1] - h->piv_off[B];
                const double *op = h->op + h->op_off[B];
                double *wB = w + h->piv_off[B];
                if (l == h->kappa) {
                    const long m = h->cend[B] - h->cbeg[B];
                    for (long b = 0; b < r; ++b) {
                        double s = 0.0;
                        for (long a = 0; a < m; ++a) s = s + op[a * r + b] * xs[h->cbeg[B] + a];
                        wB[b] = s;
                    }
                } else {
                    /* children's w^{B_c,o} are contiguous, in the order of the stacked C */
                    const long c0 = h->cch_beg[B];
                    const double *wc = w + h->piv_off[c0];
                    const long m = h->piv_off[h->cch_end[B]] - h->piv_off[c0];
                    for (long b = 0; b < r; ++b) {
                        double s = 0.0;
                        for (long a = 0; a < m; ++a) s = s + op[a * r + b] * wc[a];
                        wB[b] = s;
                    }
                }
            }
        }
        /* step 3: transverse pass */
        const long x0 = h->level_base[h->lmin <= h->kappa ? h->lmin : h->kappa + 1];
        if (form == 2) {
            /* each admissible pair once: S w^Y into u^X, S^T w^X into u^Y */
            for (long X = x0; X < nc; ++X) {
                const long *tX = h->piv_row + h->piv_off[X];
                const long rX = h->piv_off[X + 1] - h->piv_off[X];
                const double *wX = w + h->piv_off[X];
                double *uX = u + h->piv_off[X];
                for (long q = h->il_off[X]; q < h->il_off[X + 1]; ++q) {
                    const long Y = h->il_idx[q];
                    if (Y <= X) continue;
                    const long *tY = h->piv_row + h->piv_off[Y];
                    const long rY = h->piv_off[Y + 1] - h->piv_off[Y];
                    const double *wY = w + h->piv_off[Y];
                    double *uY = u + h->piv_off[Y];
                    for (long a = 0; a < rX; ++a)
                        for (long b = 0; b < rY; ++b) {
                            const double k = orc_entry(h, tX[a], tY[b]);
                            uX[a] = uX[a] + k * wY[b];
                            uY[b] = uY[b] + k * wX[a];
                        }
                }
            }
        } else {
        #pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
        for (long X = x0; X < nc; ++X) {
            const long *tX = h->piv_row + h->piv_off[X];
            const long rX = h->piv_off[X + 1] - h->piv_off[X];
            double *uX = u + h->piv_off[X];
            for (long a = 0; a < rX; ++a) {
                double s = 0.0;
                for (long q = h->il_off[X]; q < h->il_off[X + 1]; ++q) {
                    const long Y = h->il_idx[q];
                    const long *tY = h->piv_row + h->piv_off[Y];
                    const long rY = h->piv_off[Y + 1] - h->piv_off[Y];
                    const double *wY = w + h->piv_off[Y];
                    const double *S = (form == 1) ? h->s_blk + h->s_off[q] + a * rY : NULL;
                    for (long b = 0; b < rY; ++b) {
                        double k = S ? S[b] : orc_entry(h, tX[a], tY[b]);
                        s = s + k * wY[b];
                    }
                }
                uX[a] = s;
            }
        }
        }
        /* step 4: downward pass, levels top-down, then leaves */
        for (int l = h->lmin + 1; l <= h->kappa; ++l) {
            #pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
            for (long B = h->level_base[l]; B < h->level_base[l + 1]; ++B) {
                const long P = h->cpar[B];
                const long rP = h->piv_off[P + 1] - h->piv_off[P];
                const long rB = h->piv_off[B + 1] - h->piv_off[B];
                /* the rows of P's stacked C that belong to child B */
                const long row0 = h->piv_off[B] - h->piv_off[h->cch_beg[P]];
                const double *C = h->op + h->op_off[P] + row0 * rP;
                const double *uP = u + h->piv_off[P];
                double *uB = u + h->piv_off[B];
                for (long a = 0; a < rB; ++a) {
                    double s = 0.0;
                    for (long b = 0; b < rP; ++b) s = s + C[a * rP + b] * uP[b];
                    uB[a] = uB[a] + s;
                }
            }
        }
        for (long i = 0; i < n; ++i) ys[i] = 0.0;
        if (h->lmin <= h->kappa) {
            #pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
            for (long B = h->level_base[h->kappa]; B < h->level_base[h->kappa + 1]; ++B) {
                const long r = h->piv_off[B + 1] - h->piv_off[B];
                const double *op = h->op + h->op_off[B];
                const double *uB = u + h->piv_off[B];
                for (long a = h->cbeg[B]; a < h->cend[B]; ++a) {
                    double s = 0.0;
                    for (long b = 0; b < r; ++b) s = s + op[(a - h->cbeg[B]) * r + b] * uB[b];
                    ys[a] = s;
                }
            }
        }
        /* step 5: near field */
        #pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
        for (long X = h->level_base[h->kappa]; X < h->level_base[h->kappa + 1]; ++X) {
            for (long a = h->cbeg[X]; a < h->cend[X]; ++a) {
                double s = 0.0;
                for (long q = h->nb_off[X]; q < h->nb_off[X + 1]; ++q) {
                    const long Y = h->nb_idx[q];
                    const long nY = h->cend[Y] - h->cbeg[Y];
                    const double *Nb = (form == 1) ? h->near_blk + h->near_off[q] + (a - h->cbeg[X]) * nY : NULL;
                    for (long b = h->cbeg[Y]; b < h->cend[Y]; ++b) {
                        double k = Nb ? Nb[b - h->cbeg[Y]] : orc_entry(h, a, b);
                        s = s + k * xs[b];
                    }
                }
                ys[a] = ys[a] + s;
            }
        }
        for (long i = 0; i < n; ++i) y[rhs * ld + h->perm[i]] = ys[i];
    }
    free(xs); free(ys); free(w); free(u);
    return 0;
}

static double dense_row(const orc_config *cfg, const double *P, long n, long i, const double *x) {
    double s = 0.0;
    for (long j = 0; j < n; ++j) {
        double k = (j == i) ? cfg->kparam[2] : orc_kernel(cfg, P + i * cfg->d, P + j * cfg->d);
        s = s + k * x[j];
    }
    return s;
}

void orc_dense_matvec(const orc_config *cfg, const double *P, long n, const double *x, double *y,
                      long nrhs, long ld, int nthreads) {
    (void)nthreads;
    for (long rhs = 0; rhs < nrhs; ++rhs) {
        #pragma omp parallel for schedule(dynamic, 64)
        for (long i = 0; i < n; ++i) y[rhs * ld + i] = dense_row(cfg, P, n, i, x + rhs * ld);
    }
}

void orc_dense_rows(const orc_config *cfg, const double *P, long n, const long *rows, long nrows,
                    const double *x, double *y, long nrhs, long ld, int nthreads) {
    (void)nthreads;
    for (long rhs = 0; rhs < nrhs; ++rhs) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (long q = 0; q < nrows; ++q) y[rhs * nrows + q] = dense_row(cfg, P, n, rows[q], x + rhs * ld);
    }
}
