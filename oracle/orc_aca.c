/*
 * Partially pivoted ACA and the pivot-submatrix solve (oracle; test
 * infrastructure only).
 *
 * ACA (Sec. 2.2.1, Eqs. 3-4; the paper uses the partially pivoted ACA of
 * Rjasanow 2002 and fixes only the stopping rule). An m x n block A is
 * approximated by crosses, A ~ A^(k) = sum_{l<k} u_l v_l^T, with row pivots
 * i_l and column pivots j_l. The paper leaves the details open; the reading:
 *
 *  1. Start at row 0. Rows and columns are in candidate-set order.
 *  2. Residual row: r_j = A(i, j) - sum_{l<k} u_l(i) v_l(j), the sum taken in
 *     ascending l as r_j <- fma(-u_l(i), v_l(j), r_j).
 *  3. Column pivot j* = argmax over unused columns of |r_j|, ties to the
 *     smallest j. If that maximum is 0, or at round-off level (at most 2^-44
 *     times the row's largest entry max_j |A(i, j)|), the row carries nothing
 *     new: it is marked used, the smallest unused row is taken next, and no
 *     cross is formed. (A row that repeats a pivot row, as for two points at
 *     the same location, has a residual of a few units in the last place;
 *     taking it as a pivot would make the pivot block A_{tau sigma} of Eqs. 11
 *     and 14 singular.)
 *  4. v = r * (1 / r_{j*});  u(i') = A(i', j*) - sum_{l<k} v_l(j*) u_l(i')
 *     (ascending l, fused as in 2).
 *  5. ||A^(k+1)||_F^2 = ||A^(k)||_F^2 + 2 sum_{l<k} (u_l.u)(v_l.v) + |u|^2 |v|^2,
 *     the cross terms summed in ascending l with fma, then
 *     f2 <- f2 + 2*cross, f2 <- f2 + |u|^2*|v|^2.
 *  6. Stopping rule (Eq. 4): stop when |u|_2 |v|_2 <= eps ||A^(k+1)||_F,
 *     evaluated as sqrt(|u|^2) * sqrt(|v|^2) <= eps * sqrt(f2). The cross that
 *     meets the rule is NOT kept: it is negligible at tolerance eps, so the
 *     rank is the smallest that meets the rule, and a block of exact rank r
 *     gets exactly r pivots (keeping it would add a pure round-off (r+1)-th).
 *  7. Otherwise the cross is kept (pivots (i, j*)), and the iteration stops
 *     when k = min(m, n) or no unused row is left; the next row is the argmax
 *     over unused rows of |u(i')|, ties to the smallest i'.
 *
 * Every dot product and norm uses orc_cdot: element j is accumulated (with
 * fma) into partial j mod 256 in ascending j, and the 256 partials are folded
 * pairwise, p[t] += p[t + o] for o = 128, 64, ..., 1. The paper fixes no
 * summation order; a fixed one makes the pivots reproducible bit for bit.
 *
 * Pivot-submatrix solve (Sec. 2.3.1, Eq. 11 and Eq. 14): the bases are
 * X = A_{t~ sigma} (A_{tau sigma})^{-1}, computed from X M = B as
 * M^T X^T = B^T by LU with partial pivoting of M^T (pivot = largest |entry|
 * in the column, ties to the smallest row; right-looking updates
 * a_ij <- fma(-l_ic, u_cj, a_ij)), forward substitution in ascending j and
 * back substitution in ascending j, each with fma, then one division by the
 * diagonal.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#include "orc_internal.h"

#define NPART 256

double orc_cdot(const double *a, const double *b, long n) {
    double p[NPART];
    for (int t = 0; t < NPART; ++t) p[t] = 0.0;
    for (long j = 0; j < n; ++j) p[j % NPART] = fma(a[j], b[j], p[j % NPART]);
    for (int o = NPART / 2; o >= 1; o /= 2)
        for (int t = 0; t < o; ++t) p[t] = p[t] + p[t + o];
    return p[0];
}

long orc_aca(long m, long n, orc_entry_fn entry, const void *ctx, double eps,
             long *prow, long *pcol, double *Uout, double *Vout) {
    if (m <= 0 || n <= 0) return 0;
    const long kmax = m < n ? m : n;
    double *U = (double *)calloc((size_t)(m * kmax), sizeof(double));
    double *V = (double *)calloc((size_t)(n * kmax), sizeof(double));
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    char *urow = (char *)calloc((size_t)m, 1);
    char *ucol = (char *)calloc((size_t)n, 1);
    double frob2 = 0.0;
    long k = 0, i = 0;
    for (;;) {
        /* 2. residual of row i (and the row's largest entry) */
        double amax = 0.0;
        for (long j = 0; j < n; ++j) {
            double s = entry(ctx, i, j);
            if (fabs(s) > amax) amax = fabs(s);
            for (long l = 0; l < k; ++l) s = fma(-U[l * m + i], V[l * n + j], s);
            r[j] = s;
        }
        /* 3. column pivot */
        long jp = -1;
        double best = -1.0;
        for (long j = 0; j < n; ++j)
            if (!ucol[j] && fabs(r[j]) > best) { best = fabs(r[j]); jp = j; }
        if (jp < 0 || best <= ldexp(amax, -44)) {
            urow[i] = 1;
            long nxt = -1;
            for (long t = 0; t < m; ++t) if (!urow[t]) { nxt = t; break; }
            if (nxt < 0) break;
            i = nxt;
            continue;
        }
        /* 4. the new cross */
        double *v = V + k * n, *u = U + k * m;
        const double inv = 1.0 / r[jp];
        for (long j = 0; j < n; ++j) v[j] = r[j] * inv;
        for (long t = 0; t < m; ++t) {
            double s = entry(ctx, t, jp);
            for (long l = 0; l < k; ++l) s = fma(-V[l * n + jp], U[l * m + t], s);
            u[t] = s;
        }
        /* 5. Frobenius norm of the approximation including the new cross */
        const double nu2 = orc_cdot(u, u, m);
        const double nv2 = orc_cdot(v, v, n);
        double cross = 0.0;
        for (long l = 0; l < k; ++l)
            cross = fma(orc_cdot(U + l * m, u, m), orc_cdot(V + l * n, v, n), cross);
        double f2 = frob2 + 2.0 * cross;
        f2 = f2 + nu2 * nv2;
        /* 6. stopping rule: the negligible cross is not kept */
        if (sqrt(nu2) * sqrt(nv2) <= eps * sqrt(f2)) break;
        /* 7. keep it */
        urow[i] = 1;
        ucol[jp] = 1;
        prow[k] = i;
        pcol[k] = jp;
        frob2 = f2;
        ++k;
        if (k == kmax) break;
        long ip = -1;
        best = -1.0;
        for (long t = 0; t < m; ++t)
            if (!urow[t] && fabs(u[t]) > best) { best = fabs(u[t]); ip = t; }
        if (ip < 0) break;
        i = ip;
    }
    if (Uout) memcpy(Uout, U, sizeof(double) * (size_t)(m * kmax));
    if (Vout) memcpy(Vout, V, sizeof(double) * (size_t)(n * kmax));
    free(U); free(V); free(r); free(urow); free(ucol);
    return k;
}

typedef struct { const double *A; long lda; } dense_ctx;
static double dense_entry(const void *ctx, long i, long j) {
    const dense_ctx *c = (const dense_ctx *)ctx;
    return c->A[i * c->lda + j];
}

long orc_aca_dense(const double *A, long m, long n, long lda, double eps,
                   long *prow, long *pcol, double *U, double *V) {
    dense_ctx c = {A, lda};
    return orc_aca(m, n, dense_entry, &c, eps, prow, pcol, U, V);
}

int orc_solve_right(const double *M, long r, const double *B, long m, double *X) {
    /* T = M^T, factor in place: T = P^T L U */
    double *T = (double *)malloc(sizeof(double) * (size_t)(r * r > 0 ? r * r : 1));
    long *piv = (long *)malloc(sizeof(long) * (size_t)(r > 0 ? r : 1));
    double *b = (double *)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    int status = 0;
    for (long a = 0; a < r; ++a)
        for (long c = 0; c < r; ++c) T[a * r + c] = M[c * r + a];
    for (long c = 0; c < r; ++c) {
        long p = c;
        double best = fabs(T[c * r + c]);
        for (long a = c + 1; a < r; ++a)
            if (fabs(T[a * r + c]) > best) { best = fabs(T[a * r + c]); p = a; }
        piv[c] = p;
        if (p != c)
            for (long j = 0; j < r; ++j) { double t = T[c * r + j]; T[c * r + j] = T[p * r + j]; T[p * r + j] = t; }
        if (T[c * r + c] == 0.0) status = -1;
        for (long a = c + 1; a < r; ++a) T[a * r + c] = T[a * r + c] / T[c * r + c];
        for (long a = c + 1; a < r; ++a)
            for (long j = c + 1; j < r; ++j) T[a * r + j] = fma(-T[a * r + c], T[c * r + j], T[a * r + j]);
    }
    for (long row = 0; row < m; ++row) {
        for (long a = 0; a < r; ++a) b[a] = B[row * r + a];
        for (long c = 0; c < r; ++c)
            if (piv[c] != c) { double t = b[c]; b[c] = b[piv[c]]; b[piv[c]] = t; }
        for (long a = 0; a < r; ++a) {
            double s = b[a];
            for (long j = 0; j < a; ++j) s = fma(-T[a * r + j], b[j], s);
            b[a] = s;
        }
        for (long a = r - 1; a >= 0; --a) {
            double s = b[a];
            for (long j = a + 1; j < r; ++j) s = fma(-T[a * r + j], b[j], s);
            b[a] = s / T[a * r + a];
        }
        for (long a = 0; a < r; ++a) X[row * r + a] = b[a];
    }
    free(T); free(piv); free(b);
    return status;
}
