/*
 * Kernel functions K(x, y) = K(r), r = |x - y|_2 (oracle; test infrastructure only).
 *
 * The paper's matrix has entries A(i, j) = K(p_i, q_j) with K smooth away from
 * x = y (Sec. 1). The experiments use radial kernels (Sec. 5): kernels (i) and
 * (ii) of Sec. 5.1 with a = 1e-4, 1/r (Sec. 5.3-5.5), and the Gaussian and
 * Matern-type kernels of the SVM experiment (Sec. 5.6). log r, s/r and the
 * Gaussian with bandwidth h are the kernels of the benchmark workloads.
 *
 * K is singular (or undefined) at r = 0 for the log and 1/r kernels. The
 * diagonal A(i, i) is decided by index and takes the configured value
 * kparam[2]; two distinct points that coincide (r == 0) give 0 for the
 * singular kernels and K(0) for the smooth ones.
 *
 * r^2 is summed in coordinate order, each product and sum rounded on its own.
 */
#include <math.h>
#include "oracle.h"

static double r2_of(int d, const double *x, const double *y) {
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = x[k] - y[k];
        r2 = r2 + t * t;
    }
    return r2;
}

double orc_kernel(const orc_config *cfg, const double *x, const double *y) {
    const double s = cfg->kparam[0];
    const double h = cfg->kparam[1];
    const int d = cfg->d;
    switch (cfg->kernel) {
    case ORC_K_LOG: {
        double r2 = r2_of(d, x, y);
        if (r2 == 0.0) return 0.0;
        return s * log(sqrt(r2));
    }
    case ORC_K_INV_R: {
        double r2 = r2_of(d, x, y);
        if (r2 == 0.0) return 0.0;
        return s / sqrt(r2);
    }
    case ORC_K_GAUSS: {
        double r2 = r2_of(d, x, y);
        return s * exp(-r2 / (2.0 * h * h));
    }
    case ORC_K_MATERN: {
        double r2 = r2_of(d, x, y);
        return s * exp(-sqrt(r2) / h);
    }
    case ORC_K_PAPER_I: {
        /* (r (log r - 1)) / (a (log a - 1)) for r < a, log r / log a otherwise */
        double r = sqrt(r2_of(d, x, y));
        if (r == 0.0) return 0.0;
        if (r < h) return s * ((r * (log(r) - 1.0)) / (h * (log(h) - 1.0)));
        return s * (log(r) / log(h));
    }
    case ORC_K_PAPER_II: {
        /* r / a for r < a, a / r otherwise */
        double r = sqrt(r2_of(d, x, y));
        if (r < h) return s * (r / h);
        return s * (h / r);
    }
    case ORC_K_SEPARABLE: {
        double fx = 1.0, fy = 1.0;
        for (int k = 0; k < d; ++k) { fx = fx + x[k]; fy = fy + y[k]; }
        return s * (fx * fy);
    }
    case ORC_K_POLY2: {
        double t = 1.0;
        for (int k = 0; k < d; ++k) t = t + x[k] * y[k];
        return s * (t * t);
    }
    default:
        return NAN;
    }
}

/* A(i, j) for sorted positions of a built tree (P = Q): the diagonal by index. */
double orc_entry(const orc_h2 *h, long i, long j) {
    if (i == j) return h->cfg.kparam[2];
    return orc_kernel(&h->cfg, h->x + i * h->d, h->x + j * h->d);
}

/* K over all pairs of two point lists (row-major out, rows x cols); no diagonal rule. */
void orc_kernel_block(const orc_config *cfg, const double *X, long nx, const double *Y, long ny, double *out) {
    for (long i = 0; i < nx; ++i)
        for (long j = 0; j < ny; ++j) out[i * ny + j] = orc_kernel(cfg, X + i * cfg->d, Y + j * cfg->d);
}
