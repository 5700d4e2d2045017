/*
 * Neighbours and interaction lists (oracle; test infrastructure only).
 *
 * Admissibility (Sec. 2.2, Eq. 2): cells X, Y are admissible when
 *     max{diam X, diam Y} <= eta * dist(X, Y).
 * Two cells of one level are cubes of the same side s, with integer cell
 * coordinates a and b. Then diam = sqrt(d) * s and
 *     dist = s * sqrt(sum_k g_k^2),  g_k = max(0, |a_k - b_k| - 1),
 * so with eta^2 = num / den the test is exact in integers:
 *     admissible  <=>  d * den <= num * sum_k g_k^2.
 *
 * Table 1:
 *   N(B)  = cells at the level of B that are not admissible with B
 *           (this includes B itself);
 *   IL(B) = children of the neighbours of B's parent that are not
 *           neighbours of B.
 * The root has N = {root}, IL = {}. Only non-empty cells exist (the paper is
 * silent on empty cells; they hold no points and take part in nothing).
 * N(B) is formed by testing every cell of the level (the plain definition);
 * both lists are in ascending cell id, which is ascending Morton key.
 */
#include <stdlib.h>
#include "oracle.h"
#include "orc_internal.h"

int orc_level_of(const orc_h2 *h, long cell) {
    int l = 0;
    while (cell >= h->level_base[l + 1]) ++l;
    return l;
}

static int admissible_coords(int d, int num, int den, const int64_t *a, const int64_t *b) {
    int64_t g2 = 0;
    for (int k = 0; k < d; ++k) {
        int64_t t = a[k] - b[k];
        if (t < 0) t = -t;
        t = t - 1;
        if (t < 0) t = 0;
        g2 += t * t;
    }
    return (int64_t)d * den <= (int64_t)num * g2;
}

int orc_admissible(const orc_h2 *h, long X, long Y, int l) {
    int64_t a[4], b[4];
    orc_cell_coords(h->d, h->ckey[X], l, a);
    orc_cell_coords(h->d, h->ckey[Y], l, b);
    return admissible_coords(h->d, h->cfg.eta2_num, h->cfg.eta2_den, a, b);
}

typedef struct { long *v; long n, cap; } lvec;
static void lpush(lvec *a, long x) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 64;
        a->v = (long *)realloc(a->v, sizeof(long) * (size_t)a->cap);
    }
    a->v[a->n++] = x;
}

int orc_lists_build(orc_h2 *h) {
    const long nc = h->ncell;
    h->nb_off = (long *)calloc((size_t)nc + 1, sizeof(long));
    h->il_off = (long *)calloc((size_t)nc + 1, sizeof(long));
    long **nbl = (long **)calloc((size_t)(nc > 0 ? nc : 1), sizeof(long *));
    long *nbn = (long *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(long));
    long **ill = (long **)calloc((size_t)(nc > 0 ? nc : 1), sizeof(long *));
    long *iln = (long *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(long));

    const int d = h->d, num = h->cfg.eta2_num, den = h->cfg.eta2_den;
    int64_t *co = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)(nc > 0 ? nc : 1));
    for (int l = 0; l <= h->kappa && nc > 0; ++l)
        for (long c = h->level_base[l]; c < h->level_base[l + 1]; ++c) orc_cell_coords(d, h->ckey[c], l, co + 4 * c);
    for (int l = 0; l <= h->kappa && nc > 0; ++l) {
        long b0 = h->level_base[l], b1 = h->level_base[l + 1];
        /* neighbours: every cell of the level that is not admissible with X */
        #pragma omp parallel for schedule(dynamic, 16)
        for (long X = b0; X < b1; ++X) {
            lvec a = {0, 0, 0};
            for (long Y = b0; Y < b1; ++Y)
                if (!admissible_coords(d, num, den, co + 4 * X, co + 4 * Y)) lpush(&a, Y);
            nbl[X] = a.v;
            nbn[X] = a.n;
        }
        /* interaction list: children of the parent's neighbours that are not
         * neighbours of X, i.e. that are admissible with X */
        #pragma omp parallel for schedule(dynamic, 16)
        for (long X = b0; X < b1; ++X) {
            lvec a = {0, 0, 0};
            if (l > 0) {
                long P = h->cpar[X];
                for (long q = 0; q < nbn[P]; ++q) {
                    long Z = nbl[P][q];
                    for (long Y = h->cch_beg[Z]; Y < h->cch_end[Z]; ++Y)
                        if (admissible_coords(d, num, den, co + 4 * X, co + 4 * Y)) lpush(&a, Y);
                }
            }
            ill[X] = a.v;
            iln[X] = a.n;
        }
    }
    free(co);
    for (long c = 0; c < nc; ++c) {
        h->nb_off[c + 1] = h->nb_off[c] + nbn[c];
        h->il_off[c + 1] = h->il_off[c] + iln[c];
    }
    h->nb_idx = (long *)malloc(sizeof(long) * (size_t)(h->nb_off[nc] > 0 ? h->nb_off[nc] : 1));
    h->il_idx = (long *)malloc(sizeof(long) * (size_t)(h->il_off[nc] > 0 ? h->il_off[nc] : 1));
    for (long c = 0; c < nc; ++c) {
        for (long t = 0; t < nbn[c]; ++t) h->nb_idx[h->nb_off[c] + t] = nbl[c][t];
        for (long t = 0; t < iln[c]; ++t) h->il_idx[h->il_off[c] + t] = ill[c][t];
        free(nbl[c]);
        free(ill[c]);
    }
    free(nbl); free(nbn); free(ill); free(iln);
    /* first level with a non-empty interaction list */
    h->lmin = h->kappa + 1;
    for (int l = 0; l <= h->kappa; ++l) {
        long any = 0;
        for (long c = h->level_base[l]; c < h->level_base[l + 1]; ++c) any |= (h->il_off[c + 1] > h->il_off[c]);
        if (any) { h->lmin = l; break; }
    }
    return 0;
}
