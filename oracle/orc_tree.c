/*
 * Uniform 2^d tree (oracle; test infrastructure only). Sec. 2.1.
 *
 * The paper builds a uniform 2^d tree on a compact hypercube D containing the
 * points, subdividing every cell into 2^d children, and stops at the first
 * level kappa at which every cell holds at most nu points (of P and of Q; here
 * P = Q). The paper does not fix D or the point-to-cell rule; the reading used:
 *
 *  - D is the bounding cube of the points: centre c_k = (lo_k + hi_k) * 0.5,
 *    half side h = max_k (hi_k - lo_k) * 0.5 (h = 0.5 if all points coincide),
 *    corner_k = c_k - h, side = 2h.
 *  - Each coordinate is quantised once at lmax = floor(63 / d) bits:
 *    q_k = floor(((x_k - corner_k) / side) * 2^lmax), clamped to
 *    [0, 2^lmax - 1]. The level-l cell of a point is given by the top l bits
 *    of every q_k, so cells nest exactly.
 *  - The Morton key interleaves the bits: bit b of q_k goes to key bit
 *    b*d + k (dimension 0 is the least significant bit of each group).
 *  - Points are sorted by (key, original index); cells at every level are
 *    runs of equal key prefixes in that order; only non-empty cells exist.
 *  - kappa = the smallest level at which every cell holds <= nu points; if
 *    even level lmax has a larger cell (coincident points), kappa = lmax.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#include "orc_internal.h"

typedef struct { uint64_t key; long idx; } keyidx;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *p = (const keyidx *)a, *q = (const keyidx *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* Level-l prefix of a key. */
uint64_t orc_prefix(const orc_h2 *h, uint64_t key, int l) {
    int shift = h->d * (h->lmax - l);
    return shift >= 64 ? 0 : key >> shift;
}

/* Integer coordinates of a level-l cell from its key prefix. */
void orc_cell_coords(int d, uint64_t ckey, int l, int64_t *c) {
    for (int k = 0; k < d; ++k) c[k] = 0;
    for (int b = 0; b < l; ++b)
        for (int k = 0; k < d; ++k)
            c[k] |= (int64_t)((ckey >> (b * d + k)) & 1u) << b;
}

int orc_tree_build(orc_h2 *h, const double *P, long n) {
    const int d = h->d;
    const int lmax = 63 / d;
    h->lmax = lmax;
    h->n = n;

    /* bounding cube */
    double lo[4], hi[4];
    for (int k = 0; k < d; ++k) { lo[k] = P[k]; hi[k] = P[k]; }
    for (long i = 1; i < n; ++i)
        for (int k = 0; k < d; ++k) {
            double v = P[i * d + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double half = 0.0;
    for (int k = 0; k < d; ++k) {
        double e = (hi[k] - lo[k]) * 0.5;
        if (e > half) half = e;
    }
    if (half == 0.0) half = 0.5;
    for (int k = 0; k < d; ++k) h->corner[k] = (lo[k] + hi[k]) * 0.5 - half;
    h->side = 2.0 * half;

    /* quantise, Morton keys, stable sort by (key, index) */
    const double scale = ldexp(1.0, lmax);
    const uint64_t qmax = (lmax == 64) ? ~(uint64_t)0 : (((uint64_t)1 << lmax) - 1);
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) {
        uint64_t key = 0;
        for (int k = 0; k < d; ++k) {
            double t = ((P[i * d + k] - h->corner[k]) / h->side) * scale;
            double f = floor(t);
            uint64_t q;
            if (!(f >= 0.0)) q = 0;
            else if (f >= scale) q = qmax;
            else q = (uint64_t)f;
            for (int b = 0; b < lmax; ++b) key |= ((q >> b) & 1u) << (b * d + k);
        }
        ki[i].key = key;
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    h->perm = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    h->key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    h->x = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n * d : 1));
    for (long i = 0; i < n; ++i) {
        h->perm[i] = ki[i].idx;
        h->key[i] = ki[i].key;
        for (int k = 0; k < d; ++k) h->x[i * d + k] = P[ki[i].idx * d + k];
    }
    free(ki);

    /* leaf level: the first level whose largest cell holds <= nu points */
    int kappa = lmax;
    for (int l = 0; l <= lmax; ++l) {
        long run = 0, maxrun = 0;
        for (long i = 0; i < n; ++i) {
            if (i == 0 || orc_prefix(h, h->key[i], l) != orc_prefix(h, h->key[i - 1], l)) run = 0;
            ++run;
            if (run > maxrun) maxrun = run;
        }
        if (maxrun <= h->cfg.leaf_size) { kappa = l; break; }
    }
    h->kappa = kappa;

    /* cells of every level: runs of equal prefixes */
    long total = 0;
    for (int l = 0; l <= kappa; ++l) {
        long c = 0;
        for (long i = 0; i < n; ++i)
            if (i == 0 || orc_prefix(h, h->key[i], l) != orc_prefix(h, h->key[i - 1], l)) ++c;
        if (n == 0 && l == 0) c = 0;
        h->level_base[l] = total;
        total += c;
    }
    h->level_base[kappa + 1] = total;
    h->ncell = total;
    h->ckey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(total > 0 ? total : 1));
    h->cbeg = (long *)malloc(sizeof(long) * (size_t)(total > 0 ? total : 1));
    h->cend = (long *)malloc(sizeof(long) * (size_t)(total > 0 ? total : 1));
    h->cpar = (long *)malloc(sizeof(long) * (size_t)(total > 0 ? total : 1));
    h->cch_beg = (long *)malloc(sizeof(long) * (size_t)(total > 0 ? total : 1));
    h->cch_end = (long *)malloc(sizeof(long) * (size_t)(total > 0 ? total : 1));
    /* point -> cell at the previous level, to link parents */
    long *cell_of = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long *cell_prev = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (int l = 0; l <= kappa; ++l) {
        long c = h->level_base[l] - 1;
        for (long i = 0; i < n; ++i) {
            uint64_t p = orc_prefix(h, h->key[i], l);
            if (i == 0 || p != orc_prefix(h, h->key[i - 1], l)) {
                ++c;
                h->ckey[c] = p;
                h->cbeg[c] = i;
                h->cpar[c] = (l == 0) ? -1 : cell_prev[i];
                h->cch_beg[c] = h->cch_end[c] = -1;
            }
            h->cend[c] = i + 1;
            cell_of[i] = c;
        }
        if (l > 0) {
            /* children of the level-(l-1) cells: contiguous runs of this level */
            for (long cc = h->level_base[l]; cc < h->level_base[l + 1]; ++cc) {
                long p = h->cpar[cc];
                if (h->cch_beg[p] < 0) h->cch_beg[p] = cc;
                h->cch_end[p] = cc + 1;
            }
        }
        long *t = cell_prev; cell_prev = cell_of; cell_of = t;
    }
    for (long c = h->level_base[kappa]; c < h->level_base[kappa + 1]; ++c) h->cch_beg[c] = h->cch_end[c] = -1;
    for (long c = 0; c < total; ++c)
        if (h->cch_beg[c] < 0) h->cch_beg[c] = h->cch_end[c] = 0;
    free(cell_of);
    free(cell_prev);
    return 0;
}
