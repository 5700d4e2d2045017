/*
 * NNCA build: pivots, bases and translation operators (oracle; test
 * infrastructure only).
 *
 * Identification of pivots (Sec. 2.3.2): the tree is traversed bottom-up
 * (reverse level order). For each cell B two steps:
 *   1. candidate sets (Eqs. 15-18). Leaf:  t~^{B,i} = t^B,
 *        s~^{B,i} = union over B' in IL(B) of s^{B'}.
 *      Non-leaf: t~^{B,i} = union over children B' of t^{B',i},
 *        s~^{B,i} = union over B' in IL(B), B'' child of B', of s^{B'',o}.
 *   2. ACA with tolerance eps on A_{t~ s~}; its row and column pivots become
 *      t^{B,i} and s^{B,i}.
 * Symmetric shortcut (Sec. 5, the paragraph on P = Q and symmetric kernels):
 * with P = Q and K symmetric only the incoming pivots are computed, with
 * t^{B,o} := s^{B,i}, s^{B,o} := t^{B,i}; then V_B = U_B (leaf) and the
 * row translation T_{B B_c} is the transpose of C_{B_c B}. So s^{B'',o} in
 * the non-leaf candidate set is t^{B'',i}.
 *
 * Bases (Sec. 2.3.1, Eq. 11 and Eq. 14): leaf U_B = A_{t^B s^{B,i}}
 * (A_{t^{B,i} s^{B,i}})^{-1}; non-leaf C_{B_c B} = A_{t^{B_c,i} s^{B,i}}
 * (A_{t^{B,i} s^{B,i}})^{-1}. Both are X = A_{t~ sigma} A_{tau sigma}^{-1}
 * over the candidate rows t~ (for a non-leaf the rows of the stacked
 * [C_{B_1 B}; ...; C_{B_{2^d} B}], the Remark of Sec. 2.3.2). They are
 * stored per cell as a |t~| x r row-major matrix. The rows of X at the pivot
 * rows are the identity by definition and are set exactly.
 *
 * Readings where the paper is silent:
 *  - Candidate-set order: t~ in the order of the children (ascending Morton)
 *    and each child's pivots in ACA selection order; s~ over IL(B) in
 *    ascending Morton order, then children in order, then each child's
 *    pivots in selection order. Leaf sets: sorted point order.
 *  - Levels above the first level with a non-empty interaction list need no
 *    pivots (nothing there takes part in a far-field interaction).
 *  - A cell whose far-field candidate columns cannot determine its basis
 *    passes all its candidates up: t^{B,i} := t~^{B,i}, s^{B,i} := {} and its
 *    basis is the identity, so its points still reach the far field of its
 *    ancestors. That is the case when s~ is empty (the interaction list is
 *    empty or holds only rank-0 cells), and more generally when the ACA of
 *    Sec. 2.2.1 uses up every column of s~ without meeting its stopping rule
 *    while rows of t~ remain (rank = |s~| < |t~|): the cross then interpolates
 *    A_{t~ s~} exactly but says nothing about the rows it did not pick, which
 *    the ancestors' far field needs. The empty set is the case |s~| = 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#include "orc_internal.h"

typedef struct { const orc_h2 *h; const long *rows; const long *cols; } block_ctx;
static double block_entry(const void *ctx, long i, long j) {
    const block_ctx *c = (const block_ctx *)ctx;
    return orc_entry(c->h, c->rows[i], c->cols[j]);
}

typedef struct {
    long m, r;       /* candidate rows, rank */
    long *cand;      /* t~ (m)               */
    long *prow;      /* t^{B,i} (r)          */
    long *pcol;      /* s^{B,i} (r) or NULL  */
    double *op;      /* m x r                */
    int passthru;
} cell_out;

/* all m candidate rows become the pivots t^{B,i}, with the identity basis */
static void pass_through(cell_out *o, const long *rows, long m) {
    o->passthru = 1;
    o->r = m;
    o->prow = (long *)malloc(sizeof(long) * (size_t)(m > 0 ? m : 1));
    memcpy(o->prow, rows, sizeof(long) * (size_t)m);
    o->pcol = NULL;
    o->op = (double *)calloc((size_t)(m * m > 0 ? m * m : 1), sizeof(double));
    for (long t = 0; t < m; ++t) o->op[t * m + t] = 1.0;
}

static void build_cell(const orc_h2 *h, long B, int leaf, cell_out *outs, cell_out *o) {
    const double eps = h->cfg.aca_tol;
    /* step 1: candidate sets */
    long m = 0, n = 0;
    long *rows, *cols;
    if (leaf) {
        m = h->cend[B] - h->cbeg[B];
        rows = (long *)malloc(sizeof(long) * (size_t)(m > 0 ? m : 1));
        for (long t = 0; t < m; ++t) rows[t] = h->cbeg[B] + t;
        for (long q = h->il_off[B]; q < h->il_off[B + 1]; ++q) {
            long Y = h->il_idx[q];
            n += h->cend[Y] - h->cbeg[Y];
        }
        cols = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
        n = 0;
        for (long q = h->il_off[B]; q < h->il_off[B + 1]; ++q) {
            long Y = h->il_idx[q];
            for (long p = h->cbeg[Y]; p < h->cend[Y]; ++p) cols[n++] = p;
        }
    } else {
        for (long c = h->cch_beg[B]; c < h->cch_end[B]; ++c) m += outs[c].r;
        rows = (long *)malloc(sizeof(long) * (size_t)(m > 0 ? m : 1));
        m = 0;
        for (long c = h->cch_beg[B]; c < h->cch_end[B]; ++c)
            for (long t = 0; t < outs[c].r; ++t) rows[m++] = outs[c].prow[t];
        for (long q = h->il_off[B]; q < h->il_off[B + 1]; ++q) {
            long Y = h->il_idx[q];
            for (long c = h->cch_beg[Y]; c < h->cch_end[Y]; ++c) n += outs[c].r;
        }
        cols = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
        n = 0;
        for (long q = h->il_off[B]; q < h->il_off[B + 1]; ++q) {
            long Y = h->il_idx[q];
            for (long c = h->cch_beg[Y]; c < h->cch_end[Y]; ++c)
                for (long t = 0; t < outs[c].r; ++t) cols[n++] = outs[c].prow[t];
        }
    }
    o->m = m;
    o->cand = rows;
    if (n == 0) {
        /* no far-field candidates: pass everything up, identity basis */
        pass_through(o, rows, m);
        free(cols);
        return;
    }
    /* step 2: ACA on A_{t~ s~} */
    long kmax = m < n ? m : n;
    long *pr = (long *)malloc(sizeof(long) * (size_t)(kmax > 0 ? kmax : 1));
    long *pc = (long *)malloc(sizeof(long) * (size_t)(kmax > 0 ? kmax : 1));
    block_ctx ctx = {h, rows, cols};
    long r = orc_aca(m, n, block_entry, &ctx, eps, pr, pc, NULL, NULL);
    if (r == n && r < m) {
        /* every far-field column used, rows left: the basis is not determined */
        free(pr); free(pc); free(cols);
        pass_through(o, rows, m);
        return;
    }
    o->passthru = 0;
    o->r = r;
    o->prow = (long *)malloc(sizeof(long) * (size_t)(r > 0 ? r : 1));
    o->pcol = (long *)malloc(sizeof(long) * (size_t)(r > 0 ? r : 1));
    for (long t = 0; t < r; ++t) { o->prow[t] = rows[pr[t]]; o->pcol[t] = cols[pc[t]]; }
    /* bases: X = A_{t~ sigma} (A_{tau sigma})^{-1} */
    double *M = (double *)malloc(sizeof(double) * (size_t)(r * r > 0 ? r * r : 1));
    double *Bm = (double *)malloc(sizeof(double) * (size_t)(m * r > 0 ? m * r : 1));
    for (long a = 0; a < r; ++a)
        for (long b = 0; b < r; ++b) M[a * r + b] = orc_entry(h, o->prow[a], o->pcol[b]);
    for (long t = 0; t < m; ++t)
        for (long b = 0; b < r; ++b) Bm[t * r + b] = orc_entry(h, rows[t], o->pcol[b]);
    o->op = (double *)malloc(sizeof(double) * (size_t)(m * r > 0 ? m * r : 1));
    orc_solve_right(M, r, Bm, m, o->op);
    for (long a = 0; a < r; ++a)
        for (long b = 0; b < r; ++b) o->op[pr[a] * r + b] = (a == b) ? 1.0 : 0.0;
    free(M); free(Bm); free(pr); free(pc); free(cols);
}

static orc_h2 *alloc_h(const orc_config *cfg, const double *P, long n) {
    if (!cfg || (n > 0 && !P) || n < 0) return NULL;
    if (cfg->d < 1 || cfg->d > 4 || cfg->leaf_size < 1 || cfg->eta2_num < 1 || cfg->eta2_den < 1) return NULL;
    if (!(cfg->aca_tol > 0.0)) return NULL;
    for (long i = 0; i < n * cfg->d; ++i)
        if (!isfinite(P[i])) return NULL;
    orc_h2 *h = (orc_h2 *)calloc(1, sizeof(orc_h2));
    h->cfg = *cfg;
    h->d = cfg->d;
    return h;
}

orc_h2 *orc_build_structure(const orc_config *cfg, const double *P, long n, int nthreads) {
    (void)nthreads;
    orc_h2 *h = alloc_h(cfg, P, n);
    if (!h) return NULL;
    orc_tree_build(h, P, n);
    orc_lists_build(h);
    return h;
}

orc_h2 *orc_build(const orc_config *cfg, const double *P, long n, int nthreads) {
    orc_h2 *h = orc_build_structure(cfg, P, n, nthreads);
    if (!h) return NULL;
    const long nc = h->ncell;
    cell_out *outs = (cell_out *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(cell_out));
    for (int l = h->kappa; l >= h->lmin; --l) {
        const int leaf = (l == h->kappa);
        const long b0 = h->level_base[l], b1 = h->level_base[l + 1];
        #pragma omp parallel for schedule(dynamic, 1)
        for (long B = b0; B < b1; ++B) build_cell(h, B, leaf, outs, &outs[B]);
    }
    /* pack per-cell results into CSR arrays */
    h->piv_off = (long *)calloc((size_t)nc + 1, sizeof(long));
    h->cand_off = (long *)calloc((size_t)nc + 1, sizeof(long));
    h->op_off = (long *)calloc((size_t)nc + 1, sizeof(long));
    h->passthru = (int *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int));
    for (long c = 0; c < nc; ++c) {
        h->piv_off[c + 1] = h->piv_off[c] + outs[c].r;
        h->cand_off[c + 1] = h->cand_off[c] + outs[c].m;
        h->op_off[c + 1] = h->op_off[c] + outs[c].m * outs[c].r;
        h->passthru[c] = outs[c].passthru;
    }
    h->piv_row = (long *)malloc(sizeof(long) * (size_t)(h->piv_off[nc] > 0 ? h->piv_off[nc] : 1));
    h->piv_col = (long *)malloc(sizeof(long) * (size_t)(h->piv_off[nc] > 0 ? h->piv_off[nc] : 1));
    h->cand = (long *)malloc(sizeof(long) * (size_t)(h->cand_off[nc] > 0 ? h->cand_off[nc] : 1));
    h->op = (double *)malloc(sizeof(double) * (size_t)(h->op_off[nc] > 0 ? h->op_off[nc] : 1));
    for (long c = 0; c < nc; ++c) {
        for (long t = 0; t < outs[c].r; ++t) {
            h->piv_row[h->piv_off[c] + t] = outs[c].prow[t];
            h->piv_col[h->piv_off[c] + t] = outs[c].pcol ? outs[c].pcol[t] : -1;
        }
        for (long t = 0; t < outs[c].m; ++t) h->cand[h->cand_off[c] + t] = outs[c].cand[t];
        if (outs[c].m * outs[c].r > 0)
            memcpy(h->op + h->op_off[c], outs[c].op, sizeof(double) * (size_t)(outs[c].m * outs[c].r));
        free(outs[c].cand); free(outs[c].prow); free(outs[c].pcol); free(outs[c].op);
    }
    free(outs);
    return h;
}

long orc_leaf_pivots(const orc_h2 *h, long cell, long *prow, long *pcol, long cap) {
    if (cell < h->level_base[h->kappa] || cell >= h->level_base[h->kappa + 1]) return -1;
    cell_out o;
    memset(&o, 0, sizeof(o));
    build_cell(h, cell, 1, NULL, &o);
    long r = o.r;
    for (long t = 0; t < r && t < cap; ++t) {
        prow[t] = o.prow[t];
        pcol[t] = o.pcol ? o.pcol[t] : -1;
    }
    free(o.cand); free(o.prow); free(o.pcol); free(o.op);
    return r;
}

void orc_free(orc_h2 *h) {
    if (!h) return;
    free(h->perm); free(h->key); free(h->x);
    free(h->ckey); free(h->cbeg); free(h->cend); free(h->cpar); free(h->cch_beg); free(h->cch_end);
    free(h->nb_off); free(h->nb_idx); free(h->il_off); free(h->il_idx);
    free(h->piv_off); free(h->piv_row); free(h->piv_col); free(h->passthru);
    free(h->cand_off); free(h->cand); free(h->op_off); free(h->op);
    free(h->s_off); free(h->s_blk); free(h->near_off); free(h->near_blk);
    free(h);
}
