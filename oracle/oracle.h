/*
 * FP64 CPU oracle for the NNCA-based H^2 matrix-vector product of
 * Gujjula & Ambikasaran, "A new Nested Cross Approximation" (NNCA).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product links, imports or calls
 * this code: it exists so that the tests, the smoke check and the CPU-baseline
 * leg of the benchmark can check the CUDA path against an independent,
 * plainly written implementation of the paper's method. It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Everything is FP64 and compiled with -ffp-contract=off: every multiply-add
 * that the method performs as one fused step is written as an explicit IEEE
 * fma() call, every other operation rounds on its own.
 *
 * Parts (each file cites the passage of the paper it follows):
 *   orc_tree.c    uniform 2^d tree, leaf level kappa (Sec. 2.1)
 *   orc_lists.c   neighbours N(B) and interaction list IL(B) (Sec. 2.2, Eq. 2, Table 1)
 *   orc_aca.c     partially pivoted ACA (Sec. 2.2.1, Eqs. 3-4), LU solve for
 *                 the bases (Sec. 2.3.1, Eq. 11 and Eq. 14)
 *   orc_build.c   bottom-up pivot identification (Sec. 2.3.2, Eqs. 15-18),
 *                 symmetric shortcut (Sec. 5, opening paragraphs),
 *                 H^2 representation (Sec. 3)
 *   orc_matvec.c  H^2 matrix-vector product (Sec. 4, steps 1-5) in stored and
 *                 on-the-fly forms, and the dense product u = A w (Eq. 19)
 *   orc_kernel.c  kernel functions K(x, y)
 *
 * Vectors: nrhs right-hand sides, vector r stored contiguously at x[r*ld + i]
 * (i = original point index).
 */
#ifndef NNCA_ORACLE_H
#define NNCA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_K_LOG = 0,        /* s * log(r)                                  */
    ORC_K_INV_R = 1,      /* s / r                                       */
    ORC_K_GAUSS = 2,      /* s * exp(-r^2 / (2 h^2))                     */
    ORC_K_MATERN = 3,     /* s * exp(-r / h)                             */
    ORC_K_PAPER_I = 4,    /* Sec. 5.1 kernel (i), parameter a            */
    ORC_K_PAPER_II = 5,   /* Sec. 5.1 kernel (ii), parameter a           */
    ORC_K_SEPARABLE = 6,  /* s * f(x) f(y), f(x) = 1 + sum_k x_k (rank 1) */
    ORC_K_POLY2 = 7       /* s * (1 + x.y)^2 (rank <= (d+1)(d+2)/2)      */
};

typedef struct {
    int d;              /* dimension, 1..4                                    */
    int leaf_size;      /* nu: maximum points per leaf (Sec. 2.1)             */
    int eta2_num;       /* eta^2 = eta2_num / eta2_den (Sec. 2.2, Eq. 2)      */
    int eta2_den;
    double aca_tol;     /* epsilon of the ACA stopping rule (Eq. 4)           */
    int kernel;         /* ORC_K_*                                            */
    double kparam[4];   /* [0] scale s, [1] h or a, [2] diagonal value K(p_i,p_i), [3] unused */
} orc_config;

/* The H^2 representation built by orc_build. Cells are numbered globally,
 * level by level: level l holds cells [level_base[l], level_base[l+1]).
 * Point indices in the tree are positions in Morton-sorted order
 * (sorted position s holds original point perm[s]). */
typedef struct {
    int d, lmax, kappa, lmin;      /* lmin: first level with a non-empty IL (kappa+1 if none) */
    long n;
    double corner[4], side;        /* the cube D = corner + [0, side]^d          */
    long *perm;                    /* [n] original index of sorted position       */
    uint64_t *key;                 /* [n] sorted Morton keys (lmax bits per dim)  */
    double *x;                     /* [n*d] sorted coordinates, row-major         */
    long ncell;                    /* total cells, all levels                     */
    long level_base[66];
    uint64_t *ckey;                /* [ncell] cell key at its level               */
    long *cbeg, *cend;             /* [ncell] sorted point range of the cell      */
    long *cpar;                    /* [ncell] parent cell (-1 for the root)       */
    long *cch_beg, *cch_end;       /* [ncell] children cell range                 */
    long *nb_off, *nb_idx;         /* CSR: neighbours N(B), ascending cell id     */
    long *il_off, *il_idx;         /* CSR: interaction list IL(B), ascending      */
    long *piv_off;                 /* [ncell+1] CSR of incoming pivots            */
    long *piv_row;                 /* t^{B,i}: sorted point positions             */
    long *piv_col;                 /* s^{B,i}: sorted point positions (-1 if pass-through) */
    int *passthru;                 /* [ncell] 1 if the cell passed all candidates up (no far-field
                                      candidates, or an ACA that used up every column) */
    long *cand_off;                /* [ncell+1] CSR of candidate rows t~^{B,i}    */
    long *cand;                    /* t~^{B,i}: sorted point positions            */
    long *op_off;                  /* [ncell+1] offsets into op                   */
    double *op;                    /* per cell |t~| x r row-major: U_B (leaf) or stacked C_{B_c B} */
    /* stored H^2 form (Sec. 3 steps 2-3); NULL until orc_assemble */
    long *s_off;                   /* [n_il_entries+1] offsets of S_{X,Y} blocks   */
    double *s_blk;
    long *near_off;                /* [n_nb_entries+1] offsets of near-field blocks */
    double *near_blk;
    orc_config cfg;
} orc_h2;

/* Kernel K(x, y) for points x, y (d coordinates each), in FP64. Does not
 * apply the diagonal rule; callers handle i == j by index. */
double orc_kernel(const orc_config *cfg, const double *x, const double *y);
/* K over all pairs of two point lists (out is nx x ny row-major); no diagonal rule. */
void orc_kernel_block(const orc_config *cfg, const double *X, long nx, const double *Y, long ny, double *out);
/* A(i, j) for sorted positions i, j of a built tree, with the diagonal rule. */
double orc_entry(const orc_h2 *h, long i, long j);

/* Build everything (tree, lists, pivots, operators). P: n x d row-major.
 * Returns NULL on invalid input. nthreads <= 0 uses the OpenMP default. */
orc_h2 *orc_build(const orc_config *cfg, const double *P, long n, int nthreads);
/* Tree and lists only (no pivots): for structure checks at large n. */
orc_h2 *orc_build_structure(const orc_config *cfg, const double *P, long n, int nthreads);
void orc_free(orc_h2 *h);
/* Pivots of one leaf cell (Sec. 2.3.2, leaf candidate sets) computed from the
 * tree and lists alone; works on a structure-only build. Returns the rank
 * (pivots beyond cap are not written), or -1 if cell is not a leaf. */
long orc_leaf_pivots(const orc_h2 *h, long cell, long *prow, long *pcol, long cap);

/* Form the stored H^2 representation (coupling S_{X,Y} and near blocks). */
int orc_assemble(orc_h2 *h);

/* H^2 product y = A~ x. form 0: on-the-fly kernel evaluation, form 1: stored,
 * form 2: on the fly with the transverse pass (Sec. 4 step 3) taken over each
 * unordered pair {X, Y}, Y in IL(X), once: S_{X,Y} = K(t^X, t^Y) is evaluated
 * and applied as u^X += S w^Y and u^Y += S^T w^X (the kernel is symmetric and
 * Y in IL(X) iff X in IL(Y)); serial, in cell order. */
int orc_h2_matvec(const orc_h2 *h, const double *x, double *y, long nrhs, long ld, int form, int nthreads);
/* Dense product y = A x in original order (Eq. 19 evaluated exactly). */
void orc_dense_matvec(const orc_config *cfg, const double *P, long n, const double *x, double *y,
                      long nrhs, long ld, int nthreads);
/* Dense product restricted to rows[0..nrows): y[r*nrows + q] = (A x_r)[rows[q]]. */
void orc_dense_rows(const orc_config *cfg, const double *P, long n, const long *rows, long nrows,
                    const double *x, double *y, long nrhs, long ld, int nthreads);

/* Partially pivoted ACA of an explicit m x n matrix A (row-major, lda).
 * Returns the rank k and writes prow[0..k), pcol[0..k), and the crosses
 * U (m x kmax, column l at U[l*m]) and V (n x kmax, column l at V[l*n]) if
 * those are non-NULL. kmax = min(m, n). */
long orc_aca_dense(const double *A, long m, long n, long lda, double eps,
                   long *prow, long *pcol, double *U, double *V);

/* Solve X * M = B for X (m x r) with M (r x r), B (m x r), all row-major,
 * by LU with partial pivoting of M^T. X may alias B. Returns 0, or -1 if a
 * pivot is exactly zero. */
int orc_solve_right(const double *M, long r, const double *B, long m, double *X);

/* Canonical FP64 dot product used by every reduction of the ACA. */
double orc_cdot(const double *a, const double *b, long n);

#ifdef __cplusplus
}
#endif
#endif
