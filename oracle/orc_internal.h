/* Internal declarations shared by the oracle's own files (test infrastructure only). */
#ifndef NNCA_ORC_INTERNAL_H
#define NNCA_ORC_INTERNAL_H
#include "oracle.h"

uint64_t orc_prefix(const orc_h2 *h, uint64_t key, int l);
void orc_cell_coords(int d, uint64_t ckey, int l, int64_t *c);
int orc_tree_build(orc_h2 *h, const double *P, long n);
int orc_lists_build(orc_h2 *h);
int orc_level_of(const orc_h2 *h, long cell);
/* 1 if two level-l cells satisfy the admissibility condition (Eq. 2). */
int orc_admissible(const orc_h2 *h, long X, long Y, int l);

/* Entry callback for the ACA: A(i, j) of the block being approximated. */
typedef double (*orc_entry_fn)(const void *ctx, long i, long j);
long orc_aca(long m, long n, orc_entry_fn entry, const void *ctx, double eps,
             long *prow, long *pcol, double *U, double *V);
#endif
