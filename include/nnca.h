/*
 * nnca.h -- C ABI of the GB300 (sm_103a) NNCA H^2 library.
 *
 * Computes the H^2 matrix-vector product y = A x with A(i, j) = K(p_i, p_j)
 * (or K(p_i, q_j) for distinct point sets P and Q, see nnca_build) built by
 * the new Nested Cross Approximation (NNCA) of Gujjula & Ambikasaran, "A new
 * Nested Cross Approximation":
 *
 *   nnca_build   uniform 2^d tree over the points (Sec. 2.1), neighbour and
 *                interaction lists from the admissibility condition
 *                (Sec. 2.2, Eq. 2, Table 1), bottom-up pivot identification
 *                by ACA on the candidate sets (Sec. 2.3.2, Eqs. 15-18), and
 *                the nested bases and translation operators
 *                A_{t~ s^{B,i}} (A_{t^{B,i} s^{B,i}})^{-1} (Sec. 2.3.1,
 *                Eqs. 11 and 14; Remark of Sec. 2.3.2);
 *   nnca_matvec  the H^2 product of Sec. 4: upward pass (P2M, M2M),
 *                transverse pass (M2L with K evaluated on the fly over the
 *                pivot pairs of Sec. 3 step 2), downward pass (L2L, L2P) and
 *                the near field (P2P over Sec. 3 step 3 blocks, evaluated
 *                on the fly).
 *
 * Every step runs as a CUDA kernel on the GPU that is current when the call
 * is made; no step falls back to the host.
 *
 * Conventions
 *  - All pointers named "device" must be device memory of the current GPU;
 *    pointers named "host" must be host memory (pageable or pinned).
 *  - Points: n x d FP64; layout NNCA_LAYOUT_AOS (p[i*d + k]) or
 *    NNCA_LAYOUT_SOA (p[k*n + i]).
 *  - Vectors: nrhs right-hand sides; right-hand side r occupies
 *    x[r*ld + i], i the caller's point index, ld >= n (for P != Q: x on the
 *    points of Q, y on those of P, ld >= max(nP, nQ)).
 *  - Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *    default stream. nnca_build synchronises the stream (it reads sizes back
 *    to the host); nnca_matvec is asynchronous on the stream.
 *  - Errors: every call returns an nnca_status; no exception crosses the
 *    ABI. After a failure nnca_last_error() holds a one-line message
 *    (thread-local for calls without a handle). A failed nnca_build leaves
 *    *out == NULL and frees everything it allocated.
 *  - Ownership: the library copies what it needs; caller buffers are only
 *    read or written during the call (or, for nnca_matvec, until the stream
 *    reaches the end of the call's work). The handle owns all device memory
 *    it allocates; nnca_destroy frees it.
 *  - Thread safety: one handle must not be used by two host threads at once.
 */
#ifndef NNCA_H
#define NNCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nnca_handle_s *nnca_handle;

typedef enum {
    NNCA_OK = 0,
    NNCA_ERR_INVALID_ARG = 1,   /* rejected before any device work            */
    NNCA_ERR_OOM = 2,           /* a device allocation failed                 */
    NNCA_ERR_CUDA = 3,          /* a CUDA runtime call or kernel failed       */
    NNCA_ERR_UNSUPPORTED = 4,   /* valid request this build does not support  */
    NNCA_ERR_TIMEOUT = 5,       /* a bounded device wait gave up              */
    NNCA_ERR_INTERNAL = 6       /* a device-side consistency check failed     */
} nnca_status;

/* Kernel functions K(r), r = |x - y|_2 (Sec. 1: smooth away from x = y;
 * Sec. 5 uses radial kernels). s = kparam[0]. The diagonal entry A(i, i) is
 * decided by index and equals kparam[2]; two distinct coincident points give 0
 * for the kernels singular at r = 0 (LOG, INV_R, PAPER_I) and K(0) otherwise. */
enum {
    NNCA_K_LOG = 0,        /* s log r                                          */
    NNCA_K_INV_R = 1,      /* s / r                                            */
    NNCA_K_GAUSS = 2,      /* s exp(-r^2 / (2 h^2)),      h = kparam[1]        */
    NNCA_K_MATERN = 3,     /* s exp(-r / h),              h = kparam[1]        */
    NNCA_K_PAPER_I = 4,    /* Sec. 5.1 kernel (i):  r(log r - 1)/(a(log a - 1)) for r < a,
                              log r / log a otherwise,   a = kparam[1]          */
    NNCA_K_PAPER_II = 5,   /* Sec. 5.1 kernel (ii): r/a for r < a, a/r otherwise */
    NNCA_K_SEPARABLE = 6,  /* s f(x) f(y), f(x) = 1 + sum_k x_k  (rank 1)       */
    NNCA_K_POLY2 = 7       /* s (1 + x.y)^2                                     */
};

enum { NNCA_LAYOUT_AOS = 0, NNCA_LAYOUT_SOA = 1 };
enum { NNCA_F64 = 0, NNCA_F32 = 1 };                 /* element type of x and y   */
/* Arithmetic of the product. FP64: everything in double. FP32: the kernel
 * evaluations of M2L and P2P (nearly all of the work) in float, with
 * coordinates relative to their cell centre and compensated accumulation
 * across source cells; bases, translations and coefficient vectors in double.
 * Tensor-core forms (for many right-hand sides; radial kernels, d <= 3): the
 * FP32 form with the M2L of up to 64 right-hand sides at once as dense
 * contractions on the tensor cores (tcgen05.mma), the kernel values K
 * evaluated on the fly in float and multiplied with the multipole
 * coefficients of all right-hand sides, accumulated in FP32 in tensor memory:
 *   NNCA_PREC_TF32X3  both operands split into tf32 hi + lo parts, three
 *                     products per pair (hi hi + hi lo + lo hi; about 22 bits);
 *   NNCA_PREC_TF32    one tf32 product per pair (11-bit operands);
 *   NNCA_PREC_BF16    both operands rounded to bfloat16, one product per pair
 *                     (8-bit operands, FP32 accumulation).
 * The other passes run as in the FP32 form. nnca_matvec_noalloc takes FP64 and
 * FP32 only. */
enum { NNCA_PREC_FP64 = 0, NNCA_PREC_FP32 = 1, NNCA_PREC_TF32X3 = 2, NNCA_PREC_TF32 = 3, NNCA_PREC_BF16 = 4 };
/* nnca_config.m2l_form */
enum { NNCA_M2L_AUTO = 0, NNCA_M2L_FULL = 1 };

typedef struct {
    int d;             /* dimension 1..4                                         */
    int leaf_size;     /* nu >= 1: maximum points per leaf (Sec. 2.1)             */
    int eta2_num;      /* eta^2 = eta2_num / eta2_den > 0 (Eq. 2); the paper's    */
    int eta2_den;      /*   experiments use eta = sqrt(2): 2 / 1                  */
    double aca_tol;    /* epsilon > 0 of the ACA stopping rule (Eq. 4)            */
    int kernel;        /* NNCA_K_*                                                */
    double kparam[4];  /* [0] scale s, [1] h or a, [2] diagonal value, [3] unused */
    int symmetric;     /* must be 1: K symmetric (K(p, q) = K(q, p)); uses the
                          shortcut t^{B,o} = s^{B,i}, s^{B,o} = t^{B,i} (Sec. 5),
                          on P, or on the union [P; Q] for P != Q (nnca_build)   */
    int m2l_form;      /* FP32 M2L of one right-hand side: NNCA_M2L_AUTO the symmetric form
                          where it applies (every f(|p - q|) of an admissible
                          pair evaluated once, for both u_B and u_B'; ranks up
                          to 256), NNCA_M2L_FULL always the full form (each target sums
                          its whole interaction list)                            */
    int m2l_item_targets; /* tile of the FP32 M2L: targets (pivots of one parent's
                          children) per work item, 32..256, or 0 for 256; a
                          tuning parameter (it changes only the order of the
                          FP32 partial sums)                                   */
    int reserved;      /* set to 0                                                */
} nnca_config;

/* Sizes and timings of a built handle (the quantities of the paper's
 * Table of Sec. 5: memory, assembly time) plus work counts. */
typedef struct {
    int d, lmax, kappa, lmin;      /* lmin: first level with an interaction list   */
    int64_t n;
    int64_t ncell;                 /* non-empty cells, all levels                  */
    int64_t ncell_level[64];
    int64_t n_il, n_nb;            /* interaction-list and neighbour entries       */
    int64_t n_pivots;              /* sum of ranks over all cells                  */
    int64_t max_rank;
    int64_t n_passthru;            /* pass-through cells (all candidates kept)     */
    int64_t p2p_pairs;             /* sum over leaves of n_B * sum_{N(B)} n_B'     */
    int64_t m2l_pairs;             /* sum over cells of r_B * sum_{IL(B)} r_B'     */
    int64_t op_entries;            /* entries of all bases and translations        */
    int64_t device_bytes;          /* device memory held by the handle             */
    double build_ms[8];            /* tree, lists, pivots (ACA), bases, finish, total, -, - */
    int64_t aca_retries;           /* cells re-run because the scratch pool ran out */
    /* product timings, filled while profiling is on (nnca_set_profiling):
     * device time per pass summed over the profiled products, from CUDA events
     * recorded on the caller's stream between the passes:
     * [0] permutation in, [1] P2M + M2M, [2] M2L, [3] L2L, [4] L2P + P2P,
     * [5] whole product */
    double pass_ms[8];
    int64_t pass_calls;            /* products summed in pass_ms                   */
    int64_t launches_per_product;  /* kernels of this library in the last product  */
    int64_t device_status;         /* device-side check bits since the build (read
                                      by nnca_get_stats): 2 an index failed a bounds
                                      check, 16 a bounded wait on an asynchronous
                                      copy ran out; the product's result is then
                                      not valid. 1 (ACA scratch retried) is benign. */
    int64_t m2l_evals;             /* kernel evaluations of the FP32 M2L of one
                                      right-hand side: m2l_pairs / 2 when it runs
                                      in the symmetric form (each value f(|p - q|)
                                      serves both u_B and u_B'), else m2l_pairs */
} nnca_stats;

/* Build the H^2 representation of A(i, j) = K(p_i, q_j) (Sec. 2, Sec. 3).
 *  cfg    host pointer; validated (d, leaf_size, eta2, aca_tol > 0, kernel,
 *         symmetric == 1).
 *  P      device pointer, nP points (layout), FP64, all finite.
 *  Q      device pointer or NULL. NULL, or Q == P with nQ == nP: the symmetric
 *         case of Sec. 5 (A on P x P, the diagonal taking kparam[2]).
 *         Otherwise nQ >= 1 points of Q in the same layout: the representation
 *         is built on the union [P; Q] (nP + nQ < 2^31 points; P and Q may share
 *         coordinates, which count as distinct points), and the products of the
 *         handle return A(P, Q) x as the P rows of the union matrix applied to
 *         [0; x]: the same nested bases and ACA tolerance, at the cost of the
 *         union's size (the paper's separate incoming and outgoing bases, Eqs.
 *         15-18, are not built). Such a handle serves nnca_matvec and
 *         nnca_matvec_host only; the batched, no-allocation and gradient calls
 *         return NNCA_ERR_UNSUPPORTED for it. Its statistics describe the union.
 *  out    host pointer that receives the handle (NULL on failure).
 * Synchronises `stream`. nP >= 1 and nP < 2^31. */
nnca_status nnca_build(const nnca_config *cfg, const double *P, int64_t nP, const double *Q, int64_t nQ,
                       int layout, void *stream, nnca_handle *out);

/* y = A~ x for nrhs right-hand sides. x, y: device pointers, element type
 * dtype (NNCA_F64 or NNCA_F32), column r at [r*ld .. r*ld + n). y is
 * overwritten. For a P != Q handle x holds nQ entries and y nP entries per
 * column (ld >= max(nP, nQ)), and the call also uses a workspace of two union
 * vectors per right-hand side. precision: NNCA_PREC_FP64 (all arithmetic in FP64),
 * NNCA_PREC_FP32 (kernel evaluations and contractions in FP32 with
 * cell-relative coordinates and compensated accumulation across cells), or a
 * tensor-core form (NNCA_PREC_TF32X3, NNCA_PREC_TF32, NNCA_PREC_BF16).
 * Asynchronous on `stream`. The first call with a larger nrhs than before
 * allocates the handle's workspace (so make that call before capturing a
 * stream into a graph). */
nnca_status nnca_matvec(nnca_handle h, const void *x, void *y, int64_t nrhs, int64_t ld, int dtype,
                        int precision, void *stream);

/* Same product from and to HOST buffers: copies x to the device, runs
 * nnca_matvec, copies y back, and synchronises `stream` before returning. */
nnca_status nnca_matvec_host(nnca_handle h, const void *x_host, void *y_host, int64_t nrhs, int64_t ld,
                             int dtype, int precision, void *stream);

/* The product for ONE right-hand side with no device allocation. The paper
 * has no counterpart; this is a library service. nnca_matvec allocates its
 * workspace with cudaMalloc on its first call; callers that cannot allocate
 * then (a fixed device-memory budget already given to their own allocator, or
 * latency-critical loops that cannot accept cudaMalloc's implicit device
 * synchronisation) call this instead. The workspace comes from one file-scope
 * device array of NNCA_NOALLOC_BYTES that every GPU loading the library holds
 * until exit. Limit: 12 * n + 20 * pivots + 256 bytes must fit in it, else
 * NNCA_ERR_INVALID_ARG with the sizes in nnca_last_error (pivots:
 * nnca_stats.n_pivots). The first call on a device looks the array's address
 * up (cudaGetSymbolAddress): make it before any stream capture. All calls share
 * the array and it keeps the last call's contents; each call clears what must
 * start at zero, and calls that overlap on the GPU race. Profiling must be off.
 * x, y, ld, dtype, precision, stream: as for nnca_matvec with nrhs = 1. */
#define NNCA_NOALLOC_BYTES (64u << 20)
nnca_status nnca_matvec_noalloc(nnca_handle h, const void *x, void *y, int64_t ld, int dtype, int precision,
                                void *stream);

/* Products of `count` independent handles at once (batched uneven problems; the
 * paper has no counterpart). Product k is y[k] = A_k x[k] for handle h[k] with
 * leading dimension ld[k] (>= that handle's n); nrhs, dtype and precision are
 * shared. The products run on internal worker streams forked from `stream` and
 * joined back to it (event waits), so small problems overlap on the GPU and the
 * call as a whole is ordered on `stream`. Capturing `stream` into a CUDA graph
 * captures all of it: make one uncaptured call first with the same handles and
 * nrhs (it allocates the handles' workspaces and the worker streams). A handle
 * may appear at most once per call. Errors: NNCA_ERR_INVALID_ARG for NULL
 * arrays, count < 1 or > 4096, a repeated handle, or any argument nnca_matvec
 * would reject (nnca_last_error(NULL) names the first failing product). */
nnca_status nnca_matvec_batch(const nnca_handle *h, int count, const void *const *x, void *const *y,
                              const int64_t *ld, int64_t nrhs, int dtype, int precision, void *stream);

/* Gradient of L = sum_r g_r^T A~ x_r with respect to the points and the kernel
 * parameter h = kparam[1], with every index set of the build held (tree, lists,
 * pivots t^{B,i}, s^{B,i}: "pivots fixed"); A~ moves with the points through its
 * kernel entries and through the bases X_B = A_{t~ sigma} (A_{tau sigma})^{-1}
 * (Sec. 2.3.1, Eqs. 11 and 14), differentiated as
 * dX = (dA_{t~ sigma} - X dA_{tau sigma}) (A_{tau sigma})^{-1}. The derivative in x
 * is A~ g (the product, A~ being symmetric).
 *   x, g    device FP64, nrhs right-hand sides, column r at [r*ld .. r*ld + n),
 *           caller's point order;
 *   grad_p  device FP64, n x d row-major (grad_p[i*d + k]), caller's order;
 *           overwritten;
 *   grad_h  device FP64 [1] or NULL; dL/dh (0 for the log and 1/r kernels).
 * Kernels: NNCA_K_LOG, NNCA_K_INV_R, NNCA_K_GAUSS, NNCA_K_MATERN (else
 * NNCA_ERR_UNSUPPORTED). FP64 throughout (the products of x and g run in FP64).
 * Synchronises `stream`; allocates scratch for the call. */
nnca_status nnca_gradient(nnca_handle h, const double *x, const double *g, int64_t nrhs, int64_t ld, double *grad_p,
                          double *grad_h, void *stream);

/* Testing hook for the bounded waits of the FP32 product (the paper has no
 * counterpart; a failure-handling service). The FP32 M2L and near-field kernels
 * wait on shared-memory barriers of their own thread block for their own bulk
 * copies; a wait that runs out of its clock budget sets bit 16 of
 * nnca_stats.device_status, lets the block's copies in flight land and returns,
 * so the context stays usable and the product is reported invalid.
 *   wait_limit_clocks > 0 sets the budget of one wait (<= 0: the default, 2^31);
 *   extra_tx_bytes > 0 adds that many bytes to every staging round's expected
 *     byte count, more than its copies deliver, so that every wait on a round
 *     runs out although every copy lands (0: normal operation).
 * Applies on the current device to every product launched after the call;
 * synchronises the device. Products run with extra_tx_bytes > 0 are invalid:
 * restore (0, 0) before further use. */
nnca_status nnca_set_wait_test(int64_t wait_limit_clocks, unsigned extra_tx_bytes);

/* Free every device and host resource of the handle (NULL is a no-op).
 * Synchronises the device first. */
void nnca_destroy(nnca_handle h);

/* Copy the statistics. Synchronises with the profiled products first. */
nnca_status nnca_get_stats(nnca_handle h, nnca_stats *out);

/* Turn per-pass timing of nnca_matvec on (1) or off (0); turning it on
 * clears the accumulated pass_ms. While on, every product records CUDA events
 * between its passes on the caller's stream (no host synchronisation in the
 * product itself). */
nnca_status nnca_set_profiling(nnca_handle h, int on);

/* Copy one internal array to host memory, for inspection and tests. If buf
 * is NULL only *bytes is set. Otherwise at most cap bytes are written and
 * *bytes receives the array's size. Point indices are Morton-sorted
 * positions; cell ids are global (level by level, as in LEVEL_BASE).
 *   PERM        int64[n]        original index of sorted position
 *   KEYS        uint64[n]       sorted Morton keys
 *   LEVEL_BASE  int64[kappa+2]  first cell id of each level
 *   CKEY        uint64[ncell]   cell key (prefix of its level)
 *   CBEG, CEND  int64[ncell]    sorted point range of the cell
 *   CPAR        int64[ncell]    parent cell id (-1 for the root)
 *   CCH_BEG/END int64[ncell]    children cell range
 *   NB_OFF      int64[ncell+1]  CSR offsets of N(B); NB_IDX int64 cell ids
 *   IL_OFF      int64[ncell+1]  CSR offsets of IL(B); IL_IDX int64 cell ids
 *   PIV_OFF     int64[ncell+1]  CSR offsets of the pivots (ranks)
 *   PIV_ROW     int64[npiv]     t^{B,i} (sorted positions)
 *   PIV_COL     int64[npiv]     s^{B,i} (sorted positions; -1 for pass-through cells)
 *   PASSTHRU    int64[ncell]    1 if the cell passed all its candidates up (no
 *                               far-field candidates, or an ACA that used up
 *                               every candidate column with rows left)
 *   CAND_OFF    int64[ncell+1]  CSR offsets of the candidate rows t~^{B,i}
 *   OP_OFF      int64[ncell+1]  offsets of the per-cell operators
 *   OP          double[...]     per cell |t~| x r row-major: U_B (leaf) or
 *                               the stacked C_{B_c B} (non-leaf)          */
enum {
    NNCA_EXPORT_PERM = 0, NNCA_EXPORT_KEYS, NNCA_EXPORT_LEVEL_BASE, NNCA_EXPORT_CKEY,
    NNCA_EXPORT_CBEG, NNCA_EXPORT_CEND, NNCA_EXPORT_CPAR, NNCA_EXPORT_CCH_BEG, NNCA_EXPORT_CCH_END,
    NNCA_EXPORT_NB_OFF, NNCA_EXPORT_NB_IDX, NNCA_EXPORT_IL_OFF, NNCA_EXPORT_IL_IDX,
    NNCA_EXPORT_PIV_OFF, NNCA_EXPORT_PIV_ROW, NNCA_EXPORT_PIV_COL, NNCA_EXPORT_PASSTHRU,
    NNCA_EXPORT_CAND_OFF, NNCA_EXPORT_OP_OFF, NNCA_EXPORT_OP
};
nnca_status nnca_export(nnca_handle h, int what, void *buf, int64_t cap, int64_t *bytes);

/* Message of the last failure on this handle (or, for h == NULL, of the
 * last failed call without a handle on this thread). Never NULL. */
const char *nnca_last_error(nnca_handle h);
const char *nnca_status_string(nnca_status s);

#ifdef __cplusplus
}
#endif
#endif /* NNCA_H */
