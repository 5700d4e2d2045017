// Internal definitions of the NNCA CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/nnca.h"

namespace nnca {

// ---------------------------------------------------------------------------
// Errors: internal code throws nnca::Error; the C ABI converts it to a status.
struct Error : std::runtime_error {
    nnca_status status;
    Error(nnca_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define NNCA_CUDA(call)                                                                     \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            throw ::nnca::Error(e_ == cudaErrorMemoryAllocation ? NNCA_ERR_OOM : NNCA_ERR_CUDA, \
                                std::string(#call) + ": " + cudaGetErrorString(e_));       \
        }                                                                                   \
    } while (0)

#define NNCA_LAUNCH_CHECK() NNCA_CUDA(cudaGetLastError())

#define NNCA_REQUIRE(cond, st, msg)                     \
    do {                                                \
        if (!(cond)) throw ::nnca::Error((st), (msg));  \
    } while (0)

// Device-side status word bits (never a trap: a kernel that finds a problem
// records it and returns; the host reads the word and reports it).
enum : unsigned {
    DEV_OK = 0,
    DEV_POOL_EXHAUSTED = 1u,   // a cell ran out of ACA scratch: it is retried
    DEV_BAD_INDEX = 2u,        // an index failed a bounds check
    DEV_ZERO_PIVOT = 4u,       // the LU of a pivot block met an exact zero pivot
    DEV_LIST_OVERFLOW = 8u,
    DEV_WAIT_TIMEOUT = 16u     // a bounded wait on an asynchronous copy ran out
};

inline unsigned ceil_div(unsigned long long a, unsigned long long b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Kernel functions K(x, y). Parameters passed by value to every kernel.
struct KParams {
    int kind;
    int d;
    double s;      // scale
    double h;      // h or a
    double diag;   // A(i, i)
    float sf, hf;
};

// FP64 form that performs exactly the IEEE operations of the oracle's kernel
// definition (each operation rounded on its own, correctly rounded sqrt and
// division), so that pivot decisions are reproducible bit for bit. The log and
// exp kernels use CUDA's log/exp, which may differ from the host library in
// the last place.
__device__ __forceinline__ double kern_exact(const KParams &kp, const double *x, const double *y) {
    double r2 = 0.0;
    if (kp.kind != NNCA_K_SEPARABLE && kp.kind != NNCA_K_POLY2) {
        for (int k = 0; k < kp.d; ++k) {
            double t = __dsub_rn(x[k], y[k]);
            r2 = __dadd_rn(r2, __dmul_rn(t, t));
        }
    }
    switch (kp.kind) {
    case NNCA_K_LOG:
        if (r2 == 0.0) return 0.0;
        return __dmul_rn(kp.s, log(__dsqrt_rn(r2)));
    case NNCA_K_INV_R:
        if (r2 == 0.0) return 0.0;
        return __ddiv_rn(kp.s, __dsqrt_rn(r2));
    case NNCA_K_GAUSS:
        return __dmul_rn(kp.s, exp(__ddiv_rn(-r2, __dmul_rn(__dmul_rn(2.0, kp.h), kp.h))));
    case NNCA_K_MATERN:
        return __dmul_rn(kp.s, exp(__ddiv_rn(-__dsqrt_rn(r2), kp.h)));
    case NNCA_K_PAPER_I: {
        double r = __dsqrt_rn(r2);
        if (r == 0.0) return 0.0;
        if (r < kp.h)
            return __dmul_rn(kp.s, __ddiv_rn(__dmul_rn(r, __dsub_rn(log(r), 1.0)),
                                             __dmul_rn(kp.h, __dsub_rn(log(kp.h), 1.0))));
        return __dmul_rn(kp.s, __ddiv_rn(log(r), log(kp.h)));
    }
    case NNCA_K_PAPER_II: {
        double r = __dsqrt_rn(r2);
        if (r < kp.h) return __dmul_rn(kp.s, __ddiv_rn(r, kp.h));
        return __dmul_rn(kp.s, __ddiv_rn(kp.h, r));
    }
    case NNCA_K_SEPARABLE: {
        double fx = 1.0, fy = 1.0;
        for (int k = 0; k < kp.d; ++k) {
            fx = __dadd_rn(fx, x[k]);
            fy = __dadd_rn(fy, y[k]);
        }
        return __dmul_rn(kp.s, __dmul_rn(fx, fy));
    }
    case NNCA_K_POLY2: {
        double t = 1.0;
        for (int k = 0; k < kp.d; ++k) t = __dadd_rn(t, __dmul_rn(x[k], y[k]));
        return __dmul_rn(kp.s, __dmul_rn(t, t));
    }
    default:
        return 0.0;
    }
}

// K as a function of r^2 (radial kernels) or of the points (the two
// non-radial test kernels), FP64, for the product. Contraction allowed.
__device__ __forceinline__ double kern64_r2(const KParams &kp, double r2) {
    switch (kp.kind) {
    case NNCA_K_INV_R: return r2 > 0.0 ? kp.s * rsqrt(r2) : 0.0;
    case NNCA_K_LOG: return r2 > 0.0 ? 0.5 * kp.s * log(r2) : 0.0;
    case NNCA_K_GAUSS: return kp.s * exp(-r2 / (2.0 * kp.h * kp.h));
    case NNCA_K_MATERN: return kp.s * exp(-sqrt(r2) / kp.h);
    case NNCA_K_PAPER_I: {
        if (!(r2 > 0.0)) return 0.0;
        double r = sqrt(r2);
        if (r < kp.h) return kp.s * (r * (log(r) - 1.0)) / (kp.h * (log(kp.h) - 1.0));
        return kp.s * log(r) / log(kp.h);
    }
    case NNCA_K_PAPER_II: {
        double r = sqrt(r2);
        return r < kp.h ? kp.s * r / kp.h : kp.s * kp.h / r;
    }
    default: return 0.0;
    }
}

__device__ __forceinline__ float kern32_r2(const KParams &kp, float r2) {
    switch (kp.kind) {
    case NNCA_K_INV_R: return r2 > 0.f ? kp.sf * rsqrtf(r2) : 0.f;
    case NNCA_K_LOG: return r2 > 0.f ? 0.5f * kp.sf * __logf(r2) : 0.f;
    case NNCA_K_GAUSS: return kp.sf * __expf(-r2 / (2.f * kp.hf * kp.hf));
    case NNCA_K_MATERN: return kp.sf * __expf(-sqrtf(r2) / kp.hf);
    case NNCA_K_PAPER_I: {
        if (!(r2 > 0.f)) return 0.f;
        float r = sqrtf(r2);
        if (r < kp.hf) return kp.sf * (r * (logf(r) - 1.f)) / (kp.hf * (logf(kp.hf) - 1.f));
        return kp.sf * logf(r) / logf(kp.hf);
    }
    case NNCA_K_PAPER_II: {
        float r = sqrtf(r2);
        return r < kp.hf ? kp.sf * r / kp.hf : kp.sf * kp.hf / r;
    }
    default: return 0.f;
    }
}

inline bool kernel_is_radial(int kind) { return kind != NNCA_K_SEPARABLE && kind != NNCA_K_POLY2; }

// The FP32 M2L runs one thread block of M2L_GROUP_WARPS warps per group of
// sibling target cells; a group item holds at most M2L_GROUP_TARGETS
// consecutive targets (items of M2L_GROUP_TARGETS and a remainder), and its
// warps take m2l_warp_targets(targets) consecutive targets each (two per lane
// on half as many lanes; the warp's other lane groups split the sources), so
// that the four warps of an item stay busy for about the same time. Source cells
// arrive in staging rounds of at most M2L_STAGE_RECS cells and M2L_STAGE_CAP
// sources (padded counts), which bounds the largest rank it takes.
constexpr int M2L_GROUP_WARPS = 4;
constexpr int M2L_WARP_TARGETS = 64;
constexpr int M2L_GROUP_TARGETS = M2L_WARP_TARGETS * M2L_GROUP_WARPS;
// targets per warp of an item of nt targets: the least power of two (at least
// 2) with four warps covering nt, at most M2L_WARP_TARGETS
__host__ __device__ inline int m2l_warp_targets(int nt) {
    int s = 2;
    while (s * M2L_GROUP_WARPS < nt && s < M2L_WARP_TARGETS) s <<= 1;
    return s;
}
constexpr int M2L_STAGE_CAP = 512;
constexpr int M2L_STAGE_RECS = 32;
constexpr int M2L_STAGE_BUFS = 4;
// right-hand sides of one FP32 M2L pass with several (their weights travel as
// [w(2q, r) w(2q+1, r) w(2q, r+1) w(2q+1, r+1)] float4 pairs per source pair q)
constexpr int M2L_RHS = 4;
// The symmetric FP32 M2L (one right-hand side) serves each unordered pair of
// neighbouring parents {P, Q} once: a kernel value f(|s - t|) feeds the row sum
// of target t and the column sum of source s. Its rounds hold at most
// M2L_SYM_CAP padded sources (so the per-warp column sums of the rounds in
// flight fit in shared memory beside the staged sources).
constexpr int M2L_SYM_CAP = 256;
// source pairs of one chunk of the FP32 M2L pair loop when a whole warp shares it
// (two pairs per step, M2L_FOLD steps between folds into the compensated totals)
constexpr int M2L_CHUNK_PAIRS = 16;
// The FP32 near field runs independent warps, NEAR_WARPS per block, one leaf
// (up to 64 targets) per work item. The points of N(B) arrive in rounds of at
// most NEAR_RECS cells and NEAR_CAP point pairs through NEAR_BUFS buffers per
// warp, which bounds the largest leaf it takes (2 * NEAR_CAP points).
constexpr int NEAR_WARPS = 4;
constexpr int NEAR_CAP = 48;                  // point pairs of hi/lo coordinates per buffer
constexpr int NEAR_UNITS = 4 * NEAR_CAP;      // buffer size in 16-byte units
constexpr int NEAR_RECS = 16;
constexpr int NEAR_BUFS = 3;
// coordinate of a padding source: far from every target, weight 0
constexpr float FAR_AWAY = 1.0e18f;
// sources of a cell padded to a multiple of four (two packed pairs)
__host__ __device__ inline int m2l_padded(int rank) { return (rank + 3) & ~3; }

// ---------------------------------------------------------------------------
// Handle.
struct Handle;

// Device allocation tracked by the handle (freed by nnca_destroy).
void *dev_alloc(Handle *h, size_t bytes);
void dev_free(Handle *h, void *p);
template <class T> T *dalloc(Handle *h, size_t count) { return (T *)dev_alloc(h, sizeof(T) * (count ? count : 1)); }

// Scratch allocation owned by the caller of a build step (freed explicitly).
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() { for (void *p : ptrs) cudaFree(p); }
    template <class T> T *get(size_t count) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * (count ? count : 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(NNCA_ERR_OOM, std::string("scratch cudaMalloc: ") + cudaGetErrorString(e));
        }
        ptrs.push_back(p);
        return (T *)p;
    }
    void release(void *p) {
        for (auto &q : ptrs) if (q == p) { cudaFree(q); q = nullptr; }
    }
};

struct Handle {
    nnca_config cfg{};
    KParams kp{};
    uint64_t uid = 0;                 // unique per built handle (keys of cross-problem caches)
    int d = 0, lmax = 0, kappa = 0, lmin = 0;
    int64_t n = 0;
    double corner[4] = {0, 0, 0, 0};
    double side = 1.0;
    cudaStream_t stream = nullptr;

    // tree (device)
    int32_t *perm = nullptr;      // [n] original index of sorted position
    uint64_t *keys = nullptr;     // [n]
    double *xs = nullptr;         // [d][n] sorted coordinates (SoA)
    int64_t ncell = 0;
    std::vector<int64_t> level_base;   // host, kappa + 2 entries
    uint64_t *ckey = nullptr;
    int32_t *cbeg = nullptr, *cend = nullptr, *cpar = nullptr, *cch_beg = nullptr, *cch_end = nullptr;
    int32_t *ccoord = nullptr;    // [d][ncell] integer cell coordinates at the cell's level

    // lists (device CSR over global cell ids)
    int32_t *nb_off = nullptr, *nb_idx = nullptr, *il_off = nullptr, *il_idx = nullptr;
    int64_t n_nb = 0, n_il = 0;

    // pivots and operators (device)
    int32_t *piv_off = nullptr, *piv_row = nullptr, *piv_col = nullptr, *passthru = nullptr;
    int64_t *cand_off = nullptr, *op_off = nullptr;
    double *op = nullptr;
    int64_t npiv = 0, nop = 0;
    std::vector<int32_t> h_piv_off;    // host copy (ncell + 1)

    // product data (device)
    double *ccen = nullptr;       // [d][ncell] cell centres
    float *ccen_hi = nullptr;     // [d][ncell] centre rounded to float
    float *ccen_lo = nullptr;     // [d][ncell] centre - hi, rounded to float
    double *pv64 = nullptr;       // [d][npiv] pivot coordinates
    float *pv32 = nullptr;        // [d][npiv] pivot coordinates relative to their cell centre
    float *xs32 = nullptr;        // [d][n] point coordinates relative to their leaf centre
    int32_t *leaf_of = nullptr;   // [n] leaf (global id) of each sorted position
    int32_t *m2l_tgt = nullptr;   // cells with a non-empty IL, heaviest first
    int64_t n_m2l_tgt = 0;
    int32_t *leaf_order = nullptr;  // leaves, heaviest near field first
    int64_t nleaf = 0;
    // FP32 product: packed data and work items (cell, first target, count) per slice count 2^s
    int2 *prange = nullptr;       // [ncell] (first pivot, rank)
    float4 *pv4 = nullptr;        // [npiv] pivot coordinates relative to the cell centre
    float4 *chi4 = nullptr, *clo4 = nullptr;   // [ncell] centre as float hi + lo
    float4 *xh4 = nullptr, *xl4 = nullptr;     // [n] point coordinates as float hi + lo
    // FP32 M2L: items (parent, first target | targets << 16, first plan record,
    // plan records), heaviest first; plan records (cell, first source pair,
    // staging slot | pairs << 11 | child mask << 22, cells in the round or 0);
    // sources of every cell as pairs [x0 x1 y0 y1][z0 z1 w0 w1] relative to the
    // cell centre, padded to m2l_padded(rank) with far-away sources of weight 0
    // (the products write the weights w), from pair spk_off[cell]
    int4 *m2l_groups = nullptr;
    int n_m2l_groups = 0;
    std::vector<int64_t> h_m2l_weight;   // host: pairs of each item (cross-problem ordering)
    int *m2l_next = nullptr;      // item counter of the FP32 M2L launch
    // heavy items are split at staging-round boundaries: such a piece writes
    // its partial sums to m2l_parts[slot][0, targets), and a combine pass adds the
    // pieces of each split (u offset, targets, first slot, pieces) in order
    int *m2l_item_part = nullptr;   // per item: part slot, or -1 (writes u)
    double *m2l_parts = nullptr;
    int4 *m2l_split = nullptr;
    int n_m2l_split = 0;
    // FP32 near field: points of every leaf as pairs [xh0 xh1 yh0 yh1][zh0 zh1 w0 w1]
    // [xl0 xl1 yl0 yl1][zl0 zl1 0 0] (absolute coordinates as float hi + lo,
    // padded to m2l_padded(points) with far-away points of weight 0; the
    // products write the weights) from pair ppk_off[cell]; per-leaf staging plans
    // (cell, first pair, slot in 16-byte units | pairs << 11 | own leaf << 22 |
    // adjacent << 23, cells in the round or 0) and items (leaf, first target | targets << 16 | groups << 24, first
    // record, records) for 2 and 3 targets per lane
    float4 *ppk = nullptr;
    float4 *ppl = nullptr;        // the same points as [x0 x1 y0 y1][z0 z1 w0 w1] relative to the leaf centre
    int32_t *ppk_off = nullptr;   // [ncell + 1], pairs (the same for ppk and ppl)
    int4 *near_plan = nullptr;
    int64_t n_near_plan = 0;
    int4 *near_items[2] = {nullptr, nullptr};   // by targets per lane (2, 3)
    int n_near_items[2] = {0, 0};
    int *near_next = nullptr;                    // [2] item counters
    bool near_packed = false;     // false: leaves too large, the ring kernel serves them
    // FP32 near field of M2L_RHS right-hand sides at once: the weights of every
    // packed point pair for the four, [w0(p0) w0(p1) w1(p0) w1(p1)][w2(p0) w2(p1)
    // w3(p0) w3(p1)] (2 float4 per pair, pairs as in ppk), and items of at most
    // 64 targets (leaf, first target | targets << 16 | groups << 24, first record,
    // records), two targets per lane
    float4 *pw4 = nullptr;
    float4 *pw8 = nullptr;        // the same for eight right-hand sides (4 float4 per pair)
    float4 *spw_multi = nullptr;  // spw of each group of a grouped FP32 pass ([group][pairs][M2L_RHS / 2])
    int spw_multi_groups = 0;
    int64_t near_pairs = 0;       // packed point pairs (ppk)
    int4 *near_items4 = nullptr;
    int n_near_items4 = 0;
    const char *m2l_fp32_unsupported = nullptr;   // why the FP32 M2L cannot run, or null
    int4 *m2l_plan = nullptr;
    float4 *m2l_plan_sh = nullptr;   // per plan record: c_Y - c_P rounded to float
    int64_t n_m2l_plan = 0;
    float4 *spk = nullptr;
    int32_t *spk_off = nullptr;   // [ncell + 1]
    float4 *spw = nullptr;        // [pairs][M2L_RHS / 2]: weights of a pass with M2L_RHS right-hand sides
    int64_t n_spk_pairs = 0;
    // Symmetric FP32 M2L (null sym_items: not available, the full form runs):
    // the plan of parent P lists only the children of neighbours Q > P (cell
    // index), in rounds of at most M2L_SYM_CAP sources; items and split pieces as
    // for the full form. Item i writes the column sums of its staged sources, in
    // staging order, to sym_col[sym_item_col[i] ...]; cell Y gathers its column
    // sums from the slots sym_ent[sym_ent_off[Y] .. sym_ent_off[Y + 1]) (each the
    // slot of Y's first pivot) in that fixed order.
    int4 *sym_plan = nullptr;
    float4 *sym_plan_sh = nullptr;
    int64_t n_sym_plan = 0;
    bool sym_unroll = true;       // symmetric M2L: unrolled pair loop (long staged records) or counted loop
    int4 *sym_items = nullptr;
    int n_sym_items = 0;
    int *sym_item_part = nullptr;
    int *sym_item_col = nullptr;
    double *sym_parts = nullptr;
    int4 *sym_split = nullptr;
    int n_sym_split = 0;
    float *sym_col = nullptr;
    int64_t n_sym_col = 0;
    int32_t *sym_ent_off = nullptr;   // [ncell + 1]
    int32_t *sym_ent = nullptr;
    int2 *sym_tasks = nullptr;        // (cell with slots, first of 32 pivots) per warp of the column pass
    int n_sym_tasks = 0;
    // tensor-core M2L of many right-hand sides: items (parent, first target |
    // targets << 16, first record, records) of at most 64 targets over the full
    // plan (m2l_plan), heaviest first
    bool no_alloc = false;            // inside nnca_matvec_noalloc: no path may allocate
    int64_t *f64_slot_of = nullptr;   // symmetric FP64 M2L: first column slot of each IL entry (or its partner's)
    double *f64_slots = nullptr;
    int4 *tc_items = nullptr;
    int n_tc_items = 0;
    int2 *leaf_items[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int n_leaf_items[5] = {0, 0, 0, 0, 0};

    // product workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t ws_nrhs = 0;
    void *tc_ws = nullptr;        // workspace of the tensor-core forms (passes of 64 right-hand sides)
    size_t tc_ws_bytes = 0;
    void *host_stage = nullptr;   // device buffers for nnca_matvec_host
    size_t host_stage_bytes = 0;
    // P != Q: the representation is built on the union [P; Q] (n = n_rows + n_cols
    // points, caller order P then Q); a product takes x on Q, embeds it as [0; x],
    // runs the symmetric product and returns its rows on P
    bool pq = false;
    int64_t n_rows = 0, n_cols = 0;
    void *pq_buf = nullptr;
    size_t pq_buf_bytes = 0;

    // per-pass profiling of the product
    bool profile = false;
    std::vector<cudaEvent_t> prof_events;   // 6 per profiled product, pending
    std::vector<cudaEvent_t> event_pool;
    int64_t launches = 0;

    std::vector<void *> allocs;
    std::string last_error;
    nnca_stats stats{};
    unsigned *dev_status = nullptr;   // device status word
};

// Build steps (tree.cu, lists.cu, aca.cu) and product (matvec.cu).
void build_tree(Handle *h, const double *P, int layout);
void build_lists(Handle *h);
void build_pivots(Handle *h);   // pivots, bases, global pivot/operator arrays
void build_finish(Handle *h);   // data of the product: centres, FP32 coordinates, work lists
void matvec(Handle *h, const void *x, void *y, int64_t nrhs, int64_t ld, int dtype, int precision);
// Batched FP32 products of independent handles (matvec.cu): passes of four
// right-hand sides synchronised across the problems, the M2L of each pass one
// launch per kernel family over a cross-problem item list; the other passes per
// problem on the worker streams. Returns false (and does nothing) if a handle
// cannot take this path.
bool matvec_batch_fp32(Handle *const *hs, int count, const void *const *x, void *const *y, const int64_t *ld,
                       int64_t nrhs, int dtype, cudaStream_t s, cudaStream_t *workers, int nworkers, cudaEvent_t fork,
                       cudaEvent_t *join);
// frees the cross-problem item lists of every handle set that contains handle uid
void release_cross_plans(uint64_t uid);
// wait budget and extra expected bytes of the FP32 kernels' staging (nnca_set_wait_test)
void set_wait_test(int64_t wait_limit_clocks, unsigned extra_tx_bytes);
void set_wait_test_tc(int64_t wait_limit_clocks, unsigned extra_tx_bytes);
// Tensor-core M2L (m2l_tc.cu) of one pass of nr <= tc_rhs_per_pass() right-hand
// sides: w and u right-hand-side major FP64 (nr rows of npiv); tcws holds
// tc_workspace_floats(h) floats. mode: NNCA_PREC_TF32X3, NNCA_PREC_TF32 or NNCA_PREC_BF16.
// Gradient of sum_r g_r^T A~ x_r in the points (caller order, n x d) and in
// kparam[1], pivots fixed (grad.cu); x, g FP64 device, nrhs columns of ld.
// Synchronises the handle's stream.
void gradient(Handle *h, const double *x, const double *g, int64_t nrhs, int64_t ld, double *grad_p, double *grad_h);
int tc_rhs_per_pass();
size_t tc_workspace_floats(const Handle *h);
void m2l_tensor(Handle *h, int mode, int nr, const double *w, double *u, float *tcws);

// Exclusive scan of n uint32/int64 values (scan.cu). out may alias in.
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, Scratch &scr);
int64_t scan_total_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, Scratch &scr);

unsigned read_status(Handle *h);
// true for device (or managed) memory; false for host memory and unknown pointers
bool is_device_ptr(const void *p);
// Record the profiling event that ends pass `slot` (0 = start of the product).
void prof_mark(Handle *h, int slot);

}  // namespace nnca

// The opaque handle of the C ABI is the library's Handle.
struct nnca_handle_s : nnca::Handle {};
