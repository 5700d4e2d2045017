// M2L of many right-hand sides on the tensor cores (Sec. 4 step 3, Sec. 3 step 2).
//
// For one pass of up to TC_RHS right-hand sides the transverse pass is a set of
// dense contractions: for the targets t of a group of sibling cells (the pivots
// of the children of one parent P) and the sources s of the children of N(P)
// (the pivots of every cell Y admissible for the target's cell, Table 1),
//
//     u(t, r) += sum_s K(t, s) w(s, r),        K(t, s) = f(|p_t - p_s|) or 0,
//
// with K evaluated on the fly (zero where Y is not in the target's interaction
// list) and w the multipole coefficients of all right-hand sides. One thread
// block serves an item of at most TC_TGT targets. Per chunk of 32 sources:
//   - a staging warp copies the sources' coordinates and the packed weights
//     W^T (right-hand side x source, tf32 hi and lo parts) into shared memory
//     with bulk asynchronous copies (TMA), tracked by an mbarrier;
//   - four warps evaluate K for every (target, source) pair of the chunk in
//     FP32 (one MUFU operation per pair), split each value into tf32 hi and lo
//     parts and store them as the MMA's B operand;
//   - one thread issues tcgen05.mma (kind::tf32, M = 128, N = the targets
//     rounded up to a power of two of at least 16, K = 8 per instruction),
//     D[r][t] += W^T[r][s] K[t][s], accumulating in tensor memory:
//       3xTF32 (NNCA_PREC_TF32X3): Whi Khi + Whi Klo + Wlo Khi, the split of
//         Ootomo & Yokota (2022), which keeps about 22 bits of each operand;
//       TF32 (NNCA_PREC_TF32): Whi Khi;
//       BF16 (NNCA_PREC_BF16): both operands rounded to bfloat16 (exact in
//         tf32), one product per pair, FP32 accumulation.
// The main products Whi Khi accumulate in one tensor-memory accumulator D that
// two warps read out (tcgen05.ld) every TC_SEG_CHUNKS chunks and add into
// compensated float sums (two-sum) in shared memory; the correction products
// (about 2^-11 smaller) accumulate over the whole item in a second accumulator C.
// At the end of an item those two warps store u. D and C are double-buffered,
// so the MMAs of the next segment or item run while the last one is read.
// Rows 64..127 of the M = 128 instruction read the next quad's weights and are
// ignored.
//
// Every wait is bounded (g_wait_limit clocks); one that runs out sets
// DEV_WAIT_TIMEOUT, the block drains what it issued and returns, and frees
// its tensor memory.
#include <algorithm>

#include "nnca_internal.cuh"

namespace nnca {

namespace {

#include "dev_common.cuh"

constexpr int TC_RHS = 64;                    // right-hand sides of one pass: rows of W^T and of D
constexpr int TC_M = 128;                     // MMA M
constexpr int TC_TGT = 64;                    // targets of one item: MMA N up to 64
constexpr int TC_QPC = 8;                     // source quads (4 sources) per chunk: four K-steps of 8
constexpr int TC_STAGES = 2;
constexpr int TC_EVAL = 128;                  // evaluating threads (warps 0-3)
constexpr int TC_THREADS = TC_EVAL + 64;      // + staging warp (4) + MMA warp (5)
constexpr int TC_QF = TC_RHS * 4;             // floats of one quad of W^T: [8 row groups][8 rows][4 sources]
constexpr unsigned TC_TMEM_COLS = 4 * TC_TGT; // main and correction accumulators, two of each, TC_TGT columns each

// One pipeline stage: a chunk of TC_QPC source quads.
//   ahi/alo: W^T of the chunk, quad q at [q * TC_QF]: element (r, k) at
//            (r / 8) * 32 + (r % 8) * 4 + k  (K-major, no swizzle: core matrices
//            of 8 rows x 16 bytes; 128 bytes between row groups, TC_QF * 4
//            bytes between quads); one extra quad that rows 64..127 of the last
//            K-step read;
//   bhi/blo: K of the chunk, element (t, 4 q + k) at (t / 8) * 32 TC_QPC + q * 32 + (t % 8) * 4 + k
//            (1024 bytes between row groups, 128 bytes between quads).
struct __align__(128) TcStage {
    float ahi[(TC_QPC + 1) * TC_QF];
    float alo[(TC_QPC + 1) * TC_QF];
    float bhi[TC_TGT * TC_QPC * 4];
    float blo[TC_TGT * TC_QPC * 4];
    float4 src[TC_QPC][4];   // per quad the 4 sources, packed pairs [x0 x1 y0 y1][z0 z1 w0 w1]
    float4 sh[TC_QPC];       // c_Q - c_P of the quad's plan record
    int mask[TC_QPC];        // children of P that admit the quad's cell (0: empty quad)
    int item, flags, nq, pad;   // flags: TC_SEG_START, TC_SEG_END, TC_ITEM_FIRST, TC_ITEM_LAST, TC_END
};
constexpr int TC_SEG_START = 1, TC_SEG_END = 2, TC_END = 4, TC_ITEM_FIRST = 8, TC_ITEM_LAST = 16;

struct TcSmem {
    TcStage st[TC_STAGES];
    float2 acc[TC_TGT][TC_RHS];   // compensated sums (sum, error) of the item's flushed segments, target-major
    unsigned long long full[TC_STAGES], ready[TC_STAGES], freeb[TC_STAGES];
    unsigned long long dfull[2], dfree[2], cfree[2], done;
    unsigned tmem;
    int abort;
};

constexpr unsigned TC_A_LBO = TC_QF * 4;      // bytes between the quads (K direction) of W^T
constexpr unsigned TC_A_SBO = 128;            // bytes between row groups of W^T
constexpr unsigned TC_B_LBO = 128;            // bytes between the quads of K
constexpr unsigned TC_B_SBO = TC_QPC * 128;   // bytes between row groups (8 targets) of K

// ---- tcgen05 wrappers ---------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading (K direction) and
// stride (M/N direction) byte offsets, version 1, no swizzle
__device__ __forceinline__ unsigned long long sdesc(const void *p, unsigned lbo, unsigned sbo) {
    const unsigned a = smem_addr(p);
    return (unsigned long long)((a >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major, N and M
__host__ __device__ constexpr unsigned idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         unsigned acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
// arrive on bar once every tcgen05.mma this thread issued so far has completed
__device__ __forceinline__ void mma_commit(void *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
// 16 consecutive 32-bit columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                 "%14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// x rounded to bfloat16 (nearest even), as a float
__device__ __forceinline__ float to_bf16f(float x) {
    unsigned short b;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(b) : "f"(x));
    return __uint_as_float((unsigned)b << 16);
}

// the hi and lo operand parts of one value under the given mode
__device__ __forceinline__ void split_value(int mode, float v, float &hi, float &lo) {
    if (mode == NNCA_PREC_BF16) {
        hi = to_bf16f(v);
        lo = 0.f;
    } else {
        hi = to_tf32(v);
        lo = mode == NNCA_PREC_TF32X3 ? to_tf32(v - hi) : 0.f;
    }
}

__device__ __forceinline__ void tc_fail(TcSmem &S, unsigned *status) {
    atomicOr(status, DEV_WAIT_TIMEOUT);
    *(volatile int *)&S.abort = 1;
}

// ---- the kernel -----------------------------------------------------------------
// items: (parent P, first target | targets << 16, first plan record, records),
// targets the pivots of P's children from prange[cch_beg[P]].x on.
template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 2)
    k_m2l_tc(KParams kp, int mode, const int4 *items, int nitems, const int4 *plan, const float4 *plan_sh,
             const int32_t *cch_beg, const int32_t *cch_end, const int2 *prange, const float4 *pv4, const float4 *chi,
             const float4 *clo, const float4 *spk, const float *wq_hi, const float *wq_lo, int nrhs, float *utc,
             int seg_chunks, unsigned *status) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        // zero the stage buffers (a quad that is never staged reads as finite
        // values) and the compensated sums
        float4 *z = reinterpret_cast<float4 *>(S.st);
        for (int i = tid; i < (int)(sizeof(S.st) / sizeof(float4)); i += TC_THREADS) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 *za = reinterpret_cast<float4 *>(S.acc);
        for (int i = tid; i < (int)(sizeof(S.acc) / sizeof(float4)); i += TC_THREADS) za[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.ready[s], TC_EVAL);
            mbar_init(&S.freeb[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.dfull[b], 1);
            mbar_init(&S.dfree[b], 64);
            mbar_init(&S.cfree[b], 64);
        }
        mbar_init(&S.done, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(&S.tmem, TC_TMEM_COLS);
        tmem_relinquish();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = S.tmem;

    if (warp == 4) {
        // ---- staging: one lane walks the items' plan records in chunks of TC_QPC quads
        if (lane == 0) {
            unsigned cnt = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
                const int4 item = items[it];
                int k = item.z, ro = 0;
                const int kend = item.z + item.w;
                bool first = true;
                int chunk = 0;
                while (k < kend) {
                    const int s = cnt % TC_STAGES;
                    if (*(volatile int *)&S.abort ||
                        (cnt >= TC_STAGES && !mbar_wait(&S.freeb[s], (cnt / TC_STAGES - 1) & 1))) {
                        tc_fail(S, status);
                        ok = false;
                        break;
                    }
                    TcStage &T = S.st[s];
                    int nq = 0;
                    int pd[TC_QPC], pq[TC_QPC], pc[TC_QPC], np = 0;   // pieces: first quad here, global quad, quads
                    while (nq < TC_QPC && k < kend) {
                        const int4 rec = plan[k];
                        const int rq = ((rec.z >> 11) & 0x7ff) >> 1;
                        const int take = min(TC_QPC - nq, rq - ro);
                        const float4 sh = plan_sh[k];
                        const int msk = (rec.z >> 22) & 0xff;
                        for (int j = 0; j < take; ++j) {
                            T.sh[nq + j] = sh;
                            T.mask[nq + j] = msk;
                        }
                        pd[np] = nq;
                        pq[np] = (rec.y >> 1) + ro;
                        pc[np] = take;
                        ++np;
                        nq += take;
                        ro += take;
                        if (ro == rq) {
                            ++k;
                            ro = 0;
                        }
                    }
                    for (int j = nq; j < TC_QPC; ++j) T.mask[j] = 0;
                    T.item = it;
                    const bool last = k == kend;
                    T.flags = (first ? TC_ITEM_FIRST : 0) | (last ? TC_ITEM_LAST : 0) |
                              (chunk % seg_chunks == 0 ? TC_SEG_START : 0) |
                              (last || chunk % seg_chunks == seg_chunks - 1 ? TC_SEG_END : 0);
                    T.nq = nq;
                    first = false;
                    ++chunk;
                    const unsigned per_quad = 64u + (unsigned)TC_QF * 4u * (mode == NNCA_PREC_TF32X3 ? 2u : 1u);
                    mbar_arrive_tx(&S.full[s], per_quad * (unsigned)nq + g_stage_extra_tx);
                    for (int p = 0; p < np; ++p) {
                        bulk_g2s(&T.src[pd[p]][0], spk + 4 * (int64_t)pq[p], 64u * pc[p], &S.full[s]);
                        bulk_g2s(&T.ahi[pd[p] * TC_QF], wq_hi + (int64_t)pq[p] * TC_QF, 4u * TC_QF * pc[p], &S.full[s]);
                        if (mode == NNCA_PREC_TF32X3)
                            bulk_g2s(&T.alo[pd[p] * TC_QF], wq_lo + (int64_t)pq[p] * TC_QF, 4u * TC_QF * pc[p],
                                     &S.full[s]);
                    }
                    ++cnt;
                }
            }
            // let the copies of the last stages land (the latest phase of each
            // stage's barrier), then mark the end of the block's work. The end
            // marker arrives on a stage barrier only when that barrier's earlier
            // phases all completed: after a failure a phase may still wait for
            // bytes, and one more arrival would exceed its count; the consumers
            // then stop on their own bounded waits instead.
            bool clean = ok;
            for (unsigned j = cnt > (unsigned)TC_STAGES ? cnt - TC_STAGES : 0u; j < cnt; ++j)
                if (!mbar_wait(&S.full[j % TC_STAGES], (j / TC_STAGES) & 1)) {
                    tc_fail(S, status);
                    clean = false;
                }
            const int s = cnt % TC_STAGES;
            if (cnt >= TC_STAGES && !mbar_wait(&S.freeb[s], (cnt / TC_STAGES - 1) & 1)) {
                tc_fail(S, status);
                clean = false;
            }
            if (clean && !*(volatile int *)&S.abort) {
                S.st[s].flags = TC_END;
                mbar_arrive(&S.full[s]);
            }
        }
        __syncwarp();
    } else if (warp == 5) {
        // ---- MMA issue: one lane
        if (lane == 0) {
            unsigned cnt = 0, nseg = 0, nit = 0, acc = 0, accc = 0, idesc = idesc_tf32(TC_M, 16);
            for (;;) {
                const int s = cnt % TC_STAGES;
                if (!mbar_wait(&S.ready[s], (cnt / TC_STAGES) & 1)) {
                    tc_fail(S, status);
                    break;
                }
                TcStage &T = S.st[s];
                const int flags = T.flags;
                if (flags & TC_END) break;
                const int db = nseg & 1;
                const int ib = nit & 1;
                if (flags & TC_ITEM_FIRST) {
                    // the correction accumulator of item nit - 2 has been read out
                    if (nit >= 2 && !mbar_wait(&S.cfree[ib], ((nit >> 1) - 1) & 1)) {
                        tc_fail(S, status);
                        break;
                    }
                    const int nt = items[T.item].y >> 16;
                    int npad = 16;
                    while (npad < nt) npad <<= 1;
                    idesc = idesc_tf32(TC_M, npad);
                    accc = 0;
                }
                if (flags & TC_SEG_START) {
                    // the accumulator of segment nseg - 2 has been read out
                    if (nseg >= 2 && !mbar_wait(&S.dfree[db], ((nseg >> 1) - 1) & 1)) {
                        tc_fail(S, status);
                        break;
                    }
                    acc = 0;
                }
                tc_fence_after();
                // main products into D[db] (flushed per segment), the two
                // correction products (2^-11 smaller) into C[ib] (read per item)
                const unsigned d = tmem + (unsigned)(db * TC_TGT);
                const unsigned dc = tmem + (unsigned)((2 + ib) * TC_TGT);
                const int ks = (T.nq + 1) >> 1;
                for (int q = 0; q < ks; ++q) {
                    const unsigned long long ah = sdesc(&T.ahi[2 * q * TC_QF], TC_A_LBO, TC_A_SBO);
                    const unsigned long long bh = sdesc(&T.bhi[2 * q * 32], TC_B_LBO, TC_B_SBO);
                    mma_tf32(d, ah, bh, idesc, acc);
                    acc = 1;
                    if (mode == NNCA_PREC_TF32X3) {
                        const unsigned long long al = sdesc(&T.alo[2 * q * TC_QF], TC_A_LBO, TC_A_SBO);
                        const unsigned long long bl = sdesc(&T.blo[2 * q * 32], TC_B_LBO, TC_B_SBO);
                        mma_tf32(dc, ah, bl, idesc, accc);
                        accc = 1;
                        mma_tf32(dc, al, bh, idesc, 1);
                    }
                }
                mma_commit(&S.freeb[s]);
                if (flags & TC_SEG_END) {
                    mma_commit(&S.dfull[db]);
                    ++nseg;
                }
                if (flags & TC_ITEM_LAST) ++nit;
                ++cnt;
            }
            // every issued MMA done before the tensor memory is released
            mma_commit(&S.done);
            if (!mbar_wait(&S.done, 0)) tc_fail(S, status);
        }
        __syncwarp();
    } else {
        // ---- evaluation (warps 0-3) and, in warps 0-1, the results
        unsigned cnt = 0, nseg = 0, nit = 0;
        int nt = 0, npad = 16, g0 = 0, n = 0, c = 31;
        float tx = 0.f, ty = 0.f, tz = 0.f;
        for (;;) {
            const int s = cnt % TC_STAGES;
            if (!mbar_wait_warp(&S.full[s], (cnt / TC_STAGES) & 1)) {
                if (lane == 0) tc_fail(S, status);
                break;
            }
            TcStage &T = S.st[s];
            const int flags = T.flags;
            if (flags & TC_END) {
                mbar_arrive(&S.ready[s]);
                break;
            }
            if (flags & TC_ITEM_FIRST) {
                const int4 item = items[T.item];
                const int P = item.x, t0 = item.y & 0xffff;
                nt = item.y >> 16;
                npad = 16;
                while (npad < nt) npad <<= 1;
                const int cb = cch_beg[P], nch = cch_end[P] - cb;
                g0 = prange[cb].x + t0;
                n = tid & (npad - 1);
                c = 31;
                if (n < nt) {
                    const int g = g0 + n;
                    int cc = 0;
                    for (int k = 1; k < nch; ++k)
                        if (prange[cb + k].x <= g) cc = k;
                    c = cc;
                    const int X = cb + cc;
                    const float4 v = pv4[g], hX = chi[X], lX = clo[X], hP = chi[P], lP = clo[P];
                    tx = v.x + ((hX.x - hP.x) + (lX.x - lP.x));
                    ty = v.y + ((hX.y - hP.y) + (lX.y - lP.y));
                    tz = v.z + ((hX.z - hP.z) + (lX.z - lP.z));
                }
            }
            const int nq = T.nq;
            for (int q = tid / npad; q < TC_QPC; q += TC_EVAL / npad) {
                float f[4] = {0.f, 0.f, 0.f, 0.f};
                if (c < 31 && q < nq && ((T.mask[q] >> c) & 1)) {
                    const float4 sh = T.sh[q];
                    const float x = tx - sh.x, y = ty - sh.y, z = tz - sh.z;
                    const float4 a = T.src[q][0], b = T.src[q][1], e = T.src[q][2], g = T.src[q][3];
                    const float sx[4] = {a.x, a.y, e.x, e.y}, sy[4] = {a.z, a.w, e.z, e.w}, sz[4] = {b.x, b.y, g.x, g.y};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float dx = x - sx[j], dy = y - sy[j], dz = z - sz[j];
                        f[j] = KF<KIND>::f32_far(kp, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    }
                }
                float4 hi, lo;
                split_value(mode, f[0], hi.x, lo.x);
                split_value(mode, f[1], hi.y, lo.y);
                split_value(mode, f[2], hi.z, lo.z);
                split_value(mode, f[3], hi.w, lo.w);
                const int o = (n >> 3) * (TC_QPC * 32) + q * 32 + (n & 7) * 4;
                *reinterpret_cast<float4 *>(&T.bhi[o]) = hi;
                if (mode == NNCA_PREC_TF32X3) *reinterpret_cast<float4 *>(&T.blo[o]) = lo;
            }
            // the B tile (generic writes) and the source reads before the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&S.ready[s]);
            ++cnt;
            if (flags & TC_SEG_END) {
                // warps 0-1 (rows 0..63 of D): add the segment's accumulator into
                // the compensated sums; at the item's end write u and clear them
                const int db = nseg & 1;
                if (warp < 2) {
                    if (!mbar_wait_warp(&S.dfull[db], (nseg >> 1) & 1)) {
                        if (lane == 0) tc_fail(S, status);
                        break;
                    }
                    tc_fence_after();
                    const int r = warp * 32 + lane;
                    const bool last = (flags & TC_ITEM_LAST) != 0;
                    const bool corr = last && mode == NNCA_PREC_TF32X3;
                    const unsigned lanes = (unsigned)(warp * 32) << 16;
                    for (int c0 = 0; c0 < npad; c0 += 16) {
                        float v[16], vc[16];
                        tmem_ld16(tmem + lanes + (unsigned)(db * TC_TGT + c0), v);
                        if (corr) tmem_ld16(tmem + lanes + (unsigned)((2 + (nit & 1)) * TC_TGT + c0), vc);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float2 a = S.acc[c0 + j][r];
                            two_sum_add(a.x, a.y, v[j]);
                            if (last) {
                                if (corr) two_sum_add(a.x, a.y, vc[j]);
                                if (c0 + j < nt && r < nrhs) utc[(int64_t)(g0 + c0 + j) * TC_RHS + r] = a.x + a.y;
                                a = make_float2(0.f, 0.f);
                            }
                            S.acc[c0 + j][r] = a;
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(&S.dfree[db]);
                    if (last) mbar_arrive(&S.cfree[nit & 1]);
                }
                ++nseg;
                if (flags & TC_ITEM_LAST) ++nit;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

// W^T of a pass, packed per source quad of spk: quad Q holds sources 4Q .. 4Q + 3 of
// the packed order (cell y's pivots from pair spk_off[y] on, padded with weight 0),
// element (r, k) at Q * TC_QF + (r / 8) * 32 + (r % 8) * 4 + k; hi and lo parts by mode.
// One warp per cell.
__global__ void k_pack_wq(int64_t ncell, const int2 *prange, const int32_t *spk_off, const double *w, int64_t npiv,
                          int nr, int mode, float *wq_hi, float *wq_lo) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t y = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; y < ncell; y += nw) {
        const int2 pr = prange[y];
        const int npad = m2l_padded(pr.y);
        if (pr.y == 0) continue;
        const int64_t q0 = spk_off[y] >> 1;
        for (int e = lane; e < npad * TC_RHS; e += 32) {
            const int j = e % npad, r = e / npad;
            const float v = (j < pr.y && r < nr) ? (float)w[(int64_t)r * npiv + pr.x + j] : 0.f;
            float hi, lo;
            split_value(mode, v, hi, lo);
            const int64_t o = (q0 + (j >> 2)) * TC_QF + (r >> 3) * 32 + (r & 7) * 4 + (j & 3);
            wq_hi[o] = hi;
            if (mode == NNCA_PREC_TF32X3) wq_lo[o] = lo;
        }
    }
}

// u(r, p) = s * utc(p, r) for the pass's right-hand sides (u right-hand-side major)
__global__ void k_unpack_u(int64_t npiv, int nr, double s, const float *utc, double *u) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npiv * nr; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / npiv, p = e - r * npiv;
        u[e] = s * (double)utc[p * TC_RHS + r];
    }
}

// Chunks of 32 sources whose main products accumulate in tensor memory between
// two flushes into the compensated sums. The tensor core's FP32 accumulation
// loses about one unit in the last place per accumulating instruction (measured:
// the error of the 3xTF32 product grows linearly with this period); with 2 chunks
// (8 main products) the 1,048,576- and 262,144-point workloads' products stay
// within 1e-6 of the FP64 form.
constexpr int TC_SEG_CHUNKS = 2;

template <int KIND>
void launch_tc(Handle *h, int mode, int nr, const float *wq_hi, const float *wq_lo, float *utc) {
    int dev = 0, nsm = 152;
    NNCA_CUDA(cudaGetDevice(&dev));
    NNCA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int smem = (int)sizeof(TcSmem);
    NNCA_CUDA(cudaFuncSetAttribute(k_m2l_tc<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const unsigned grid = (unsigned)std::max(1, std::min(h->n_tc_items, 2 * nsm));
    k_m2l_tc<KIND><<<grid, TC_THREADS, smem, h->stream>>>(h->kp, mode, h->tc_items, h->n_tc_items, h->m2l_plan,
                                                          h->m2l_plan_sh, h->cch_beg, h->cch_end, h->prange, h->pv4,
                                                          h->chi4, h->clo4, h->spk, wq_hi, wq_lo, nr, utc,
                                                          TC_SEG_CHUNKS, h->dev_status);
    NNCA_LAUNCH_CHECK();
    ++h->launches;
}

unsigned grid_tc(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 64));
}

}  // namespace

int tc_rhs_per_pass() { return TC_RHS; }

size_t tc_workspace_floats(const Handle *h) {
    const int64_t nquads = h->n_spk_pairs / 2;
    return (size_t)h->npiv * TC_RHS + 2 * (size_t)(nquads + 1) * TC_QF;
}

void m2l_tensor(Handle *h, int mode, int nr, const double *w, double *u, float *tcws) {
    NNCA_REQUIRE(nr >= 1 && nr <= TC_RHS, NNCA_ERR_INTERNAL, "tensor-core M2L: bad pass width");
    const int64_t npiv = h->npiv, nquads = h->n_spk_pairs / 2;
    float *utc = tcws;
    float *wq_hi = utc + (size_t)npiv * TC_RHS;
    float *wq_lo = wq_hi + (size_t)(nquads + 1) * TC_QF;
    cudaStream_t s = h->stream;
    k_pack_wq<<<grid_tc(h->ncell * 32, 256), 256, 0, s>>>(h->ncell, h->prange, h->spk_off, w, npiv, nr, mode, wq_hi,
                                                        wq_lo);
    NNCA_LAUNCH_CHECK();
    NNCA_CUDA(cudaMemsetAsync(utc, 0, sizeof(float) * (size_t)npiv * TC_RHS, s));
    h->launches += 1;
    if (h->n_tc_items > 0) {
        switch (h->kp.kind) {
        case NNCA_K_INV_R: launch_tc<NNCA_K_INV_R>(h, mode, nr, wq_hi, wq_lo, utc); break;
        case NNCA_K_LOG: launch_tc<NNCA_K_LOG>(h, mode, nr, wq_hi, wq_lo, utc); break;
        case NNCA_K_GAUSS: launch_tc<NNCA_K_GAUSS>(h, mode, nr, wq_hi, wq_lo, utc); break;
        case NNCA_K_MATERN: launch_tc<NNCA_K_MATERN>(h, mode, nr, wq_hi, wq_lo, utc); break;
        case NNCA_K_PAPER_I: launch_tc<NNCA_K_PAPER_I>(h, mode, nr, wq_hi, wq_lo, utc); break;
        case NNCA_K_PAPER_II: launch_tc<NNCA_K_PAPER_II>(h, mode, nr, wq_hi, wq_lo, utc); break;
        default: NNCA_REQUIRE(false, NNCA_ERR_UNSUPPORTED, "tensor-core M2L: radial kernels only");
        }
    }
    k_unpack_u<<<grid_tc(npiv * nr, 256), 256, 0, s>>>(npiv, nr, h->kp.s, utc, u);
    NNCA_LAUNCH_CHECK();
    h->launches += 1;
}

void set_wait_test_tc(int64_t wait_limit_clocks, unsigned extra_tx_bytes) {
    const long long lim = wait_limit_clocks > 0 ? (long long)wait_limit_clocks : (1ll << 31);
    NNCA_CUDA(cudaMemcpyToSymbol(g_wait_limit, &lim, sizeof(lim)));
    NNCA_CUDA(cudaMemcpyToSymbol(g_stage_extra_tx, &extra_tx_bytes, sizeof(extra_tx_bytes)));
}

}  // namespace nnca
