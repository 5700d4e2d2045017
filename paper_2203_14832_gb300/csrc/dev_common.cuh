// Device helpers shared by the product's kernels (matvec.cu, m2l_tc.cu): MUFU
// forms of the kernel functions, compensated float sums, packed f32x2
// arithmetic, mbarrier and bulk-copy (TMA) wrappers with bounded waits.
//
// Included inside an anonymous namespace of nnca: every translation unit gets
// its own copy, including its own g_wait_limit and g_stage_extra_tx (which
// set_wait_test sets in every unit that has them).
#pragma once

// Single-instruction MUFU forms (flush-to-zero approximations).
__device__ __forceinline__ float mufu_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// f(r^2) with K = s f(r); FP32 and FP64 forms, one instantiation per kernel.
// f32_far: r^2 > 0 guaranteed (distinct cells); f32: any r^2 >= 0.
template <int KIND> struct KF;
template <> struct KF<NNCA_K_INV_R> {
    static __device__ __forceinline__ float f32(const KParams &, float r2) { return r2 > 0.f ? mufu_rsqrt(r2) : 0.f; }
    static __device__ __forceinline__ float f32_far(const KParams &, float r2) { return mufu_rsqrt(r2); }
    static __device__ __forceinline__ double f64(const KParams &, double r2) { return r2 > 0.0 ? rsqrt(r2) : 0.0; }
};
template <> struct KF<NNCA_K_LOG> {
    // 0.5 ln(r^2) = (0.5 ln 2) log2(r^2)
    static __device__ __forceinline__ float f32(const KParams &, float r2) {
        return r2 > 0.f ? 0.34657359f * mufu_lg2(r2) : 0.f;
    }
    static __device__ __forceinline__ float f32_far(const KParams &, float r2) { return 0.34657359f * mufu_lg2(r2); }
    static __device__ __forceinline__ double f64(const KParams &, double r2) { return r2 > 0.0 ? 0.5 * log(r2) : 0.0; }
};
template <> struct KF<NNCA_K_GAUSS> {
    // exp(-r^2 / (2 h^2)) = 2^(r^2 * c), c = -log2(e) / (2 h^2) precomputed in kp.hf
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) { return mufu_ex2(r2 * kp.hf); }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return mufu_ex2(r2 * kp.hf); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) { return exp(-r2 / (2.0 * kp.h * kp.h)); }
};
template <> struct KF<NNCA_K_MATERN> {
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) { return __expf(-sqrtf(r2) / (float)kp.h); }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return f32(kp, r2); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) { return exp(-sqrt(r2) / kp.h); }
};
template <> struct KF<NNCA_K_PAPER_I> {
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) {
        if (!(r2 > 0.f)) return 0.f;
        const float a = (float)kp.h, r = sqrtf(r2);
        return r < a ? (r * (logf(r) - 1.f)) / (a * (logf(a) - 1.f)) : logf(r) / logf(a);
    }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return f32(kp, r2); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) {
        if (!(r2 > 0.0)) return 0.0;
        const double a = kp.h, r = sqrt(r2);
        return r < a ? (r * (log(r) - 1.0)) / (a * (log(a) - 1.0)) : log(r) / log(a);
    }
};
template <> struct KF<NNCA_K_PAPER_II> {
    static __device__ __forceinline__ float f32(const KParams &kp, float r2) {
        const float a = (float)kp.h, r = sqrtf(r2);
        return r < a ? r / a : a / r;
    }
    static __device__ __forceinline__ float f32_far(const KParams &kp, float r2) { return f32(kp, r2); }
    static __device__ __forceinline__ double f64(const KParams &kp, double r2) {
        const double a = kp.h, r = sqrt(r2);
        return r < a ? r / a : a / r;
    }
};

// compensated accumulation: (s, c) += v
__device__ __forceinline__ void two_sum_add(float &s, float &c, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (v - bp);
    s = t;
    c += err;
}

// ---- packed FP32 arithmetic (two lanes of float in one 64-bit register) ------
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(f2 a) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// f(r^2) on a packed pair; SAFE maps r^2 = 0 to f(0) of the singular kernels (0).
#ifndef NNCA_RSQRT_NEWTON
#define NNCA_RSQRT_NEWTON 0
#endif
template <int KIND, bool SAFE> struct KF2 {
    static __device__ __forceinline__ f2 eval(const KParams &kp, f2 r2) {
        const float2 v = f2_unpack(r2);
        return f2_pack(SAFE ? KF<KIND>::f32(kp, v.x) : KF<KIND>::f32_far(kp, v.x),
                       SAFE ? KF<KIND>::f32(kp, v.y) : KF<KIND>::f32_far(kp, v.y));
    }
};
// rsqrt of both halves of a packed pair, unpacked and repacked inside one PTX
// block so that the halves can stay in their register pair
__device__ __forceinline__ f2 f2_rsqrt(f2 a) {
    f2 r;
    asm("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\trsqrt.approx.ftz.f32 lo, lo;\n\t"
        "rsqrt.approx.ftz.f32 hi, hi;\n\tmov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r)
        : "l"(a));
    return r;
}

template <bool SAFE> struct KF2<NNCA_K_INV_R, SAFE> {
    // 1/r: one MUFU rsqrt (relative error ~1e-7). An optional Newton step
    // f <- f - (f/2)(r^2 f^2 - 1) takes it to float rounding, at 4 more packed
    // operations per pair; measured, it changes the product's error by ~3%.
    static __device__ __forceinline__ f2 eval(const KParams &, f2 r2) {
        f2 f = f2_rsqrt(r2);
#if NNCA_RSQRT_NEWTON
        const f2 h = f2_mul(r2, f);
        const f2 e = f2_fma(h, f, f2_pack(-1.f, -1.f));
        const f2 hf = f2_mul(f, f2_pack(-0.5f, -0.5f));
        f = f2_fma(hf, e, f);
#endif
        if (SAFE) {
            const float2 v = f2_unpack(r2);
            float2 g = f2_unpack(f);
            g.x = v.x > 0.f ? g.x : 0.f;
            g.y = v.y > 0.f ? g.y : 0.f;
            f = f2_pack(g.x, g.y);
        }
        return f;
    }
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(void *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(void *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(void *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// The bounded waits' clock budget and the bytes added to every staging round's
// expected transaction count, in device memory so that a test can change them
// (nnca_set_wait_test): 2^31 clocks and 0 in normal use. With extra bytes the
// rounds' phases never complete although every copy lands, so every wait on
// them runs out.
__device__ long long g_wait_limit = 1ll << 31;
__device__ unsigned g_stage_extra_tx = 0u;

// wait until the phase of the given parity has completed; false after g_wait_limit clocks
__device__ __forceinline__ bool mbar_wait(void *bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    const long long lim = g_wait_limit;
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > lim) return false;
    }
}
// the same wait taken by a whole warp: it succeeds only if it succeeds for every lane
__device__ __forceinline__ bool mbar_wait_warp(void *bar, unsigned parity) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity));
}
// bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, void *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

