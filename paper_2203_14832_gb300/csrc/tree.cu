// Uniform 2^d tree on the GPU (Sec. 2.1): bounding cube, Morton keys, LSD
// radix sort, leaf level kappa, and the cell tables of every level.
//
// The cube, the quantisation and the key layout follow one fixed reading of
// the paper's "compact hypercube containing the points" (every floating-point
// step rounded on its own, in the order written below), so that keys, cells
// and lists are reproducible bit for bit:
//   centre_k = (lo_k + hi_k) * 0.5, half = max_k (hi_k - lo_k) * 0.5
//   (0.5 if all points coincide), corner_k = centre_k - half, side = 2 half,
//   q_k = clamp(floor(((x_k - corner_k) / side) * 2^lmax), 0, 2^lmax - 1),
//   lmax = floor(63 / d); bit b of q_k is key bit b*d + k.
// Points are sorted by (key, original index) with a stable LSD radix sort,
// and kappa is the first level at which no cell holds more than nu points.
#include "nnca_internal.cuh"

namespace nnca {

namespace {

constexpr int BB_THREADS = 256;

__global__ void k_check_finite(const double *P, int64_t total, unsigned *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(P[i])) atomicOr(status, DEV_BAD_INDEX);
}

__global__ void k_bbox_partial(const double *P, int64_t n, int d, int layout, double *plo, double *phi) {
    double lo[4], hi[4];
    for (int k = 0; k < 4; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < d; ++k) {
            double v = layout == NNCA_LAYOUT_AOS ? P[i * d + k] : P[(int64_t)k * n + i];
            lo[k] = fmin(lo[k], v);
            hi[k] = fmax(hi[k], v);
        }
    __shared__ double slo[4][BB_THREADS / 32], shi[4][BB_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < d; ++k) {
        double a = lo[k], b = hi[k];
        for (int o = 16; o; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { slo[k][wid] = a; shi[k][wid] = b; }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < d; ++k) {
            double a = INFINITY, b = -INFINITY;
            for (int w = 0; w < BB_THREADS / 32; ++w) { a = fmin(a, slo[k][w]); b = fmax(b, shi[k][w]); }
            plo[blockIdx.x * 4 + k] = a;
            phi[blockIdx.x * 4 + k] = b;
        }
}

// geom[0..3] = corner, geom[4] = side
__global__ void k_bbox_final(const double *plo, const double *phi, int nb, int d, double *geom) {
    if (threadIdx.x != 0) return;
    double lo[4], hi[4];
    for (int k = 0; k < d; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < d; ++k) { lo[k] = fmin(lo[k], plo[b * 4 + k]); hi[k] = fmax(hi[k], phi[b * 4 + k]); }
    double half = 0.0;
    for (int k = 0; k < d; ++k) {
        double e = __dmul_rn(__dsub_rn(hi[k], lo[k]), 0.5);
        if (e > half) half = e;
    }
    if (half == 0.0) half = 0.5;
    for (int k = 0; k < d; ++k) geom[k] = __dsub_rn(__dmul_rn(__dadd_rn(lo[k], hi[k]), 0.5), half);
    geom[4] = __dmul_rn(2.0, half);
}

__global__ void k_morton(const double *P, int64_t n, int d, int layout, int lmax, const double *geom,
                         uint64_t *keys, int32_t *vals) {
    const double side = geom[4];
    const double scale = ldexp(1.0, lmax);
    const uint64_t qmax = (lmax >= 64) ? ~0ull : ((1ull << lmax) - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
        for (int k = 0; k < d; ++k) {
            double v = layout == NNCA_LAYOUT_AOS ? P[i * d + k] : P[(int64_t)k * n + i];
            double t = __dmul_rn(__ddiv_rn(__dsub_rn(v, geom[k]), side), scale);
            double f = floor(t);
            uint64_t q;
            if (!(f >= 0.0)) q = 0;
            else if (f >= scale) q = qmax;
            else q = (uint64_t)f;
            for (int b = 0; b < lmax; ++b) key |= ((q >> b) & 1ull) << (b * d + k);
        }
        keys[i] = key;
        vals[i] = (int32_t)i;
    }
}

// ---- LSD radix sort of (uint64 key, int32 value), 8-bit digits, stable ------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void k_radix_hist(const uint64_t *keys, int64_t n, int shift, int64_t *hist, int nblocks) {
    __shared__ unsigned sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&sh[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout, int64_t n,
                                int shift, const int64_t *offs, int nblocks) {
    __shared__ int64_t base[256];
    __shared__ unsigned wcnt[RS_THREADS / 32][257];
    __shared__ unsigned rtot[256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = tile + (int64_t)r * RS_THREADS + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int32_t val = valid ? vin[i] : 0;
        unsigned dg = valid ? (unsigned)((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        unsigned rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) wcnt[wid][dg] = __popc(peers);
        __syncthreads();
        {   // exclusive prefix over warps for digit threadIdx.x
            unsigned run = 0;
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                unsigned c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = run;
                run += c;
            }
            rtot[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base[dg] + wcnt[wid][dg] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        base[threadIdx.x] += rtot[threadIdx.x];
        for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

__global__ void k_kappa(const uint64_t *keys, int64_t n, int nu, int d, int lmax, int *maxeq) {
    const int nbits = d * lmax;
    int best = -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + nu < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = keys[i] ^ keys[i + nu];
        int eqbits = x == 0 ? nbits : (__clzll((long long)x) - (64 - nbits));
        int eqg = eqbits / d;
        best = max(best, eqg);
    }
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best >= 0) atomicMax(maxeq, best);
}

__device__ __forceinline__ uint64_t prefix_of(uint64_t key, int d, int lmax, int l) {
    int sh = d * (lmax - l);
    return sh >= 64 ? 0ull : key >> sh;
}

// per-level count of cells: a point starts a cell where its prefix changes
__global__ void k_cell_count(const uint64_t *keys, int64_t n, int d, int lmax, int kappa,
                             unsigned long long *counts) {
    __shared__ unsigned sc[64];
    if (threadIdx.x < 64) sc[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i], kp = i ? keys[i - 1] : 0;
        for (int l = 0; l <= kappa; ++l)
            if (i == 0 || prefix_of(k, d, lmax, l) != prefix_of(kp, d, lmax, l)) atomicAdd(&sc[l], 1u);
    }
    __syncthreads();
    if (threadIdx.x <= (unsigned)kappa && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)sc[threadIdx.x]);
}

__global__ void k_cell_flags(const uint64_t *keys, int64_t n, int d, int lmax, int l, int64_t *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || prefix_of(keys[i], d, lmax, l) != prefix_of(keys[i - 1], d, lmax, l)) ? 1 : 0;
}

__global__ void k_cell_fill(const uint64_t *keys, int64_t n, int d, int lmax, int l, const int64_t *pos,
                            int64_t base, uint64_t *ckey, int32_t *cbeg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t p = prefix_of(keys[i], d, lmax, l);
        if (i == 0 || p != prefix_of(keys[i - 1], d, lmax, l)) {
            int64_t c = base + pos[i];
            ckey[c] = p;
            cbeg[c] = (int32_t)i;
        }
    }
}

__global__ void k_cell_links(int64_t b0, int64_t b1, int64_t pb0, int64_t n, int d, int l, const uint64_t *ckey,
                             const int32_t *cbeg, int32_t *cend, int32_t *cpar, int32_t *ccoord, int64_t ncell) {
    for (int64_t c = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < b1; c += (int64_t)gridDim.x * blockDim.x) {
        cend[c] = (c + 1 < b1) ? cbeg[c + 1] : (int32_t)n;
        if (l == 0) {
            cpar[c] = -1;
        } else {
            uint64_t pk = ckey[c] >> d;
            int64_t lo = pb0, hi = b0;   // parent level range [pb0, b0)
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) >> 1;
                if (ckey[mid] <= pk) lo = mid; else hi = mid;
            }
            cpar[c] = (int32_t)lo;
        }
        uint64_t key = ckey[c];
        for (int k = 0; k < d; ++k) {
            int32_t v = 0;
            for (int b = 0; b < l; ++b) v |= (int32_t)((key >> (b * d + k)) & 1ull) << b;
            ccoord[(int64_t)k * ncell + c] = v;
        }
    }
}

__global__ void k_cell_children(int64_t b0, int64_t b1, const int32_t *cpar, int32_t *cch_beg, int32_t *cch_end) {
    for (int64_t c = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < b1; c += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = cpar[c];
        if (c == b0 || cpar[c - 1] != p) cch_beg[p] = (int32_t)c;
        if (c == b1 - 1 || cpar[c + 1] != p) cch_end[p] = (int32_t)(c + 1);
    }
}

__global__ void k_gather_points(const double *P, int64_t n, int d, int layout, const int32_t *perm, double *xs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t src = perm[i];
        for (int k = 0; k < d; ++k)
            xs[(int64_t)k * n + i] = layout == NNCA_LAYOUT_AOS ? P[src * d + k] : P[(int64_t)k * n + src];
    }
}

unsigned grid_for(int64_t n, int threads, unsigned cap = 152 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace

void build_tree(Handle *h, const double *P, int layout) {
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    const int d = h->d;
    h->lmax = 63 / d;
    Scratch scr;

    k_check_finite<<<grid_for(n * d, 256), 256, 0, s>>>(P, n * d, h->dev_status);
    NNCA_LAUNCH_CHECK();

    // bounding cube
    const unsigned nbb = grid_for(n, BB_THREADS, 1024);
    double *plo = scr.get<double>(nbb * 4), *phi = scr.get<double>(nbb * 4), *geom = scr.get<double>(8);
    k_bbox_partial<<<nbb, BB_THREADS, 0, s>>>(P, n, d, layout, plo, phi);
    NNCA_LAUNCH_CHECK();
    k_bbox_final<<<1, 32, 0, s>>>(plo, phi, (int)nbb, d, geom);
    NNCA_LAUNCH_CHECK();
    double hg[8];
    NNCA_CUDA(cudaMemcpyAsync(hg, geom, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));

    // Morton keys and stable radix sort
    uint64_t *k0 = scr.get<uint64_t>(n), *k1 = scr.get<uint64_t>(n);
    int32_t *v0 = scr.get<int32_t>(n), *v1 = scr.get<int32_t>(n);
    k_morton<<<grid_for(n, 256), 256, 0, s>>>(P, n, d, layout, h->lmax, geom, k0, v0);
    NNCA_LAUNCH_CHECK();
    const int nbits = d * h->lmax;
    const int npass = (nbits + 7) / 8;
    const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    int64_t *hist = scr.get<int64_t>((size_t)256 * nblk);
    for (int pass = 0; pass < npass; ++pass) {
        const int shift = pass * 8;
        k_radix_hist<<<nblk, RS_THREADS, 0, s>>>(k0, n, shift, hist, nblk);
        NNCA_LAUNCH_CHECK();
        scan_exclusive_i64(hist, hist, (int64_t)256 * nblk, s, scr);
        k_radix_scatter<<<nblk, RS_THREADS, 0, s>>>(k0, v0, k1, v1, n, shift, hist, nblk);
        NNCA_LAUNCH_CHECK();
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    h->keys = dalloc<uint64_t>(h, n);
    h->perm = dalloc<int32_t>(h, n);
    NNCA_CUDA(cudaMemcpyAsync(h->keys, k0, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    NNCA_CUDA(cudaMemcpyAsync(h->perm, v0, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    h->xs = dalloc<double>(h, (size_t)n * d);
    k_gather_points<<<grid_for(n, 256), 256, 0, s>>>(P, n, d, layout, h->perm, h->xs);
    NNCA_LAUNCH_CHECK();

    // leaf level kappa
    int *maxeq = scr.get<int>(1);
    NNCA_CUDA(cudaMemsetAsync(maxeq, 0xff, sizeof(int), s));   // -1
    const int nu = h->cfg.leaf_size;
    if (n > nu) {
        k_kappa<<<grid_for(n, 256), 256, 0, s>>>(h->keys, n, nu, d, h->lmax, maxeq);
        NNCA_LAUNCH_CHECK();
    }
    int hmax = -1;
    NNCA_CUDA(cudaMemcpyAsync(&hmax, maxeq, sizeof(int), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < d; ++k) h->corner[k] = hg[k];
    h->side = hg[4];
    h->kappa = (n <= nu) ? 0 : std::min(hmax + 1, h->lmax);
    const int kappa = h->kappa;

    // cell tables, level by level
    unsigned long long *cnt = scr.get<unsigned long long>(64);
    NNCA_CUDA(cudaMemsetAsync(cnt, 0, 64 * sizeof(unsigned long long), s));
    k_cell_count<<<grid_for(n, 256), 256, 0, s>>>(h->keys, n, d, h->lmax, kappa, cnt);
    NNCA_LAUNCH_CHECK();
    unsigned long long hc[64];
    NNCA_CUDA(cudaMemcpyAsync(hc, cnt, 64 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaStreamSynchronize(s));
    h->level_base.assign(kappa + 2, 0);
    for (int l = 0; l <= kappa; ++l) h->level_base[l + 1] = h->level_base[l] + (int64_t)hc[l];
    const int64_t nc = h->level_base[kappa + 1];
    h->ncell = nc;
    h->ckey = dalloc<uint64_t>(h, nc);
    h->cbeg = dalloc<int32_t>(h, nc);
    h->cend = dalloc<int32_t>(h, nc);
    h->cpar = dalloc<int32_t>(h, nc);
    h->cch_beg = dalloc<int32_t>(h, nc);
    h->cch_end = dalloc<int32_t>(h, nc);
    h->ccoord = dalloc<int32_t>(h, (size_t)nc * d);
    NNCA_CUDA(cudaMemsetAsync(h->cch_beg, 0, nc * sizeof(int32_t), s));
    NNCA_CUDA(cudaMemsetAsync(h->cch_end, 0, nc * sizeof(int32_t), s));
    int64_t *flags = scr.get<int64_t>(n);
    for (int l = 0; l <= kappa; ++l) {
        k_cell_flags<<<grid_for(n, 256), 256, 0, s>>>(h->keys, n, d, h->lmax, l, flags);
        NNCA_LAUNCH_CHECK();
        scan_exclusive_i64(flags, flags, n, s, scr);
        k_cell_fill<<<grid_for(n, 256), 256, 0, s>>>(h->keys, n, d, h->lmax, l, flags, h->level_base[l], h->ckey,
                                                     h->cbeg);
        NNCA_LAUNCH_CHECK();
        const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1];
        k_cell_links<<<grid_for(b1 - b0, 256), 256, 0, s>>>(b0, b1, l ? h->level_base[l - 1] : 0, n, d, l, h->ckey,
                                                             h->cbeg, h->cend, h->cpar, h->ccoord, nc);
        NNCA_LAUNCH_CHECK();
        if (l > 0) {
            k_cell_children<<<grid_for(b1 - b0, 256), 256, 0, s>>>(b0, b1, h->cpar, h->cch_beg, h->cch_end);
            NNCA_LAUNCH_CHECK();
        }
    }
    NNCA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace nnca
