// Device-wide exclusive prefix sum of int64 values (reduce, scan of tile sums,
// down-sweep). Used to turn per-item counts into CSR offsets.
#include "nnca_internal.cuh"

namespace nnca {

namespace {
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of one value per thread across the block; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t &excl) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t block_tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;   // exclusive warp offsets
        if (lane == nw - 1) block_tot = ti;       // block total (nw <= 32)
    }
    __syncthreads();
    excl = inc - v + warp_tot[wid];
    int64_t total = block_tot;
    __syncthreads();
    return total;
}

__global__ void k_scan_reduce(const int64_t *in, int64_t n, int64_t *tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += in[i];
    }
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_down(const int64_t *in, int64_t *out, int64_t n, const int64_t *tile_off,
                            int64_t *total) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, excl);
    int64_t run = excl + (tile_off ? tile_off[blockIdx.x] : 0);
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *total = (tile_off ? tile_off[blockIdx.x] : 0) + tot;
}

void scan_rec(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s, Scratch &scr) {
    if (n <= 0) {
        if (total) NNCA_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        return;
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_down<<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, total);
        NNCA_LAUNCH_CHECK();
        return;
    }
    int64_t *sums = scr.get<int64_t>(tiles);
    k_scan_reduce<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums);
    NNCA_LAUNCH_CHECK();
    scan_rec(sums, sums, tiles, nullptr, s, scr);
    k_scan_down<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums, total);
    NNCA_LAUNCH_CHECK();
}
}  // namespace

void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, Scratch &scr) {
    scan_rec(in, out, n, nullptr, s, scr);
}

int64_t scan_total_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, Scratch &scr) {
    int64_t *tot = scr.get<int64_t>(1);
    scan_rec(in, out, n, tot, s, scr);
    int64_t h = 0;
    NNCA_CUDA(cudaMemcpyAsync(&h, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NNCA_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace nnca
