// Neighbour lists N(B) and interaction lists IL(B) on the GPU (Sec. 2.2,
// Eq. 2, Table 1).
//
// Admissibility of two cells of one level with integer coordinates a, b is
// exact in integers: with g_k = max(0, |a_k - b_k| - 1) and eta^2 = num/den,
//     max{diam X, diam Y} <= eta dist(X, Y)  <=>  d * den <= num * sum g_k^2.
// A neighbour of X has a parent that is a neighbour of X's parent (parents are
// twice as large and no farther apart, so non-admissible children have
// non-admissible parents). Hence the children of N(parent(X)) hold both N(X)
// and IL(X): the admissible ones form IL(X) (Table 1), the others N(X).
// Walking N(parent) in ascending cell id and each parent's children in order
// yields both lists in ascending cell id (= ascending Morton key) with no sort.
#include "nnca_internal.cuh"

namespace nnca {

namespace {

__device__ __forceinline__ bool admissible(const int32_t *ccoord, int64_t ncell, int d, int num, int den,
                                           int64_t X, int64_t Y) {
    int64_t g2 = 0;
    for (int k = 0; k < d; ++k) {
        int64_t t = (int64_t)ccoord[(int64_t)k * ncell + X] - ccoord[(int64_t)k * ncell + Y];
        if (t < 0) t = -t;
        t -= 1;
        if (t < 0) t = 0;
        g2 += t * t;
    }
    return (int64_t)d * den <= (int64_t)num * g2;
}

// pass 0: count, pass 1: fill. Per cell X of the level (local index x).
template <int PASS>
__global__ void k_lists(int64_t b0, int64_t b1, const int32_t *cpar, const int32_t *cch_beg, const int32_t *cch_end,
                        const int32_t *ccoord, int64_t ncell, int d, int num, int den,
                        const int64_t *pnb_off, const int32_t *pnb_idx, int64_t pb0,
                        int64_t *nb_cnt, int64_t *il_cnt, int32_t *nb_idx, int32_t *il_idx) {
    for (int64_t X = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; X < b1; X += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = X - b0;
        const int64_t P = cpar[X];
        const int64_t p = P - pb0;
        int64_t cn = 0, ci = 0;
        int64_t on = PASS ? nb_cnt[x] : 0, oi = PASS ? il_cnt[x] : 0;
        for (int64_t q = pnb_off[p]; q < pnb_off[p + 1]; ++q) {
            const int64_t Z = pnb_idx[q];
            for (int64_t Y = cch_beg[Z]; Y < cch_end[Z]; ++Y) {
                if (admissible(ccoord, ncell, d, num, den, X, Y)) {
                    if (PASS) il_idx[oi + ci] = (int32_t)Y;
                    ++ci;
                } else {
                    if (PASS) nb_idx[on + cn] = (int32_t)Y;
                    ++cn;
                }
            }
        }
        if (!PASS) {
            nb_cnt[x] = cn;
            il_cnt[x] = ci;
        }
    }
}

__global__ void k_offsets_to_global(const int64_t *loc, int64_t cnt, int64_t base_entry, int64_t first_cell,
                                    int32_t *goff) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x <= cnt; x += (int64_t)gridDim.x * blockDim.x)
        goff[first_cell + x] = (int32_t)(base_entry + loc[x]);
}

unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

}  // namespace

void build_lists(Handle *h) {
    cudaStream_t s = h->stream;
    Scratch scr;
    const int kappa = h->kappa, d = h->d;
    const int num = h->cfg.eta2_num, den = h->cfg.eta2_den;
    std::vector<int64_t *> nb_off(kappa + 1), il_off(kappa + 1);
    std::vector<int32_t *> nb_idx(kappa + 1), il_idx(kappa + 1);
    std::vector<int64_t> nb_tot(kappa + 1), il_tot(kappa + 1);

    // level 0: N(root) = {root}, IL(root) = {}
    {
        int64_t ho[2] = {0, 1}, hi[2] = {0, 0};
        int32_t root = 0;
        nb_off[0] = scr.get<int64_t>(2);
        il_off[0] = scr.get<int64_t>(2);
        nb_idx[0] = scr.get<int32_t>(1);
        il_idx[0] = scr.get<int32_t>(1);
        NNCA_CUDA(cudaMemcpyAsync(nb_off[0], ho, sizeof(ho), cudaMemcpyHostToDevice, s));
        NNCA_CUDA(cudaMemcpyAsync(il_off[0], hi, sizeof(hi), cudaMemcpyHostToDevice, s));
        NNCA_CUDA(cudaMemcpyAsync(nb_idx[0], &root, sizeof(root), cudaMemcpyHostToDevice, s));
        nb_tot[0] = 1;
        il_tot[0] = 0;
        NNCA_CUDA(cudaStreamSynchronize(s));
    }
    for (int l = 1; l <= kappa; ++l) {
        const int64_t b0 = h->level_base[l], b1 = h->level_base[l + 1], cnt = b1 - b0;
        nb_off[l] = scr.get<int64_t>(cnt + 1);
        il_off[l] = scr.get<int64_t>(cnt + 1);
        NNCA_CUDA(cudaMemsetAsync(nb_off[l] + cnt, 0, sizeof(int64_t), s));
        NNCA_CUDA(cudaMemsetAsync(il_off[l] + cnt, 0, sizeof(int64_t), s));
        k_lists<0><<<grid_for(cnt, 128), 128, 0, s>>>(b0, b1, h->cpar, h->cch_beg, h->cch_end, h->ccoord, h->ncell, d,
                                                      num, den, nb_off[l - 1], nb_idx[l - 1], h->level_base[l - 1],
                                                      nb_off[l], il_off[l], nullptr, nullptr);
        NNCA_LAUNCH_CHECK();
        nb_tot[l] = scan_total_i64(nb_off[l], nb_off[l], cnt + 1, s, scr);
        il_tot[l] = scan_total_i64(il_off[l], il_off[l], cnt + 1, s, scr);
        nb_idx[l] = scr.get<int32_t>(nb_tot[l]);
        il_idx[l] = scr.get<int32_t>(il_tot[l]);
        k_lists<1><<<grid_for(cnt, 128), 128, 0, s>>>(b0, b1, h->cpar, h->cch_beg, h->cch_end, h->ccoord, h->ncell, d,
                                                      num, den, nb_off[l - 1], nb_idx[l - 1], h->level_base[l - 1],
                                                      nb_off[l], il_off[l], nb_idx[l], il_idx[l]);
        NNCA_LAUNCH_CHECK();
    }
    int64_t NB = 0, IL = 0;
    for (int l = 0; l <= kappa; ++l) { NB += nb_tot[l]; IL += il_tot[l]; }
    NNCA_REQUIRE(NB < (1ll << 31) && IL < (1ll << 31), NNCA_ERR_UNSUPPORTED, "list sizes exceed 2^31 entries");
    h->n_nb = NB;
    h->n_il = IL;
    h->nb_off = dalloc<int32_t>(h, h->ncell + 1);
    h->il_off = dalloc<int32_t>(h, h->ncell + 1);
    h->nb_idx = dalloc<int32_t>(h, NB);
    h->il_idx = dalloc<int32_t>(h, IL);
    int64_t eb = 0, ei = 0;
    for (int l = 0; l <= kappa; ++l) {
        const int64_t b0 = h->level_base[l], cnt = h->level_base[l + 1] - b0;
        k_offsets_to_global<<<grid_for(cnt + 1, 256), 256, 0, s>>>(nb_off[l], cnt, eb, b0, h->nb_off);
        NNCA_LAUNCH_CHECK();
        k_offsets_to_global<<<grid_for(cnt + 1, 256), 256, 0, s>>>(il_off[l], cnt, ei, b0, h->il_off);
        NNCA_LAUNCH_CHECK();
        if (nb_tot[l]) NNCA_CUDA(cudaMemcpyAsync(h->nb_idx + eb, nb_idx[l], nb_tot[l] * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (il_tot[l]) NNCA_CUDA(cudaMemcpyAsync(h->il_idx + ei, il_idx[l], il_tot[l] * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        eb += nb_tot[l];
        ei += il_tot[l];
    }
    // first level with a non-empty interaction list
    h->lmin = kappa + 1;
    for (int l = 0; l <= kappa; ++l)
        if (il_tot[l] > 0) { h->lmin = l; break; }
    NNCA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace nnca
