// Spatial reordering of a fit batch's kernels, an aid to the binning of
// Sec. IV-C and not part of the method: each image's kernels are permuted
// into tile-major order of their centres (ascending current index within a
// tile), so that kernels with consecutive indices are neighbours again after
// the fit has moved the centres.  Consecutive kernels then share tiles, which
// the binning's warp-aggregated walks and run merge exploit.  The model is
// the same set of kernels; only the order of the terms of the per-pixel sums
// changes (FP32 rounding).
//
//   k_centre_count / k_centre_scatter   counting sort of the kernels by the
//                                       tile of their centre (then the lists'
//                                       own sort: ascending index per tile)
//   k_move_rows                         gather a parameter set's rows into
//                                       the new order, then copy them back
//   k_move_order                        the same for the original-index map
#include "smoe_internal.cuh"

namespace smoe {

namespace {

constexpr int kThreads = 256;

// Global index of the tile holding kernel k's centre; centres outside the
// raster clamp to the nearest edge tile, a non-finite centre goes to its
// image's last tile.
__device__ __forceinline__ int64_t centre_tile(const Geo &g, int64_t k) {
    const ImgDev &im = img_of(g, img_by_kernel(g, k));
    const int64_t kl = k - im.k_off;
    const float mx = __fmul_rn(im.p.mu[2 * kl], (float)im.W);
    const float my = __fmul_rn(im.p.mu[2 * kl + 1], (float)im.H);
    int tx = im.tiles_x - 1, ty = im.tiles_y - 1;
    if (isfinite(mx) && isfinite(my)) {
        const float fx = floorf(__fdiv_rn(mx, (float)g.T));
        const float fy = floorf(__fdiv_rn(my, (float)g.T));
        tx = (int)fminf(fmaxf(fx, 0.0f), (float)(im.tiles_x - 1));
        ty = (int)fminf(fmaxf(fy, 0.0f), (float)(im.tiles_y - 1));
    }
    return im.t_off + (int64_t)ty * im.tiles_x + tx;
}

__global__ void k_centre_count(const __grid_constant__ Geo g, Bufs w) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (status_bad(w.status) || k >= g.K_total) return;
    atomicAdd(&w.tile_cnt[centre_tile(g, k)], 1);
}

// The prefix sum left each cursor at its tile's first slot; every id is its
// own block for the lists' sort (top bit set).
__global__ void k_centre_scatter(const __grid_constant__ Geo g, Bufs w) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (status_bad(w.status) || k >= g.K_total) return;
    w.pair_tmp[atomicAdd(&w.cursor[centre_tile(g, k)], 1)] = (int32_t)k | (int32_t)0x80000000u;
}

// Slot s receives kernel ids[s] (of the same image).  One thread per slot
// moves the whole row of parameter set SET (0 parameters, 1 first moments,
// 2 second moments): mu 2, chol 3, ea C, eW 2C and logpi 1 values.  Pass 0
// gathers the row of kernel ids[s] into scratch row s (GS floats per row);
// pass 1 copies scratch row s back to slot s.
template <int C, bool LIN, int SET>
__global__ void k_move_rows(const __grid_constant__ Geo g, const int32_t *__restrict__ ids,
                            float *__restrict__ scratch, int pass, const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= g.K_total) return;
    const ImgDev &im = img_of(g, img_by_kernel(g, s));
    const smoe_params &x = SET == 0 ? im.p : SET == 1 ? im.m : im.v;
    const int64_t r = (pass == 0 ? (int64_t)ids[s] : s) - im.k_off;   // the image's own row
    float *row = scratch + s * g.GS;
    float *dst[4] = {x.mu + 2 * r, x.chol + 3 * r, x.ea + C * r, LIN ? x.eW + 2 * C * r : nullptr};
    constexpr int n[4] = {2, 3, C, LIN ? 2 * C : 0};
    int at = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int j = 0; j < n[q]; ++j) {
            if (pass == 0) row[at + j] = dst[q][j];
            else dst[q][j] = row[at + j];
        }
        at += n[q];
    }
    if (x.logpi) {
        if (pass == 0) row[at] = x.logpi[r];
        else x.logpi[r] = row[at];
    }
}

// Each set in turn: gather into scratch, then copy back (the scratch holds
// one set).
template <int C, bool LIN>
void move_sets(const Geo &g, const int32_t *ids, float *scratch, const int32_t *status,
               unsigned blocks, int threads, cudaStream_t st) {
    for (int pass = 0; pass < 2; ++pass)
        k_move_rows<C, LIN, 0><<<blocks, threads, 0, st>>>(g, ids, scratch, pass, status);
    for (int pass = 0; pass < 2; ++pass)
        k_move_rows<C, LIN, 1><<<blocks, threads, 0, st>>>(g, ids, scratch, pass, status);
    for (int pass = 0; pass < 2; ++pass)
        k_move_rows<C, LIN, 2><<<blocks, threads, 0, st>>>(g, ids, scratch, pass, status);
}

__global__ void k_move_order(int64_t K, const int32_t *__restrict__ ids, int32_t *order,
                             int32_t *__restrict__ scratch, int pass, const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= K) return;
    if (pass == 0) scratch[s] = order[ids[s]];
    else order[s] = scratch[s];
}

__global__ void k_scatter_rows(const float *__restrict__ src, const int32_t *__restrict__ index,
                               int64_t base, int64_t K, int n, float *__restrict__ dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= K * n) return;
    const int64_t r = i / n;
    dst[((int64_t)index[r] - base) * n + (i - r * n)] = src[i];
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_reorder(const Geo &g, const Bufs &w, int32_t *order, cudaStream_t st) {
    const int64_t K = g.K_total, n = g.tiles_total;
    if (K == 0 || n == 0) return cudaSuccess;
    // Index scratch inside the record buffer (K x S ints, S >= 8; the next
    // binning rebuilds it): the ids as scattered, as sorted, and the order map.
    int32_t *tmp = reinterpret_cast<int32_t *>(w.rec);
    int32_t *ids = tmp + K;
    Bufs r = w;
    r.pair_tmp = tmp;
    r.pair_k = ids;
    r.huge = nullptr;                  // the centre lists have no queued kernels
    cudaError_t e = cudaMemsetAsync(w.tile_cnt, 0, sizeof(int32_t) * n, st);
    if (e != cudaSuccess) return e;
    k_centre_count<<<blocks_for(K), kThreads, 0, st>>>(g, r);
    e = launch_exscan(n, w.tile_cnt, w.bsum, w.tile_off, w.n_pairs, w.n_long, w.cursor, K,
                      w.status, st);
    if (e != cudaSuccess) return e;
    k_centre_scatter<<<blocks_for(K), kThreads, 0, st>>>(g, r);
    e = launch_sort_lists(g, r, st);
    if (e != cudaSuccess) return e;
    // Rows move through the gradient-sum buffer (K x GS floats, GS at least
    // the values per kernel; zero between iterations, so zeroed again after).
    const unsigned bk = blocks_for(K);
    if (g.C == 1 && !g.linear) move_sets<1, false>(g, ids, w.acc, w.status, bk, kThreads, st);
    else if (g.C == 1) move_sets<1, true>(g, ids, w.acc, w.status, bk, kThreads, st);
    else if (!g.linear) move_sets<3, false>(g, ids, w.acc, w.status, bk, kThreads, st);
    else move_sets<3, true>(g, ids, w.acc, w.status, bk, kThreads, st);
    if (order) {
        int32_t *ov = tmp + 2 * K;                  // after the ids, still in the record buffer
        for (int pass = 0; pass < 2; ++pass)
            k_move_order<<<blocks_for(K), kThreads, 0, st>>>(K, ids, order, ov, pass, w.status);
    }
    e = cudaMemsetAsync(w.acc, 0, sizeof(float) * g.GS * K, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_scatter_params(const smoe_params &src, const int32_t *index, int64_t base,
                                  int64_t K, int C, const smoe_params &dst, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const float *s[5] = {src.mu, src.chol, src.ea, src.eW, src.logpi};
    float *d[5] = {dst.mu, dst.chol, dst.ea, dst.eW, dst.logpi};
    const int width[5] = {2, 3, C, 2 * C, 1};
    for (int grp = 0; grp < 5; ++grp) {
        if (!s[grp] || !d[grp]) continue;
        k_scatter_rows<<<blocks_for(K * width[grp]), kThreads, 0, st>>>(s[grp], index, base, K,
                                                                      width[grp], d[grp]);
    }
    return cudaGetLastError();
}

}  // namespace smoe
