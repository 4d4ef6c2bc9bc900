// Internal declarations shared by the CUDA translation units of libsmoe.so.
//
// Data layout in HBM
//   - user parameters: FP32 SoA (mu[K][2] normalised, chol[K][3], ea[K][C],
//     eW[K][C][2]), see include/smoe.h;
//   - prepared record per kernel (written by the prep/bbox kernel, read by
//     every tile kernel with one contiguous load): S floats,
//       [0] mx  [1] my   centre in output pixels (float product mu * W)
//       [2] a   [3] b  [4] c   L / s
//       [5] log2(e) * logpi (the gate weight pi = exp(logpi), Eq. 4; 0 for pi = 1)
//       [6] spare
//       [7 + c*E + 0] ea_c, [7 + c*E + 1] eW_c0 / s, [7 + c*E + 2] eW_c1 / s
//     with E = 3 for linear and 1 for constant experts, S = round_up(7+C*E, 4)
//     (16 floats = 64 B for RGB linear experts);
//   - backward accumulator per kernel: GS floats of raw per-kernel sums
//     (see render.cu), GS = round_up(6 + C*E, 4);
//   - tile lists: CSR tile_off / pair_k over the global tile index of a batch
//     (image b's tiles start at t_off, row-major inside the image).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/smoe.h"

namespace smoe {

constexpr int kMaxC = 3;
// Rectangles of more tiles than this are queued by the binning (Bufs::huge).
#ifndef SMOE_HUGE_RECT
#define SMOE_HUGE_RECT 1024
#endif
constexpr int kHugeRect = SMOE_HUGE_RECT;
// Largest cutoff: exp(-q/2) of an included pair stays an FP32 normal number
// (q log2(e) / 2 <= 125.5), so no included kernel is flushed to zero.
constexpr float kMaxQmax = 174.0f;
// Largest tile table of one launch (the prefix sum's capacity, 4096 chunks).
constexpr int64_t kMaxTiles = 4096LL * 4096LL;

// A raster description every entry point accepts (host side): positive
// size, C 1 or 3, tile 8 / 16 / 32, known expert and gate modes, a cutoff in
// (0, kMaxQmax], a finite positive scale and a tile count within kMaxTiles.
inline bool desc_valid(const smoe_desc *d) {
    if (!d) return false;
    if (d->W <= 0 || d->H <= 0) return false;
    if (d->C != 1 && d->C != 3) return false;
    if (d->tile != 8 && d->tile != 16 && d->tile != 32) return false;
    if (d->expert != 0 && d->expert != 1) return false;
    if (d->gate != 0 && d->gate != 1) return false;
    if (!(d->qmax > 0.0f) || !(d->qmax <= kMaxQmax)) return false;
    if (!(d->scale > 0.0f) || !std::isfinite(d->scale)) return false;
    const int64_t tiles = (int64_t)((d->W + d->tile - 1) / d->tile) * ((d->H + d->tile - 1) / d->tile);
    return tiles <= kMaxTiles;
}
constexpr float kNegHalfLog2e = -0.72134752044448170368f;   // -log2(e) / 2
constexpr float kLog2e = 1.44269504088896340736f;

// One image of a launch.  Its kernels have global ids [k_off, k_off + K) and
// its tiles [t_off, t_off + tiles_x * tiles_y); p / m / v are the image's own
// SoA parameters and Adam moments (local kernel ids).
struct ImgDev {
    int32_t W, H, tiles_x, tiles_y;
    int64_t K, k_off, t_off;
    const float *target;
    smoe_params p, m, v;
    int32_t iters;
    float lr_mu0, lr_mu1, lr_chol, lr_ea, lr_eW, lr_pi;
    double mu_rho;         // per-iteration factor of the centre rate: (lr_mu1 / lr_mu0)^(1 / (iters - 1))
};

struct Geo {
    int32_t C, T, linear, S, GS;
    int32_t rbf;           // 1: RBF sum of Eq. 1 (y = N, D = 1); 0: softmax gates (Eq. 4)
    float qmax, scale;
    int32_t B;
    int64_t K_total, tiles_total;
    const ImgDev *table;   // device array of B entries, or nullptr (then `one`)
    ImgDev one;
};

struct Bufs {
    float *rec;
    int4 *rect;
    int32_t *tile_cnt;
    int32_t *cursor;
    long long *bsum;
    int32_t *pair_tmp;
    int32_t *long_q;     // tiles whose list is too long for the warp sort
    int32_t *n_long;
    float *acc;
    int32_t *tile_off;
    int32_t *pair_k;
    int64_t *n_pairs;
    int64_t pair_cap;
    int32_t *status;
    uint32_t *work;      // tile queue of the persistent fit launch (fit only)
    // Kernels whose rectangle holds more than kHugeRect tiles (a kernel that
    // a near-zero Cholesky entry stretches across the image): the binning
    // queues their ids here instead of walking their tiles, adds their
    // coverage to the tile counts one thread per tile and appends them to
    // each covered tile's list before the sort.  Null: every kernel walked.
    int32_t *huge;
    int32_t *n_huge;
    // Deterministic fit (all null otherwise): GS partial sums per (tile,
    // kernel) pair at the pair's list position, and a kernel-major index of
    // those positions: kernel k's pairs are pidx[koff[k] .. koff[k] +
    // kcnt[k] - 1], one per tile of its rectangle in row-major order (every
    // tile of the rectangle lists the kernel).  kcnt / koff / pidx are
    // written by the binning (areas, their exclusive scan, the index).
    float *part;
    int32_t *kcnt, *koff, *pidx;
    long long *kbsum;    // scan block sums of the kernel areas
    int64_t *ktot;       // their total (the pair count again)
    int32_t *kn_long;    // unused output of the scan
};

// Index entry of the (tile (tx, ty) of its image, kernel k) pair: the
// tile's row-major position inside the kernel's rectangle rc, after the
// kernel's first entry.
__device__ __forceinline__ int64_t part_slot(const Bufs &w, int64_t k, int4 rc, int tx, int ty) {
    return (int64_t)w.koff[k] + (int64_t)(ty - rc.y) * (rc.z - rc.x + 1) + (tx - rc.x);
}

// Deterministic gradient sums of kernel k: the partial sums of its (tile, k)
// pairs added in row-major tile order over its rectangle rc (the order of
// its index entries).  The loads are independent of each other.  GS sums,
// in registers.
template <int GS>
__device__ __forceinline__ void gather_sums(const Bufs &w, const ImgDev &im, int64_t k, int4 rc,
                                            float (&out)[GS]) {
#pragma unroll
    for (int q = 0; q < GS; ++q) out[q] = 0.0f;
    const int n = (rc.z - rc.x + 1) * (rc.w - rc.y + 1);
    const int32_t *idx = w.pidx + w.koff[k];
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
        const float4 *src = reinterpret_cast<const float4 *>(w.part + (int64_t)idx[i] * GS);
#pragma unroll
        for (int q = 0; q < GS / 4; ++q) {
            const float4 v = src[q];
            out[4 * q] += v.x; out[4 * q + 1] += v.y; out[4 * q + 2] += v.z; out[4 * q + 3] += v.w;
        }
    }
}

__host__ __device__ inline int rec_stride(int C, int linear) {
    return (7 + C * (linear ? 3 : 1) + 3) & ~3;
}
__host__ __device__ inline int acc_stride(int C, int linear) {
    return (6 + C * (linear ? 3 : 1) + 3) & ~3;
}

__device__ __forceinline__ const ImgDev &img_of(const Geo &g, int b) {
    return g.table ? g.table[b] : g.one;
}

// Image that owns global kernel k / global tile t (binary search, B small).
__device__ __forceinline__ int img_by_kernel(const Geo &g, int64_t k) {
    if (!g.table) return 0;
    int lo = 0, hi = g.B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g.table[mid].k_off <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int img_by_tile(const Geo &g, int64_t t) {
    if (!g.table) return 0;
    int lo = 0, hi = g.B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g.table[mid].t_off <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Hardware base-2 exponential (MUFU.EX2), flush-to-zero.  Arguments on the
// hot path lie in [-0.72 q_max, 0], far from the subnormal range.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Truncation predicate pieces, one IEEE rounding per step (no contraction):
//   per row:   dy = y0 - my, t = b*dy, z1 = c*dy, u = z1*z1
//   per pixel: dx = x0 - mx, z0 = fma(a, dx, t), q = fma(z0, z0, u)
__device__ __forceinline__ float q_of(float a, float dx, float t, float u, float &z0) {
    z0 = __fmaf_rn(a, dx, t);
    return __fmaf_rn(z0, z0, u);
}

// Gate numerator for a pair: exp(-q/2) if q <= q_max else 0.
__device__ __forceinline__ float gate_e(float q, float qmax) {
    float e = ex2(__fmul_rn(q, kNegHalfLog2e));
    return q <= qmax ? e : 0.0f;
}

__device__ __forceinline__ bool status_bad(const int32_t *status) {
    return status && *(volatile const int32_t *)status != 0;
}

// --------------------------------------------------------------------------
// launchers (host side, no synchronisation)
// --------------------------------------------------------------------------
cudaError_t launch_bin(const Geo &g, const Bufs &w, cudaStream_t st);
// Sort every tile's segment pair_tmp[tile_off[t] .. tile_off[t+1]) into
// pair_k in ascending order (the last step of launch_bin).
cudaError_t launch_sort_lists(const Geo &g, const Bufs &w, cudaStream_t st);
// Spatial reordering of a fit batch's kernels (see smoe_fit_reorder).
cudaError_t launch_reorder(const Geo &g, const Bufs &w, int32_t *order, cudaStream_t st);
// dst row index[i] - base <- src row i, for every group present in both sets.
cudaError_t launch_scatter_params(const smoe_params &src, const int32_t *index, int64_t base,
                                  int64_t K, int C, const smoe_params &dst, cudaStream_t st);
cudaError_t launch_render(const Geo &g, const Bufs &w, float *y, float *inv_d,
                          cudaStream_t st);
// Exclusive prefix sum of n counters into off[0..n] (off[n] = min(total, cap),
// *total = the sum, cursor[i] = off[i] (a scatter's first slot); a total above cap sets
// SMOE_ERR_CAPACITY); needs ceil(n / 4096) entries of bsum.
cudaError_t launch_exscan(int64_t n, const int32_t *cnt, long long *bsum, int32_t *off,
                          int64_t *total, int32_t *n_long, int32_t *cursor, int64_t cap,
                          int32_t *status, cudaStream_t st);
// Scratch of smoe_render_points: per-tile counts / cursors / offsets of the
// points, prefix-sum block sums, each point's tile and the tile-sorted order.
struct PointBufs {
    int32_t *cnt, *cursor, *off, *pt_tile, *order, *n_long;
    long long *bsum;
    int64_t *n_in;
};
// Adds to *out the number of (pixel, kernel) pairs of the lists with q <= q_max.
cudaError_t launch_count_inrange(const Geo &g, const float *rec, const int32_t *tile_off,
                                 const int32_t *pair_k, unsigned long long *out,
                                 const int32_t *status, cudaStream_t st);
// out = f * in elementwise (one rounding), n floats.
cudaError_t launch_scale(const float *in, float *out, int64_t n, float f, cudaStream_t st);
// y(x) of one model (g.B == 1) at n points xy (n x 2, pixel units of g.one's
// raster) from the model's prepared records and tile lists.
cudaError_t launch_render_points(const Geo &g, const float *rec, const int32_t *tile_off,
                                 const int32_t *pair_k, int64_t n, const float *xy,
                                 const PointBufs &pb, float *y, float *inv_d,
                                 const int32_t *status, cudaStream_t st);
// Mean of the renders of a batch's B models (all images one size), Eq. 11.
cudaError_t launch_render_mean(const Geo &g, const Bufs &w, float *y, cudaStream_t st);
cudaError_t launch_render_bwd(const Geo &g, const Bufs &w, const float *y, const float *inv_d,
                              const float *gy, const float *target, const smoe_params &grad,
                              cudaStream_t st);
cudaError_t launch_fit_tiles(const Geo &g, const Bufs &w, double *loss, int32_t hist,
                             const int32_t *step, bool persistent, cudaStream_t st);
cudaError_t launch_adam_soa(const smoe_params &p, const smoe_params &gr, const smoe_params &m,
                            const smoe_params &v, int C, const float lr[5], double b1, double b2,
                            double eps, int32_t step, cudaStream_t st);
cudaError_t launch_fit_adam(const Geo &g, const Bufs &w, double b1, double b2, double eps,
                            int32_t *step, uint32_t *done, float *coef, cudaStream_t st);
// The finalized gradients of the fit's current iteration (the sums of the
// fused tile launch through the same chain rule as launch_fit_adam) written
// to grad at the batch's global kernel index; zeroes the atomic sums.
cudaError_t launch_fit_grads(const Geo &g, const Bufs &w, const int32_t *step,
                             const smoe_params &grad, cudaStream_t st);
cudaError_t launch_adam_coefs(const Geo &g, const int32_t *step, double b1, double b2,
                              float *coef, cudaStream_t st);
cudaError_t launch_sq_error(const float *y, const float *t, int64_t n, int clamp, double *out,
                            cudaStream_t st);

}  // namespace smoe
