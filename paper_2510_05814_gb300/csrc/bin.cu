// Binning: the "geometry shader" (Sec. IV-B) and the subset kernel selection
// per block (Sec. IV-C, Eq. 5) as a counting sort of (tile, kernel) pairs.
//
//   k_prep_bbox     one thread per kernel: prepared record, tile rectangle,
//                   per-tile counts (one atomic per tile of a warp's union box
//                   when the warp's rectangles are compact, else one per
//                   covered tile; a large rectangle is walked by the whole warp)
//   k_scan_*        exclusive prefix sum of the per-tile counts -> tile_off
//                   (three phases: block sums, scan of the sums, block scans)
//   k_scatter       one thread per kernel: a slot in each covered tile (claimed
//                   per union tile for the warp, or one atomic per tile)
//   k_segsort_warp  one warp per tile: restore ascending kernel order for lists
//                   of up to 512 ids (register bitonic sorts; from 129 ids on
//                   first a merge of the ascending per-warp runs the
//                   aggregated scatter writes)
//   k_segsort_long  one CTA per longer list (up to 1024 ids the run merge
//                   first; a bitonic sort in shared memory up to 2048 ids, a
//                   bitmap sweep over the kernel-id range above)
//
// The per-tile lists are the unique sets {k : tile in rect_k} in ascending k,
// so the output is bit-exact whatever order the atomics took.
#include "smoe_internal.cuh"

namespace smoe {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr int kSortThreads = 256;
constexpr int kSortMax = 2048;                 // bitonic in shared memory up to this
constexpr int kBitmapWords = 8192;             // 262144 kernel ids per bitmap pass
constexpr int kLongGrid = 152;                 // CTAs sweeping the queue of long lists (> 512 ids)
#ifndef SMOE_BIN_BIG
#define SMOE_BIN_BIG 32
#endif
#ifndef SMOE_BIN_AGG
#define SMOE_BIN_AGG 128
#endif
constexpr int kBig = SMOE_BIN_BIG;             // rectangles of more tiles are walked by a whole warp
// The scatter marks the first id of every block it writes contiguously and
// in ascending order (a warp's covering kernels, or a single id) in the top
// bit of the 32-bit slot; ids are below 2^31.  The sorts strip it.
constexpr int32_t kBlockHead = (int32_t)0x80000000u;
constexpr int32_t kIdMask = 0x7fffffff;

// Add 1 to the count (or claim a slot) of every tile of the rectangles of
// the warp's kernels.  Small rectangles are walked by their own lane; a large
// one (a wide or degenerate kernel, up to the whole image) by the whole warp.
template <bool SCATTER>
__device__ __forceinline__ void walk_rects(const Bufs &w, bool valid, int4 rect, int64_t t_off,
                                           int tiles_x, int32_t k) {
    const int lane = threadIdx.x & 31;
    const int wdt = rect.z - rect.x + 1;
    const int n = valid && rect.x <= rect.z ? wdt * (rect.w - rect.y + 1) : 0;
    auto visit = [&](int64_t t, int32_t kid) {
        if (SCATTER) w.pair_tmp[atomicAdd(&w.cursor[t], 1)] = kid | kBlockHead;
        else atomicAdd(&w.tile_cnt[t], 1);
    };
    if (n <= kBig) {             // small rectangles: each lane walks its own
        if (SCATTER) {
            // four slot claims in flight before their stores
            int tx = rect.x;
            int64_t row = t_off + (int64_t)rect.y * tiles_x;
            for (int i = 0; i < n; i += 4) {
                int slot[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    slot[u] = -1;
                    if (i + u < n) {
                        slot[u] = atomicAdd(&w.cursor[row + tx], 1);
                        if (++tx > rect.z) { tx = rect.x; row += tiles_x; }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (slot[u] >= 0) w.pair_tmp[slot[u]] = k | kBlockHead;
            }
        } else {
            for (int ty = rect.y; n > 0 && ty <= rect.w; ++ty)
                for (int tx = rect.x; tx <= rect.z; ++tx)
                    visit(t_off + (int64_t)ty * tiles_x + tx, k);
        }
    }
    unsigned big = __ballot_sync(0xffffffffu, n > kBig);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const int4 r = make_int4(__shfl_sync(0xffffffffu, rect.x, src),
                                 __shfl_sync(0xffffffffu, rect.y, src),
                                 __shfl_sync(0xffffffffu, rect.z, src),
                                 __shfl_sync(0xffffffffu, rect.w, src));
        const int64_t to = __shfl_sync(0xffffffffu, t_off, src);
        const int tx_n = __shfl_sync(0xffffffffu, tiles_x, src);
        const int32_t kk = __shfl_sync(0xffffffffu, k, src);
        const int rw = r.z - r.x + 1, nn = rw * (r.w - r.y + 1);
        if (SCATTER) {
            // four slot claims in flight per lane before their stores
            for (int i0 = lane; i0 < nn; i0 += 128) {
                int slot[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + 32 * u;
                    slot[u] = i < nn ? atomicAdd(&w.cursor[to + (int64_t)(r.y + i / rw) * tx_n +
                                                           r.x + i % rw], 1)
                                     : -1;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (slot[u] >= 0) w.pair_tmp[slot[u]] = kk | kBlockHead;
            }
        } else {
            for (int i = lane; i < nn; i += 32)
                visit(to + (int64_t)(r.y + i / rw) * tx_n + r.x + i % rw, kk);
        }
    }
}

// Per-warp aggregation of the walks.  A warp's 32 consecutive kernels are
// mostly neighbours, so their rectangles overlap.  The union box of the
// warp's small rectangles (at most kBig tiles each) is visited tile by tile:
// each box tile gets the number of the warp's kernels covering it (large
// ones included) with one atomic, and the scatter places the covering
// kernels at base + their rank in lane order, so each warp leaves one
// ascending block of ids per tile.  The parts of large rectangles outside
// the box are walked tile by tile by the whole warp.  Warps whose box spans
// two images, holds more than kAggMax tiles or no fewer tiles than the small
// rectangles' total walk lane by lane (walk_rects).  Both passes take the
// same decisions from the same rectangles, so counts and slots agree.
constexpr int kAggMax = SMOE_BIN_AGG;
constexpr int kBinThreads = 256;

struct WarpAgg {
    int4 rect[32];              // the warp's rectangles
    int base[kAggMax];          // scatter, per box tile: first slot claimed for the warp
    unsigned bal[kAggMax];      // and the lanes covering it
};

template <bool SCATTER>
__device__ __forceinline__ void walk_warp(const Bufs &w, bool valid, int4 rect, int64_t t_off,
                                          int tiles_x, int32_t k, WarpAgg &wa) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool has = valid && rect.x <= rect.z && rect.y <= rect.w;
    const unsigned any = __ballot_sync(full, has);
    if (!any) return;
    const int src = __ffs(any) - 1;
    // the image of the warp's kernels with a rectangle: every lane, also one
    // of another image whose rectangle is empty, indexes that image's tiles
    const int64_t t0 = __shfl_sync(full, t_off, src);
    const int tx_n = __shfl_sync(full, tiles_x, src);
    const bool one_image = __all_sync(full, !has || t_off == t0);
    const int own = has ? (rect.z - rect.x + 1) * (rect.w - rect.y + 1) : 0;
    const bool small = has && own <= kBig;
    const int ux0 = __reduce_min_sync(full, small ? rect.x : 0x7fffffff);
    const int uy0 = __reduce_min_sync(full, small ? rect.y : 0x7fffffff);
    const int ux1 = __reduce_max_sync(full, small ? rect.z : -1);
    const int uy1 = __reduce_max_sync(full, small ? rect.w : -1);
    const int uw = ux1 - ux0 + 1;
    const long long nu = ux1 >= 0 ? (long long)uw * (uy1 - uy0 + 1) : 0;
    const unsigned total = __reduce_add_sync(full, small ? (unsigned)own : 0u);
    if (!one_image || nu == 0 || nu > kAggMax || nu >= (long long)total) {
        walk_rects<SCATTER>(w, valid, rect, t_off, tiles_x, k);
        return;
    }
    // One box tile per lane: the mask of the warp's lanes covering it (the
    // rectangles from shared memory); the count adds its popcount, the
    // scatter claims that many slots and keeps the mask for the ranks.
    wa.rect[lane] = has ? rect : make_int4(1, 1, 0, 0);
    __syncwarp();
    for (int u = lane; u < (int)nu; u += 32) {
        const int tx = ux0 + u % uw, ty = uy0 + u / uw;
        unsigned msk = 0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) {
            const int4 r = wa.rect[l];
            msk |= (r.x <= tx && tx <= r.z && r.y <= ty && ty <= r.w) ? 1u << l : 0u;
        }
        const int64_t t = t0 + (int64_t)ty * tx_n + tx;
        if (SCATTER) {
            wa.bal[u] = msk;
            if (msk) wa.base[u] = atomicAdd(&w.cursor[t], __popc(msk));
        } else if (msk) {
            atomicAdd(&w.tile_cnt[t], __popc(msk));
        }
    }
    __syncwarp();
    if (SCATTER && has) {
        // each lane places its kernel in its tiles inside the box
        const unsigned lower = (1u << lane) - 1u;
        const int y0 = max(rect.y, uy0), y1 = min(rect.w, uy1);
        const int x0 = max(rect.x, ux0), x1 = min(rect.z, ux1);
        for (int y = y0; y <= y1; ++y) {
            const int ub = (y - uy0) * uw - ux0;
            for (int x = x0; x <= x1; ++x) {
                const int uu = ub + x;
                const int rank = __popc(wa.bal[uu] & lower);
                w.pair_tmp[wa.base[uu] + rank] = rank ? k : (k | kBlockHead);
            }
        }
    }
    // the parts of large rectangles outside the box, one rectangle at a time
    unsigned big = __ballot_sync(full, has && !small &&
                                           !(rect.x >= ux0 && rect.z <= ux1 && rect.y >= uy0 &&
                                             rect.w <= uy1));
    while (big) {
        const int bl = __ffs(big) - 1;
        big &= big - 1;
        const int4 r = wa.rect[bl];
        const int32_t kk = __shfl_sync(full, k, bl);
        const int rw = r.z - r.x + 1, nn = rw * (r.w - r.y + 1);
        // four tiles per lane at a time: the scatter's slot claims in flight
        // before their stores
        for (int i0 = lane; i0 < nn; i0 += 128) {
            int slot[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u;
                slot[u] = -1;
                if (i >= nn) continue;
                const int tx = r.x + i % rw, ty = r.y + i / rw;
                if (tx >= ux0 && tx <= ux1 && ty >= uy0 && ty <= uy1) continue;
                const int64_t t = t0 + (int64_t)ty * tx_n + tx;
                if (SCATTER) slot[u] = atomicAdd(&w.cursor[t], 1);
                else atomicAdd(&w.tile_cnt[t], 1);
            }
            if (SCATTER)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (slot[u] >= 0) w.pair_tmp[slot[u]] = kk | kBlockHead;
        }
    }
    __syncwarp();
}

// A rectangle the binning queues instead of walking (see Bufs::huge).
__device__ __forceinline__ bool is_huge(const Bufs &w, int4 r) {
    return w.huge && r.x <= r.z && (r.z - r.x + 1) * (r.w - r.y + 1) > kHugeRect;
}

__global__ void __launch_bounds__(kBinThreads, 4) k_prep_bbox(const __grid_constant__ Geo g, Bufs w) {
    __shared__ WarpAgg agg[kBinThreads / 32];
    if (status_bad(w.status)) return;
    const int64_t k_raw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = k_raw < g.K_total;
    const int64_t k = valid ? k_raw : g.K_total - 1;   // inactive lanes mirror the last kernel
    const ImgDev &im = img_of(g, img_by_kernel(g, k));
    const int64_t kl = k - im.k_off;                   // the image's own kernel index
    // Every input is loaded before the first store (the record's stores may
    // alias nothing, but the compiler cannot know that): one memory round
    // trip per kernel instead of one per channel.
    const float mu0 = im.p.mu[2 * kl], mu1 = im.p.mu[2 * kl + 1];
    float a = im.p.chol[3 * kl], b = im.p.chol[3 * kl + 1], c = im.p.chol[3 * kl + 2];
    const float lp = im.p.logpi ? im.p.logpi[kl] : 0.0f;
    float ex[3], w0[3], w1[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const bool on = ch < g.C;
        ex[ch] = on ? im.p.ea[kl * g.C + ch] : 0.0f;
        w0[ch] = on && g.linear ? im.p.eW[(kl * g.C + ch) * 2] : 0.0f;
        w1[ch] = on && g.linear ? im.p.eW[(kl * g.C + ch) * 2 + 1] : 0.0f;
    }
    // Kernel in output-pixel units, one rounding per operation.
    const float mx = __fmul_rn(mu0, (float)im.W);
    const float my = __fmul_rn(mu1, (float)im.H);
    const bool scaled = g.scale != 1.0f;
    if (scaled) {
        a = __fdiv_rn(a, g.scale);
        b = __fdiv_rn(b, g.scale);
        c = __fdiv_rn(c, g.scale);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            w0[ch] = __fdiv_rn(w0[ch], g.scale);
            w1[ch] = __fdiv_rn(w1[ch], g.scale);
        }
    }
    if (valid) {
        // record: [0..4] mx my a b c, [5] log2 pi, [6] 0, [7 + ch E + e] experts,
        // zero-padded to S floats (S <= 16), written as float4
        float r[16];
        r[0] = mx; r[1] = my; r[2] = a; r[3] = b; r[4] = c;
        r[5] = __fmul_rn(lp, kLog2e);              // pi = 1 stores 0
#pragma unroll
        for (int x = 6; x < 16; ++x) r[x] = 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (ch < g.C) {
                if (g.linear) {
                    r[7 + 3 * ch] = ex[ch]; r[8 + 3 * ch] = w0[ch]; r[9 + 3 * ch] = w1[ch];
                } else {
                    r[7 + ch] = ex[ch];
                }
            }
        }
        float4 *dst = reinterpret_cast<float4 *>(w.rec + k * g.S);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * q < g.S) dst[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }

    // Bounding box: square of half side r = sqrt(q_max * lambda_max(Sigma))
    // * (1 + 2^-10), lambda_max(Sigma) = lambda_max(P) / det(P), P = L L^T.
    int4 rect = make_int4(0, 0, -1, -1);
    const bool finite = isfinite(mx) && isfinite(my) && isfinite(a) && isfinite(b) && isfinite(c);
    if (finite) {
        float p00 = __fmul_rn(a, a);
        float p01 = __fmul_rn(a, b);
        float cc = __fmul_rn(c, c);
        float p11 = __fmaf_rn(b, b, cc);
        float h = __fmul_rn(0.5f, __fsub_rn(p00, p11));
        float p01sq = __fmul_rn(p01, p01);
        float rt = __fsqrt_rn(__fmaf_rn(h, h, p01sq));
        float half_tr = __fmul_rn(0.5f, __fadd_rn(p00, p11));
        float lmax_p = __fadd_rn(half_tr, rt);
        float ac = __fmul_rn(a, c);
        float det = __fmul_rn(ac, ac);
        bool whole = false;
        float lo_x = 0.f, hi_x = 0.f, lo_y = 0.f, hi_y = 0.f;
        if (det == 0.0f) {
            whole = true;
        } else {
            float lmax_s = __fdiv_rn(lmax_p, det);
            float rad = __fsqrt_rn(__fmul_rn(g.qmax, lmax_s));
            rad = __fmul_rn(rad, 1.0f + 0x1p-10f);
            const float T = (float)g.T;
            lo_x = __fdiv_rn(__fsub_rn(mx, rad), T);
            hi_x = __fdiv_rn(__fadd_rn(mx, rad), T);
            lo_y = __fdiv_rn(__fsub_rn(my, rad), T);
            hi_y = __fdiv_rn(__fadd_rn(my, rad), T);
            if (!isfinite(rad) || !isfinite(lo_x) || !isfinite(hi_x) || !isfinite(lo_y) ||
                !isfinite(hi_y))
                whole = true;
        }
        if (whole) {
            rect = make_int4(0, 0, im.tiles_x - 1, im.tiles_y - 1);
        } else {
            float fx0 = fmaxf(floorf(lo_x), 0.0f);
            float fy0 = fmaxf(floorf(lo_y), 0.0f);
            float fx1 = fminf(floorf(hi_x), (float)(im.tiles_x - 1));
            float fy1 = fminf(floorf(hi_y), (float)(im.tiles_y - 1));
            if (fx0 <= fx1 && fy0 <= fy1)
                rect = make_int4((int)fx0, (int)fy0, (int)fx1, (int)fy1);
        }
    }
    if (valid) w.rect[k] = rect;
    if (valid && w.kcnt)    // deterministic fit: the kernel's pair count (rectangle area)
        w.kcnt[k] = rect.x <= rect.z ? (rect.z - rect.x + 1) * (rect.w - rect.y + 1) : 0;
    int4 walk = rect;
    if (valid && is_huge(w, rect)) {      // counted per tile by k_huge_cover instead
        w.huge[atomicAdd(w.n_huge, 1)] = (int32_t)k;
        walk = make_int4(0, 0, -1, -1);
    }
    walk_warp<false>(w, valid, walk, im.t_off, im.tiles_x, (int32_t)k, agg[threadIdx.x >> 5]);
}

// Block-wide exclusive scan of one long long per thread (1024 threads).
__device__ long long block_exscan(long long v, long long *total) {
    __shared__ long long warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        long long s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    long long base = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(int64_t n, const int32_t *cnt,
                                                              long long *bsum,
                                                              const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += cnt[base + i];
    long long total;
    block_exscan(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int nb, long long *bsum, int64_t n,
                                                           int32_t *tile_off, int64_t *n_pairs,
                                                           int32_t *n_long, int64_t cap,
                                                           int32_t *status) {
    if (status_bad(status)) return;
    // nb <= kScanChunk: each thread scans up to kScanItems consecutive sums.
    const int base = threadIdx.x * kScanItems;
    long long v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < nb ? bsum[base + i] : 0;
        s += v[i];
    }
    long long total;
    long long run = block_exscan(s, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < nb) bsum[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) {
        *n_pairs = total;
        *n_long = 0;
        tile_off[n] = (int32_t)(total < cap ? total : cap);
        if (total > cap) atomicCAS(status, 0, (int32_t)SMOE_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(int64_t n, const int32_t *cnt,
                                                            const long long *bsum,
                                                            int32_t *tile_off, int32_t *cursor,
                                                            int64_t cap,
                                                            const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
    long long v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? cnt[base + i] : 0;
        s += v[i];
    }
    long long total;
    long long run = block_exscan(s, &total) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) {
            const int32_t o = (int32_t)(run < cap ? run : cap);
            tile_off[base + i] = o;
            cursor[base + i] = o;                 // scatter cursor: the tile's first slot
        }
        run += v[i];
    }
}

__global__ void __launch_bounds__(kBinThreads) k_scatter(const __grid_constant__ Geo g, Bufs w) {
    __shared__ WarpAgg agg[kBinThreads / 32];
    if (status_bad(w.status)) return;
    const int64_t k_raw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = k_raw < g.K_total;
    const int64_t k = valid ? k_raw : g.K_total - 1;
    int4 rect = w.rect[k];
    if (is_huge(w, rect)) rect = make_int4(0, 0, -1, -1);   // appended by k_segsort_warp
    const ImgDev &im = img_of(g, img_by_kernel(g, k));
    walk_warp<true>(w, valid, rect, im.t_off, im.tiles_x, (int32_t)k, agg[threadIdx.x >> 5]);
}

// Coverage of the queued (huge) rectangles, one thread per tile: each tile's
// count gains the number of queued rectangles of its image that hold it (the
// count kernel's atomics are complete; the prefix sum follows).
constexpr int kHugeThreads = 256;

__global__ void __launch_bounds__(kHugeThreads) k_huge_cover(const __grid_constant__ Geo g,
                                                             Bufs w) {
    __shared__ int4 hr[kHugeThreads];
    __shared__ int hb[kHugeThreads];
    if (status_bad(w.status)) return;
    const int nh = *w.n_huge;
    if (nh == 0) return;                      // the same for every thread
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool in = t < g.tiles_total;
    int b = -1, tx = 0, ty = 0;
    if (in) {
        b = img_by_tile(g, t);
        const ImgDev &im = img_of(g, b);
        const int64_t local = t - im.t_off;
        tx = (int)(local % im.tiles_x);
        ty = (int)(local / im.tiles_x);
    }
    int cnt = 0;
    for (int c0 = 0; c0 < nh; c0 += kHugeThreads) {
        __syncthreads();
        const int i = c0 + (int)threadIdx.x;
        if (i < nh) {
            const int32_t k = w.huge[i];
            hr[threadIdx.x] = w.rect[k];
            hb[threadIdx.x] = img_by_kernel(g, k);
        }
        __syncthreads();
        const int m = min(kHugeThreads, nh - c0);
        for (int j = 0; j < m; ++j) {
            const int4 r = hr[j];
            cnt += (hb[j] == b && r.x <= tx && tx <= r.z && r.y <= ty && ty <= r.w) ? 1 : 0;
        }
    }
    if (in && cnt) w.tile_cnt[t] += cnt;
}

__device__ int block_exscan_int(int v, int *total) {
    __shared__ int ws[kSortThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    int base = 0, tot = 0;
    for (int i = 0; i < kSortThreads / 32; ++i) {
        if (i < wid) base += ws[i];
        tot += ws[i];
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

__device__ void segsort_tile(const Geo &g, const Bufs &w, int64_t t, uint32_t *s);

// Bitonic sort of the warp's 32 E ids in registers, ascending; element
// p = lane E + i.  Compare-exchange stages whose partner is in another lane
// (distance j >= E) go through shuffles, the others stay inside the lane.
template <int E, typename V>
__device__ __forceinline__ void warp_bitonic(V (&v)[E], int lane) {
    constexpr int P = 32 * E;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const bool up = ((lane * E + i) & k) == 0;
                    const V o = __shfl_xor_sync(0xffffffffu, v[i], lj);
                    v[i] = (lower == up) ? min(v[i], o) : max(v[i], o);
                }
            } else {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int ip = i ^ j;
                    if (ip > i) {
                        const bool up = ((lane * E + i) & k) == 0;
                        const V a = v[i], b = v[ip];
                        v[i] = up ? min(a, b) : max(a, b);
                        v[ip] = up ? max(a, b) : min(a, b);
                    }
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_list(const Bufs &w, int64_t start, int n, int lane) {
    int v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = lane * E + i;
        v[i] = p < n ? w.pair_tmp[start + p] & kIdMask : 0x7fffffff;
    }
    warp_bitonic<E, int>(v, lane);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = lane * E + i;
        if (p < n) w.pair_k[start + p] = v[i];
    }
}

// The scatter writes each list as blocks, each marked at its first id and
// ascending (a warp's covering kernels, or a single id), placed in any order.
// When every block is ascending, there are at most kMaxRuns of them and,
// ordered by their first ids, each starts above the end of the one before,
// the sorted list is the blocks in that order: sort the first ids (two per
// lane), scan the block lengths, move each id.  Returns false, having
// written nothing, when the list is not of that form (the caller sorts it in
// full).  E ids per lane: n <= 32 E.
constexpr int kMaxRuns = 64;

struct WarpRuns {
    int start[kMaxRuns + 1], dest[kMaxRuns];
    int first[kMaxRuns], last[kMaxRuns];
};

template <int E>
__device__ __forceinline__ bool warp_merge_runs(const Bufs &w, int64_t start, int n, int lane,
                                                WarpRuns &sr) {
    const unsigned full = 0xffffffffu;
    int v[E];
    unsigned hmask = 0;                                // bit i: element i opens a block
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = lane * E + i;
        const int raw = p < n ? w.pair_tmp[start + p] : kIdMask;
        v[i] = raw & kIdMask;
        if (p < n && (raw < 0 || p == 0)) hmask |= 1u << i;
    }
    const int prev_last = __shfl_up_sync(full, v[E - 1], 1);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = lane * E + i;
        if (p < n && !((hmask >> i) & 1u) && v[i] <= (i ? v[i - 1] : prev_last)) ok = false;
    }
    if (!__all_sync(full, ok)) return false;
    const int hc = __popc(hmask);
    int incl = hc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    const int R = __shfl_sync(full, incl, 31);
    if (R > kMaxRuns) return false;
    // block starts, first and last ids (an element ends its block when the
    // next one opens a block or the list ends)
    const unsigned next_first = __shfl_down_sync(full, hmask & 1u, 1);
    int r = incl - hc;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = lane * E + i;
        if ((hmask >> i) & 1u) {
            sr.start[r] = p;
            sr.first[r] = v[i];
            ++r;
        }
        const bool ends = p == n - 1 ||
                          (i + 1 < E ? ((hmask >> (i + 1)) & 1u) != 0 : (lane < 31 && next_first));
        if (p < n && ends) sr.last[r - 1] = v[i];
    }
    if (lane == 0) sr.start[R] = n;
    __syncwarp();
    // blocks by first id: first << 32 | block, two per lane
    constexpr int KE = kMaxRuns / 32;
    unsigned long long x[KE];
#pragma unroll
    for (int e = 0; e < KE; ++e) {
        const int b = KE * lane + e;
        x[e] = b < R ? ((unsigned long long)(unsigned)sr.first[b] << 32) | (unsigned)b : ~0ull;
    }
    warp_bitonic<KE, unsigned long long>(x, lane);
    // each block starts above the end of the block before it
    const unsigned long long prev = __shfl_up_sync(full, x[KE - 1], 1);
    bool disjoint = true;
#pragma unroll
    for (int e = 0; e < KE; ++e) {
        const int q = KE * lane + e;
        const unsigned long long pq = e ? x[e - 1] : prev;
        if (q > 0 && q < R &&
            (int)(x[e] >> 32) <= sr.last[(int)(pq & 0xffffffffull)])
            disjoint = false;
    }
    if (!__all_sync(full, disjoint)) return false;
    int len[KE], d = 0;
#pragma unroll
    for (int e = 0; e < KE; ++e) {
        const int q = KE * lane + e;
        const int bi = (int)(x[e] & 0xffffffffull);
        len[e] = q < R ? sr.start[bi + 1] - sr.start[bi] : 0;
        d += len[e];
    }
    int incl_d = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, incl_d, o);
        if (lane >= o) incl_d += y;
    }
    int at = incl_d - d;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < KE; ++e) {
        const int q = KE * lane + e;
        if (q < R) sr.dest[x[e] & 0xffffffffull] = at;
        at += len[e];
    }
    __syncwarp();
    int rb = incl - hc - 1;                            // block of the elements before my first head
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = lane * E + i;
        if (p < n) {
            if ((hmask >> i) & 1u) ++rb;
            w.pair_k[start + sr.dest[rb] + (p - sr.start[rb])] = v[i];
        }
    }
    __syncwarp();
    return true;
}

// One warp per tile: lists of up to 512 ids are sorted in registers (a
// bitonic sort of the smallest power of two >= 32 that holds the list, 1 to
// 16 ids per lane; from 129 ids on the run merge first); longer ones are
// queued for k_segsort_long.
constexpr int kShortSortThreads = 128;

// The sort kernel's CTAs take 8 tiles, so that a pass over the queue of
// huge kernels is staged in shared memory once for 8 tiles.
#ifndef SMOE_SEGSORT_THREADS
#define SMOE_SEGSORT_THREADS 256
#endif
constexpr int kSegThreads = SMOE_SEGSORT_THREADS;
constexpr int kHugeStage = kSegThreads;          // queued kernels staged per pass

__global__ void __launch_bounds__(kSegThreads) k_segsort_warp(const __grid_constant__ Geo g,
                                                              int64_t n_tiles, Bufs w) {
    __shared__ WarpRuns runs[kSegThreads / 32];
    __shared__ int4 hq_rect[kHugeStage];
    __shared__ int32_t hq_k[kHugeStage], hq_b[kHugeStage];
    if (status_bad(w.status)) return;
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const bool tile_ok = t < n_tiles;
    // queued kernels appended to this list: each is a block of its own and
    // they span the kernel order, so the block merge below would not apply
    // (the list takes the full sort)
    int n_app = 0;
    const int nh = w.huge ? *w.n_huge : 0;         // the same for every thread
    if (nh > 0) {
        // the queued (huge) kernels that hold this tile go after the slots the
        // scatter filled, up to the tile's end, each as its own block; the
        // queue passes through shared memory a CTA-wide pass at a time
        int b = -1, tx = 0, ty = 0;
        int32_t at = 0;
        if (tile_ok) {
            b = img_by_tile(g, t);
            const ImgDev &im = img_of(g, b);
            const int64_t local = t - im.t_off;
            tx = (int)(local % im.tiles_x);
            ty = (int)(local / im.tiles_x);
            at = w.cursor[t];
        }
        for (int c0 = 0; c0 < nh; c0 += kHugeStage) {
            __syncthreads();                           // the previous pass is read
            const int i = c0 + (int)threadIdx.x;
            if (i < nh) {
                const int32_t k = w.huge[i];
                hq_k[threadIdx.x] = k;
                hq_rect[threadIdx.x] = w.rect[k];
                hq_b[threadIdx.x] = img_by_kernel(g, k);
            }
            __syncthreads();
            const int m = min(kHugeStage, nh - c0);
            if (tile_ok) {
                for (int j0 = 0; j0 < m; j0 += 32) {
                    const int j = j0 + lane;
                    int32_t k = 0;
                    bool cov = false;
                    if (j < m) {
                        const int4 r = hq_rect[j];
                        k = hq_k[j];
                        cov = hq_b[j] == b && r.x <= tx && tx <= r.z && r.y <= ty && ty <= r.w;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, cov);
                    if (cov) w.pair_tmp[at + __popc(bal & ((1u << lane) - 1u))] = k | kBlockHead;
                    at += __popc(bal);
                    n_app += __popc(bal);
                }
            }
        }
        __syncwarp();
    }
    if (!tile_ok) return;
    const int64_t start = w.tile_off[t];
    const int n = (int)(w.tile_off[t + 1] - start);
    if (n <= 1) {
        if (n == 1 && lane == 0) w.pair_k[start] = w.pair_tmp[start] & kIdMask;
        return;
    }
    if (n <= 32) {
        warp_sort_list<1>(w, start, n, lane);
    } else if (n <= 64) {
        warp_sort_list<2>(w, start, n, lane);
    } else if (n <= 128) {
        warp_sort_list<4>(w, start, n, lane);
    } else if (n <= 256) {
        if (n_app > 0 || !warp_merge_runs<8>(w, start, n, lane, runs[threadIdx.x >> 5]))
            warp_sort_list<8>(w, start, n, lane);
    } else if (n <= 512) {
        if (n_app > 0 || !warp_merge_runs<16>(w, start, n, lane, runs[threadIdx.x >> 5]))
            warp_sort_list<16>(w, start, n, lane);
    } else if (lane == 0) {
        // the top bit marks a list that carries appended queued kernels
        w.long_q[atomicAdd(w.n_long, 1)] = (int32_t)t | (n_app > 0 ? kBlockHead : 0);
    }
}

// One CTA per queued long list (grid-stride over the queue).
__global__ void __launch_bounds__(kSortThreads) k_segsort_long(const __grid_constant__ Geo g,
                                                               Bufs w) {
    if (status_bad(w.status)) return;
    __shared__ uint32_t s[kBitmapWords];
    constexpr int kWarps = kSortThreads / 32;
    __shared__ WarpRuns runs[kWarps];
    __shared__ bool merged[kWarps];
    const int n_long = *w.n_long;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's lists are q = blockIdx.x + j gridDim.x; kWarps at a time its
    // warps try the run merge (up to 1024 ids), then the CTA sorts the rest
    for (int q0 = blockIdx.x; q0 < n_long; q0 += gridDim.x * kWarps) {
        const int q = q0 + warp * gridDim.x;
        bool ok = false;
        if (q < n_long) {
            const int32_t e = w.long_q[q];
            const int64_t t = e & kIdMask;
            const int64_t start = w.tile_off[t];
            const int n = (int)(w.tile_off[t + 1] - start);
            ok = e >= 0 && n <= 1024 && warp_merge_runs<32>(w, start, n, lane, runs[warp]);
        }
        if (lane == 0) merged[warp] = ok;
        __syncthreads();
        for (int j = 0; j < kWarps; ++j) {
            const int qq = q0 + j * gridDim.x;
            if (qq >= n_long) break;
            if (!merged[j]) segsort_tile(g, w, w.long_q[qq] & kIdMask, s);
            __syncthreads();
        }
    }
}

__device__ void segsort_tile(const Geo &g, const Bufs &w, int64_t t, uint32_t *s) {
    const int64_t start = w.tile_off[t];
    const int n = (int)(w.tile_off[t + 1] - start);
    if (n <= 0) return;
    const int tid = threadIdx.x;
    if (n <= kSortMax) {
        int P = 1;
        while (P < n) P <<= 1;
        int *v = reinterpret_cast<int *>(s);
        for (int i = tid; i < P; i += kSortThreads)
            v[i] = i < n ? w.pair_tmp[start + i] & kIdMask : 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < P; i += kSortThreads) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const int a = v[i], b = v[ixj];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) { v[i] = b; v[ixj] = a; }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < n; i += kSortThreads) w.pair_k[start + i] = v[i];
        return;
    }
    // Long list: sweep the owning image's kernel-id range with a bitmap.
    const ImgDev &im = img_of(g, img_by_tile(g, t));
    const int64_t win = (int64_t)kBitmapWords * 32;
    int64_t out = start;
    for (int64_t w0 = im.k_off; w0 < im.k_off + im.K; w0 += win) {
        for (int i = tid; i < kBitmapWords; i += kSortThreads) s[i] = 0u;
        __syncthreads();
        for (int i = tid; i < n; i += kSortThreads) {
            const int64_t d = (int64_t)(w.pair_tmp[start + i] & kIdMask) - w0;
            if (d >= 0 && d < win) atomicOr(&s[d >> 5], 1u << (d & 31));
        }
        __syncthreads();
        constexpr int per = kBitmapWords / kSortThreads;
        int cnt = 0;
        for (int q = 0; q < per; ++q) cnt += __popc(s[tid * per + q]);
        int total;
        int64_t pos = out + block_exscan_int(cnt, &total);
        for (int q = 0; q < per; ++q) {
            uint32_t word = s[tid * per + q];
            while (word) {
                const int bit = __ffs(word) - 1;
                word &= word - 1;
                w.pair_k[pos++] = (int32_t)(w0 + (int64_t)(tid * per + q) * 32 + bit);
            }
        }
        out += total;
        __syncthreads();
    }
}

}  // namespace

// Deterministic fit: the kernel-major index of the pairs' list positions
// (see Bufs::pidx).  One warp per tile, lanes over its list.
__global__ void __launch_bounds__(kShortSortThreads) k_pair_index(const __grid_constant__ Geo g,
                                                                  Bufs w) {
    if (status_bad(w.status)) return;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= g.tiles_total) return;
    const ImgDev &im = img_of(g, img_by_tile(g, t));
    const int64_t local = t - im.t_off;
    const int tx = (int)(local % im.tiles_x), ty = (int)(local / im.tiles_x);
    const int32_t p0 = w.tile_off[t], p1 = w.tile_off[t + 1];
    for (int32_t p = p0 + (int32_t)(threadIdx.x & 31); p < p1; p += 32) {
        const int32_t k = w.pair_k[p];
        w.pidx[part_slot(w, k, w.rect[k], tx, ty)] = p;
    }
}

cudaError_t launch_bin(const Geo &g, const Bufs &w, cudaStream_t st) {
    const int64_t n = g.tiles_total;
    cudaError_t e = cudaMemsetAsync(w.tile_cnt, 0, sizeof(int32_t) * n, st);
    if (e == cudaSuccess && w.huge) e = cudaMemsetAsync(w.n_huge, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (g.K_total > 0) {
        const unsigned gb = (unsigned)((g.K_total + kBinThreads - 1) / kBinThreads);
        k_prep_bbox<<<gb, kBinThreads, 0, st>>>(g, w);
        if (w.huge && n > 0)
            k_huge_cover<<<(unsigned)((n + kHugeThreads - 1) / kHugeThreads), kHugeThreads, 0, st>>>(
                g, w);
    }
    const int nb = (int)((n + kScanChunk - 1) / kScanChunk);
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(n, w.tile_cnt, w.bsum, w.status);
    k_scan_top<<<1, kScanThreads, 0, st>>>(nb, w.bsum, n, w.tile_off, w.n_pairs, w.n_long,
                                           w.pair_cap, w.status);
    k_scan_down<<<nb, kScanThreads, 0, st>>>(n, w.tile_cnt, w.bsum, w.tile_off, w.cursor,
                                             w.pair_cap, w.status);
    if (g.K_total > 0) {
        const unsigned gb = (unsigned)((g.K_total + kBinThreads - 1) / kBinThreads);
        k_scatter<<<gb, kBinThreads, 0, st>>>(g, w);
    }
    if (w.kcnt && g.K_total > 0) {
        // deterministic fit: each kernel's first index entry (the same total
        // as the tiles'; the offsets are written twice over, as offsets and
        // cursors)
        e = launch_exscan(g.K_total, w.kcnt, w.kbsum, w.koff, w.ktot, w.kn_long, w.koff,
                          w.pair_cap, w.status, st);
        if (e != cudaSuccess) return e;
    }
    e = launch_sort_lists(g, w, st);
    if (e == cudaSuccess && w.kcnt && n > 0) {
        constexpr int wpb = kShortSortThreads / 32;
        k_pair_index<<<(unsigned)((n + wpb - 1) / wpb), kShortSortThreads, 0, st>>>(g, w);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_sort_lists(const Geo &g, const Bufs &w, cudaStream_t st) {
    const int64_t n = g.tiles_total;
    if (n > 0) {
        constexpr int wpb = kSegThreads / 32;
        k_segsort_warp<<<(unsigned)((n + wpb - 1) / wpb), kSegThreads, 0, st>>>(g, n, w);
        const int64_t gl = n < kLongGrid ? n : kLongGrid;
        k_segsort_long<<<(unsigned)gl, kSortThreads, 0, st>>>(g, w);
    }
    return cudaGetLastError();
}


cudaError_t launch_exscan(int64_t n, const int32_t *cnt, long long *bsum, int32_t *off,
                          int64_t *total, int32_t *n_long, int32_t *cursor, int64_t cap,
                          int32_t *status, cudaStream_t st) {
    const int nb = (int)((n + kScanChunk - 1) / kScanChunk);
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(n, cnt, bsum, status);
    k_scan_top<<<1, kScanThreads, 0, st>>>(nb, bsum, n, off, total, n_long, cap, status);
    k_scan_down<<<nb, kScanThreads, 0, st>>>(n, cnt, bsum, off, cursor, cap, status);
    return cudaGetLastError();
}

}  // namespace smoe
