// Resampling and kernel editing (Sec. II-B, Sec. VII-C):
//   - smoe_sharpen: native sharpening, L' = f L (bandwidths divided by f);
//   - smoe_render_points: the continuous regression function y(x) (Eq. 5)
//     at arbitrary sample points, i.e. super-resolution on a regular or an
//     irregular raster.
//
// Points: each in-image point gets the tile of the model raster it lies in;
// a counting sort by tile (count, the binning's prefix sum, scatter) puts
// the points of one tile next to each other, and one thread per point then
// walks its tile's kernel list.  Neighbouring threads of a warp mostly share
// a tile, so their reads of a kernel's prepared record are the same address
// (one transaction for the warp) and the records stay in L2; such a warp
// first culls the list against its points' rows (k_render_points).
#include <cmath>

#include "smoe_internal.cuh"

namespace smoe {

namespace {

constexpr int kPtThreads = 256;

__global__ void k_scale(const float *__restrict__ in, float *__restrict__ out, int64_t n,
                        float f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __fmul_rn(in[i], f);
}

// Tile of each point (-1 outside [0,W) x [0,H) or non-finite; such a point's
// outputs are written as 0 here) and the per-tile counts.
__global__ void k_pt_tile(int64_t n, const float2 *__restrict__ xy, int W, int H, int T,
                          int tiles_x, int C, int32_t *__restrict__ pt_tile,
                          int32_t *__restrict__ cnt, float *__restrict__ y,
                          float *__restrict__ inv_d, const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = i < n;
    const float2 p = live ? xy[i] : make_float2(-1.0f, -1.0f);
    int32_t t = -1;
    if (p.x >= 0.0f && p.x < (float)W && p.y >= 0.0f && p.y < (float)H) {
        // floor of a float in [0, W): exact integer conversion
        const int tx = min((int)p.x / T, tiles_x - 1);
        const int ty = (int)p.y / T;
        t = ty * tiles_x + tx;
    } else if (live) {
        for (int ch = 0; ch < C; ++ch) y[ch * n + i] = 0.0f;
        if (inv_d) inv_d[i] = 0.0f;
    }
    // neighbouring points mostly share a tile: one atomic per tile per warp
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    if (t >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[t], __popc(peers));
    if (live) pt_tile[i] = t;
}

__global__ void k_pt_scatter(int64_t n, const int32_t *__restrict__ pt_tile,
                             int32_t *__restrict__ cursor,
                             int32_t *__restrict__ order, const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t t = i < n ? pt_tile[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    if (t < 0) return;
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[t], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    order[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;   // cursor starts at off[t]
}

// One kernel's contribution to a point (p): the predicate's own FP32
// operations, then pi exp(-q/2) and the expert values.
template <int C, bool LIN>
__device__ __forceinline__ void point_pair(const float *r, float2 p, float qmax, float &D,
                                           float (&N)[C]) {
    constexpr int E = LIN ? 3 : 1;
    const float4 r0 = __ldg(reinterpret_cast<const float4 *>(r));
    const float c = __ldg(r + 4), lp = __ldg(r + 5);
    const float dy = __fsub_rn(p.y, r0.y);
    const float z1 = __fmul_rn(c, dy);
    const float u = __fmul_rn(z1, z1);
    if (!(u <= qmax)) return;                // q = fma(z0, z0, u) >= u: not included
    const float dx = __fsub_rn(p.x, r0.x);
    const float tb = __fmul_rn(r0.w, dy);
    float z0;
    const float qv = q_of(r0.z, dx, tb, u, z0);
    if (!(qv <= qmax)) return;
    const float ev = ex2(__fmaf_rn(qv, kNegHalfLog2e, lp));       // pi exp(-q/2)
    D += ev;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        float m = __ldg(r + 7 + ch * E);
        if (LIN) m = __fmaf_rn(__ldg(r + 7 + ch * E + 1), dx,
                               __fmaf_rn(__ldg(r + 7 + ch * E + 2), dy, m));
        N[ch] = __fmaf_rn(ev, m, N[ch]);
    }
}

// One thread per sorted in-image point: D = sum e_k, N_c = sum e_k m_kc over
// the tile's list in ascending kernel order, y_c = N_c / D (0 where D = 0).
// A warp whose points share one tile first culls the list 32 kernels at a
// time against its points' rows: a kernel passes when some point of the
// warp has u = (c dy)^2 <= q_max, computed with the predicate's own
// operations at the warp's lowest and highest point (u is monotone in the
// point's y on each side of the centre; a centre between them passes).  A
// culled kernel includes none of the warp's points, so the sums, taken over
// the passing kernels in list order, are the per-point walk's bit for bit.
template <int C, bool LIN>
__global__ void __launch_bounds__(kPtThreads) k_render_points(
    int64_t n, const int64_t *__restrict__ n_in, const float2 *__restrict__ xy,
    const int32_t *__restrict__ order, const int32_t *__restrict__ pt_tile,
    const int32_t *__restrict__ tile_off, const int32_t *__restrict__ pair_k,
    const float *__restrict__ rec, int S, float qmax, int rbf, float *__restrict__ y,
    float *__restrict__ inv_d, const int32_t *status) {
    const unsigned full = 0xffffffffu;
    if (status_bad(status)) return;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nin = *n_in;
    if (j - (threadIdx.x & 31) >= nin) return;          // the whole warp is past the end
    const bool active = j < nin;
    const int lane = threadIdx.x & 31;
    const int32_t i = active ? order[j] : 0;
    const int32_t t = active ? pt_tile[i] : -1;
    const float2 p = active ? xy[i] : make_float2(0.0f, 0.0f);
    float D = 0.0f, N[C];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) N[ch] = 0.0f;
    const int32_t t0 = __shfl_sync(full, t, 0);         // lane 0 is active
    if (__all_sync(full, !active || t == t0)) {
        float ylo = active ? p.y : INFINITY, yhi = active ? p.y : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ylo = fminf(ylo, __shfl_xor_sync(full, ylo, o));
            yhi = fmaxf(yhi, __shfl_xor_sync(full, yhi, o));
        }
        const int32_t s0 = tile_off[t0], e0 = tile_off[t0 + 1];
        for (int32_t q0 = s0; q0 < e0; q0 += 32) {
            const int32_t q = q0 + lane;
            int32_t kid = 0;
            bool pass = false;
            if (q < e0) {
                kid = pair_k[q];
                const float *r = rec + (int64_t)kid * S;
                const float my = __ldg(r + 1), c = __ldg(r + 4);
                const float zl = __fmul_rn(c, __fsub_rn(ylo, my));
                const float zh = __fmul_rn(c, __fsub_rn(yhi, my));
                pass = (my >= ylo && my <= yhi) || __fmul_rn(zl, zl) <= qmax ||
                       __fmul_rn(zh, zh) <= qmax;
            }
            unsigned bal = __ballot_sync(full, pass);
            while (bal) {
                const int l = __ffs(bal) - 1;
                bal &= bal - 1;
                const int32_t k = __shfl_sync(full, kid, l);
                if (active) point_pair<C, LIN>(rec + (int64_t)k * S, p, qmax, D, N);
            }
        }
    } else if (active) {
        const int32_t e = tile_off[t + 1];
        for (int32_t q = tile_off[t]; q < e; ++q)
            point_pair<C, LIN>(rec + (int64_t)pair_k[q] * S, p, qmax, D, N);
    }
    if (!active) return;
    const float inv = D > 0.0f ? 1.0f / D : 0.0f;
    const float sc = rbf ? 1.0f : inv;                // Eq. 1 does not normalise
#pragma unroll
    for (int ch = 0; ch < C; ++ch) y[ch * n + i] = N[ch] * sc;
    if (inv_d) inv_d[i] = inv;
}

template <int C, bool LIN>
void launch_points_kernel(unsigned grid, cudaStream_t st, int64_t n, const int64_t *n_in,
                          const float2 *xy, const int32_t *order, const int32_t *pt_tile,
                          const int32_t *tile_off, const int32_t *pair_k, const float *rec,
                          int S, float qmax, int rbf, float *y, float *inv_d,
                          const int32_t *status) {
    k_render_points<C, LIN><<<grid, kPtThreads, 0, st>>>(n, n_in, xy, order, pt_tile, tile_off,
                                                         pair_k, rec, S, qmax, rbf, y, inv_d,
                                                         status);
}

// In-range pairs: one CTA per tile, one thread per pixel of the tile; every
// pixel tests the tile's whole list with the exact predicate and the CTA adds
// its count of (pixel, kernel) pairs with q <= q_max to *out.
__global__ void __launch_bounds__(1024) k_count_inrange(const __grid_constant__ Geo g,
                                                        const float *__restrict__ rec,
                                                        const int32_t *__restrict__ tile_off,
                                                        const int32_t *__restrict__ pair_k,
                                                        unsigned long long *out,
                                                        const int32_t *status) {
    if (status_bad(status)) return;
    const int64_t t = blockIdx.x;
    const int tiles_x = g.one.tiles_x;
    const int x0 = (int)(t % tiles_x) * g.T, y0 = (int)(t / tiles_x) * g.T;
    const int xi = x0 + (int)threadIdx.x % g.T, yi = y0 + (int)threadIdx.x / g.T;
    unsigned long long n = 0;
    if (xi < g.one.W && yi < g.one.H) {
        const float px = (float)xi + 0.5f, py = (float)yi + 0.5f;
        for (int32_t q = tile_off[t]; q < tile_off[t + 1]; ++q) {
            const float *r = rec + (int64_t)pair_k[q] * g.S;
            const float4 r0 = __ldg(reinterpret_cast<const float4 *>(r));
            const float c = __ldg(r + 4);
            const float dx = __fsub_rn(px, r0.x), dy = __fsub_rn(py, r0.y);
            const float z1 = __fmul_rn(c, dy);
            float z0;
            const float qv = q_of(r0.z, dx, __fmul_rn(r0.w, dy), __fmul_rn(z1, z1), z0);
            n += qv <= g.qmax ? 1ull : 0ull;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

}  // namespace

cudaError_t launch_count_inrange(const Geo &g, const float *rec, const int32_t *tile_off,
                                 const int32_t *pair_k, unsigned long long *out,
                                 const int32_t *status, cudaStream_t st) {
    if (g.tiles_total == 0) return cudaSuccess;
    k_count_inrange<<<(unsigned)g.tiles_total, g.T * g.T, 0, st>>>(g, rec, tile_off, pair_k, out,
                                                                 status);
    return cudaGetLastError();
}

cudaError_t launch_scale(const float *in, float *out, int64_t n, float f, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_scale<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(in, out, n, f);
    return cudaGetLastError();
}

cudaError_t launch_render_points(const Geo &g, const float *rec, const int32_t *tile_off,
                                 const int32_t *pair_k, int64_t n, const float *xy,
                                 const PointBufs &pb, float *y, float *inv_d,
                                 const int32_t *status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t tiles = g.tiles_total;
    cudaError_t e = cudaMemsetAsync(pb.cnt, 0, sizeof(int32_t) * tiles, st);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((n + kPtThreads - 1) / kPtThreads);
    const float2 *p2 = reinterpret_cast<const float2 *>(xy);
    k_pt_tile<<<grid, kPtThreads, 0, st>>>(n, p2, g.one.W, g.one.H, g.T, g.one.tiles_x, g.C,
                                           pb.pt_tile, pb.cnt, y, inv_d, status);
    // the points counted never exceed n: no capacity error is possible
    e = launch_exscan(tiles, pb.cnt, pb.bsum, pb.off, pb.n_in, pb.n_long, pb.cursor, n,
                      const_cast<int32_t *>(status), st);
    if (e != cudaSuccess) return e;
    k_pt_scatter<<<grid, kPtThreads, 0, st>>>(n, pb.pt_tile, pb.cursor, pb.order, status);
    const int S = g.S;
    if (g.C == 1 && !g.linear)
        launch_points_kernel<1, false>(grid, st, n, pb.n_in, p2, pb.order, pb.pt_tile, tile_off,
                                       pair_k, rec, S, g.qmax, g.rbf, y, inv_d, status);
    else if (g.C == 1)
        launch_points_kernel<1, true>(grid, st, n, pb.n_in, p2, pb.order, pb.pt_tile, tile_off,
                                      pair_k, rec, S, g.qmax, g.rbf, y, inv_d, status);
    else if (!g.linear)
        launch_points_kernel<3, false>(grid, st, n, pb.n_in, p2, pb.order, pb.pt_tile, tile_off,
                                       pair_k, rec, S, g.qmax, g.rbf, y, inv_d, status);
    else
        launch_points_kernel<3, true>(grid, st, n, pb.n_in, p2, pb.order, pb.pt_tile, tile_off,
                                      pair_k, rec, S, g.qmax, g.rbf, y, inv_d, status);
    return cudaGetLastError();
}

}  // namespace smoe
