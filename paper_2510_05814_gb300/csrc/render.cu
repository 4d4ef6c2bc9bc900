// Tile kernels of the rasterised SMoE regression: forward render (Eqs. 2-5),
// the backward of the gradient-descent fit through the rasteriser
// (Sec. III-D), and the fused forward + MSE + backward fit tile.
//
// One CTA (4 warps) per tile.  The tile's kernel list is processed in chunks
// of up to NCH kernels (256 for the render kernels; 512 for the fused fit
// tile at T = 16, whose backward re-stages every chunk but the last, so
// that the longer lists of a fit's later iterations are staged once); each
// chunk is staged in shared memory: the kernel's
// prepared record and a ROW MASK, bit r clear only where row r of the tile
// holds no included pixel.  The row test evaluates the predicate's own FP32
// value at the row's minimising column (see stage_chunk), so skipping the
// clear rows changes no result; a listed kernel whose ellipse misses the
// tile's pixels has an empty mask and costs only its staging.
//
// Forward (pixel-major): a warp owns a band of 64 pixels (2 adjacent pixels
// per lane, 64/T rows) and walks the chunk, skipping every kernel whose mask
// misses the band's rows (ballot compaction), four kernels in flight on two
// pairs of accumulators; D = sum e and N_c = sum e m_c stay in FP32
// registers.  Pixel pairs use packed f32x2 arithmetic (IEEE per lane, the
// same single rounding as the scalar predicate, so the inclusion decision is
// bit-identical).  T = 8 has one band: its warps split the chunk and meet in
// shared memory.
//
// Backward (row-synchronous, lane = kernel): the chunk's kernels are grouped
// 16 at a time by the centre of their row span; a warp walks the rows where
// its group has a live row two at a time, lanes 0-15 on the first and 16-31
// on the second, every lane evaluating its kernel on the row's pixel pairs
// against the pixel state read by broadcast from shared memory; a kernel's
// raw sums (below) stay in its two lanes' registers, are added once, and
// leave the SM as one float4 atomic per 4 sums per (tile, kernel).  With
// float atomics the last round's groups are shared by all warps
// row-interleaved, so no warp idles.  The chunks of a long list are walked
// last to first (the forward's last chunk is still staged).
//
// Raw per-kernel sums (e = pi exp(-q/2); s = g sum_c G_c (m_c - y_c), g = e / D,
// H_c = G_c / D, so s = e (sum_c H_c m_c - sum_c H_c y_c) and g G_c = e H_c;
// in the RBF mode of Eq. 1 (y = N, D = 1) the same holds with H_c = G_c and
// the y term dropped):
//   [0] A1 = sum s z0 dx  [1] B1 = sum s z0 dy  [2] C1 = sum s z1 dy
//   [3] A2 = sum s z0     [4] Z3 = sum s z1
//   [5+c] E_c = sum e H_c,   linear: [5+C+c] F_c = sum e H_c dx,
//                                    [5+2C+c] Fy_c = sum e H_c dy
//   [5+C*E] S0 = sum s
// and the gradients (chain rule of Eqs. 2-4):
//   dL/da = -A1, dL/db = -B1, dL/dc = -C1,
//   dL/dmx = a A2 - sum_c W_c0 E_c,  dL/dmy = b A2 + c Z3 - sum_c W_c1 E_c,
//   dL/dea_c = E_c, dL/dW_c0 = F_c, dL/dW_c1 = Fy_c, dL/dlogpi = S0.
#include "smoe_internal.cuh"

#include <type_traits>

namespace smoe {

namespace {

#ifndef SMOE_NW
#define SMOE_NW 4
#endif
constexpr int kNW = SMOE_NW;          // warps per CTA
constexpr int kThreads = kNW * 32;
// Resident CTAs per SM that the register budget targets, and the chunk of a
// tile's list staged in shared memory at once (tiles of 8 and 16 pixels).
#ifndef SMOE_MIN_BLOCKS
#define SMOE_MIN_BLOCKS 4
#endif
#ifndef SMOE_NCH
#define SMOE_NCH 256
#endif
#ifndef SMOE_FIT_NCH
#define SMOE_FIT_NCH 512
#endif
#ifndef SMOE_FWD_UNROLL
#define SMOE_FWD_UNROLL 4
#endif
// Backward: rows of the tile one warp step covers (a group of 32 / rows
// kernels, each on that many rows at once).
#ifndef SMOE_BWD_ROWS
#define SMOE_BWD_ROWS 2
#endif

constexpr int kMinBlocks = SMOE_MIN_BLOCKS;
constexpr int kBwdRows = SMOE_BWD_ROWS;
static_assert(kBwdRows == 1 || kBwdRows == 2 || kBwdRows == 4, "rows per backward step");
// The forward-only kernels (render, fused mean) need fewer registers than
// the backward: one more resident CTA per SM measured faster for them.
#ifndef SMOE_MIN_BLOCKS_FWD
#define SMOE_MIN_BLOCKS_FWD 5
#endif
constexpr int kMinBlocksFwd = SMOE_MIN_BLOCKS_FWD;

template <int C, bool LIN>
struct Rec {
    static constexpr int E = LIN ? 3 : 1;
    static constexpr int S = (7 + C * E + 3) & ~3;        // global record stride (floats)
    static constexpr int SS = (S % 8 == 0) ? S + 4 : S;   // shared stride: spreads banks
    static constexpr int PI = 5 + C * E;                  // sum slot of dL/dlogpi
    static constexpr int GS = (PI + 1 + 3) & ~3;          // accumulator stride (raw sums)
};

// Kernels per staged chunk of a tile's list: the render kernels' and the
// fused fit kernel's (whose backward re-stages every chunk but the last).
constexpr int default_nch(int T) { return T >= 32 ? 128 : SMOE_NCH; }
constexpr int fit_nch(int T) { return T == 16 ? SMOE_FIT_NCH : default_nch(T); }

template <int C, int T>
struct Geom {
    static constexpr int NPX = T * T;
    static constexpr int BANDS = NPX / 64;                // 64-pixel bands per tile
    static constexpr int BROWS = 64 / T;                  // rows per band
    static constexpr int LROW = T / 2;                    // lanes per row (2 px each)
    static constexpr int KSPLIT = BANDS >= kNW ? 1 : kNW / BANDS;
    static constexpr int BPW = BANDS >= kNW ? BANDS / kNW : 1;   // bands per warp
    static constexpr int PS = 2 * (C + 1);                // floats per pixel pair of state
    static constexpr int RS = (T / 2) * PS + 4;           // floats per row of state (padded)
};

// A staged chunk of NC kernels.  The forward's per-warp band lists index a
// sub-chunk of at most 256 of them in one byte (a longer chunk is walked in
// sub-chunks: two-byte indices in its inner loop measured 1.6 % slower); the
// backward groups the whole chunk (its index is read once per group).
template <int NC>
struct Chunk {
    static constexpr int NCH = NC;
    static constexpr int NSUB = NC < 256 ? NC : 256;
    using Ord = typename std::conditional<(NC > 256), uint16_t, uint8_t>::type;
};

template <int C, bool LIN, int T, int NC = default_nch(T)>
struct Smem {
    using R = Rec<C, LIN>;
    using G = Geom<C, T>;
    using K = Chunk<NC>;
    alignas(16) float rec[K::NCH * R::SS];
    alignas(16) float pst[T * G::RS];
    alignas(16) float red[(G::KSPLIT - 1) * (C + 1) * G::NPX + 1];
    uint32_t mask[K::NCH];
    int32_t kid[K::NCH];
    uint8_t flist[kNW][K::NSUB];         // per-warp compacted kernel list of a band
    typename K::Ord order[K::NCH];       // backward: kernels grouped by row-span centre
    int bcnt[2 * T], boff[2 * T];        // backward grouping buckets (2T - 1 keys)
    double lsum[kNW];
    long long next;                      // persistent launch: the CTA's next tile
};

template <int C, bool LIN, int T, int NC = default_nch(T)>
constexpr size_t smem_bytes() { return sizeof(Smem<C, LIN, T, NC>); }

struct TileInfo {
    int b, x0, y0, W, H;
    int64_t start;
    int n;
};

__device__ __forceinline__ TileInfo tile_info(const Geo &g, const Bufs &w, int64_t t) {
    TileInfo ti;
    ti.b = img_by_tile(g, t);
    const ImgDev &im = img_of(g, ti.b);
    const int64_t local = t - im.t_off;
    ti.x0 = (int)(local % im.tiles_x) * g.T;
    ti.y0 = (int)(local / im.tiles_x) * g.T;
    ti.W = im.W;
    ti.H = im.H;
    ti.start = w.tile_off[t];
    ti.n = (int)(w.tile_off[t + 1] - ti.start);
    return ti;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Stage kernels [c0, c0 + nc) of the tile's list: records and row masks.
template <int C, bool LIN, int T, int NC>
__device__ __forceinline__ void stage_chunk(const Geo &g, const Bufs &w, const TileInfo &ti,
                                            int c0, int nc, Smem<C, LIN, T, NC> &sm) {
    using R = Rec<C, LIN>;
    constexpr int Q = R::S / 4;                // float4 per record
    for (int i = threadIdx.x; i < nc * Q; i += kThreads) {
        const int j = i / Q, q = i - j * Q;
        const int kid = w.pair_k[ti.start + c0 + j];
        const float4 v = __ldg(reinterpret_cast<const float4 *>(w.rec + (int64_t)kid * R::S) + q);
        *reinterpret_cast<float4 *>(sm.rec + j * R::SS + 4 * q) = v;
        if (q == 0) sm.kid[j] = kid;
    }
    __syncthreads();
    // Row masks: bit r is clear only if no pixel of row r inside the tile
    // passes the predicate, evaluated with the render's own FP32 operations
    // q32 = fma(z0, z0, u), z0 = fma(a, x - mx, b dy), u = (c dy)^2.  Along
    // a row z0 is monotone in the column (each operation rounds
    // monotonically) and q32 is monotone in |z0|, so where z0 has one sign at
    // the tile's first and last column the row's least q32 is fma(zm, zm, u),
    // zm = min |z0| of those two columns, exactly.  Where the sign changes
    // inside the tile the row keeps the test u <= q_max (q32 >= u): a
    // superset, nearly always live anyway.  T / 8 adjacent lanes share a
    // kernel, each taking 8 of its rows; every lane of a warp runs every round.
    {
        constexpr int LPK = T / 8;                         // lanes per kernel
        const int lane = threadIdx.x & 31;
        const float y0f = (float)ti.y0 + 0.5f;
        const float xl = (float)ti.x0 + 0.5f;              // first and last column centres
        const float xr = (float)ti.x0 + ((float)T - 0.5f);
        // least q32 of a row over the columns between two of them (exact
        // where z0 keeps one sign there, else the u test)
        auto row_min = [](float zl, float zr, float u) {
            const float zm = fminf(fabsf(zl), fabsf(zr));
            const bool one_sign = (zl >= 0.0f) == (zr >= 0.0f);
            return one_sign ? __fmaf_rn(zm, zm, u) : u;
        };
        for (int base = threadIdx.x & ~31; base < LPK * nc; base += kThreads) {
            const int i = base + lane;
            const int j = i < LPK * nc ? i / LPK : 0;
            const int r0 = (i % LPK) * 8;
            const float *rj = sm.rec + j * R::SS;
            const float mx = rj[0], my = rj[1], a = rj[2], b = rj[3], c = rj[4];
            const float dxl = __fsub_rn(xl, mx), dxr = __fsub_rn(xr, mx);
            uint32_t m = 0;
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const float dy = __fsub_rn(__fadd_rn(y0f, (float)(r0 + rr)), my);
                const float t = __fmul_rn(b, dy);
                const float z1 = __fmul_rn(c, dy);
                const float u = __fmul_rn(z1, z1);
                const float zl = __fmaf_rn(a, dxl, t), zr = __fmaf_rn(a, dxr, t);
                m |= (row_min(zl, zr, u) <= g.qmax ? 1u : 0u) << rr;
            }
            m <<= r0;
#pragma unroll
            for (int o = 1; o < LPK; o <<= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
            if (i % LPK == 0 && i < LPK * nc) sm.mask[j] = m;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- forward

// Pixel (row, col) of the lane's pair for band slot bi, and whether this warp
// finalises it (T = 8: only warp 0 after the reduction).
template <int C, int T>
__device__ __forceinline__ bool lane_pixels(int bi, int &row, int &col) {
    using G = Geom<C, T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int band = G::KSPLIT > 1 ? 0 : warp + bi * kNW;
    row = band * G::BROWS + lane / G::LROW;
    col = 2 * (lane % G::LROW);
    return G::KSPLIT == 1 || warp == 0;
}

// One kernel's contribution to a lane's two pixels (row y0, columns x2).
template <int C, bool LIN>
__device__ __forceinline__ void fwd_pair(const float *r, float y0, float2 x2, float qmax,
                                         float2 &D, float2 (&N)[C]) {
    using R = Rec<C, LIN>;
    const float4 r0 = *reinterpret_cast<const float4 *>(r);
    const float4 r1 = *reinterpret_cast<const float4 *>(r + 4);
    float ex[R::SS - 8 > 0 ? R::SS - 8 : 1];
    if (R::S > 8) {
#pragma unroll
        for (int q = 0; q < (R::S - 8) / 4; ++q) {
            const float4 v = *reinterpret_cast<const float4 *>(r + 8 + 4 * q);
            ex[4 * q] = v.x; ex[4 * q + 1] = v.y; ex[4 * q + 2] = v.z; ex[4 * q + 3] = v.w;
        }
    }
    // record: [0..4] mx my a b c, [5..6] spare, [7 + ch*E + k] experts
    auto rv = [&](int i) -> float {
        return i < 4 ? (i == 0 ? r0.x : i == 1 ? r0.y : i == 2 ? r0.z : r0.w)
             : i < 8 ? (i == 4 ? r1.x : i == 5 ? r1.y : i == 6 ? r1.z : r1.w)
                     : ex[i - 8];
    };
    const float mx = r0.x, my = r0.y, a = r0.z, b = r0.w, c = r1.x;
    const float dy = __fsub_rn(y0, my);
    const float t = __fmul_rn(b, dy);
    const float z1 = __fmul_rn(c, dy);
    const float u = __fmul_rn(z1, z1);
    const float2 dx = __fadd2_rn(x2, f2(-mx));
    const float2 z0 = __ffma2_rn(f2(a), dx, f2(t));
    const float2 q = __ffma2_rn(z0, z0, f2(u));
    // log2 of pi exp(-q/2): one FMA (pi = 1 stores 0, giving the plain product)
    const float2 arg = __ffma2_rn(q, f2(kNegHalfLog2e), f2(r1.y));
    float2 e = make_float2(ex2(arg.x), ex2(arg.y));
    e.x = q.x <= qmax ? e.x : 0.0f;
    e.y = q.y <= qmax ? e.y : 0.0f;
    D = __fadd2_rn(D, e);
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        const float ea = rv(7 + ch * R::E);
        float2 m;
        if (LIN) {
            const float mb = fmaf(rv(7 + ch * R::E + 2), dy, ea);
            m = __ffma2_rn(f2(rv(7 + ch * R::E + 1)), dx, f2(mb));
        } else {
            m = f2(ea);
        }
        N[ch] = __ffma2_rn(e, m, N[ch]);
    }
}

// Accumulate D and N_c of one lane's two pixels (row `row`, columns col,
// col+1 of the tile) over the staged kernels s0 + j, j = j0, j0 + step, ...
// < nc (a sub-chunk of at most 256) whose mask meets `band_mask`: the warp
// first compacts those kernels (ballot), then evaluates them four at a time
// on two pairs of accumulators.
template <int C, bool LIN, int T, int NC>
__device__ __forceinline__ void fwd_band(const Geo &g, const TileInfo &ti,
                                         Smem<C, LIN, T, NC> &sm, int s0, int nc, int j0, int step,
                                         uint32_t band_mask, int row, int col, float2 &D,
                                         float2 (&N)[C]) {
    using R = Rec<C, LIN>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *lst = sm.flist[warp];
    int cnt = 0;
    for (int base = 0; base < nc; base += 32) {
        const int j = base + lane;
        const bool hit = j < nc && (j - j0) % step == 0 && j >= j0 && (sm.mask[s0 + j] & band_mask);
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) lst[cnt + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)j;
        cnt += __popc(bal);
    }
    __syncwarp();
    const float *rec = sm.rec + s0 * R::SS;
    const float qmax = g.qmax;
    const float y0 = (float)(ti.y0 + row) + 0.5f;
    const float2 x2 = make_float2((float)(ti.x0 + col) + 0.5f, (float)(ti.x0 + col) + 1.5f);
    float2 D2 = f2(0.0f), N2[C];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) N2[ch] = f2(0.0f);
    int i = 0;
#if SMOE_FWD_UNROLL >= 4
    // four kernels in flight: two pairs of accumulators, each pair fed twice
    for (; i + 3 < cnt; i += 4) {
        fwd_pair<C, LIN>(rec + lst[i] * R::SS, y0, x2, qmax, D, N);
        fwd_pair<C, LIN>(rec + lst[i + 1] * R::SS, y0, x2, qmax, D2, N2);
        fwd_pair<C, LIN>(rec + lst[i + 2] * R::SS, y0, x2, qmax, D, N);
        fwd_pair<C, LIN>(rec + lst[i + 3] * R::SS, y0, x2, qmax, D2, N2);
    }
#endif
    for (; i + 1 < cnt; i += 2) {
        fwd_pair<C, LIN>(rec + lst[i] * R::SS, y0, x2, qmax, D, N);
        fwd_pair<C, LIN>(rec + lst[i + 1] * R::SS, y0, x2, qmax, D2, N2);
    }
    if (i < cnt) fwd_pair<C, LIN>(rec + lst[i] * R::SS, y0, x2, qmax, D, N);
    D = __fadd2_rn(D, D2);
#pragma unroll
    for (int ch = 0; ch < C; ++ch) N[ch] = __fadd2_rn(N[ch], N2[ch]);
    __syncwarp();
}

// Forward over the whole list.  On return, for every band b the warp owns
// (bands w, w + 4, ...; T = 8: band 0 summed over the warps), lane l holds
// D and N_c of pixels (row, col), (row, col + 1) in Dv[bi], Nv[bi].
template <int C, bool LIN, int T, int NC>
__device__ __forceinline__ void fwd_tile(const Geo &g, const Bufs &w, const TileInfo &ti,
                                         Smem<C, LIN, T, NC> &sm, float2 (&Dv)[Geom<C, T>::BPW],
                                         float2 (&Nv)[Geom<C, T>::BPW][C]) {
    using G = Geom<C, T>;
    using K = Chunk<NC>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int split = warp % G::KSPLIT;
#pragma unroll
    for (int bi = 0; bi < G::BPW; ++bi) {
        Dv[bi] = f2(0.0f);
#pragma unroll
        for (int ch = 0; ch < C; ++ch) Nv[bi][ch] = f2(0.0f);
    }
    for (int c0 = 0; c0 < ti.n; c0 += K::NCH) {
        const int nc = min(K::NCH, ti.n - c0);
        if (c0 > 0) __syncthreads();              // previous chunk fully consumed
        stage_chunk<C, LIN, T>(g, w, ti, c0, nc, sm);
#pragma unroll
        for (int bi = 0; bi < G::BPW; ++bi) {
            const int band = G::KSPLIT > 1 ? 0 : warp + bi * kNW;
            int row, col;
            lane_pixels<C, T>(bi, row, col);
            const uint32_t bm = (G::BROWS >= 32 ? 0xffffffffu : ((1u << G::BROWS) - 1u))
                                << (band * G::BROWS);
            for (int s0 = 0; s0 < nc; s0 += K::NSUB)
                fwd_band<C, LIN, T>(g, ti, sm, s0, min(K::NSUB, nc - s0), split, G::KSPLIT, bm, row,
                                    col, Dv[bi], Nv[bi]);
        }
    }
    if (G::KSPLIT > 1) {
        // T = 8: warps 1..3 hand their partial sums to warp 0.
        const int p = 2 * lane;                   // pixel index of the lane's pair (band 0)
        if (split > 0) {
            float *dst = sm.red + (split - 1) * (C + 1) * G::NPX;
            dst[p] = Dv[0].x;
            dst[p + 1] = Dv[0].y;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                dst[(1 + ch) * G::NPX + p] = Nv[0][ch].x;
                dst[(1 + ch) * G::NPX + p + 1] = Nv[0][ch].y;
            }
        }
        __syncthreads();
        if (split == 0) {
#pragma unroll
            for (int k = 0; k < G::KSPLIT - 1; ++k) {
                const float *src = sm.red + k * (C + 1) * G::NPX;
                Dv[0].x += src[p];
                Dv[0].y += src[p + 1];
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    Nv[0][ch].x += src[(1 + ch) * G::NPX + p];
                    Nv[0][ch].y += src[(1 + ch) * G::NPX + p + 1];
                }
            }
        }
    }
}

template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads, kMinBlocksFwd) k_render(const __grid_constant__ Geo g, Bufs w,
                                                        float *__restrict__ y,
                                                        float *__restrict__ inv_d) {
    using G = Geom<C, T>;
    if (status_bad(w.status)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C, LIN, T> &sm = *reinterpret_cast<Smem<C, LIN, T> *>(smem_raw);
    const TileInfo ti = tile_info(g, w, blockIdx.x);
    float2 Dv[G::BPW], Nv[G::BPW][C];
    fwd_tile<C, LIN, T>(g, w, ti, sm, Dv, Nv);
    const int64_t HW = (int64_t)ti.W * ti.H;
#pragma unroll
    for (int bi = 0; bi < G::BPW; ++bi) {
        int row, col;
        if (!lane_pixels<C, T>(bi, row, col)) continue;
        const int yi = ti.y0 + row;
        if (yi >= ti.H) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xi = ti.x0 + col + h;
            if (xi >= ti.W) continue;
            const float D = h ? Dv[bi].y : Dv[bi].x;
            const float inv = D > 0.0f ? 1.0f / D : 0.0f;
            const float sc = g.rbf ? 1.0f : inv;          // Eq. 1 does not normalise
            const int64_t o = (int64_t)yi * ti.W + xi;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) y[ch * HW + o] = (h ? Nv[bi][ch].y : Nv[bi][ch].x) * sc;
            if (inv_d) inv_d[o] = inv;
        }
    }
}

// Multi-model fusion (Sec. V-C, Eq. 11): the B models of a batch whose
// images share one size are rendered tile by tile and averaged per pixel,
// y = (sum_h y_h) / B, with y_h = N_h / D_h (0 where D_h = 0) exactly as
// k_render computes it.  The models are visited in index order, so the sum
// is deterministic, and B = 1 gives k_render's output bit for bit.  The grid
// covers the tiles of one image; image b's tiles follow image b-1's.
template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads, kMinBlocksFwd) k_render_mean(const __grid_constant__ Geo g, Bufs w,
                                                             float *__restrict__ y) {
    using G = Geom<C, T>;
    if (status_bad(w.status)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C, LIN, T> &sm = *reinterpret_cast<Smem<C, LIN, T> *>(smem_raw);
    const int64_t tiles_img = g.tiles_total / g.B;
    float2 Sv[G::BPW][C];
#pragma unroll
    for (int bi = 0; bi < G::BPW; ++bi)
#pragma unroll
        for (int ch = 0; ch < C; ++ch) Sv[bi][ch] = f2(0.0f);
    TileInfo ti{};
    for (int b = 0; b < g.B; ++b) {
        if (b > 0) __syncthreads();               // the previous model's chunk is consumed
        ti = tile_info(g, w, (int64_t)b * tiles_img + blockIdx.x);
        float2 Dv[G::BPW], Nv[G::BPW][C];
        fwd_tile<C, LIN, T>(g, w, ti, sm, Dv, Nv);
#pragma unroll
        for (int bi = 0; bi < G::BPW; ++bi) {
            const float ia = g.rbf ? 1.0f : (Dv[bi].x > 0.0f ? 1.0f / Dv[bi].x : 0.0f);
            const float ib = g.rbf ? 1.0f : (Dv[bi].y > 0.0f ? 1.0f / Dv[bi].y : 0.0f);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                Sv[bi][ch].x = __fadd_rn(Sv[bi][ch].x, __fmul_rn(Nv[bi][ch].x, ia));
                Sv[bi][ch].y = __fadd_rn(Sv[bi][ch].y, __fmul_rn(Nv[bi][ch].y, ib));
            }
        }
    }
    const float nb = (float)g.B;
    const int64_t HW = (int64_t)ti.W * ti.H;
#pragma unroll
    for (int bi = 0; bi < G::BPW; ++bi) {
        int row, col;
        if (!lane_pixels<C, T>(bi, row, col)) continue;
        const int yi = ti.y0 + row;
        if (yi >= ti.H) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xi = ti.x0 + col + h;
            if (xi >= ti.W) continue;
            const int64_t o = (int64_t)yi * ti.W + xi;
#pragma unroll
            for (int ch = 0; ch < C; ++ch)
                y[ch * HW + o] = __fdiv_rn(h ? Sv[bi][ch].y : Sv[bi][ch].x, nb);
        }
    }
}

// ---------------------------------------------------------------- backward

// Write the state of pixels (row, col), (row, col+1): H_c = G_c / D and
// -Hy = -sum_c H_c y_c, as pairs {H_0a, H_0b, ..., -Hy_a, -Hy_b}.  Pixels
// outside the image get zeros.
template <int C, int T>
__device__ __forceinline__ void put_state(float *pst, int row, int col, const float (&H)[2][C],
                                          const float (&nHy)[2]) {
    using G = Geom<C, T>;
    float *dst = pst + row * G::RS + (col / 2) * G::PS;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        dst[2 * ch] = H[0][ch];
        dst[2 * ch + 1] = H[1][ch];
    }
    dst[2 * C] = nHy[0];
    dst[2 * C + 1] = nHy[1];
}

// Running per-kernel sums of one lane (registers).
template <int C, bool LIN>
struct BwdAcc {
    float v[Rec<C, LIN>::GS];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < Rec<C, LIN>::GS; ++q) v[q] = 0.0f;
    }
};

// Backward over the tile's list; the pixel state is in sm.pst.  `staged`:
// the forward's last chunk is still in shared memory.  The chunk's kernels
// with a live row are grouped by the centre of their row span, 16 to a
// warp; a lane owns one kernel and every second row of the group's rows
// (see `group` below): every read of pixel state is a broadcast, lanes
// whose kernel misses the row contribute zero, and each kernel's sums stay
// in its two lanes' registers until one float4 atomic per 4 sums at the end.
template <int C, bool LIN, int T, int NC>
__device__ __forceinline__ void bwd_tile(const Geo &g, const Bufs &w, const TileInfo &ti,
                                         Smem<C, LIN, T, NC> &sm, bool staged) {
    using R = Rec<C, LIN>;
    using G = Geom<C, T>;
    using K = Chunk<NC>;
    const float qmax = g.qmax;
    const float2 k2 = f2(kNegHalfLog2e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float x0f = (float)ti.x0, y0f = (float)ti.y0 + 0.5f;   // exact: integers < 2^24
    // The chunks last to first: the forward leaves its last chunk staged, so
    // a list longer than one chunk is staged once less (each kernel's sums
    // come from the one chunk that holds it, so the order changes none).
    const int last = ti.n > 0 ? (ti.n - 1) / K::NCH * K::NCH : 0;
    for (int c0 = last; c0 >= 0; c0 -= K::NCH) {
        const int nc = min(K::NCH, ti.n - c0);
        __syncthreads();                          // previous users of the chunk are done
        if (!(staged && c0 == last)) stage_chunk<C, LIN, T>(g, w, ti, c0, nc, sm);
        // Group the kernels by the centre of their row span, first + last row
        // (counting sort over 2T - 1 keys), so that a warp's 32 kernels cover
        // similar rows; kernels that miss every row are dropped.  The order
        // inside a group does not change any kernel's sums.
        constexpr int NB = 2 * T - 1;
        if (threadIdx.x < 2 * T) sm.bcnt[threadIdx.x] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            const uint32_t m = sm.mask[j];
            if (m) atomicAdd(&sm.bcnt[(__ffs(m) - 1) + (31 - __clz(m))], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int r = 0; r < NB; ++r) {
                sm.boff[r] = acc;
                acc += sm.bcnt[r];
                sm.bcnt[r] = 0;
            }
            sm.boff[NB] = acc;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) {
            const uint32_t m = sm.mask[j];
            if (m) {
                const int key = (__ffs(m) - 1) + (31 - __clz(m));
                sm.order[sm.boff[key] + atomicAdd(&sm.bcnt[key], 1)] = (typename K::Ord)j;
            }
        }
        __syncthreads();
        const int n_live = sm.boff[NB];
        // One group of KG = 32 / RPS kernels.  The rows it walks are the
        // selected rows base + stride i (all rows, or every fourth when the
        // warps share a group), taken RPS at a time: lane l works on kernel
        // grp KG + l % KG and, in block b, on selected row RPS b + l / KG.  A
        // block is skipped when no kernel of the group has a live row in it.
        // Which lane takes a row depends on the row alone, so a kernel's sums
        // do not depend on the other kernels of its group.
        constexpr int RPS = kBwdRows;
        constexpr int KG = 32 / RPS;
        auto group = [&](int grp, int base, int stride) {
            const int sub = lane / KG;
            const int idx = grp * KG + (lane % KG);
            const bool valid = idx < n_live;
            const int j = valid ? sm.order[idx] : 0;
            const uint32_t m = valid ? sm.mask[j] : 0u;
            float v[R::S];
#pragma unroll
            for (int q = 0; q < R::S / 4; ++q) {
                const float4 f = valid ? *reinterpret_cast<const float4 *>(sm.rec + j * R::SS + 4 * q)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
            }
            const float mx = v[0], my = v[1], a = v[2], b = v[3], c = v[4];
            float ea[C], w0[C], w1[C];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                ea[ch] = v[7 + ch * R::E];
                w0[ch] = LIN ? v[7 + ch * R::E + 1] : 0.0f;
                w1[ch] = LIN ? v[7 + ch * R::E + 2] : 0.0f;
            }
            BwdAcc<C, LIN> acc;
            acc.zero();
            const float2 nmx = f2(-mx), a2 = f2(a), lp2 = f2(v[5]);
            // blocks of RPS selected rows that hold a live row of the group
            const uint32_t um = __reduce_or_sync(0xffffffffu, m);
            const int nsel = T / stride;
            uint32_t blocks = 0;
#pragma unroll
            for (int bb = 0; bb < (T + RPS - 1) / RPS; ++bb) {
                bool any = false;
#pragma unroll
                for (int q = 0; q < RPS; ++q) {
                    const int i = RPS * bb + q;
                    if (i < nsel) any |= ((um >> (base + stride * i)) & 1u) != 0;
                }
                blocks |= (any ? 1u : 0u) << bb;
            }
            const uint32_t msel = m;
            while (blocks) {
                const int bb = __ffs(blocks) - 1;
                blocks &= blocks - 1;
                const int i = RPS * bb + sub;
                const bool in = i < nsel;
                const int r = in ? base + stride * i : 0;
                // lanes whose kernel has no live pixel in row r add zero
                const float qm = in && ((msel >> r) & 1u) ? qmax : -1.0f;
                const float dy = __fsub_rn(__fadd_rn(y0f, (float)r), my);
                const float t = __fmul_rn(b, dy);
                const float z1 = __fmul_rn(c, dy);
                const float u = __fmul_rn(z1, z1);
                float2 mb[C];
#pragma unroll
                for (int ch = 0; ch < C; ++ch) mb[ch] = f2(LIN ? fmaf(w1[ch], dy, ea[ch]) : ea[ch]);
                const float2 t2 = f2(t), u2 = f2(u);
                float2 A1 = f2(0.f), rA2 = f2(0.f), rS = f2(0.f), rE[C], F[C];
#pragma unroll
                for (int ch = 0; ch < C; ++ch) { rE[ch] = f2(0.f); F[ch] = f2(0.f); }
                const float *prow = sm.pst + r * G::RS;
                const float2 xt = f2(x0f);
#pragma unroll
                for (int p = 0; p < T / 2; ++p) {
                    const float *ps = prow + p * G::PS;
                    float2 H[C], nHy;
                    if (C == 3) {
                        const float4 s0 = *reinterpret_cast<const float4 *>(ps);
                        const float4 s1 = *reinterpret_cast<const float4 *>(ps + 4);
                        H[0] = make_float2(s0.x, s0.y);
                        H[C > 1 ? 1 : 0] = make_float2(s0.z, s0.w);
                        H[C > 2 ? 2 : 0] = make_float2(s1.x, s1.y);
                        nHy = make_float2(s1.z, s1.w);
                    } else {
                        const float4 s0 = *reinterpret_cast<const float4 *>(ps);
                        H[0] = make_float2(s0.x, s0.y);
                        nHy = make_float2(s0.z, s0.w);
                    }
                    // pixel centres x0 + 2p + 0.5, x0 + 2p + 1.5 (exact in FP32)
                    const float2 x2 = __fadd2_rn(xt, make_float2(2 * p + 0.5f, 2 * p + 1.5f));
                    const float2 dx = __fadd2_rn(x2, nmx);
                    const float2 z0 = __ffma2_rn(a2, dx, t2);
                    const float2 q = __ffma2_rn(z0, z0, u2);
                    const float2 arg = __ffma2_rn(q, k2, lp2);
                    float2 e = make_float2(ex2(arg.x), ex2(arg.y));
                    e.x = q.x <= qm ? e.x : 0.0f;
                    e.y = q.y <= qm ? e.y : 0.0f;
                    float2 rp = nHy;
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) {
                        const float2 mm = LIN ? __ffma2_rn(f2(w0[ch]), dx, mb[ch]) : mb[ch];
                        rp = __ffma2_rn(H[ch], mm, rp);
                    }
                    const float2 sv = __fmul2_rn(e, rp);
                    const float2 sz = __fmul2_rn(sv, z0);
                    A1 = __ffma2_rn(sz, dx, A1);
                    rA2 = __fadd2_rn(rA2, sz);
                    rS = __fadd2_rn(rS, sv);
                    const float2 edx = __fmul2_rn(e, dx);
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) {
                        rE[ch] = __ffma2_rn(e, H[ch], rE[ch]);
                        if (LIN) F[ch] = __ffma2_rn(edx, H[ch], F[ch]);
                    }
                }
                const float a2s = rA2.x + rA2.y, ss = rS.x + rS.y;
                acc.v[0] += A1.x + A1.y;
                acc.v[1] = fmaf(dy, a2s, acc.v[1]);
                acc.v[2] = fmaf(z1 * dy, ss, acc.v[2]);
                acc.v[3] += a2s;
                acc.v[4] = fmaf(z1, ss, acc.v[4]);
                acc.v[R::PI] += ss;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float es = rE[ch].x + rE[ch].y;
                    acc.v[5 + ch] += es;
                    if (LIN) {
                        acc.v[5 + C + ch] += F[ch].x + F[ch].y;
                        acc.v[5 + 2 * C + ch] = fmaf(dy, es, acc.v[5 + 2 * C + ch]);
                    }
                }
            }
            // the RPS lanes of each kernel add their sums (a fixed order)
#pragma unroll
            for (int o = KG; o < 32; o <<= 1)
#pragma unroll
                for (int q = 0; q < R::GS; ++q) acc.v[q] += __shfl_xor_sync(0xffffffffu, acc.v[q], o);
            // every stride-th row from base (stride 1, 2, 4 or 8)
            const uint32_t every = stride == 1 ? 0xffffffffu : stride == 2 ? 0x55555555u
                                 : stride == 4 ? 0x11111111u : 0x01010101u;
            const uint32_t rowsel = every << base;
            if (sub == 0 && (m & rowsel)) {
                if (w.part) {        // deterministic: this pair's own slot
                    float4 *dst = reinterpret_cast<float4 *>(w.part + (ti.start + c0 + j) * R::GS);
#pragma unroll
                    for (int q = 0; q < R::GS / 4; ++q)
                        dst[q] = make_float4(acc.v[4 * q], acc.v[4 * q + 1], acc.v[4 * q + 2],
                                             acc.v[4 * q + 3]);
                } else {
                    float4 *dst = reinterpret_cast<float4 *>(w.acc + (int64_t)sm.kid[j] * R::GS);
#pragma unroll
                    for (int q = 0; q < R::GS / 4; ++q)
                        atomicAdd(dst + q, make_float4(acc.v[4 * q], acc.v[4 * q + 1],
                                                       acc.v[4 * q + 2], acc.v[4 * q + 3]));
                }
            }
        };
        // Whole groups round-robin over the warps; with float atomics the
        // n_groups mod kNW groups of the last round are shared by all warps,
        // each taking the rows r = warp (mod kNW) and adding its own partial
        // sums (the deterministic mode keeps whole groups: one writer per pair).
        const int n_groups = (n_live + KG - 1) / KG;
        const int whole = w.part ? n_groups : n_groups - n_groups % kNW;
        for (int grp = warp; grp < whole; grp += kNW) group(grp, 0, 1);
        for (int grp = whole; grp < n_groups; ++grp) group(grp, warp, kNW);
        if (w.part) {                // pairs whose kernel misses every row add zero
            for (int i = threadIdx.x; i < nc * (R::GS / 4); i += kThreads) {
                const int j = i / (R::GS / 4), q = i - j * (R::GS / 4);
                if (!sm.mask[j])
                    reinterpret_cast<float4 *>(w.part + (ti.start + c0 + j) * R::GS)[q] =
                        make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
}

template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_render_bwd(const __grid_constant__ Geo g, Bufs w,
                                                            const float *__restrict__ y,
                                                            const float *__restrict__ inv_d,
                                                            const float *__restrict__ gy,
                                                            const float *__restrict__ target) {
    if (status_bad(w.status)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C, LIN, T> &sm = *reinterpret_cast<Smem<C, LIN, T> *>(smem_raw);
    const TileInfo ti = tile_info(g, w, blockIdx.x);
    if (ti.n == 0) return;
    const int64_t HW = (int64_t)ti.W * ti.H;
    const float norm = 2.0f / ((float)C * (float)HW);
    for (int pp = threadIdx.x; pp < T * T / 2; pp += kThreads) {
        const int row = pp / (T / 2), col = 2 * (pp % (T / 2));
        float H[2][C], nHy[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xi = ti.x0 + col + h, yi = ti.y0 + row;
            nHy[h] = 0.0f;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) H[h][ch] = 0.0f;
            if (xi < ti.W && yi < ti.H) {
                const int64_t o = (int64_t)yi * ti.W + xi;
                const float inv = g.rbf ? 1.0f : inv_d[o];   // Eq. 1: D = 1, no y term
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float yv = y[ch * HW + o];
                    const float Gv = gy ? gy[ch * HW + o] : norm * (yv - target[ch * HW + o]);
                    H[h][ch] = inv * Gv;
                    if (!g.rbf) nHy[h] = fmaf(-H[h][ch], yv, nHy[h]);
                }
            }
        }
        put_state<C, T>(sm.pst, row, col, H, nHy);
    }
    bwd_tile<C, LIN, T>(g, w, ti, sm, false);
}

// ---------------------------------------------------------------- fused fit tile

// Forward, MSE and backward of global tile t (all threads of the CTA).
template <int C, bool LIN, int T, int NC>
__device__ __forceinline__ void fit_tile_body(const Geo &g, const Bufs &w, int64_t t,
                                              Smem<C, LIN, T, NC> &sm, double *loss, int32_t hist,
                                              const int32_t *__restrict__ step) {
    using G = Geom<C, T>;
    const TileInfo ti = tile_info(g, w, t);
    const ImgDev &im = img_of(g, ti.b);
    const int32_t it = step ? step[ti.b] : 0;
    if (it >= im.iters) return;                      // this image has finished its run
    const int64_t HW = (int64_t)ti.W * ti.H;
    // With one band per warp (T <= 16) the lane's target values are loaded
    // before the forward, so that they arrive while it runs (0 outside the
    // image, where they are not read); with more bands they would hold too
    // many registers and are read after it.
    constexpr bool kEarly = G::BPW == 1;
    float tg[G::BPW][2][C];
#pragma unroll
    for (int bi = 0; bi < (kEarly ? G::BPW : 0); ++bi) {
        int row, col;
        const bool mine = lane_pixels<C, T>(bi, row, col);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xi = ti.x0 + col + h, yi = ti.y0 + row;
            const bool in = mine && xi < ti.W && yi < ti.H;
            const int64_t o = (int64_t)yi * ti.W + xi;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) tg[bi][h][ch] = in ? __ldg(im.target + ch * HW + o) : 0.0f;
        }
    }
    float2 Dv[G::BPW], Nv[G::BPW][C];
    fwd_tile<C, LIN, T>(g, w, ti, sm, Dv, Nv);
    const float norm = 2.0f / ((float)C * (float)HW);
    float se = 0.0f;                                 // this thread's <= 2 C squared errors per band
#pragma unroll
    for (int bi = 0; bi < G::BPW; ++bi) {
        int row, col;
        if (!lane_pixels<C, T>(bi, row, col)) continue;
        float H[2][C], nHy[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xi = ti.x0 + col + h, yi = ti.y0 + row;
            nHy[h] = 0.0f;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) H[h][ch] = 0.0f;
            if (xi < ti.W && yi < ti.H) {
                const int64_t o = (int64_t)yi * ti.W + xi;
                const float D = h ? Dv[bi].y : Dv[bi].x;
                // softmax gates: y = N / D; RBF sum (Eq. 1): y = N and D = 1
                const float inv = g.rbf ? 1.0f : (D > 0.0f ? 1.0f / D : 0.0f);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float yv = (h ? Nv[bi][ch].y : Nv[bi][ch].x) * inv;
                    const float d = yv - (kEarly ? tg[bi][h][ch] : im.target[ch * HW + o]);
                    se = fmaf(d, d, se);
                    H[h][ch] = inv * (norm * d);
                    if (!g.rbf) nHy[h] = fmaf(-H[h][ch], yv, nHy[h]);
                }
            }
        }
        put_state<C, T>(sm.pst, row, col, H, nHy);
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        if ((threadIdx.x & 31) == 0) sm.lsum[threadIdx.x >> 5] = (double)se;
    }
    __syncthreads();
    if (loss && threadIdx.x == 0 && it < hist) {
        double s = 0.0;
        for (int i = 0; i < kNW; ++i) s += sm.lsum[i];
        atomicAdd(loss + (int64_t)ti.b * hist + it, s / ((double)C * (double)HW));
    }
    if (ti.n == 0) return;
    bwd_tile<C, LIN, T>(g, w, ti, sm, true);
}

template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_fit_tile(const __grid_constant__ Geo g, Bufs w,
                                                          double *loss, int32_t hist,
                                                          const int32_t *__restrict__ step) {
    if (status_bad(w.status)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C, LIN, T, fit_nch(T)> &sm = *reinterpret_cast<Smem<C, LIN, T, fit_nch(T)> *>(smem_raw);
    fit_tile_body<C, LIN, T>(g, w, blockIdx.x, sm, loss, hist, step);
}

// The same work as one persistent grid: each CTA takes the next tile from a
// queue (a counter zeroed before the launch) until the table is exhausted.
template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_fit_tile_persistent(const __grid_constant__ Geo g, Bufs w, double *loss, int32_t hist,
                          const int32_t *__restrict__ step) {
    if (status_bad(w.status)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C, LIN, T, fit_nch(T)> &sm = *reinterpret_cast<Smem<C, LIN, T, fit_nch(T)> *>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) sm.next = (long long)atomicAdd(w.work, 1u);
        __syncthreads();
        const int64_t t = sm.next;
        __syncthreads();
        if (t >= g.tiles_total) break;
        fit_tile_body<C, LIN, T>(g, w, t, sm, loss, hist, step);
    }
}

// ---------------------------------------------------------------- finalize

// Raw sums -> gradients in API units, ADDED into the SoA gradient arrays.
__global__ void k_finalize(const __grid_constant__ Geo g, Bufs w, smoe_params grad) {
    if (status_bad(w.status)) return;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K_total) return;
    const int4 rc = w.rect[k];
    if (rc.x > rc.z) return;       // listed in no tile: its gradient is exactly 0
    const ImgDev &im = img_of(g, img_by_kernel(g, k));
    const float *s = w.acc + k * g.GS;
    const float *r = w.rec + k * g.S;
    const int C = g.C, E = g.linear ? 3 : 1;
    float gmx = r[2] * s[3], gmy = fmaf(r[3], s[3], r[4] * s[4]);
    for (int ch = 0; ch < C; ++ch) {
        grad.ea[k * C + ch] += s[5 + ch];
        if (g.linear) {
            gmx -= r[7 + ch * E + 1] * s[5 + ch];
            gmy -= r[7 + ch * E + 2] * s[5 + ch];
            grad.eW[(k * C + ch) * 2] += s[5 + C + ch] / g.scale;
            grad.eW[(k * C + ch) * 2 + 1] += s[5 + 2 * C + ch] / g.scale;
        }
    }
    grad.mu[2 * k] += gmx * (float)im.W;
    grad.mu[2 * k + 1] += gmy * (float)im.H;
    grad.chol[3 * k] += -s[0] / g.scale;
    grad.chol[3 * k + 1] += -s[1] / g.scale;
    grad.chol[3 * k + 2] += -s[2] / g.scale;
    if (grad.logpi) grad.logpi[k] += s[5 + C * E];
}

// Raise a tile kernel's dynamic shared-memory limit once per instantiation.
template <typename K>
cudaError_t smem_attr(K kern, size_t smem, bool &done) {
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int C, bool LIN, int T>
cudaError_t dispatch_one(const Geo &g, const Bufs &w, int which, const float *y, float *yo,
                         float *inv_do, const float *inv_d, const float *gy, const float *target,
                         double *loss, int32_t hist, const int32_t *step, cudaStream_t st) {
    const unsigned grid = (unsigned)g.tiles_total;
    if (grid == 0) return cudaSuccess;
    constexpr size_t smem = smem_bytes<C, LIN, T>();
    constexpr size_t smem_fit = smem_bytes<C, LIN, T, fit_nch(T)>();
    static bool a0 = false, a1 = false, a2 = false;
    cudaError_t e;
    if (which == 0) {
        if ((e = smem_attr(k_render<C, LIN, T>, smem, a0)) != cudaSuccess) return e;
        k_render<C, LIN, T><<<grid, kThreads, smem, st>>>(g, w, yo, inv_do);
    } else if (which == 1) {
        if ((e = smem_attr(k_render_bwd<C, LIN, T>, smem, a1)) != cudaSuccess) return e;
        k_render_bwd<C, LIN, T><<<grid, kThreads, smem, st>>>(g, w, y, inv_d, gy, target);
    } else if (which == 2) {
        if ((e = smem_attr(k_fit_tile<C, LIN, T>, smem_fit, a2)) != cudaSuccess) return e;
        k_fit_tile<C, LIN, T><<<grid, kThreads, smem_fit, st>>>(g, w, loss, hist, step);
    } else if (which == 4) {
        static bool a4 = false;
        if ((e = smem_attr(k_render_mean<C, LIN, T>, smem, a4)) != cudaSuccess) return e;
        k_render_mean<C, LIN, T><<<(unsigned)(g.tiles_total / g.B), kThreads, smem, st>>>(g, w, yo);
    } else {
        static bool a3 = false;
        static int resident = 0;
        if ((e = smem_attr(k_fit_tile_persistent<C, LIN, T>, smem_fit, a3)) != cudaSuccess) return e;
        if (!resident) {
            int dev = 0, sms = 0, per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &per_sm, k_fit_tile_persistent<C, LIN, T>, kThreads, smem_fit)) != cudaSuccess)
                return e;
            resident = sms * (per_sm > 0 ? per_sm : 1);
        }
        if ((e = cudaMemsetAsync(w.work, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
        const unsigned pg = grid < (unsigned)resident ? grid : (unsigned)resident;
        k_fit_tile_persistent<C, LIN, T><<<pg, kThreads, smem_fit, st>>>(g, w, loss, hist, step);
    }
    return cudaGetLastError();
}

template <int C, bool LIN>
cudaError_t dispatch_T(const Geo &g, const Bufs &w, int which, const float *y, float *yo,
                       float *inv_do, const float *inv_d, const float *gy, const float *target,
                       double *loss, int32_t hist, const int32_t *step, cudaStream_t st) {
    switch (g.T) {
        case 8:
            return dispatch_one<C, LIN, 8>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss,
                                           hist, step, st);
        case 16:
            return dispatch_one<C, LIN, 16>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss,
                                            hist, step, st);
        case 32:
            return dispatch_one<C, LIN, 32>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss,
                                            hist, step, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch(const Geo &g, const Bufs &w, int which, const float *y, float *yo,
                     float *inv_do, const float *inv_d, const float *gy, const float *target,
                     double *loss, int32_t hist, const int32_t *step, cudaStream_t st) {
    if (g.C == 1 && !g.linear)
        return dispatch_T<1, false>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss, hist, step, st);
    if (g.C == 1 && g.linear)
        return dispatch_T<1, true>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss, hist, step, st);
    if (g.C == 3 && !g.linear)
        return dispatch_T<3, false>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss, hist, step, st);
    if (g.C == 3 && g.linear)
        return dispatch_T<3, true>(g, w, which, y, yo, inv_do, inv_d, gy, target, loss, hist, step, st);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_render(const Geo &g, const Bufs &w, float *y, float *inv_d, cudaStream_t st) {
    return dispatch(g, w, 0, nullptr, y, inv_d, nullptr, nullptr, nullptr, nullptr, 0, nullptr, st);
}

cudaError_t launch_render_bwd(const Geo &g, const Bufs &w, const float *y, const float *inv_d,
                              const float *gy, const float *target, const smoe_params &grad,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(w.acc, 0, sizeof(float) * g.GS * g.K_total, st);
    if (e != cudaSuccess) return e;
    e = dispatch(g, w, 1, y, nullptr, nullptr, inv_d, gy, target, nullptr, 0, nullptr, st);
    if (e != cudaSuccess) return e;
    if (g.K_total > 0)
        k_finalize<<<(unsigned)((g.K_total + 255) / 256), 256, 0, st>>>(g, w, grad);
    return cudaGetLastError();
}

cudaError_t launch_render_mean(const Geo &g, const Bufs &w, float *y, cudaStream_t st) {
    return dispatch(g, w, 4, nullptr, y, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, st);
}

cudaError_t launch_fit_tiles(const Geo &g, const Bufs &w, double *loss, int32_t hist,
                             const int32_t *step, bool persistent, cudaStream_t st) {
    return dispatch(g, w, persistent ? 3 : 2, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, loss, hist, step, st);
}

}  // namespace smoe
