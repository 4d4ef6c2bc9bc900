// Tile kernels of the rasterised SMoE regression.
//
// Forward (Eqs. 2-5, per tile, pixel-major): each lane owns a few pixels of
// the tile and walks the tile's kernel list, keeping the gate denominator
// D = sum e and the numerators N_c = sum e m_c in FP32 registers; the warps of
// a CTA split the list (T = 8, 16) or the tile (T = 32) and meet in shared
// memory at the end.  Kernel records are staged per warp in shared memory,
// 32 at a time, and the next 32 are fetched into registers while the current
// ones are evaluated.
//
// Backward (the gradient-descent fit through the rasteriser, Sec. III-D;
// kernel-major): each lane owns ONE kernel of the tile's list and walks the
// tile's pixels, whose per-pixel upstream state sits in shared memory, so the
// per-kernel sums need no cross-lane reduction.  Gates are recomputed.  The
// sums are raw moments (below); a finalize pass turns them into gradients.
// One float4 atomic add per 4 sums per (tile, kernel).
//
// Raw per-kernel sums (s = g * sum_c G_c (m_c - y_c), g = e / D,
// H_c = G_c / D, so s = e (sum_c H_c m_c - sum_c H_c y_c) and g G_c = e H_c):
//   [0] A1 = sum s z0 dx  [1] B1 = sum s z0 dy  [2] C1 = sum s z1 dy
//   [3] A2 = sum s z0     [4] Z3 = sum s z1
//   [5+c] E_c = sum e H_c,   linear: [5+C+c] F_c = sum e H_c dx,
//                                    [5+2C+c] Fy_c = sum e H_c dy
// and the gradients (Sec. III-D chain rule of Eqs. 2-4):
//   dL/da = -A1, dL/db = -B1, dL/dc = -C1,
//   dL/dmx = a A2 - sum_c W_c0 E_c,  dL/dmy = b A2 + c Z3 - sum_c W_c1 E_c,
//   dL/dea_c = E_c, dL/dW_c0 = F_c, dL/dW_c1 = Fy_c.
#include "smoe_internal.cuh"

namespace smoe {

namespace {

constexpr int kNW = 4;                // warps per CTA
constexpr int kThreads = kNW * 32;

template <int T>
struct Shape {
    static constexpr int SUB = T >= 16 ? 16 : 8;       // side of one warp's pixel block
    static constexpr int NSUB = (T / SUB) * (T / SUB);  // pixel blocks per tile
    static constexpr int KSPLIT = kNW / NSUB;           // warps sharing a pixel block
    static constexpr int PX = SUB / 4;                  // pixels per lane along a row
    static constexpr int RY = SUB / 8;                  // rows per lane
    static constexpr int NPX = PX * RY;
};

template <int C, bool LIN>
struct Rec {
    static constexpr int E = LIN ? 3 : 1;
    static constexpr int S = (7 + C * E + 3) & ~3;
    static constexpr int GS = (5 + C * E + 3) & ~3;
};

// Tile coordinates of global tile t.
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

// ---------------------------------------------------------------- forward

template <int C, bool LIN, int T>
__device__ __forceinline__ void fwd_accumulate(const Geo &g, const float *__restrict__ rec,
                                               const int32_t *__restrict__ list, int n,
                                               float x0_px, float y0_px, float *stage,
                                               float (&D)[Shape<T>::NPX],
                                               float (&N)[C][Shape<T>::NPX]) {
    using Sh = Shape<T>;
    using R = Rec<C, LIN>;
    constexpr int S = R::S;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int split = warp % Sh::KSPLIT;
    const int lr = lane >> 2, lc = lane & 3;
    float xc[Sh::PX], yc[Sh::RY];
#pragma unroll
    for (int px = 0; px < Sh::PX; ++px) xc[px] = x0_px + (float)(lc * Sh::PX + px) + 0.5f;
#pragma unroll
    for (int ry = 0; ry < Sh::RY; ++ry) yc[ry] = y0_px + (float)(lr + 8 * ry) + 0.5f;
#pragma unroll
    for (int i = 0; i < Sh::NPX; ++i) {
        D[i] = 0.0f;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) N[ch][i] = 0.0f;
    }
    const float qmax = g.qmax;
    const int nchunk = (n + 31) >> 5;
    float4 nxt[S / 4];
#pragma unroll
    for (int q = 0; q < S / 4; ++q) nxt[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int ci = split;
    if (ci < nchunk) {
        const int j = ci * 32 + lane;
        if (j < n) {
            const float4 *src = reinterpret_cast<const float4 *>(rec + (int64_t)list[j] * S);
#pragma unroll
            for (int q = 0; q < S / 4; ++q) nxt[q] = __ldg(src + q);
        }
    }
    for (; ci < nchunk; ci += Sh::KSPLIT) {
        __syncwarp();
        float4 *dst = reinterpret_cast<float4 *>(stage + lane * S);
#pragma unroll
        for (int q = 0; q < S / 4; ++q) dst[q] = nxt[q];
        __syncwarp();
        const int cnt = min(32, n - ci * 32);
        const int cn = ci + Sh::KSPLIT;
        if (cn < nchunk) {
            const int j = cn * 32 + lane;
            if (j < n) {
                const float4 *src = reinterpret_cast<const float4 *>(rec + (int64_t)list[j] * S);
#pragma unroll
                for (int q = 0; q < S / 4; ++q) nxt[q] = __ldg(src + q);
            }
        }
        for (int kk = 0; kk < cnt; ++kk) {
            const float *r = stage + kk * S;
            const float4 r0 = *reinterpret_cast<const float4 *>(r);
            const float mx = r0.x, my = r0.y, a = r0.z, b = r0.w;
            const float c = r[4];
            float ea[C], w0[C], w1[C];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                ea[ch] = r[7 + ch * R::E];
                w0[ch] = LIN ? r[7 + ch * R::E + 1] : 0.0f;
                w1[ch] = LIN ? r[7 + ch * R::E + 2] : 0.0f;
            }
            float dx[Sh::PX];
#pragma unroll
            for (int px = 0; px < Sh::PX; ++px) dx[px] = __fsub_rn(xc[px], mx);
#pragma unroll
            for (int ry = 0; ry < Sh::RY; ++ry) {
                const float dy = __fsub_rn(yc[ry], my);
                const float t = __fmul_rn(b, dy);
                const float z1 = __fmul_rn(c, dy);
                const float u = __fmul_rn(z1, z1);
                float mb[C];
#pragma unroll
                for (int ch = 0; ch < C; ++ch) mb[ch] = LIN ? fmaf(w1[ch], dy, ea[ch]) : ea[ch];
#pragma unroll
                for (int px = 0; px < Sh::PX; ++px) {
                    float z0;
                    const float q = q_of(a, dx[px], t, u, z0);
                    const float e = gate_e(q, qmax);
                    const int i = ry * Sh::PX + px;
                    D[i] += e;
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) {
                        const float m = LIN ? fmaf(w0[ch], dx[px], mb[ch]) : mb[ch];
                        N[ch][i] = fmaf(e, m, N[ch][i]);
                    }
                }
            }
        }
    }
}

// Shared memory for the forward phase.
template <int C, bool LIN, int T>
struct FwdSmem {
    float stage[kNW][32 * Rec<C, LIN>::S];
    float red[Shape<T>::KSPLIT][C + 1][T * T];
};

// Run the forward over one tile and leave per-pixel D and N_c (summed over
// the warps sharing a pixel) in red[0][.][px] for px in [0, T*T).
template <int C, bool LIN, int T>
__device__ __forceinline__ void fwd_tile(const Geo &g, const Bufs &w, const TileInfo &ti,
                                         FwdSmem<C, LIN, T> &sm) {
    using Sh = Shape<T>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = warp / Sh::KSPLIT, split = warp % Sh::KSPLIT;
    const int sx = (sub % (T / Sh::SUB)) * Sh::SUB, sy = (sub / (T / Sh::SUB)) * Sh::SUB;
    float D[Sh::NPX], N[C][Sh::NPX];
    fwd_accumulate<C, LIN, T>(g, w.rec, w.pair_k + ti.start, ti.n, (float)(ti.x0 + sx),
                              (float)(ti.y0 + sy), sm.stage[warp], D, N);
    const int lr = lane >> 2, lc = lane & 3;
#pragma unroll
    for (int ry = 0; ry < Sh::RY; ++ry)
#pragma unroll
        for (int px = 0; px < Sh::PX; ++px) {
            const int p = (sy + lr + 8 * ry) * T + sx + lc * Sh::PX + px;
            const int i = ry * Sh::PX + px;
            sm.red[split][0][p] = D[i];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) sm.red[split][1 + ch][p] = N[ch][i];
        }
    __syncthreads();
    if (Sh::KSPLIT > 1) {
        for (int p = threadIdx.x; p < T * T; p += kThreads) {
#pragma unroll
            for (int v = 0; v < C + 1; ++v) {
                float s = sm.red[0][v][p];
#pragma unroll
                for (int k = 1; k < Sh::KSPLIT; ++k) s += sm.red[k][v][p];
                sm.red[0][v][p] = s;
            }
        }
        __syncthreads();
    }
}

template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads) k_render(const __grid_constant__ Geo g, Bufs w,
                                                     float *__restrict__ y,
                                                     float *__restrict__ inv_d) {
    if (status_bad(w.status)) return;
    __shared__ __align__(16) FwdSmem<C, LIN, T> sm;
    const TileInfo ti = tile_info(g, w, blockIdx.x);
    fwd_tile<C, LIN, T>(g, w, ti, sm);
    const int64_t HW = (int64_t)ti.W * ti.H;
    for (int p = threadIdx.x; p < T * T; p += kThreads) {
        const int xi = ti.x0 + (p % T), yi = ti.y0 + (p / T);
        if (xi >= ti.W || yi >= ti.H) continue;
        const float D = sm.red[0][0][p];
        const float inv = D > 0.0f ? 1.0f / D : 0.0f;
        const int64_t o = (int64_t)yi * ti.W + xi;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) y[ch * HW + o] = sm.red[0][1 + ch][p] * inv;
        if (inv_d) inv_d[o] = inv;
    }
}

// ---------------------------------------------------------------- backward

// Per-pixel upstream state: (H_0 .. H_{C-1}, Hy) with H_c = G_c / D and
// Hy = sum_c H_c y_c; zero for pixels outside the image or with D = 0.
template <int C>
struct PixState {
    static constexpr int N = C + 1 <= 2 ? 2 : 4;
};

template <int C, bool LIN, int T>
__device__ __forceinline__ void bwd_accumulate(const Geo &g, const Bufs &w, const TileInfo &ti,
                                               const float *pstate) {
    using R = Rec<C, LIN>;
    constexpr int S = R::S, GS = R::GS;
    constexpr int PN = PixState<C>::N;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nchunk = (ti.n + 31) >> 5;
    for (int ci = warp; ci < nchunk; ci += kNW) {
        const int j = ci * 32 + lane;
        const bool valid = j < ti.n;
        float r[S];
        int kid = 0;
        if (valid) {
            kid = w.pair_k[ti.start + j];
            const float4 *src = reinterpret_cast<const float4 *>(w.rec + (int64_t)kid * S);
#pragma unroll
            for (int q = 0; q < S / 4; ++q) {
                const float4 v = __ldg(src + q);
                r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < S; ++q) r[q] = 0.0f;
        }
        const float qm = valid ? g.qmax : -1.0f;     // inactive lanes include nothing
        const float mx = r[0], my = r[1], a = r[2], b = r[3], c = r[4];
        float ea[C], w0[C], w1[C];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            ea[ch] = r[7 + ch * R::E];
            w0[ch] = LIN ? r[7 + ch * R::E + 1] : 0.0f;
            w1[ch] = LIN ? r[7 + ch * R::E + 2] : 0.0f;
        }
        float dxs[T];
#pragma unroll
        for (int col = 0; col < T; ++col) dxs[col] = __fsub_rn((float)(ti.x0 + col) + 0.5f, mx);
        float A1 = 0.f, B1 = 0.f, C1 = 0.f, A2 = 0.f, Z3 = 0.f;
        float E[C], F[C], Fy[C];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) { E[ch] = 0.f; F[ch] = 0.f; Fy[ch] = 0.f; }
        for (int row = 0; row < T; ++row) {
            const float dy = __fsub_rn((float)(ti.y0 + row) + 0.5f, my);
            const float t = __fmul_rn(b, dy);
            const float z1 = __fmul_rn(c, dy);
            const float u = __fmul_rn(z1, z1);
            float mb[C], rE[C];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                mb[ch] = LIN ? fmaf(w1[ch], dy, ea[ch]) : ea[ch];
                rE[ch] = 0.f;
            }
            float rA2 = 0.f, rS = 0.f;
            const float *prow = pstate + row * T * PN;
#pragma unroll
            for (int col = 0; col < T; ++col) {
                float H[C], Hy;
                if (PN == 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(prow + col * 4);
                    H[0] = v.x;
                    if (C > 1) H[1] = v.y;
                    if (C > 2) H[2] = v.z;
                    Hy = v.w;
                } else {
                    const float2 v = *reinterpret_cast<const float2 *>(prow + col * 2);
                    H[0] = v.x;
                    Hy = v.y;
                }
                const float dx = dxs[col];
                float z0;
                const float q = q_of(a, dx, t, u, z0);
                const float e = gate_e(q, qm);
                float rp = -Hy;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float m = LIN ? fmaf(w0[ch], dx, mb[ch]) : mb[ch];
                    rp = fmaf(H[ch], m, rp);
                }
                const float s = e * rp;
                const float sz = s * z0;
                A1 = fmaf(sz, dx, A1);
                rA2 += sz;
                rS += s;
                const float edx = e * dx;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    rE[ch] = fmaf(e, H[ch], rE[ch]);
                    if (LIN) F[ch] = fmaf(edx, H[ch], F[ch]);
                }
            }
            A2 += rA2;
            B1 = fmaf(dy, rA2, B1);
            Z3 = fmaf(z1, rS, Z3);
            C1 = fmaf(z1 * dy, rS, C1);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                E[ch] += rE[ch];
                if (LIN) Fy[ch] = fmaf(dy, rE[ch], Fy[ch]);
            }
        }
        if (valid) {
            float o[GS];
#pragma unroll
            for (int q = 0; q < GS; ++q) o[q] = 0.f;
            o[0] = A1; o[1] = B1; o[2] = C1; o[3] = A2; o[4] = Z3;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                o[5 + ch] = E[ch];
                if (LIN) { o[5 + C + ch] = F[ch]; o[5 + 2 * C + ch] = Fy[ch]; }
            }
            float4 *dst = reinterpret_cast<float4 *>(w.acc + (int64_t)kid * GS);
#pragma unroll
            for (int q = 0; q < GS / 4; ++q)
                atomicAdd(dst + q, make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]));
        }
    }
}

template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads) k_render_bwd(const __grid_constant__ Geo g, Bufs w,
                                                         const float *__restrict__ y,
                                                         const float *__restrict__ inv_d,
                                                         const float *__restrict__ gy,
                                                         const float *__restrict__ target) {
    if (status_bad(w.status)) return;
    constexpr int PN = PixState<C>::N;
    __shared__ __align__(16) float pstate[T * T * PN];
    const TileInfo ti = tile_info(g, w, blockIdx.x);
    if (ti.n == 0) return;
    const int64_t HW = (int64_t)ti.W * ti.H;
    const float norm = 2.0f / ((float)C * (float)HW);
    for (int p = threadIdx.x; p < T * T; p += kThreads) {
        const int xi = ti.x0 + (p % T), yi = ti.y0 + (p / T);
        float H[4] = {0.f, 0.f, 0.f, 0.f}, Hy = 0.f;
        if (xi < ti.W && yi < ti.H) {
            const int64_t o = (int64_t)yi * ti.W + xi;
            const float inv = inv_d[o];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const float yv = y[ch * HW + o];
                const float G = gy ? gy[ch * HW + o] : norm * (yv - target[ch * HW + o]);
                H[ch] = inv * G;
                Hy = fmaf(H[ch], yv, Hy);
            }
        }
        if (PN == 4) {
            reinterpret_cast<float4 *>(pstate)[p] = make_float4(H[0], H[1], H[2], Hy);
        } else {
            reinterpret_cast<float2 *>(pstate)[p] = make_float2(H[0], Hy);
        }
    }
    __syncthreads();
    bwd_accumulate<C, LIN, T>(g, w, ti, pstate);
}

// ---------------------------------------------------------------- fused fit tile

template <int C, bool LIN, int T>
__global__ void __launch_bounds__(kThreads) k_fit_tile(const __grid_constant__ Geo g, Bufs w,
                                                       double *loss, int32_t hist,
                                                       const int32_t *__restrict__ step) {
    if (status_bad(w.status)) return;
    constexpr int PN = PixState<C>::N;
    __shared__ __align__(16) FwdSmem<C, LIN, T> sm;
    __shared__ __align__(16) float pstate[T * T * PN];
    __shared__ double lsum[kNW];
    const TileInfo ti = tile_info(g, w, blockIdx.x);
    const ImgDev &im = img_of(g, ti.b);
    const int32_t it = step ? step[ti.b] : 0;
    if (it >= im.iters) return;                      // this image has finished its run
    fwd_tile<C, LIN, T>(g, w, ti, sm);
    const int64_t HW = (int64_t)ti.W * ti.H;
    const float norm = 2.0f / ((float)C * (float)HW);
    double se = 0.0;
    for (int p = threadIdx.x; p < T * T; p += kThreads) {
        const int xi = ti.x0 + (p % T), yi = ti.y0 + (p / T);
        float H[4] = {0.f, 0.f, 0.f, 0.f}, Hy = 0.f;
        if (xi < ti.W && yi < ti.H) {
            const int64_t o = (int64_t)yi * ti.W + xi;
            const float D = sm.red[0][0][p];
            const float inv = D > 0.0f ? 1.0f / D : 0.0f;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const float yv = sm.red[0][1 + ch][p] * inv;
                const float d = yv - im.target[ch * HW + o];
                se += (double)d * d;
                H[ch] = inv * (norm * d);
                Hy = fmaf(H[ch], yv, Hy);
            }
        }
        if (PN == 4) {
            reinterpret_cast<float4 *>(pstate)[p] = make_float4(H[0], H[1], H[2], Hy);
        } else {
            reinterpret_cast<float2 *>(pstate)[p] = make_float2(H[0], Hy);
        }
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        if ((threadIdx.x & 31) == 0) lsum[threadIdx.x >> 5] = se;
    }
    __syncthreads();
    if (loss && threadIdx.x == 0 && it < hist) {
        double s = 0.0;
        for (int i = 0; i < kNW; ++i) s += lsum[i];
        atomicAdd(loss + (int64_t)ti.b * hist + it, s / ((double)C * (double)HW));
    }
    if (ti.n == 0) return;
    bwd_accumulate<C, LIN, T>(g, w, ti, pstate);
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
}

template <int C, bool LIN>
cudaError_t dispatch_T(const Geo &g, const Bufs &w, int which, const float *y, float *yo,
                       float *inv_do, const float *inv_d, const float *gy, const float *target,
                       double *loss, int32_t hist, const int32_t *step, cudaStream_t st) {
    const unsigned grid = (unsigned)g.tiles_total;
    if (grid == 0) return cudaSuccess;
#define SMOE_LAUNCH(TT)                                                                   \
    if (which == 0) k_render<C, LIN, TT><<<grid, kThreads, 0, st>>>(g, w, yo, inv_do);    \
    else if (which == 1)                                                                  \
        k_render_bwd<C, LIN, TT><<<grid, kThreads, 0, st>>>(g, w, y, inv_d, gy, target);  \
    else k_fit_tile<C, LIN, TT><<<grid, kThreads, 0, st>>>(g, w, loss, hist, step);
    switch (g.T) {
        case 8: SMOE_LAUNCH(8) break;
        case 16: SMOE_LAUNCH(16) break;
        case 32: SMOE_LAUNCH(32) break;
        default: return cudaErrorInvalidValue;
    }
#undef SMOE_LAUNCH
    return cudaGetLastError();
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

cudaError_t launch_fit_tiles(const Geo &g, const Bufs &w, double *loss, int32_t hist,
                             const int32_t *step, cudaStream_t st) {
    return dispatch(g, w, 2, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, loss, hist,
                    step, st);
}

}  // namespace smoe
