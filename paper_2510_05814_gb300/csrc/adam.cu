// Adam (Sec. VI-B: all groups optimised with Adam; per-group learning rates;
// the centre rate decays exponentially over the run), torch semantics in FP32:
//   m <- m + (1 - b1) (g - m);  v <- b2 v + (1 - b2) g^2
//   p <- p - (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
#include <cmath>

#include "smoe_internal.cuh"

namespace smoe {

namespace {

struct Betas {
    float b2, omb1, omb2, eps;   // b2, 1 - b1, 1 - b2 (rounded once from FP64), eps
};

struct AdamK {
    Betas be;
    float step_size;       // lr / (1 - b1^t)
    float inv_sqrt_bc2;    // 1 / sqrt(1 - b2^t)
};

// Every operation rounded explicitly: the update is the same bit for bit in
// every kernel and code path that inlines it (no contraction left to the
// compiler), so a fit does not depend on how its kernels share CTAs.
__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, const AdamK &k) {
    m = __fmaf_rn(k.be.omb1, __fsub_rn(g, m), m);
    v = __fmaf_rn(k.be.b2, v, __fmul_rn(__fmul_rn(k.be.omb2, g), g));
    const float denom = __fmaf_rn(__fsqrt_rn(v), k.inv_sqrt_bc2, k.be.eps);
    p = __fmaf_rn(-k.step_size, __fdiv_rn(m, denom), p);
}

// One launch over the groups of a SoA parameter set; zeroes g.
__global__ void k_adam_soa(int64_t K, int C, int has_w, int has_pi, smoe_params p,
                           smoe_params gr, smoe_params m, smoe_params v, float lr0, float lr1,
                           float lr2, float lr3, float lr4, Betas be, float bc1, float isb2) {
    const int64_t n_mu = 2 * K, n_ch = 3 * K, n_ea = (int64_t)C * K;
    const int64_t n_w = has_w ? 2 * (int64_t)C * K : 0;
    const int64_t n_pi = has_pi ? K : 0;
    const int64_t total = n_mu + n_ch + n_ea + n_w + n_pi;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        float *pp, *gg, *mm, *vv;
        float lr;
        int64_t x = i;
        if (x < n_mu) { pp = p.mu; gg = gr.mu; mm = m.mu; vv = v.mu; lr = lr0; }
        else if ((x -= n_mu) < n_ch) { pp = p.chol; gg = gr.chol; mm = m.chol; vv = v.chol; lr = lr1; }
        else if ((x -= n_ch) < n_ea) { pp = p.ea; gg = gr.ea; mm = m.ea; vv = v.ea; lr = lr2; }
        else if ((x -= n_ea) < n_w) { pp = p.eW; gg = gr.eW; mm = m.eW; vv = v.eW; lr = lr3; }
        else { x -= n_w; pp = p.logpi; gg = gr.logpi; mm = m.logpi; vv = v.logpi; lr = lr4; }
        AdamK k{be, lr / bc1, isb2};
        float pv = pp[x], mv = mm[x], vv_ = vv[x];
        adam1(pv, gg[x], mv, vv_, k);
        pp[x] = pv; mm[x] = mv; vv[x] = vv_;
        gg[x] = 0.0f;
    }
}

// x^n by squaring: FP64 multiplies only (no transcendental, whose FP64
// form is slow on this part); relative error about 2 log2(n) ulp.
__device__ __forceinline__ double ipow(double x, uint32_t n) {
    double r = 1.0;
    while (n) {
        if (n & 1u) r *= x;
        x *= x;
        n >>= 1;
    }
    return r;
}

// Per-image Adam coefficients of the current step, formed in FP64 and rounded
// once: the four step sizes lr_g / (1 - b1^t) (the centre rate follows the
// exponential schedule lr_mu0 (lr_mu1 / lr_mu0)^(it / (iters - 1)), i.e.
// lr_mu0 rho^it) and 1 / sqrt(1 - b2^t).  Threads stride over images.
__device__ void adam_coefs(const Geo &g, const int32_t *step, double b1, double b2,
                           float *coef) {
    for (int b = threadIdx.x; b < g.B; b += blockDim.x) {
        const ImgDev &im = img_of(g, b);
        const int32_t it = step[b];
        const uint32_t t = (uint32_t)it + 1u;
        const double bc1 = 1.0 - ipow(b1, t);
        const double bc2 = 1.0 - ipow(b2, t);
        const double lr_mu = im.lr_mu0 > 0.0f ? (double)im.lr_mu0 * ipow(im.mu_rho, (uint32_t)it) : 0.0;
        float *c = coef + 8 * b;
        c[0] = (float)(lr_mu / bc1);
        c[1] = (float)(im.lr_chol / bc1);
        c[2] = (float)(im.lr_ea / bc1);
        c[3] = (float)(im.lr_eW / bc1);
        c[4] = (float)(1.0 / sqrt(bc2));
        c[5] = (float)(im.lr_pi / bc1);
    }
}

__global__ void k_adam_coefs(const __grid_constant__ Geo g, const int32_t *step, double b1,
                             double b2, float *coef) {
    adam_coefs(g, step, b1, b2, coef);
}

// Fit: raw per-kernel sums -> gradients (see render.cu) -> Adam on the 5 + C
// (+ 2C, + 1 with gate weights) parameters of the kernel; zeroes the sums.
// Two phases per CTA of kAdamThreads kernels: (1) each thread turns its
// kernel's sums and prepared record (loaded whole, float4) into gradients in
// shared memory, laid out like the parameter arrays; (2) the CTA updates the
// parameters and moments group by group, consecutive threads on consecutive
// elements, so every global access is coalesced.  The last CTA to finish
// advances every running image's step counter and forms the coefficients of
// the next step.
// Kernels per CTA of the Adam launches: 128 measured 4 % faster than 256
// on the 2048^2 fit (38.9 against 40.5 us; 512 spills).
#ifndef SMOE_ADAM_THREADS
#define SMOE_ADAM_THREADS 128
#endif
constexpr int kAdamThreads = SMOE_ADAM_THREADS;

// Adam on one parameter group of a CTA's kernels (N values per kernel):
// gradients in shared memory (gs[e], e = t N + j for kernel k0 + t), `img`
// the kernel's image or -1, `ptr` picks the group's array from a parameter
// set, `ci` its step-size coefficient.
template <int N, typename F>
__device__ __forceinline__ void adam_group(const Geo &g, const Betas &be, const float *coef,
                                           int64_t k0, const int32_t *img, const float *gs,
                                           int ci, F ptr) {
    float pv[N], mv[N], vv[N];
    float *pp[N], *mp[N], *vp[N];
    int bb[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int e = threadIdx.x + i * kAdamThreads;
        const int t = e / N;
        bb[i] = img[t];
        pp[i] = nullptr;
        if (bb[i] >= 0) {
            const ImgDev &im = img_of(g, bb[i]);
            float *base = ptr(im.p);
            if (base) {
                const int64_t x = (k0 + t - im.k_off) * N + (e - t * N);
                pp[i] = base + x;
                mp[i] = ptr(im.m) + x;
                vp[i] = ptr(im.v) + x;
                pv[i] = *pp[i];
                mv[i] = *mp[i];
                vv[i] = *vp[i];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (!pp[i]) continue;
        const float *cf = coef + 8 * bb[i];
        const AdamK kk{be, cf[ci], cf[4]};
        adam1(pv[i], gs[threadIdx.x + i * kAdamThreads], mv[i], vv[i], kk);
        *pp[i] = pv[i];
        *mp[i] = mv[i];
        *vp[i] = vv[i];
    }
}

// Phase 2 for a CTA whose kernels all belong to one running image (base
// pointers uniform): every group's p, m and v values are loaded before any
// is stored, one memory round trip for the whole update.
template <int C, bool LIN>
__device__ __forceinline__ void adam_uniform(const ImgDev &im, const Betas &be, const float *cf,
                                             int64_t kl0, const float *gsm, bool has_pi) {
    constexpr int NW = LIN ? 2 * C : 0;
    constexpr int NT = 2 + 3 + C + NW + 1;                 // values per thread (logpi last)
    const int tid = threadIdx.x;
    float pv[NT], mv[NT], vv[NT];
    // element i of the thread: group, elements per kernel n, index j within it
    auto elem = [&](int i, const smoe_params &q, float *&ptr, int64_t &x) {
        int n, j, base = 0;
        if (i < 2) { ptr = q.mu; n = 2; j = i; }
        else if (i < 5) { ptr = q.chol; n = 3; j = i - 2; base = 2 * kAdamThreads; }
        else if (i < 5 + C) { ptr = q.ea; n = C; j = i - 5; base = 5 * kAdamThreads; }
        else if (i < 5 + C + NW) { ptr = q.eW; n = NW ? NW : 1; j = i - 5 - C; base = (5 + C) * kAdamThreads; }
        else { ptr = q.logpi; n = 1; j = 0; base = (5 + C + NW) * kAdamThreads; }
        const int e = tid + j * kAdamThreads;               // element of the CTA's range
        x = kl0 * n + e;
        return base + e;                                    // its gradient in shared memory
    };
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        float *pp; int64_t x;
        elem(i, im.p, pp, x);
        if (i == NT - 1 && !has_pi) continue;
        float *mp, *vp; int64_t xm, xv;
        elem(i, im.m, mp, xm);
        elem(i, im.v, vp, xv);
        pv[i] = pp[x]; mv[i] = mp[xm]; vv[i] = vp[xv];
    }
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        if (i == NT - 1 && !has_pi) continue;
        float *pp, *mp, *vp; int64_t x, xm, xv;
        const int gi = elem(i, im.p, pp, x);
        elem(i, im.m, mp, xm);
        elem(i, im.v, vp, xv);
        const int ci = i < 2 ? 0 : i < 5 ? 1 : i < 5 + C ? 2 : i < 5 + C + NW ? 3 : 5;
        const AdamK kk{be, cf[ci], cf[4]};
        adam1(pv[i], gsm[gi], mv[i], vv[i], kk);
        pp[x] = pv[i]; mp[xm] = mv[i]; vp[xv] = vv[i];
    }
}

// The gradient of kernel k (global id, image im) in API units, from its raw
// per-kernel sums (the float-atomic sums, or in deterministic mode the
// per-pair partials added in tile order) and its prepared record: the chain
// rule of Eqs. 2-4 (the sums and their formulas are listed in render.cu),
// the centre's gradient in normalised units (x W, x H).  Zeroes the kernel's
// atomic sums for the next iteration.  A kernel listed in no tile touched no
// pixel, so its gradient is exactly 0 (and must not become inf * 0 for
// non-finite parameters).  Adam (k_fit_adam) and the gradient read-out
// (k_fit_grads) both take their gradients from here.
template <int C, bool LIN>
struct KGrad {
    static constexpr int NW = LIN ? 2 * C : 0;
    float mu[2], chol[3], ea[C], eW[NW > 0 ? NW : 1], pi;
};

template <int C, bool LIN>
__device__ __forceinline__ void kernel_grad(const Bufs &w, const ImgDev &im, int64_t k,
                                            KGrad<C, LIN> &o) {
    constexpr int E = LIN ? 3 : 1;
    constexpr int S = (7 + C * E + 3) & ~3;       // record stride (floats)
    constexpr int GS = (6 + C * E + 3) & ~3;      // sums stride (floats)
    constexpr int PI = 5 + C * E;                 // dL/dlogpi slot
    const int4 rc = w.rect[k];
    const bool listed = rc.x <= rc.z;
    float s[GS];
    float4 *acc = reinterpret_cast<float4 *>(w.acc + k * GS);
    if (!listed) {
#pragma unroll
        for (int q = 0; q < GS; ++q) s[q] = 0.0f;
    } else if (w.part) {
        gather_sums<GS>(w, im, k, rc, s);
    } else {
#pragma unroll
        for (int q = 0; q < GS / 4; ++q) {
            const float4 v = acc[q];
            s[4 * q] = v.x; s[4 * q + 1] = v.y; s[4 * q + 2] = v.z; s[4 * q + 3] = v.w;
        }
    }
    float r[S];
    const float4 *rec = reinterpret_cast<const float4 *>(w.rec + k * S);
#pragma unroll
    for (int q = 0; q < S / 4; ++q) {
        const float4 v = rec[q];
        r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
    }
    float gmx = 0.f, gmy = 0.f;
    if (listed) { gmx = r[2] * s[3]; gmy = fmaf(r[3], s[3], r[4] * s[4]); }
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        o.ea[ch] = s[5 + ch];
        if (LIN) {
            if (listed) {
                gmx -= r[7 + ch * E + 1] * s[5 + ch];
                gmy -= r[7 + ch * E + 2] * s[5 + ch];
            }
#pragma unroll
            for (int d = 0; d < 2; ++d) o.eW[2 * ch + d] = s[5 + (1 + d) * C + ch];
        }
    }
    o.mu[0] = gmx * (float)im.W;
    o.mu[1] = gmy * (float)im.H;
#pragma unroll
    for (int d = 0; d < 3; ++d) o.chol[d] = -s[d];
    o.pi = s[PI];                                 // dL/dlogpi = S0
    if (!w.part && listed)     // an unlisted kernel's sums received nothing: still 0
#pragma unroll
        for (int q = 0; q < GS / 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int C, bool LIN>
__global__ void __launch_bounds__(kAdamThreads, 2)
k_fit_adam(const __grid_constant__ Geo g, Bufs w, double b1, double b2, Betas be, int32_t *step,
           uint32_t *done, float *coef) {
    constexpr int NW = LIN ? 2 * C : 0;           // slopes per kernel
    // gradient groups in shared memory: mu (2), chol (3), ea (C), eW (2C), logpi (1)
    constexpr int O_MU = 0, O_CH = O_MU + 2 * kAdamThreads, O_EA = O_CH + 3 * kAdamThreads;
    constexpr int O_EW = O_EA + C * kAdamThreads, O_PI = O_EW + NW * kAdamThreads;
    __shared__ float gsm[O_PI + kAdamThreads];
    __shared__ int32_t kimg[kAdamThreads];        // the kernel's image, -1: nothing to update
    __shared__ bool last;
    if (status_bad(w.status)) return;
    const int tid = threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.x * kAdamThreads;
    const int64_t k = k0 + tid;
    {
        int bk = -1;
        if (k < g.K_total) {
            const int b = img_by_kernel(g, k);
            if (step[b] < img_of(g, b).iters) bk = b;
        }
        kimg[tid] = bk;
        if (bk >= 0) {
            KGrad<C, LIN> kg;
            kernel_grad<C, LIN>(w, img_of(g, bk), k, kg);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                gsm[O_EA + tid * C + ch] = kg.ea[ch];
                if (LIN)
#pragma unroll
                    for (int d = 0; d < 2; ++d) gsm[O_EW + tid * NW + 2 * ch + d] = kg.eW[2 * ch + d];
            }
            gsm[O_MU + 2 * tid] = kg.mu[0];
            gsm[O_MU + 2 * tid + 1] = kg.mu[1];
#pragma unroll
            for (int d = 0; d < 3; ++d) gsm[O_CH + 3 * tid + d] = kg.chol[d];
            gsm[O_PI + tid] = kg.pi;
        }
    }
    // One image for the whole CTA (and it is running): the single-round-trip update.
    const int b0 = kimg[0];
    if (__syncthreads_and(kimg[tid] == b0 && b0 >= 0)) {
        const ImgDev &im = img_of(g, b0);
        adam_uniform<C, LIN>(im, be, coef + 8 * b0, k0 - im.k_off, gsm, im.p.logpi != nullptr);
    } else {
    // Phase 2: group by group, element e of the CTA's range is parameter
    // e % N of kernel k0 + e / N; a thread loads its N elements of p, m and v
    // before it stores any.
    adam_group<2>(g, be, coef, k0, kimg, gsm + O_MU, 0, [](const smoe_params &q) { return q.mu; });
    adam_group<3>(g, be, coef, k0, kimg, gsm + O_CH, 1, [](const smoe_params &q) { return q.chol; });
    adam_group<C>(g, be, coef, k0, kimg, gsm + O_EA, 2, [](const smoe_params &q) { return q.ea; });
    if (LIN)
        adam_group<NW ? NW : 1>(g, be, coef, k0, kimg, gsm + O_EW, 3,
                                [](const smoe_params &q) { return q.eW; });
    adam_group<1>(g, be, coef, k0, kimg, gsm + O_PI, 5, [](const smoe_params &q) { return q.logpi; });
    }
    // Step counters advance once every CTA has read them.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(done, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        for (int b = threadIdx.x; b < g.B; b += blockDim.x)
            if (step[b] < img_of(g, b).iters) step[b] += 1;
        __syncthreads();
        adam_coefs(g, step, b1, b2, coef);
        if (threadIdx.x == 0) *done = 0u;
        __threadfence();
    }
}

// Gradient read-out of the fit: the gradients that k_fit_adam would apply
// this iteration (same sums, same kernel_grad), written to the caller's
// arrays at the kernel's global (batch) index instead of stepping Adam.
// Kernels of an image whose run has ended get 0 (its tiles were skipped).
template <int C, bool LIN>
__global__ void __launch_bounds__(kAdamThreads)
k_fit_grads(const __grid_constant__ Geo g, Bufs w, const int32_t *step, smoe_params grad) {
    constexpr int NW = LIN ? 2 * C : 0;
    if (status_bad(w.status)) return;
    const int64_t k = (int64_t)blockIdx.x * kAdamThreads + threadIdx.x;
    if (k >= g.K_total) return;
    const int b = img_by_kernel(g, k);
    const ImgDev &im = img_of(g, b);
    KGrad<C, LIN> kg{};
    if (step[b] < im.iters) kernel_grad<C, LIN>(w, im, k, kg);
    grad.mu[2 * k] = kg.mu[0];
    grad.mu[2 * k + 1] = kg.mu[1];
#pragma unroll
    for (int d = 0; d < 3; ++d) grad.chol[3 * k + d] = kg.chol[d];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) grad.ea[k * C + ch] = kg.ea[ch];
    if (LIN)
#pragma unroll
        for (int i = 0; i < NW; ++i) grad.eW[k * NW + i] = kg.eW[i];
    if (grad.logpi) grad.logpi[k] = kg.pi;
}

__global__ void k_sq_error(const float *y, const float *t, int64_t n, int clamp, double *out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = y[i];
        if (clamp) v = fminf(fmaxf(v, 0.0f), 1.0f);
        const double d = (double)v - (double)t[i];
        s += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += ws[i];
        atomicAdd(out, a);
    }
}

}  // namespace

cudaError_t launch_adam_soa(const smoe_params &p, const smoe_params &gr, const smoe_params &m,
                            const smoe_params &v, int C, const float lr[5], double b1, double b2,
                            double eps, int32_t step, cudaStream_t st) {
    const int has_w = p.eW != nullptr;
    const int has_pi = p.logpi != nullptr;
    const int64_t total = p.K * (5 + (int64_t)C * (has_w ? 3 : 1) + has_pi);
    if (total == 0) return cudaSuccess;
    const double bc1 = 1.0 - std::pow((double)b1, (double)step);
    const double isb2 = 1.0 / std::sqrt(1.0 - std::pow((double)b2, (double)step));
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    const Betas be{(float)b2, (float)(1.0 - b1), (float)(1.0 - b2), (float)eps};
    k_adam_soa<<<(unsigned)blocks, 256, 0, st>>>(p.K, C, has_w, has_pi, p, gr, m, v, lr[0],
                                                 lr[1], lr[2], lr[3], lr[4], be, (float)bc1,
                                                 (float)isb2);
    return cudaGetLastError();
}

cudaError_t launch_fit_adam(const Geo &g, const Bufs &w, double b1, double b2, double eps,
                            int32_t *step, uint32_t *done, float *coef, cudaStream_t st) {
    const unsigned blocks = (unsigned)((g.K_total + kAdamThreads - 1) / kAdamThreads);
    if (blocks == 0) return cudaSuccess;
    const Betas be{(float)b2, (float)(1.0 - b1), (float)(1.0 - b2), (float)eps};
    if (g.C == 1 && !g.linear) k_fit_adam<1, false><<<blocks, kAdamThreads, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    else if (g.C == 1) k_fit_adam<1, true><<<blocks, kAdamThreads, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    else if (!g.linear) k_fit_adam<3, false><<<blocks, kAdamThreads, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    else k_fit_adam<3, true><<<blocks, kAdamThreads, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    return cudaGetLastError();
}

cudaError_t launch_fit_grads(const Geo &g, const Bufs &w, const int32_t *step,
                             const smoe_params &grad, cudaStream_t st) {
    const unsigned blocks = (unsigned)((g.K_total + kAdamThreads - 1) / kAdamThreads);
    if (blocks == 0) return cudaSuccess;
    if (g.C == 1 && !g.linear) k_fit_grads<1, false><<<blocks, kAdamThreads, 0, st>>>(g, w, step, grad);
    else if (g.C == 1) k_fit_grads<1, true><<<blocks, kAdamThreads, 0, st>>>(g, w, step, grad);
    else if (!g.linear) k_fit_grads<3, false><<<blocks, kAdamThreads, 0, st>>>(g, w, step, grad);
    else k_fit_grads<3, true><<<blocks, kAdamThreads, 0, st>>>(g, w, step, grad);
    return cudaGetLastError();
}

cudaError_t launch_adam_coefs(const Geo &g, const int32_t *step, double b1, double b2,
                              float *coef, cudaStream_t st) {
    k_adam_coefs<<<1, 256, 0, st>>>(g, step, b1, b2, coef);
    return cudaGetLastError();
}

cudaError_t launch_sq_error(const float *y, const float *t, int64_t n, int clamp, double *out,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_sq_error<<<(unsigned)blocks, 256, 0, st>>>(y, t, n, clamp, out);
    return cudaGetLastError();
}

}  // namespace smoe
