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

__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, const AdamK &k) {
    m = fmaf(k.be.omb1, g - m, m);
    v = fmaf(k.be.b2, v, k.be.omb2 * g * g);
    const float denom = sqrtf(v) * k.inv_sqrt_bc2 + k.be.eps;
    p -= k.step_size * (m / denom);
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

// Per-image Adam coefficients of the current step, formed in FP64 and rounded
// once: the four step sizes lr_g / (1 - b1^t) (the centre rate follows the
// exponential schedule) and 1 / sqrt(1 - b2^t).  Threads stride over images.
__device__ void adam_coefs(const Geo &g, const int32_t *step, double b1, double b2,
                           float *coef) {
    for (int b = threadIdx.x; b < g.B; b += blockDim.x) {
        const ImgDev &im = img_of(g, b);
        const int32_t it = step[b];
        const double t = (double)(it + 1);
        const double bc1 = 1.0 - pow(b1, t);
        const double f = im.iters > 1 ? (double)it / (double)(im.iters - 1) : 0.0;
        const double lr_mu =
            im.lr_mu0 > 0.0f ? (double)im.lr_mu0 * pow((double)im.lr_mu1 / im.lr_mu0, f) : 0.0;
        float *c = coef + 8 * b;
        c[0] = (float)(lr_mu / bc1);
        c[1] = (float)(im.lr_chol / bc1);
        c[2] = (float)(im.lr_ea / bc1);
        c[3] = (float)(im.lr_eW / bc1);
        c[4] = (float)(1.0 / sqrt(1.0 - pow(b2, t)));
        c[5] = (float)(im.lr_pi / bc1);
    }
}

__global__ void k_adam_coefs(const __grid_constant__ Geo g, const int32_t *step, double b1,
                             double b2, float *coef) {
    adam_coefs(g, step, b1, b2, coef);
}

// Fit: raw per-kernel sums -> gradients (see render.cu) -> Adam on the 5 + C
// (+ 2C, + 1 with gate weights) parameters of the kernel; zeroes the sums.
// The sums and the prepared record are loaded whole (float4) into registers.
// The last CTA to finish advances every running image's step counter and
// forms the coefficients of the next step.
template <int C, bool LIN>
__global__ void k_fit_adam(const __grid_constant__ Geo g, Bufs w, double b1, double b2,
                           Betas be, int32_t *step, uint32_t *done, float *coef) {
    constexpr int E = LIN ? 3 : 1;
    constexpr int S = (7 + C * E + 3) & ~3;       // record stride (floats)
    constexpr int GS = (6 + C * E + 3) & ~3;      // sums stride (floats)
    constexpr int PI = 5 + C * E;                 // dL/dlogpi slot
    if (status_bad(w.status)) return;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < g.K_total) {
        const int b = img_by_kernel(g, k);
        const ImgDev &im = img_of(g, b);
        const int32_t it = step[b];
        if (it < im.iters) {
            const int64_t kl = k - im.k_off;
            // A kernel listed in no tile touched no pixel: its gradient is 0
            // (and must not become inf * 0 for non-finite parameters).
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
            const float *cf = coef + 8 * b;
            const float isb2 = cf[4];
            const AdamK kmu{be, cf[0], isb2}, kch{be, cf[1], isb2}, kea{be, cf[2], isb2};
            const AdamK kew{be, cf[3], isb2}, kpi{be, cf[5], isb2};
            float gmx = 0.f, gmy = 0.f;
            if (listed) { gmx = r[2] * s[3]; gmy = fmaf(r[3], s[3], r[4] * s[4]); }
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const int64_t x = kl * C + ch;
                float pv = im.p.ea[x], mv = im.m.ea[x], vv = im.v.ea[x];
                adam1(pv, s[5 + ch], mv, vv, kea);
                im.p.ea[x] = pv; im.m.ea[x] = mv; im.v.ea[x] = vv;
                if (LIN) {
                    if (listed) {
                        gmx -= r[7 + ch * E + 1] * s[5 + ch];
                        gmy -= r[7 + ch * E + 2] * s[5 + ch];
                    }
#pragma unroll
                    for (int d = 0; d < 2; ++d) {
                        const int64_t xw = x * 2 + d;
                        float pw = im.p.eW[xw], mw = im.m.eW[xw], vw = im.v.eW[xw];
                        adam1(pw, s[5 + (1 + d) * C + ch], mw, vw, kew);
                        im.p.eW[xw] = pw; im.m.eW[xw] = mw; im.v.eW[xw] = vw;
                    }
                }
            }
            const float gm[2] = {gmx * (float)im.W, gmy * (float)im.H};
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                float pv = im.p.mu[2 * kl + d], mv = im.m.mu[2 * kl + d], vv = im.v.mu[2 * kl + d];
                adam1(pv, gm[d], mv, vv, kmu);
                im.p.mu[2 * kl + d] = pv; im.m.mu[2 * kl + d] = mv; im.v.mu[2 * kl + d] = vv;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float pv = im.p.chol[3 * kl + d], mv = im.m.chol[3 * kl + d];
                float vv = im.v.chol[3 * kl + d];
                adam1(pv, -s[d], mv, vv, kch);
                im.p.chol[3 * kl + d] = pv; im.m.chol[3 * kl + d] = mv; im.v.chol[3 * kl + d] = vv;
            }
            if (im.p.logpi) {                              // gate weight: dL/dlogpi = S0
                float pv = im.p.logpi[kl], mv = im.m.logpi[kl], vv = im.v.logpi[kl];
                adam1(pv, s[PI], mv, vv, kpi);
                im.p.logpi[kl] = pv; im.m.logpi[kl] = mv; im.v.logpi[kl] = vv;
            }
            if (!w.part && listed)     // an unlisted kernel's sums received nothing: still 0
#pragma unroll
                for (int q = 0; q < GS / 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // Step counters advance once every CTA has read them.
    __shared__ bool last;
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
    const unsigned blocks = (unsigned)((g.K_total + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    const Betas be{(float)b2, (float)(1.0 - b1), (float)(1.0 - b2), (float)eps};
    if (g.C == 1 && !g.linear) k_fit_adam<1, false><<<blocks, 256, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    else if (g.C == 1) k_fit_adam<1, true><<<blocks, 256, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    else if (!g.linear) k_fit_adam<3, false><<<blocks, 256, 0, st>>>(g, w, b1, b2, be, step, done, coef);
    else k_fit_adam<3, true><<<blocks, 256, 0, st>>>(g, w, b1, b2, be, step, done, coef);
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
