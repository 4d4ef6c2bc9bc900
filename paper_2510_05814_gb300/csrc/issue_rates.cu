// Issue-rate micro-benchmark (libsmoe_rates.so, separate from libsmoe.so):
// lane operations per clock per SM of the three instruction kinds the tile
// kernels are made of -- MUFU ex2.approx, scalar FFMA and packed
// fma.rn.f32x2 -- measured with clock64 on a full grid of independent
// dependency chains (8 chains per thread, 2048 threads per SM).  It gives
// the ALU roofline of the tile kernels its per-clock peaks.
#include <cuda_runtime.h>

#include <vector>

namespace {

constexpr int kIters = 4096;
constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Each thread writes one float of `out` (grid x block entries) and thread 0
// of each block its cycle count; nothing else is written.
__global__ void __launch_bounds__(kThreads) k_rate_ex2(float *out, float seed, long long *cyc) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = seed * (float)(i + 1) * 1e-3f;
    const long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = ex2_approx(-x[i]);
    }
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) k_rate_ffma(float *out, float seed, long long *cyc) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = seed * (float)(i + 1);
    const long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __fmaf_rn(x[i], 0.999f, 1e-3f);
    }
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) k_rate_ffma2(float *out, float seed, long long *cyc) {
    float2 x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = make_float2(seed * (float)(i + 1), seed * (float)(i + 2));
    const float2 a = make_float2(0.999f, 0.999f), b = make_float2(1e-3f, 1e-3f);
    const long long t0 = clock64();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a, b);
    }
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

}  // namespace

// out[0..2]: ex2, FFMA, packed f32x2 FMA lane operations per clock per SM
// (the best of three repetitions); clock_mhz: the SM clock the ex2 run
// implies (cycles / elapsed time).  Returns 0, or the CUDA error code.
extern "C" __attribute__((visibility("default"))) int smoe_issue_rates(double *out,
                                                                        double *clock_mhz) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 8;
    void (*kernels[3])(float *, float, long long *) = {k_rate_ex2, k_rate_ffma, k_rate_ffma2};
    for (auto k : kernels) {
        int r = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k, kThreads, 0)) != cudaSuccess)
            return (int)e;
        if (r < per_sm) per_sm = r;
    }
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    const int blocks = sms * per_sm;                // every block resident at once
    float *d_out = nullptr;
    long long *d_cyc = nullptr;
    if ((e = cudaMalloc(&d_out, sizeof(float) * blocks * kThreads)) != cudaSuccess) return (int)e;
    if ((e = cudaMalloc(&d_cyc, sizeof(long long) * blocks)) != cudaSuccess) {
        cudaFree(d_out);
        return (int)e;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<long long> cyc(blocks);
    const double lanes[3] = {1.0, 1.0, 2.0};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        double best = 0.0;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0);
            kernels[k]<<<blocks, kThreads>>>(d_out, 1.0f, d_cyc);
            cudaEventRecord(e1);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpy(cyc.data(), d_cyc, sizeof(long long) * blocks,
                                cudaMemcpyDeviceToHost)) != cudaSuccess)
                break;
            long long mc = 1;
            for (long long c : cyc) mc = c > mc ? c : mc;
            const double ops = (double)blocks * kThreads * kIters * kChains * lanes[k];
            const double rate = ops / sms / (double)mc;
            if (rate > best) {
                best = rate;
                if (k == 0 && clock_mhz) {
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    *clock_mhz = (double)mc / (ms * 1e3);
                }
            }
        }
        out[k] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    cudaFree(d_cyc);
    return (int)e;
}
