// palmad_measure_peak: arithmetic throughput of this GPU's FP32 and FP64
// pipes, the denominator of the pair kernels' roofline (they are bound by
// FP32 arithmetic, not by memory).  Every thread runs kChains independent
// fused multiply-add chains, so the pipe, not latency, limits the rate; the
// grid fills every SM with 32 warps.  The rate is the best of several timed
// launches (CUDA events on a private stream) after one warm-up launch.
#include "palmad.h"
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long pack2(float x, float y) {
    return (static_cast<unsigned long long>(__float_as_uint(y)) << 32) | __float_as_uint(x);
}

// x <- x*a + b keeps every chain finite and non-constant (|a| < 1).
__global__ void __launch_bounds__(kThreads) k_peak_f32(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = float(threadIdx.x + c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_peak_f32x2(float* out, int iters, float a, float b) {
    unsigned long long x[kChains];
    const unsigned long long av = pack2(a, a), bv = pack2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = pack2(float(threadIdx.x + c), float(c));
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma_f32x2(x[c], av, bv);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += __uint_as_float(unsigned(x[c])) + __uint_as_float(unsigned(x[c] >> 32));
    if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f64(float* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = double(threadIdx.x + c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5) out[blockIdx.x] = float(s);
}

}  // namespace

}  // namespace palmad

extern "C" palmad_status palmad_measure_peak(int device, int32_t kind, double* tflops) {
    using namespace palmad;
    if (!tflops || kind < PALMAD_PEAK_FP32 || kind > PALMAD_PEAK_FP64) return PALMAD_ERR_ARG;
    *tflops = 0.0;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PALMAD_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = sms * kBlocksPerSm;
    // FP64 runs far slower on this part: fewer iterations keep a launch short
    const int iters = kind == PALMAD_PEAK_FP64 ? 512 : 16384;
    float* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    palmad_status st = PALMAD_OK;
    float best = 0.f;
    if (cudaMalloc(&out, sizeof(float) * grid) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = PALMAD_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 6 && st == PALMAD_OK; ++rep) {
            cudaEventRecord(e0, s);
            if (kind == PALMAD_PEAK_FP32) k_peak_f32<<<grid, kThreads, 0, s>>>(out, iters, 0.999f, 0.001f);
            else if (kind == PALMAD_PEAK_FP32X2) k_peak_f32x2<<<grid, kThreads, 0, s>>>(out, iters, 0.999f, 0.001f);
            else k_peak_f64<<<grid, kThreads, 0, s>>>(out, iters, 0.999, 0.001);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                st = PALMAD_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;  // rep 0 warms up
        }
    }
    if (st == PALMAD_OK && best > 0.f) {
        const double lanes = kind == PALMAD_PEAK_FP32X2 ? 2.0 : 1.0;
        const double flops = 2.0 * lanes * kChains * double(iters) * double(grid) * kThreads;
        *tflops = flops / (double(best) * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    cudaGetLastError();
    cudaSetDevice(prev);
    return st;
}
