// sigkernel_fma_peak: the FP32 / FP64 multiply-add throughput of the current GPU, measured with
// independent FMA chains.  The paper has no counterpart: the roofline fractions the library's
// benchmark reports for its ALU-bound wavefront kernels divide by this measured figure instead of
// a peak derived from unit counts and the nominal clock.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/sigkernel.h"
#include "sk_dispatch.h"

namespace {

constexpr int kThreads = 384;  // 4 blocks of 12 warps per SM: 48 resident warps

// Sink of the chains' final values, so that the compiler keeps every FMA.
__device__ double g_peak_sink;

// Scalar chains: each thread runs C independent recurrences v <- v * m + c (|m| < 1, so the
// values stay normal and bounded), `iters` times.
template <typename T, int C>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T m, T c) {
    T v[C];
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = static_cast<T>(threadIdx.x + k) * static_cast<T>(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < C; ++k) v[k] = fma(v[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < C; ++k) s += v[k];
    if (s == static_cast<T>(-1.0)) g_peak_sink = static_cast<double>(s);  // never true: keeps the chains live
}

// The same with packed pairs through the two-wide FP32 instruction (two FMAs per instruction).
template <int C>
__global__ void __launch_bounds__(kThreads) ffma2_chain_kernel(int iters, float m, float c) {
    float2 v[C];
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = make_float2((threadIdx.x + k) * 1e-3f, (threadIdx.x + k + C) * 1e-3f);
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < C; ++k) v[k] = __ffma2_rn(v[k], m2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < C; ++k) s += v[k].x + v[k].y;
    if (s == -1.0f) g_peak_sink = static_cast<double>(s);
}

int peak_fail(int code, const char* what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "sigkernel_fma_peak: %s: %s", what, cudaGetErrorString(e));
    sk::set_last_error(buf);
    return code;
}

}  // namespace

extern "C" {

int sigkernel_fma_peak(int32_t compute, int32_t packed, int32_t reps, double* tflops, void* stream) {
    sk::set_last_error("");
    if (!tflops || reps < 1 || reps > 100 || (compute != SK_COMPUTE_F32 && compute != SK_COMPUTE_F64) ||
        (packed && compute != SK_COMPUTE_F32)) {
        sk::set_last_error("sigkernel_fma_peak: bad argument");
        return SK_ERR_INVALID_ARG;
    }
    *tflops = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return peak_fail(SK_ERR_CUDA, "cudaGetDevice", e);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return peak_fail(SK_ERR_CUDA, "cudaDeviceGetAttribute", e);
    const int blocks = sms * 4;
    // chains per thread and iterations: a few milliseconds per launch at the expected rates
    constexpr int kC32 = 16, kC64 = 8;
    const int iters = compute == SK_COMPUTE_F32 ? 32768 : 2048;
    const double fmas = static_cast<double>(blocks) * kThreads * iters *
                        (compute == SK_COMPUTE_F32 ? (packed ? 2.0 * (kC32 / 2) : kC32) : kC64);
    auto launch = [&]() {
        if (compute == SK_COMPUTE_F64) fma_chain_kernel<double, kC64><<<blocks, kThreads, 0, st>>>(iters, 0.9999, 1e-4);
        else if (packed) ffma2_chain_kernel<kC32 / 2><<<blocks, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f);
        else fma_chain_kernel<float, kC32><<<blocks, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f);
        return cudaGetLastError();
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return peak_fail(SK_ERR_CUDA, "cudaEventCreate", e);
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return peak_fail(SK_ERR_CUDA, "cudaEventCreate", e);
    }
    float best = -1.f;
    int rc = SK_OK;
    for (int r = 0; r <= reps && rc == SK_OK; ++r) {  // r = 0 warms up
        float ms = 0.f;
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess || (e = launch()) != cudaSuccess ||
            (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            rc = peak_fail(SK_ERR_CUDA, "timed launch", e);
            break;
        }
        if (r > 0 && (best < 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SK_OK) return rc;
    *tflops = 2.0 * fmas / (static_cast<double>(best) * 1e-3) / 1e12;
    return SK_OK;
}

}  // extern "C"
