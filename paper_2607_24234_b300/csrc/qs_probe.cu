// qs_probe.cu -- arithmetic-rate probes (qs_probe_alu, see qs.h).
//
// The resident and Green's-function sweeps are bound by FP32 arithmetic and
// the FP64 sweep by FP64 arithmetic, not by HBM.  Their roofline fractions
// need the rate the GPU at hand actually sustains, so these kernels measure
// it: every thread runs NC independent dependent chains of fused multiply-
// adds (x <- x * b + c), long enough that the launch lasts about a second.
// The chains keep each scheduler's pipe full (NC in flight per thread, many
// warps per SM); nothing else is issued in the loop.
//
// Counting: an FMA on one value is one "lane-op"; a packed f32x2 FMA
// (__ffma2_rn) is two.  This is the unit of the sweep's algorithmic op count.
#include <cuda_runtime.h>

#include <cstdint>

#include "qs.h"

namespace {

constexpr int NC = 8;   // independent chains per thread

// The result is stored only if it has one particular NaN bit pattern, which
// the chains never produce; the compiler cannot prove that, so the
// arithmetic stays.
__global__ void __launch_bounds__(256) k_probe_ffma2(long long iters, float *sink) {
    float2 x[NC];
    const float t = 1e-3f * (float)(threadIdx.x + 1);
#pragma unroll
    for (int k = 0; k < NC; ++k) x[k] = make_float2(t + k, t - k);
    const float2 b = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, -1e-7f);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NC; ++k) x[k] = __ffma2_rn(x[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NC; ++k) s += x[k].x + x[k].y;
    if (__float_as_uint(s) == 0x7fc0dead) sink[0] = s;
}

__global__ void __launch_bounds__(256) k_probe_ffma(long long iters, float *sink) {
    float x[2 * NC];
    const float t = 1e-3f * (float)(threadIdx.x + 1);
#pragma unroll
    for (int k = 0; k < 2 * NC; ++k) x[k] = t + k;
    const float b = 0.9999999f, c = 1e-7f;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 2 * NC; ++k) x[k] = __fmaf_rn(x[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 2 * NC; ++k) s += x[k];
    if (__float_as_uint(s) == 0x7fc0dead) sink[0] = s;
}

__global__ void __launch_bounds__(256) k_probe_dfma(long long iters, double *sink) {
    double x[NC];
    const double t = 1e-3 * (double)(threadIdx.x + 1);
#pragma unroll
    for (int k = 0; k < NC; ++k) x[k] = t + k;
    const double b = 0.9999999999, c = 1e-10;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NC; ++k) x[k] = __fma_rn(x[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NC; ++k) s += x[k];
    if (__double_as_longlong(s) == 0x7ff8deaddeadbeefLL) sink[0] = s;
}

// FP64 add and multiply chains (the FP64 sweep issues 16 FMA, 4 MUL and 2
// ADD per update; these show whether the latter issue at the FMA rate)
__global__ void __launch_bounds__(256) k_probe_dadd(long long iters, double *sink) {
    double x[NC];
    const double t = 1e-3 * (double)(threadIdx.x + 1);
#pragma unroll
    for (int k = 0; k < NC; ++k) x[k] = t + k;
    const double c = 1e-12;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NC; ++k) x[k] = __dadd_rn(x[k], c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NC; ++k) s += x[k];
    if (__double_as_longlong(s) == 0x7ff8deaddeadbeefLL) sink[0] = s;
}

__global__ void __launch_bounds__(256) k_probe_dmul(long long iters, double *sink) {
    double x[NC];
    const double t = 1e-3 * (double)(threadIdx.x + 1);
#pragma unroll
    for (int k = 0; k < NC; ++k) x[k] = t + k;
    const double b = 0.9999999999;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NC; ++k) x[k] = __dmul_rn(x[k], b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NC; ++k) s += x[k];
    if (__double_as_longlong(s) == 0x7ff8deaddeadbeefLL) sink[0] = s;
}

}  // namespace

extern "C" qs_status qs_probe_alu(int kind, int blocks, int threads, int64_t iters, void *dev_sink,
                                  void *stream, double *lane_ops) {
    if (kind < 0 || kind > 4 || blocks < 1 || threads < 32 || threads > 256 || threads % 32 || iters < 1 ||
        !dev_sink)
        return QS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double per_iter = kind == QS_PROBE_FFMA2 ? 2.0 * NC : kind == QS_PROBE_FFMA ? 2.0 * NC : 1.0 * NC;
    if (kind == QS_PROBE_FFMA2)
        k_probe_ffma2<<<blocks, threads, 0, s>>>(iters, static_cast<float *>(dev_sink));
    else if (kind == QS_PROBE_FFMA)
        k_probe_ffma<<<blocks, threads, 0, s>>>(iters, static_cast<float *>(dev_sink));
    else if (kind == QS_PROBE_DFMA)
        k_probe_dfma<<<blocks, threads, 0, s>>>(iters, static_cast<double *>(dev_sink));
    else if (kind == QS_PROBE_DADD)
        k_probe_dadd<<<blocks, threads, 0, s>>>(iters, static_cast<double *>(dev_sink));
    else
        k_probe_dmul<<<blocks, threads, 0, s>>>(iters, static_cast<double *>(dev_sink));
    if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
    if (lane_ops) *lane_ops = per_iter * (double)iters * (double)blocks * (double)threads;
    return QS_OK;
}
