// Arithmetic-rate probe: the roofline denominators of the ALU-bound kernels (FP32 FMA, packed
// FP32 FMA, the MUFU reciprocal square root, FP64 FMA), measured on the running device at
// its current clocks with CUDA events.  Not part of the paper's method: a measurement
// utility, so that the FP32 fractions reported beside the HMM and all-pairs kernels are
// fractions of a measured rate, not of a nominal one.
//
// Each thread runs kChains independent dependency chains (enough instruction-level
// parallelism to cover the pipe latency at 8 warps per scheduler) for `iters` rounds; the
// grid is 4 CTAs of 512 threads per SM.  The chains' results are written out so that
// nothing is removed by the compiler.
#include "common.cuh"

#include <cuda_fp16.h>

namespace accel {
namespace probe {

constexpr int kThreads = 512;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) k_ffma(int64_t iters, float a, float b, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_ffma2(int64_t iters, float a, float b, float* out) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_rsqrt(int64_t iters, float a, float b, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = rsqrtf(x[c]);   // converges to 1: stays finite
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s + a * b;
}

__global__ void __launch_bounds__(kThreads) k_dfma(int64_t iters, float a, float b, float* out) {
    double x[kChains];
    const double da = a, db = b;
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], da, db);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kThreads + threadIdx.x] = (float)s;
}

}  // namespace probe
}  // namespace accel

using namespace accel;

extern "C" accel_status accel_alu_rate(int32_t kind, int64_t iters, float* d_scratch, double* h_rate, void* stream) {
    ACCEL_REQUIRE(kind >= ACCEL_PROBE_FFMA && kind <= ACCEL_PROBE_DFMA, ACCEL_ERR_INVALID_ARG,
                  "accel_alu_rate: bad kind %d", kind);
    ACCEL_REQUIRE(iters >= 1 && d_scratch && h_rate, ACCEL_ERR_INVALID_ARG, "accel_alu_rate: bad argument");
    cudaStream_t st = as_stream(stream);
    const int grid = 4 * num_sms();
    auto kern = kind == ACCEL_PROBE_FFMA ? probe::k_ffma
              : kind == ACCEL_PROBE_FFMA2 ? probe::k_ffma2
              : kind == ACCEL_PROBE_RSQRT ? probe::k_rsqrt : probe::k_dfma;
    // operations per inner step of one chain: an FMA is 2 flop, a packed FMA 4, a rsqrt 1
    const double per = kind == ACCEL_PROBE_FFMA2 ? 4.0 : kind == ACCEL_PROBE_RSQRT ? 1.0 : 2.0;
    const float a = 0.999999f, b = 1e-7f;
    kern<<<grid, probe::kThreads, 0, st>>>(1, a, b, d_scratch);         // warm-up (clocks, caches)
    cudaEvent_t e0, e1;
    ACCEL_CUDA_TRY(cudaEventCreate(&e0));
    ACCEL_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    kern<<<grid, probe::kThreads, 0, st>>>(iters, a, b, d_scratch);
    cudaEventRecord(e1, st);
    count_launches(2);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(ACCEL_ERR_CUDA, "accel_alu_rate: %s", cudaGetErrorString(e));
    const double ops = (double)grid * probe::kThreads * probe::kChains * 8.0 * (double)iters * per;
    *h_rate = ops / (ms * 1e-3);
    return ok();
}
