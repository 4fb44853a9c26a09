// Re-estimation after the adjoint: the softmax-parameterised gradient and the Baum-Welch
// M-step of every parameter row (textbook; the paper has no HMM).  Its shape is the paper's
// map of a reduce (Appendix A): a map over the rows of (reductions over the row, then a map
// over the row).
//
// Rows: r < K is row r of A (length K), K <= r < 2K row r-K of B (length M), r = 2K is pi
// (length K).  g is the gradient with respect to log P read as free parameters (the expected
// counts hmm_adjoint returns).  One warp per row; the row's sums are accumulated in FP64, the
// per-element exp and log in FP32 (each result is one FP32 rounding from its FP64 value up to
// the few-ulp error of expf / logf):
//   P_j      = exp(logP_j - max) / sum_j' exp(logP_j' - max)       (softmax of the row)
//   gtheta_j = g_j - P_j * sum_j' g_j'                              (P = softmax(theta))
//   newlog_j = log g_j - log sum_j' g_j'   (a row with zero count sum keeps logP_j)
#include "common.cuh"
#include "hmm_internal.cuh"

#include <math.h>

namespace accel {
namespace hmm {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    return v;
}

__global__ void __launch_bounds__(kThreads)
k_mstep(int K, int M, const float* __restrict__ logA, const float* __restrict__ logB, const float* __restrict__ logpi,
        const float* __restrict__ gA, const float* __restrict__ gB, const float* __restrict__ gpi,
        float* __restrict__ tA, float* __restrict__ tB, float* __restrict__ tpi,
        float* __restrict__ nA, float* __restrict__ nB, float* __restrict__ npi) {
    const int row = (int)((blockIdx.x * (unsigned)kThreads + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (row > 2 * K) return;                      // the whole warp
    const float *lp, *g;
    float *to, *no;
    int n;
    if (row < K) {
        const size_t o = (size_t)row * K;
        n = K; lp = logA + o; g = gA + o; to = tA ? tA + o : nullptr; no = nA ? nA + o : nullptr;
    } else if (row < 2 * K) {
        const size_t o = (size_t)(row - K) * M;
        n = M; lp = logB + o; g = gB + o; to = tB ? tB + o : nullptr; no = nB ? nB + o : nullptr;
    } else {
        n = K; lp = logpi; g = gpi; to = tpi; no = npi;
    }
    double mx = -INFINITY, gs = 0.0;
    for (int j = lane; j < n; j += 32) {
        mx = fmax(mx, (double)lp[j]);
        gs += (double)g[j];
    }
    mx = warp_max(mx);
    gs = warp_sum(gs);
    const float mxf = (float)mx;                  // the row's largest entry, exactly
    if (to) {
        double es = 0.0;
        for (int j = lane; j < n; j += 32) es += (double)expf(lp[j] - mxf);
        es = warp_sum(es);
        const double scale = gs / es;
        for (int j = lane; j < n; j += 32) to[j] = (float)((double)g[j] - (double)expf(lp[j] - mxf) * scale);
    }
    if (no) {
        const double lgs = log(gs);
        for (int j = lane; j < n; j += 32) no[j] = gs > 0.0 ? (float)((double)logf(g[j]) - lgs) : lp[j];
    }
}

}  // namespace

accel_status check_model(const accel_hmm_model* m, const char* who);

}  // namespace hmm
}  // namespace accel

using namespace accel;
using namespace accel::hmm;

extern "C" {

accel_status hmm_mstep(const accel_hmm_model* m, const float* d_grad_log_A, const float* d_grad_log_B,
                       const float* d_grad_log_pi, float* d_grad_theta_A, float* d_grad_theta_B,
                       float* d_grad_theta_pi, float* d_new_log_A, float* d_new_log_B, float* d_new_log_pi,
                       void* stream) {
    accel_status r = check_model(m, "hmm_mstep");
    if (r != ACCEL_OK) return r;
    ACCEL_REQUIRE(d_grad_log_A && d_grad_log_B && d_grad_log_pi, ACCEL_ERR_INVALID_ARG, "hmm_mstep: null gradient");
    const int K = m->K, M = m->M;
    const int64_t warps = 2 * (int64_t)K + 1;
    const int blocks = (int)((warps * 32 + kThreads - 1) / kThreads);
    cudaStream_t st = as_stream(stream);
    k_mstep<<<blocks, kThreads, 0, st>>>(K, M, m->log_A, m->log_B, m->log_pi, d_grad_log_A, d_grad_log_B,
                                         d_grad_log_pi, d_grad_theta_A, d_grad_theta_B, d_grad_theta_pi, d_new_log_A,
                                         d_new_log_B, d_new_log_pi);
    return after_launch(st, "hmm_mstep", 1);
}

}  // extern "C"
