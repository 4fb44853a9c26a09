// Plain FP32 log-space HMM forward recursion (K7).
//
// The recursion is a map over states j of a reduce over states i inside a sequential
// loop over t (Appendix A patterns; Listing 1's loop/reduce pairing).  The paper does
// not discuss HMMs; the arithmetic is the textbook forward algorithm in log space:
//     la_1(j) = log pi_j + log B[j, o_1]
//     la_t(j) = LSE_i(la_{t-1}(i) + log A[i, j]) + log B[j, o_t],   logL = LSE_j la_T(j)
// evaluated as la_t(j) = m + log sum_i exp(la_{t-1}(i) - m) A[i, j] + log B[j, o_t] with
// m = max_i la_{t-1}(i) (max-shifted sum of exponentials; A = exp(log A) precomputed).
// Each sequence keeps la = c + r with r in FP32 and the running offset c (the sum of the
// per-step maxima, a sum of log scale factors) in FP64.
//
// Two kernels:
//  * k_plain_warp<J> (K <= 32 J, J <= 2): one warp per sequence, lane l owns states
//    l and l + 32; the two columns of A it needs live in registers (K floats each), the
//    emission table log B^T in shared memory; no block-wide synchronisation.
//  * k_plain_cta (K <= 256): one CTA per group of G sequences (ordered by length so a
//    group's lengths are alike); thread j owns state j of all G sequences and streams A's
//    column j from L2, reusing each element G times.
#include "common.cuh"
#include "hmm_internal.cuh"
#include "simt_stream.cuh"

namespace accel {
namespace hmm {

// ---------------------------------------------------------------- warp per sequence
template <int J>
__global__ void __launch_bounds__(128)
k_plain_warp(const float* __restrict__ logA, const float* __restrict__ logB, const float* __restrict__ logpi,
             int K, int M, const int32_t* __restrict__ obs, const int64_t* __restrict__ off, int64_t S,
             double* __restrict__ loglik) {
    extern __shared__ float smem[];
    float* sB = smem;                                  // [M][K]  log B^T
    float* sP = smem + (((size_t)M * K + 3) & ~(size_t)3);   // [4][32 J] per-warp, 16-byte aligned
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int idx = threadIdx.x; idx < M * K; idx += blockDim.x) {
        int j = idx / M, k = idx - j * M;
        sB[k * K + j] = logB[idx];
    }
    __syncthreads();
    const int64_t s = blockIdx.x * 4 + w;
    if (s >= S) return;

    float a[J][32 * J];                      // a[jj][i] = A[i, lane + 32 jj]
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        int j = lane + 32 * jj;
#pragma unroll
        for (int i = 0; i < 32 * J; ++i) a[jj][i] = (j < K && i < K) ? __expf(logA[i * K + j]) : 0.f;
    }
    float* P = sP + w * 32 * J;
    const int64_t o0 = off[s];
    const int64_t T = off[s + 1] - o0;
    const int32_t* o = obs + o0;

    float r[J];
    int32_t ob = o[0];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        int j = lane + 32 * jj;
        r[jj] = j < K ? logpi[j] + sB[ob * K + j] : -INFINITY;
    }
    double c = 0.0;
    int32_t ochunk = 0;
    for (int64_t t = 1; t < T; ++t) {
        int sl = (int)(t & 31);
        if (sl == 0 || t == 1) {             // refill: lane l holds o[32 floor(t/32) + l]
            int64_t tt = t + lane - sl;
            ochunk = (tt < T) ? o[tt] : 0;
        }
        ob = __shfl_sync(0xffffffffu, ochunk, sl);
        float m = r[0];
#pragma unroll
        for (int jj = 1; jj < J; ++jj) m = fmaxf(m, r[jj]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
#pragma unroll
        for (int jj = 0; jj < J; ++jj) P[lane + 32 * jj] = __expf(r[jj] - m);
        __syncwarp();
        float acc[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) acc[jj] = 0.f;
#pragma unroll
        for (int i4 = 0; i4 < 8 * J; ++i4) {
            float4 p = reinterpret_cast<const float4*>(P)[i4];
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                acc[jj] = fmaf(p.x, a[jj][4 * i4 + 0], acc[jj]);
                acc[jj] = fmaf(p.y, a[jj][4 * i4 + 1], acc[jj]);
                acc[jj] = fmaf(p.z, a[jj][4 * i4 + 2], acc[jj]);
                acc[jj] = fmaf(p.w, a[jj][4 * i4 + 3], acc[jj]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
            int j = lane + 32 * jj;
            r[jj] = j < K ? __logf(acc[jj]) + sB[ob * K + j] : -INFINITY;
        }
        c += (double)m;
    }
    float m = r[0];
#pragma unroll
    for (int jj = 1; jj < J; ++jj) m = fmaxf(m, r[jj]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
    float e = 0.f;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) e += __expf(r[jj] - m);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) e += __shfl_xor_sync(0xffffffffu, e, d);
    if (lane == 0) loglik[s] = c + (double)m + log((double)e);
}

// ---------------------------------------------------------------- CTA per G sequences
constexpr int kCtaThreads = 256;
constexpr int kG = 8;

// exp(log A) with row stride Kp (padding zero)
__global__ void k_exp_f32(const float* __restrict__ in, float* __restrict__ out, int K, int Kp) {
    int64_t n = (int64_t)K * Kp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(i / Kp), c = (int)(i % Kp);
        out[i] = c < K ? __expf(in[(int64_t)r * K + c]) : 0.f;
    }
}

__host__ __device__ inline size_t cta_off_b(int Kp) { return align_up(simt::stream_smem_bytes(Kp), 16); }

__global__ void __launch_bounds__(kCtaThreads)
k_plain_cta(const float* __restrict__ Aexp, const float* __restrict__ logB, const float* __restrict__ logpi,
            int K, int M, const int32_t* __restrict__ obs, const int64_t* __restrict__ off, int64_t S,
            const int32_t* __restrict__ order, double* __restrict__ loglik, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) float smem_f[];
    char* smem = reinterpret_cast<char*>(smem_f);
    const int Kp = (K + 3) & ~3;                // padded row stride (16-byte rows)
    simt::AStream as;
    simt::as_init(as, smem, K, Kp);
    float* sB = reinterpret_cast<float*>(smem + cta_off_b(Kp));                        // [M][K]
    float* sP = sB + (((size_t)M * K + 3) & ~(size_t)3);                               // [kG][Kp]
    __shared__ float s_red[kG][kCtaThreads / 32];
    __shared__ int64_t s_T[kG], s_o0[kG];
    const int j = threadIdx.x, lane = j & 31, w = j >> 5;
    for (int idx = threadIdx.x; idx < M * K; idx += blockDim.x) {
        int jj = idx / M, k = idx - jj * M;
        sB[k * K + jj] = logB[idx];
    }
    int64_t seq[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        int64_t q = blockIdx.x * (int64_t)kG + g;
        seq[g] = q < S ? order[q] : -1;
    }
    if (j < kG) {
        int64_t sq = seq[j];
        s_o0[j] = sq >= 0 ? off[sq] : 0;
        s_T[j] = sq >= 0 ? off[sq + 1] - off[sq] : 0;
    }
    __syncthreads();
    int64_t T[kG], o0[kG], Tmax = 0;
#pragma unroll
    for (int g = 0; g < kG; ++g) { T[g] = s_T[g]; o0[g] = s_o0[g]; Tmax = T[g] > Tmax ? T[g] : Tmax; }
    const bool jv = j < K;
    float r[kG];
    double c[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        c[g] = 0.0;
        r[g] = (jv && T[g] > 0) ? logpi[j] + sB[obs[o0[g]] * K + j] : -INFINITY;
    }
    simt::as_begin(as, Aexp);
    for (int64_t t = 1; t < Tmax; ++t) {
        // per-sequence maxima over states
        float m[kG];
        bool act[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            act[g] = t < T[g];
            float v = r[g];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
            if (lane == 0) s_red[g][w] = v;
        }
        __syncthreads();
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            float v = s_red[g][0];
            for (int q = 1; q < kCtaThreads / 32; ++q) v = fmaxf(v, s_red[g][q]);
            m[g] = v;
            if (jv) sP[g * Kp + j] = act[g] ? __expf(r[g] - v) : 0.f;
        }
        __syncthreads();
        float acc[kG];
        if (!simt::as_matvec<kG>(as, sP, Kp, act, acc)) {
            if (threadIdx.x == 0) report_status(status, ACCEL_ERR_TIMEOUT);
            simt::as_drain(as);
            return;
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            if (act[g]) {
                int32_t ob = obs[o0[g] + t];
                r[g] = jv ? __logf(acc[g]) + sB[ob * K + j] : -INFINITY;
                c[g] += (double)m[g];
            }
        }
        __syncthreads();   // sP and s_red reuse
    }
    if (!simt::as_end(as)) {
        if (threadIdx.x == 0) report_status(status, ACCEL_ERR_TIMEOUT);
        simt::as_drain(as);
        return;
    }
    // logL = c + LSE_j r
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        float v = r[g];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
        if (lane == 0) s_red[g][w] = v;
    }
    __syncthreads();
    float m[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        float v = s_red[g][0];
        for (int q = 1; q < kCtaThreads / 32; ++q) v = fmaxf(v, s_red[g][q]);
        m[g] = v;
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        float e = jv ? __expf(r[g] - m[g]) : 0.f;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) e += __shfl_xor_sync(0xffffffffu, e, d);
        if (lane == 0) s_red[g][w] = e;
    }
    __syncthreads();
    if (j < kG) {
        int g = j;
        float e = 0.f;
        for (int q = 0; q < kCtaThreads / 32; ++q) e += s_red[g][q];
        if (seq[g] >= 0) loglik[seq[g]] = c[g] + (double)m[g] + log((double)e);
    }
}

size_t plain_ws_bytes(int K, int M, int64_t S) {
    (void)M;
    if (K <= 64) return 0;
    return align_up((size_t)K * ((K + 3) & ~3) * 4, 256) + order_ws_bytes(S);
}

accel_status plain_forward(const accel_hmm_model* m, const int32_t* obs, const int64_t* off, int64_t S,
                           double* loglik, char* ws, int32_t* d_status, cudaStream_t st) {
    const int K = m->K, M = m->M;
    if (K <= 64) {
        size_t smem = ((((size_t)M * K + 3) & ~(size_t)3) + 4 * 64) * sizeof(float);
        ACCEL_REQUIRE(smem <= (size_t)max_smem_optin(), ACCEL_ERR_UNSUPPORTED, "hmm_forward: M*K too large for the FP32 kernel");
        unsigned grid = (unsigned)((S + 3) / 4);
        if (K <= 32) {
            ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_plain_warp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_plain_warp<1><<<grid, 128, smem, st>>>(m->log_A, m->log_B, m->log_pi, K, M, obs, off, S, loglik);
        } else {
            ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_plain_warp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_plain_warp<2><<<grid, 128, smem, st>>>(m->log_A, m->log_B, m->log_pi, K, M, obs, off, S, loglik);
        }
        return after_launch(st, "hmm_forward(fp32 warp)", 1);
    }
    const int Kp = (K + 3) & ~3;
    size_t smem = cta_off_b(Kp) + ((((size_t)M * K + 3) & ~(size_t)3) + (size_t)kG * Kp) * sizeof(float);
    ACCEL_REQUIRE(smem <= (size_t)max_smem_optin(), ACCEL_ERR_UNSUPPORTED, "hmm_forward: M*K too large for the FP32 kernel");
    float* Aexp = (float*)ws;
    int32_t* order = (int32_t*)(ws + align_up((size_t)K * Kp * 4, 256));
    char* order_scratch = (char*)order + align_up((size_t)S * 4, 256);
    k_exp_f32<<<num_sms() * 2, 256, 0, st>>>(m->log_A, Aexp, K, Kp);
    accel_status r = order_by_length(off, S, order, order_scratch, st);
    if (r != ACCEL_OK) return r;
    ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_plain_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = (unsigned)((S + kG - 1) / kG);
    k_plain_cta<<<grid, kCtaThreads, smem, st>>>(Aexp, m->log_B, m->log_pi, K, M, obs, off, S, order, loglik, d_status);
    return after_launch(st, "hmm_forward(fp32 cta)", 5);
}

}  // namespace hmm
}  // namespace accel
