// Streaming a dense K x K FP32 matrix through shared memory for the SIMT HMM kernels.
//
// The batched SIMT steps compute acc_g(j) = sum_i X_g(i) Mat(i, j) for a few sequences g
// per CTA (thread j owns output j).  Mat does not fit shared memory at K = 256 (256 KB in
// FP32), and reading it straight from L2 leaves every warp waiting on loads.  Instead the
// rows of Mat are streamed in chunks of 32 rows through a ring of kNB shared buffers by
// 1-D bulk copies (cp.async.bulk, one thread issues them), each completing on its own
// mbarrier; while the CTA works on chunk c the next kNB - 1 chunks are in flight.  The
// chunk order repeats every step, so a stream "phase" (consecutive steps with the same
// matrix) keeps the ring full across step boundaries.  Mat rows are stored with a stride
// of Kp floats (a multiple of 4) so every copy is 16-byte aligned.
// Every wait is bounded (2 s of wall clock); on expiry the calling kernel reports
// ACCEL_ERR_TIMEOUT and drains its copies in flight (again bounded) before returning.
#pragma once
#include "common.cuh"
#include "tc_ptx.cuh"

namespace accel {
namespace simt {

constexpr int kChunkRows = 32;
constexpr int kNB = 3;
constexpr uint64_t kWaitNs = 2000000000ull;

struct AStream {
    const float* g;     // matrix rows (stride Kp floats), 16-byte aligned
    float* buf;         // kNB x kChunkRows x Kp shared floats
    uint64_t* full;     // kNB mbarriers, initialised with count 1
    int K, Kp, nchunk;
    uint32_t c;         // chunks consumed so far
    uint32_t phase0;    // value of c when the current phase began
};

__host__ __device__ constexpr size_t stream_smem_bytes(int Kp) { return (size_t)kNB * kChunkRows * Kp * 4 + kNB * 8; }

// Carve the ring and its barriers from `smem` (16-byte aligned); thread 0 initialises the
// barriers.  The caller syncs before the first as_begin.
__device__ __forceinline__ void as_init(AStream& s, char* smem, int K, int Kp) {
    s.buf = reinterpret_cast<float*>(smem);
    s.full = reinterpret_cast<uint64_t*>(smem + (size_t)kNB * kChunkRows * Kp * 4);
    s.K = K;
    s.Kp = Kp;
    s.nchunk = (K + kChunkRows - 1) / kChunkRows;
    s.c = 0;
    s.phase0 = 0;
    s.g = nullptr;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kNB; ++b) tc::mbar_init(&s.full[b], 1);
        tc::fence_mbar_init();
    }
}

__device__ __forceinline__ void as_issue(AStream& s, uint32_t gi) {   // thread 0 only
    const int b = (int)(gi % kNB);
    const int cc = (int)((gi - s.phase0) % (uint32_t)s.nchunk);
    const int rows = min(kChunkRows, s.K - cc * kChunkRows);
    const uint32_t bytes = (uint32_t)rows * s.Kp * 4;
    tc::mbar_arrive_expect_tx(&s.full[b], bytes);
    tc::bulk_g2s(s.buf + (size_t)b * kChunkRows * s.Kp, s.g + (size_t)cc * kChunkRows * s.Kp, bytes, &s.full[b]);
}

// Start a phase streaming `g` (all threads call; thread 0 fills the ring).
__device__ __forceinline__ void as_begin(AStream& s, const float* g) {
    s.g = g;
    s.phase0 = s.c;
    if (threadIdx.x == 0)
        for (int k = 0; k < kNB; ++k) as_issue(s, s.c + k);
}

// End a phase: wait for the kNB prefetched chunks nobody will use (all threads call).
__device__ __forceinline__ bool as_end(AStream& s) {
    bool ok = true;
    for (int k = 0; k < kNB; ++k) {
        uint32_t gi = s.c + k;
        ok = tc::mbar_wait_bounded(&s.full[gi % kNB], (gi / kNB) & 1, kWaitNs) && ok;
    }
    s.c += kNB;
    return !__syncthreads_or(!ok);
}

// After a failed wait: wait (bounded) for the copies still in flight, then give up.
__device__ __forceinline__ void as_drain(AStream& s) {
    for (int k = 0; k < kNB; ++k) {
        uint32_t gi = s.c + k;
        tc::mbar_wait_bounded(&s.full[gi % kNB], (gi / kNB) & 1, kWaitNs / 4);
    }
}

// acc_g(j) = sum_i X[g * ld + i] Mat(i, j) for the active g, thread j = threadIdx.x.
// Returns false (in every thread) if a chunk did not arrive in time.
template <int G>
__device__ __forceinline__ bool as_matvec(AStream& s, const float* X, int ld, const bool (&act)[G], float (&acc)[G]) {
    const int j = threadIdx.x;
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.f;
    for (int cc = 0; cc < s.nchunk; ++cc) {
        const uint32_t gi = s.c;
        const int b = (int)(gi % kNB);
        const bool arrived = tc::mbar_wait_bounded(&s.full[b], (gi / kNB) & 1, kWaitNs);
        if (arrived && j < s.K) {
            const float* A = s.buf + (size_t)b * kChunkRows * s.Kp + j;
            const int i0 = cc * kChunkRows;
            const int rows = min(kChunkRows, s.K - i0);
            int r = 0;
            for (; r + 4 <= rows; r += 4) {
                const float a0 = A[(r + 0) * s.Kp], a1 = A[(r + 1) * s.Kp];
                const float a2 = A[(r + 2) * s.Kp], a3 = A[(r + 3) * s.Kp];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (!act[g]) continue;
                    const float4 x = *reinterpret_cast<const float4*>(X + g * ld + i0 + r);
                    acc[g] = fmaf(x.x, a0, acc[g]);
                    acc[g] = fmaf(x.y, a1, acc[g]);
                    acc[g] = fmaf(x.z, a2, acc[g]);
                    acc[g] = fmaf(x.w, a3, acc[g]);
                }
            }
            for (; r < rows; ++r) {
                const float a0 = A[r * s.Kp];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (act[g]) acc[g] = fmaf(X[g * ld + i0 + r], a0, acc[g]);
            }
        }
        s.c = gi + 1;
        if (__syncthreads_or(!arrived)) return false;   // also: buffer b is free
        if (threadIdx.x == 0) as_issue(s, gi + kNB);
    }
    return true;
}

}  // namespace simt
}  // namespace accel
