// Sequence ordering for the persistent HMM kernels: a counting sort of the sequences by
// decreasing length into 1024 logarithmic buckets (64 buckets per octave), so the longest
// sequences are taken first from the work queue (longest-processing-time-first) and
// consecutive sequences have similar lengths.  Order inside a bucket is arbitrary; no HMM
// result depends on which row or group a sequence lands in.
#include "hmm_internal.cuh"

#include <math.h>

namespace accel {
namespace hmm {

constexpr int kBuckets = 1024;

__device__ __forceinline__ int len_bucket(int64_t len) {
    // bucket 0 = longest: 1023 - floor(64 log2(len + 1)), clamped
    float l = log2f((float)len + 1.0f) * 64.0f;
    int b = (int)l;
    b = b < 0 ? 0 : (b > kBuckets - 1 ? kBuckets - 1 : b);
    return kBuckets - 1 - b;
}

__global__ void k_len_hist(const int64_t* __restrict__ off, int64_t S, int32_t* __restrict__ count) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&count[len_bucket(off[s + 1] - off[s])], 1);
}

__global__ void __launch_bounds__(kBuckets) k_len_scan(const int32_t* __restrict__ count, int32_t* __restrict__ cursor) {
    __shared__ int32_t s[kBuckets];
    int t = threadIdx.x;
    s[t] = count[t];
    __syncthreads();
    for (int d = 1; d < kBuckets; d <<= 1) {
        int32_t v = t >= d ? s[t - d] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    cursor[t] = s[t] - count[t];
}

__global__ void k_len_scatter(const int64_t* __restrict__ off, int64_t S, int32_t* __restrict__ cursor,
                              int32_t* __restrict__ order) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = atomicAdd(&cursor[len_bucket(off[s + 1] - off[s])], 1);
        order[p] = (int32_t)s;
    }
}

size_t order_ws_bytes(int64_t S) { return align_up((size_t)S * 4, 256) + 2 * kBuckets * 4; }

accel_status order_by_length(const int64_t* d_off, int64_t S, int32_t* d_order, char* scratch, cudaStream_t st) {
    ACCEL_REQUIRE(S <= INT32_MAX, ACCEL_ERR_UNSUPPORTED, "HMM: more than 2^31-1 sequences");
    int32_t* count = (int32_t*)scratch;
    int32_t* cursor = count + kBuckets;
    ACCEL_CUDA_TRY(cudaMemsetAsync(count, 0, kBuckets * 4, st));
    int g = (int)((S + 255) / 256);
    if (g > 4 * num_sms()) g = 4 * num_sms();
    if (g < 1) g = 1;
    k_len_hist<<<g, 256, 0, st>>>(d_off, S, count);
    k_len_scan<<<1, kBuckets, 0, st>>>(count, cursor);
    k_len_scatter<<<g, 256, 0, st>>>(d_off, S, cursor, d_order);
    // these three are counted by the calling entry point
    ACCEL_CUDA_TRY(cudaGetLastError());
    return ACCEL_OK;
}

// Largest segment length max_s (off[s+1] - off[s]), one CTA (0 for S = 0).
__global__ void __launch_bounds__(1024) k_max_len(const int64_t* __restrict__ off, int64_t S,
                                                  int64_t* __restrict__ out) {
    __shared__ int64_t s_max[32];
    int64_t m = 0;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
        const int64_t len = off[s + 1] - off[s];
        m = len > m ? len : m;
    }
    for (int d = 16; d > 0; d >>= 1) {
        const int64_t o = __shfl_xor_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? s_max[threadIdx.x] : 0;
        for (int d = 16; d > 0; d >>= 1) {
            const int64_t o = __shfl_xor_sync(0xffffffffu, m, d);
            m = o > m ? o : m;
        }
        if (threadIdx.x == 0) *out = m;
    }
}

}  // namespace hmm
}  // namespace accel

extern "C" accel_status hmm_max_length(const int64_t* d_offsets, int64_t S, int64_t* d_max_T, void* stream) {
    using namespace accel;
    ACCEL_REQUIRE(S >= 0, ACCEL_ERR_INVALID_ARG, "hmm_max_length: negative S");
    ACCEL_REQUIRE(d_offsets && d_max_T, ACCEL_ERR_INVALID_ARG, "hmm_max_length: null pointer");
    hmm::k_max_len<<<1, 1024, 0, as_stream(stream)>>>(d_offsets, S, d_max_T);
    return after_launch(as_stream(stream), "hmm_max_length", 1);
}
