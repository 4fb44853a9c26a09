// Sequence ordering for the persistent HMM kernels: a counting sort of the sequences by
// decreasing length into 1024 logarithmic buckets (64 buckets per octave), so the longest
// sequences are taken first from the work queue (longest-processing-time-first) and
// consecutive sequences have similar lengths.  The sort is stable: inside a bucket the
// sequences keep increasing index.  The order is therefore a function of the lengths alone,
// which the adjoint needs -- its sequence groups, and with them the order of its partial
// sums, follow the order -- so that repeated calls give bit-identical results.
//
// Three launches over nb contiguous blocks of sequences: per-block bucket histograms; one CTA
// that turns them into each block's first position per bucket (buckets in order, blocks in
// order inside a bucket); and the scatter, in which a block places its sequences in index
// order (rounds of 256: lanes of a warp ranked by __match_any_sync, warps one after another).
#include "hmm_internal.cuh"

#include <math.h>

namespace accel {
namespace hmm {

constexpr int kBuckets = 1024;
constexpr int kSortThreads = 256;
constexpr int kSortChunk = 1024;      // sequences per block (fewer blocks past kSortBlocksMax)
constexpr int kSortBlocksMax = 512;

static int sort_blocks(int64_t S) {
    const int64_t b = (S + kSortChunk - 1) / kSortChunk;
    return (int)(b < 1 ? 1 : (b > kSortBlocksMax ? kSortBlocksMax : b));
}

__device__ __forceinline__ int len_bucket(int64_t len) {
    // bucket 0 = longest: 1023 - floor(64 log2(len + 1)), clamped
    float l = log2f((float)len + 1.0f) * 64.0f;
    int b = (int)l;
    b = b < 0 ? 0 : (b > kBuckets - 1 ? kBuckets - 1 : b);
    return kBuckets - 1 - b;
}

// sequences [s0, s1) of block b of nb
__device__ __forceinline__ void sort_range(int64_t S, int nb, int b, int64_t& s0, int64_t& s1) {
    s0 = S * b / nb;
    s1 = S * (b + 1) / nb;
}

// hist[b][k] = number of sequences of block b in bucket k
__global__ void __launch_bounds__(kSortThreads) k_len_hist(const int64_t* __restrict__ off, int64_t S,
                                                           int32_t* __restrict__ hist) {
    __shared__ int32_t h[kBuckets];
    for (int k = threadIdx.x; k < kBuckets; k += kSortThreads) h[k] = 0;
    __syncthreads();
    int64_t s0, s1;
    sort_range(S, (int)gridDim.x, (int)blockIdx.x, s0, s1);
    for (int64_t s = s0 + threadIdx.x; s < s1; s += kSortThreads) atomicAdd(&h[len_bucket(off[s + 1] - off[s])], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < kBuckets; k += kSortThreads) hist[(int64_t)blockIdx.x * kBuckets + k] = h[k];
}

// In place: hist[b][k] <- (sequences in buckets < k) + (sequences of bucket k in blocks < b).
__global__ void __launch_bounds__(kBuckets) k_len_scan(int32_t* __restrict__ hist, int nb) {
    __shared__ int32_t s[kBuckets];
    const int k = threadIdx.x;
    int32_t run = 0;
    for (int b = 0; b < nb; ++b) {
        const int32_t c = hist[(int64_t)b * kBuckets + k];
        hist[(int64_t)b * kBuckets + k] = run;
        run += c;
    }
    s[k] = run;
    __syncthreads();
    for (int d = 1; d < kBuckets; d <<= 1) {
        const int32_t v = k >= d ? s[k - d] : 0;
        __syncthreads();
        s[k] += v;
        __syncthreads();
    }
    const int32_t base = s[k] - run;   // exclusive prefix over the buckets
    for (int b = 0; b < nb; ++b) hist[(int64_t)b * kBuckets + k] += base;
}

__global__ void __launch_bounds__(kSortThreads) k_len_scatter(const int64_t* __restrict__ off, int64_t S,
                                                              const int32_t* __restrict__ start,
                                                              int32_t* __restrict__ order) {
    __shared__ int32_t cur[kBuckets];
    for (int k = threadIdx.x; k < kBuckets; k += kSortThreads) cur[k] = start[(int64_t)blockIdx.x * kBuckets + k];
    __syncthreads();
    int64_t s0, s1;
    sort_range(S, (int)gridDim.x, (int)blockIdx.x, s0, s1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = s0; base < s1; base += kSortThreads) {
        const int64_t s = base + threadIdx.x;
        const bool in = s < s1;
        // lanes past the range get keys of their own, so they match nothing
        const int key = in ? len_bucket(off[s + 1] - off[s]) : kBuckets + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        for (int w = 0; w < kSortThreads / 32; ++w) {
            if (warp == w) {
                int32_t p = 0;
                if (in && lane == leader) {
                    p = cur[key];
                    cur[key] = p + __popc(peers);
                }
                p = __shfl_sync(0xffffffffu, p, leader);
                if (in) order[p + rank] = (int32_t)s;
            }
            __syncthreads();
        }
    }
}

size_t order_ws_bytes(int64_t S) { return align_up((size_t)S * 4, 256) + (size_t)sort_blocks(S) * kBuckets * 4; }

accel_status order_by_length(const int64_t* d_off, int64_t S, int32_t* d_order, char* scratch, cudaStream_t st) {
    ACCEL_REQUIRE(S <= INT32_MAX, ACCEL_ERR_UNSUPPORTED, "HMM: more than 2^31-1 sequences");
    int32_t* hist = (int32_t*)scratch;
    const int nb = sort_blocks(S);
    k_len_hist<<<nb, kSortThreads, 0, st>>>(d_off, S, hist);
    k_len_scan<<<1, kBuckets, 0, st>>>(hist, nb);
    k_len_scatter<<<nb, kSortThreads, 0, st>>>(d_off, S, hist, d_order);
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
