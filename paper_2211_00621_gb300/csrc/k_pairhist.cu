// All-pairs histogram of angular separations (the two-point angular correlation shape the
// paper names as its tpacf workload, Table 1): a map over point pairs of a bin lookup,
// reduced into a histogram.  For unit vectors p_i, p_j the separation enters through the dot
// product d = (x_i x_j + y_i y_j) + z_i z_j, computed in FP32 with every product and sum
// rounded separately (no fused multiply-add), and the bin of d is the number of edges
// e_k >= d of a descending edge list (the cosines of increasing angles): bin 0 holds pairs
// closer than the first edge, bin n_edges those beyond the last one.
//
// Self mode (B is A) counts the unordered pairs i < j; cross mode all pairs (i in A, j in B).
// Tiles of 256 x 256 pairs: one CTA holds its 256 points of A in registers (one per thread)
// and streams the tile's points of B through shared memory (read as broadcasts).  The bin is
// found by binary lifting over the edges, padded to 32 with -inf, in shared memory (32
// words: conflict-free).  Each thread counts into its own column of a shared [bin][thread]
// array (no atomics, conflict-free for any bins); at the end of the launch a CTA sums its
// columns and adds them to the global int64 histogram.
#include "common.cuh"

#include <math.h>

namespace accel {
namespace pairhist {

constexpr int kThreads = 256;
constexpr int kTile = 256;
constexpr int kMaxBins = 32;             // n_edges + 1 <= 32

struct HistPrm {
    const float *ax, *ay, *az;
    const float *bx, *by, *bz;
    int64_t NA, NB;
    int self;                          // 1: B is A, count i < j
    int nbins;                         // n_edges + 1
    float edges[kMaxBins];             // descending, padded with -inf
    unsigned long long* hist;          // [nbins]
    int64_t ti, tj, ntiles;            // tiles along A, along B, tiles in the launch
};

// Tile q of the launch -> (tile of A, tile of B).  Self mode enumerates the upper triangle
// (tb >= ta) row by row.
__device__ __forceinline__ void tile_of(const HistPrm& p, int64_t q, int64_t& ta, int64_t& tb) {
    if (!p.self) {
        ta = q / p.tj;
        tb = q - ta * p.tj;
        return;
    }
    // row ta holds ti - ta tiles; find ta with prefix(ta) <= q < prefix(ta + 1),
    // prefix(a) = a ti - a (a - 1) / 2
    int64_t lo = 0, hi = p.ti - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        const int64_t pre = mid * p.ti - mid * (mid - 1) / 2;
        if (pre <= q) lo = mid; else hi = mid - 1;
    }
    ta = lo;
    tb = ta + (q - (lo * p.ti - lo * (lo - 1) / 2));
}

__global__ void __launch_bounds__(kThreads) k_pairhist(HistPrm p) {
    __shared__ float sx[kTile], sy[kTile], sz[kTile];
    __shared__ float se[kMaxBins];
    __shared__ unsigned int cnt[kMaxBins][kThreads];
    const int tid = threadIdx.x;
    if (tid < kMaxBins) se[tid] = p.edges[tid];
    for (int b = 0; b < kMaxBins; ++b) cnt[b][tid] = 0u;
    for (int64_t q = blockIdx.x; q < p.ntiles; q += gridDim.x) {
        int64_t ta, tb;
        tile_of(p, q, ta, tb);
        const int64_t i = ta * kTile + tid;
        const bool has_i = i < p.NA;
        const float xi = has_i ? p.ax[i] : 0.f, yi = has_i ? p.ay[i] : 0.f, zi = has_i ? p.az[i] : 0.f;
        const int64_t j0 = tb * kTile;
        int64_t nj = p.NB - j0;
        if (nj > kTile) nj = kTile;
        __syncthreads();                  // the previous tile's points are no longer read
        if (tid < nj) {
            sx[tid] = p.bx[j0 + tid];
            sy[tid] = p.by[j0 + tid];
            sz[tid] = p.bz[j0 + tid];
        }
        __syncthreads();
        if (has_i) {
            // self mode, diagonal tile: only j > i
            const int jstart = (p.self && ta == tb) ? tid + 1 : 0;
            auto bin_of = [&](int jj) {
                const float d = __fadd_rn(__fadd_rn(__fmul_rn(xi, sx[jj]), __fmul_rn(yi, sy[jj])), __fmul_rn(zi, sz[jj]));
                int b = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (se[b + step - 1] >= d) b += step;
                return b;
            };
            int jj = jstart;
            // four independent lookups in flight, then their counts
            for (; jj + 4 <= (int)nj; jj += 4) {
                const int b0 = bin_of(jj), b1 = bin_of(jj + 1), b2 = bin_of(jj + 2), b3 = bin_of(jj + 3);
                cnt[b0][tid] += 1u;
                cnt[b1][tid] += 1u;
                cnt[b2][tid] += 1u;
                cnt[b3][tid] += 1u;
            }
            for (; jj < (int)nj; ++jj) cnt[bin_of(jj)][tid] += 1u;
        }
    }
    __syncthreads();
    // sum the columns: warp w sums bins w, w + 8, ...
    const int w = tid >> 5, lane = tid & 31;
    for (int b = w; b < p.nbins; b += kThreads / 32) {
        unsigned long long s = 0;
        for (int t = lane; t < kThreads; t += 32) s += cnt[b][t];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0 && s) atomicAdd(&p.hist[b], s);
    }
}

}  // namespace pairhist
}  // namespace accel

using namespace accel;
using namespace accel::pairhist;

extern "C" {

accel_status accel_pair_histogram(const float* d_ax, const float* d_ay, const float* d_az, int64_t NA,
                                  const float* d_bx, const float* d_by, const float* d_bz, int64_t NB,
                                  const float* h_edges, int32_t n_edges, int64_t* d_hist, void* stream) {
    ACCEL_REQUIRE(NA >= 0 && NB >= 0, ACCEL_ERR_INVALID_ARG, "accel_pair_histogram: negative size");
    ACCEL_REQUIRE(n_edges >= 1 && n_edges <= kMaxBins - 1, ACCEL_ERR_UNSUPPORTED,
                  "accel_pair_histogram: n_edges=%d outside [1, %d]", n_edges, kMaxBins - 1);
    ACCEL_REQUIRE(h_edges && d_hist, ACCEL_ERR_INVALID_ARG, "accel_pair_histogram: null pointer");
    // self mode: B is A (the same arrays and count)
    const bool self = d_bx == d_ax && d_by == d_ay && d_bz == d_az && NB == NA;
    ACCEL_REQUIRE(NA == 0 || (d_ax && d_ay && d_az), ACCEL_ERR_INVALID_ARG, "accel_pair_histogram: null point array");
    ACCEL_REQUIRE(NB == 0 || (d_bx && d_by && d_bz), ACCEL_ERR_INVALID_ARG, "accel_pair_histogram: null point array");
    HistPrm p{};
    for (int k = 0; k < n_edges; ++k) {
        ACCEL_REQUIRE(!isnan(h_edges[k]), ACCEL_ERR_INVALID_ARG, "accel_pair_histogram: edge %d is NaN", k);
        ACCEL_REQUIRE(k == 0 || h_edges[k] < h_edges[k - 1], ACCEL_ERR_SHAPE,
                      "accel_pair_histogram: edges must be strictly decreasing (edge %d)", k);
        p.edges[k] = h_edges[k];
    }
    for (int k = n_edges; k < kMaxBins; ++k) p.edges[k] = -INFINITY;
    p.nbins = n_edges + 1;
    p.self = self ? 1 : 0;
    p.ax = d_ax; p.ay = d_ay; p.az = d_az;
    p.NA = NA;
    p.bx = d_bx; p.by = d_by; p.bz = d_bz;
    p.NB = NB;
    p.hist = (unsigned long long*)d_hist;
    p.ti = (p.NA + kTile - 1) / kTile;
    p.tj = (p.NB + kTile - 1) / kTile;
    p.ntiles = self ? p.ti * (p.ti + 1) / 2 : p.ti * p.tj;
    cudaStream_t st = as_stream(stream);
    ACCEL_CUDA_TRY(cudaMemsetAsync(d_hist, 0, (size_t)p.nbins * sizeof(int64_t), st));
    if (p.ntiles == 0) return after_launch(st, "accel_pair_histogram", 0);
    // a thread counts at most 256 pairs per tile in uint32: at most 2^24 tiles per CTA
    int64_t grid = 4LL * num_sms();
    const int64_t min_grid = (p.ntiles + (1LL << 24) - 1) >> 24;
    if (grid < min_grid) grid = min_grid;
    if (grid > p.ntiles) grid = p.ntiles;
    k_pairhist<<<(unsigned)grid, kThreads, 0, st>>>(p);
    return after_launch(st, "accel_pair_histogram", 1);
}

}  // extern "C"
