// All-pairs map-of-reduce (K10): for every body i a reduce over all bodies j
// (Appendix A: a map whose function is a reduce; the paper's tpacf / mri-q workloads,
// Table 1, have this shape).  Softened gravity, G = 1, FP32:
//     a_i = sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2)
//
// FP32-ALU bound (FFMA + MUFU rsqrt), no tensor cores.  A CTA owns 64 bodies and splits
// the j range four ways (256 threads), so the grid is N/64 CTAs -- enough to balance 152
// SMs at N = 65,536.  j bodies are staged in shared memory as float4 tiles (x, y, z, m)
// and read as warp-wide broadcasts; each thread carries two bodies (i and i + 32) to
// reuse every loaded j twice.  The four partial sums of a body are added in a fixed order
// in shared memory, so results are deterministic.
#include "common.cuh"

namespace accel {
namespace pair {

constexpr int kThreads = 256;
constexpr int kBodies = 64;   // bodies per CTA
constexpr int kSplit = 4;     // j-range split inside the CTA
constexpr int kTile = 256;    // j bodies per shared-memory tile

__global__ void __launch_bounds__(kThreads)
k_gravity(const float* __restrict__ X, const float* __restrict__ Y, const float* __restrict__ Z,
          const float* __restrict__ Mass, int64_t n, float eps2, float* __restrict__ AX,
          float* __restrict__ AY, float* __restrict__ AZ) {
    __shared__ float4 s_j[kTile];
    __shared__ float3 s_part[kSplit][kBodies];
    // Thread t: j quarter q = t / 64 (warps 2q and 2q+1); both warps of a quarter hold
    // all 64 bodies of the CTA (slots il and il + 32) and take alternate j's (parity
    // `half`) of the quarter, so every j read from shared memory is a warp broadcast.
    const int t = threadIdx.x;
    const int q = t >> 6;
    const int il = t & 31;
    const int half = (t >> 5) & 1;
    const int64_t ib = blockIdx.x * (int64_t)kBodies;
    const int64_t i0 = ib + il, i1 = ib + il + 32;
    float x0 = 0, y0 = 0, z0 = 0, x1 = 0, y1 = 0, z1 = 0;
    if (i0 < n) { x0 = X[i0]; y0 = Y[i0]; z0 = Z[i0]; }
    if (i1 < n) { x1 = X[i1]; y1 = Y[i1]; z1 = Z[i1]; }
    float ax0 = 0.f, ay0 = 0.f, az0 = 0.f, ax1 = 0.f, ay1 = 0.f, az1 = 0.f;

    for (int64_t jb = 0; jb < n; jb += kTile) {
        __syncthreads();
        {
            int64_t j = jb + t;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);   // padding bodies have zero mass
            if (j < n) v = make_float4(X[j], Y[j], Z[j], Mass[j]);
            s_j[t] = v;
        }
        __syncthreads();
        // this warp's j's in the tile: quarter q = [q*64, q*64+64), split by parity
        const float4* pj = s_j + q * (kTile / kSplit) + half;
#pragma unroll 8
        for (int k = 0; k < kTile / kSplit / 2; ++k) {
            float4 b = pj[2 * k];
            float dx0 = b.x - x0, dy0 = b.y - y0, dz0 = b.z - z0;
            float dx1 = b.x - x1, dy1 = b.y - y1, dz1 = b.z - z1;
            float r0 = fmaf(dx0, dx0, fmaf(dy0, dy0, fmaf(dz0, dz0, eps2)));
            float r1 = fmaf(dx1, dx1, fmaf(dy1, dy1, fmaf(dz1, dz1, eps2)));
            float inv0 = rsqrtf(r0), inv1 = rsqrtf(r1);
            float s0 = b.w * inv0 * inv0 * inv0;
            float s1 = b.w * inv1 * inv1 * inv1;
            ax0 = fmaf(s0, dx0, ax0); ay0 = fmaf(s0, dy0, ay0); az0 = fmaf(s0, dz0, az0);
            ax1 = fmaf(s1, dx1, ax1); ay1 = fmaf(s1, dy1, ay1); az1 = fmaf(s1, dz1, az1);
        }
    }
    // combine: parity halves via shared memory, then the four quarters in order
    __shared__ float3 s_half[kSplit][kBodies];
    if (half == 1) {
        s_half[q][il] = make_float3(ax0, ay0, az0);
        s_half[q][il + 32] = make_float3(ax1, ay1, az1);
    }
    __syncthreads();
    if (half == 0) {
        float3 o0 = s_half[q][il], o1 = s_half[q][il + 32];
        s_part[q][il] = make_float3(ax0 + o0.x, ay0 + o0.y, az0 + o0.z);
        s_part[q][il + 32] = make_float3(ax1 + o1.x, ay1 + o1.y, az1 + o1.z);
    }
    __syncthreads();
    if (t < kBodies) {
        int64_t i = ib + t;
        float3 a = s_part[0][t];
#pragma unroll
        for (int r = 1; r < kSplit; ++r) {
            float3 b = s_part[r][t];
            a.x += b.x; a.y += b.y; a.z += b.z;
        }
        if (i < n) { AX[i] = a.x; AY[i] = a.y; AZ[i] = a.z; }
    }
}

}  // namespace pair
}  // namespace accel

using namespace accel;

extern "C" {

accel_status pairwise_mapreduce(int32_t op, const float* d_x, const float* d_y, const float* d_z, const float* d_m,
                                int64_t n, float eps, float* d_ax, float* d_ay, float* d_az, void* stream) {
    ACCEL_REQUIRE(op == ACCEL_PAIR_GRAVITY_SOFTENED, ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: bad op %d", op);
    ACCEL_REQUIRE(n >= 0, ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: n < 0");
    if (n == 0) return ok();
    ACCEL_REQUIRE(d_x && d_y && d_z && d_m && d_ax && d_ay && d_az, ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: null pointer");
    ACCEL_REQUIRE(n <= (int64_t)INT32_MAX * pair::kBodies, ACCEL_ERR_UNSUPPORTED, "pairwise_mapreduce: n too large");
    cudaStream_t st = as_stream(stream);
    unsigned grid = (unsigned)((n + pair::kBodies - 1) / pair::kBodies);
    pair::k_gravity<<<grid, pair::kThreads, 0, st>>>(d_x, d_y, d_z, d_m, n, eps * eps, d_ax, d_ay, d_az);
    return after_launch(st, "pairwise_mapreduce", 1);
}

}  // extern "C"
