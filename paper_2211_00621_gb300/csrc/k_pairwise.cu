// All-pairs map-of-reduce (K10): for every body i a reduce over all bodies j
// (Appendix A: a map whose function is a reduce; the paper's tpacf / mri-q workloads,
// Table 1, have this shape).  Softened gravity, G = 1, FP32:
//     a_i = sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2)
//
// FP32-pipe bound (12 FP32 operations + 1 MUFU rsqrt per interaction), no tensor cores.
// The FP32 work is issued as packed pairs (add/mul/fma .f32x2, one instruction for two
// lanes' worth of operations): with scalar FFMAs the FP32 pipe alone needs one issue slot per
// cycle, so every shared-memory load, MUFU and loop instruction came out of its time; with
// pairs the pipe keeps its rate at half the issue slots.  A pair is two j bodies against one
// i body, so the i coordinates are duplicated into both halves once, and the j bodies are
// staged in shared memory as a structure of arrays, read four at a time as float4 warp
// broadcasts.  The reciprocal square root is the MUFU approximation with denormal inputs
// flushed: r >= eps^2, and the host accepts only eps whose eps^2 is a normal float, so no
// input of it is denormal and the flush never applies.
//
// Decomposition: a CTA owns 64 bodies (lane l holds bodies l and l + 32) and its four warps
// take the four quarters of every j tile.  A cluster of P CTAs (P in {1, 2, 4, 8}) shares one
// group of 64 bodies and splits the j range P ways; the P partial sums are added through
// distributed shared memory, so nothing leaves the cluster before the final sums.  The host
// picks P so that the grid holds about six waves of resident CTAs (eight per SM at <= 64
// registers) -- finer work units, so that every SM stays full to the end instead of running
// a partial last wave.
// Each body's sums are kept per parity of j (the two halves of a pair) and added in a fixed
// order: the halves, the four quarters, then the P cluster ranks -- results are
// deterministic for a given N and P.
#include "common.cuh"

#include <cfloat>
#include <cmath>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace accel {
namespace pair {

constexpr int kThreads = 128;
constexpr int kBodies = 64;   // bodies per CTA (per cluster)
constexpr int kSplit = 4;     // j quarters per tile, one per warp
constexpr int kTile = 512;    // j bodies per shared-memory tile
constexpr int kMaxCluster = 8;

__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One pair of interactions: the j pair (xj, yj, zj, mj) against body i, whose negated
// coordinates are duplicated in (nx, ny, nz).  The arithmetic of each half is that of the
// scalar form: d = p_j - p_i, r = dx^2 + (dy^2 + (dz^2 + eps^2)), s = m r^(-1/2)^3,
// a += s d.
__device__ __forceinline__ void interact2(float2 xj, float2 yj, float2 zj, float2 mj, float2 nx, float2 ny,
                                          float2 nz, float2 e2, float2& ax, float2& ay, float2& az) {
    const float2 dx = __fadd2_rn(xj, nx), dy = __fadd2_rn(yj, ny), dz = __fadd2_rn(zj, nz);
    float2 r = __ffma2_rn(dz, dz, e2);
    r = __ffma2_rn(dy, dy, r);
    r = __ffma2_rn(dx, dx, r);
    const float2 inv = make_float2(rsqrt_ftz(r.x), rsqrt_ftz(r.y));
    const float2 s = __fmul2_rn(__fmul2_rn(__fmul2_rn(mj, inv), inv), inv);
    ax = __ffma2_rn(s, dx, ax);
    ay = __ffma2_rn(s, dy, ay);
    az = __ffma2_rn(s, dz, az);
}

// Launched in clusters of P CTAs along x: cluster c owns bodies [64 c, 64 c + 64), its rank r
// the j range [r per, min(n, (r + 1) per)).
__global__ void __launch_bounds__(kThreads, 8)
k_gravity(const float* __restrict__ X, const float* __restrict__ Y, const float* __restrict__ Z,
          const float* __restrict__ Mass, int64_t n, int64_t per, float eps2, float* __restrict__ AX,
          float* __restrict__ AY, float* __restrict__ AZ) {
    __shared__ __align__(16) float s_x[kTile];
    __shared__ __align__(16) float s_y[kTile];
    __shared__ __align__(16) float s_z[kTile];
    __shared__ __align__(16) float s_m[kTile];
    __shared__ float3 s_part[kSplit][kBodies];
    __shared__ float3 s_sum[kBodies];
    cg::cluster_group cluster = cg::this_cluster();
    const int P = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int t = threadIdx.x;
    const int w = t >> 5;
    const int l = t & 31;
    const int64_t ib = (int64_t)(blockIdx.x / P) * kBodies;
    const int64_t jbeg = rank * per;
    const int64_t jend = jbeg + per < n ? jbeg + per : n;
    const int64_t i0 = ib + l, i1 = ib + l + 32;
    float x0 = 0, y0 = 0, z0 = 0, x1 = 0, y1 = 0, z1 = 0;
    if (i0 < n) { x0 = X[i0]; y0 = Y[i0]; z0 = Z[i0]; }
    if (i1 < n) { x1 = X[i1]; y1 = Y[i1]; z1 = Z[i1]; }
    const float2 nx0 = make_float2(-x0, -x0), ny0 = make_float2(-y0, -y0), nz0 = make_float2(-z0, -z0);
    const float2 nx1 = make_float2(-x1, -x1), ny1 = make_float2(-y1, -y1), nz1 = make_float2(-z1, -z1);
    const float2 e2 = make_float2(eps2, eps2);
    float2 ax0 = make_float2(0.f, 0.f), ay0 = ax0, az0 = ax0, ax1 = ax0, ay1 = ax0, az1 = ax0;

    for (int64_t jb = jbeg; jb < jend; jb += kTile) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTile / kThreads; ++k) {
            // padding bodies (past the range) sit at the origin with zero mass
            const int s = t + k * kThreads;
            const int64_t j = jb + s;
            const bool in = j < jend;
            s_x[s] = in ? X[j] : 0.f;
            s_y[s] = in ? Y[j] : 0.f;
            s_z[s] = in ? Z[j] : 0.f;
            s_m[s] = in ? Mass[j] : 0.f;
        }
        __syncthreads();
        const int q0 = w * (kTile / kSplit);
        const float4* px = reinterpret_cast<const float4*>(s_x + q0);
        const float4* py = reinterpret_cast<const float4*>(s_y + q0);
        const float4* pz = reinterpret_cast<const float4*>(s_z + q0);
        const float4* pm = reinterpret_cast<const float4*>(s_m + q0);
#pragma unroll 2
        for (int g = 0; g < kTile / kSplit / 4; ++g) {
            const float4 bx = px[g], by = py[g], bz = pz[g], bm = pm[g];
            const float2 xa = make_float2(bx.x, bx.y), ya = make_float2(by.x, by.y);
            const float2 za = make_float2(bz.x, bz.y), ma = make_float2(bm.x, bm.y);
            const float2 xb = make_float2(bx.z, bx.w), yb = make_float2(by.z, by.w);
            const float2 zb = make_float2(bz.z, bz.w), mb = make_float2(bm.z, bm.w);
            interact2(xa, ya, za, ma, nx0, ny0, nz0, e2, ax0, ay0, az0);
            interact2(xa, ya, za, ma, nx1, ny1, nz1, e2, ax1, ay1, az1);
            interact2(xb, yb, zb, mb, nx0, ny0, nz0, e2, ax0, ay0, az0);
            interact2(xb, yb, zb, mb, nx1, ny1, nz1, e2, ax1, ay1, az1);
        }
    }
    // this CTA's sums: the two halves of each pair, then the four quarters in order
    s_part[w][l] = make_float3(ax0.x + ax0.y, ay0.x + ay0.y, az0.x + az0.y);
    s_part[w][l + 32] = make_float3(ax1.x + ax1.y, ay1.x + ay1.y, az1.x + az1.y);
    __syncthreads();
    if (t < kBodies) {
        float3 a = s_part[0][t];
#pragma unroll
        for (int r = 1; r < kSplit; ++r) {
            const float3 b = s_part[r][t];
            a.x += b.x; a.y += b.y; a.z += b.z;
        }
        s_sum[t] = a;
    }
    // the cluster's ranks in order; rank r finishes bodies [r 64/P, (r + 1) 64/P)
    cluster.sync();
    const int nb = kBodies / P;
    if (t < nb) {
        const int b = rank * nb + t;
        float3 a = cluster.map_shared_rank(s_sum, 0)[b];
        for (int r = 1; r < P; ++r) {
            const float3 c = cluster.map_shared_rank(s_sum, r)[b];
            a.x += c.x; a.y += c.y; a.z += c.z;
        }
        const int64_t i = ib + b;
        if (i < n) { AX[i] = a.x; AY[i] = a.y; AZ[i] = a.z; }
    }
    cluster.sync();   // no CTA leaves while a peer still reads its sums
}

// Cluster size for n bodies: double P while the grid holds under six waves of resident CTAs
// and every rank keeps at least two j tiles (the best measured P at N = 16,384, 65,536 and
// 262,144 bodies: 8, 8 and 2).
int choose_cluster(int64_t n) {
    static int slots = -1;
    if (slots < 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gravity, kThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
        slots = (per_sm > 0 ? per_sm : 1) * num_sms();
    }
    const int64_t groups = (n + kBodies - 1) / kBodies;
    int P = 1;
    while (P < kMaxCluster && groups * P < 6 * (int64_t)slots && n >= (int64_t)2 * P * 2 * kTile) P *= 2;
    return P;
}

accel_status launch_gravity(const float* d_x, const float* d_y, const float* d_z, const float* d_m, int64_t n,
                            float eps, float* d_ax, float* d_ay, float* d_az, int P, cudaStream_t st) {
    const int64_t groups = (n + kBodies - 1) / kBodies;
    const int64_t per = (n + P - 1) / P;
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.gridDim = dim3((unsigned)(groups * P), 1, 1);
    lc.blockDim = dim3(kThreads, 1, 1);
    lc.dynamicSmemBytes = 0;
    lc.stream = st;
    lc.attrs = attr;
    lc.numAttrs = 1;
    ACCEL_CUDA_TRY(cudaLaunchKernelEx(&lc, k_gravity, d_x, d_y, d_z, d_m, n, per, eps * eps, d_ax, d_ay, d_az));
    return after_launch(st, "pairwise_mapreduce", 1);
}

}  // namespace pair
}  // namespace accel

using namespace accel;

extern "C" {

accel_status pairwise_mapreduce(int32_t op, const float* d_x, const float* d_y, const float* d_z, const float* d_m,
                                int64_t n, float eps, float* d_ax, float* d_ay, float* d_az, void* stream) {
    ACCEL_REQUIRE(op == ACCEL_PAIR_GRAVITY_SOFTENED, ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: bad op %d", op);
    ACCEL_REQUIRE(n >= 0, ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: n < 0");
    // the j = i term (and a padding body's) is 0 * r^(-3/2) with r >= eps^2: it stays 0 only
    // while eps^-3 is finite in FP32, with a margin for the rounding of r and the rsqrt
    ACCEL_REQUIRE(eps > 0.f && std::isfinite(eps) && 1.0 / ((double)eps * eps * eps) <= FLT_MAX / 4.0,
                  ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: eps must be positive and finite with eps^-3 < FLT_MAX/4 (eps = %g)",
                  (double)eps);
    if (n == 0) return ok();
    ACCEL_REQUIRE(d_x && d_y && d_z && d_m && d_ax && d_ay && d_az, ACCEL_ERR_INVALID_ARG, "pairwise_mapreduce: null pointer");
    ACCEL_REQUIRE((n + pair::kBodies - 1) / pair::kBodies * pair::kMaxCluster <= (int64_t)INT32_MAX,
                  ACCEL_ERR_UNSUPPORTED, "pairwise_mapreduce: n too large");
    return pair::launch_gravity(d_x, d_y, d_z, d_m, n, eps, d_ax, d_ay, d_az, pair::choose_cluster(n),
                                as_stream(stream));
}

}  // extern "C"
