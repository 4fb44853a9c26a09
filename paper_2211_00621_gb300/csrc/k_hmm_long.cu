// Parallel-in-T HMM forward for few, very long sequences.
//
// The forward recursion alpha_1 = pi o b(o_1), alpha_t = (alpha_{t-1} A) o b(o_t) is a chain
// of vector-matrix products alpha_T = alpha_1 M_2 M_3 ... M_T with M_t = A diag(b(o_t)).
// Matrix products are associative, so the chain can be cut into chunks whose products are
// formed independently (the scan/reduce pattern of Appendix A applied to the loop of
// Listing 1; the HMM itself is textbook, not in the paper):
//   phase 1 (k_long_chunk, one CTA per chunk of a sequence):  P_c = prod_{t in chunk} M_t,
//            starting from the identity, one K x K x K product per step;
//   phase 2 (k_long_combine, one CTA per sequence):  v <- v P_c over the chunks in order,
//            logL = log sum_j v_j.
// Depth is T / n_chunks steps instead of T; work is K^3 per step instead of K^2, so this
// pays for sequences far longer than the GPU has parallel lanes for otherwise.
//
// Scaling: a chunk product is kept as diag(2^E) X with one integer exponent per row: after
// every step each row of X is divided by the power of two of its largest entry (exact), and
// the exponent is added to the row's E.  Row scales pass through right-multiplication
// ((D X) A = D (X A)), so no step needs a global reduction.  Phase 2 folds E into the vector
// before each product (shifted by the largest exponent of the rows in use) and keeps the
// vector's own scale as a log2 sum in FP64.
//
// States are padded to KP = 64 (zero rows and columns of A, zero emissions); K <= 64.
// Per step of phase 1 a CTA of 64 threads computes a 64 x 64 x 64 product from shared
// memory (X stored transposed, A row-major; each thread an 8 x 8 block from four float4
// loads per k, packed FP32 FMAs over column pairs), scales the columns by the step's emission (prefetched one step ahead), and
// renormalises its rows with a max over the row's 8 lanes.  FP32 throughout; exponents int32.
#include "common.cuh"
#include "hmm_internal.cuh"

#include <climits>
#include <math.h>

#include "tc_ptx.cuh"

namespace accel {
namespace hmm {
namespace {

constexpr int KP = 64;
constexpr int kChunkThreads = 64;       // chunk products: 8 x 8 outputs per thread

struct LongPrm {
    const float* Ap;        // [KP][KP] exp(log A), zero padded
    const float* BT;        // [M][KP]  exp(log B)^T, zero padded
    const float* log_pi;    // [K]
    int K, M;
    const int32_t* obs;
    const int64_t* off;
    int64_t S;
    int nchunk;             // chunks per sequence
    float* X;               // [S][nchunk][KP][KP] chunk products (row-scaled), row-major
    int32_t* E;             // [S][nchunk][KP] row exponents
    double* loglik;
};

__global__ void k_long_prep(const float* __restrict__ logA, const float* __restrict__ logB, int K, int M,
                            float* __restrict__ Ap, float* __restrict__ BT) {
    const int64_t nA = (int64_t)KP * KP, nB = (int64_t)M * KP;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nA + nB;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < nA) {
            const int i = (int)(idx / KP), j = (int)(idx % KP);
            Ap[idx] = (i < K && j < K) ? expf(logA[(int64_t)i * K + j]) : 0.f;
        } else {
            const int64_t q = idx - nA;
            const int o = (int)(q / KP), j = (int)(q % KP);
            BT[q] = j < K ? expf(logB[(int64_t)j * M + o]) : 0.f;
        }
    }
}

// Steps [t0, t1) of the sequence (obs indices; the matrices M_{t+1} in 1-based terms).
__device__ __forceinline__ void chunk_range(const LongPrm& p, int64_t s, int c, int64_t& o0, int64_t& t0, int64_t& t1) {
    o0 = p.off[s];
    const int64_t T = p.off[s + 1] - o0;
    const int64_t nmat = T > 1 ? T - 1 : 0;
    const int64_t L = (nmat + p.nchunk - 1) / p.nchunk;
    t0 = 1 + (int64_t)c * L;
    t1 = 1 + (int64_t)(c + 1) * L;
    if (t1 > T) t1 = T;
    if (t0 > t1) t0 = t1;
}

// X is stored transposed, row k = column k of X, in 16-byte chunks of 4 entries; chunk q of
// row k sits at chunk position q ^ xsw(k), so that the 8 rows a warp writes in one store hit
// different banks (the readers of a row read whole chunks, unaffected).
__device__ __forceinline__ int xsw(int k) { return (k >> 2) & 7; }

__global__ void __launch_bounds__(kChunkThreads) k_long_chunk(LongPrm p) {
    __shared__ __align__(16) float sA[KP][KP];         // A[k][j]
    __shared__ __align__(16) float sX[2][KP][KP];      // X transposed (chunk-swizzled rows)
    const int c = blockIdx.x;
    const int64_t s = blockIdx.y;
    const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
    // this thread's 8 x 8 block of X A: rows i0..i0+7, columns 4tx..4tx+3 and 32+4tx..32+4tx+3
    // (the two float4 loads of a row of A by a warp then cover all banks once)
    const int i0 = 8 * ty, jA = 4 * tx, jB = 32 + 4 * tx;
    for (int idx = tid; idx < KP * KP / 4; idx += kChunkThreads) {
        reinterpret_cast<float4*>(&sA[0][0])[idx] = reinterpret_cast<const float4*>(p.Ap)[idx];
        const int k = (4 * idx) / KP, i = 4 * (((4 * idx) % KP / 4) ^ xsw(k));   // identity
        reinterpret_cast<float4*>(&sX[0][0][0])[idx] =
            make_float4(k == i ? 1.f : 0.f, k == i + 1 ? 1.f : 0.f, k == i + 2 ? 1.f : 0.f, k == i + 3 ? 1.f : 0.f);
    }
    int64_t o0, t0, t1;
    chunk_range(p, s, c, o0, t0, t1);
    int32_t erow[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float4 bn0 = make_float4(0.f, 0.f, 0.f, 0.f), bn1 = bn0;
    if (t0 < t1) {
        const float* bp = p.BT + (int64_t)p.obs[o0 + t0] * KP;
        bn0 = *reinterpret_cast<const float4*>(bp + jA);
        bn1 = *reinterpret_cast<const float4*>(bp + jB);
    }
    __syncthreads();
    int buf = 0;
    for (int64_t t = t0; t < t1; ++t) {
        // packed FMAs over column pairs: (acc[a][2q], acc[a][2q+1]) += x[a] (A[k][2q], A[k][2q+1])
        float2 acc2[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc2[a][q] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int k = 0; k < KP; ++k) {
            const int sk = xsw(k);
            const float4 xa = *reinterpret_cast<const float4*>(&sX[buf][k][4 * ((2 * ty) ^ sk)]);
            const float4 xb = *reinterpret_cast<const float4*>(&sX[buf][k][4 * ((2 * ty + 1) ^ sk)]);
            const float4 aa = *reinterpret_cast<const float4*>(&sA[k][jA]);
            const float4 ab = *reinterpret_cast<const float4*>(&sA[k][jB]);
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float2 av[4] = {make_float2(aa.x, aa.y), make_float2(aa.z, aa.w), make_float2(ab.x, ab.y),
                                  make_float2(ab.z, ab.w)};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const float2 xx = make_float2(xv[a], xv[a]);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc2[a][q] = __ffma2_rn(xx, av[q], acc2[a][q]);
            }
        }
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[a][2 * q] = acc2[a][q].x;
                acc[a][2 * q + 1] = acc2[a][q].y;
            }
        const float bv[8] = {bn0.x, bn0.y, bn0.z, bn0.w, bn1.x, bn1.y, bn1.z, bn1.w};
        if (t + 1 < t1) {
            const float* bp = p.BT + (int64_t)p.obs[o0 + t + 1] * KP;
            bn0 = *reinterpret_cast<const float4*>(bp + jA);
            bn1 = *reinterpret_cast<const float4*>(bp + jB);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            float m = 0.f;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                acc[a][b] *= bv[b];
                m = fmaxf(m, acc[a][b]);
            }
            // the row's 8 threads are 8 consecutive lanes
#pragma unroll
            for (int d = 1; d < 8; d <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
            const int e = m > 0.f ? ilogbf(m) : 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = ldexpf(acc[a][b], -e);
            erow[a] += e;
        }
        float* dst = &sX[buf ^ 1][0][0];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int j = b < 4 ? jA + b : jB + b - 4;
            const int sj = xsw(j);
            *reinterpret_cast<float4*>(dst + j * KP + 4 * ((2 * ty) ^ sj)) =
                make_float4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
            *reinterpret_cast<float4*>(dst + j * KP + 4 * ((2 * ty + 1) ^ sj)) =
                make_float4(acc[4][b], acc[5][b], acc[6][b], acc[7][b]);
        }
        buf ^= 1;
        __syncthreads();
    }
    const int64_t slot = s * p.nchunk + c;
    float* Xo = p.X + slot * KP * KP;
    for (int idx = tid; idx < KP * KP; idx += kChunkThreads) {
        const int i = idx / KP, j = idx % KP;
        Xo[idx] = sX[buf][j][4 * ((i >> 2) ^ xsw(j)) + (i & 3)];
    }
    if (tx == 0) {
#pragma unroll
        for (int a = 0; a < 8; ++a) p.E[slot * KP + i0 + a] = erow[a];
    }
}

// Block-wide (64 threads) max / sum through shared memory.
__device__ __forceinline__ float block_max64(float v, float* red) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    const float r = fmaxf(red[0], red[1]);
    __syncthreads();
    return r;
}
__device__ __forceinline__ int block_max64i(int v, int* red) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    const int r = max(red[0], red[1]);
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_sum64(double v, double* red) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    const double r = red[0] + red[1];
    __syncthreads();
    return r;
}

// Chunk product `slot` into shared memory with cp.async (16 B per copy, 16 per thread).
__device__ __forceinline__ void prefetch_chunk(const float* X, int64_t slot, float* dst) {
    const float* src = X + slot * KP * KP;
#pragma unroll
    for (int q = 0; q < KP * KP / 4 / KP; ++q) {
        const int idx = (int)threadIdx.x + KP * q;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst + 4 * idx)), "l"(src + 4 * idx)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One CTA of KP threads per sequence: thread j owns v_j.  The chunk products stream
// through two shared-memory buffers, the next one in flight while the current one is used.
__global__ void __launch_bounds__(KP) k_long_combine(LongPrm p) {
    __shared__ __align__(16) float sXc[2][KP * KP];
    __shared__ float su[KP];
    __shared__ float redf[2];
    __shared__ int redi[2];
    __shared__ double redd[2];
    const int64_t s = blockIdx.x;
    const int j = threadIdx.x;
    const int64_t o0 = p.off[s];
    prefetch_chunk(p.X, s * p.nchunk, sXc[0]);
    float v = j < p.K ? expf(p.log_pi[j]) * p.BT[(int64_t)p.obs[o0] * KP + j] : 0.f;
    double l2 = 0.0;                                     // v_true = v 2^l2
    auto renorm = [&]() {
        const float m = block_max64(v, redf);
        const int e = m > 0.f ? ilogbf(m) : 0;
        v = ldexpf(v, -e);
        l2 += (double)e;
    };
    renorm();
    for (int c = 0; c < p.nchunk; ++c) {
        const int64_t slot = s * p.nchunk + c;
        if (c + 1 < p.nchunk) {
            prefetch_chunk(p.X, slot + 1, sXc[(c + 1) & 1]);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        const int ej = p.E[slot * KP + j];
        // u_i = v_i 2^{E_i - Emax} over the rows in use, Emax added to the scale
        const int emax = block_max64i(v > 0.f ? ej : INT_MIN, redi);   // (its barriers publish the copies)
        su[j] = v > 0.f ? ldexpf(v, ej - emax) : 0.f;
        if (emax != INT_MIN) l2 += (double)emax;
        __syncthreads();
        const float* Xc = sXc[c & 1];
        float acc = 0.f;
#pragma unroll 8
        for (int i = 0; i < KP; ++i) acc = fmaf(su[i], Xc[i * KP + j], acc);
        v = acc;
        __syncthreads();                                 // buffer c&1 is refilled two chunks on
        renorm();
    }
    const double tot = block_sum64((double)v, redd);
    if (j == 0) p.loglik[s] = 0.6931471805599453 * l2 + log(tot);
}

struct LongLayout {
    size_t ap_off, bt_off, x_off, e_off, total;
};

LongLayout long_layout(int M, int64_t S, int nchunk) {
    LongLayout L;
    L.ap_off = align_up(kStatusBytes, 256);
    L.bt_off = align_up(L.ap_off + (size_t)KP * KP * 4, 256);
    L.x_off = align_up(L.bt_off + (size_t)M * KP * 4, 256);
    L.e_off = align_up(L.x_off + (size_t)S * nchunk * KP * KP * 4, 256);
    L.total = align_up(L.e_off + (size_t)S * nchunk * KP * 4, 256);
    return L;
}

// Chunks per sequence: about four CTAs per SM in total, each chunk at least 64 steps.
int long_chunks(int64_t S, int64_t max_T) {
    if (S <= 0) return 1;
    const int64_t target = 4LL * num_sms();
    int64_t n = (target + S - 1) / S;
    const int64_t cap = max_T > 1 ? (max_T - 1 + 63) / 64 : 1;
    if (n > cap) n = cap;
    if (n < 1) n = 1;
    if (n > 65535) n = 65535;
    return (int)n;
}

}  // namespace

accel_status check_model(const accel_hmm_model* m, const char* who);

}  // namespace hmm
}  // namespace accel

using namespace accel;
using namespace accel::hmm;

extern "C" {

size_t hmm_forward_long_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T, int64_t max_T) {
    (void)total_T;
    if (!m || S < 0 || max_T < 0) return 0;
    return long_layout(m->M, S, long_chunks(S, max_T)).total;
}

accel_status hmm_forward_long(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets, int64_t S,
                              int64_t total_T, int64_t max_T, double* d_loglik, void* d_ws, size_t ws_bytes,
                              void* stream) {
    accel_status r = check_model(m, "hmm_forward_long");
    if (r != ACCEL_OK) return r;
    ACCEL_REQUIRE(m->K <= KP, ACCEL_ERR_UNSUPPORTED, "hmm_forward_long: K=%d > %d", m->K, KP);
    ACCEL_REQUIRE(S >= 0 && total_T >= 0 && max_T >= 0, ACCEL_ERR_INVALID_ARG, "hmm_forward_long: negative size");
    ACCEL_REQUIRE(d_offsets && d_ws && (S == 0 || (d_loglik && d_obs)), ACCEL_ERR_INVALID_ARG,
                  "hmm_forward_long: null pointer");
    ACCEL_REQUIRE(((uintptr_t)d_ws % 256) == 0, ACCEL_ERR_INVALID_ARG, "hmm_forward_long: d_ws must be 256-byte aligned");
    const size_t need = hmm_forward_long_workspace_size(m, S, total_T, max_T);
    ACCEL_REQUIRE(ws_bytes >= need, ACCEL_ERR_WORKSPACE, "hmm_forward_long: workspace %zu < %zu bytes", ws_bytes, need);
    if (S == 0) return ok();
    ACCEL_REQUIRE(S <= 65535, ACCEL_ERR_UNSUPPORTED, "hmm_forward_long: S=%lld > 65535 sequences", (long long)S);
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    if (debug_mode()) {
        r = debug_check_offsets(d_offsets, S, total_T, 1, ws + kDebugScratchOff, st);
        if (r != ACCEL_OK) return r;
        r = debug_check_symbols(d_obs, total_T, m->M, ws + kDebugScratchOff, st);
        if (r != ACCEL_OK) return r;
    }
    const int nchunk = long_chunks(S, max_T);
    const LongLayout L = long_layout(m->M, S, nchunk);
    LongPrm p;
    p.Ap = (const float*)(ws + L.ap_off);
    p.BT = (const float*)(ws + L.bt_off);
    p.log_pi = m->log_pi;
    p.K = m->K;
    p.M = m->M;
    p.obs = d_obs;
    p.off = d_offsets;
    p.S = S;
    p.nchunk = nchunk;
    p.X = (float*)(ws + L.x_off);
    p.E = (int32_t*)(ws + L.e_off);
    p.loglik = d_loglik;
    const int64_t nprep = (int64_t)KP * KP + (int64_t)m->M * KP;
    int pg = (int)((nprep + 255) / 256);
    if (pg > 4 * num_sms()) pg = 4 * num_sms();
    k_long_prep<<<pg, 256, 0, st>>>(m->log_A, m->log_B, m->K, m->M, (float*)p.Ap, (float*)p.BT);
    k_long_chunk<<<dim3((unsigned)nchunk, (unsigned)S), kChunkThreads, 0, st>>>(p);
    k_long_combine<<<(unsigned)S, KP, 0, st>>>(p);
    return after_launch(st, "hmm_forward_long", 3);
}

}  // extern "C"
