// Batched scaled HMM forward on the tensor cores (K8).
//
// The forward recursion (map over states j of a reduce over states i inside a sequential
// loop over t; Appendix A patterns) for a tile of 128 sequences is one dense contraction
// per step:  D = X_{t-1} A  with X the [128 x K] tile of scaled forward vectors.
//   alpha~_t = (X_{t-1} A) o b(o_t),   c'_t = sum_j alpha~_t(j)
//   X_t      = alpha~_t * 2^-e_t       with c'_t = f 2^e_t, f in [0.5, 1)
//   logL     = ln2 * sum_{t<T} e_t + ln c'_T
// Rescaling by an exact power of two keeps X in range like the textbook c_t normalisation
// but leaves no rounding in the log-scale bookkeeping (an integer sum per sequence); only
// the final ln c'_T is evaluated, in FP64.  The HMM itself is not in the paper; this is
// the textbook scaled forward algorithm.
//
// Per CTA (one per SM, persistent): A^T (BF16, the MMA's B operand, N = K rows by K) and
// the emission table b(j, k) (BF16) stay in shared memory for the whole launch; X is the
// MMA's A operand (BF16, 128 x K) in shared memory; D accumulates in FP32 in tensor memory
// (K columns x 128 lanes).  One thread issues the K/16 MMAs of a step (M=128, N=K, K=16
// each) and commits them to an mbarrier; the 128 threads then read their row of D
// (tcgen05.ld), apply the emission, sum, rescale, round to BF16 and write the row of X
// for the next step.  Rows take sequences from a global queue ordered by decreasing
// length; a row whose sequence ends writes logL and starts the next sequence in the same
// step (alpha~_1 = pi o b(o_1)), so uneven lengths are packed in one launch.
#include "common.cuh"
#include "hmm_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace accel {
namespace hmm {

constexpr int kRows = 128;
constexpr int kTcThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;   // bounded mbarrier wait: 2 s of wall clock

struct TcLayout {
    // workspace (after the status block)
    size_t at_off, e_off, pi_off, order_off, order_scratch_off, total;
    // dynamic shared memory
    uint32_t s_at, s_x, s_e, s_pi, s_bar, s_slot, smem_bytes;
};

static TcLayout tc_layout(int K, int M, int64_t S) {
    TcLayout L;
    L.at_off = align_up(kStatusBytes, 1024);
    L.e_off = align_up(L.at_off + (size_t)K * K * 2, 1024);
    L.pi_off = align_up(L.e_off + (size_t)M * K * 2, 1024);
    L.order_off = align_up(L.pi_off + (size_t)K * 4, 256);
    L.order_scratch_off = align_up(L.order_off + (size_t)S * 4, 256);
    L.total = L.order_off + order_ws_bytes(S);
    uint32_t o = 0;
    L.s_at = o; o += (uint32_t)K * K * 2;
    L.s_x = o;  o += (uint32_t)kRows * K * 2;
    L.s_e = o;  o += (uint32_t)M * K * 2;
    L.s_pi = o; o += (uint32_t)K * 4;
    o = (o + 15) & ~15u;
    L.s_bar = o; o += 8;
    L.s_slot = o; o += 8;
    L.smem_bytes = o;
    return L;
}

bool tc_supported(int K, int M) {
    if (K < 32 || K > 256 || K % 32 != 0 || M < 1) return false;
    return (int)tc_layout(K, M, 0).smem_bytes <= max_smem_optin();
}

size_t tc_ws_bytes(int K, int M, int64_t S) { return tc_layout(K, M, S).total; }

// Byte offset of element (row r, col k) in the no-swizzle K-major canonical layout with
// LBO = 128 (core matrices along K contiguous) and SBO = 16 * Kdim.
__host__ __device__ __forceinline__ uint32_t canon_off(int r, int k, int Kdim) {
    return (uint32_t)((r >> 3) * (16 * Kdim) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Emission table row o (symbol), state j: row of K BF16 values whose 16-byte chunks are
// rotated by o, so threads reading the same chunk of different rows hit different banks.
__host__ __device__ __forceinline__ uint32_t etab_off(int o, int j, int K) {
    int nch = K >> 3;
    int q = ((j >> 3) + o) % nch;
    return (uint32_t)(o * K * 2 + q * 16 + (j & 7) * 2);
}

// A^T in canonical layout (B operand: row n = j, column k = i), emission table, pi.
__global__ void k_tc_prep(const float* __restrict__ logA, const float* __restrict__ logB,
                          const float* __restrict__ logpi, int K, int M, char* __restrict__ at,
                          char* __restrict__ etab, float* __restrict__ pi) {
    int64_t nA = (int64_t)K * K, nB = (int64_t)K * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nA + nB + K;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < nA) {
            int i = (int)(idx / K), j = (int)(idx % K);
            *reinterpret_cast<__nv_bfloat16*>(at + canon_off(j, i, K)) = __float2bfloat16_rn(__expf(logA[idx]));
        } else if (idx < nA + nB) {
            int64_t q = idx - nA;
            int j = (int)(q / M), k = (int)(q % M);
            *reinterpret_cast<__nv_bfloat16*>(etab + etab_off(k, j, K)) = __float2bfloat16_rn(__expf(logB[q]));
        } else {
            int j = (int)(idx - nA - nB);
            pi[j] = __expf(logpi[j]);
        }
    }
}

__device__ __forceinline__ float bf_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf_hi(uint32_t x) { return __uint_as_float(x & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_hmm_tc(int K, int M, const char* __restrict__ g_at, const char* __restrict__ g_etab,
         const float* __restrict__ g_pi, const int32_t* __restrict__ obs, const int64_t* __restrict__ off,
         int64_t S, const int32_t* __restrict__ order, unsigned long long* __restrict__ next,
         double* __restrict__ loglik, int32_t* __restrict__ status, TcLayout L) {
    extern __shared__ __align__(1024) char smem[];
    char* sAT = smem + L.s_at;
    char* sX = smem + L.s_x;
    char* sE = smem + L.s_e;
    float* sPi = reinterpret_cast<float*>(smem + L.s_pi);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.s_bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + L.s_slot);
    const int m = threadIdx.x, w = m >> 5;

    // ---- stage A^T, the emission table and pi (linear copies of prepared layouts)
    {
        const int4* src = reinterpret_cast<const int4*>(g_at);
        int4* dst = reinterpret_cast<int4*>(sAT);
        for (int i = m; i < K * K * 2 / 16; i += kTcThreads) dst[i] = src[i];
        src = reinterpret_cast<const int4*>(g_etab);
        dst = reinterpret_cast<int4*>(sE);
        for (int i = m; i < M * K * 2 / 16; i += kTcThreads) dst[i] = src[i];
        for (int i = m; i < K; i += kTcThreads) sPi[i] = g_pi[i];
    }
    const uint32_t ncols = K <= 32 ? 32 : K <= 64 ? 64 : K <= 128 ? 128 : 256;
    if (w == 0) {
        tc::tmem_alloc(slot, ncols);
        tc::tmem_relinquish();
    }
    if (m == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t trow = tmem + ((uint32_t)(w * 32) << 16);   // this warp's lane quarter

    const uint32_t idesc = tc::idesc_bf16_f32(kRows, K);
    const uint32_t sx_addr = tc::smem_u32(sX), sat_addr = tc::smem_u32(sAT);
    const uint32_t sbo = 16u * (uint32_t)K;
    const int nch = K >> 3;

    int64_t seq = -1, T = 0, pos = 0;
    const int32_t* o = nullptr;
    int64_t E = 0;
    bool queue_empty = false, zeroed = false, timed_out = false;

    // write (v[j] * scale) for j in [jc, jc+32) as BF16 into row m of X
    auto store_chunk = [&](int jc, const float (&v)[32], float scale) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint4 pk;
            pk.x = pack_bf16(v[8 * u + 0] * scale, v[8 * u + 1] * scale);
            pk.y = pack_bf16(v[8 * u + 2] * scale, v[8 * u + 3] * scale);
            pk.z = pack_bf16(v[8 * u + 4] * scale, v[8 * u + 5] * scale);
            pk.w = pack_bf16(v[8 * u + 6] * scale, v[8 * u + 7] * scale);
            *reinterpret_cast<uint4*>(sX + canon_off(m, jc + 8 * u, K)) = pk;
        }
    };
    // emission b(j, ob) for j in [jc, jc+32), FP32
    auto load_emis = [&](int ob, int jc, float (&b)[32]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int q = ((jc >> 3) + u + ob) % nch;
            uint4 r = *reinterpret_cast<const uint4*>(sE + ob * K * 2 + q * 16);
            b[8 * u + 0] = bf_lo(r.x); b[8 * u + 1] = bf_hi(r.x);
            b[8 * u + 2] = bf_lo(r.y); b[8 * u + 3] = bf_hi(r.y);
            b[8 * u + 4] = bf_lo(r.z); b[8 * u + 5] = bf_hi(r.z);
            b[8 * u + 6] = bf_lo(r.w); b[8 * u + 7] = bf_hi(r.w);
        }
    };

    for (uint32_t iter = 0;; ++iter) {
        if (iter > 0) {
            bool okw = tc::mbar_wait_bounded(bar, (iter - 1) & 1, kWaitNs);
            timed_out = !okw;
            tc::tc_fence_after();
        }
        if (__syncthreads_or(timed_out)) {
            if (m == 0) atomicExch(status, ACCEL_ERR_TIMEOUT);
            break;
        }
        // ---- epilogue of step `pos` for the row's current sequence.  tcgen05.ld is
        // warp-collective (.sync.aligned): every thread of a warp executes the loads, and
        // rows without a sequence ignore what they read.
        if (iter > 0 && __any_sync(0xffffffffu, seq >= 0)) {
            const bool act = seq >= 0;
            const int ob = act ? o[pos] : 0;
            float csum = 0.f;
            for (int jc = 0; jc < K; jc += 32) {
                uint32_t d[32];
                float b[32];
                tc::tmem_ld32(trow + jc, d);
                load_emis(ob, jc, b);
#pragma unroll
                for (int u = 0; u < 32; ++u) csum = fmaf(__uint_as_float(d[u]), b[u], csum);
            }
            bool cont = false;
            float scale = 1.f;
            if (act) {
                if (pos == T - 1) {
                    loglik[seq] = 0.6931471805599453 * (double)E + log((double)csum);
                    seq = -1;
                } else {
                    int e;
                    frexpf(csum, &e);
                    scale = ldexpf(1.0f, -e);
                    E += e;
                    cont = true;
                }
            }
            if (__any_sync(0xffffffffu, cont)) {
                for (int jc = 0; jc < K; jc += 32) {
                    uint32_t d[32];
                    tc::tmem_ld32(trow + jc, d);
                    if (cont) {
                        float b[32], v[32];
                        load_emis(ob, jc, b);
#pragma unroll
                        for (int u = 0; u < 32; ++u) v[u] = __uint_as_float(d[u]) * b[u];
                        store_chunk(jc, v, scale);
                    }
                }
            }
            if (cont) ++pos;
        }
        // ---- idle row: start the next sequence of the queue (alpha~_1 = pi o b(o_1))
        while (seq < 0 && !queue_empty) {
            unsigned long long q = atomicAdd(next, 1ull);
            if (q >= (unsigned long long)S) { queue_empty = true; break; }
            seq = order[q];
            const int64_t o0 = off[seq];
            T = off[seq + 1] - o0;
            o = obs + o0;
            pos = 0;
            E = 0;
            const int ob = o[0];
            float csum = 0.f;
            for (int jc = 0; jc < K; jc += 32) {
                float b[32];
                load_emis(ob, jc, b);
#pragma unroll
                for (int u = 0; u < 32; ++u) csum = fmaf(sPi[jc + u], b[u], csum);
            }
            if (T == 1) {
                loglik[seq] = log((double)csum);
                seq = -1;
                continue;
            }
            int e;
            frexpf(csum, &e);
            const float scale = ldexpf(1.0f, -e);
            E = e;
            for (int jc = 0; jc < K; jc += 32) {
                float b[32], v[32];
                load_emis(ob, jc, b);
#pragma unroll
                for (int u = 0; u < 32; ++u) v[u] = sPi[jc + u] * b[u];
                store_chunk(jc, v, scale);
            }
            pos = 1;
            zeroed = false;
        }
        if (seq < 0 && !zeroed) {
            float z[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) z[u] = 0.f;
            for (int jc = 0; jc < K; jc += 32) store_chunk(jc, z, 1.f);
            zeroed = true;
        }
        // ---- publish X to the tensor core and issue the next step's MMAs
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        const bool any = __syncthreads_or(seq >= 0);
        if (!any) break;
        if (m == 0) {
            tc::tc_fence_after();
            for (int ks = 0; ks < K / 16; ++ks) {
                uint64_t ad = tc::smem_desc_noswizzle(sx_addr + ks * 256, 128, sbo);
                uint64_t bd = tc::smem_desc_noswizzle(sat_addr + ks * 256, 128, sbo);
                tc::mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(bar);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, ncols);
}

accel_status tc_forward(const accel_hmm_model* mdl, const int32_t* obs, const int64_t* off, int64_t S,
                        double* loglik, char* ws, int32_t* d_status, cudaStream_t st) {
    const int K = mdl->K, M = mdl->M;
    ACCEL_REQUIRE(tc_supported(K, M), ACCEL_ERR_UNSUPPORTED,
                  "hmm_forward(bf16): K must be a multiple of 32 in [32, 256] and the tables must fit shared memory (K=%d, M=%d)", K, M);
    TcLayout L = tc_layout(K, M, S);
    char* at = ws + L.at_off;
    char* et = ws + L.e_off;
    float* pi = (float*)(ws + L.pi_off);
    int32_t* order = (int32_t*)(ws + L.order_off);
    unsigned long long* next = (unsigned long long*)(ws + kQueueOff);   // inside the status block
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + kQueueOff, 0, 8, st));
    int64_t nprep = (int64_t)K * K + (int64_t)K * M + K;
    int pg = (int)((nprep + 255) / 256);
    if (pg > 4 * num_sms()) pg = 4 * num_sms();
    k_tc_prep<<<pg, 256, 0, st>>>(mdl->log_A, mdl->log_B, mdl->log_pi, K, M, at, et, pi);
    accel_status r = order_by_length(off, S, order, ws + L.order_scratch_off, st);
    if (r != ACCEL_OK) return r;
    ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_hmm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes));
    int64_t tiles = (S + kRows - 1) / kRows;
    int grid = (int)(tiles < num_sms() ? tiles : num_sms());
    k_hmm_tc<<<grid, kTcThreads, L.smem_bytes, st>>>(K, M, at, et, pi, obs, off, S, order, next, loglik, d_status, L);
    return after_launch(st, "hmm_forward(bf16 tcgen05)", 5);
}

}  // namespace hmm
}  // namespace accel
