// Batched scaled HMM forward on the tensor cores (K8).
//
// The forward recursion (map over states j of a reduce over states i inside a sequential
// loop over t; Appendix A patterns) for a tile of 128 sequences is one dense contraction
// per step:  D = X_{t-1} A  with X the [128 x K] tile of scaled forward vectors.  The HMM
// itself is not in the paper; this is the textbook scaled forward algorithm, with the
// rescaling done by exact powers of two:
//   alpha~_t = (X_{t-1} A) o b(o_t),   s_t = sum_j alpha~_t(j),   X_t = alpha~_t 2^-k_t
//   logL     = ln2 * sum_{t<T-1} k_t + ln s_{T-1}
// Any integers k_t give the same logL exactly (alpha_t = alpha~_t 2^{k_0+...+k_{t-1}}); they
// only keep X in range.  k_t is predicted one step ahead -- from log2 sum(X_{t-1}) and the
// previous growth ratio s_{t-1} / sum(X_{t-2}) -- so the epilogue makes a single pass over
// the accumulator: the row sum is needed only afterwards.  sum(X_t) then stays within a
// factor of the step-to-step change of the emission scale, with no drift.
//
// Per CTA (one per SM, persistent, 128 x NSPLIT threads; NSPLIT = 2 or 4 column parts per
// row, chosen by the autotuner):
//  * shared memory holds, for the whole launch, A^T (BF16, the MMA's B operand: N = K rows
//    of K, no-swizzle K-major canonical layout) and the emission table b(j, k) (BF16, rows
//    rotated by the symbol so different symbols hit different banks); the X tile
//    (BF16, 128 x K, canonical layout) is the MMA's A operand;
//  * D (FP32, 128 lanes x K columns) accumulates in tensor memory; one thread issues the
//    K/16 tcgen05.mma (M=128, N=K, K=16) of a step and commits them to an mbarrier;
//  * 4 x NSPLIT warps read D back (tcgen05.ld): warps w, w+4, ... share the lane quarter of
//    rows 32(w%4)..+31 and split the columns in NSPLIT parts; each thread multiplies its part
//    of the row by the emission, accumulates its partial row sum, scales by the predicted
//    2^-k, rounds to BF16 and writes its part of the next X row;
//  * while the next step's MMAs run, one thread per row combines the partial sums and
//    advances the row's bookkeeping; when its sequence ends it writes logL and takes the
//    next sequence from a global queue ordered by decreasing length, whose first vector
//    alpha~_0 = pi o b(o_0) the row's threads write in the next epilogue (so uneven lengths
//    are packed into one launch).  The row's next symbol is loaded one step ahead, so no
//    global load sits on the step's critical path.
// All mbarrier waits are bounded (2 s); on expiry the kernel reports ACCEL_ERR_TIMEOUT.  The
// single-CTA kernel also has a watchdog on its whole run time (accel_set_watchdog_ns), checked
// at step boundaries, which stops it cleanly with ACCEL_ERR_TIMEOUT.
#include "common.cuh"
#include "hmm_internal.cuh"
#include "tc_ptx.cuh"

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <map>
#include <mutex>
#include <utility>

namespace accel {
namespace hmm {

constexpr int kRows = 128;
constexpr uint64_t kWaitNs = 2000000000ull;   // bounded mbarrier wait: 2 s of wall clock

struct TcLayout {
    // workspace (after the status block)
    size_t at_off, e_off, order_off, order_scratch_off, total;
    // dynamic shared memory
    uint32_t s_at, s_x, s_e, s_rowinfo, s_psum, s_bar, s_slot, smem_bytes;
};

// Per-row values the column-part threads need (written by the row's owner thread).
struct RowInfo {
    int16_t ob;     // symbol o_t of the step being computed; -1: no sequence; -(o_0 + 2): the
                    // row starts a sequence whose first symbol is o_0
    int16_t k;      // exponent k_t: this step's X_t is scaled by 2^-k_t
};

static TcLayout tc_layout(int K, int M, int64_t S) {
    TcLayout L;
    L.at_off = align_up(kStatusBytes, 1024);
    L.e_off = align_up(L.at_off + (size_t)K * K * 2, 1024);
    L.order_off = align_up(L.e_off + (size_t)M * K * 2, 256);
    L.order_scratch_off = align_up(L.order_off + (size_t)S * 4, 256);
    L.total = L.order_off + order_ws_bytes(S);
    uint32_t o = 0;
    L.s_at = o; o += (uint32_t)K * K * 2;
    L.s_x = o;  o += (uint32_t)kRows * K * 2;
    L.s_e = o;  o += (uint32_t)M * K * 2;
    o = (o + 15) & ~15u;
    L.s_rowinfo = o; o += kRows * (uint32_t)sizeof(RowInfo);
    L.s_psum = o; o += 4 * kRows * 4;
    L.s_bar = o; o += 8;
    L.s_slot = o; o += 8;
    L.smem_bytes = o;
    return L;
}

bool tc_supported(int K, int M) {
    if (K < 64 || K > 256 || K % 64 != 0 || M < 1 || M > 32767) return false;
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

// A^T in canonical layout (B operand: row n = j, column k = i) and the emission table.
__global__ void k_tc_prep(const float* __restrict__ logA, const float* __restrict__ logB, int K, int M,
                          char* __restrict__ at, char* __restrict__ etab) {
    int64_t nA = (int64_t)K * K, nB = (int64_t)K * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nA + nB;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < nA) {
            int i = (int)(idx / K), j = (int)(idx % K);
            *reinterpret_cast<__nv_bfloat16*>(at + canon_off(j, i, K)) = __float2bfloat16_rn(__expf(logA[idx]));
        } else {
            int64_t q = idx - nA;
            int j = (int)(q / M), k = (int)(q % M);
            *reinterpret_cast<__nv_bfloat16*>(etab + etab_off(k, j, K)) = __float2bfloat16_rn(__expf(logB[q]));
        }
    }
}

__device__ __forceinline__ float bf_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf_hi(uint32_t x) { return __uint_as_float(x & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// NSPLIT = column parts per row: 2 (8 warps) or 4 (16 warps; needs K/4 a multiple of 32).
// MT = rows of the MMA tile: 128, or 64 when a CTA runs at most 64 sequence rows (half the
// tensor-core work per step).  With M = 64, row r of D sits in TMEM lane 32 (r / 16) + r % 16,
// so in each warp's lane quarter only lanes 0-15 carry a row.
template <int NSPLIT, int MT>
__global__ void __launch_bounds__(128 * NSPLIT, 1)
k_hmm_tc(int K, int M, const char* __restrict__ g_at, const char* __restrict__ g_etab,
         const float* __restrict__ log_pi, const int32_t* __restrict__ obs, const int64_t* __restrict__ off,
         int64_t S, const int32_t* __restrict__ order, unsigned long long* __restrict__ next, int rows_active,
         double* __restrict__ loglik, int32_t* __restrict__ status, uint64_t watchdog_ns, TcLayout L) {
    extern __shared__ __align__(1024) char smem[];
    char* sAT = smem + L.s_at;
    char* sX = smem + L.s_x;
    char* sE = smem + L.s_e;
    RowInfo* rinfo = reinterpret_cast<RowInfo*>(smem + L.s_rowinfo);
    float* psum = reinterpret_cast<float*>(smem + L.s_psum);        // [NSPLIT][kRows]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.s_bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + L.s_slot);
    constexpr int kThreads = 128 * NSPLIT;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int quarter = w & 3, part = w >> 2;
    constexpr int RPQ = MT / 4;                   // rows per lane quarter
    const bool has_row = lane < RPQ;
    const int row = RPQ * quarter + (has_row ? lane : 0);   // row this thread reads and writes
    const int KH = K / NSPLIT;                    // columns per part
    const int c0 = part * KH;                     // first column of this thread's part
    const int nch = K >> 3;

    // ---- stage A^T and the emission table (linear copies of prepared layouts)
    {
        const int4* src = reinterpret_cast<const int4*>(g_at);
        int4* dst = reinterpret_cast<int4*>(sAT);
        for (int i = tid; i < K * K * 2 / 16; i += kThreads) dst[i] = src[i];
        src = reinterpret_cast<const int4*>(g_etab);
        dst = reinterpret_cast<int4*>(sE);
        for (int i = tid; i < M * K * 2 / 16; i += kThreads) dst[i] = src[i];
    }
    const uint32_t ncols = K <= 64 ? 64 : K <= 128 ? 128 : 256;
    if (w == 0) {
        tc::tmem_alloc(slot, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;

    const uint32_t idesc = tc::idesc_bf16_f32(MT, K);
    const uint32_t sx_addr = tc::smem_u32(sX), sat_addr = tc::smem_u32(sAT);
    const uint32_t sbo = 16u * (uint32_t)K;
    const uint64_t adesc0 = tc::smem_desc_noswizzle(sx_addr, 128, sbo);
    const uint64_t bdesc0 = tc::smem_desc_noswizzle(sat_addr, 128, sbo);

    // row bookkeeping, kept by the row's owner thread (part 0)
    const bool owner = part == 0 && has_row;
    int64_t seq = -1, T = 0, pos = 0, E = 0;
    const int32_t* o = nullptr;
    int32_t nob = 0;             // o[pos + 1], loaded one step ahead of its use
    int32_t kcur = 0;            // exponent applied to this step's X
    float uprev = 0.f;           // log2 sum(X_{t-1})
    bool queue_empty = !has_row || row >= rows_active;   // rows past rows_active never take sequences
    volatile uint32_t* s_flag = slot + 1;                 // set by a thread whose wait timed out
    if (tid == 0) *s_flag = 0;
    // watchdog: when the launch has run longer than watchdog_ns (0 = no limit), thread 0 stops
    // it at the next step boundary -- after the previous step's MMAs have completed and before
    // new ones are issued, so no tensor-core work is in flight -- and every thread leaves
    // through the normal exit that frees the tensor memory
    const uint64_t t_launch = watchdog_ns != 0 ? tc::globaltimer_ns() : 0;

    // emission b(j, ob) for j in [jc, jc+32), FP32, times `scale` (a power of two: exact)
    auto load_emis = [&](int ob, int jc, float (&b)[32], float scale) {
        const int qb = ((jc >> 3) + ob) % nch;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = qb + u < nch ? qb + u : qb + u - nch;
            uint4 r = *reinterpret_cast<const uint4*>(sE + ob * K * 2 + q * 16);
            b[8 * u + 0] = bf_lo(r.x) * scale; b[8 * u + 1] = bf_hi(r.x) * scale;
            b[8 * u + 2] = bf_lo(r.y) * scale; b[8 * u + 3] = bf_hi(r.y) * scale;
            b[8 * u + 4] = bf_lo(r.z) * scale; b[8 * u + 5] = bf_hi(r.z) * scale;
            b[8 * u + 6] = bf_lo(r.w) * scale; b[8 * u + 7] = bf_hi(r.w) * scale;
        }
    };
    // row values of columns [jc, jc+32): X = a o bs (a = D, or pi for a fresh row), packed to
    // BF16 and stored; returns their sum (a fixed pairwise tree)
    auto epi_chunk = [&](const float* a, const float (&bs)[32], int jc) -> float {
        float part8[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = a[8 * u + e] * bs[8 * u + e];
            uint4 pk;
            pk.x = pack_bf16(v[0], v[1]);
            pk.y = pack_bf16(v[2], v[3]);
            pk.z = pack_bf16(v[4], v[5]);
            pk.w = pack_bf16(v[6], v[7]);
            *reinterpret_cast<uint4*>(sX + canon_off(row, jc + 8 * u, K)) = pk;
            part8[2 * u] = (v[0] + v[1]) + (v[2] + v[3]);
            part8[2 * u + 1] = (v[4] + v[5]) + (v[6] + v[7]);
        }
        return ((part8[0] + part8[1]) + (part8[2] + part8[3])) + ((part8[4] + part8[5]) + (part8[6] + part8[7]));
    };
    // take the next sequence of the queue on this row (owner thread).  Its first vector
    // alpha~_0 = pi o b(o_0) (unscaled: k_0 = 0) is written by the row's epilogue threads in
    // the next epilogue, flagged by rinfo.ob = -(o_0 + 2).
    auto take_next = [&]() {
        seq = -1;
        if (!queue_empty) {
            const unsigned long long q = atomicAdd(next, 1ull);
            if (q >= (unsigned long long)S) {
                queue_empty = true;
            } else {
                seq = order[q];
                const int64_t o0 = off[seq];
                T = off[seq + 1] - o0;
                o = obs + o0;
                pos = 0;
                E = 0;
                kcur = 0;
                nob = T > 1 ? o[1] : 0;
                rinfo[row].ob = (int16_t)(-(o[0] + 2));
                rinfo[row].k = 0;
                return;
            }
        }
        rinfo[row].ob = -1;
        rinfo[row].k = 0;
    };

    // Step loop.  Iteration i: (A) X is complete -> one thread issues the MMAs D = X A;
    // meanwhile the owners process the row sums of the previous epilogue (logL at a
    // sequence's end, the next exponent, the next symbol, or the next sequence); (B) every
    // thread waits for the MMAs and writes the next X (or a fresh row's alpha~_0).
    if (owner) take_next();
    for (uint32_t iter = 0;; ++iter) {
        // ---- (A) publish X; the MMAs of this iteration
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        if (watchdog_ns != 0 && tid == 0 && tc::globaltimer_ns() - t_launch > watchdog_ns) *s_flag = 2;
        const bool any = __syncthreads_or(owner && seq >= 0);
        if (*s_flag != 0) {
            if (tid == 0) report_status(status, ACCEL_ERR_TIMEOUT);
            break;
        }
        if (!any) break;
        if (tid == kRows) {              // a thread of column part 1: never a row owner
            tc::tc_fence_after();
            // k-step ks is 256 bytes further: 16 in the descriptors' address field
            uint64_t ad = adesc0, bd = bdesc0;
            tc::mma_bf16(tmem, ad, bd, idesc, 0u);
            for (int ks = 1; ks < K / 16; ++ks) {
                ad += 16;
                bd += 16;
                tc::mma_bf16(tmem, ad, bd, idesc, 1u);
            }
            tc::mma_commit(bar);
        }
        // ---- bookkeeping of the previous epilogue's rows (owner threads), overlapping the MMAs
        if (owner && seq >= 0 && iter > 0) {
            float s = psum[row];
#pragma unroll
            for (int q = 1; q < NSPLIT; ++q) s += psum[q * kRows + row];
            if (pos == T - 1) {
                loglik[seq] = 0.6931471805599453 * (double)E + log((double)s);
                take_next();
            } else {
                E += kcur;
                const float ls = __log2f(s);
                const float u = ls - (float)kcur;       // log2 sum(X_t)
                const float lr = pos == 0 ? ls : ls - uprev;   // log2 of the growth sum(X_{t-1}) -> s_t
                uprev = u;
                kcur = (int)rintf(u + lr);
                ++pos;
                rinfo[row].ob = (int16_t)nob;
                rinfo[row].k = (int16_t)kcur;
                nob = pos + 1 < T ? o[pos + 1] : 0;
            }
        }
        __syncthreads();
        // ---- (B) epilogue
        const RowInfo ri = rinfo[row];
        const bool fresh = has_row && ri.ob <= -2;
        const bool act = has_row && ri.ob >= 0;
        const int ob = fresh ? -ri.ob - 2 : ri.ob;
        const float mult = ldexpf(1.0f, -(int)ri.k);
        // the first chunk's emission (scaled by 2^-k) is read while the MMAs run
        float bs[32];
        if (act || fresh) load_emis(ob, c0, bs, mult);
        const bool ok = tc::mbar_wait_bounded(bar, iter & 1, kWaitNs);
        if (!ok) *s_flag = 1;
        tc::tc_fence_after();
        // each thread's part of the row of D (tcgen05.ld is warp-collective); the row sum is
        // accumulated over the scaled values and unscaled by 2^k (exact) at the end
        float ps = 0.f;
        if (__any_sync(0xffffffffu, act)) {
            if (KH % 64 == 0) {
                for (int jc = 0; jc < KH; jc += 64) {
                    uint32_t d[64];
                    tc::tmem_ld64(taddr + jc, d);
                    if (act) {
                        if (jc > 0) load_emis(ob, c0 + jc, bs, mult);
                        ps += epi_chunk(reinterpret_cast<const float*>(d), bs, c0 + jc);
                        load_emis(ob, c0 + jc + 32, bs, mult);
                        ps += epi_chunk(reinterpret_cast<const float*>(d) + 32, bs, c0 + jc + 32);
                    }
                }
            } else {
                for (int jc = 0; jc < KH; jc += 32) {
                    uint32_t d[32];
                    tc::tmem_ld32(taddr + jc, d);
                    if (act) {
                        if (jc > 0) load_emis(ob, c0 + jc, bs, mult);
                        ps += epi_chunk(reinterpret_cast<const float*>(d), bs, c0 + jc);
                    }
                }
            }
            ps *= ldexpf(1.0f, (int)ri.k);
        }
        if (fresh) {
            // alpha~_0 = pi o b(o_0) for this thread's columns
            for (int jc = 0; jc < KH; jc += 32) {
                if (jc > 0) load_emis(ob, c0 + jc, bs, 1.f);
                float pv[32];
#pragma unroll
                for (int u = 0; u < 32; ++u) pv[u] = __expf(log_pi[c0 + jc + u]);
                ps += epi_chunk(pv, bs, c0 + jc);
            }
        }
        if (has_row) psum[part * kRows + row] = ps;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, ncols);
}

// ============================================================================================
// Cluster-pair variant.  The two CTAs of a cluster run the same tile of sequence rows and
// split the state columns: CTA r computes D_r = X A[:, r K/2 : (r+1) K/2] (MMA N = K/2, half
// the tensor-core time of a step), holds only its half of A^T and of the emission table, and
// runs the epilogue of its own columns (half the per-row work).  Each CTA writes its half of
// X_t into its own tile and, with st.async, into its peer's, together with its partial row
// sums; the stores count their bytes on the receiver's mbarrier of that step's parity, so a
// CTA waits for its peer's half with no cluster barrier per step -- and only after issuing the
// MMAs over its own half of X (half of the K/16 k-steps), which hide the exchange latency.
// X is double-buffered by
// step parity: a peer can be one step ahead and must not overwrite the tile the MMA reads.
// Both CTAs do the same row bookkeeping on the same sums (added in the same order), so they
// agree on every exponent and on the end of every sequence; CTA 0 alone writes logL and pops
// the sequence queue, and sends the popped index to CTA 1 in the same exchange.  A row that
// takes a new sequence this way idles for one step while the index travels.
// ============================================================================================
struct PairLayout {
    uint32_t s_at, s_x, x_bytes, s_e, s_rowinfo, s_psum, s_mail, s_bar, s_slot, smem_bytes;
};

// NC = CTAs of the cluster (2 or 4); each holds KC = K / NC state columns.
static PairLayout pair_layout(int K, int M, int MT, int NSPLIT, int NC) {
    PairLayout L;
    const uint32_t KC = (uint32_t)(K / NC);
    uint32_t o = 0;
    L.s_at = o; o += KC * (uint32_t)K * 2;                 // this CTA's part of A^T (N = K/NC rows)
    L.x_bytes = (uint32_t)MT * (uint32_t)K * 2;
    L.s_x = o;  o += 2 * L.x_bytes;                        // X, one buffer per step parity
    L.s_e = o;  o += (uint32_t)M * KC * 2;                 // emission columns of this part
    o = (o + 15) & ~15u;
    L.s_rowinfo = o; o += (uint32_t)MT * (uint32_t)sizeof(RowInfo);
    L.s_psum = o; o += 2 * (uint32_t)NC * (uint32_t)NSPLIT * (uint32_t)MT * 4;   // [parity][cta][part][row]
    L.s_mail = o; o += 2 * (uint32_t)MT * 4;                                     // [parity][row] popped index
    o = (o + 7) & ~7u;
    L.s_bar = o; o += 3 * 8;                                          // MMA, exchange x 2 parities
    L.s_slot = o; o += 8;
    L.smem_bytes = o;
    return L;
}

bool tc_cl_supported(int K, int M, int rows, int split, int nc) {
    if (nc != 2 && nc != 4) return false;
    if (K < 64 * nc || K > 256 || K % 64 != 0 || M < 1 || M > 32767 || (split != 2 && split != 4)) return false;
    if ((K / nc / split) % 32 != 0) return false;
    const int MT = rows <= 64 ? 64 : 128;
    return (int)pair_layout(K, M, MT, split, nc).smem_bytes <= max_smem_optin();
}

// Launched with a cluster of NC CTAs (cudaLaunchKernelEx, cluster-dimension attribute).
template <int NSPLIT, int MT, int NC>
__global__ void __launch_bounds__(128 * NSPLIT, 1)
k_hmm_tc_pair(int K, int M, const char* __restrict__ g_at, const char* __restrict__ g_etab,
              const float* __restrict__ log_pi, const int32_t* __restrict__ obs, const int64_t* __restrict__ off,
              int64_t S, const int32_t* __restrict__ order, unsigned long long* __restrict__ next, int rows_active,
              double* __restrict__ loglik, int32_t* __restrict__ status, PairLayout L) {
    extern __shared__ __align__(1024) char smem[];
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int cid = (int)(blockIdx.x / NC), ncl = (int)(gridDim.x / NC);
    char* sAT = smem + L.s_at;
    char* sX = smem + L.s_x;
    char* sE = smem + L.s_e;
    RowInfo* rinfo = reinterpret_cast<RowInfo*>(smem + L.s_rowinfo);
    float* psum = reinterpret_cast<float*>(smem + L.s_psum);
    int32_t* mail = reinterpret_cast<int32_t*>(smem + L.s_mail);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.s_bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + L.s_slot);
    constexpr int kThreads = 128 * NSPLIT;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int quarter = w & 3, part = w >> 2;
    // MT = 128: row 32 q + lane of lane quarter q, one thread per row and part.  MT = 64: the
    // rows sit in lanes 0-15 of each quarter, and threads t and t + 16 share row 16 q + t%16,
    // each taking half of the part's columns (16-lane TMEM loads).
    constexpr bool HL = MT == 64;
    const int hsel = HL ? lane >> 4 : 0;
    const int row = HL ? 16 * quarter + (lane & 15) : 32 * quarter + lane;
    const int KC = K / NC;                        // columns of this CTA
    const int KH = KC / NSPLIT;                   // columns per part
    const int CPT = HL ? KH / 2 : KH;             // columns per thread
    const int l0 = part * KH;                     // first column of the part, within the half
    const int lt = l0 + hsel * CPT;               // first column of this thread, within the half
    const int gt = rank * KC + lt;                // ... and in the full row
    const int nch = K >> 3, nchh = KC >> 3;

    // ---- stage this half of A^T (rows rank*KC.. of the canonical layout are one block) and
    // the emission columns of this half (16-byte chunks re-rotated within the half)
    {
        const int4* src = reinterpret_cast<const int4*>(g_at + (size_t)rank * KC * K * 2);
        int4* dst = reinterpret_cast<int4*>(sAT);
        for (int i = tid; i < KC * K * 2 / 16; i += kThreads) dst[i] = src[i];
        for (int i = tid; i < M * nchh; i += kThreads) {
            const int ob = i / nchh, c = i - ob * nchh;
            const int qs = (rank * nchh + c + ob) % nch, qd = (c + ob) % nchh;
            reinterpret_cast<int4*>(sE + (size_t)ob * KC * 2)[qd] =
                reinterpret_cast<const int4*>(g_etab + (size_t)ob * K * 2)[qs];
        }
        for (int i = tid; i < 2 * MT; i += kThreads) mail[i] = -1;
    }
    if (w == 0) {
        tc::tmem_alloc(slot, (uint32_t)KC);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_init(&bar[2], 1);
        tc::fence_mbar_init();
    }
    volatile uint32_t* s_flag = slot + 1;
    if (tid == 0) *s_flag = 0;
    tc::tc_fence_before();
    cl.sync();                                    // both CTAs' barriers exist before any st.async
    tc::tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(HL ? l0 : lt);
    const uint32_t idesc = tc::idesc_bf16_f32(MT, KC);
    const uint32_t sx_addr = tc::smem_u32(sX), sat_addr = tc::smem_u32(sAT);
    const uint32_t sbo = 16u * (uint32_t)K;
    // the other CTAs of the cluster, d = 1 .. NC-1: CTA (rank + d) % NC
    uint32_t rx[NC - 1], rpsum[NC - 1], rmail[NC - 1], rbar0[NC - 1], rbar1[NC - 1];
#pragma unroll
    for (int d = 1; d < NC; ++d) {
        const uint32_t pr = (uint32_t)((rank + d) % NC);
        rx[d - 1] = tc::cluster_addr(sX, pr);
        rpsum[d - 1] = tc::cluster_addr(psum, pr);
        rmail[d - 1] = tc::cluster_addr(mail, pr);
        rbar0[d - 1] = tc::cluster_addr(&bar[1], pr);
        rbar1[d - 1] = tc::cluster_addr(&bar[2], pr);
    }
    // bytes a CTA receives per step: the other CTAs' parts of X and partial sums, and (CTAs
    // other than 0) the indices CTA 0 popped
    const uint32_t xbytes = (uint32_t)((NC - 1) * (MT * KC * 2 + MT * NSPLIT * 4) + (rank != 0 ? MT * 4 : 0));

    const bool owner = part == 0 && hsel == 0;
    int64_t seq = -1, T = 0, pos = 0, E = 0;     // seq: -1 none, -2 waiting for CTA 0's index
    const int32_t* o = nullptr;
    int32_t nob = 0;
    int32_t kcur = 0;
    float uprev = 0.f;
    bool queue_empty = row >= rows_active;
    const int64_t qbase = (int64_t)rows_active * ncl;   // the first rows_active x ncl entries are dealt out

    // emission b(j, ob) for the 16 columns [jc, jc+16) of this half, times `scale` (a power of two)
    auto load_emis = [&](int ob, int jc, float (&b)[16], float scale) {
        const int qb = ((jc >> 3) + ob) % nchh;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = qb + u < nchh ? qb + u : qb + u - nchh;
            uint4 r = *reinterpret_cast<const uint4*>(sE + ob * KC * 2 + q * 16);
            b[8 * u + 0] = bf_lo(r.x) * scale; b[8 * u + 1] = bf_hi(r.x) * scale;
            b[8 * u + 2] = bf_lo(r.y) * scale; b[8 * u + 3] = bf_hi(r.y) * scale;
            b[8 * u + 4] = bf_lo(r.z) * scale; b[8 * u + 5] = bf_hi(r.z) * scale;
            b[8 * u + 6] = bf_lo(r.w) * scale; b[8 * u + 7] = bf_hi(r.w) * scale;
        }
    };
    // columns [jc, jc+16) of this half: X = a o bs packed to BF16 into the buffer at xo of both
    // CTAs; returns their sum (a fixed pairwise tree)
    auto epi16 = [&](const float* a, const float (&bs)[16], int jc, uint32_t xo, const uint32_t (&rb)[NC - 1]) -> float {
        float part4[4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = a[8 * u + e] * bs[8 * u + e];
            uint4 pk;
            pk.x = pack_bf16(v[0], v[1]);
            pk.y = pack_bf16(v[2], v[3]);
            pk.z = pack_bf16(v[4], v[5]);
            pk.w = pack_bf16(v[6], v[7]);
            const uint32_t co = xo + canon_off(row, rank * KC + jc + 8 * u, K);
            *reinterpret_cast<uint4*>(sX + co) = pk;
#pragma unroll
            for (int d = 0; d < NC - 1; ++d) tc::st_async_u4(rx[d] + co, pk, rb[d]);
            part4[2 * u] = (v[0] + v[1]) + (v[2] + v[3]);
            part4[2 * u + 1] = (v[4] + v[5]) + (v[6] + v[7]);
        }
        return (part4[0] + part4[1]) + (part4[2] + part4[3]);
    };
    auto start = [&](int32_t sq) {
        seq = sq;
        const int64_t o0 = off[sq];
        T = off[sq + 1] - o0;
        o = obs + o0;
        pos = 0;
        E = 0;
        kcur = 0;
        nob = T > 1 ? o[1] : 0;
        rinfo[row].ob = (int16_t)(-(o[0] + 2));
        rinfo[row].k = 0;
    };
    auto idle = [&](int64_t state) {
        seq = state;
        rinfo[row].ob = -1;
        rinfo[row].k = 0;
    };
    if (owner) {
        const int64_t q0 = (int64_t)row * ncl + cid;
        if (row < rows_active && q0 < S) start(order[q0]);
        else idle(-1);
    }

    uint32_t xph = 0;                             // bit p: parity of the next completion of exchange barrier p
    // bounded wait for the peer's bytes of step parity q
    auto xchg_wait = [&](int q) {
        const uint32_t ph = (xph >> q) & 1u;
        uint64_t t0 = 0;
        for (uint32_t i = 0;; ++i) {
            if (tc::mbar_try_wait_cluster(&bar[1 + q], ph)) break;
            if ((i & 255) == 0) {
                const uint64_t now = tc::globaltimer_ns();
                if (i == 0) t0 = now;
                else if (now - t0 > kWaitNs) { *s_flag = 1; break; }
            }
        }
        xph ^= 1u << q;
    };
    const int ks_own = rank * (KC / 16);
    // descriptors of k-step 0 of X buffer 0 and of A^T; a k-step is 256 bytes further (16 in
    // the descriptor's address field), a buffer x_bytes
    const uint64_t adesc0 = tc::smem_desc_noswizzle(sx_addr, 128, sbo);
    const uint64_t bdesc0 = tc::smem_desc_noswizzle(sat_addr, 128, sbo);
    const int nks = KC / 16;
    for (uint32_t iter = 0;; ++iter) {
        const int par = (int)(iter & 1u);
        // ---- (A) this CTA's half of X_{t-1} is complete (buffer par^1): its MMAs start while
        // the peer's half is still in flight
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        const bool any = __syncthreads_or(owner && seq != -1);
        if (*s_flag != 0 || !any) {
            if (*s_flag != 0 && tid == 0) report_status(status, ACCEL_ERR_TIMEOUT);
            if (iter > 0) xchg_wait(par ^ 1);     // the peer's last stores have landed (bounded)
            break;
        }
        const uint64_t xdesc = adesc0 + (uint64_t)((par ^ 1) * (L.x_bytes >> 4));
        if (tid == kRows) {                       // a thread of column part 1: never a row owner
            tc::tc_fence_after();
            uint64_t ad = xdesc + (uint64_t)(ks_own * 16), bd = bdesc0 + (uint64_t)(ks_own * 16);
            tc::mma_bf16(tmem, ad, bd, idesc, 0u);
            for (int u = 1; u < nks; ++u) {
                ad += 16;
                bd += 16;
                tc::mma_bf16(tmem, ad, bd, idesc, 1u);
            }
        }
        // the peer's half of X_{t-1}, its row sums and (CTA 1) the indices it popped
        if (iter > 0) xchg_wait(par ^ 1);
        if (tid == kRows) {
            tc::fence_proxy_async_smem();         // the peers' stores, seen through the barrier, to the tensor core
#pragma unroll
            for (int d = 1; d < NC; ++d) {
                const int ks_peer = ((rank + d) % NC) * (KC / 16);
                uint64_t ad = xdesc + (uint64_t)(ks_peer * 16), bd = bdesc0 + (uint64_t)(ks_peer * 16);
                for (int u = 0; u < nks; ++u) {
                    tc::mma_bf16(tmem, ad, bd, idesc, 1u);
                    ad += 16;
                    bd += 16;
                }
            }
            tc::mma_commit(&bar[0]);
        }
        // ---- bookkeeping of the previous step's rows (both CTAs alike), overlapping the MMAs
        if (owner && iter > 0) {
            const int pp = par ^ 1;
            if (seq == -2) {
                const int32_t sq = mail[pp * MT + row];
                if (sq >= 0) start(sq);
                else idle(-1);
            } else if (seq >= 0) {
                float s = 0.f;                    // the same order in every CTA of the cluster
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int q = 0; q < NSPLIT; ++q) s += psum[((pp * NC + c) * NSPLIT + q) * MT + row];
                if (pos == T - 1) {
                    if (rank == 0) {
                        loglik[seq] = 0.6931471805599453 * (double)E + log((double)s);
                        int32_t sq = -1;
                        if (!queue_empty) {
                            const int64_t q = qbase + (int64_t)atomicAdd(next, 1ull);
                            if (q >= S) queue_empty = true;
                            else sq = order[q];
                        }
                        mail[par * MT + row] = sq;
                    }
                    idle(-2);
                } else {
                    E += kcur;
                    const float ls = __log2f(s);
                    const float u = ls - (float)kcur;
                    const float lr = pos == 0 ? ls : ls - uprev;
                    uprev = u;
                    kcur = (int)rintf(u + lr);
                    ++pos;
                    rinfo[row].ob = (int16_t)nob;
                    rinfo[row].k = (int16_t)kcur;
                    nob = pos + 1 < T ? o[pos + 1] : 0;
                }
            }
        }
        uint32_t rb[NC - 1];
#pragma unroll
        for (int d = 0; d < NC - 1; ++d) rb[d] = par ? rbar1[d] : rbar0[d];
        if (rank == 0 && owner)
#pragma unroll
            for (int d = 0; d < NC - 1; ++d)
                tc::st_async_u1(rmail[d] + 4u * (uint32_t)(par * MT + row), (uint32_t)mail[par * MT + row], rb[d]);
        __syncthreads();
        // ---- (B) epilogue of this CTA's columns into buffer par of both CTAs
        const RowInfo ri = rinfo[row];
        const bool fresh = ri.ob <= -2;
        const bool act = ri.ob >= 0;
        const int ob = fresh ? -ri.ob - 2 : ri.ob;
        const float mult = ldexpf(1.0f, -(int)ri.k);
        const uint32_t xo = (uint32_t)par * L.x_bytes;
        float bs[16];
        if (act || fresh) load_emis(ob, lt, bs, mult);
        const bool ok = tc::mbar_wait_bounded(&bar[0], iter & 1u, kWaitNs);
        if (!ok) *s_flag = 1;
        tc::tc_fence_after();
        float ps = 0.f;
        if (__any_sync(0xffffffffu, act)) {
            if (HL) {
                if (CPT == 16) {
                    uint32_t d[16];
                    tc::tmem_ld16x2_16(taddr, d);
                    if (act) ps = epi16(reinterpret_cast<const float*>(d), bs, lt, xo, rb);
                } else {
                    uint32_t d[32];
                    tc::tmem_ld16x2_32(taddr, d);
                    if (act) {
                        ps = epi16(reinterpret_cast<const float*>(d), bs, lt, xo, rb);
                        load_emis(ob, lt + 16, bs, mult);
                        ps += epi16(reinterpret_cast<const float*>(d) + 16, bs, lt + 16, xo, rb);
                    }
                }
            } else {
                for (int jc = 0; jc < CPT; jc += 32) {
                    uint32_t d[32];
                    tc::tmem_ld32(taddr + jc, d);
                    if (act) {
                        if (jc > 0) load_emis(ob, lt + jc, bs, mult);
                        ps += epi16(reinterpret_cast<const float*>(d), bs, lt + jc, xo, rb);
                        load_emis(ob, lt + jc + 16, bs, mult);
                        ps += epi16(reinterpret_cast<const float*>(d) + 16, bs, lt + jc + 16, xo, rb);
                    }
                }
            }
            ps *= ldexpf(1.0f, (int)ri.k);
        }
        if (fresh) {
            // alpha~_0 = pi o b(o_0) for this thread's columns
            for (int jc = 0; jc < CPT; jc += 16) {
                if (jc > 0) load_emis(ob, lt + jc, bs, 1.f);
                float pv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) pv[u] = __expf(log_pi[gt + jc + u]);
                ps += epi16(pv, bs, lt + jc, xo, rb);
            }
        }
        if (!act && !fresh) {
            // no sequence on the row: zeros keep the peer's byte count fixed
            for (int jc = 0; jc < CPT; jc += 8) {
                const uint32_t co = xo + canon_off(row, gt + jc, K);
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(sX + co) = z;
#pragma unroll
                for (int d = 0; d < NC - 1; ++d) tc::st_async_u4(rx[d] + co, z, rb[d]);
            }
        }
        if (HL) ps += __shfl_xor_sync(0xffffffffu, ps, 16);   // the row's two threads
        if (hsel == 0) {
            const int idx = ((par * NC + rank) * NSPLIT + part) * MT + row;
            psum[idx] = ps;
#pragma unroll
            for (int d = 0; d < NC - 1; ++d) tc::st_async1(rpsum[d] + 4u * (uint32_t)idx, ps, rb[d]);
        }
        // the peer's bytes of this step complete the barrier's phase (waited for next step)
        if (tid == 0) tc::mbar_arrive_expect_tx(&bar[1 + par], xbytes);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tmem, (uint32_t)KC);
    cl.sync();                                    // the peer no longer addresses this CTA's shared memory
}

// Clusters of nc CTAs of a cluster kernel that fit on the device at once (cached per kernel).
template <typename Kern>
static int pair_max_clusters(Kern kern, uint32_t smem, int threads, int nc) {
    static std::mutex mu;
    static std::map<std::pair<const void*, uint32_t>, int> cache;
    const auto key = std::make_pair(reinterpret_cast<const void*>(kern), smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(num_sms() / nc * nc), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    cache[key] = n;
    return n;
}

template <int NC>
static accel_status tc_forward_cluster(const accel_hmm_model* mdl, const int32_t* obs, const int64_t* off, int64_t S,
                                       double* loglik, char* ws, int32_t* d_status, TcConfig cfg, cudaStream_t st) {
    const int K = mdl->K, M = mdl->M;
    ACCEL_REQUIRE(tc_cl_supported(K, M, cfg.rows, cfg.split, NC), ACCEL_ERR_UNSUPPORTED,
                  "hmm_forward(bf16, cluster of %d): unsupported configuration (K=%d, M=%d, split=%d, rows=%d)", NC, K,
                  M, cfg.split, cfg.rows);
    const int MT = cfg.rows <= 64 ? 64 : 128;
    const PairLayout P = pair_layout(K, M, MT, cfg.split, NC);
    TcLayout L = tc_layout(K, M, S);
    char* at = ws + L.at_off;
    char* et = ws + L.e_off;
    int32_t* order = (int32_t*)(ws + L.order_off);
    unsigned long long* next = (unsigned long long*)(ws + kQueueOff);
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + kQueueOff, 0, 8, st));
    int64_t nprep = (int64_t)K * K + (int64_t)K * M;
    int pg = (int)((nprep + 255) / 256);
    if (pg > 4 * num_sms()) pg = 4 * num_sms();
    k_tc_prep<<<pg, 256, 0, st>>>(mdl->log_A, mdl->log_B, K, M, at, et);
    accel_status r = order_by_length(off, S, order, ws + L.order_scratch_off, st);
    if (r != ACCEL_OK) return r;
    auto kern = cfg.split == 4 ? (MT == 64 ? k_hmm_tc_pair<4, 64, NC> : k_hmm_tc_pair<4, 128, NC>)
                               : (MT == 64 ? k_hmm_tc_pair<2, 64, NC> : k_hmm_tc_pair<2, 128, NC>);
    ACCEL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem_bytes));
    const int threads = 128 * cfg.split;
    const int maxcl = pair_max_clusters(kern, P.smem_bytes, threads, NC);
    ACCEL_REQUIRE(maxcl > 0, ACCEL_ERR_UNSUPPORTED, "hmm_forward(bf16): no cluster of %d CTAs fits the device", NC);
    const int64_t tiles = (S + cfg.rows - 1) / cfg.rows;
    int ncl = (int)(tiles < maxcl ? tiles : maxcl);
    if (cfg.units > 0 && cfg.units < ncl) ncl = cfg.units;
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.gridDim = dim3((unsigned)(NC * ncl), 1, 1);
    lc.blockDim = dim3((unsigned)threads, 1, 1);
    lc.dynamicSmemBytes = P.smem_bytes;
    lc.stream = st;
    lc.attrs = attr;
    lc.numAttrs = 1;
    ACCEL_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, K, M, (const char*)at, (const char*)et, mdl->log_pi, obs, off, S,
                                      (const int32_t*)order, next, cfg.rows, loglik, d_status, P));
    return after_launch(st, NC == 2 ? "hmm_forward(bf16 tcgen05, cluster pair)" : "hmm_forward(bf16 tcgen05, cluster of 4)", 5);
}

accel_status tc_forward_cfg(const accel_hmm_model* mdl, const int32_t* obs, const int64_t* off, int64_t S,
                            double* loglik, char* ws, int32_t* d_status, TcConfig cfg, cudaStream_t st) {
    const int K = mdl->K, M = mdl->M;
    ACCEL_REQUIRE(tc_supported(K, M), ACCEL_ERR_UNSUPPORTED,
                  "hmm_forward(bf16): K must be a multiple of 64 in [64, 256] and the tables must fit shared "
                  "memory (K=%d, M=%d)", K, M);
    if (cfg.split == 4 && (K / 4) % 32 != 0) cfg.split = 2;
    if (cfg.rows < 32 || cfg.rows > kRows) cfg.rows = kRows;
    if (cfg.pair == 2 && !tc_cl_supported(K, M, cfg.rows, cfg.split, 4)) cfg.pair = 1;
    if (cfg.pair == 2) return tc_forward_cluster<4>(mdl, obs, off, S, loglik, ws, d_status, cfg, st);
    if (cfg.pair == 1) {
        if (tc_cl_supported(K, M, cfg.rows, cfg.split, 2))
            return tc_forward_cluster<2>(mdl, obs, off, S, loglik, ws, d_status, cfg, st);
        cfg.pair = 0;
    }
    TcLayout L = tc_layout(K, M, S);
    char* at = ws + L.at_off;
    char* et = ws + L.e_off;
    int32_t* order = (int32_t*)(ws + L.order_off);
    unsigned long long* next = (unsigned long long*)(ws + kQueueOff);   // inside the status block
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + kQueueOff, 0, 8, st));
    int64_t nprep = (int64_t)K * K + (int64_t)K * M;
    int pg = (int)((nprep + 255) / 256);
    if (pg > 4 * num_sms()) pg = 4 * num_sms();
    k_tc_prep<<<pg, 256, 0, st>>>(mdl->log_A, mdl->log_B, K, M, at, et);
    accel_status r = order_by_length(off, S, order, ws + L.order_scratch_off, st);
    if (r != ACCEL_OK) return r;
    int64_t tiles = (S + cfg.rows - 1) / cfg.rows;
    int grid = (int)(tiles < num_sms() ? tiles : num_sms());
    if (cfg.units > 0 && cfg.units < grid) grid = cfg.units;
    // rows <= 64 per CTA: M = 64 tiles
    auto kern = cfg.split == 4 ? (cfg.rows <= 64 ? k_hmm_tc<4, 64> : k_hmm_tc<4, 128>)
                               : (cfg.rows <= 64 ? k_hmm_tc<2, 64> : k_hmm_tc<2, 128>);
    ACCEL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes));
    kern<<<grid, 128 * cfg.split, L.smem_bytes, st>>>(K, M, at, et, mdl->log_pi, obs, off, S, order, next, cfg.rows,
                                                      loglik, d_status, watchdog_ns(), L);
    return after_launch(st, "hmm_forward(bf16 tcgen05)", 5);
}

accel_status tc_forward(const accel_hmm_model* mdl, const int32_t* obs, const int64_t* off, int64_t S,
                        double* loglik, char* ws, int32_t* d_status, cudaStream_t st) {
    return tc_forward_cfg(mdl, obs, off, S, loglik, ws, d_status, tuned_config(mdl->K, mdl->M, S), st);
}

}  // namespace hmm
}  // namespace accel
