// Hand-written adjoint of the scaled HMM forward recursion (K9), with sqrt(T)
// checkpointing.
//
// Gradients of L = sum_s w_s logL_s with respect to log A, log B, log pi taken as free
// parameters are the (weighted) forward-backward expected counts.  The HMM is not in the
// paper; the recursion is its pattern vocabulary (a map of a reduce inside a sequential
// loop, Appendix A) and the adjoint is the textbook backward recursion, arranged so that
// the power-of-two scaling of the forward pass carries over without logarithms:
//
//   forward (0-based t):  S_t = alpha~_t 2^-e_t, alpha~_0 = pi o b(o_0),
//                         alpha~_t = (S_{t-1} A) o b(o_t),  c'_t = sum_j alpha~_t(j) = f 2^e_t
//   logL = ln2 sum_{t<T-1} e_t + ln c'_{T-1}
//   backward:             R_{T-1} = 1 / c'_{T-1}
//                         R_t     = 2^-e_t  A (b(o_{t+1}) o R_{t+1})
//   expected counts:      xi(i,j)  = A_ij sum_t S_t(i) b_j(o_{t+1}) R_{t+1}(j)
//                         gamma_t  = S_t o R_t 2^e_t,   counts(j,k) = sum_t gamma_t(j)[o_t = k]
// (R_t equals beta_t 2^{E_{t-1}} / P(o) with E the running exponent sum, so every product
// above equals the textbook alpha, beta, P(o) expression.)
//
// Memory: the forward keeps S_t only every C_s = ceil(sqrt(T_s)) steps (plus e_t).  The
// backward runs in rounds r = 0, 1, ...: round r takes segment n_s - 1 - r of every
// sequence (n_s = ceil(T_s / C_s)), recomputes its S_t from the checkpoint into a row
// buffer P, runs the backward recursion across it writing the matching rows
// Q = w_s b(o_{t+1}) o R_{t+1}, and a split-K GEMM accumulates U += P^T Q, so that
// xi = A o U at the end.  Storage is O(S sqrt(T_max) K) instead of O(sum_s T_s K).
//
// The recurrences are FP32 SIMT: for K in {64, 128, 256} on CTA pairs (thread-block clusters)
// that split the states, each pair running one or two groups of up to 16 length-sorted
// sequences as planned by k_plan; otherwise one CTA per 8 sequences.  The count
// contractions of each backward round run on the tensor cores (k_xi_tc.cu).  On the cluster
// path the backward of round r, the recomputation of round r + 1 and the counts of earlier
// rounds run at the same time on three streams, each round's rows in buffers of its own.
// Every accumulation has a fixed order, so results are deterministic.
#include "hmm_internal.cuh"
#include "simt_stream.cuh"

#include <cooperative_groups.h>
#include <map>
#include <math.h>
#include <vector>

namespace accel {
namespace hmm {
namespace adj {

constexpr int kT = 256;     // threads per CTA; thread j <-> state j
constexpr int kG = 8;       // sequences per CTA
constexpr int kTile = 64;   // GEMM tile of U
constexpr int kSplit = 16;  // GEMM split over rows

// cluster path: row buffers of the rounds (see Prm)
constexpr int kPBufs = 4;      // P rows: rounds r mod 4
constexpr int kQBufs = 3;      // Q, gamma and symbol rows: rounds r mod 3

struct Prm {
    int K, M, Cmax;
    int64_t S;
    const float* A;     // exp(log A) [K][K]
    const float* At;    // its transpose
    const float* BT;    // exp(log B)^T [M][K]
    const float* pi;    // exp(log pi) [K]
    const int32_t* obs;
    const int64_t* off;
    const int32_t* order;
    const double* w;    // weights or null
    float* cp;          // checkpoints [S][Cmax][K]
    int32_t* cp_e;      // their exponents [S][Cmax]
    float* clast;       // c'_{T-1} [S]
    double* loglik;     // [S] or null
    float* P;           // rows [S][Cmax][K]
    float* Q;           // rows [S][Cmax][K]
    float* Rc;          // carried R [S][K]
    float* cnt;         // per group [ngroups][K][M]
    float* pig;         // per group [ngroups][K]
    int32_t* status;    // device status word (ACCEL_ERR_SHAPE / ACCEL_ERR_TIMEOUT)
    int Kp;             // padded row stride (multiple of 4) of A, At and the shared vectors
    int32_t* rows;      // per round: rows of P/Q that may be non-zero (sorted-position order)
    int32_t* ebuf;      // exponents e_t of the P rows [S][Cmax] (cluster path)
    float* gam;         // weighted posteriors gamma_t of the rows [S][Cmax][K] (cluster path)
    int32_t* osym;      // o_t of each row, -1 for none [S][Cmax] (cluster path)
    int64_t ncl;        // cluster path: number of CTA pairs (the backward rounds; the plans' stride)
    int64_t ncl_fwd;    // cluster path: CTA pairs of the forward recursion (<= ncl; the SM budget)
    const int64_t* plan;  // cluster path: per pass (0: the forward; 1 + r: the backward of round r;
                          // 1 + Cmax + r: the recomputation of round r) and per pair (start0,
                          // size0, start1, size1) of its sequence groups (size1 = 0: one group),
                          // or null: group_range with ncl groups
    // cluster path, per round r: the sorted positions of the sequences with a segment in round
    // r (rlist[r][i], in sorted order), the first row of each in the round's row buffers
    // (rrow[r][i]: rows are packed, each sequence taking its segment length), and their number
    const int32_t* rlist;
    const int32_t* rrow;
    const int32_t* rcount;
    // cluster path: more row buffers, so that the recomputation of round r + 1 may run
    // beside the backward of round r, and the counts of round r beside the passes of the
    // rounds after it: P rows of round r in Pb[r mod kPBufs] (Pb[0] = P); exponents in ebuf,
    // ebuf2 (r mod 2); Q, gamma and symbol rows in Qb / Gb / Ob[r mod kQBufs] (the first
    // ones Q, gam, osym)
    float* Pb[kPBufs];
    int32_t* ebuf2;
    float* Qb[kQBufs];
    float* Gb[kQBufs];
    int32_t* Ob[kQBufs];
    // cluster path with plans: per backward launch l (the backward of round l - 1 beside the
    // recomputation of round l), the CTA pairs given to the backward; the rest recompute
    const int32_t* split;
};

// The scale exponent of a row sum c: c = m 2^e with m in [0.5, 1) (the frexp convention),
// read from the IEEE-754 exponent field of a normal c; zero, subnormal and non-finite c take
// frexpf.  pow2_scale(e) = 2^-e, built from the field where that is a normal float.  Both
// give exactly what frexpf / ldexpf give, at a few integer instructions on the per-step path.
__device__ __forceinline__ int scale_exp(float c) {
    const int f = (int)((__float_as_uint(c) >> 23) & 0xffu);
    if (f == 0 || f == 0xff) {
        int e = 0;
        frexpf(c, &e);
        return e;
    }
    return f - 126;
}
__device__ __forceinline__ float pow2_scale(int e) {     // 2^-e
    return (e > -127 && e < 127) ? __uint_as_float((uint32_t)(127 - e) << 23) : ldexpf(1.0f, -e);
}

__host__ __device__ __forceinline__ int seg_len(int64_t T) {
    int c = (int)ceil(sqrt((double)T));
    while ((int64_t)c * c < T) ++c;
    while (c > 1 && (int64_t)(c - 1) * (c - 1) >= T) --c;
    return c < 1 ? 1 : c;
}

struct GroupInfo {
    int64_t seq[kG], T[kG], o0[kG];
    int C[kG];
};

__device__ void load_group(const Prm& p, GroupInfo& gi) {
    for (int g = 0; g < kG; ++g) {
        int64_t q = blockIdx.x * (int64_t)kG + g;
        int64_t s = q < p.S ? p.order[q] : -1;
        gi.seq[g] = s;
        gi.T[g] = s >= 0 ? p.off[s + 1] - p.off[s] : 0;
        gi.o0[g] = s >= 0 ? p.off[s] : 0;
        gi.C[g] = s >= 0 ? seg_len(gi.T[g]) : 1;
        if (s >= 0 && gi.C[g] > p.Cmax) {   // longer than max_T: skip, report
            if (threadIdx.x == 0) report_status(p.status, ACCEL_ERR_SHAPE);
            gi.seq[g] = -1;
            gi.T[g] = 0;
            gi.C[g] = 1;
        }
    }
}

// Block-wide sums of kG per-thread values (deterministic order); result in all threads.
__device__ __forceinline__ void block_sum_g(float (&v)[kG], float (*s_red)[kT / 32]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        float x = v[g];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane == 0) s_red[g][w] = x;
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        float x = 0.f;
#pragma unroll
        for (int q = 0; q < kT / 32; ++q) x += s_red[g][q];
        v[g] = x;
    }
    __syncthreads();
}

// One forward step for the active sequences with A streamed through shared memory: sS
// holds S_{t-1} on entry and S_t on exit; returns e_t and c'_t per sequence.  obs_t[g] is
// o_t of sequence g.  Returns false if a bulk copy did not arrive in time.
__device__ __forceinline__ bool fwd_step(const Prm& p, simt::AStream& as, float* sS, const float* sBT,
                                         float (*s_red)[kT / 32], const bool (&act)[kG], const int (&obs_t)[kG],
                                         int (&e)[kG], float (&c)[kG]) {
    const int j = threadIdx.x, K = p.K, Kp = p.Kp;
    float acc[kG];
    if (!simt::as_matvec<kG>(as, sS, Kp, act, acc)) return false;
    float v[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        acc[g] = (act[g] && j < K) ? acc[g] * sBT[obs_t[g] * K + j] : 0.f;
        v[g] = acc[g];
    }
    block_sum_g(v, s_red);   // its barriers follow every read of sS
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        c[g] = v[g];
        int ex = 0;
        frexpf(v[g], &ex);
        e[g] = ex;
        if (act[g] && j < K) sS[g * Kp + j] = acc[g] * ldexpf(1.0f, -ex);
    }
    __syncthreads();
    return true;
}

__device__ __forceinline__ void report_timeout(const Prm& p, simt::AStream& as) {
    if (threadIdx.x == 0) report_status(p.status, ACCEL_ERR_TIMEOUT);
    simt::as_drain(as);
}

// A and At with row stride Kp (padding zero), the emission table transposed, pi.
__global__ void k_prep(const float* __restrict__ logA, const float* __restrict__ logB, const float* __restrict__ logpi,
                       int K, int Kp, int M, float* __restrict__ A, float* __restrict__ At, float* __restrict__ BT,
                       float* __restrict__ pi) {
    int64_t nA = (int64_t)K * Kp, nB = (int64_t)K * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * nA + nB + K;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < nA) {
            int i = (int)(idx / Kp), j = (int)(idx % Kp);
            A[idx] = j < K ? __expf(logA[(int64_t)i * K + j]) : 0.f;
        } else if (idx < 2 * nA) {
            int64_t q = idx - nA;
            int j = (int)(q / Kp), i = (int)(q % Kp);
            At[q] = i < K ? __expf(logA[(int64_t)i * K + j]) : 0.f;
        } else if (idx < 2 * nA + nB) {
            int64_t q = idx - 2 * nA;
            int j = (int)(q / M), k = (int)(q % M);
            BT[(int64_t)k * K + j] = __expf(logB[q]);
        } else {
            int j = (int)(idx - 2 * nA - nB);
            pi[j] = __expf(logpi[j]);
        }
    }
}

// Shared-memory layout of both kernels: [A stream ring + barriers][emission table M x K]
// [sS kG x Kp][sR kG x Kp][sE kG x Cmax ints]
__host__ __device__ inline size_t off_bt(int Kp) { return align_up(simt::stream_smem_bytes(Kp), 16); }
__host__ __device__ inline size_t off_ss(int K, int M, int Kp) { return align_up(off_bt(Kp) + (size_t)M * K * 4, 16); }

// ---------------------------------------------------------------- forward + checkpoints
__global__ void __launch_bounds__(kT) k_forward_cp(Prm p) {
    extern __shared__ __align__(16) char smem[];
    const int K = p.K, M = p.M, Kp = p.Kp, j = threadIdx.x;
    simt::AStream as;
    simt::as_init(as, smem, K, Kp);
    float* sBT = reinterpret_cast<float*>(smem + off_bt(Kp));          // [M][K]
    float* sS = reinterpret_cast<float*>(smem + off_ss(K, M, Kp));     // [kG][Kp]
    __shared__ float s_red[kG][kT / 32];
    for (int idx = j; idx < M * K; idx += kT) sBT[idx] = p.BT[idx];
    GroupInfo gi;
    load_group(p, gi);
    int64_t Tmax = 0;
    for (int g = 0; g < kG; ++g) Tmax = gi.T[g] > Tmax ? gi.T[g] : Tmax;
    __syncthreads();
    simt::as_begin(as, p.A);
    // t = 0: alpha~_0 = pi o b(o_0)
    bool act[kG];
    int ob[kG], e[kG];
    float c[kG], v[kG], a0[kG];
    int64_t E[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        act[g] = gi.T[g] > 0;
        ob[g] = act[g] ? p.obs[gi.o0[g]] : 0;
        a0[g] = (act[g] && j < K) ? p.pi[j] * sBT[ob[g] * K + j] : 0.f;
        v[g] = a0[g];
        E[g] = 0;
    }
    block_sum_g(v, s_red);
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        int ex = 0;
        frexpf(v[g], &ex);
        e[g] = ex;
        c[g] = v[g];
        if (act[g] && j < K) {
            float sv = a0[g] * ldexpf(1.0f, -ex);
            sS[g * Kp + j] = sv;
            p.cp[((int64_t)gi.seq[g] * p.Cmax) * K + j] = sv;
        }
        if (act[g] && j == 0) p.cp_e[(int64_t)gi.seq[g] * p.Cmax] = ex;
        if (act[g] && gi.T[g] == 1 && j == 0) {
            p.clast[gi.seq[g]] = c[g];
            if (p.loglik) p.loglik[gi.seq[g]] = log((double)c[g]);
        }
        E[g] = ex;
    }
    __syncthreads();
    for (int64_t t = 1; t < Tmax; ++t) {
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            act[g] = t < gi.T[g];
            ob[g] = act[g] ? p.obs[gi.o0[g] + t] : 0;
        }
        if (!fwd_step(p, as, sS, sBT, s_red, act, ob, e, c)) { report_timeout(p, as); return; }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            if (!act[g]) continue;
            if (t == gi.T[g] - 1 && j == 0) {
                p.clast[gi.seq[g]] = c[g];
                if (p.loglik) p.loglik[gi.seq[g]] = 0.6931471805599453 * (double)E[g] + log((double)c[g]);
            }
            E[g] += e[g];
            if (t % gi.C[g] == 0) {
                int64_t k = t / gi.C[g];
                if (j < K) p.cp[((int64_t)gi.seq[g] * p.Cmax + k) * K + j] = sS[g * Kp + j];
                if (j == 0) p.cp_e[(int64_t)gi.seq[g] * p.Cmax + k] = e[g];
            }
        }
    }
    if (!simt::as_end(as)) report_timeout(p, as);
}

// ---------------------------------------------------------------- one backward round
// P/Q rows of the sequence at sorted position q are rows [q Cmax, (q+1) Cmax).
__global__ void __launch_bounds__(kT) k_backward_round(Prm p, int r) {
    extern __shared__ __align__(16) char smem[];
    const int K = p.K, M = p.M, Kp = p.Kp, j = threadIdx.x;
    simt::AStream as;
    simt::as_init(as, smem, K, Kp);
    float* sBT = reinterpret_cast<float*>(smem + off_bt(Kp));          // [M][K]
    float* sS = reinterpret_cast<float*>(smem + off_ss(K, M, Kp));     // [kG][Kp] recompute state / v
    float* sR = sS + (size_t)kG * Kp;                                  // [kG][Kp] R_{t+1}
    int* sE = reinterpret_cast<int*>(sR + (size_t)kG * Kp);            // [kG][Cmax] exponents of the segment
    __shared__ float s_red[kG][kT / 32];
    for (int idx = j; idx < M * K; idx += kT) sBT[idx] = p.BT[idx];
    GroupInfo gi;
    load_group(p, gi);
    int64_t t0[kG], L[kG], rowbase[kG];
    int maxL = 0;
    float wgt[kG];
    bool just_done[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        t0[g] = 0;
        L[g] = 0;
        wgt[g] = 0.f;
        just_done[g] = false;
        rowbase[g] = (blockIdx.x * (int64_t)kG + g) * p.Cmax;
        if (gi.seq[g] < 0) continue;
        int64_t n = (gi.T[g] + gi.C[g] - 1) / gi.C[g];
        int64_t k = n - 1 - r;
        just_done[g] = k == -1;
        if (k < 0) continue;
        t0[g] = k * gi.C[g];
        int64_t t1 = t0[g] + gi.C[g] < gi.T[g] ? t0[g] + gi.C[g] : gi.T[g];
        L[g] = t1 - t0[g];
        maxL = L[g] > maxL ? (int)L[g] : maxL;
        wgt[g] = p.w ? (float)p.w[gi.seq[g]] : 1.0f;
        if (j == 0) atomicMax(&p.rows[r], (int32_t)(rowbase[g] + p.Cmax));
    }
    // rows that must read as zero: all rows of a sequence whose last segment was done in
    // the previous round, and rows past the segment length of an active one
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        if (gi.seq[g] < 0 || !(just_done[g] || L[g] > 0)) continue;
        for (int64_t tt = L[g]; tt < p.Cmax; ++tt)
            if (j < K) p.Q[(rowbase[g] + tt) * K + j] = 0.f;
    }
    if (maxL == 0) return;
    // ---- recompute S_t for t in [t0, t0 + L) into the P rows (and e_t into sE)
    bool act[kG];
    int ob[kG], e[kG];
    float c[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        act[g] = L[g] > 0;
        if (!act[g]) continue;
        int64_t base = (int64_t)gi.seq[g] * p.Cmax;
        int64_t k = t0[g] / gi.C[g];
        if (j < K) {
            float sv = p.cp[(base + k) * K + j];
            sS[g * Kp + j] = sv;
            p.P[rowbase[g] * K + j] = sv;
        }
        if (j == 0) sE[g * p.Cmax] = p.cp_e[base + k];
    }
    __syncthreads();
    simt::as_begin(as, p.A);
    for (int tt = 1; tt < maxL; ++tt) {
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            act[g] = tt < L[g];
            ob[g] = act[g] ? p.obs[gi.o0[g] + t0[g] + tt] : 0;
        }
        if (!fwd_step(p, as, sS, sBT, s_red, act, ob, e, c)) { report_timeout(p, as); return; }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            if (!act[g]) continue;
            if (j < K) p.P[(rowbase[g] + tt) * K + j] = sS[g * Kp + j];
            if (j == 0) sE[g * p.Cmax + tt] = e[g];
        }
    }
    if (!simt::as_end(as)) { report_timeout(p, as); return; }
    // ---- backward across the segment: R_{t+1} in sR, v = b(o_{t+1}) o R_{t+1} in sS
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        if (L[g] == 0 || j >= K) continue;
        bool last_seg = t0[g] + L[g] == gi.T[g];
        sR[g * Kp + j] = last_seg ? 0.f : p.Rc[(int64_t)gi.seq[g] * K + j];
    }
    __syncthreads();
    simt::as_begin(as, p.At);
    float* cnt = p.cnt + (int64_t)blockIdx.x * K * M;
    for (int tt = maxL - 1; tt >= 0; --tt) {
        bool trans[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            act[g] = tt < L[g];
            int64_t t = t0[g] + tt;
            trans[g] = act[g] && t < gi.T[g] - 1;          // transition t -> t+1 exists
            if (act[g] && j < K) {
                float vv = trans[g] ? sBT[p.obs[gi.o0[g] + t + 1] * K + j] * sR[g * Kp + j] : 0.f;
                sS[g * Kp + j] = vv;
                p.Q[(rowbase[g] + tt) * K + j] = wgt[g] * vv;
            }
        }
        __syncthreads();
        float acc[kG];
        if (!simt::as_matvec<kG>(as, sS, Kp, trans, acc)) { report_timeout(p, as); return; }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            if (!act[g]) continue;
            int64_t t = t0[g] + tt;
            const int et = sE[g * p.Cmax + tt];
            float Rt = trans[g] ? acc[g] * ldexpf(1.0f, -et) : 1.0f / p.clast[gi.seq[g]];
            if (j < K) {
                float St = p.P[(rowbase[g] + tt) * K + j];
                float gam = wgt[g] * St * Rt * ldexpf(1.0f, et);
                int ot = p.obs[gi.o0[g] + t];
                cnt[(int64_t)j * M + ot] += gam;
                if (t == 0) p.pig[(int64_t)blockIdx.x * K + j] += gam;
                sR[g * Kp + j] = Rt;
            }
        }
        __syncthreads();
    }
    if (!simt::as_end(as)) { report_timeout(p, as); return; }
    // carry R_{t0} to the next round
#pragma unroll
    for (int g = 0; g < kG; ++g)
        if (L[g] > 0 && j < K) p.Rc[(int64_t)gi.seq[g] * K + j] = sR[g * Kp + j];
}

// ---------------------------------------------------------------- U += P^T Q (split-K)
// CTA (tile i-block, j-block, split) takes rows [split*R/kSplit, (split+1)*R/kSplit) of the
// rows R = rows[round] that may be non-zero.
__global__ void __launch_bounds__(256) k_gemm_ptq(const float* __restrict__ P, const float* __restrict__ Q,
                                                 const int32_t* __restrict__ rows_r, int K, float* __restrict__ Upart) {
    __shared__ float sP[32][kTile + 4];
    __shared__ float sQ[32][kTile + 4];
    const int64_t rows = *rows_r;
    const int nb = (K + kTile - 1) / kTile;
    const int bi = blockIdx.x % nb, bj = (blockIdx.x / nb) % nb, sp = blockIdx.x / (nb * nb);
    const int64_t r0 = rows * sp / kSplit, r1 = rows * (sp + 1) / kSplit;
    if (r0 >= r1) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x 4 outputs each
    float acc[4][4] = {};
    for (int64_t rb = r0; rb < r1; rb += 32) {
        for (int q = threadIdx.x; q < 32 * kTile; q += 256) {
            int rr = q / kTile, cc = q % kTile;
            int64_t row = rb + rr;
            int ci = bi * kTile + cc, cj = bj * kTile + cc;
            sP[rr][cc] = (row < r1 && ci < K) ? P[row * K + ci] : 0.f;
            sQ[rr][cc] = (row < r1 && cj < K) ? Q[row * K + cj] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = sP[rr][ty * 4 + u]; b[u] = sQ[rr][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
    float* U = Upart + (int64_t)sp * K * K;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int i = bi * kTile + ty * 4 + u, jj = bj * kTile + tx * 4 + v;
            if (i < K && jj < K) U[(int64_t)i * K + jj] += acc[u][v];
        }
}

// Emission counts of one round (cluster path): cntp[split][j][k] += sum over the split's rows
// with o(row) = k of gam[row][j].  Thread j owns column j of a shared [M][256] block, so the
// accumulation is conflict-free and in row order (deterministic).
constexpr int kCntSplit = 64;
__global__ void __launch_bounds__(256) k_counts(const float* __restrict__ gam, const int32_t* __restrict__ osym,
                                               const int32_t* __restrict__ rows_r, int K, int M,
                                               float* __restrict__ cntp) {
    extern __shared__ float sc[];          // [M][256]
    const int64_t rows = *rows_r;
    const int nb = (K + 255) / 256;
    const int jb = blockIdx.x % nb, sp = blockIdx.x / nb;
    const int64_t r0 = rows * sp / kCntSplit, r1 = rows * (sp + 1) / kCntSplit;
    if (r0 >= r1) return;
    const int j = jb * 256 + threadIdx.x;
    for (int k = 0; k < M; ++k) sc[k * 256 + threadIdx.x] = 0.f;
    if (j < K) {
        for (int64_t row = r0; row < r1; ++row) {
            const int o = osym[row];
            if (o >= 0) sc[o * 256 + threadIdx.x] += gam[row * K + j];
        }
        float* dst = cntp + (int64_t)sp * K * M;
        for (int k = 0; k < M; ++k) dst[(int64_t)j * M + k] += sc[k * 256 + threadIdx.x];
    }
}

// grad_log_A = A o sum_split U, grad_log_B = sum_groups counts, grad_log_pi = sum_groups pig
// (A has row stride Kp)
__global__ void k_finish(const float* __restrict__ A, int Kp, const float* __restrict__ Upart,
                         const float* __restrict__ cnt, const float* __restrict__ cntp, const float* __restrict__ pig,
                         int K, int M, int64_t ngroups, int64_t npig, int nsU, int nsC, float* __restrict__ gA,
                         float* __restrict__ gB, float* __restrict__ gpi) {
    int64_t nA = (int64_t)K * K, nB = (int64_t)K * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nA + nB + K;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < nA) {
            float u = 0.f;
            for (int s = 0; s < nsU; ++s) u += Upart[(int64_t)s * nA + idx];
            gA[idx] = A[(idx / K) * Kp + idx % K] * u;
        } else if (idx < nA + nB) {
            int64_t q = idx - nA;
            float x = 0.f;
            for (int64_t b = 0; b < ngroups; ++b) x += cnt[b * nB + q];
            for (int b = 0; b < nsC; ++b) x += cntp[(int64_t)b * nB + q];
            gB[q] = x;
        } else {
            int64_t q = idx - nA - nB;
            float x = 0.f;
            for (int64_t b = 0; b < npig; ++b) x += pig[b * K + q];
            if (gpi) gpi[q] = x;
        }
    }
}


// ============================================================================================
// Cluster-pair path (K a multiple of 64): the matrix the step multiplies by stays resident in
// shared memory in FP32.  A pair of CTAs (a thread-block cluster of 2) owns 16 sequences;
// CTA r holds the K x K/2 column half r of the matrix and computes output states
// [r K/2, (r+1) K/2) of every sequence.  After each step the two CTAs write their halves
// of the new vectors, and their partial row sums, into both CTAs' shared memory through
// distributed shared memory, then meet at one cluster barrier.  Vectors and partial sums are
// double-buffered by step parity, so a CTA never overwrites what its peer may still read.
// ============================================================================================
namespace clu {
namespace cg = cooperative_groups;

constexpr int kG = 16;      // sequences per cluster
constexpr int kT = 256;     // threads per CTA (8 warps)
constexpr int kNW = 8;

// Work split for K in {64, 128, 256}.  Each CTA of the pair owns Kh = K/2 states (output
// columns of the contraction out[g][j] = sum_i X[g][i] Mx[i][j]).
//  * Contraction: warp w takes the i-part w (rows w IPART .. w IPART + IPART - 1) and lane l
//    the CW = Kh/32 columns l CW .. l CW + CW - 1.  The thread's IPART x CW block of the
//    matrix is loaded into registers once per kernel, so the step reads only the vectors
//    from shared memory, and those as whole-warp broadcasts (every lane of a warp reads the
//    same address).  Packed FMAs pair rows: the accumulator of (g, c) is a float2 of the
//    even-row and odd-row partial sums, so both operands, (x[g][i], x[g][i+1]) and
//    (Mx[i][c], Mx[i+1][c]), are natural register pairs.  At K = 256 the 16 sequences are
//    taken in two passes of 8 to bound the accumulator registers.
//  * The eight warps' partial outputs meet in shared memory (fixed order: deterministic).
//  * Epilogue: thread t takes sequence g = t / 16 and the EC = Kh/16 consecutive states
//    (t % 16) EC .. +EC - 1, so vector, row and parameter accesses are 8-16 byte vectors.
template <int K>
struct Sh {
    static constexpr int Kh = K / 2;
    static constexpr int IPART = K / kNW;
    static constexpr int CW = Kh / 32;
    static constexpr int EC = Kh / 16;
    static constexpr int NPASS = K == 256 ? 2 : 1;
    static constexpr int GP = kG / NPASS;
    static_assert(IPART % 4 == 0 && (CW == 4 || CW == 2 || CW == 1) && EC % 2 == 0, "unsupported K");
};
__host__ __device__ inline bool cluster_shape_ok(int K) { return K == 64 || K == 128 || K == 256; }

struct SL { size_t bth, sx, part, red, st, total; };

__host__ __device__ inline SL smem_layout(int K, int M) {
    const int Kh = K / 2;
    SL L;
    size_t o = 0;
    L.bth = o;   o += (size_t)M * Kh * 4;                 // emission columns [M][Kh]
    L.sx = o;    o += (size_t)2 * kG * K * 4;             // full vectors, two step parities [2][16][K]
    L.part = o;  o += (size_t)kNW * kG * Kh * 4;          // per-warp partial outputs [8][16][Kh]
    L.red = o;   o += (size_t)2 * 2 * kG * 4;             // partial row sums [parity][rank][16]
    L.st = o;    o += (size_t)kG * Kh * 4;                // backward: this step's S_t rows (own half)
    L.total = o;
    return L;
}

// Group state in shared memory (read as broadcasts).
struct GS {
    int64_t seq[kG], T[kG], o0[kG];
    int C[kG];
    float w[kG];
    int64_t t0[kG], L[kG];
    int just_done[kG];
    int sym[2][kG];      // per step parity: the step's symbol (see the kernels)
    int eb[2][kG];       // per step parity: e_t (backward)
    int sym_end[kG];     // backward: symbol after the segment, -1 if none
    int32_t rowb[kG];    // rounds: the sequence's first row in the round's row buffers
};

// Sorted positions [start, start + size) of group j when the S sequences (in order of
// decreasing length) are split into `ngroups` contiguous groups of at most 16 (ngroups >=
// S / 16).  The longest sequences set the critical path, so when there is room the first
// groups take 8 (half the contraction work per step) and the rest share the remainder
// evenly.  Without a plan, CTA pair cidx runs group cidx of p.ncl.
__device__ __forceinline__ void group_range_n(int64_t S, int64_t ngroups, int64_t j, int64_t& start, int& size) {
    int64_t n8 = 0;                                    // leading groups of at most 8
    if (S > 8 * ngroups) {
        n8 = (16 * ngroups - S) / 8;
        if (n8 < 0) n8 = 0;
    }
    if (j < n8) {
        start = 8 * j;
        size = 8;
        return;
    }
    const int64_t rem = S - 8 * n8, m = ngroups - n8, jj = j - n8;
    const int64_t base = rem / m, extra = rem % m, firstbig = m - extra;
    start = 8 * n8 + jj * base + (jj > firstbig ? jj - firstbig : 0);
    size = (int)(base + (jj >= firstbig ? 1 : 0));
}

// The sequence groups CTA pair cidx runs in pass `pass` (0: the forward; 1 + r: the backward
// of round r; 1 + Cmax + r: the recomputation of round r), one after the other (1 or 2).
// Groups are ranges of the pass's sequence list (the forward: all sorted positions; round r:
// rlist[r]) of n entries.
__device__ __forceinline__ const int64_t* pass_plan(const Prm& p, int pass) {
    return p.plan ? p.plan + (int64_t)pass * p.ncl * 4 : nullptr;
}
// The row buffers of round r on the cluster path (see Prm).
__host__ __device__ __forceinline__ float* round_P(const Prm& p, int r) { return p.Pb[r % kPBufs]; }
__host__ __device__ __forceinline__ int32_t* round_e(const Prm& p, int r) { return (r & 1) ? p.ebuf2 : p.ebuf; }
__host__ __device__ __forceinline__ float* round_Q(const Prm& p, int r) { return p.Qb[r % kQBufs]; }
__host__ __device__ __forceinline__ float* round_gam(const Prm& p, int r) { return p.Gb[r % kQBufs]; }
__host__ __device__ __forceinline__ int32_t* round_osym(const Prm& p, int r) { return p.Ob[r % kQBufs]; }
__device__ __forceinline__ int cluster_groups(const Prm& p, int pass, int64_t cidx) {
    const int64_t* pl = pass_plan(p, pass);
    return (pl && pl[cidx * 4 + 3] > 0) ? 2 : 1;
}
__device__ __forceinline__ void cluster_group_range(const Prm& p, int pass, int64_t n, int64_t cidx, int gi,
                                                    int64_t& start, int& size) {
    const int64_t* pl = pass_plan(p, pass);
    if (pl) {
        start = pl[cidx * 4 + 2 * gi];
        size = (int)pl[cidx * 4 + 2 * gi + 1];
    } else {
        group_range_n(n, pass == 0 ? p.ncl_fwd : p.ncl, cidx, start, size);
    }
}

// ---- group plans.  More groups than CTA pairs lets more of the longest sequences run in
// groups of 8 (one contraction pass per step instead of two); the surplus groups, the
// shortest, then share a pair with another group and run after it.  A step of a group of g
// sequences costs about (0.92 + ceil(g / GP)) contraction passes (measured: a pass of 8
// sequences ~2,840 cycles at K = 256, the rest of the step ~2,620), so a pair's time in a pass
// is the sum over its groups of (the group's longest step count) x that cost.  A plan of nv
// groups on c pairs gives the first c groups (the longest) one pair each, and surplus group
// c + k joins pair c - 1 - k (the least loaded first); the group count with the smallest
// maximum load wins.
//
// One plan per pass: the forward (step counts T over all sequences) and, for every round r,
// the backward and the recomputation (step counts = the segment lengths of round r over the
// sequences that have one).  Segment lengths grow like sqrt(T), so a grouping balanced for T
// would leave the pairs that run two groups of short sequences as the slowest of every round.
//
// The backward of round r and the recomputation of round r + 1 are independent, so they run
// at the same time (backward launch r + 1: k_bwd_cl and k_rec_cl on two streams).  Either they
// run side by side, the backward on nb pairs and the recomputation on the other ncl - nb, or
// each on all ncl pairs, sharing them.  The planner takes the split with the smallest
// estimated time: the larger of the two passes' maximum loads side by side, their sum
// otherwise (a backward step weighs 1.05 recomputation steps: measured fastest among
// 0.95-1.25 at K = 256 with the two passes running side by side).  One pass alone on all
// pairs has to round 13-14 sequences a pair up to two contraction passes a step; two passes
// side by side can use groups of 16 and balance what is left between them.
//
// One CTA per launch (block 0: the forward).  The step counts of a pass's list sit in shared
// memory with their maxima over 2, 4, 8 and 16 consecutive entries, so a group's cost is two
// reads.  Candidate splits: every nb for ncl <= 32, else the multiples of 4 and then the three
// on each side of the best of them; one thread per (pass, candidate, group count).
constexpr int kPlanThreads = 1024;
constexpr int kPlanMaxGroups = 256;
constexpr int kPlanMaxSeq = 16 * kPlanMaxGroups;
constexpr int kPlanMaxCand = 40;
constexpr int kPlanLevels = 5;
constexpr float kBwdStepCost = 1.05f;

__host__ __device__ inline size_t plan_smem_bytes() { return (size_t)2 * kPlanLevels * kPlanMaxSeq * 4; }

// step count of the sequence with T steps in pass `pass` (0: T; 1 + r: its round-r segment)
__host__ __device__ __forceinline__ int64_t pass_steps(int64_t T, int pass) {
    if (pass == 0) return T;
    if (T <= 0) return 0;
    const int64_t C = seg_len(T), n = (T + C - 1) / C, k = n - pass;   // segment n - 1 - r
    if (k < 0) return 0;
    const int64_t t1 = (k + 1) * C < T ? (k + 1) * C : T;
    return t1 - k * C;
}

// A pass's list in shared memory: level k (lv(k)[i]) = max of the step counts of entries
// i .. i + 2^k - 1.
struct PlanList {
    int* lv0;
    int64_t n;
    __device__ __forceinline__ int* lv(int k) const { return lv0 + k * kPlanMaxSeq; }
};

// max over entries [st, st + sz), 1 <= sz < 32: two overlapping windows of the level below sz
__device__ __forceinline__ int list_max(const PlanList& t, int st, int sz) {
    const int k = 31 - __clz(sz);
    const int* v = t.lv(k);
    const int a = v[st], b = v[st + sz - (1 << k)];
    return a > b ? a : b;
}

// group_range_n(n, nv, .) with its divisions done once per group count (n <= kPlanMaxSeq and
// nv <= kPlanMaxGroups: 32-bit arithmetic)
struct Groups {
    int n8, base, firstbig;
};
__device__ __forceinline__ Groups groups_of(int n, int nv) {
    Groups g;
    g.n8 = 0;
    if (n > 8 * nv) {
        g.n8 = (16 * nv - n) / 8;
        if (g.n8 < 0) g.n8 = 0;
    }
    const int rem = n - 8 * g.n8, m = nv - g.n8;
    g.base = rem / m;
    g.firstbig = m - rem % m;
    return g;
}
__device__ __forceinline__ float group_cost(const PlanList& t, const Groups& g, int j, int gp) {
    int st, sz;
    if (j < g.n8) {
        st = 8 * j;
        sz = 8;
    } else {
        const int jj = j - g.n8;
        st = 8 * g.n8 + jj * g.base + (jj > g.firstbig ? jj - g.firstbig : 0);
        sz = g.base + (jj >= g.firstbig ? 1 : 0);
    }
    return sz > 0 ? (float)list_max(t, st, sz) * (0.92f + (float)((sz + gp - 1) / gp)) : 0.f;
}

// the largest pair load of nv groups of the list's n > 0 entries on c pairs
__device__ float plan_worst(const PlanList& t, int c, int nv, int gp) {
    const Groups g = groups_of((int)t.n, nv);
    const int extra = nv > c ? nv - c : 0;
    const int nq = c < nv ? c : nv;
    float worst = 0.f;
    for (int q = 0; q < nq; ++q) {
        float l = group_cost(t, g, q, gp);
        const int k = c - 1 - q;
        if (k < extra) l += group_cost(t, g, c + k, gp);
        worst = fmaxf(worst, l);
    }
    return worst;
}

// candidate group counts of n > 0 entries on c > 0 pairs: groups of at most 16, at most two
// groups a pair, at most 128 candidates (lo > hi: none)
__device__ __forceinline__ void nv_range(int64_t n, int64_t c, int64_t& lo, int64_t& hi) {
    const int64_t lo16 = (n + 15) / 16, m = c < n ? c : n;
    lo = lo16 > m ? lo16 : m;
    hi = 2 * c < n ? 2 * c : n;
    if (hi > lo + 127) hi = lo + 127;
}

// plan entries [0, stride) of one pass: nv groups on pairs [0, c), the rest empty
__device__ void write_plan(const PlanList& t, int64_t* pl, int64_t stride, int64_t c, int64_t nv) {
    const int64_t extra = nv > c ? nv - c : 0;
    for (int64_t q = threadIdx.x; q < stride; q += blockDim.x) {
        int64_t st = 0;
        int sz = 0;
        if (t.n > 0 && q < c && q < nv) group_range_n(t.n, nv, q, st, sz);
        pl[q * 4] = st;
        pl[q * 4 + 1] = sz;
        pl[q * 4 + 2] = 0;
        pl[q * 4 + 3] = 0;
        const int64_t k = c - 1 - q;
        if (t.n > 0 && q < c && k < extra) {
            group_range_n(t.n, nv, c + k, st, sz);
            pl[q * 4 + 2] = st;
            pl[q * 4 + 3] = sz;
        }
    }
}

// Block 0 plans the forward on ncl_fwd pairs.  Block 1 + l plans backward launch l (l in
// [0, Cmax]): the backward of round l - 1 (list 0, if l >= 1) and the recomputation of round l
// (list 1, if l < Cmax), and writes split[2 l] = the backward's pairs, split[2 l + 1] = the
// recomputation's.
__global__ void __launch_bounds__(kPlanThreads) k_plan(Prm p, int64_t* plan, int32_t* split, int gp) {
    extern __shared__ __align__(16) int s_lv[];          // [2][kPlanLevels][kPlanMaxSeq]
    __shared__ uint64_t s_key[2][kPlanMaxCand];
    __shared__ int s_lo[2][kPlanMaxCand];
    __shared__ int s_cnt[2 * kPlanMaxCand + 1];
    __shared__ int s_cb[kPlanMaxCand], s_cc[kPlanMaxCand];
    __shared__ int s_ncand;
    __shared__ float s_bf;
    __shared__ int s_bcb, s_bcc;
    __shared__ int64_t s_bnv[2];
    const int tid = threadIdx.x;
    const int blk = blockIdx.x, l = blk - 1;
    const bool fwd = blk == 0;
    const int rnd[2] = {fwd ? -1 : l - 1, (!fwd && l < p.Cmax) ? l : -1};
    const int64_t ncl = fwd ? p.ncl_fwd : p.ncl;
    // list k of the two passes (0: the forward or the backward; 1: the recomputation)
    auto list = [&](int k) -> PlanList {
        PlanList t;
        t.lv0 = s_lv + k * kPlanLevels * kPlanMaxSeq;
        t.n = fwd ? (k == 0 ? p.S : 0) : (rnd[k] >= 0 ? p.rcount[rnd[k]] : 0);
        return t;
    };
    for (int k = 0; k < 2; ++k) {
        const PlanList t = list(k);
        for (int64_t i = tid; i < t.n; i += kPlanThreads) {
            const int64_t q = fwd ? i : p.rlist[(int64_t)rnd[k] * p.S + i];
            const int64_t sq = p.order[q];
            t.lv0[i] = (int)pass_steps(p.off[sq + 1] - p.off[sq], fwd ? 0 : 1 + rnd[k]);
        }
    }
    __syncthreads();
    for (int v = 1; v < kPlanLevels; ++v) {
        const int h = 1 << (v - 1);
        for (int k = 0; k < 2; ++k) {
            const PlanList t = list(k);
            for (int64_t i = tid; i + 2 * h <= t.n; i += kPlanThreads) {
                const int a = t.lv(v - 1)[i], b = t.lv(v - 1)[i + h];
                t.lv(v)[i] = a > b ? a : b;
            }
        }
        __syncthreads();
    }
    const bool both = !fwd && rnd[0] >= 0 && rnd[1] >= 0;
    const int step = ncl <= 32 ? 1 : 4;
    if (tid == 0) {
        s_bf = INFINITY;
        s_bcb = (int)ncl;
        s_bcc = fwd ? 0 : (int)ncl;
        s_bnv[0] = s_bnv[1] = 0;
    }
    for (int phase = 0; phase < 2; ++phase) {
        if (tid == 0) {
            int nc = 0;
            if (phase == 0) {
                if (fwd) {
                    s_cb[nc] = (int)ncl; s_cc[nc++] = 0;
                } else if (!both) {
                    s_cb[nc] = rnd[0] >= 0 ? (int)ncl : 0;
                    s_cc[nc++] = rnd[1] >= 0 ? (int)ncl : 0;
                } else {
                    s_cb[nc] = (int)ncl; s_cc[nc++] = (int)ncl;          // each on all pairs
                    s_cb[nc] = (int)ncl; s_cc[nc++] = 0;                 // (an empty list)
                    for (int nb = step; nb < ncl; nb += step) { s_cb[nc] = nb; s_cc[nc++] = (int)ncl - nb; }
                }
            } else if (both && step > 1 && s_bcb + s_bcc == ncl) {
                for (int nb = s_bcb - step + 1; nb < s_bcb + step; ++nb)
                    if (nb >= 1 && nb < ncl && nb % step != 0) { s_cb[nc] = nb; s_cc[nc++] = (int)ncl - nb; }
            }
            s_ncand = nc;
        }
        __syncthreads();
        const int nc = s_ncand;
        // per problem (pass k, candidate j): its group-count range, its first item, and the
        // best (load, group count) so far as one 64-bit key (load bits above the count: the
        // loads are non-negative, so integer order is value order, ties to the fewest groups)
        if (tid < 2 * nc) {
            const int k = tid / nc, j = tid - k * nc;
            const int64_t c = k == 0 ? s_cb[j] : s_cc[j], n = list(k).n;
            int64_t lo = 0, hi = -1;
            uint64_t key = (uint64_t)__float_as_uint(INFINITY) << 32;
            if (n == 0) key = 0;
            else if (c > 0) nv_range(n, c, lo, hi);
            s_lo[k][j] = (int)lo;
            s_cnt[tid] = hi >= lo ? (int)(hi - lo + 1) : 0;
            s_key[k][j] = key;
        }
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int i = 0; i < 2 * nc; ++i) {
                const int c = s_cnt[i];
                s_cnt[i] = acc;
                acc += c;
            }
            s_cnt[2 * nc] = acc;
        }
        __syncthreads();
        // one thread per item (problem, group count)
        const int nitems = s_cnt[2 * nc];
        for (int it = tid; it < nitems; it += kPlanThreads) {
            int pi = 0;
            while (s_cnt[pi + 1] <= it) ++pi;
            const int k = pi / nc, j = pi - k * nc;
            const int c = k == 0 ? s_cb[j] : s_cc[j];
            const int nv = s_lo[k][j] + (it - s_cnt[pi]);
            const float w = plan_worst(list(k), c, nv, gp);
            atomicMin((unsigned long long*)&s_key[k][j],
                      (unsigned long long)(((uint64_t)__float_as_uint(w) << 32) | (uint32_t)nv));
        }
        __syncthreads();
        if (tid == 0) {
            for (int j = 0; j < nc; ++j) {
                float w2[2];
                int64_t v2[2];
                for (int k = 0; k < 2; ++k) {
                    w2[k] = __uint_as_float((uint32_t)(s_key[k][j] >> 32));
                    v2[k] = (int64_t)(s_key[k][j] & 0xffffffffu);
                }
                const float wb = kBwdStepCost * w2[0], wc = w2[1];
                const float f = s_cb[j] + s_cc[j] <= ncl ? fmaxf(wb, wc) : wb + wc;
                if (f < s_bf) {
                    s_bf = f;
                    s_bcb = s_cb[j];
                    s_bcc = s_cc[j];
                    s_bnv[0] = v2[0];
                    s_bnv[1] = v2[1];
                }
            }
        }
        __syncthreads();
    }
    // every launch has a feasible candidate: each list alone fits on all ncl pairs
    const int64_t stride = p.ncl;
    if (fwd) {
        write_plan(list(0), plan, stride, s_bcb, s_bnv[0]);
        return;
    }
    if (rnd[0] >= 0) write_plan(list(0), plan + (int64_t)(1 + rnd[0]) * stride * 4, stride, s_bcb, s_bnv[0]);
    if (rnd[1] >= 0) write_plan(list(1), plan + (int64_t)(1 + p.Cmax + rnd[1]) * stride * 4, stride, s_bcc, s_bnv[1]);
    if (tid == 0) {
        split[2 * l] = s_bcb;
        split[2 * l + 1] = s_bcc;
    }
}

// Round lists: block r writes rlist[r] (the sorted positions with a segment in round r, in
// sorted order), rrow[r] (their first rows: the exclusive prefix sum of the segment lengths),
// rcount[r] and rows[r] (the round's total rows).  Sequences longer than the workspace was
// sized for are left out (the forward reports them).
constexpr int kListThreads = 1024;
__global__ void __launch_bounds__(kListThreads) k_round_lists(Prm p, int32_t* rlist, int32_t* rrow, int32_t* rcount) {
    __shared__ int32_t s_n[32], s_l[32];
    const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t base_n = 0, base_rows = 0;
    for (int64_t q0 = 0; q0 < p.S; q0 += kListThreads) {
        const int64_t q = q0 + tid;
        int32_t L = 0;
        if (q < p.S) {
            const int64_t sq = p.order[q];
            const int64_t T = p.off[sq + 1] - p.off[sq];
            if (seg_len(T) <= p.Cmax) L = (int32_t)pass_steps(T, 1 + r);
        }
        const int32_t a = L > 0 ? 1 : 0;
        // block-wide inclusive scans of a and L (warps, then the warp totals)
        int32_t sa = a, sl = L;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t va = __shfl_up_sync(0xffffffffu, sa, d), vl = __shfl_up_sync(0xffffffffu, sl, d);
            if (lane >= d) { sa += va; sl += vl; }
        }
        if (lane == 31) { s_n[warp] = sa; s_l[warp] = sl; }
        __syncthreads();
        if (warp == 0) {
            int32_t wa = s_n[lane], wl = s_l[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t va = __shfl_up_sync(0xffffffffu, wa, d), vl = __shfl_up_sync(0xffffffffu, wl, d);
                if (lane >= d) { wa += va; wl += vl; }
            }
            s_n[lane] = wa;
            s_l[lane] = wl;
        }
        __syncthreads();
        const int32_t pa = (warp > 0 ? s_n[warp - 1] : 0) + sa - a;   // exclusive
        const int32_t pl = (warp > 0 ? s_l[warp - 1] : 0) + sl - L;
        if (a) {
            rlist[(int64_t)r * p.S + base_n + pa] = (int32_t)q;
            rrow[(int64_t)r * p.S + base_n + pa] = base_rows + pl;
        }
        base_n += s_n[31];
        base_rows += s_l[31];
        __syncthreads();                      // s_n / s_l are rewritten by the next chunk
    }
    if (tid == 0) {
        rcount[r] = base_n;
        p.rows[r] = base_rows;
    }
}

// Group state of entries [gstart, gstart + gsize) of the pass's list: round < 0, the forward
// (sorted positions); else round `round` (rlist / rrow of the round).
__device__ void load_gs(const Prm& p, GS& gs, int round, int64_t gstart, int gsize) {
    const int g = threadIdx.x;
    if (g < kG) {
        int64_t pos = -1;
        gs.rowb[g] = 0;
        if (g < gsize) {
            if (round < 0) {
                pos = gstart + g;
            } else {
                pos = p.rlist[(int64_t)round * p.S + gstart + g];
                gs.rowb[g] = p.rrow[(int64_t)round * p.S + gstart + g];
            }
        }
        int64_t sq = pos >= 0 ? p.order[pos] : -1;
        int64_t T = sq >= 0 ? p.off[sq + 1] - p.off[sq] : 0;
        int C = sq >= 0 ? seg_len(T) : 1;
        if (sq >= 0 && C > p.Cmax) {
            report_status(p.status, ACCEL_ERR_SHAPE);
            sq = -1;
            T = 0;
            C = 1;
        }
        gs.seq[g] = sq;
        gs.T[g] = T;
        gs.o0[g] = sq >= 0 ? p.off[sq] : 0;
        gs.C[g] = C;
        gs.w[g] = (sq >= 0 && p.w) ? (float)p.w[sq] : 1.0f;
    }
}

__device__ void round_bounds_gs(GS& gs, int r) {
    const int g = threadIdx.x;
    if (g < kG) {
        gs.t0[g] = 0;
        gs.L[g] = 0;
        gs.just_done[g] = 0;
        if (gs.seq[g] >= 0) {
            const int64_t n = (gs.T[g] + gs.C[g] - 1) / gs.C[g];
            const int64_t k = n - 1 - r;
            gs.just_done[g] = k == -1;
            if (k >= 0) {
                gs.t0[g] = k * gs.C[g];
                const int64_t t1 = gs.t0[g] + gs.C[g] < gs.T[g] ? gs.t0[g] + gs.C[g] : gs.T[g];
                gs.L[g] = t1 - gs.t0[g];
            }
        }
    }
}

// dst[k][c] = BT[k][r Kh + c]
// Rows of the shared-memory arrays that the epilogue threads address 8 floats at a time
// (16 threads per row: the vectors X, the emission half-rows, the partial sums, the S_t rows)
// are stored with their 16-byte chunks permuted: chunk q at chunk position q ^ ((q >> 3) & 1).
// Unpermuted, those accesses would use half of the banks twice.  (An involution: the same
// function maps positions back to chunks.)
__device__ __forceinline__ int pswz(int q) { return q ^ ((q >> 3) & 1); }
__device__ __forceinline__ int pcol(int col) { return 4 * pswz(col >> 2) + (col & 3); }

template <int K>
__device__ void load_bt(const float* __restrict__ BT, int M, int r, float* dst) {
    using S = Sh<K>;
    constexpr int Q = S::Kh / 4;
    const int N = M * Q;
    for (int b0 = threadIdx.x; b0 < N; b0 += kT * 8) {
        float4 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = b0 + e * kT;
            if (idx < N) v[e] = *reinterpret_cast<const float4*>(BT + (int64_t)(idx / Q) * K + r * S::Kh + 4 * (idx % Q));
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = b0 + e * kT;
            if (idx < N) *reinterpret_cast<float4*>(dst + (idx / Q) * S::Kh + 4 * pswz(idx % Q)) = v[e];
        }
    }
}

// The thread's block of the contraction matrix Mx[i][r Kh + c] (row stride Kp), i in its
// warp's part, c in its lane's columns: a[q][h] = (Mx[2q][c0 + h], Mx[2q + 1][c0 + h]).
template <int K>
struct MatRegs {
    using S = Sh<K>;
    float2 a[S::IPART / 2][S::CW];

    __device__ void load(const float* __restrict__ Mx, int Kp, int r) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const float* base = Mx + (int64_t)(w * S::IPART) * Kp + r * S::Kh + lane * S::CW;
        const int cb = w * S::IPART / 4;   // first chunk of the warp's part of a vector
#pragma unroll
        for (int q = 0; q < S::IPART / 2; ++q) {
            // the contraction reads the vector's chunk positions in order; position q/2 holds
            // chunk pswz(cb + q/2), so the matrix rows are taken in that order
            const int lr = 4 * (pswz(cb + (q >> 1)) - cb) + 2 * (q & 1);
            float v0[S::CW], v1[S::CW];
            if constexpr (S::CW == 4) {
                const float4 x0 = *reinterpret_cast<const float4*>(base + (int64_t)lr * Kp);
                const float4 x1 = *reinterpret_cast<const float4*>(base + (int64_t)(lr + 1) * Kp);
                v0[0] = x0.x; v0[1] = x0.y; v0[2] = x0.z; v0[3] = x0.w;
                v1[0] = x1.x; v1[1] = x1.y; v1[2] = x1.z; v1[3] = x1.w;
            } else {
#pragma unroll
                for (int h = 0; h < S::CW; ++h) {
                    v0[h] = base[(int64_t)lr * Kp + h];
                    v1[h] = base[(int64_t)(lr + 1) * Kp + h];
                }
            }
#pragma unroll
            for (int h = 0; h < S::CW; ++h) a[q][h] = make_float2(v0[h], v1[h]);
        }
    }
};

// part[w][g][lane CW + h] = sum_{i in part w} X[g][i] Mx[i][lane CW + h] (chunk-permuted), for
// the 16 g (the second pass is skipped when the group has at most 8 sequences; its slots are
// then stale and unused).
template <int K>
__device__ __forceinline__ void contract(const MatRegs<K>& m, const float* __restrict__ X, float* __restrict__ part,
                                         int gcount) {
    using S = Sh<K>;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* xb = X + w * S::IPART;
    // this lane's CW columns within a row: chunk (lane CW) / 4, offset (lane CW) % 4
    float* pb = part + (w * kG) * S::Kh + 4 * pswz((lane * S::CW) >> 2) + ((lane * S::CW) & 3);
    // the passes are not unrolled: one copy of the unrolled pass body keeps the kernels' hot
    // code small enough for the instruction caches
#pragma unroll 1
    for (int ps = 0; ps < S::NPASS; ++ps) {
        if (ps > 0 && ps * S::GP >= gcount) break;   // (uniform) a group of at most GP sequences
        float2 acc[S::GP][S::CW];
#pragma unroll
        for (int g = 0; g < S::GP; ++g)
#pragma unroll
            for (int h = 0; h < S::CW; ++h) acc[g][h] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < S::IPART / 4; ++q) {
#pragma unroll
            for (int g = 0; g < S::GP; ++g) {
                const float4 x = *reinterpret_cast<const float4*>(xb + (ps * S::GP + g) * K + 4 * q);
#pragma unroll
                for (int h = 0; h < S::CW; ++h) {
                    acc[g][h] = __ffma2_rn(make_float2(x.x, x.y), m.a[2 * q][h], acc[g][h]);
                    acc[g][h] = __ffma2_rn(make_float2(x.z, x.w), m.a[2 * q + 1][h], acc[g][h]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < S::GP; ++g) {
            float* dst = pb + (ps * S::GP + g) * S::Kh;
            if constexpr (S::CW == 4)
                *reinterpret_cast<float4*>(dst) = make_float4(acc[g][0].x + acc[g][0].y, acc[g][1].x + acc[g][1].y,
                                                              acc[g][2].x + acc[g][2].y, acc[g][3].x + acc[g][3].y);
            else if constexpr (S::CW == 2)
                *reinterpret_cast<float2*>(dst) = make_float2(acc[g][0].x + acc[g][0].y, acc[g][1].x + acc[g][1].y);
            else
                *dst = acc[g][0].x + acc[g][0].y;
        }
    }
}

// EC consecutive floats <-> registers (EC is a multiple of 2; 16-byte pieces where possible).
template <int EC>
__device__ __forceinline__ void ldv(const float* __restrict__ src, float (&v)[EC]) {
    if constexpr (EC % 4 == 0) {
#pragma unroll
        for (int e = 0; e < EC; e += 4) {
            const float4 x = *reinterpret_cast<const float4*>(src + e);
            v[e] = x.x; v[e + 1] = x.y; v[e + 2] = x.z; v[e + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < EC; e += 2) {
            const float2 x = *reinterpret_cast<const float2*>(src + e);
            v[e] = x.x; v[e + 1] = x.y;
        }
    }
}
template <int EC>
__device__ __forceinline__ void stv(float* dst, const float (&v)[EC]) {
    if constexpr (EC % 4 == 0) {
#pragma unroll
        for (int e = 0; e < EC; e += 4) *reinterpret_cast<float4*>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
    } else {
#pragma unroll
        for (int e = 0; e < EC; e += 2) *reinterpret_cast<float2*>(dst + e) = make_float2(v[e], v[e + 1]);
    }
}

// EC consecutive floats from / to column c0 (a multiple of EC) of a chunk-permuted row.
template <int EC>
__device__ __forceinline__ void ldv_p(const float* __restrict__ row, int c0, float (&v)[EC]) {
    if constexpr (EC % 4 == 0) {
#pragma unroll
        for (int e = 0; e < EC; e += 4) {
            const float4 x = *reinterpret_cast<const float4*>(row + 4 * pswz((c0 + e) >> 2));
            v[e] = x.x; v[e + 1] = x.y; v[e + 2] = x.z; v[e + 3] = x.w;
        }
    } else {
        const float2 x = *reinterpret_cast<const float2*>(row + pcol(c0));
        v[0] = x.x; v[1] = x.y;
    }
}
template <int EC>
__device__ __forceinline__ void stv_p(float* row, int c0, const float (&v)[EC]) {
    if constexpr (EC % 4 == 0) {
#pragma unroll
        for (int e = 0; e < EC; e += 4)
            *reinterpret_cast<float4*>(row + 4 * pswz((c0 + e) >> 2)) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
    } else {
        *reinterpret_cast<float2*>(row + pcol(c0)) = make_float2(v[0], v[1]);
    }
}

// o = sum over the 8 warps' partials of the thread's epilogue outputs (fixed order).
template <int K>
__device__ __forceinline__ void gather(const float* __restrict__ part, int g, int c0, float (&o)[Sh<K>::EC]) {
    using S = Sh<K>;
    static_assert(S::EC % 4 == 0 || S::EC == 2, "gather: 2 or a multiple of 4 floats per thread");
    ldv_p<S::EC>(part + g * S::Kh, c0, o);
#pragma unroll
    for (int w = 1; w < kNW; ++w) {
        float v[S::EC];
        ldv_p<S::EC>(part + (w * kG + g) * S::Kh, c0, v);
#pragma unroll
        for (int e = 0; e < S::EC; ++e) o[e] += v[e];
    }
}

struct Views {
    float *BTh, *sX, *part, *red, *sX_peer, *red_peer, *St;
};

__device__ __forceinline__ Views make_views(char* smem, int K, int M, cg::cluster_group& cl, int peer) {
    const SL Ls = smem_layout(K, M);
    Views v;
    v.BTh = reinterpret_cast<float*>(smem + Ls.bth);
    v.sX = reinterpret_cast<float*>(smem + Ls.sx);
    v.part = reinterpret_cast<float*>(smem + Ls.part);
    v.red = reinterpret_cast<float*>(smem + Ls.red);
    v.St = reinterpret_cast<float*>(smem + Ls.st);
    v.sX_peer = cl.map_shared_rank(v.sX, peer);
    v.red_peer = cl.map_shared_rank(v.red, peer);
    return v;
}

// ---- the per-step exchange between the two CTAs of a pair.  A CTA writes its half of the
// next vectors (and its partial row sums) into its own shared memory with plain stores and
// into its peer's with st.async, which counts the bytes on the peer's mbarrier of that step
// parity; a CTA then waits on its own mbarrier for the peer's bytes (one arrival: its own
// thread 0 announcing the expected byte count).  No cluster-wide memory fence per step.
struct Xchg {
    uint64_t* bar;           // this CTA's mbarriers, one per step parity
    uint32_t bar_peer0, bar_peer1;   // the peer's, as shared::cluster addresses
    uint32_t sx_peer;        // the peer's vector buffer
    uint32_t red_peer;       // the peer's row-sum slots
    uint32_t phase;          // bit p: parity of the next completion of bar[p]
};

using tc::cluster_addr;
using tc::mbar_try_wait_cluster;
using tc::st_async1;
using tc::st_async2;
using tc::st_async4;

// N floats at column c0 of the chunk-permuted row starting at element `row` of the peer's
// vector buffer (N = 2 or a multiple of 4)
template <int N>
__device__ __forceinline__ void st_peer(const Xchg& xc, uint32_t base, int row, int c0, const float (&v)[N], uint32_t rbar) {
    const uint32_t a = base + 4u * (uint32_t)row;
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int e = 0; e < N; e += 4)
            st_async4(a + 16u * (uint32_t)pswz((c0 + e) >> 2), make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]), rbar);
    } else {
        st_async2(a + 4u * (uint32_t)pcol(c0), make_float2(v[0], v[1]), rbar);
    }
}

// End of a step's writes of parity par: local visibility, then the peer's `bytes`.  Only the
// threads with `wait` set -- the warps whose part of the next contraction reads the peer's
// half of the vectors -- wait for them; the other warps start the next contraction on the
// local half at once, which hides the exchange latency behind their work.  Everything else a
// thread reads of the peer's data (the row sums) it reads after the contraction's CTA
// barrier, which the waiting warps pass only after their wait.  A wait that gives up (2 s)
// records ACCEL_ERR_TIMEOUT; the kernel then finishes its bounded loops with unusable
// values, and the caller sees the status.
__device__ __forceinline__ void xchg_finish(Xchg& xc, int par, uint32_t bytes, int32_t* status, bool wait) {
    __syncthreads();
    uint64_t* bar = par ? &xc.bar[1] : &xc.bar[0];
    if (threadIdx.x == 0) tc::mbar_arrive_expect_tx(bar, bytes);
    const uint32_t ph = (xc.phase >> par) & 1u;
    uint64_t t0 = 0;
    for (uint32_t i = 0; wait; ++i) {
        if (mbar_try_wait_cluster(bar, ph)) break;
        if ((i & 255) == 0) {
            const uint64_t now = tc::globaltimer_ns();
            if (i == 0) t0 = now;
            else if (now - t0 > 2000000000ull) { report_status(status, ACCEL_ERR_TIMEOUT); break; }
        }
    }
    xc.phase ^= 1u << par;
}

// Whether the calling thread's warp reads the peer's half of the vectors in the contraction
// (warp w takes rows w K/8 .. of the matrix, so warps [4r, 4r + 4) read CTA r's half).
__device__ __forceinline__ bool reads_peer_half(int rank) { return (int)(threadIdx.x >> 5) / (kNW / 2) != rank; }

// Sum over the 16 threads of a sequence (a half warp), published as slot (rank) of parity
// par in both CTAs.
__device__ __forceinline__ void publish_sum(float ps, const Views& V, const Xchg& xc, int par, int rank, int g) {
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) ps += __shfl_xor_sync(0xffffffffu, ps, d);
    if ((threadIdx.x & 15) == 0) {
        const int idx = (par * 2 + rank) * kG + g;
        V.red[idx] = ps;
        st_async1(xc.red_peer + 4u * (uint32_t)idx, ps, (par ? xc.bar_peer1 : xc.bar_peer0));
    }
}

__device__ __forceinline__ float row_sum(const float* red, int par, int g) {
    return red[(par * 2) * kG + g] + red[(par * 2 + 1) * kG + g];
}

// X_t = o * sc o b(ob) (or zero when the sequence has ended) into parity nxt of both CTAs,
// and its row sum.
template <int K>
__device__ __forceinline__ void fwd_epilogue(const Views& V, const Xchg& xc, int r, int nxt, int g, int c0, bool on,
                                             int ob, const float (&o)[Sh<K>::EC], float sc) {
    using S = Sh<K>;
    float b[S::EC], v[S::EC];
    ldv_p<S::EC>(V.BTh + ob * S::Kh, c0, b);
    float ps = 0.f;
#pragma unroll
    for (int e = 0; e < S::EC; ++e) {
        v[e] = on ? o[e] * sc * b[e] : 0.f;
        ps += v[e];
    }
    const int row = (nxt * kG + g) * K;
    stv_p<S::EC>(V.sX + row, r * S::Kh + c0, v);
    st_peer<S::EC>(xc, xc.sx_peer, row, r * S::Kh + c0, v, (nxt ? xc.bar_peer1 : xc.bar_peer0));
    publish_sum(ps, V, xc, nxt, r, g);
}

// bytes a CTA receives from its peer per step: its half of the vectors (+ the row sums)
template <int K>
__host__ __device__ constexpr uint32_t xchg_bytes(bool sums) {
    return (uint32_t)(kG * (K / 2) * 4 + (sums ? kG * 4 : 0));
}

__device__ __forceinline__ Xchg make_xchg(const Views& V, uint64_t* bar, int peer) {
    Xchg xc;
    xc.bar = bar;
    xc.bar_peer0 = cluster_addr(&bar[0], (uint32_t)peer);
    xc.bar_peer1 = cluster_addr(&bar[1], (uint32_t)peer);
    xc.sx_peer = cluster_addr(V.sX, (uint32_t)peer);
    xc.red_peer = cluster_addr(V.red, (uint32_t)peer);
    xc.phase = 0;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    return xc;
}

// ---------------------------------------------------------------- forward + checkpoints
// Step t (1 <= t < Tmax) reads X_{t-1} (parity cur) and the row sums of X_{t-1}, takes
// e_{t-1} from them, stores checkpoint t-1 where due, and writes X_t (parity nxt) to both
// CTAs through the pair exchange (no cluster barrier per step).  A last pass (t = Tmax)
// only finishes T-1.
template <int K>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kT, 1) k_fwd_cl(Prm p) {
    using S = Sh<K>;
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank(), peer = r ^ 1;
    const int64_t cidx = blockIdx.x >> 1;
    const int tid = threadIdx.x, g = tid >> 4, c0 = (tid & 15) * S::EC;
    const bool lead = (tid & 15) == 0;    // one thread per sequence
    const bool peer_half = reads_peer_half(r);
    extern __shared__ __align__(16) char smem[];
    __shared__ GS gs;
    __shared__ __align__(8) uint64_t s_xbar[2];
    const Views V = make_views(smem, K, p.M, cl, peer);
    Xchg xc = make_xchg(V, s_xbar, peer);
    MatRegs<K> m;
    m.load(p.A, p.Kp, r);
    load_bt<K>(p.BT, p.M, r, V.BTh);
    // the pair's sequence groups, one after the other
    const int ngr = cluster_groups(p, 0, cidx);
    for (int gi = 0; gi < ngr; ++gi) {
        int64_t gstart;
        int gsize;
        cluster_group_range(p, 0, p.S, cidx, gi, gstart, gsize);
        load_gs(p, gs, -1, gstart, gsize);
        __syncthreads();
        int ob_next = 0;                      // thread g < 16: o_{t+1} for the next symbol write
        if (tid < kG) {
            const int64_t T = gs.T[tid], o0 = gs.o0[tid];
            gs.sym[0][tid] = T > 0 ? p.obs[o0] : 0;
            gs.sym[1][tid] = T > 1 ? p.obs[o0 + 1] : 0;
            ob_next = T > 2 ? p.obs[o0 + 2] : 0;
        }
        int64_t Tmax = 0;
    #pragma unroll
        for (int q = 0; q < kG; ++q) Tmax = gs.T[q] > Tmax ? gs.T[q] : Tmax;
        const int64_t Tg = gs.T[g], base = gs.seq[g] * p.Cmax;
        const int Cg = gs.C[g];
        __syncthreads();
        cl.sync();                            // both CTAs started: shared memory may be written remotely
        {
            // t = 0: alpha~_0 = pi o b(o_0)
            float o[S::EC];
            ldv<S::EC>(p.pi + r * S::Kh + c0, o);
            fwd_epilogue<K>(V, xc, r, 0, g, c0, Tg > 0, gs.sym[0][g], o, 1.f);
        }
        xchg_finish(xc, 0, xchg_bytes<K>(true), p.status, peer_half);
        // the sequence's running exponent sum (used by the lead threads), steps to the next
        // checkpoint and its index
        int64_t E = 0;
        int cp_left = 0, cp_idx = 0;
        for (int64_t t = 1; t <= Tmax; ++t) {
            const int cur = (int)((t - 1) & 1), nxt = (int)(t & 1);
            const int64_t tp = t - 1;
            if (t < Tmax) contract<K>(m, V.sX + cur * kG * K, V.part, gsize);
            __syncthreads();                  // partials complete; the peer's half of X_{t-1} and
                                              // its row sums visible to every thread
            const float c = row_sum(V.red, cur, g);
            const int ex = scale_exp(c);
            const float sc = pow2_scale(ex);
            if (t < Tmax) {
                float o[S::EC];
                gather<K>(V.part, g, c0, o);
                fwd_epilogue<K>(V, xc, r, nxt, g, c0, t < Tg, gs.sym[nxt][g], o, sc);
                if (tid < kG) {
                    gs.sym[cur][tid] = ob_next;   // o_{t+1}, read at step t+1 (parity of t+1 == cur)
                    ob_next = t + 2 < gs.T[tid] ? p.obs[gs.o0[tid] + t + 2] : 0;
                }
            }
            // the bookkeeping of step t-1, off the path to the exchange: X_t is on its way; the
            // checkpoint reads this CTA's half of X_{t-1}, which the peer never writes
            if (tp < Tg) {
                const bool due = cp_left == 0;
                if (lead && r == 0) {
                    if (due) p.cp_e[base + cp_idx] = ex;
                    if (tp == Tg - 1) {
                        const int64_t sq = gs.seq[g];
                        p.clast[sq] = c;
                        if (p.loglik) p.loglik[sq] = 0.6931471805599453 * (double)E + log((double)c);
                    }
                }
                E += ex;
                if (due) {
                    float v[S::EC];
                    ldv_p<S::EC>(V.sX + (cur * kG + g) * K, r * S::Kh + c0, v);
    #pragma unroll
                    for (int e = 0; e < S::EC; ++e) v[e] *= sc;
                    stv<S::EC>(p.cp + (base + cp_idx) * K + r * S::Kh + c0, v);
                    ++cp_idx;
                    cp_left = Cg - 1;
                } else {
                    --cp_left;
                }
            }
            if (t == Tmax) break;
            xchg_finish(xc, nxt, xchg_bytes<K>(true), p.status, peer_half);
        }
        cl.sync();
        cl.sync();                        // the peer is done with this CTA's shared memory
    }
}

// ---------------------------------------------------------------- recompute a segment
// S_t for t in the round's segment into the P rows (normalised), e_t into ebuf; the same
// step structure as the forward, starting from the checkpoint row (e = its stored
// exponent, scale 1).
// (the groups of CTA pair cidx of the recomputation pass of round `round`; m holds A)
template <int K>
__device__ __forceinline__ void rec_groups(const Prm& p, int round, int64_t cidx, cg::cluster_group& cl,
                                           const Views& V, Xchg& xc, const MatRegs<K>& m, GS& gs) {
    using S = Sh<K>;
    const int r = (int)cl.block_rank();
    const int tid = threadIdx.x, g = tid >> 4, c0 = (tid & 15) * S::EC;
    const bool lead = (tid & 15) == 0;
    const bool peer_half = reads_peer_half(r);
    float* const Pw = round_P(p, round);
    int32_t* const ew = round_e(p, round);
    // the pair's sequence groups, one after the other
    const int pass = 1 + p.Cmax + round;
    const int64_t nlist = p.rcount[round];
    const int ngr = cluster_groups(p, pass, cidx);
    for (int gi = 0; gi < ngr; ++gi) {
        int64_t gstart;
        int gsize;
        cluster_group_range(p, pass, nlist, cidx, gi, gstart, gsize);
        load_gs(p, gs, round, gstart, gsize);
        __syncthreads();
        round_bounds_gs(gs, round);
        __syncthreads();
        int maxL = 0;
    #pragma unroll
        for (int q = 0; q < kG; ++q) maxL = gs.L[q] > maxL ? (int)gs.L[q] : maxL;
        const int Lg = (int)gs.L[g];
        const int64_t rowb = gs.rowb[g];
        // row 0: the checkpoint itself, into the local vector buffer and the P row
        for (int idx = tid; idx < kG * K / 4; idx += kT) {
            const int gg = idx / (K / 4), cc = 4 * (idx - gg * (K / 4));
            float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gs.L[gg] > 0) {
                sv = *reinterpret_cast<const float4*>(p.cp + (gs.seq[gg] * p.Cmax + gs.t0[gg] / gs.C[gg]) * K + cc);
                if (cc / S::Kh == r) *reinterpret_cast<float4*>(Pw + (int64_t)gs.rowb[gg] * K + cc) = sv;
            }
            *reinterpret_cast<float4*>(V.sX + gg * K + pcol(cc)) = sv;
        }
        int ob_next = 0;
        if (tid < kG) {
            const int q = tid;
            if (gs.L[q] > 0 && r == 0) ew[gs.rowb[q]] = p.cp_e[gs.seq[q] * p.Cmax + gs.t0[q] / gs.C[q]];
            const int64_t b0 = gs.o0[q] + gs.t0[q];
            gs.sym[1][q] = gs.L[q] > 1 ? p.obs[b0 + 1] : 0;
            ob_next = gs.L[q] > 2 ? p.obs[b0 + 2] : 0;
        }
        if (maxL <= 1) {                      // no remote access made; the peer skips it too
            __syncthreads();                  // (gs is rewritten for the next group)
            continue;
        }
        __syncthreads();
        cl.sync();
        for (int tt = 1; tt <= maxL; ++tt) {
            const int cur = (tt - 1) & 1, nxt = tt & 1;
            if (tt < maxL) contract<K>(m, V.sX + cur * kG * K, V.part, gsize);
            __syncthreads();                  // partials complete; the peer's half of X_{tt-1} and
                                              // its row sums visible to every thread
            int ex = 0;
            float sc = 1.f;
            if (tt >= 2) {
                ex = scale_exp(row_sum(V.red, cur, g));
                sc = pow2_scale(ex);
            }
            if (tt < maxL) {
                float o[S::EC];
                gather<K>(V.part, g, c0, o);
                fwd_epilogue<K>(V, xc, r, nxt, g, c0, tt < Lg, gs.sym[nxt][g], o, sc);
                if (tid < kG) {
                    gs.sym[cur][tid] = ob_next;
                    ob_next = tt + 2 < gs.L[tid] ? p.obs[gs.o0[tid] + gs.t0[tid] + tt + 2] : 0;
                }
            }
            // the P row of step tt-1, off the path to the exchange: X_tt is on its way; the row
            // is this CTA's half of X_{tt-1}, which the peer never writes
            if (tt >= 2 && tt - 1 < Lg) {
                const int tp = tt - 1;
                if (lead && r == 0) ew[rowb + tp] = ex;
                float v[S::EC];
                ldv_p<S::EC>(V.sX + (cur * kG + g) * K, r * S::Kh + c0, v);
    #pragma unroll
                for (int e = 0; e < S::EC; ++e) v[e] *= sc;
                stv<S::EC>(Pw + (rowb + tp) * K + r * S::Kh + c0, v);
            }
            if (tt == maxL) break;
            xchg_finish(xc, nxt, xchg_bytes<K>(true), p.status, peer_half);
        }
        cl.sync();
        cl.sync();                        // the peer is done with this CTA's shared memory
    }
}

// ---------------------------------------------------------------- backward over a segment
// Step tt (from L-1 down to 0) reads v_{t+1} = b(o_{t+1}) o R_{t+1} (parity tt), forms
// R_t = 2^-e_t A v_{t+1} (or 1/c'_{T-1} at the last step of a sequence) and
// gamma_t = w 2^e_t S_t o R_t, then writes v_t = b(o_t) o R_t (parity tt-1) to both CTAs
// together with the Q row of step tt-1 (the pair exchange, no cluster barrier).  R_t stays in the
// registers of the thread that owns the (sequence, state) pair.
//   sym(tt) = o_{t0+tt} if t0+tt < T and tt <= L, else -1: the epilogue symbol o_t of an
//   active step and the symbol of v_t; sym(tt+1) >= 0 says whether step tt is a transition.
// (the groups of CTA pair cidx of the backward pass of round `round`; m holds A^T)
template <int K>
__device__ __forceinline__ void bwd_groups(const Prm& p, int round, int64_t cidx, cg::cluster_group& cl,
                                           const Views& V, Xchg& xc, const MatRegs<K>& m, GS& gs) {
    using S = Sh<K>;
    const int r = (int)cl.block_rank();
    const int tid = threadIdx.x, g = tid >> 4, c0 = (tid & 15) * S::EC;
    const bool lead = (tid & 15) == 0;
    const bool peer_half = reads_peer_half(r);
    const float* const Pr = round_P(p, round);
    const int32_t* const er = round_e(p, round);
    float* const Qw = round_Q(p, round);
    float* const Gw = round_gam(p, round);
    int32_t* const Ow = round_osym(p, round);
    // the pair's sequence groups, one after the other
    const int pass = 1 + round;
    const int64_t nlist = p.rcount[round];
    const int ngr = cluster_groups(p, pass, cidx);
    for (int gi = 0; gi < ngr; ++gi) {
        int64_t gstart;
        int gsize;
        cluster_group_range(p, pass, nlist, cidx, gi, gstart, gsize);
        load_gs(p, gs, round, gstart, gsize);
        __syncthreads();
        round_bounds_gs(gs, round);
        __syncthreads();
        int maxL = 0;
    #pragma unroll
        for (int q = 0; q < kG; ++q) maxL = gs.L[q] > maxL ? (int)gs.L[q] : maxL;
        const int Lg = (int)gs.L[g];
        const int64_t rowb = gs.rowb[g];
        const int jc = r * S::Kh + c0;        // first state of the thread's epilogue block
        // (the round's rows are packed: every row below rows[round] belongs to a step of a
        // sequence in the round and is written below, so no row needs clearing)
        if (maxL == 0) {                      // no remote access made; the peer skips it too
            __syncthreads();                  // (gs is rewritten for the next group)
            continue;
        }
        auto sym_at = [&](int q, int tt) -> int {
            const int64_t t = gs.t0[q] + tt;
            return (tt <= gs.L[q] && t < gs.T[q] && gs.seq[q] >= 0) ? p.obs[gs.o0[q] + t] : -1;
        };
        auto e_at = [&](int q, int tt) -> int { return tt < gs.L[q] ? er[(int64_t)gs.rowb[q] + tt] : 0; };
        int nsym = -1, ne = 0;                // thread q < 16: scalars of step tt-1, loaded one step ahead
        if (tid < kG) {
            const int q = tid;
            gs.sym_end[q] = sym_at(q, maxL);
            gs.sym[(maxL - 1) & 1][q] = sym_at(q, maxL - 1);
            gs.eb[(maxL - 1) & 1][q] = e_at(q, maxL - 1);
            if (maxL >= 2) {
                nsym = sym_at(q, maxL - 2);
                ne = e_at(q, maxL - 2);
            }
        }
        for (int idx = tid; idx < 2 * kG * K; idx += kT) V.sX[idx] = 0.f;
        __syncthreads();
        cl.sync();                            // both CTAs started and zeroed before any remote write
        const float wg = gs.w[g];
        const bool last_seg = gs.t0[g] + Lg == gs.T[g];
        float R[S::EC];                       // R_{t+1} of the thread's (sequence, state) pairs
        if (Lg > 0 && !last_seg) {
            ldv<S::EC>(p.Rc + gs.seq[g] * K + jc, R);
        } else {
    #pragma unroll
            for (int e = 0; e < S::EC; ++e) R[e] = 0.f;
        }
        int prev_sym = gs.sym_end[g];
        // v = b(s) o R for step tt into both CTAs, and the Q row of step tt
        // (every thread sends its part each step -- zeros for a sequence not in step tt -- so the
        // peer's expected byte count is constant; the Q row is written only for active steps)
        auto write_v = [&](int tt, int s, bool active) {
            float v[S::EC], b[S::EC];
            if (active && s >= 0) {
                ldv_p<S::EC>(V.BTh + s * S::Kh, c0, b);
    #pragma unroll
                for (int e = 0; e < S::EC; ++e) v[e] = b[e] * R[e];
            } else {
    #pragma unroll
                for (int e = 0; e < S::EC; ++e) v[e] = 0.f;
            }
            const int row = ((tt & 1) * kG + g) * K;
            stv_p<S::EC>(V.sX + row, jc, v);
            st_peer<S::EC>(xc, xc.sx_peer, row, jc, v, ((tt & 1) ? xc.bar_peer1 : xc.bar_peer0));
            if (active) {
    #pragma unroll
                for (int e = 0; e < S::EC; ++e) v[e] *= wg;
                stv<S::EC>(Qw + (rowb + tt) * K + jc, v);
            }
        };
        write_v(maxL - 1, prev_sym, maxL - 1 < Lg);
        xchg_finish(xc, (maxL - 1) & 1, xchg_bytes<K>(false), p.status, peer_half);
        for (int tt = maxL - 1; tt >= 0; --tt) {
            const int buf = tt & 1;
            const int sym = gs.sym[buf][g], e_t = gs.eb[buf][g];
            const bool on = tt < Lg;
            // S_t of the thread's pairs, copied asynchronously into shared memory while the
            // contraction runs (keeps registers free)
            float* st_row = V.St + g * S::Kh;      // chunk-permuted like the vectors
            if (on) {
                const float* src = Pr + (rowb + tt) * K + jc;
    #pragma unroll
                for (int e = 0; e < S::EC; e += 2) {
                    if constexpr (S::EC % 4 == 0) {
                        if (e % 4 == 0)
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                         ::"r"(tc::smem_u32(st_row + 4 * pswz((c0 + e) >> 2))), "l"(src + e) : "memory");
                    } else {
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(st_row + pcol(c0 + e))),
                                     "l"(src + e) : "memory");
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            contract<K>(m, V.sX + buf * kG * K, V.part, gsize);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            float St[S::EC];
            if (on) ldv_p<S::EC>(st_row, c0, St);
            if (on) {
                float o[S::EC];
                gather<K>(V.part, g, c0, o);
                const bool trans = prev_sym >= 0;
                const float down = pow2_scale(e_t);
                const float up = wg * pow2_scale(-e_t);
                const float cinv = trans ? 0.f : 1.0f / p.clast[gs.seq[g]];
                float gm[S::EC];
    #pragma unroll
                for (int e = 0; e < S::EC; ++e) {
                    R[e] = trans ? o[e] * down : cinv;
                    gm[e] = up * St[e] * R[e];
                }
                stv<S::EC>(Gw + (rowb + tt) * K + jc, gm);
                if (lead && r == 0) Ow[rowb + tt] = sym;
            }
            if (tt > 0) write_v(tt - 1, sym, tt - 1 < Lg);
            prev_sym = sym;
            if (tid < kG && tt > 0) {
                gs.sym[(tt - 1) & 1][tid] = nsym;
                gs.eb[(tt - 1) & 1][tid] = ne;
                if (tt >= 2) {
                    nsym = sym_at(tid, tt - 2);
                    ne = e_at(tid, tt - 2);
                }
            }
            if (tt > 0) xchg_finish(xc, (tt - 1) & 1, xchg_bytes<K>(false), p.status, peer_half);
        }
        if (Lg > 0) stv<S::EC>(p.Rc + gs.seq[g] * K + jc, R);
        // gamma_0 of the sequences that started in this round, summed in a fixed order by one
        // thread per state (the gam rows written above are visible after the barrier)
        __syncthreads();
        for (int cc = tid; cc < S::Kh; cc += kT) {
            const int j = r * S::Kh + cc;
            float s = 0.f;
            for (int q = 0; q < kG; ++q)
                if (gs.L[q] > 0 && gs.t0[q] == 0) s += Gw[(int64_t)gs.rowb[q] * K + j];
            p.pig[cidx * K + j] += s;
        }
        cl.sync();                        // the peer is done with this CTA's shared memory
    }
}

// The recomputation of round `round` and the backward of round `round`, each on the CTA pairs
// its pass was planned for (see k_plan): np >= 0 pairs from the host, else from the plan --
// backward launch l holds the backward of round l - 1 (split[2 l] pairs) beside the
// recomputation of round l (split[2 l + 1] pairs), as two kernels on two streams.  Pairs past
// the count leave at once (both CTAs of a pair alike, before any remote access).
template <int K>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kT, 1) k_rec_cl(Prm p, int round, int np) {
    const int64_t pair = blockIdx.x >> 1;
    if (pair >= (np >= 0 ? (int64_t)np : (int64_t)p.split[2 * round + 1])) return;
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank(), peer = r ^ 1;
    extern __shared__ __align__(16) char smem[];
    __shared__ GS gs;
    __shared__ __align__(8) uint64_t s_xbar[2];
    const Views V = make_views(smem, K, p.M, cl, peer);
    Xchg xc = make_xchg(V, s_xbar, peer);
    MatRegs<K> m;
    m.load(p.A, p.Kp, r);
    load_bt<K>(p.BT, p.M, r, V.BTh);
    rec_groups<K>(p, round, pair, cl, V, xc, m, gs);
}

template <int K>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kT, 1) k_bwd_cl(Prm p, int round, int np) {
    const int64_t pair = blockIdx.x >> 1;
    if (pair >= (np >= 0 ? (int64_t)np : (int64_t)p.split[2 * (round + 1)])) return;
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank(), peer = r ^ 1;
    extern __shared__ __align__(16) char smem[];
    __shared__ GS gs;
    __shared__ __align__(8) uint64_t s_xbar[2];
    const Views V = make_views(smem, K, p.M, cl, peer);
    Xchg xc = make_xchg(V, s_xbar, peer);
    MatRegs<K> m;
    m.load(p.At, p.Kp, r);
    load_bt<K>(p.BT, p.M, r, V.BTh);
    bwd_groups<K>(p, round, pair, cl, V, xc, m, gs);
}

struct Kernels {
    void (*fwd)(Prm);
    void (*rec)(Prm, int, int);
    void (*bwd)(Prm, int, int);
};

inline Kernels kernels_for(int K) {
    switch (K) {
        case 64: return Kernels{k_fwd_cl<64>, k_rec_cl<64>, k_bwd_cl<64>};
        case 128: return Kernels{k_fwd_cl<128>, k_rec_cl<128>, k_bwd_cl<128>};
        default: return Kernels{k_fwd_cl<256>, k_rec_cl<256>, k_bwd_cl<256>};
    }
}

}  // namespace clu

struct Layout {
    size_t A, At, BT, pi, cp, cp_e, clast, P, Q, Rc, cnt, pig, Upart, rows, ebuf, gam, osym, cntp, plan, rlist, rrow,
        rcount, Pb[kPBufs], ebuf2, Qb[kQBufs], Gb[kQBufs], Ob[kQBufs], split, order, total;
    int Cmax;
    int64_t ngroups;
    int64_t npig;       // rows of pig: one per group of either path (clusters: up to S)
};

static Layout layout(int K, int M, int64_t S, int64_t max_T) {
    Layout L;
    L.Cmax = seg_len(max_T < 1 ? 1 : max_T);
    L.ngroups = (S + kG - 1) / kG;
    size_t o = kStatusBytes;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    const size_t Kp = (size_t)((K + 3) & ~3);
    L.A = take((size_t)K * Kp * 4);
    L.At = take((size_t)K * Kp * 4);
    L.BT = take((size_t)M * K * 4);
    L.pi = take((size_t)K * 4);
    L.cp = take((size_t)S * L.Cmax * K * 4);
    L.cp_e = take((size_t)S * L.Cmax * 4);
    L.clast = take((size_t)S * 4);
    L.P = take((size_t)S * L.Cmax * K * 4);
    L.Q = take((size_t)S * L.Cmax * K * 4);
    L.Rc = take((size_t)S * K * 4);
    L.cnt = take((size_t)L.ngroups * K * M * 4);
    L.npig = L.ngroups > S ? L.ngroups : S;
    L.pig = take((size_t)L.npig * K * 4);
    const int ns_max = xi_tc_supported(K) ? (kXiSplitMax > kSplit ? kXiSplitMax : kSplit) : kSplit;
    L.Upart = take((size_t)ns_max * K * K * 4);
    L.rows = take((size_t)L.Cmax * 4);
    L.ebuf = take((size_t)S * L.Cmax * 4);
    L.gam = take((size_t)S * L.Cmax * K * 4);
    L.osym = take((size_t)S * L.Cmax * 4);
    L.cntp = take((size_t)(ns_max > kCntSplit ? ns_max : kCntSplit) * K * M * 4);
    // group plans of the CTA pairs: the forward, and every round's backward and recomputation
    L.plan = take((size_t)(2 * L.Cmax + 1) * (adj::clu::kPlanMaxGroups / 2) * 4 * 8);
    L.rlist = take((size_t)L.Cmax * S * 4);
    L.rrow = take((size_t)L.Cmax * S * 4);
    L.rcount = take((size_t)L.Cmax * 4);
    // cluster path: the further row buffers of the rounds, and each backward launch's split
    const bool clu_rows = adj::clu::cluster_shape_ok(K);
    const size_t rowsK = clu_rows ? (size_t)S * L.Cmax * K * 4 : 0, rows1 = clu_rows ? (size_t)S * L.Cmax * 4 : 0;
    L.Pb[0] = L.P;
    L.Qb[0] = L.Q;
    L.Gb[0] = L.gam;
    L.Ob[0] = L.osym;
    for (int k = 1; k < kPBufs; ++k) L.Pb[k] = take(rowsK);
    L.ebuf2 = take(rows1);
    for (int k = 1; k < kQBufs; ++k) {
        L.Qb[k] = take(rowsK);
        L.Gb[k] = take(rowsK);
        L.Ob[k] = take(rows1);
    }
    L.split = take((size_t)(L.Cmax + 1) * 2 * 4);
    L.order = o;
    L.total = o + order_ws_bytes(S);
    return L;
}

static int padK(int K) { return (K + 3) & ~3; }
static size_t smem_fwd(int K, int M) { return off_ss(K, M, padK(K)) + (size_t)kG * padK(K) * 4; }
static size_t smem_bwd(int K, int M, int Cmax) {
    return off_ss(K, M, padK(K)) + 2 * (size_t)kG * padK(K) * 4 + (size_t)kG * Cmax * 4;
}

}  // namespace adj
}  // namespace hmm
}  // namespace accel

using namespace accel;
using namespace accel::hmm;

namespace accel {
namespace hmm {
accel_status check_model(const accel_hmm_model* m, const char* who);
}
}  // namespace accel

extern "C" {

size_t hmm_adjoint_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T, int64_t max_T) {
    (void)total_T;
    if (!m || S < 0) return 0;
    return adj::layout(m->K, m->M, S, max_T).total;
}

}  // extern "C"

namespace accel {
namespace hmm {
namespace adj {

// What both phases of the adjoint derive from the arguments (the same decisions every call).
struct Plan {
    Layout L;
    Prm p;
    int K, M, nb, nsU, nsC;
    size_t sm_b, sm_c;
    bool use_cluster, xi_tc, counts_tc, planned;
    float* cntp;
    float* Upart;
    char* ws;
};

static accel_status setup(const char* who, const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets,
                          int64_t S, int64_t total_T, int64_t max_T, void* d_ws, size_t ws_bytes, Plan& P) {
    accel_status r = check_model(m, who);
    if (r != ACCEL_OK) return r;
    ACCEL_REQUIRE(S >= 0 && total_T >= 0 && max_T >= 0, ACCEL_ERR_INVALID_ARG, "%s: negative size", who);
    ACCEL_REQUIRE(d_offsets && d_ws && (total_T == 0 || d_obs), ACCEL_ERR_INVALID_ARG, "%s: null pointer", who);
    ACCEL_REQUIRE(((uintptr_t)d_ws % 256) == 0, ACCEL_ERR_INVALID_ARG, "%s: d_ws must be 256-byte aligned", who);
    const int K = m->K, M = m->M;
    P.K = K;
    P.M = M;
    P.L = layout(K, M, S, max_T);
    const Layout& L = P.L;
    ACCEL_REQUIRE(ws_bytes >= L.total, ACCEL_ERR_WORKSPACE, "%s: workspace %zu < %zu bytes", who, ws_bytes, L.total);
    ACCEL_REQUIRE(S * (int64_t)L.Cmax <= (int64_t)INT32_MAX, ACCEL_ERR_UNSUPPORTED,
                  "%s: S x ceil(sqrt(max_T)) = %lld rows exceeds 2^31-1", who, (long long)(S * (int64_t)L.Cmax));
    P.sm_b = smem_bwd(K, M, L.Cmax);
    char* ws = (char*)d_ws;
    P.ws = ws;
    Prm& p = P.p;
    p.K = K; p.M = M; p.Cmax = L.Cmax; p.S = S; p.Kp = padK(K);
    p.status = status_word((int32_t*)(ws + kStatusOff));
    p.rows = (int32_t*)(ws + L.rows);
    p.ebuf = (int32_t*)(ws + L.ebuf);
    p.gam = (float*)(ws + L.gam);
    p.osym = (int32_t*)(ws + L.osym);
    p.ncl = 0;
    p.ncl_fwd = 0;
    p.plan = nullptr;
    p.rlist = (int32_t*)(ws + L.rlist);
    p.rrow = (int32_t*)(ws + L.rrow);
    p.rcount = (int32_t*)(ws + L.rcount);
    for (int k = 0; k < kPBufs; ++k) p.Pb[k] = (float*)(ws + L.Pb[k]);
    p.ebuf2 = (int32_t*)(ws + L.ebuf2);
    for (int k = 0; k < kQBufs; ++k) {
        p.Qb[k] = (float*)(ws + L.Qb[k]);
        p.Gb[k] = (float*)(ws + L.Gb[k]);
        p.Ob[k] = (int32_t*)(ws + L.Ob[k]);
    }
    p.split = nullptr;
    P.cntp = (float*)(ws + L.cntp);
    p.A = (float*)(ws + L.A); p.At = (float*)(ws + L.At); p.BT = (float*)(ws + L.BT); p.pi = (float*)(ws + L.pi);
    p.obs = d_obs; p.off = d_offsets; p.order = (int32_t*)(ws + L.order); p.w = nullptr;
    p.cp = (float*)(ws + L.cp); p.cp_e = (int32_t*)(ws + L.cp_e); p.clast = (float*)(ws + L.clast);
    p.loglik = nullptr; p.P = (float*)(ws + L.P); p.Q = (float*)(ws + L.Q); p.Rc = (float*)(ws + L.Rc);
    p.cnt = (float*)(ws + L.cnt); p.pig = (float*)(ws + L.pig);
    P.Upart = (float*)(ws + L.Upart);
    P.nb = (K + kTile - 1) / kTile;
    P.sm_c = clu::smem_layout(K, M).total;
    // the cluster kernels leave the emission counts to the tensor-core kernel or to k_counts
    // (an [M][256] table in shared memory); otherwise the streaming kernels take the shape
    const bool counts_fit = xi_tc_counts_supported(K, M) || (size_t)M * 256 * 4 <= (size_t)max_smem_optin();
    P.use_cluster = S > 0 && clu::cluster_shape_ok(K) && P.sm_c <= (size_t)max_smem_optin() && counts_fit;
    // the streaming kernels hold the whole emission table in shared memory
    ACCEL_REQUIRE(P.use_cluster || S == 0 || P.sm_b <= (size_t)max_smem_optin(), ACCEL_ERR_UNSUPPORTED,
                  "%s: emission table too large for shared memory (K=%d, M=%d)", who, K, M);
    P.xi_tc = P.use_cluster && xi_tc_supported(K);
    P.counts_tc = P.xi_tc && xi_tc_counts_supported(K, M);
    P.nsU = P.xi_tc ? xi_tc_partials(K, M, P.counts_tc) : kSplit;
    P.nsC = P.counts_tc ? xi_tc_partials(K, M, true) : kCntSplit;
    P.planned = false;
    if (P.use_cluster) {
        // groups: at most 16 sequences each, and at least one pair of CTAs per two SMs
        const int64_t ncl_min = (S + clu::kG - 1) / clu::kG;
        const int64_t ncl_sm = S < (int64_t)(num_sms() / 2) ? S : (int64_t)(num_sms() / 2);
        if (ncl_min <= 2 * ncl_sm && 2 * ncl_sm <= clu::kPlanMaxGroups && S <= clu::kPlanMaxSeq) {
            // one pair per two SMs, each running one or two groups (planned on the device
            // from the sorted lengths by the forward phase); the forward recursion within the
            // SM budget, with at least the pairs that hold every sequence in two groups
            p.ncl = ncl_sm;
            p.ncl_fwd = ncl_sm;
            const int64_t budget = sm_budget();
            if (budget > 0 && budget / 2 < ncl_sm) {
                const int64_t need = (ncl_min + 1) / 2;
                p.ncl_fwd = budget / 2 > need ? budget / 2 : need;
                if (p.ncl_fwd < 1) p.ncl_fwd = 1;
            }
            p.plan = (int64_t*)(ws + L.plan);
            p.split = (int32_t*)(ws + L.split);
            P.planned = true;
        } else {
            p.ncl = ncl_min > ncl_sm ? ncl_min : ncl_sm;
            p.ncl_fwd = p.ncl;
        }
    }
    return ACCEL_OK;
}

// Phase 1: parameters prepared, sequences ordered and (cluster path) grouped, the forward pass
// with its checkpoints and logL.  Everything phase 2 reads stays in the workspace.
static accel_status run_forward(Plan& P, const accel_hmm_model* m, double* d_loglik, cudaStream_t st, int& nlaunch) {
    Prm& p = P.p;
    const Layout& L = P.L;
    const int K = P.K, M = P.M;
    char* ws = P.ws;
    p.loglik = d_loglik;
    int pg = num_sms() * 4;
    k_prep<<<pg, 256, 0, st>>>(m->log_A, m->log_B, m->log_pi, K, p.Kp, M, (float*)p.A, (float*)p.At, (float*)p.BT,
                               (float*)p.pi);
    ++nlaunch;
    if (p.S == 0) return ACCEL_OK;
    accel_status r = order_by_length(p.off, p.S, (int32_t*)(ws + L.order), ws + L.order + align_up((size_t)p.S * 4, 256), st);
    if (r != ACCEL_OK) return r;
    nlaunch += 3;
    if (P.use_cluster) {
        // the backward rounds' sequence lists and packed row offsets (they depend on the
        // lengths only, so they belong to the saved state), then the plans of every pass
        clu::k_round_lists<<<(unsigned)L.Cmax, clu::kListThreads, 0, st>>>(p, (int32_t*)p.rlist, (int32_t*)p.rrow,
                                                                          (int32_t*)p.rcount);
        ++nlaunch;
        if (P.planned) {
            const size_t sm_plan = clu::plan_smem_bytes();
            ACCEL_CUDA_TRY(cudaFuncSetAttribute(clu::k_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_plan));
            clu::k_plan<<<(unsigned)(L.Cmax + 2), clu::kPlanThreads, sm_plan, st>>>(p, (int64_t*)p.plan,
                                                                                   (int32_t*)p.split, K == 256 ? 8 : 16);
            ++nlaunch;
        }
        const unsigned grid = (unsigned)(2 * p.ncl_fwd);
        const clu::Kernels kc = clu::kernels_for(K);
        ACCEL_CUDA_TRY(cudaFuncSetAttribute(kc.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.sm_c));
        kc.fwd<<<grid, clu::kT, P.sm_c, st>>>(p);
        ++nlaunch;
    } else {
        size_t sm_f = smem_fwd(K, M);
        ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_forward_cp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_f));
        k_forward_cp<<<(unsigned)L.ngroups, kT, sm_f, st>>>(p);
        ++nlaunch;
    }
    p.loglik = nullptr;
    return ACCEL_OK;
}

// The backward phase's streams on the cluster path, created once per host thread and device
// (non-blocking, so they order only against the caller's stream through events): the
// backward passes and the recomputations at the highest priority, the counts at the lowest.
struct BwdStreams {
    cudaStream_t hi = nullptr, hi2 = nullptr, lo = nullptr;
};
static accel_status bwd_streams(BwdStreams& out) {
    thread_local std::map<int, BwdStreams> cache;
    int dev = 0;
    ACCEL_CUDA_TRY(cudaGetDevice(&dev));
    auto it = cache.find(dev);
    if (it == cache.end()) {
        int least = 0, greatest = 0;
        ACCEL_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BwdStreams s;
        ACCEL_CUDA_TRY(cudaStreamCreateWithPriority(&s.hi, cudaStreamNonBlocking, greatest));
        ACCEL_CUDA_TRY(cudaStreamCreateWithPriority(&s.hi2, cudaStreamNonBlocking, greatest));
        ACCEL_CUDA_TRY(cudaStreamCreateWithPriority(&s.lo, cudaStreamNonBlocking, least));
        it = cache.emplace(dev, s).first;
    }
    out = it->second;
    return ACCEL_OK;
}

// Events of one call, destroyed when it returns (the waits already enqueued still hold).
struct EventSet {
    std::vector<cudaEvent_t> ev;
    cudaError_t make(cudaEvent_t& e) {
        const cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r == cudaSuccess) ev.push_back(e);
        return r;
    }
    ~EventSet() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// Phase 2: the rounds of recomputation and the backward recursion, the count accumulation, and
// the gradients.  Reads phase 1's checkpoints, order and plan; clears its own accumulators.
static accel_status run_backward(Plan& P, const double* d_weights, float* d_grad_log_A, float* d_grad_log_B,
                                 float* d_grad_log_pi, cudaStream_t st, int& nlaunch) {
    Prm& p = P.p;
    const Layout& L = P.L;
    const int K = P.K, M = P.M;
    const int64_t S = p.S;
    char* ws = P.ws;
    p.w = d_weights;
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.cnt, 0, (size_t)L.ngroups * K * M * 4, st));
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.pig, 0, (size_t)L.npig * K * 4, st));
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.Upart, 0, (size_t)P.nsU * K * K * 4, st));
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.cntp, 0, (size_t)P.nsC * K * M * 4, st));
    if (!P.use_cluster) {
        // the streaming kernels keep Cmax row slots per sequence and clear the ones they
        // leave; the cluster path packs each round's rows (all written in the round) and its
        // row counts were set by the forward phase
        ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.P, 0, (size_t)S * L.Cmax * K * 4, st));
        ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.Q, 0, (size_t)S * L.Cmax * K * 4, st));
        ACCEL_CUDA_TRY(cudaMemsetAsync(ws + L.rows, 0, (size_t)L.Cmax * 4, st));
    }
    if (S > 0) {
        if (P.use_cluster) {
            const clu::Kernels kc = clu::kernels_for(K);
            ACCEL_CUDA_TRY(cudaFuncSetAttribute(kc.rec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.sm_c));
            ACCEL_CUDA_TRY(cudaFuncSetAttribute(kc.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.sm_c));
            const size_t sm_cnt = (size_t)M * 256 * 4;
            if (!P.counts_tc) {
                ACCEL_REQUIRE(sm_cnt <= (size_t)max_smem_optin(), ACCEL_ERR_UNSUPPORTED, "hmm_adjoint: M=%d too large", M);
                ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cnt));
            }
            const int nbc = (K + 255) / 256;
            // Three streams of this thread's phase: the backward passes (hi) and the
            // recomputations (hi2) at the highest priority, the counts (lo) at the lowest.  The
            // backward of round l - 1 runs beside the recomputation of round l on the CTA pairs
            // the plan splits between them; the counts of round r run beside what follows
            // (their rows are in other buffers).  Before a pass writes a buffer again, it waits
            // for the last reader of the round that used it; the caller's stream waits for all
            // three at the end.
            BwdStreams bs;
            accel_status rs = bwd_streams(bs);
            if (rs != ACCEL_OK) return rs;
            EventSet ev;
            cudaEvent_t e_fork;
            ACCEL_CUDA_TRY(ev.make(e_fork));
            ACCEL_CUDA_TRY(cudaEventRecord(e_fork, st));
            ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.hi, e_fork, 0));
            ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.hi2, e_fork, 0));
            ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.lo, e_fork, 0));
            const size_t nr = (size_t)L.Cmax;
            std::vector<cudaEvent_t> e_rec(nr, nullptr), e_bwd(nr, nullptr), done(nr, nullptr);
            // the counts of a round, once its backward has written its rows
            auto counts = [&](int round) -> accel_status {
                ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.lo, e_bwd[round], 0));
                const float* Pr = clu::round_P(p, round);
                const float* Qr = clu::round_Q(p, round);
                const float* Gr = clu::round_gam(p, round);
                const int32_t* Or = clu::round_osym(p, round);
                if (P.xi_tc) {
                    accel_status r = xi_tc_round(Pr, Qr, Gr, Or, p.rows + round, K, M, P.Upart,
                                                 P.counts_tc ? P.cntp : nullptr, p.status, bs.lo);
                    if (r != ACCEL_OK) return r;
                } else {
                    k_gemm_ptq<<<P.nb * P.nb * kSplit, 256, 0, bs.lo>>>(Pr, Qr, p.rows + round, K, P.Upart);
                }
                ++nlaunch;
                if (!P.counts_tc) {
                    k_counts<<<nbc * kCntSplit, 256, sm_cnt, bs.lo>>>(Gr, Or, p.rows + round, K, M, P.cntp);
                    ++nlaunch;
                }
                ACCEL_CUDA_TRY(ev.make(done[round]));
                ACCEL_CUDA_TRY(cudaEventRecord(done[round], bs.lo));
                return ACCEL_OK;
            };
            // with plans each pass takes its pairs from the plan; without, all ncl pairs
            const int np = P.planned ? -1 : (int)p.ncl;
            const unsigned grid = (unsigned)(2 * p.ncl);
            auto passes = [&]() -> accel_status {
                for (int l = 0; l <= L.Cmax; ++l) {
                    if (l >= 1) {
                        // the backward of round l - 1: after its recomputation; its Q / gamma /
                        // symbol buffers were last read by the counts of round l - 1 - kQBufs
                        const int rb = l - 1;
                        ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.hi, e_rec[rb], 0));
                        if (rb >= kQBufs) ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.hi, done[rb - kQBufs], 0));
                        kc.bwd<<<grid, clu::kT, P.sm_c, bs.hi>>>(p, rb, np);
                        ++nlaunch;
                        ACCEL_CUDA_TRY(ev.make(e_bwd[rb]));
                        ACCEL_CUDA_TRY(cudaEventRecord(e_bwd[rb], bs.hi));
                        accel_status r = counts(rb);
                        if (r != ACCEL_OK) return r;
                    }
                    if (l < L.Cmax) {
                        // the recomputation of round l: its P rows' buffer was last read by the
                        // backward and the counts of round l - kPBufs, its exponents' by the
                        // backward of round l - 2
                        if (l >= kPBufs) ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.hi2, done[l - kPBufs], 0));
                        if (l >= 2) ACCEL_CUDA_TRY(cudaStreamWaitEvent(bs.hi2, e_bwd[l - 2], 0));
                        kc.rec<<<grid, clu::kT, P.sm_c, bs.hi2>>>(p, l, np);
                        ++nlaunch;
                        ACCEL_CUDA_TRY(ev.make(e_rec[l]));
                        ACCEL_CUDA_TRY(cudaEventRecord(e_rec[l], bs.hi2));
                    }
                }
                return ACCEL_OK;
            };
            const accel_status rp = passes();
            // the caller's stream waits for all three streams, also after an error on the way,
            // so that nothing enqueued so far outlives the call's ordering
            cudaEvent_t e_join[3];
            cudaStream_t own[3] = {bs.hi, bs.hi2, bs.lo};
            for (int k = 0; k < 3; ++k) {
                ACCEL_CUDA_TRY(ev.make(e_join[k]));
                ACCEL_CUDA_TRY(cudaEventRecord(e_join[k], own[k]));
                ACCEL_CUDA_TRY(cudaStreamWaitEvent(st, e_join[k], 0));
            }
            if (rp != ACCEL_OK) return rp;
        } else {
            ACCEL_CUDA_TRY(cudaFuncSetAttribute(k_backward_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.sm_b));
            for (int round = 0; round < L.Cmax; ++round) {
                k_backward_round<<<(unsigned)L.ngroups, kT, P.sm_b, st>>>(p, round);
                k_gemm_ptq<<<P.nb * P.nb * kSplit, 256, 0, st>>>(p.P, p.Q, p.rows + round, K, P.Upart);
                nlaunch += 2;
            }
        }
    }
    int pg = num_sms() * 4;
    k_finish<<<pg, 256, 0, st>>>(p.A, p.Kp, P.Upart, p.cnt, P.cntp, p.pig, K, M, L.ngroups,
                                 P.use_cluster ? p.ncl : L.ngroups, P.nsU, P.nsC, d_grad_log_A, d_grad_log_B,
                                 d_grad_log_pi);
    ++nlaunch;
    return ACCEL_OK;
}

static accel_status debug_checks(const Plan& P, const int64_t* d_offsets, const int32_t* d_obs, int64_t total_T,
                                 cudaStream_t st) {
    if (!debug_mode() || P.p.S == 0) return ACCEL_OK;
    accel_status r = debug_check_offsets(d_offsets, P.p.S, total_T, 1, P.ws + kDebugScratchOff, st);
    if (r != ACCEL_OK) return r;
    return debug_check_symbols(d_obs, total_T, P.M, P.ws + kDebugScratchOff, st);
}

static accel_status finish_call(const char* who, const Plan& P, int64_t max_T, cudaStream_t st, int nlaunch) {
    accel_status r = after_launch(st, who, nlaunch);
    if (r != ACCEL_OK) return r;
    if (debug_mode()) {
        int32_t h = 0;
        ACCEL_CUDA_TRY(cudaMemcpyAsync(&h, P.p.status, 4, cudaMemcpyDeviceToHost, st));
        ACCEL_CUDA_TRY(cudaStreamSynchronize(st));
        if (h == ACCEL_ERR_SHAPE) return set_error(h, "%s: a sequence is longer than max_T=%lld", who, (long long)max_T);
        if (h != ACCEL_OK) return set_error(h, "%s: device status %d (a bounded wait gave up)", who, h);
    }
    return ok();
}

}  // namespace adj
}  // namespace hmm
}  // namespace accel

extern "C" {

accel_status hmm_adjoint(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets, int64_t S,
                         int64_t total_T, int64_t max_T, const double* d_weights, double* d_loglik,
                         float* d_grad_log_A, float* d_grad_log_B, float* d_grad_log_pi, void* d_ws, size_t ws_bytes,
                         void* stream) {
    adj::Plan P;
    accel_status r = adj::setup("hmm_adjoint", m, d_obs, d_offsets, S, total_T, max_T, d_ws, ws_bytes, P);
    if (r != ACCEL_OK) return r;
    ACCEL_REQUIRE(d_grad_log_A && d_grad_log_B, ACCEL_ERR_INVALID_ARG, "hmm_adjoint: null pointer");
    cudaStream_t st = as_stream(stream);
    r = adj::debug_checks(P, d_offsets, d_obs, total_T, st);
    if (r != ACCEL_OK) return r;
    ACCEL_CUDA_TRY(cudaMemsetAsync(P.ws + kStatusOff, 0, 4, st));
    int nlaunch = 0;
    r = adj::run_forward(P, m, d_loglik, st, nlaunch);
    if (r != ACCEL_OK) return r;
    r = adj::run_backward(P, d_weights, d_grad_log_A, d_grad_log_B, d_grad_log_pi, st, nlaunch);
    if (r != ACCEL_OK) return r;
    return adj::finish_call("hmm_adjoint", P, max_T, st, nlaunch);
}

accel_status hmm_adjoint_forward(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets, int64_t S,
                                 int64_t total_T, int64_t max_T, double* d_loglik, void* d_ws, size_t ws_bytes,
                                 void* stream) {
    adj::Plan P;
    accel_status r = adj::setup("hmm_adjoint_forward", m, d_obs, d_offsets, S, total_T, max_T, d_ws, ws_bytes, P);
    if (r != ACCEL_OK) return r;
    cudaStream_t st = as_stream(stream);
    r = adj::debug_checks(P, d_offsets, d_obs, total_T, st);
    if (r != ACCEL_OK) return r;
    ACCEL_CUDA_TRY(cudaMemsetAsync(P.ws + kStatusOff, 0, 4, st));
    int nlaunch = 0;
    r = adj::run_forward(P, m, d_loglik, st, nlaunch);
    if (r != ACCEL_OK) return r;
    return adj::finish_call("hmm_adjoint_forward", P, max_T, st, nlaunch);
}

accel_status hmm_adjoint_backward(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets, int64_t S,
                                  int64_t total_T, int64_t max_T, const double* d_weights, float* d_grad_log_A,
                                  float* d_grad_log_B, float* d_grad_log_pi, void* d_ws, size_t ws_bytes,
                                  void* stream) {
    adj::Plan P;
    accel_status r = adj::setup("hmm_adjoint_backward", m, d_obs, d_offsets, S, total_T, max_T, d_ws, ws_bytes, P);
    if (r != ACCEL_OK) return r;
    ACCEL_REQUIRE(d_grad_log_A && d_grad_log_B, ACCEL_ERR_INVALID_ARG, "hmm_adjoint_backward: null pointer");
    cudaStream_t st = as_stream(stream);
    ACCEL_CUDA_TRY(cudaMemsetAsync(P.ws + kStatusOff, 0, 4, st));
    int nlaunch = 0;
    r = adj::run_backward(P, d_weights, d_grad_log_A, d_grad_log_B, d_grad_log_pi, st, nlaunch);
    if (r != ACCEL_OK) return r;
    return adj::finish_call("hmm_adjoint_backward", P, max_T, st, nlaunch);
}

}  // extern "C"
