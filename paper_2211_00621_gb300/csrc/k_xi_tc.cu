// Tensor-core accumulation of the adjoint's two contractions over the row buffers of one
// backward round (the expected transition and emission counts):
//
//   U[i][j]      += sum_rows P[row][i] Q[row][j]                     (xi = A o U at the end)
//   counts[i][k] += sum_rows Gamma[row][i] [osym[row] == k]           (a product with a one-hot
//                                                                      matrix, exact in TF32)
//
// Both are dense products with a long reduction (the rows) and a small K x K (K x M) result,
// so each CTA takes a 128-row block of i and a contiguous range of rows, accumulates the
// whole result block in tensor memory with tcgen05.mma kind::tf32 (M = 128, N = K and N = Mp,
// 8 rows of the reduction per instruction), and adds it once into its own partial buffer
// (deterministic: fixed row ranges, fixed order; the partials are summed by the finishing
// kernel).
//
// FP32 accuracy from TF32 tensor cores: every operand x is split as x = hi + lo with
// hi = tf32(x) and lo = tf32(x - hi) (round to nearest), and a b is accumulated as
// hi_a hi_b + hi_a lo_b + lo_a hi_b; the dropped lo_a lo_b term is below 2^-21 relative.
// The one-hot operand needs no split.
//
// Operands are staged by all 256 threads (coalesced global loads, split, 16-byte shared
// stores into the no-swizzle K-major canonical layout: core matrices of 8 rows x 4 values),
// up to three stages deep; the loads of the next two chunks are in flight (in registers)
// while the current chunk is split and stored.  One thread issues the MMAs of a stage and commits them
// to the stage's mbarrier, which the threads wait on (bounded) before they refill it.
#include "hmm_internal.cuh"
#include "tc_ptx.cuh"

namespace accel {
namespace hmm {

namespace {

constexpr int kThreads = 256;
constexpr int kKC = 16;                 // reduction rows per stage
constexpr int kMaxStages = 3;
constexpr uint64_t kWaitNs = 2000000000ull;

// Instruction descriptor, kind::tf32: TF32 A and B (K-major), FP32 accumulator, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
    return (1u << 4)                      // D format: F32
         | (2u << 7)                      // A format: TF32
         | (2u << 10)                     // B format: TF32
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

struct XiPrm {
    const float* P;
    const float* Q;
    const float* G;
    const int32_t* osym;
    const int32_t* rows_r;
    int K, M, Mp, nib, nsplit, stages;
    uint32_t tmem_cols;
    float* Upart;                         // [nsplit][K][K]
    float* cntp;                          // [nsplit][K][M] (null: counts not taken here)
    int32_t* status;
};

// Byte offsets of one stage's operand blocks (each [rows][kKC] in the canonical layout).
struct StageLayout {
    uint32_t a_hi, a_lo, b_hi, b_lo, g_hi, g_lo, h, bytes;
};
__host__ __device__ inline StageLayout stage_layout(int K, int Mp, bool counts) {
    StageLayout s;
    uint32_t o = 0;
    const uint32_t blk128 = 128u * kKC * 4, blkK = (uint32_t)K * kKC * 4, blkM = (uint32_t)Mp * kKC * 4;
    s.a_hi = o; o += blk128;
    s.a_lo = o; o += blk128;
    s.b_hi = o; o += blkK;
    s.b_lo = o; o += blkK;
    s.g_hi = o; o += counts ? blk128 : 0;
    s.g_lo = o; o += counts ? blk128 : 0;
    s.h = o;    o += counts ? blkM : 0;
    s.bytes = o;
    return s;
}

// Canonical K-major offset of element (n, k) of a [rows][kKC] block: core matrix (n/8, k/4)
// at (n/8) * SBO + (k/4) * LBO, with LBO = 128 and SBO = (kKC/4) * 128 bytes.
__device__ __forceinline__ uint32_t canon(int n, int kq) {
    return (uint32_t)(n >> 3) * (kKC / 4 * 128) + (uint32_t)kq * 128 + (uint32_t)(n & 7) * 16;
}

// Stores hi / lo of 4 reduction rows (k = 4kq .. 4kq+3) of column n.
__device__ __forceinline__ void put_split(char* hi, char* lo, int n, int kq, float4 v) {
    float4 h, l;
    h.x = tf32_rn(v.x); l.x = tf32_rn(v.x - h.x);
    h.y = tf32_rn(v.y); l.y = tf32_rn(v.y - h.y);
    h.z = tf32_rn(v.z); l.z = tf32_rn(v.z - h.z);
    h.w = tf32_rn(v.w); l.w = tf32_rn(v.w - h.w);
    const uint32_t off = canon(n, kq);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
}

// Column `col` of rows row0 + 4kq .. +3 of a [rows][K] buffer, zero past r1 or past K.
__device__ __forceinline__ float4 load4(const float* __restrict__ X, int K, int64_t row0, int kq, int64_t r1,
                                        int col) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col < K) {
        const int64_t r = row0 + 4 * kq;
        if (r + 0 < r1) v.x = X[(r + 0) * K + col];
        if (r + 1 < r1) v.y = X[(r + 1) * K + col];
        if (r + 2 < r1) v.z = X[(r + 2) * K + col];
        if (r + 3 < r1) v.w = X[(r + 3) * K + col];
    }
    return v;
}

// The operand values one thread stages per chunk: the index e of each group is the thread's
// e-th slot idx = tid + e * 256 of the block's (column, row quad) pairs.
template <int K, bool CNT>
struct Frag {
    static constexpr int NA = 128 * (kKC / 4) / kThreads;        // P^T and Gamma^T groups
    static constexpr int NB = K * (kKC / 4) / kThreads;          // Q^T groups
    float4 a[NA], g[CNT ? NA : 1], b[NB];
    int4 o;                                                      // osym of the thread's H row quad
};

template <int K, bool CNT>
__device__ __forceinline__ void frag_load(Frag<K, CNT>& f, const XiPrm& p, int64_t row0, int64_t r1, int icol0,
                                          bool valid) {
    using F = Frag<K, CNT>;
    const int tid = threadIdx.x;
#pragma unroll
    for (int e = 0; e < F::NA; ++e) {
        const int idx = tid + e * kThreads, n = idx % 128, kq = idx / 128;
        f.a[e] = valid ? load4(p.P, K, row0, kq, r1, icol0 + n) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (CNT) f.g[e] = valid ? load4(p.G, K, row0, kq, r1, icol0 + n) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < F::NB; ++e) {
        const int idx = tid + e * kThreads, n = idx % K, kq = idx / K;
        f.b[e] = valid ? load4(p.Q, K, row0, kq, r1, n) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (CNT) {
        // H: thread tid takes row quad tid % 4 for the columns tid / 4 + 64 m (see frag_store)
        const int kq = tid & 3;
        const int64_t r = row0 + 4 * kq;
        f.o.x = (valid && r + 0 < r1) ? p.osym[r + 0] : -1;
        f.o.y = (valid && r + 1 < r1) ? p.osym[r + 1] : -1;
        f.o.z = (valid && r + 2 < r1) ? p.osym[r + 2] : -1;
        f.o.w = (valid && r + 3 < r1) ? p.osym[r + 3] : -1;
    }
}

template <int K, bool CNT>
__device__ __forceinline__ void frag_store(const Frag<K, CNT>& f, char* st, const StageLayout& sl, int icol0, int Mp) {
    using F = Frag<K, CNT>;
    const int tid = threadIdx.x;
#pragma unroll
    for (int e = 0; e < F::NA; ++e) {
        const int idx = tid + e * kThreads, n = idx % 128, kq = idx / 128;
        if (icol0 + n >= K) continue;
        put_split(st + sl.a_hi, st + sl.a_lo, n, kq, f.a[e]);
        if (CNT) put_split(st + sl.g_hi, st + sl.g_lo, n, kq, f.g[e]);
    }
#pragma unroll
    for (int e = 0; e < F::NB; ++e) {
        const int idx = tid + e * kThreads, n = idx % K, kq = idx / K;
        put_split(st + sl.b_hi, st + sl.b_lo, n, kq, f.b[e]);
    }
    if (CNT) {
        // quad kq = tid % 4, columns n = tid / 4 + 64 m (m < Mp / 64)
        const int kq = tid & 3;
        for (int n = tid >> 2; n < Mp; n += kThreads / 4) {
            float4 v;
            v.x = f.o.x == n ? 1.f : 0.f;
            v.y = f.o.y == n ? 1.f : 0.f;
            v.z = f.o.z == n ? 1.f : 0.f;
            v.w = f.o.w == n ? 1.f : 0.f;
            *reinterpret_cast<float4*>(st + sl.h + canon(n, kq)) = v;
        }
    }
}

template <int K, bool CNT>
__global__ void __launch_bounds__(kThreads, 1) k_xi_tc(XiPrm p) {
    extern __shared__ __align__(1024) char smem[];
    __shared__ __align__(8) uint64_t s_bar[kMaxStages];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ib = blockIdx.x % p.nib, sp = blockIdx.x / p.nib;
    const int64_t rows = *p.rows_r;
    const int64_t r0 = rows * sp / p.nsplit, r1 = rows * (sp + 1) / p.nsplit;
    if (r0 >= r1) return;                 // uniform over the CTA; nothing allocated yet
    const int Mp = p.Mp, NS = p.stages;
    const StageLayout sl = stage_layout(K, Mp, CNT);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) tc::mbar_init(&s_bar[s], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, p.tmem_cols);
        tc::tmem_relinquish();
    }
    // rows of the i block past K stay zero in every stage
    if (K - ib * 128 < 128) {
        for (int s = 0; s < NS; ++s)
            for (int idx = tid; idx < 128 * kKC / 4; idx += kThreads) {
                const int n = idx % 128, kq = idx / 128;
                if (ib * 128 + n < K) continue;
                char* st = smem + (size_t)s * sl.bytes;
                const uint32_t off = canon(n, kq);
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4*>(st + sl.a_hi + off) = z;
                *reinterpret_cast<float4*>(st + sl.a_lo + off) = z;
                if (CNT) {
                    *reinterpret_cast<float4*>(st + sl.g_hi + off) = z;
                    *reinterpret_cast<float4*>(st + sl.g_lo + off) = z;
                }
            }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idU = idesc_tf32_f32(128, K), idC = idesc_tf32_f32(128, CNT ? Mp : 16);
    const int64_t nchunks = (r1 - r0 + kKC - 1) / kKC;
    const int icol0 = ib * 128;
    bool failed = false;
    // register ring of three chunks: chunk c is split and stored while the loads of chunks
    // c+1 and c+2 are in flight
    Frag<K, CNT> f0, f1, f2;
    frag_load<K, CNT>(f0, p, r0, r1, icol0, true);
    frag_load<K, CNT>(f1, p, r0 + kKC, r1, icol0, 1 < nchunks);
    auto chunk = [&](int64_t c, const Frag<K, CNT>& cur, Frag<K, CNT>& ahead) -> bool {
        const int s = (int)(c % NS);
        char* st = smem + (size_t)s * sl.bytes;
        frag_load<K, CNT>(ahead, p, r0 + (c + 2) * kKC, r1, icol0, c + 2 < nchunks);
        if (c >= NS) {
            const uint32_t par = (uint32_t)((c / NS - 1) & 1);
            const bool ok = tc::mbar_wait_bounded(&s_bar[s], par, kWaitNs);
            if (__syncthreads_or(!ok)) return false;
        }
        frag_store<K, CNT>(cur, st, sl, icol0, Mp);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t base = tc::smem_u32(st);
            const uint32_t sbo = kKC / 4 * 128;
#pragma unroll
            for (int ks = 0; ks < kKC / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 256;   // 8 reduction rows = two core matrices
                const uint64_t ah = tc::smem_desc_noswizzle(base + sl.a_hi + koff, 128, sbo);
                const uint64_t al = tc::smem_desc_noswizzle(base + sl.a_lo + koff, 128, sbo);
                const uint64_t bh = tc::smem_desc_noswizzle(base + sl.b_hi + koff, 128, sbo);
                const uint64_t bl = tc::smem_desc_noswizzle(base + sl.b_lo + koff, 128, sbo);
                const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                mma_tf32(tmem, ah, bh, idU, acc0);
                mma_tf32(tmem, ah, bl, idU, 1u);
                mma_tf32(tmem, al, bh, idU, 1u);
                if (CNT) {
                    const uint64_t gh = tc::smem_desc_noswizzle(base + sl.g_hi + koff, 128, sbo);
                    const uint64_t gl = tc::smem_desc_noswizzle(base + sl.g_lo + koff, 128, sbo);
                    const uint64_t hh = tc::smem_desc_noswizzle(base + sl.h + koff, 128, sbo);
                    mma_tf32(tmem + (uint32_t)K, gh, hh, idC, acc0);
                    mma_tf32(tmem + (uint32_t)K, gl, hh, idC, 1u);
                }
            }
            tc::mma_commit(&s_bar[s]);
        }
        return true;
    };
    for (int64_t c = 0; c < nchunks; c += 3) {
        if (!chunk(c, f0, f2)) { failed = true; break; }
        if (c + 1 >= nchunks) break;
        if (!chunk(c + 1, f1, f0)) { failed = true; break; }
        if (c + 2 >= nchunks) break;
        if (!chunk(c + 2, f2, f1)) { failed = true; break; }
    }
    if (!failed) {
        // the last commit covers every MMA issued before it
        const int64_t cl = nchunks - 1;
        const bool ok = tc::mbar_wait_bounded(&s_bar[cl % NS], (uint32_t)((cl / NS) & 1), kWaitNs);
        failed = __syncthreads_or(!ok);
    }
    if (failed) {
        if (tid == 0) report_status(p.status, ACCEL_ERR_TIMEOUT);
    } else {
        tc::tc_fence_after();
        // warp w reads TMEM lanes 32 (w % 4) .. +31 (rows i of the block), column half w / 4
        const int q = warp & 3, half = warp >> 2;
        const int i = icol0 + 32 * q + (tid & 31);
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        float* U = p.Upart + (int64_t)sp * K * K;
#pragma unroll 1
        for (int j0 = half * (K / 2); j0 < (half + 1) * (K / 2); j0 += 32) {
            uint32_t v[32];
            tc::tmem_ld32(lane_base + (uint32_t)j0, v);
            if (i < K) {
                float* dst = U + (int64_t)i * K + j0;
#pragma unroll
                for (int e = 0; e < 32; e += 4) {
                    float4 d = *reinterpret_cast<float4*>(dst + e);
                    d.x += __uint_as_float(v[e]);
                    d.y += __uint_as_float(v[e + 1]);
                    d.z += __uint_as_float(v[e + 2]);
                    d.w += __uint_as_float(v[e + 3]);
                    *reinterpret_cast<float4*>(dst + e) = d;
                }
            }
        }
        if (CNT) {
            float* Cn = p.cntp + (int64_t)sp * K * p.M;
#pragma unroll 1
            for (int k0 = half * (Mp / 2); k0 < (half + 1) * (Mp / 2); k0 += 32) {
                uint32_t v[32];
                tc::tmem_ld32(lane_base + (uint32_t)(K + k0), v);
                if (i < K)
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        if (k0 + e < p.M) Cn[(int64_t)i * p.M + k0 + e] += __uint_as_float(v[e]);
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, p.tmem_cols);
}

int xi_counts_cols(int M) { return (M + 63) / 64 * 64; }

}  // namespace

bool xi_tc_supported(int K) { return K == 64 || K == 128 || K == 256; }
bool xi_tc_counts_supported(int K, int M) { return xi_tc_supported(K) && K + xi_counts_cols(M) <= 512 && xi_counts_cols(M) <= 256; }

int xi_tc_splits(int K) {
    const int nib = (K + 127) / 128;
    int n = num_sms() / nib;
    return n < 1 ? 1 : (n > kXiSplitMax ? kXiSplitMax : n);
}

accel_status xi_tc_round(const float* P, const float* Q, const float* G, const int32_t* osym, const int32_t* rows_r,
                         int K, int M, float* Upart, float* cntp, int32_t* status, cudaStream_t st) {
    const bool counts = cntp != nullptr;
    XiPrm p;
    p.P = P; p.Q = Q; p.G = G; p.osym = osym; p.rows_r = rows_r;
    p.K = K; p.M = M; p.Mp = counts ? xi_counts_cols(M) : 0;
    p.nib = (K + 127) / 128;
    p.nsplit = xi_tc_splits(K);
    p.Upart = Upart; p.cntp = cntp; p.status = status;
    const int need_cols = K + p.Mp;
    uint32_t cols = 32;
    while ((int)cols < need_cols) cols <<= 1;
    p.tmem_cols = cols;
    const StageLayout sl = stage_layout(K, p.Mp, counts);
    const int optin = max_smem_optin();
    int stages = kMaxStages;
    while (stages > 2 && (size_t)stages * sl.bytes + 1024 > (size_t)optin) --stages;
    ACCEL_REQUIRE((size_t)stages * sl.bytes + 1024 <= (size_t)optin, ACCEL_ERR_UNSUPPORTED,
                  "hmm_adjoint: count/transition stages do not fit in shared memory (K=%d, M=%d)", K, M);
    p.stages = stages;
    const size_t smem = (size_t)stages * sl.bytes + 1024;   // + alignment slack of the dynamic block
    void (*kern)(XiPrm) = nullptr;
    switch (K) {
        case 64: kern = counts ? k_xi_tc<64, true> : k_xi_tc<64, false>; break;
        case 128: kern = counts ? k_xi_tc<128, true> : k_xi_tc<128, false>; break;
        default: kern = counts ? k_xi_tc<256, true> : k_xi_tc<256, false>; break;
    }
    ACCEL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)(p.nib * p.nsplit), kThreads, smem, st>>>(p);
    return ACCEL_OK;
}

}  // namespace hmm
}  // namespace accel
