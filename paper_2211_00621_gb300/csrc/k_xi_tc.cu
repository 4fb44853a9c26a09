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
// Operand path of a chunk of kKC = 16 reduction rows: 512 splitter threads load the chunk's
// rows of Q (all K columns) and of P and Gamma (the CTA's 128 columns) straight from global
// memory, four rows of one column per piece (warp loads of 32 consecutive columns), and write
// their hi / lo parts into the operand blocks of a split stage (the no-swizzle K-major
// canonical layout: core matrices of 8 rows x 4 values) together with the one-hot block.  The
// stage's mbarrier counts the 512 splitters; one thread of a seventeenth warp then issues the
// chunk's MMAs and commits them to the stage's second mbarrier, which the splitters wait on
// (bounded) before they refill that stage.  The rows are the round's packed rows, read once
// per CTA; thread 0 keeps the rows of the next kPrefetch chunks on their way into L2, so the
// splitters' loads wait on L2, not on DRAM.
#include "hmm_internal.cuh"
#include "tc_ptx.cuh"

#include <cooperative_groups.h>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

namespace accel {
namespace hmm {

namespace {

constexpr int kSplitThreads = 512;      // warps 0-15: loads, operand split, epilogue
constexpr int kThreads = kSplitThreads + 32;   // + warp 16: issues the MMAs
constexpr int kColParts = kSplitThreads / 128; // epilogue: column parts per TMEM lane quarter
constexpr int kCluster = 4;            // CTAs of consecutive row ranges of one i block
constexpr int kKC = 16;                 // reduction rows per stage
constexpr int kMaxStages = 3;          // split stages
constexpr int kPrefetch = 6;           // chunks brought into L2 ahead
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
    int two_phase;                        // epilogue: U and the counts staged one after the other
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

template <int K, bool CNT>
__global__ void __launch_bounds__(kThreads, 1) k_xi_tc(XiPrm p) {
    extern __shared__ __align__(1024) char smem[];
    __shared__ __align__(8) uint64_t s_bar[kMaxStages];     // split stage s: its MMAs done
    __shared__ __align__(8) uint64_t s_full[kMaxStages];    // split stage s: operands written
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ int64_t s_committed;       // chunks whose MMAs the MMA warp committed
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool splitter = tid < kSplitThreads;
    // cluster cid = (i block ib, split group sg); its rank crank takes split sp of the rows
    const int cid = (int)blockIdx.x / kCluster, crank = (int)blockIdx.x % kCluster;
    const int ib = cid % p.nib, sg = cid / p.nib, sp = sg * kCluster + crank;
    const int64_t rows = *p.rows_r;
    if (rows == 0) return;                // uniform over the grid; nothing allocated yet
    const int64_t r0 = rows * sp / p.nsplit, r1 = rows * (sp + 1) / p.nsplit;
    const bool has_rows = r0 < r1;        // a rank without rows still joins the cluster's sums
    const int Mp = p.Mp, NS = p.stages;
    const StageLayout sl = stage_layout(K, Mp, CNT);
    const int icol0 = ib * 128;
    const int ncols = K - icol0 < 128 ? K - icol0 : 128;     // valid i columns of the block
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&s_bar[s], 1);
            tc::mbar_init(&s_full[s], kSplitThreads);
        }
        tc::fence_mbar_init();
        s_fail = 0;
        s_committed = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, p.tmem_cols);
        tc::tmem_relinquish();
    }
    // rows of the i block past K stay zero in every stage
    if (ncols < 128 && splitter) {
        for (int s = 0; s < NS; ++s)
            for (int idx = tid; idx < 128 * kKC / 4; idx += kSplitThreads) {
                const int n = idx % 128, kq = idx / 128;
                if (n < ncols) continue;
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
    const int64_t nchunks = has_rows ? (r1 - r0 + kKC - 1) / kKC : 0;
    bool failed = false;
    int64_t c = 0;
    if (!splitter) {
        // ---- the last warp: lane 0 issues each chunk's MMAs once its operands are written
        if (lane == 0) {
            const uint32_t idU = idesc_tf32_f32(128, K), idC = idesc_tf32_f32(128, CNT ? Mp : 16);
            const uint32_t sbo = kKC / 4 * 128;
            for (int64_t q = 0; q < nchunks; ++q) {
                const int s = (int)(q % NS);
                if (!tc::mbar_wait_bounded(&s_full[s], (uint32_t)((q / NS) & 1), kWaitNs)) {
                    s_fail = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t base = tc::smem_u32(smem + (size_t)s * sl.bytes);
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint32_t koff = (uint32_t)ks * 256;   // 8 reduction rows = two core matrices
                    const uint64_t ah = tc::smem_desc_noswizzle(base + sl.a_hi + koff, 128, sbo);
                    const uint64_t al = tc::smem_desc_noswizzle(base + sl.a_lo + koff, 128, sbo);
                    const uint64_t bh = tc::smem_desc_noswizzle(base + sl.b_hi + koff, 128, sbo);
                    const uint64_t bl = tc::smem_desc_noswizzle(base + sl.b_lo + koff, 128, sbo);
                    const uint32_t acc0 = (q > 0 || ks > 0) ? 1u : 0u;
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
                s_committed = q + 1;
            }
        }
        __syncwarp();
    } else {
        // ---- the other warps: the operand split, straight from global memory.  Each splitter
        // loads its pieces of chunk c (four rows of one column per piece; the rows are on
        // their way into L2, thread 0 bringing them kPrefetch chunks ahead) and writes their
        // hi / lo parts into the chunk's stage; the stage's mbarrier counts the 512 splitters
        // before the MMA warp issues, and a splitter refills a stage once its MMAs completed.
        constexpr int QI = (K * 4 + kSplitThreads - 1) / kSplitThreads;   // Q pieces per splitter
        const int pn = tid % 128, pkq = tid / 128;    // the P / Gamma piece: column pn, rows 4 pkq ..
        const bool pin = pn < ncols;
        auto load4 = [&](const float* base, int n, int kq, int64_t row0, int nrow) -> float4 {
            const int r = 4 * kq;
            const float* src = base + (row0 + r) * K + n;
            float4 v;
            v.x = r + 0 < nrow ? __ldcg(src) : 0.f;
            v.y = r + 1 < nrow ? __ldcg(src + K) : 0.f;
            v.z = r + 2 < nrow ? __ldcg(src + 2 * K) : 0.f;
            v.w = r + 3 < nrow ? __ldcg(src + 3 * K) : 0.f;
            return v;
        };
        auto prefetch = [&](int64_t q) {
            const int64_t prow0 = r0 + q * kKC;
            const uint32_t bytes = (uint32_t)(r1 - prow0 < kKC ? r1 - prow0 : kKC) * K * 4;
            tc::bulk_prefetch_l2(p.Q + prow0 * K, bytes);
            tc::bulk_prefetch_l2(p.P + prow0 * K, bytes);
            if (CNT) tc::bulk_prefetch_l2(p.G + prow0 * K, bytes);
        };
        // this splitter's pieces of chunk q (all loads issued before the first use)
        struct Pieces {
            float4 p, g, q[QI];
            int4 o;                       // osym of the thread's H row quad tid % 4
        };
        auto load = [&](Pieces& v, int64_t q) {
            const int64_t row0 = r0 + q * kKC;
            const int nrow = (int)(r1 - row0 < kKC ? r1 - row0 : kKC);
            v.p = pin ? load4(p.P + icol0, pn, pkq, row0, nrow) : make_float4(0.f, 0.f, 0.f, 0.f);
            v.g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (CNT && pin) v.g = load4(p.G + icol0, pn, pkq, row0, nrow);
#pragma unroll
            for (int i = 0; i < QI; ++i) {
                const int idx = tid + i * kSplitThreads;
                v.q[i] = idx < K * 4 ? load4(p.Q, idx % K, idx / K, row0, nrow) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            v.o = make_int4(-1, -1, -1, -1);
            if (CNT) {
                const int64_t r = row0 + 4 * (tid & 3);
                if (r + 0 < r1) v.o.x = p.osym[r + 0];
                if (r + 1 < r1) v.o.y = p.osym[r + 1];
                if (r + 2 < r1) v.o.z = p.osym[r + 2];
                if (r + 3 < r1) v.o.w = p.osym[r + 3];
            }
        };
        if (tid == 0)
            for (int64_t q = 0; q < kPrefetch && q < nchunks; ++q) prefetch(q);
        // the pieces of chunk c + 1 load while chunk c is split
        Pieces cur, nxt;
        if (nchunks > 0) load(cur, 0);
        for (; c < nchunks; ++c) {
            const int s = (int)(c % NS);
            char* st = smem + (size_t)s * sl.bytes;
            if (tid == 0 && c + kPrefetch < nchunks) prefetch(c + kPrefetch);
            if (c + 1 < nchunks) load(nxt, c + 1);
            const float4 vp = cur.p, vg = cur.g;
            const int4 o = cur.o;
            // the stage's previous MMAs (chunk c - NS) have completed
            if (c >= NS) {
                const bool ok = *reinterpret_cast<volatile int*>(&s_fail) == 0 &&
                                tc::mbar_wait_bounded(&s_bar[s], (uint32_t)((c / NS - 1) & 1), kWaitNs);
                if (!ok) {
                    failed = true;
                    break;
                }
            }
            if (pin) {
                put_split(st + sl.a_hi, st + sl.a_lo, pn, pkq, vp);
                if (CNT) put_split(st + sl.g_hi, st + sl.g_lo, pn, pkq, vg);
            }
#pragma unroll
            for (int i = 0; i < QI; ++i) {
                const int idx = tid + i * kSplitThreads;
                if (idx < K * 4) put_split(st + sl.b_hi, st + sl.b_lo, idx % K, idx / K, cur.q[i]);
            }
            if (CNT) {
                // quad kq = tid % 4, columns n = tid / 4 + 128 m (m < Mp / 128)
                const int kq = tid & 3;
                for (int n = tid >> 2; n < Mp; n += kSplitThreads / 4) {
                    float4 v;
                    v.x = o.x == n ? 1.f : 0.f;
                    v.y = o.y == n ? 1.f : 0.f;
                    v.z = o.z == n ? 1.f : 0.f;
                    v.w = o.w == n ? 1.f : 0.f;
                    *reinterpret_cast<float4*>(st + sl.h + canon(n, kq)) = v;
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&s_full[s]);                       // the MMA warp may issue chunk c
            cur = nxt;
        }
        if (failed) s_fail = 1;
    }
    __syncthreads();                      // the MMA warp is done issuing
    failed = s_fail != 0;
    if (!failed && tid == 0 && nchunks > 0) {
        // the last commit covers every MMA issued before it
        const int64_t cl = nchunks - 1;
        if (!tc::mbar_wait_bounded(&s_bar[cl % NS], (uint32_t)((cl / NS) & 1), kWaitNs)) s_fail = 1;
    }
    if (failed && tid == 0) {
        // a wait gave up: let the MMAs already committed finish (bounded) before the tensor
        // memory and the CTA go away
        const int64_t nc = s_committed;
        if (nc > 0) tc::mbar_wait_bounded(&s_bar[(nc - 1) % NS], (uint32_t)(((nc - 1) / NS) & 1), kWaitNs);
    }
    __syncthreads();
    failed = s_fail != 0;
    if (failed && tid == 0) report_status(p.status, ACCEL_ERR_TIMEOUT);
    // ---- epilogue.  Each CTA stages its accumulators in its own (now idle) shared memory --
    // zeros for a rank without rows or after a failed wait, so that every rank still takes
    // both cluster barriers -- then rank r adds the cluster's kCluster blocks for rows
    // [32 r, 32 r + 32) of the i block through distributed shared memory, in rank order, and
    // adds the sums into the cluster's partial: one read-modify-write of the partials per
    // cluster instead of one per CTA.
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int ULD = K + 4;            // staging row strides (floats): 16-byte stores, 4 wavefronts
    const int CLD = Mp + 4;
    float* stU = reinterpret_cast<float*>(smem);
    // U and the counts are staged together when both fit, else one after the other in the
    // same area (two rounds of the two barriers)
    const bool two_phase = CNT && p.two_phase;
    float* stC = two_phase ? stU : stU + 128 * ULD;
    const bool live = !failed && has_rows;
    for (int ph = 0; ph < (two_phase ? 2 : 1); ++ph) {
        const bool do_u = !two_phase || ph == 0, do_c = CNT && (!two_phase || ph == 1);
        if (splitter) {
            const int q = warp & 3, part = warp >> 2;
            const int row = 32 * q + lane;
            const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
            if (live) tc::tc_fence_after();
#pragma unroll 1
            for (int j0 = 32 * part; do_u && j0 < K; j0 += 32 * kColParts) {
                uint32_t v[32];
                if (live) {
                    tc::tmem_ld32(lane_base + (uint32_t)j0, v);
                } else {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = 0u;
                }
                float4* dst = reinterpret_cast<float4*>(stU + row * ULD + j0);
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    dst[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                         __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
            }
            if (do_c) {
#pragma unroll 1
                for (int k0 = 32 * part; k0 < Mp; k0 += 32 * kColParts) {
                    uint32_t v[32];
                    if (live) {
                        tc::tmem_ld32(lane_base + (uint32_t)(K + k0), v);
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e) v[e] = 0u;
                    }
                    float4* dst = reinterpret_cast<float4*>(stC + row * CLD + k0);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        dst[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                             __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
                }
            }
        }
        cluster.sync();                       // every rank's block staged
        if (splitter) {
            const int rb = 32 * crank;        // this rank's rows of the block
            constexpr int NQ = K / 4;         // float4 per row
            constexpr int UIT = (32 * NQ + kSplitThreads - 1) / kSplitThreads;
            float* U = p.Upart + (int64_t)sg * K * K;
            if (do_u) {
            float4 acc[UIT], cur[UIT];
#pragma unroll
            for (int it = 0; it < UIT; ++it) {
                const int idx = tid + it * kSplitThreads, rr = idx / NQ, c4 = idx % NQ;
                acc[it] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (idx < 32 * NQ && icol0 + rb + rr < K) {
#pragma unroll
                    for (int c = 0; c < kCluster; ++c) {
                        const float4 b = reinterpret_cast<const float4*>(cluster.map_shared_rank(stU, c) + (rb + rr) * ULD)[c4];
                        acc[it].x += b.x; acc[it].y += b.y; acc[it].z += b.z; acc[it].w += b.w;
                    }
                    cur[it] = reinterpret_cast<const float4*>(U + (int64_t)(icol0 + rb + rr) * K)[c4];
                }
            }
#pragma unroll
            for (int it = 0; it < UIT; ++it) {
                const int idx = tid + it * kSplitThreads, rr = idx / NQ, c4 = idx % NQ;
                if (idx < 32 * NQ && icol0 + rb + rr < K) {
                    float4 d = cur[it];
                    d.x += acc[it].x; d.y += acc[it].y; d.z += acc[it].z; d.w += acc[it].w;
                    reinterpret_cast<float4*>(U + (int64_t)(icol0 + rb + rr) * K)[c4] = d;
                }
            }
            }
            if (do_c) {
                const int M = p.M;
                float* Cn = p.cntp + (int64_t)sg * K * M;
                // batches of four entries per thread: their loads first, then their stores
                constexpr int CB = 4;
                for (int base = tid; base < 32 * M; base += CB * kSplitThreads) {
                    float cacc[CB], ccur[CB];
#pragma unroll
                    for (int it = 0; it < CB; ++it) {
                        const int idx = base + it * kSplitThreads, rr = idx / M, k = idx % M;
                        cacc[it] = 0.f;
                        ccur[it] = 0.f;
                        if (idx < 32 * M && icol0 + rb + rr < K) {
#pragma unroll
                            for (int c = 0; c < kCluster; ++c) cacc[it] += cluster.map_shared_rank(stC, c)[(rb + rr) * CLD + k];
                            ccur[it] = Cn[(int64_t)(icol0 + rb + rr) * M + k];
                        }
                    }
#pragma unroll
                    for (int it = 0; it < CB; ++it) {
                        const int idx = base + it * kSplitThreads, rr = idx / M, k = idx % M;
                        if (idx < 32 * M && icol0 + rb + rr < K) Cn[(int64_t)(icol0 + rb + rr) * M + k] = ccur[it] + cacc[it];
                    }
                }
            }
        }
        cluster.sync();                       // no CTA leaves while a peer still reads its staging
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, p.tmem_cols);
}

int xi_counts_cols(int M) { return (M + 63) / 64 * 64; }

}  // namespace

bool xi_tc_supported(int K) { return K == 64 || K == 128 || K == 256; }
bool xi_tc_counts_supported(int K, int M) { return xi_tc_supported(K) && K + xi_counts_cols(M) <= 512 && xi_counts_cols(M) <= 256; }

namespace {
// Dynamic shared memory of a launch: the split stages (as many as fit, at most kMaxStages;
// + alignment slack of the block), at least the epilogue's staging of the accumulators -- U
// and the counts together if that fits, else one after the other (*two_phase).
size_t xi_smem_bytes(int K, int Mp, bool counts, int* stages_out, bool* two_phase) {
    const StageLayout sl = stage_layout(K, Mp, counts);
    const size_t optin = (size_t)max_smem_optin();
    int stages = kMaxStages;
    while (stages > 2 && (size_t)stages * sl.bytes + 1024 > optin) --stages;
    if (stages_out) *stages_out = stages;
    size_t smem = (size_t)stages * sl.bytes + 1024;
    const size_t su = (size_t)128 * (K + 4) * 4, sc = counts ? (size_t)128 * (Mp + 4) * 4 : 0;
    const bool two = su + sc + 1024 > optin;
    if (two_phase) *two_phase = two;
    const size_t staging = (two ? (su > sc ? su : sc) : su + sc) + 1024;
    return smem < staging ? staging : smem;
}

void (*xi_kernel(int K, bool counts))(XiPrm) {
    switch (K) {
        case 64: return counts ? k_xi_tc<64, true> : k_xi_tc<64, false>;
        case 128: return counts ? k_xi_tc<128, true> : k_xi_tc<128, false>;
        default: return counts ? k_xi_tc<256, true> : k_xi_tc<256, false>;
    }
}
}  // namespace

// Row splits of a launch: one CTA per split and i block, in whole clusters, no more CTAs
// than are resident at once (clusters of four fit 144 of 152 SMs: a second wave of the last
// clusters would double the call).
int xi_tc_splits(int K, int M, bool counts) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const int Mp = counts ? xi_counts_cols(M) : 0;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, K, Mp, counts ? 1 : 0);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int nib = (K + 127) / 128;
    int n = num_sms() / nib;
    void (*kern)(XiPrm) = xi_kernel(K, counts);
    const size_t smem = xi_smem_bytes(K, Mp, counts, nullptr, nullptr);
    int maxcl = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.gridDim = dim3((unsigned)(kCluster * nib), 1, 1);
        lc.blockDim = dim3(kThreads, 1, 1);
        lc.dynamicSmemBytes = smem;
        lc.attrs = attr;
        lc.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&maxcl, kern, &lc) != cudaSuccess) maxcl = 0;
    }
    cudaGetLastError();
    if (maxcl > 0 && maxcl * kCluster / nib < n) n = maxcl * kCluster / nib;
    n = n > kXiSplitMax ? kXiSplitMax : n;
    n = n / kCluster * kCluster;                  // whole clusters
    if (n < kCluster) n = kCluster;
    cache[key] = n;
    return n;
}

int xi_tc_partials(int K, int M, bool counts) { return xi_tc_splits(K, M, counts) / kCluster; }

accel_status xi_tc_round(const float* P, const float* Q, const float* G, const int32_t* osym, const int32_t* rows_r,
                         int K, int M, float* Upart, float* cntp, int32_t* status, cudaStream_t st) {
    const bool counts = cntp != nullptr;
    XiPrm p;
    p.P = P; p.Q = Q; p.G = G; p.osym = osym; p.rows_r = rows_r;
    p.K = K; p.M = M; p.Mp = counts ? xi_counts_cols(M) : 0;
    p.nib = (K + 127) / 128;
    p.nsplit = xi_tc_splits(K, M, counts);
    p.Upart = Upart; p.cntp = cntp; p.status = status;
    const int need_cols = K + p.Mp;
    uint32_t cols = 32;
    while ((int)cols < need_cols) cols <<= 1;
    p.tmem_cols = cols;
    int stages = 2;
    bool two = false;
    const size_t smem = xi_smem_bytes(K, p.Mp, counts, &stages, &two);
    p.two_phase = two ? 1 : 0;
    ACCEL_REQUIRE(smem <= (size_t)max_smem_optin(), ACCEL_ERR_UNSUPPORTED,
                  "hmm_adjoint: count/transition stages do not fit in shared memory (K=%d, M=%d)", K, M);
    p.stages = stages;
    void (*kern)(XiPrm) = xi_kernel(K, counts);
    ACCEL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.gridDim = dim3((unsigned)(p.nib * p.nsplit), 1, 1);
    lc.blockDim = dim3(kThreads, 1, 1);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    lc.attrs = attr;
    lc.numAttrs = 1;
    ACCEL_CUDA_TRY(cudaLaunchKernelEx(&lc, kern, p));
    return ACCEL_OK;
}

}  // namespace hmm
}  // namespace accel
