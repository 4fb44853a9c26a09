// Segmented reduce with a fused map (K5): the nested pattern
//     map (lam s. reduce f ne (map g s))   over a flattened [[T]]     (Appendix A)
// d_out[s] = f-fold of g(data[k]) over k in [off[s], off[s+1]), ne for an empty segment.
//
// Design (HBM-bound streaming):
//  * The flat data is cut into fixed tiles of 16 KB (4096 4-byte or 2048 8-byte
//    elements), one CTA of 256 threads per tile, so the load is balanced whatever the
//    segment lengths are.  A segment is OWNED by the tile holding its last element (an
//    empty segment by the tile holding its position, clamped to N-1).  Owned segments of
//    tile b are the contiguous range [lo[b], lo[b+1]), scattered by a small partition
//    kernel from the monotone keys.
//  * Loads are 16-byte vectors, coalesced across the CTA, staged through shared memory
//    with an XOR swizzle so that each thread then reads its 16 contiguous elements
//    conflict-free.  The tile's offsets are cached in shared memory too.
//  * Each thread folds its elements in order, writing every segment that starts and
//    ends inside it.  Partial segments crossing thread boundaries are combined by a
//    CTA-wide key-segmented scan; segments crossing tile boundaries by a deterministic
//    fixup kernel that folds the preceding tiles' carry-outs in tile order.
#include "common.cuh"

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

namespace accel {
namespace segred {

constexpr int kThreads = 256;
constexpr int kTileBytes = 16384;
constexpr int kVecs = kTileBytes / 16;            // 1024 16-byte vectors per tile
constexpr int kVecPerThread = kVecs / kThreads;   // 4
constexpr int kOffCap = 1024;                     // offsets cached in shared memory

template <typename Tin> constexpr int items() { return kTileBytes / kThreads / (int)sizeof(Tin); }
template <typename Tin> constexpr int tile_elems() { return kTileBytes / (int)sizeof(Tin); }

__device__ __forceinline__ int swz(int v) { return v ^ ((v >> 3) & 7); }

// key(s): last element of a non-empty segment, position of an empty one, clamped to N-1.
__device__ __forceinline__ int64_t seg_key(const int64_t* __restrict__ off, int64_t s, int64_t N) {
    int64_t a = off[s], b = off[s + 1];
    int64_t k = b > a ? b - 1 : a;
    return k < N - 1 ? k : N - 1;
}

// lo[b] = first segment with key >= b * TILE, for b in [0, ntiles]; lo[ntiles] = S.  Built by
// a scatter: segment s writes lo[b] = s for every tile b
// in (tile(key(s-1)), tile(key(s))] (keys are monotone, so each b is written exactly once),
// and thread S writes lo[b] = S for the tiles past the last key.  One coalesced pass over
// the offsets, with no dependent-load chain.
__global__ void k_partition_scatter(const int64_t* __restrict__ off, int64_t S, int64_t N, int64_t tile,
                                    int64_t ntiles, int64_t* __restrict__ lo) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s > S) return;
    const int64_t tprev = s == 0 ? -1 : seg_key(off, s - 1, N) / tile;
    const int64_t tcur = s == S ? ntiles : seg_key(off, s, N) / tile;
    for (int64_t b = tprev + 1; b <= tcur; ++b) lo[b] = s;
}

// Bring the 16 KB tile `b` into L2 ahead of its CTA (full tiles only; no completion to wait
// for).  A CTA prefetches the tile about half a wave of resident CTAs ahead of its own, so
// the CTA that later takes it finds it in L2: more bytes in flight than the resident CTAs'
// own loads alone.
template <typename Tin>
__device__ __forceinline__ void prefetch_tile(const Tin* data, int64_t N, int64_t b) {
    constexpr int64_t TE = kTileBytes / (int64_t)sizeof(Tin);
    if ((b + 1) * TE <= N)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(data + b * TE), "r"((uint32_t)kTileBytes) : "memory");
}

template <typename C> struct KV { int32_t k; C v; };

template <int OP, typename C>
__device__ __forceinline__ KV<C> seg_combine(KV<C> a, KV<C> b) {
    // (k1, v1) + (k2, v2) = (k2, k1 == k2 ? v1 f v2 : v2); associative for monotone keys.
    KV<C> r;
    r.k = b.k;
    r.v = (a.k == b.k) ? red_combine<OP, C>(a.v, b.v) : b.v;
    return r;
}

template <typename C> __device__ __forceinline__ C shfl_up_val(C v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }

__device__ __forceinline__ int64_t sq_wide(int32_t x) { return (int64_t)x * (int64_t)x; }
__device__ __forceinline__ uint64_t sq_wide(int64_t x) { return (uint64_t)x * (uint64_t)x; }
template <typename T> __device__ __forceinline__ T sq_wide(T x) { return x * x; }

// Fold of g(x) over the first n of a thread's IT raw items, in item order: the map
// switch sits outside the (unrolled) element loop.  For an integer sum of x*x + 1 the
// fold is sum(x*x) + n: one widening multiply-add per element, exact in int64.
template <int OP, typename Tin, typename C, int IT>
__device__ __forceinline__ C fused_fold(int map_op, const Tin* __restrict__ xs, int n, C sc, C nel) {
    C acc = nel;
    if constexpr (OP == ACCEL_RED_ADD && std::is_integral<C>::value) {
        if (map_op == ACCEL_MAP_SQ_PLUS_ONE) {
            // x*x of a 32-bit x is exact in 64 bits (a widening multiply); only the running
            // sum wraps, so accumulate unsigned
            uint64_t u = (uint64_t)acc;
            if (n == IT) {
#pragma unroll
                for (int i = 0; i < IT; ++i) u += (uint64_t)sq_wide(xs[i]);
            } else {
#pragma unroll
                for (int i = 0; i < IT; ++i)
                    if (i < n) u += (uint64_t)sq_wide(xs[i]);
            }
            return (C)(u + (uint64_t)n);
        }
    }
    switch (map_op) {
#define ACCEL_FOLD_CASE(MAPID)                                                                   \
        case MAPID:                                                                              \
            _Pragma("unroll") for (int i = 0; i < IT; ++i)                                      \
                if (i < n) acc = red_combine<OP, C>(acc, map_apply<MAPID, C>((C)xs[i], C(0), sc)); \
            break;
        ACCEL_FOLD_CASE(ACCEL_MAP_SQ_PLUS_ONE)
        ACCEL_FOLD_CASE(ACCEL_MAP_NEG)
        ACCEL_FOLD_CASE(ACCEL_MAP_ABS)
        ACCEL_FOLD_CASE(ACCEL_MAP_SCALE)
        ACCEL_FOLD_CASE(ACCEL_MAP_IDENTITY)
#undef ACCEL_FOLD_CASE
    }
    return acc;
}

template <typename C> __device__ __forceinline__ C map_one(int op, C x, C s) {
    switch (op) {
        case ACCEL_MAP_SQ_PLUS_ONE: return map_apply<ACCEL_MAP_SQ_PLUS_ONE, C>(x, C(0), s);
        case ACCEL_MAP_NEG: return map_apply<ACCEL_MAP_NEG, C>(x, C(0), s);
        case ACCEL_MAP_ABS: return map_apply<ACCEL_MAP_ABS, C>(x, C(0), s);
        case ACCEL_MAP_SCALE: return map_apply<ACCEL_MAP_SCALE, C>(x, C(0), s);
        default: return x;
    }
}

template <typename Tin, typename Tout, int OP>
__global__ void __launch_bounds__(kThreads)
k_segreduce(const Tin* __restrict__ data, int64_t N, const int64_t* __restrict__ off, int64_t S,
            const int64_t* __restrict__ lo_arr, int map_op, double scalar, Tout* __restrict__ out,
            int64_t* __restrict__ tail_seg, typename compute_of<Tout>::type* __restrict__ tail_val, int64_t pf) {
    using C = typename compute_of<Tout>::type;
    constexpr int IT = items<Tin>();
    constexpr int TE = tile_elems<Tin>();
    constexpr int PV = 16 / (int)sizeof(Tin);     // elements per 16-byte vector
    __shared__ int4 s_data[kVecs];
    __shared__ int32_t s_pos[kOffCap];              // offsets relative to the tile, clamped
    __shared__ KV<C> s_warp[kThreads / 32];

    const int t = threadIdx.x;
    const int64_t b = blockIdx.x;
    const int64_t e0 = b * TE;
    const int ne = (int)((e0 + TE < N) ? TE : N - e0);   // elements in this tile
    const int64_t lo_b = lo_arr[b], hi_b = lo_arr[b + 1];
    if (t == 0 && pf > 0) prefetch_tile(data, N, b + pf);
    const C nel = red_neutral<C>(OP);
    const Tout nel_out = red_neutral<Tout>(OP);   // an empty segment: the output type's own neutral
    const C sc = (C)scalar;

    // ---- stage the tile (16-byte vectors, coalesced) and the tile's offsets
    if (ne == TE) {
        const int4* src = reinterpret_cast<const int4*>(data + e0);
#pragma unroll
        for (int r = 0; r < kVecPerThread; ++r) {
            int v = r * kThreads + t;
            s_data[swz(v)] = __ldg(src + v);
        }
    } else {
        Tin* sd = reinterpret_cast<Tin*>(s_data);
        for (int e = t; e < TE; e += kThreads) sd[swz(e / PV) * PV + e % PV] = e < ne ? data[e0 + e] : Tin(0);
    }
    // positions off[lo_b .. last] - e0, clamped to [-1, TE + 1]; last = min(hi_b + 1, S)
    const int64_t last = (hi_b + 1 < S) ? hi_b + 1 : S;
    const int64_t cnt = last - lo_b + 1;
    const bool in_smem = cnt <= kOffCap;
    auto clamp_rel = [&](int64_t x) -> int32_t {
        int64_t r = x - e0;
        return (int32_t)(r < -1 ? -1 : (r > TE + 1 ? TE + 1 : r));
    };
    if (in_smem)
        for (int i = t; i < cnt; i += kThreads) s_pos[i] = clamp_rel(off[lo_b + i]);
    __syncthreads();
    // start of segment lo_b + q (relative index q), and its end; past the cached range: TE+1
    auto rel = [&](int q) -> int32_t { return in_smem ? s_pos[q] : clamp_rel(off[lo_b + q]); };
    const int qlast = (int)(last - lo_b);
    auto rel_end = [&](int q) -> int32_t { return q + 1 <= qlast ? rel(q + 1) : TE + 1; };

    // ---- this thread's elements [r0, r1) relative to the tile
    const int r0 = t * IT;
    const int r1 = min(r0 + IT, ne);
    const bool active = r0 < ne;
    const int rN = (int)((N - e0 < (int64_t)TE + 2) ? N - e0 : (int64_t)TE + 2);   // position of N (the end of the data)

    KV<C> tail;                 // (relative segment index, partial) handed to the scan
    bool tail_open = false;     // elements accumulated after the last segment end
    bool has_head = false;
    int head_q = 0;
    C head_val = nel;

    if (active) {
        // segment containing r0: largest q in [0, hi_b - lo_b] with rel(q) <= r0
        int a = 0, z = (int)(hi_b - lo_b);
        while (a < z) {
            int mid = (a + z + 1) >> 1;
            if (rel(mid) <= r0) a = mid; else z = mid - 1;
        }
        int q = a;
        // empty segments positioned at r0 precede q: they are owned here
        for (int p = q - 1; p >= 0 && rel(p) == r0 && rel(p + 1) == r0; --p) out[lo_b + p] = nel_out;
        int nend = rel_end(q);
        if (nend > r1) {
            // no segment ends among this thread's items: one fused map + fold
            int4 raw[kVecPerThread];
#pragma unroll
            for (int r = 0; r < kVecPerThread; ++r) raw[r] = s_data[swz(t * kVecPerThread + r)];
            tail.k = q;
            tail.v = fused_fold<OP, Tin, C, IT>(map_op, reinterpret_cast<const Tin*>(raw), r1 - r0, sc, nel);
            tail_open = true;
        } else {
            // general path: walk the items (read from shared memory), ending segments as met
            const Tin* sd = reinterpret_cast<const Tin*>(s_data);
            bool started_here = rel(q) >= r0;
            C acc = nel;
#pragma unroll 1
            for (int k = r0; k < r1; ++k) {
                acc = red_combine<OP, C>(acc, map_one<C>(map_op, (C)sd[swz(k / PV) * PV + k % PV], sc));
                tail_open = true;
                if (k == nend - 1) {
                    tail_open = false;
                    if (started_here) out[lo_b + q] = (Tout)acc;
                    else { has_head = true; head_q = q; head_val = acc; }
                    acc = nel;
                    started_here = true;
                    ++q;
                    // empty segments at position k+1 belong here if k+1 < r1, or if k+1 is the
                    // end of the data (their key is clamped to N-1)
                    while (lo_b + q < S && (k + 1 < r1 || k + 1 == rN)) {
                        if (!(rel(q) == k + 1 && rel_end(q) == k + 1)) break;
                        out[lo_b + q] = nel_out;
                        ++q;
                    }
                    nend = (lo_b + q < S) ? rel_end(q) : TE + 2;
                }
            }
            tail.k = q;
            tail.v = acc;
        }
    } else {
        tail.k = INT32_MAX;
        tail.v = nel;
    }

    // ---- CTA-wide inclusive key-segmented scan of the tails (keys are relative indices)
    const int lane = t & 31, warp = t >> 5;
    KV<C> qv = tail;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        KV<C> o;
        o.k = __shfl_up_sync(0xffffffffu, qv.k, d);
        o.v = shfl_up_val<C>(qv.v, d);
        if (lane >= d) qv = seg_combine<OP, C>(o, qv);
    }
    if (lane == 31) s_warp[warp] = qv;
    __syncthreads();
    KV<C> wpre;  // fold of warps 0..warp-1
    wpre.k = INT32_MIN;
    wpre.v = nel;
    for (int w = 0; w < warp; ++w) wpre = (w == 0) ? s_warp[0] : seg_combine<OP, C>(wpre, s_warp[w]);
    if (warp > 0) qv = seg_combine<OP, C>(wpre, qv);
    // exclusive value for this thread = inclusive value of thread t-1
    KV<C> ex;
    ex.k = __shfl_up_sync(0xffffffffu, qv.k, 1);
    ex.v = shfl_up_val<C>(qv.v, 1);
    if (lane == 0) ex = wpre;

    if (has_head) {
        C carry = (t > 0 && ex.k == head_q) ? ex.v : nel;
        out[lo_b + head_q] = (Tout)red_combine<OP, C>(carry, head_val);
    }
    // tile carry-out: the last active thread
    const int t_last = (ne - 1) / IT;
    if (t == t_last) {
        if (tail_open) { tail_seg[b] = lo_b + tail.k; tail_val[b] = qv.v; }
        else tail_seg[b] = -1;
    }
}

// Integer sums: a branch-free variant with few instructions per element.  The tile's mapped
// values are prefix-summed across the CTA (each thread scans its IT contiguous items, a
// CTA-wide scan adds the thread offsets) into shared memory, and every owned segment's sum
// is P[end-1] - P[start-1].  Wrapping 64-bit addition forms a group, so the differences are
// exact whatever the magnitudes; every thread does the same work whatever the segment
// lengths.  For the common map x*x + 1 on a full tile, P' = prefix of x*x is formed with one
// widening multiply-add per element and P[k] = P'[k] + k + 1 is applied at lookup.  The
// prefix array is item-major (item i of thread t at i * kThreads + t), so the stores are
// conflict-free with constant offsets.  The tile's open segment (if its last element does
// not end a segment) is handed to the fixup kernel.
template <typename Tin>
__device__ __forceinline__ uint64_t gmap(int map_op, int64_t x, int64_t sc) {
    switch (map_op) {
        case ACCEL_MAP_SQ_PLUS_ONE: return (uint64_t)x * (uint64_t)x + 1ull;
        case ACCEL_MAP_NEG: return 0ull - (uint64_t)x;
        case ACCEL_MAP_ABS: return x < 0 ? 0ull - (uint64_t)x : (uint64_t)x;
        case ACCEL_MAP_SCALE: return (uint64_t)sc * (uint64_t)x;
        default: return (uint64_t)x;
    }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads)
k_segsum(const Tin* __restrict__ data, int64_t N, const int64_t* __restrict__ off, int64_t S,
         const int64_t* __restrict__ lo_arr, int map_op, double scalar, Tout* __restrict__ out,
         int64_t* __restrict__ tail_seg, int64_t* __restrict__ tail_val, int64_t pf) {
    constexpr int IT = items<Tin>();
    constexpr int TE = tile_elems<Tin>();
    constexpr int PV = 16 / (int)sizeof(Tin);
    // the staged tile and, once every thread holds its items, the prefix sums share storage
    __shared__ __align__(16) uint64_t s_buf[TE];
    int4* s_data = reinterpret_cast<int4*>(s_buf);  // kVecs 16-byte vectors (16 KB)
    uint64_t* s_P = s_buf;                          // prefix of the mapped values, item-major
    __shared__ int32_t s_pos[kOffCap];
    __shared__ uint64_t s_wtot[kThreads / 32];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t b = blockIdx.x;
    const int64_t e0 = b * TE;
    const int ne = (int)((e0 + TE < N) ? TE : N - e0);
    const int64_t lo_b = lo_arr[b], hi_b = lo_arr[b + 1];
    const int64_t sc = (int64_t)scalar;
    const bool fast = map_op == ACCEL_MAP_SQ_PLUS_ONE && ne == TE;
    if (t == 0 && pf > 0) prefetch_tile(data, N, b + pf);

    if (ne == TE) {
        const int4* src = reinterpret_cast<const int4*>(data + e0);
#pragma unroll
        for (int r = 0; r < kVecPerThread; ++r) {
            int v = r * kThreads + t;
            s_data[swz(v)] = __ldg(src + v);
        }
    } else {
        Tin* sd = reinterpret_cast<Tin*>(s_data);
        for (int e = t; e < TE; e += kThreads) sd[swz(e / PV) * PV + e % PV] = e < ne ? data[e0 + e] : Tin(0);
    }
    const int64_t last = (hi_b + 1 < S) ? hi_b + 1 : S;
    const int64_t cnt = last - lo_b + 1;
    const bool in_smem = cnt <= kOffCap;
    // segment start relative to the tile, clamped to [0, ne]
    auto clamp_rel = [&](int64_t x) -> int32_t {
        const int64_t r = x - e0;
        return (int32_t)(r < 0 ? 0 : (r > ne ? ne : r));
    };
    if (in_smem)
        for (int i = t; i < cnt; i += kThreads) s_pos[i] = clamp_rel(off[lo_b + i]);
    __syncthreads();
    auto rel = [&](int64_t q) -> int32_t { return in_smem ? s_pos[q] : clamp_rel(off[lo_b + q]); };

    // ---- per-thread items and their total
    const int r0 = t * IT;
    const int n = max(0, min(IT, ne - r0));
    int4 raw[kVecPerThread];
#pragma unroll
    for (int r = 0; r < kVecPerThread; ++r) raw[r] = s_data[swz(t * kVecPerThread + r)];
    const Tin* xs = reinterpret_cast<const Tin*>(raw);
    uint64_t run = 0;
    if (fast) {
#pragma unroll
        for (int i = 0; i < IT; ++i) run += (uint64_t)sq_wide(xs[i]);
    } else {
#pragma unroll
        for (int i = 0; i < IT; ++i)
            if (i < n) run += gmap<Tin>(map_op, (int64_t)xs[i], sc);
    }
    // ---- CTA-wide exclusive scan of the thread totals
    uint64_t inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) s_wtot[warp] = inc;
    __syncthreads();   // also: every thread has read its items from the staging buffer
    uint64_t acc = inc - run;
    for (int w = 0; w < warp; ++w) acc += s_wtot[w];
    if (fast) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            acc += (uint64_t)sq_wide(xs[i]);
            s_P[i * kThreads + t] = acc;
        }
    } else {
#pragma unroll
        for (int i = 0; i < IT; ++i)
            if (i < n) { acc += gmap<Tin>(map_op, (int64_t)xs[i], sc); s_P[i * kThreads + t] = acc; }
    }
    __syncthreads();

    // ---- owned segments: sum over [start, end) of the tile = P(end) - P(start), where
    // P(p) = sum of g over the tile's positions < p
    auto Pb = [&](int32_t p) -> uint64_t {
        if (p <= 0) return 0ull;
        const int k = p - 1;
        const uint64_t v = s_P[(k % IT) * kThreads + k / IT];
        return fast ? v + (uint64_t)p : v;
    };
    const int64_t nown = hi_b - lo_b;
    for (int64_t q = t; q < nown; q += kThreads) out[lo_b + q] = (Tout)(int64_t)(Pb(rel(q + 1)) - Pb(rel(q)));
    // ---- the tile's open segment: segment hi_b if it starts at or before the last element
    if (t == 0) {
        const int32_t a = (hi_b < S) ? rel(nown) : ne;
        if (a <= ne - 1) {
            tail_seg[b] = hi_b;
            tail_val[b] = (int64_t)(Pb(ne) - Pb(a));
        } else {
            tail_seg[b] = -1;
        }
    }
}

// Folds the carry-outs of the tiles preceding b into the first segment b owns, when that
// segment started in an earlier tile.  Tile order is kept, so float results are
// deterministic.
template <typename Tout, int OP>
__global__ void k_fixup(const int64_t* __restrict__ off, const int64_t* __restrict__ lo_arr, int64_t ntiles,
                        int64_t tile, const int64_t* __restrict__ tail_seg,
                        const typename compute_of<Tout>::type* __restrict__ tail_val, Tout* __restrict__ out) {
    using C = typename compute_of<Tout>::type;
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= ntiles || b == 0) return;
    int64_t s = lo_arr[b];
    if (s >= lo_arr[b + 1]) return;            // owns nothing
    if (off[s] >= b * tile) return;            // first owned segment starts in this tile
    if (off[s + 1] == off[s]) return;          // empty (cannot cross)
    int64_t a = b - 1;
    while (a >= 0 && tail_seg[a] == s) --a;
    C carry = red_neutral<C>(OP);
    for (int64_t i = a + 1; i < b; ++i) carry = red_combine<OP, C>(carry, tail_val[i]);
    out[s] = (Tout)red_combine<OP, C>(carry, (C)out[s]);
}

template <typename Tout>
__global__ void k_fill(Tout* __restrict__ out, int64_t S, Tout v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) out[i] = v;
}

// Small inputs (N <= kWarpPathMaxN elements, segments of at most 4,096 elements on
// average): one warp per segment, straight from the offsets -- one launch instead of three (partition, tiles, fix-up).  At these sizes the
// call's time is its launches, not its bytes, and the tiled kernel's load balance buys
// nothing.  Lane l folds elements off[s] + l, + 32, ... in order (warp loads of 32
// consecutive elements), then the 32 lane values combine in a fixed butterfly: the result
// is deterministic (bit-exact for integers; for floats a fixed order, not the tiled one).
constexpr int64_t kWarpPathMaxN = int64_t(1) << 20;

template <typename Tin, typename Tout, int OP>
__global__ void __launch_bounds__(kThreads)
k_segreduce_warp(const Tin* __restrict__ data, const int64_t* __restrict__ off, int64_t S, int map_op,
                 double scalar, Tout* __restrict__ out) {
    using C = typename compute_of<Tout>::type;
    const C sc = (C)scalar;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t s = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; s < S; s += nw) {
        const int64_t a = off[s], b = off[s + 1];
        C acc = red_neutral<C>(OP);
        bool done = false;
        if constexpr (OP == ACCEL_RED_ADD && std::is_integral<C>::value) {
            if (map_op == ACCEL_MAP_SQ_PLUS_ONE) {
                // x*x of the input is exact in 64 bits; only the running sum wraps
                uint64_t u = 0;
                for (int64_t k = a + lane; k < b; k += 32) u += (uint64_t)sq_wide(data[k]) + 1u;
                acc = (C)u;
                done = true;
            }
        }
        if (!done)
            for (int64_t k = a + lane; k < b; k += 32) acc = red_combine<OP, C>(acc, map_one<C>(map_op, (C)data[k], sc));
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc = red_combine<OP, C>(acc, (C)__shfl_xor_sync(0xffffffffu, acc, d));
        if (lane == 0) out[s] = b > a ? (Tout)acc : red_neutral<Tout>(OP);
    }
}

struct Layout {
    int64_t ntiles;
    size_t lo_off, seg_off, val_off, total;
};

static Layout layout(int64_t N, int64_t S, size_t in_size) {
    Layout L;
    int64_t te = kTileBytes / (int64_t)in_size;
    L.ntiles = (N + te - 1) / te;
    L.lo_off = kStatusBytes;
    L.seg_off = align_up(L.lo_off + (size_t)(L.ntiles + 1) * 8, 256);
    L.val_off = align_up(L.seg_off + (size_t)L.ntiles * 8, 256);
    L.total = align_up(L.val_off + (size_t)L.ntiles * 8, 256);
    (void)S;
    return L;
}

// Tiles half a wave ahead: half the CTAs resident at once on the device (measured at 2^20
// segments: half a wave 3,452 GB/s, one wave 3,409, two waves 3,342, none 3,187).
template <typename KernT>
static int64_t prefetch_distance(KernT kern) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int64_t> cache;   // per device and kernel
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(dev, (const void*)kern);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    const int64_t d = (int64_t)per_sm * num_sms() / 2;
    cache[key] = d;
    return d;
}

template <typename Tin, typename Tout>
static accel_status run(int32_t op, int32_t map_op, const void* d_data, int64_t N, const int64_t* d_off,
                        int64_t S, double scalar, void* d_out, void* d_ws, cudaStream_t st) {
    using C = typename compute_of<Tout>::type;
    Layout L = layout(N, S, sizeof(Tin));
    char* ws = (char*)d_ws;
    int64_t* lo = (int64_t*)(ws + L.lo_off);
    int64_t* tseg = (int64_t*)(ws + L.seg_off);
    C* tval = (C*)(ws + L.val_off);
    Tout* out = (Tout*)d_out;
    if (N == 0) {
        Tout nel = 0;
        ACCEL_DISPATCH_RED(op, OPC, (nel = red_neutral<Tout>(OPC)));
        int g = (int)((S + 255) / 256);
        if (g > 8 * num_sms()) g = 8 * num_sms();
        k_fill<Tout><<<g, 256, 0, st>>>(out, S, nel);
        return after_launch(st, "accel_segreduce(fill)", 1);
    }
    if (N <= kWarpPathMaxN && N <= 4096 * S) {
        int64_t g = (S + kThreads / 32 - 1) / (kThreads / 32);
        if (g > 8 * (int64_t)num_sms()) g = 8 * (int64_t)num_sms();
        ACCEL_DISPATCH_RED(op, OPC, {
            k_segreduce_warp<Tin, Tout, OPC><<<(unsigned)g, kThreads, 0, st>>>((const Tin*)d_data, d_off, S, map_op,
                                                                                scalar, out);
        });
        return after_launch(st, "accel_segreduce", 1);
    }
    int64_t te = tile_elems<Tin>();
    k_partition_scatter<<<(unsigned)((S + 1 + 255) / 256), 256, 0, st>>>(d_off, S, N, te, L.ntiles, lo);
    if constexpr (std::is_integral<C>::value) {
        if (op == ACCEL_RED_ADD) {
            k_segsum<Tin, Tout><<<(unsigned)L.ntiles, kThreads, 0, st>>>(
                (const Tin*)d_data, N, d_off, S, lo, map_op, scalar, out, tseg, (int64_t*)tval,
                prefetch_distance(k_segsum<Tin, Tout>));
            k_fixup<Tout, ACCEL_RED_ADD><<<(unsigned)((L.ntiles + 255) / 256), 256, 0, st>>>(d_off, lo, L.ntiles, te,
                                                                                            tseg, tval, out);
            return after_launch(st, "accel_segreduce", 3);
        }
    }
    ACCEL_DISPATCH_RED(op, OPC, {
        k_segreduce<Tin, Tout, OPC><<<(unsigned)L.ntiles, kThreads, 0, st>>>(
            (const Tin*)d_data, N, d_off, S, lo, map_op, scalar, out, tseg, tval,
            prefetch_distance(k_segreduce<Tin, Tout, OPC>));
        k_fixup<Tout, OPC><<<(unsigned)((L.ntiles + 255) / 256), 256, 0, st>>>(d_off, lo, L.ntiles, te, tseg, tval, out);
    });
    return after_launch(st, "accel_segreduce", 3);
}

}  // namespace segred
}  // namespace accel

using namespace accel;

extern "C" {

size_t accel_segreduce_workspace_size(int64_t N, int64_t S) {
    // sized for the largest element (8 bytes: the fewest elements per tile, so the most tiles)
    return segred::layout(N < 0 ? 0 : N, S, 8).total;
}

accel_status accel_segreduce(int32_t op, int32_t fused_map, int32_t in_dtype, int32_t out_dtype, const void* d_data,
                             int64_t N, const int64_t* d_offsets, int64_t S, double scalar, void* d_out, void* d_ws,
                             size_t ws_bytes, void* stream) {
    ACCEL_REQUIRE(op >= ACCEL_RED_ADD && op <= ACCEL_RED_MAX, ACCEL_ERR_INVALID_ARG, "accel_segreduce: bad op %d", op);
    ACCEL_REQUIRE(fused_map >= ACCEL_MAP_IDENTITY && fused_map <= ACCEL_MAP_SCALE, ACCEL_ERR_INVALID_ARG,
                  "accel_segreduce: fused map must be a single-operand map (got %d)", fused_map);
    ACCEL_REQUIRE(dtype_valid(in_dtype) && dtype_valid(out_dtype), ACCEL_ERR_DTYPE, "accel_segreduce: bad dtype");
    ACCEL_REQUIRE(dtype_is_int(in_dtype) == dtype_is_int(out_dtype), ACCEL_ERR_DTYPE,
                  "accel_segreduce: input and output must both be integer or both float");
    ACCEL_REQUIRE(N >= 0 && S >= 0, ACCEL_ERR_INVALID_ARG, "accel_segreduce: negative size");
    ACCEL_REQUIRE(d_offsets && d_ws && (S == 0 || d_out) && (N == 0 || d_data), ACCEL_ERR_INVALID_ARG,
                  "accel_segreduce: null pointer");
    ACCEL_REQUIRE(((uintptr_t)d_data % 16) == 0, ACCEL_ERR_INVALID_ARG, "accel_segreduce: d_data must be 16-byte aligned");
    ACCEL_REQUIRE(((uintptr_t)d_ws % 256) == 0, ACCEL_ERR_INVALID_ARG, "accel_segreduce: d_ws must be 256-byte aligned");
    ACCEL_REQUIRE(ws_bytes >= accel_segreduce_workspace_size(N, S), ACCEL_ERR_WORKSPACE,
                  "accel_segreduce: workspace %zu < %zu bytes", ws_bytes, accel_segreduce_workspace_size(N, S));
    if (S == 0) return ok();
    cudaStream_t st = as_stream(stream);
    if (debug_mode()) {
        accel_status r = debug_check_offsets(d_offsets, S, N, 0, d_ws, st);
        if (r != ACCEL_OK) return r;
    }
    accel_status r = ACCEL_OK;
    switch (in_dtype * 4 + out_dtype) {
        case ACCEL_I32 * 4 + ACCEL_I32: r = segred::run<int32_t, int32_t>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        case ACCEL_I32 * 4 + ACCEL_I64: r = segred::run<int32_t, int64_t>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        case ACCEL_I64 * 4 + ACCEL_I64: r = segred::run<int64_t, int64_t>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        case ACCEL_I64 * 4 + ACCEL_I32: r = segred::run<int64_t, int32_t>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        case ACCEL_F32 * 4 + ACCEL_F32: r = segred::run<float, float>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        case ACCEL_F32 * 4 + ACCEL_F64: r = segred::run<float, double>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        case ACCEL_F64 * 4 + ACCEL_F64: r = segred::run<double, double>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
        default: r = segred::run<double, float>(op, fused_map, d_data, N, d_offsets, S, scalar, d_out, d_ws, st); break;
    }
    return r;
}

}  // extern "C"

// ----------------------------------------------------------------------------------------
// accel_segreduce_noalloc: the same segmented reduce for callers that cannot allocate
// device memory -- code running where cudaMalloc is unavailable or forbidden, such as
// inside a custom allocator's own callbacks, a plugin host that owns every allocation, or
// a real-time loop that must never reach the allocator.  Its scratch space is the
// file-scope array below, created when the library is loaded on a device and kept until
// the process exits; nothing is allocated or freed per call.
//
// Limits and sharing: the array holds kNoAllocScratchBytes (2 MiB), enough for
// N <= 178,913,280 flat elements per call (any element type; S is not limited); larger
// inputs are rejected with ACCEL_ERR_UNSUPPORTED.  All calls in the process share the array and it
// keeps the last call's contents; every byte a call reads is first written by that same
// call, so nothing has to be cleared in between.  Calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on the array.
// Set-up: the first call on each device looks up the array's device address with
// cudaGetSymbolAddress while that device is current, and caches it; make that first call
// before any stream capture begins.  The cached address belongs to the device's context of
// that moment: resetting the device (cudaDeviceReset) after the first call is not supported.
// ----------------------------------------------------------------------------------------
#include <mutex>

namespace accel {
namespace segred {

constexpr size_t kNoAllocScratchBytes = 2u << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
static accel_status noalloc_scratch(void** out) {
    int dev = 0;
    ACCEL_CUDA_TRY(cudaGetDevice(&dev));
    ACCEL_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, ACCEL_ERR_UNSUPPORTED,
                  "accel_segreduce_noalloc: device index %d >= %d", dev, kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return set_error(ACCEL_ERR_CUDA, "accel_segreduce_noalloc: cudaGetSymbolAddress failed: %s",
                             cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return ACCEL_OK;
}

}  // namespace segred
}  // namespace accel

extern "C" {

accel_status accel_segreduce_noalloc(int32_t op, int32_t fused_map, int32_t in_dtype, int32_t out_dtype,
                                     const void* d_data, int64_t N, const int64_t* d_offsets, int64_t S, double scalar,
                                     void* d_out, void* stream) {
    ACCEL_REQUIRE(N >= 0 && S >= 0, ACCEL_ERR_INVALID_ARG, "accel_segreduce_noalloc: negative size");
    const size_t need = accel_segreduce_workspace_size(N, S);
    ACCEL_REQUIRE(need <= segred::kNoAllocScratchBytes, ACCEL_ERR_UNSUPPORTED,
                  "accel_segreduce_noalloc: N=%lld needs %zu bytes of scratch; the built-in area holds %zu bytes "
                  "(at most 178,913,280 elements); use accel_segreduce with a workspace",
                  (long long)N, need, segred::kNoAllocScratchBytes);
    void* scratch = nullptr;
    accel_status r = segred::noalloc_scratch(&scratch);
    if (r != ACCEL_OK) return r;
    r = accel_segreduce(op, fused_map, in_dtype, out_dtype, d_data, N, d_offsets, S, scalar, d_out, scratch,
                        segred::kNoAllocScratchBytes, stream);
    if (r != ACCEL_OK) {
        // name this entry point in the message of an error found by the shared implementation
        char msg[400];
        snprintf(msg, sizeof(msg), "%s", accel_last_error());
        return set_error(r, "accel_segreduce_noalloc (via %s)", msg);
    }
    return r;
}

}  // extern "C"
