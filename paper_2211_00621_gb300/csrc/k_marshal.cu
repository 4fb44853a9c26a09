// Marshaling (Sec. 3.3): converting the sequential representation of an accelerated
// binding's arguments into the backend format.
//  K1 accel_marshal_ragged  -- [[T]] as a host list of S separately stored sequences ->
//                              flat data + int64 offsets (flatten, Appendix A).
//  K2 accel_marshal_records -- a sequence of records {l_i = e_i} stored as an array of
//                              structures -> one array per field, or back.
//  accel_marshal_nested     -- [[[T]]] (groups of separately stored sequences) -> flat data,
//                              int64 offsets of the sequences, int64 offsets of the groups
//                              into those (two levels of flatten).
//  accel_unmarshal_ragged   -- the inverse of K1: flat data + offsets -> S separately stored
//                              destination arrays (device memory or pinned host memory
//                              written by the kernel directly).
#include "common.cuh"

namespace accel {
namespace marshal {

constexpr int kScanThreads = 1024;   // elements scanned per block = kScanThreads

// ---------------------------------------------------------------- exclusive scan
// Block-local inclusive scan of int64 (warp shuffles + one shared level).
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) s_warp[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t x = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t o = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += o;
        }
        s_warp[lane] = x;  // inclusive warp prefix
    }
    __syncthreads();
    if (w > 0) v += s_warp[w - 1];
    return v;
}

// pass 1: per-block totals of the lengths; `copy` (may be null) receives the lengths read
// (when they are read from host memory, so the third pass reads them from the device)
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const int64_t* __restrict__ len, int64_t S,
                                                               int64_t* __restrict__ bsum, int64_t* __restrict__ copy) {
    __shared__ int64_t s_warp[32];
    int64_t i = blockIdx.x * (int64_t)kScanThreads + threadIdx.x;
    int64_t v = i < S ? len[i] : 0;
    if (copy && i < S) copy[i] = v;
    v = block_incl_scan(v, s_warp);
    if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = v;
}

// pass 2: exclusive scan of the block totals, in place, by one block (chunks with carry)
__global__ void __launch_bounds__(kScanThreads) k_scan_totals(int64_t* __restrict__ bsum, int64_t nb) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t inc = block_incl_scan(v, s_warp);
        int64_t carry = s_carry;
        if (i < nb) bsum[i] = carry + inc - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = carry + inc;
        __syncthreads();
    }
}

// pass 3: offsets[i] = block prefix + exclusive in-block prefix; offsets[S] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_final(const int64_t* __restrict__ len, int64_t S,
                                                              const int64_t* __restrict__ bpre,
                                                              int64_t* __restrict__ off) {
    __shared__ int64_t s_warp[32];
    int64_t i = blockIdx.x * (int64_t)kScanThreads + threadIdx.x;
    int64_t v = i < S ? len[i] : 0;
    int64_t inc = block_incl_scan(v, s_warp);
    int64_t p = bpre[blockIdx.x];
    if (i < S) off[i] = p + inc - v;
    if (i == S - 1) off[S] = p + inc;
}

// small inputs (S <= kScanSmall): the whole exclusive scan in one CTA, chunk by chunk with a
// running carry -- one launch instead of three
constexpr int64_t kScanSmall = 16 * kScanThreads;
__global__ void __launch_bounds__(kScanThreads) k_scan_one(const int64_t* __restrict__ len, int64_t S,
                                                            int64_t* __restrict__ off) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < S; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < S ? len[i] : 0;
        const int64_t inc = block_incl_scan(v, s_warp);
        const int64_t carry = s_carry;
        if (i < S) off[i] = carry + inc - v;
        if (i == S - 1) off[S] = carry + inc;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = carry + inc;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- ragged gather
// Each warp takes batches of SPB consecutive sequences (grid-stride over batches): lane l
// loads the metadata of sequence b0 + l (offset, length, source pointer) with one coalesced
// load per table -- the pointer table may be page-locked host memory read over the
// chip-to-chip link -- then the warp copies the batch's sequences four at a time, the loads of
// a round issued before any of its stores, broadcasting the metadata with shuffles.  SPB
// (1 .. 32) is chosen by the host so that there are enough batches to fill the device.
// Four sequences at a time, in rounds of 128 elements of each: every lane issues its 4 x 4
// loads before any of the round's stores, so a warp keeps 2 KB (int32) in flight even when
// the sequences are short.
template <typename T>
__device__ __forceinline__ void gather_quad(const T* const (&src)[4], T* const (&dst)[4], const int (&n)[4], int lane) {
    const int nmax = max(max(n[0], n[1]), max(n[2], n[3]));
    for (int base = 0; base < nmax; base += 32 * 4) {
        T v[4][4];
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = base + r * 32 + lane;
                if (k < n[g]) v[g][r] = src[g][k];
            }
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = base + r * 32 + lane;
                if (k < n[g]) dst[g][k] = v[g][r];
            }
    }
}

// One warp copies a batch of cnt <= 32 consecutive sequences whose metadata lane l holds
// (offset mo, length mn, source ms of sequence l of the batch).
template <typename T>
__device__ __forceinline__ void gather_batch(int64_t mo, int64_t mn, const T* ms, int cnt, T* __restrict__ flat,
                                             int lane) {
    if (__any_sync(0xffffffffu, mn > (int64_t)INT32_MAX)) {
        // a sequence longer than 2^31 - 1 elements: the batch one sequence at a time, 64-bit
        for (int j = 0; j < cnt; ++j) {
            const int64_t o = __shfl_sync(0xffffffffu, mo, j), ng = __shfl_sync(0xffffffffu, mn, j);
            const T* sp = reinterpret_cast<const T*>(__shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(ms), j));
            for (int64_t k = lane; k < ng; k += 32) flat[o + k] = sp[k];
        }
        return;
    }
    for (int j = 0; j < cnt; j += 4) {
        const T* src[4];
        T* dst[4];
        int n[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int jj = j + g < cnt ? j + g : j;          // a missing sequence copies nothing
            const int64_t o = __shfl_sync(0xffffffffu, mo, jj);
            const int ng = __shfl_sync(0xffffffffu, (int)mn, jj);
            src[g] = reinterpret_cast<const T*>(__shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(ms), jj));
            dst[g] = flat + o;
            n[g] = j + g < cnt ? ng : 0;
        }
        gather_quad<T>(src, dst, n, lane);
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_gather(const T* const* __restrict__ ptrs, const int64_t* __restrict__ off,
                                                  int64_t S, int spb, T* __restrict__ flat) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b0 = warp * spb; b0 < S; b0 += nwarps * spb) {
        const int cnt = (int)(S - b0 < spb ? S - b0 : spb);
        int64_t mo = 0, mn = 0;
        const T* ms = nullptr;
        if (lane < cnt) {
            mo = off[b0 + lane];
            mn = off[b0 + lane + 1] - mo;
            ms = ptrs[b0 + lane];
        }
        gather_batch<T>(mo, mn, ms, cnt, flat, lane);
    }
}

// One warp per sequence: dst[s][k] = flat[off[s] + k] (the inverse of k_gather).
template <typename T>
__global__ void __launch_bounds__(256) k_scatter(const T* __restrict__ flat, const int64_t* __restrict__ off, int64_t S,
                                                T* const* __restrict__ ptrs) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < S; s += nwarps) {
        const int64_t o = off[s];
        const int64_t n = off[s + 1] - o;
        const T* src = flat + o;
        T* dst = ptrs[s];
        for (int64_t base = 0; base < n; base += 32 * 8) {
            T v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                int64_t k = base + r * 32 + lane;
                if (k < n) v[r] = src[k];
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                int64_t k = base + r * 32 + lane;
                if (k < n) dst[k] = v[r];
            }
        }
    }
}

// A host table into device memory, in stream order: a page-locked table is read when the
// stream reaches the copy (keep it until then), a pageable one is staged before this returns.
static cudaError_t table_to_device(void* d_dst, const void* h_src, size_t bytes, cudaStream_t st) {
    return cudaMemcpyAsync(d_dst, h_src, bytes, cudaMemcpyHostToDevice, st);
}

// The device address of a page-locked (mapped) host table, or null for pageable memory,
// which must be copied.
static const void* mapped_host(const void* h) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// pointer table (copied there when the host tables are pageable), the length table (ditto,
// or the scan's copy of page-locked lengths), then the scan's block totals
size_t ws_layout(int64_t S, size_t* ptr_off, size_t* len_off, size_t* bsum_off) {
    int64_t nb = (S + kScanThreads - 1) / kScanThreads;
    *ptr_off = kStatusBytes;
    *len_off = *ptr_off + (size_t)S * 8;
    *bsum_off = align_up(*len_off + (size_t)S * 8, 256);
    return align_up(*bsum_off + (size_t)(nb > 0 ? nb : 1) * 8, 256);
}

// ---------------------------------------------------------------- records
struct FieldDesc {
    int32_t nfields;
    int32_t record_bytes;
    int32_t off[ACCEL_MAX_FIELDS];
    int32_t size[ACCEL_MAX_FIELDS];
    void* soa[ACCEL_MAX_FIELDS];
};

// Fast path: 16-byte records of four 4-byte fields at offsets 0, 4, 8, 12.
template <bool INV>
__global__ void __launch_bounds__(256) k_records16(int4* __restrict__ aos, int64_t n, FieldDesc fd) {
    int32_t* f0 = (int32_t*)fd.soa[0];
    int32_t* f1 = (int32_t*)fd.soa[1];
    int32_t* f2 = (int32_t*)fd.soa[2];
    int32_t* f3 = (int32_t*)fd.soa[3];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (!INV) {
            int4 r = aos[i];
            f0[i] = r.x; f1[i] = r.y; f2[i] = r.z; f3[i] = r.w;
        } else {
            aos[i] = make_int4(f0[i], f1[i], f2[i], f3[i]);
        }
    }
}

// General path: one thread per (record, field) pair, 4- or 8-byte scalars.
template <bool INV>
__global__ void __launch_bounds__(256) k_records(char* __restrict__ aos, int64_t n, FieldDesc fd) {
    int64_t total = n * fd.nfields;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / fd.nfields;
        int f = (int)(q - i * fd.nfields);
        char* rec = aos + i * fd.record_bytes + fd.off[f];
        if (fd.size[f] == 4) {
            int32_t* col = (int32_t*)fd.soa[f];
            if constexpr (!INV) col[i] = *(const int32_t*)rec; else *(int32_t*)rec = col[i];
        } else {
            int64_t* col = (int64_t*)fd.soa[f];
            if constexpr (!INV) col[i] = *(const int64_t*)rec; else *(int64_t*)rec = col[i];
        }
    }
}

}  // namespace marshal
}  // namespace accel

using namespace accel;
using namespace accel::marshal;

extern "C" {

size_t accel_marshal_ragged_workspace_size(int64_t S) {
    size_t a, b, c;
    return ws_layout(S < 0 ? 0 : S, &a, &b, &c);
}

accel_status accel_marshal_ragged(const void* const* h_ptrs, const int64_t* h_lengths, int64_t S, int32_t dtype,
                                  void* d_flat, int64_t* d_offsets, void* d_ws, size_t ws_bytes, void* stream) {
    ACCEL_REQUIRE(S >= 0, ACCEL_ERR_INVALID_ARG, "accel_marshal_ragged: S < 0");
    ACCEL_REQUIRE(dtype_valid(dtype), ACCEL_ERR_DTYPE, "accel_marshal_ragged: bad dtype");
    ACCEL_REQUIRE(d_offsets && d_ws && (S == 0 || (h_ptrs && h_lengths)), ACCEL_ERR_INVALID_ARG,
                  "accel_marshal_ragged: null pointer");
    ACCEL_REQUIRE(((uintptr_t)d_ws % 256) == 0, ACCEL_ERR_INVALID_ARG, "accel_marshal_ragged: d_ws must be 256-byte aligned");
    size_t po, lo, bo;
    size_t need = ws_layout(S, &po, &lo, &bo);
    ACCEL_REQUIRE(ws_bytes >= need, ACCEL_ERR_WORKSPACE, "accel_marshal_ragged: workspace %zu < %zu bytes", ws_bytes, need);
    if (debug_mode()) {
        // O(S) checks of the host tables only in debug mode (accelerate mode: O(1) checks)
        int64_t total = 0;
        for (int64_t s = 0; s < S; ++s) {
            ACCEL_REQUIRE(h_lengths[s] >= 0, ACCEL_ERR_SHAPE, "accel_marshal_ragged: length[%lld] < 0", (long long)s);
            ACCEL_REQUIRE(h_lengths[s] == 0 || h_ptrs[s], ACCEL_ERR_INVALID_ARG, "accel_marshal_ragged: ptr[%lld] is null",
                          (long long)s);
            total += h_lengths[s];
        }
        ACCEL_REQUIRE(total == 0 || d_flat, ACCEL_ERR_INVALID_ARG, "accel_marshal_ragged: d_flat is null");
    }
    cudaStream_t st = as_stream(stream);
    if (S == 0) {
        ACCEL_CUDA_TRY(cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), st));
        return after_launch(st, "accel_marshal_ragged", 0);
    }
    char* ws = (char*)d_ws;
    const int64_t* d_len = (int64_t*)(ws + lo);
    int64_t* d_bsum = (int64_t*)(ws + bo);
    const void* const* d_ptrs = (const void* const*)(ws + po);
    const void* dp = mapped_host(h_ptrs);
    const void* dl = mapped_host(h_lengths);
    if (dp && dl) {
        // page-locked tables: the kernels read them in place over the host link (no copy)
        d_ptrs = (const void* const*)dp;
        d_len = (const int64_t*)dl;
    } else {
        ACCEL_CUDA_TRY(table_to_device(ws + po, h_ptrs, (size_t)S * sizeof(void*), st));
        ACCEL_CUDA_TRY(table_to_device(ws + lo, h_lengths, (size_t)S * sizeof(int64_t), st));
    }
    int64_t nb = (S + kScanThreads - 1) / kScanThreads;
    int nscan = 1;
    if (S <= kScanSmall) {
        k_scan_one<<<1, kScanThreads, 0, st>>>(d_len, S, d_offsets);
    } else {
        int64_t* dev_len = (int64_t*)(ws + lo);
        k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(d_len, S, d_bsum, d_len != dev_len ? dev_len : nullptr);
        k_scan_totals<<<1, kScanThreads, 0, st>>>(d_bsum, nb);
        k_scan_final<<<(unsigned)nb, kScanThreads, 0, st>>>(dev_len, S, d_bsum, d_offsets);
        nscan = 3;
    }
    // sequences per warp batch: as many as keep every warp slot of the device busy (8 CTAs of
    // 8 warps per SM), at most 32
    const int64_t slots = (int64_t)num_sms() * 64;
    int spb = 1;
    while (spb < 32 && S / (2 * spb) >= slots) spb *= 2;
    int64_t blocks = ((S + spb - 1) / spb + 7) / 8;
    int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (dtype_size(dtype) == 4)
        k_gather<int32_t><<<(unsigned)blocks, 256, 0, st>>>((const int32_t* const*)d_ptrs, d_offsets, S, spb,
                                                            (int32_t*)d_flat);
    else
        k_gather<int64_t><<<(unsigned)blocks, 256, 0, st>>>((const int64_t* const*)d_ptrs, d_offsets, S, spb,
                                                            (int64_t*)d_flat);
    return after_launch(st, "accel_marshal_ragged", nscan + 1);
}

// offsets[0..n] = exclusive scan of the n host lengths (copied into the workspace first)
static accel_status scan_lengths(const int64_t* h_len, int64_t n, int64_t* d_off, char* ws, cudaStream_t st) {
    size_t po, lo, bo;
    ws_layout(n, &po, &lo, &bo);
    int64_t* d_len = (int64_t*)(ws + lo);
    int64_t* d_bsum = (int64_t*)(ws + bo);
    ACCEL_CUDA_TRY(table_to_device(d_len, h_len, (size_t)n * sizeof(int64_t), st));
    if (n <= kScanSmall) {
        k_scan_one<<<1, kScanThreads, 0, st>>>(d_len, n, d_off);
        count_launches(1);
        return ACCEL_OK;
    }
    int64_t nb = (n + kScanThreads - 1) / kScanThreads;
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(d_len, n, d_bsum, nullptr);
    k_scan_totals<<<1, kScanThreads, 0, st>>>(d_bsum, nb);
    k_scan_final<<<(unsigned)nb, kScanThreads, 0, st>>>(d_len, n, d_bsum, d_off);
    count_launches(3);
    return ACCEL_OK;
}

size_t accel_marshal_nested_workspace_size(int64_t S, int64_t G) {
    size_t a, b, c;
    const size_t x = ws_layout(S < 0 ? 0 : S, &a, &b, &c), y = ws_layout(G < 0 ? 0 : G, &a, &b, &c);
    return x > y ? x : y;
}

accel_status accel_marshal_nested(const void* const* h_ptrs, const int64_t* h_lengths, int64_t S,
                                  const int64_t* h_group_sizes, int64_t G, int32_t dtype, void* d_flat,
                                  int64_t* d_offsets, int64_t* d_group_offsets, void* d_ws, size_t ws_bytes,
                                  void* stream) {
    ACCEL_REQUIRE(G >= 0 && S >= 0, ACCEL_ERR_INVALID_ARG, "accel_marshal_nested: negative size");
    ACCEL_REQUIRE(d_group_offsets && (G == 0 || h_group_sizes), ACCEL_ERR_INVALID_ARG, "accel_marshal_nested: null pointer");
    ACCEL_REQUIRE(ws_bytes >= accel_marshal_nested_workspace_size(S, G), ACCEL_ERR_WORKSPACE,
                  "accel_marshal_nested: workspace %zu < %zu bytes", ws_bytes, accel_marshal_nested_workspace_size(S, G));
    int64_t total = 0;
    for (int64_t g = 0; g < G; ++g) {
        ACCEL_REQUIRE(h_group_sizes[g] >= 0, ACCEL_ERR_SHAPE, "accel_marshal_nested: group size[%lld] < 0", (long long)g);
        total += h_group_sizes[g];
    }
    ACCEL_REQUIRE(total == S, ACCEL_ERR_SHAPE, "accel_marshal_nested: group sizes sum to %lld, not S=%lld",
                  (long long)total, (long long)S);
    // inner level: the sequences, as accel_marshal_ragged
    accel_status r = accel_marshal_ragged(h_ptrs, h_lengths, S, dtype, d_flat, d_offsets, d_ws, ws_bytes, stream);
    if (r != ACCEL_OK) return r;
    // outer level: group offsets into the sequence offsets (stream order: after the gather)
    cudaStream_t st = as_stream(stream);
    if (G == 0) {
        ACCEL_CUDA_TRY(cudaMemsetAsync(d_group_offsets, 0, sizeof(int64_t), st));
        return after_launch(st, "accel_marshal_nested", 0);
    }
    r = scan_lengths(h_group_sizes, G, d_group_offsets, (char*)d_ws, st);
    if (r != ACCEL_OK) return r;
    return after_launch(st, "accel_marshal_nested", 0);
}

size_t accel_unmarshal_ragged_workspace_size(int64_t S) {
    return align_up(kStatusBytes + (size_t)(S > 0 ? S : 0) * sizeof(void*), 256);
}

accel_status accel_unmarshal_ragged(const void* d_flat, int64_t N, const int64_t* d_offsets, int64_t S, int32_t dtype,
                                    void* const* h_dst_ptrs, void* d_ws, size_t ws_bytes, void* stream) {
    ACCEL_REQUIRE(S >= 0 && N >= 0, ACCEL_ERR_INVALID_ARG, "accel_unmarshal_ragged: negative size");
    ACCEL_REQUIRE(dtype_valid(dtype), ACCEL_ERR_DTYPE, "accel_unmarshal_ragged: bad dtype");
    ACCEL_REQUIRE(d_offsets && d_ws && (S == 0 || (h_dst_ptrs && d_flat)), ACCEL_ERR_INVALID_ARG,
                  "accel_unmarshal_ragged: null pointer");
    ACCEL_REQUIRE(((uintptr_t)d_ws % 256) == 0, ACCEL_ERR_INVALID_ARG, "accel_unmarshal_ragged: d_ws must be 256-byte aligned");
    ACCEL_REQUIRE(ws_bytes >= accel_unmarshal_ragged_workspace_size(S), ACCEL_ERR_WORKSPACE,
                  "accel_unmarshal_ragged: workspace %zu < %zu bytes", ws_bytes, accel_unmarshal_ragged_workspace_size(S));
    if (S == 0) return ok();
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    if (debug_mode()) {
        accel_status r = debug_check_offsets(d_offsets, S, N, 0, ws + 0, st);
        if (r != ACCEL_OK) return r;
    }
    void** d_ptrs = (void**)(ws + kStatusBytes);
    ACCEL_CUDA_TRY(table_to_device(d_ptrs, h_dst_ptrs, (size_t)S * sizeof(void*), st));
    int64_t blocks = (S + 7) / 8;
    int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (dtype_size(dtype) == 4)
        k_scatter<int32_t><<<(unsigned)blocks, 256, 0, st>>>((const int32_t*)d_flat, d_offsets, S, (int32_t* const*)d_ptrs);
    else
        k_scatter<int64_t><<<(unsigned)blocks, 256, 0, st>>>((const int64_t*)d_flat, d_offsets, S, (int64_t* const*)d_ptrs);
    return after_launch(st, "accel_unmarshal_ragged", 1);
}

accel_status accel_marshal_records(void* d_aos, int64_t n, int32_t record_bytes, int32_t nfields,
                                   const int32_t* h_field_offsets, const int32_t* h_field_dtypes, void* const* h_soa,
                                   int32_t inverse, void* stream) {
    ACCEL_REQUIRE(n >= 0 && record_bytes > 0, ACCEL_ERR_INVALID_ARG, "accel_marshal_records: bad size");
    ACCEL_REQUIRE(nfields >= 1 && nfields <= ACCEL_MAX_FIELDS, ACCEL_ERR_INVALID_ARG,
                  "accel_marshal_records: nfields must be 1..%d", ACCEL_MAX_FIELDS);
    ACCEL_REQUIRE(h_field_offsets && h_field_dtypes && h_soa, ACCEL_ERR_INVALID_ARG, "accel_marshal_records: null pointer");
    FieldDesc fd{};
    fd.nfields = nfields;
    fd.record_bytes = record_bytes;
    for (int f = 0; f < nfields; ++f) {
        ACCEL_REQUIRE(dtype_valid(h_field_dtypes[f]), ACCEL_ERR_DTYPE, "accel_marshal_records: bad dtype of field %d", f);
        int sz = (int)dtype_size(h_field_dtypes[f]);
        ACCEL_REQUIRE(h_field_offsets[f] >= 0 && h_field_offsets[f] + sz <= record_bytes, ACCEL_ERR_SHAPE,
                      "accel_marshal_records: field %d outside the record", f);
        ACCEL_REQUIRE(h_field_offsets[f] % sz == 0 && record_bytes % sz == 0, ACCEL_ERR_DTYPE,
                      "accel_marshal_records: field %d not naturally aligned", f);
        ACCEL_REQUIRE(n == 0 || h_soa[f], ACCEL_ERR_INVALID_ARG, "accel_marshal_records: field %d array is null", f);
        fd.off[f] = h_field_offsets[f];
        fd.size[f] = sz;
        fd.soa[f] = h_soa[f];
    }
    if (n == 0) return ok();
    ACCEL_REQUIRE(d_aos, ACCEL_ERR_INVALID_ARG, "accel_marshal_records: d_aos is null");
    cudaStream_t st = as_stream(stream);
    bool fast = record_bytes == 16 && nfields == 4 && ((uintptr_t)d_aos % 16) == 0;
    for (int f = 0; fast && f < 4; ++f) fast = fd.off[f] == 4 * f && fd.size[f] == 4;
    int64_t work = fast ? n : n * nfields;
    int64_t blocks = (work + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (fast) {
        if (inverse) k_records16<true><<<(unsigned)blocks, 256, 0, st>>>((int4*)d_aos, n, fd);
        else k_records16<false><<<(unsigned)blocks, 256, 0, st>>>((int4*)d_aos, n, fd);
    } else {
        if (inverse) k_records<true><<<(unsigned)blocks, 256, 0, st>>>((char*)d_aos, n, fd);
        else k_records<false><<<(unsigned)blocks, 256, 0, st>>>((char*)d_aos, n, fd);
    }
    return after_launch(st, "accel_marshal_records", 1);
}

}  // extern "C"
