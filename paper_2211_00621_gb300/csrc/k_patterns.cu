// map / map2 (K3), loop (K6) and reduce (K4): the flat parallel patterns of Appendix A,
// Fig. "pmexpr-extension".  All three are HBM-streaming kernels: grid-stride loops over
// 16-byte vectors with several independent vectors in flight per thread, grids sized as
// a multiple of the SM count.
#include "common.cuh"

namespace accel {

constexpr int kThreads = 256;

template <typename T, int N> struct alignas(16) vec { T v[N]; };

template <typename Tin> constexpr int vec_of() { return 16 / (int)sizeof(Tin); }

static int grid_for(int64_t work_items, int per_block) {
    int64_t b = (work_items + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms() * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------------------- map
// out[k] = g(in[k] [, in2[k]]) computed in C (int64 for integer results).
template <typename Tin, typename Tout, int OP, bool BIN>
__global__ void __launch_bounds__(kThreads)
k_map(const Tin* __restrict__ in, const Tin* __restrict__ in2, Tout* __restrict__ out, int64_t n,
      double scalar, bool vec_ok) {
    using C = typename compute_of<Tout>::type;
    const C s = (C)scalar;
    constexpr int V = vec_of<Tin>();
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec_ok) {
        int64_t nv = n / V;
        const vec<Tin, V>* vin = reinterpret_cast<const vec<Tin, V>*>(in);
        const vec<Tin, V>* vin2 = reinterpret_cast<const vec<Tin, V>*>(in2);
        for (int64_t i = tid; i < nv; i += nthreads) {
            vec<Tin, V> a = vin[i];
            vec<Tin, V> b;
            if constexpr (BIN) b = vin2[i];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                C y = BIN ? (C)b.v[e] : C(0);
                out[i * V + e] = (Tout)map_apply<OP, C>((C)a.v[e], y, s);
            }
        }
        done = nv * V;
    }
    for (int64_t i = done + tid; i < n; i += nthreads) {
        C y = BIN ? (C)in2[i] : C(0);
        out[i] = (Tout)map_apply<OP, C>((C)in[i], y, s);
    }
}

template <typename Tin, typename Tout>
static accel_status launch_map(int32_t op, const void* in, const void* in2, void* out, int64_t n,
                               double scalar, cudaStream_t st) {
    constexpr int V = vec_of<Tin>();
    bool vec_ok = ((uintptr_t)in % 16 == 0) && (in2 == nullptr || (uintptr_t)in2 % 16 == 0);
    int grid = grid_for(n / V + 1, kThreads);
    const Tin* a = (const Tin*)in;
    const Tin* b = (const Tin*)in2;
    Tout* o = (Tout*)out;
    switch (op) {
        case ACCEL_MAP_ADD2: k_map<Tin, Tout, ACCEL_MAP_ADD2, true><<<grid, kThreads, 0, st>>>(a, b, o, n, scalar, vec_ok); break;
        case ACCEL_MAP_MUL2: k_map<Tin, Tout, ACCEL_MAP_MUL2, true><<<grid, kThreads, 0, st>>>(a, b, o, n, scalar, vec_ok); break;
        default: ACCEL_DISPATCH_MAP1(op, OPC, (k_map<Tin, Tout, OPC, false><<<grid, kThreads, 0, st>>>(a, nullptr, o, n, scalar, vec_ok)));
    }
    return after_launch(st, "accel_map", 1);
}

// ------------------------------------------------------------------------ loop
template <typename T, int BODY>
__global__ void __launch_bounds__(kThreads)
k_loop(T* __restrict__ t0, const T* __restrict__ t1, int64_t n, double scalar) {
    using C = typename compute_of<T>::type;
    const C c = (C)scalar;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        C y = (C)t1[i];
        if constexpr (BODY == ACCEL_LOOP_AXPY) t0[i] = (T)wrap_add<C>((C)t0[i], wrap_mul<C>(c, y));
        else t0[i] = (T)wrap_mul<C>(c, y);
    }
}

// ---------------------------------------------------------------------- reduce
template <int OP, typename C>
__device__ __forceinline__ C block_reduce(C v, C* smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = red_combine<OP, C>(v, __shfl_down_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        v = l < nw ? smem[l] : red_neutral<C>(OP);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = red_combine<OP, C>(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;  // valid in thread 0
}

// Pass 1: per-CTA partial of a contiguous grid-stride share, written to partials[blockIdx].
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads)
k_reduce_partial(const T* __restrict__ in, int64_t n, typename compute_of<T>::type* __restrict__ partials) {
    using C = typename compute_of<T>::type;
    __shared__ C smem[kThreads / 32];
    C acc = red_neutral<C>(OP);
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // four independent loads in flight per thread
    for (; i + 3 * stride < n; i += 4 * stride) {
        T a = in[i], b = in[i + stride], c = in[i + 2 * stride], d = in[i + 3 * stride];
        acc = red_combine<OP, C>(acc, red_combine<OP, C>(red_combine<OP, C>((C)a, (C)b), red_combine<OP, C>((C)c, (C)d)));
    }
    for (; i < n; i += stride) acc = red_combine<OP, C>(acc, (C)in[i]);
    acc = block_reduce<OP, C>(acc, smem);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Pass 2: one CTA combines the partials in index order.  The int64 result of an int32
// reduction is narrowed; an empty reduction gives the neutral element of T itself (for an
// int32 max, INT32_MIN -- not the narrowed int64 neutral element).
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads)
k_reduce_final(const typename compute_of<T>::type* __restrict__ partials, int nparts, int64_t n, T* __restrict__ out) {
    using C = typename compute_of<T>::type;
    __shared__ C smem[kThreads / 32];
    C acc = red_neutral<C>(OP);
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc = red_combine<OP, C>(acc, partials[i]);
    acc = block_reduce<OP, C>(acc, smem);
    if (threadIdx.x == 0) *out = n == 0 ? red_neutral<T>(OP) : (T)acc;
}

// Small inputs (n <= kReduceOne): one CTA reduces everything (one launch instead of two);
// the same fixed combination order on every call.
constexpr int64_t kReduceOne = 1 << 16;
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) k_reduce_one(const T* __restrict__ in, int64_t n, T* __restrict__ out) {
    using C = typename compute_of<T>::type;
    __shared__ C smem[kThreads / 32];
    C acc = red_neutral<C>(OP);
    for (int64_t i = threadIdx.x; i < n; i += kThreads) acc = red_combine<OP, C>(acc, (C)in[i]);
    acc = block_reduce<OP, C>(acc, smem);
    if (threadIdx.x == 0) *out = n == 0 ? red_neutral<T>(OP) : (T)acc;
}

static int reduce_grid(int64_t n) {
    int g = grid_for(n / 4 + 1, kThreads);
    return g > 1024 ? 1024 : g;
}

}  // namespace accel

using namespace accel;

extern "C" {

accel_status accel_map(int32_t op, int32_t in_dtype, const void* d_in, const void* d_in2, int32_t out_dtype,
                       void* d_out, int64_t n, double scalar, void* stream) {
    ACCEL_REQUIRE(op >= ACCEL_MAP_IDENTITY && op <= ACCEL_MAP_MUL2, ACCEL_ERR_INVALID_ARG, "accel_map: bad op %d", op);
    ACCEL_REQUIRE(dtype_valid(in_dtype) && dtype_valid(out_dtype), ACCEL_ERR_DTYPE, "accel_map: bad dtype");
    ACCEL_REQUIRE(n >= 0, ACCEL_ERR_INVALID_ARG, "accel_map: n < 0");
    bool bin = op == ACCEL_MAP_ADD2 || op == ACCEL_MAP_MUL2;
    ACCEL_REQUIRE(bin == (d_in2 != nullptr), ACCEL_ERR_INVALID_ARG, "accel_map: d_in2 must be given exactly for map2 operators");
    ACCEL_REQUIRE(!(dtype_is_int(out_dtype) && !dtype_is_int(in_dtype)), ACCEL_ERR_DTYPE, "accel_map: float input with integer output");
    if (n == 0) return ok();
    ACCEL_REQUIRE(d_in && d_out, ACCEL_ERR_INVALID_ARG, "accel_map: null pointer");
    cudaStream_t st = as_stream(stream);
    accel_status r = ACCEL_OK;
    ACCEL_DISPATCH_DTYPE(in_dtype, Tin, ACCEL_DISPATCH_DTYPE(out_dtype, Tout, (r = launch_map<Tin, Tout>(op, d_in, d_in2, d_out, n, scalar, st))));
    return r;
}

accel_status accel_loop(int32_t body, int64_t n, const accel_tensor* args, int32_t nargs, double scalar, void* stream) {
    ACCEL_REQUIRE(body == ACCEL_LOOP_AXPY || body == ACCEL_LOOP_SCALE, ACCEL_ERR_INVALID_ARG, "accel_loop: bad body %d", body);
    ACCEL_REQUIRE(args && nargs == 2, ACCEL_ERR_INVALID_ARG, "accel_loop: need exactly 2 tensor arguments");
    ACCEL_REQUIRE(n >= 0, ACCEL_ERR_INVALID_ARG, "accel_loop: n < 0");
    for (int a = 0; a < 2; ++a) {
        ACCEL_REQUIRE(args[a].rank >= 0 && args[a].rank <= ACCEL_MAX_RANK, ACCEL_ERR_SHAPE,
                      "accel_loop: tensor %d has rank %d > %d", a, args[a].rank, ACCEL_MAX_RANK);
        ACCEL_REQUIRE(dtype_valid(args[a].dtype), ACCEL_ERR_DTYPE, "accel_loop: bad dtype");
        int64_t numel = 1;
        for (int d = 0; d < args[a].rank; ++d) {
            ACCEL_REQUIRE(args[a].dims[d] >= 0, ACCEL_ERR_SHAPE, "accel_loop: negative dim");
            numel *= args[a].dims[d];
        }
        ACCEL_REQUIRE(numel >= n, ACCEL_ERR_SHAPE, "accel_loop: tensor %d has %lld < n elements", a, (long long)numel);
        ACCEL_REQUIRE(n == 0 || args[a].data, ACCEL_ERR_INVALID_ARG, "accel_loop: null tensor");
    }
    ACCEL_REQUIRE(args[0].dtype == args[1].dtype, ACCEL_ERR_DTYPE, "accel_loop: dtypes differ");
    if (n == 0) return ok();
    cudaStream_t st = as_stream(stream);
    int grid = grid_for(n, kThreads * 4);
    ACCEL_DISPATCH_DTYPE(args[0].dtype, T,
        if (body == ACCEL_LOOP_AXPY) k_loop<T, ACCEL_LOOP_AXPY><<<grid, kThreads, 0, st>>>((T*)args[0].data, (const T*)args[1].data, n, scalar);
        else k_loop<T, ACCEL_LOOP_SCALE><<<grid, kThreads, 0, st>>>((T*)args[0].data, (const T*)args[1].data, n, scalar));
    return after_launch(st, "accel_loop", 1);
}

size_t accel_reduce_workspace_size(int64_t n, int32_t dtype) {
    (void)n; (void)dtype;
    return kStatusBytes + 1024 * sizeof(int64_t);
}

accel_status accel_reduce(int32_t op, int32_t dtype, const void* d_in, int64_t n, void* d_out, void* d_ws,
                          size_t ws_bytes, void* stream) {
    ACCEL_REQUIRE(op >= ACCEL_RED_ADD && op <= ACCEL_RED_MAX, ACCEL_ERR_INVALID_ARG, "accel_reduce: bad op %d", op);
    ACCEL_REQUIRE(dtype_valid(dtype), ACCEL_ERR_DTYPE, "accel_reduce: bad dtype");
    ACCEL_REQUIRE(n >= 0 && d_out && d_ws && (n == 0 || d_in), ACCEL_ERR_INVALID_ARG, "accel_reduce: bad pointer or size");
    ACCEL_REQUIRE(ws_bytes >= accel_reduce_workspace_size(n, dtype), ACCEL_ERR_WORKSPACE, "accel_reduce: workspace too small");
    cudaStream_t st = as_stream(stream);
    if (n <= kReduceOne) {
        ACCEL_DISPATCH_DTYPE(dtype, T, ACCEL_DISPATCH_RED(op, OPC, {
            k_reduce_one<T, OPC><<<1, kThreads, 0, st>>>((const T*)d_in, n, (T*)d_out);
        }));
        return after_launch(st, "accel_reduce", 1);
    }
    int grid = reduce_grid(n);
    void* partials = (char*)d_ws + kStatusBytes;
    ACCEL_DISPATCH_DTYPE(dtype, T, ACCEL_DISPATCH_RED(op, OPC, {
        using C = typename compute_of<T>::type;
        k_reduce_partial<T, OPC><<<grid, kThreads, 0, st>>>((const T*)d_in, n, (C*)partials);
        k_reduce_final<T, OPC><<<1, kThreads, 0, st>>>((const C*)partials, grid, n, (T*)d_out);
    }));
    return after_launch(st, "accel_reduce", 2);
}

}  // extern "C"
