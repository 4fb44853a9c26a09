// Shared host/device helpers of libaccel: status handling, debug mode, dtype traits,
// device properties.  Every kernel file includes this; the C ABI is declared in accel.h.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <climits>
#include <cfloat>

#include "../../include/accel.h"

namespace accel {

// ----------------------------------------------------------------- status / errors
accel_status set_error(accel_status st, const char* fmt, ...);
accel_status ok();
bool debug_mode();

#define ACCEL_CUDA_TRY(expr)                                                          \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess)                                                        \
            return ::accel::set_error(ACCEL_ERR_CUDA, "%s: %s (%s:%d)", #expr,        \
                                      cudaGetErrorString(_e), __FILE__, __LINE__);    \
    } while (0)

#define ACCEL_REQUIRE(cond, st, ...)                                                  \
    do {                                                                              \
        if (!(cond)) return ::accel::set_error((st), __VA_ARGS__);                   \
    } while (0)

// After the launches of one call: count them (accel_launch_count), report launch errors,
// and in debug mode synchronize the stream so asynchronous faults surface as
// ACCEL_ERR_CUDA from the call that caused them.
accel_status after_launch(cudaStream_t stream, const char* what, int nkernels);
void count_launches(int n);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------------------- device properties
int num_sms();             // SM count of the current device
int max_smem_optin();      // max dynamic shared memory per block (opt-in)

// ----------------------------------------------------------------- dtypes
inline bool dtype_valid(int32_t d) { return d >= ACCEL_I32 && d <= ACCEL_F64; }
inline bool dtype_is_int(int32_t d) { return d == ACCEL_I32 || d == ACCEL_I64; }
inline size_t dtype_size(int32_t d) { return (d == ACCEL_I32 || d == ACCEL_F32) ? 4 : 8; }

template <int32_t D> struct dtype_of;
template <> struct dtype_of<ACCEL_I32> { using type = int32_t; };
template <> struct dtype_of<ACCEL_I64> { using type = int64_t; };
template <> struct dtype_of<ACCEL_F32> { using type = float; };
template <> struct dtype_of<ACCEL_F64> { using type = double; };

// Computation type of a map/reduce whose result has type T: int64 for integers (the
// paper's single 64-bit integer type), the float type itself otherwise.
template <typename T> struct compute_of { using type = T; };
template <> struct compute_of<int32_t> { using type = int64_t; };

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ----------------------------------------------------------------- device helpers
template <typename T> __host__ __device__ inline T red_neutral(int op);
template <> __host__ __device__ inline int64_t red_neutral<int64_t>(int op) {
    return op == ACCEL_RED_ADD ? 0 : op == ACCEL_RED_MUL ? 1 : op == ACCEL_RED_MIN ? LLONG_MAX : LLONG_MIN;
}
template <> __host__ __device__ inline int32_t red_neutral<int32_t>(int op) {
    return op == ACCEL_RED_ADD ? 0 : op == ACCEL_RED_MUL ? 1 : op == ACCEL_RED_MIN ? INT_MAX : INT_MIN;
}
template <> __host__ __device__ inline float red_neutral<float>(int op) {
    return op == ACCEL_RED_ADD ? 0.f : op == ACCEL_RED_MUL ? 1.f : op == ACCEL_RED_MIN ? __builtin_huge_valf() : -__builtin_huge_valf();
}
template <> __host__ __device__ inline double red_neutral<double>(int op) {
    return op == ACCEL_RED_ADD ? 0.0 : op == ACCEL_RED_MUL ? 1.0 : op == ACCEL_RED_MIN ? __builtin_huge_val() : -__builtin_huge_val();
}

// Integer add/mul wrap (two's complement) via unsigned arithmetic.
template <typename T> __device__ __forceinline__ T wrap_add(T a, T b) { return a + b; }
template <> __device__ __forceinline__ int64_t wrap_add<int64_t>(int64_t a, int64_t b) {
    return (int64_t)((uint64_t)a + (uint64_t)b);
}
template <> __device__ __forceinline__ int32_t wrap_add<int32_t>(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a + (uint32_t)b);
}
template <typename T> __device__ __forceinline__ T wrap_mul(T a, T b) { return a * b; }
template <> __device__ __forceinline__ int64_t wrap_mul<int64_t>(int64_t a, int64_t b) {
    return (int64_t)((uint64_t)a * (uint64_t)b);
}
template <> __device__ __forceinline__ int32_t wrap_mul<int32_t>(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a * (uint32_t)b);
}

template <int OP, typename T> __device__ __forceinline__ T red_combine(T a, T b) {
    if constexpr (OP == ACCEL_RED_ADD) return wrap_add<T>(a, b);
    else if constexpr (OP == ACCEL_RED_MUL) return wrap_mul<T>(a, b);
    else if constexpr (OP == ACCEL_RED_MIN) return b < a ? b : a;
    else return b > a ? b : a;
}

// Map operators applied in computation type C (see accel.h for the definitions).
template <int OP, typename C> __device__ __forceinline__ C map_apply(C x, C y, C s) {
    if constexpr (OP == ACCEL_MAP_IDENTITY) return x;
    else if constexpr (OP == ACCEL_MAP_SQ_PLUS_ONE) return wrap_add<C>(wrap_mul<C>(x, x), C(1));
    else if constexpr (OP == ACCEL_MAP_NEG) return C(0) - x;
    else if constexpr (OP == ACCEL_MAP_ABS) return x < C(0) ? C(0) - x : x;
    else if constexpr (OP == ACCEL_MAP_SCALE) return wrap_mul<C>(s, x);
    else if constexpr (OP == ACCEL_MAP_ADD2) return wrap_add<C>(x, y);
    else return wrap_mul<C>(x, y);
}

// Dispatch a runtime operator id onto a template parameter.
#define ACCEL_DISPATCH_RED(op, OPC, ...)                                              \
    switch (op) {                                                                     \
        case ACCEL_RED_ADD: { constexpr int OPC = ACCEL_RED_ADD; __VA_ARGS__; } break; \
        case ACCEL_RED_MUL: { constexpr int OPC = ACCEL_RED_MUL; __VA_ARGS__; } break; \
        case ACCEL_RED_MIN: { constexpr int OPC = ACCEL_RED_MIN; __VA_ARGS__; } break; \
        default:            { constexpr int OPC = ACCEL_RED_MAX; __VA_ARGS__; } break; \
    }

#define ACCEL_DISPATCH_MAP1(op, OPC, ...)                                                         \
    switch (op) {                                                                                 \
        case ACCEL_MAP_IDENTITY:    { constexpr int OPC = ACCEL_MAP_IDENTITY; __VA_ARGS__; } break;    \
        case ACCEL_MAP_SQ_PLUS_ONE: { constexpr int OPC = ACCEL_MAP_SQ_PLUS_ONE; __VA_ARGS__; } break; \
        case ACCEL_MAP_NEG:         { constexpr int OPC = ACCEL_MAP_NEG; __VA_ARGS__; } break;         \
        case ACCEL_MAP_ABS:         { constexpr int OPC = ACCEL_MAP_ABS; __VA_ARGS__; } break;         \
        default:                    { constexpr int OPC = ACCEL_MAP_SCALE; __VA_ARGS__; } break;       \
    }

#define ACCEL_DISPATCH_DTYPE(dt, T, ...)                                              \
    switch (dt) {                                                                     \
        case ACCEL_I32: { using T = int32_t; __VA_ARGS__; } break;                    \
        case ACCEL_I64: { using T = int64_t; __VA_ARGS__; } break;                    \
        case ACCEL_F32: { using T = float; __VA_ARGS__; } break;                      \
        default:        { using T = double; __VA_ARGS__; } break;                     \
    }

// Debug-mode check of an offsets array on the device: offsets[0] == 0, non-decreasing,
// offsets[S] == N, and (if min_len > 0) every segment at least min_len long.  Returns
// ACCEL_ERR_SHAPE with a message naming the first bad index.  d_scratch is 16 bytes of
// the caller's workspace.  Synchronizes the stream.
accel_status debug_check_offsets(const int64_t* d_offsets, int64_t S, int64_t N, int64_t min_len,
                                 void* d_scratch, cudaStream_t stream);

// Debug-mode check that every int32 symbol in d_obs[0..n) lies in [0, M).
accel_status debug_check_symbols(const int32_t* d_obs, int64_t n, int32_t M, void* d_scratch,
                                 cudaStream_t stream);

// Bytes every workspace reserves at its start for debug / device status words.
constexpr size_t kStatusBytes = 256;

// Device status word of a call made on this thread: the word the caller registered with
// accel_set_device_status, or `fallback` (the call's own word in its workspace) if none.
int32_t* status_word(int32_t* fallback);
// Watchdog budget of the persistent single-CTA BF16 forward (accel_set_watchdog_ns; 0 = off).
uint64_t watchdog_ns();
// SM budget of the adjoint's forward recursion on this host thread (accel_set_sm_budget; 0 = all).
int32_t sm_budget();

// Record a device-side error: the first error stays (compare-and-swap from ACCEL_OK), so a
// word shared by several calls keeps the earliest failure until the caller clears it.
__device__ __forceinline__ void report_status(int32_t* word, int32_t code) { atomicCAS(word, ACCEL_OK, code); }

}  // namespace accel
