/*
 * accel.h -- C ABI of libaccel, a GB300 (sm_103a) library for the data-parallel hot path
 * of expression acceleration (Expression Acceleration: Seamless Parallelization of Typed
 * High-Level Languages, arXiv 2211.00621).
 *
 * One call = one accelerated expression (Sec. 3.1 "Key Idea": `accelerate e` runs e on the
 * GPU, its free variables passed in).  Arguments arrive already in the backend format or
 * are marshaled by the library (Sec. 3.3 "Marshaling").  There are no function-valued
 * arguments (Sec. 3.4 and Appendix B, rules WF-BC-1/2 forbid higher-order functions in
 * accelerated code), so every pattern takes an operator from a FIXED enumeration.  Tensor
 * elements are integers or floats (Appendix B, WF-TC-Ten) and tensors have rank <= 3
 * (Appendix B, "Dynamic Assumptions": the CUDA backend's maximum rank, default 3).
 *
 * Conventions (all entry points)
 * ------------------------------
 *  - Every call returns accel_status; ACCEL_OK (0) on success.  On failure nothing has
 *    been launched unless the code is ACCEL_ERR_CUDA / ACCEL_ERR_TIMEOUT, and
 *    accel_last_error() returns a message (thread-local, valid until the next call on the
 *    same thread).
 *  - Pointers named d_* are device pointers (or host pointers the device can address, where
 *    stated); h_* are host pointers read before the call returns.  The caller owns ALL
 *    memory: the library never allocates device memory.  Scratch space is passed as
 *    (d_ws, ws_bytes); the matching *_workspace_size() reports how much is needed
 *    (256-byte aligned pointer required).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every call is
 *    asynchronous on that stream unless debug mode is on.
 *  - Debug mode (accel_set_debug(1)) follows the paper's debug mode (Sec. 3.2 "Recommended
 *    Workflow" and Appendix B "Dynamic Assumptions"): arguments are validated on the host
 *    and on the device (offsets monotone and in range, symbols < M, rank <= 3, lengths),
 *    the stream is synchronized after the call and device-side errors are returned as
 *    status codes.  With debug mode off ("accelerate mode") only O(1) host checks run, and
 *    errors that only the device can see (a bounded wait that gave up, a sequence longer
 *    than the max_T a call was sized for) are recorded in a device status word: the
 *    caller's, registered with accel_set_device_status, and read with accel_sync_status.
 *  - Integers are 64-bit wherever the paper's compiler would use its single int type
 *    (Sec. 5: the compiler always uses 64-bit integers): offsets, sizes, integer results of
 *    maps and reductions computed from int32 data.
 */
#ifndef ACCEL_H
#define ACCEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
typedef int32_t accel_status;
#define ACCEL_OK                 0
#define ACCEL_ERR_INVALID_ARG    1  /* null pointer, bad enum, negative size            */
#define ACCEL_ERR_SHAPE          2  /* rank > 3, offsets not monotone, symbol >= M, ... */
#define ACCEL_ERR_DTYPE          3  /* dtype combination not supported by the operator  */
#define ACCEL_ERR_WORKSPACE      4  /* ws_bytes smaller than *_workspace_size()         */
#define ACCEL_ERR_CUDA           5  /* a CUDA runtime call failed                        */
#define ACCEL_ERR_TIMEOUT        6  /* a bounded device-side wait gave up                */
#define ACCEL_ERR_UNSUPPORTED    7  /* size outside the kernels' limits (e.g. K > 256)   */

/* ------------------------------------------------------------------ element types */
#define ACCEL_I32 0
#define ACCEL_I64 1
#define ACCEL_F32 2
#define ACCEL_F64 3

/* ----------------------------------------------------------- fixed operator sets */
/* map / map2 operators g (Appendix A: map f s, map2 f s1 s2).  For integer outputs the
 * arithmetic is int64 narrowed to the output type; for float outputs it is done in the
 * output type.  SCALE multiplies by `scalar`; ADD2/MUL2 are map2 operators.           */
#define ACCEL_MAP_IDENTITY     0  /* g(x) = x          */
#define ACCEL_MAP_SQ_PLUS_ONE  1  /* g(x) = x*x + 1    */
#define ACCEL_MAP_NEG          2  /* g(x) = -x         */
#define ACCEL_MAP_ABS          3  /* g(x) = |x|        */
#define ACCEL_MAP_SCALE        4  /* g(x) = scalar*x   */
#define ACCEL_MAP_ADD2         5  /* g(x,y) = x + y    */
#define ACCEL_MAP_MUL2         6  /* g(x,y) = x * y    */

/* reduce operators f with neutral element ne (Appendix A: reduce f ne s; Appendix B:
 * f must be associative and ne its neutral element).                                  */
#define ACCEL_RED_ADD 0  /* ne = 0                         */
#define ACCEL_RED_MUL 1  /* ne = 1                         */
#define ACCEL_RED_MIN 2  /* ne = max of type / +inf        */
#define ACCEL_RED_MAX 3  /* ne = min of type / -inf        */

/* loop bodies (Appendix A: loop n f calls f i for i in [0,n) in undefined order).     */
#define ACCEL_LOOP_AXPY  0  /* t0[i] = t0[i] + scalar*t1[i]   (Listing 1, axpy)      */
#define ACCEL_LOOP_SCALE 1  /* t0[i] = scalar*t1[i]           (Appendix A, b = 2a)   */

/* all-pairs operators */
#define ACCEL_PAIR_GRAVITY_SOFTENED 0

/* HMM forward precisions */
#define ACCEL_HMM_FP32_LOG    0  /* log-space forward in FP32 SIMT                     */
#define ACCEL_HMM_BF16_SCALED 1  /* scaled forward, BF16 tcgen05 step, FP32 accumulate */

#define ACCEL_MAX_RANK   3
#define ACCEL_MAX_FIELDS 8
#define ACCEL_HMM_MAX_K  256

/* ------------------------------------------------------------------- housekeeping */
const char* accel_version(void);
/* Message of the last failing call on the calling thread ("" if none). */
const char* accel_last_error(void);
/* Debug mode on (1) / off (0); process-wide, default off. */
void accel_set_debug(int32_t on);
int32_t accel_get_debug(void);
/* Number of CUDA kernels this library has launched in the process so far (diagnostic;
 * used to count the launches inside a timed region). */
uint64_t accel_launch_count(void);

/*
 * accel_alu_rate -- measure one arithmetic rate of the running device at its current clocks
 * (a measurement utility with no counterpart in the paper: the denominators of the ALU
 * rooflines reported beside the kernels).  One warm-up launch, then one timed launch
 * (CUDA events) of 4 CTAs x 512 threads per SM, each thread running 8 independent chains of
 * 8 x iters dependent operations:
 *   ACCEL_PROBE_FFMA   FP32 fused multiply-add (counted as 2 flop)
 *   ACCEL_PROBE_FFMA2  packed FP32 FMA on float pairs (4 flop)
 *   ACCEL_PROBE_RSQRT  FP32 reciprocal square root (1 op, the special-function unit)
 *   ACCEL_PROBE_DFMA   FP64 fused multiply-add (2 flop)
 * *h_rate receives operations per second.  d_scratch: device float32 scratch of 2048 x SM
 * count elements (written).  Synchronizes `stream`.  Errors: INVALID_ARG, CUDA.
 */
#define ACCEL_PROBE_FFMA  0
#define ACCEL_PROBE_FFMA2 1
#define ACCEL_PROBE_RSQRT 2
#define ACCEL_PROBE_DFMA  3
accel_status accel_alu_rate(int32_t kind, int64_t iters, float* d_scratch, double* h_rate, void* stream);

/*
 * Device-side status in accelerate mode (the asynchronous counterpart of the paper's
 * debug-mode runtime checks, Sec. 3.2 and Appendix B "Dynamic Assumptions").
 *
 * accel_set_device_status -- register d_status (a caller-owned device int32, set to
 *   ACCEL_OK = 0 by the caller) for the calls made afterwards on the calling thread; NULL
 *   unregisters.  Every call that can detect an error on the device (hmm_forward,
 *   hmm_adjoint; their bounded waits and the adjoint's max_T check) then records it there:
 *   the FIRST error stays (compare-and-swap from ACCEL_OK), later calls do not clear it.
 *   Without a registered word each call keeps its status in its own workspace, where only
 *   debug mode reads it.  Kernels captured into a CUDA graph keep the word they were
 *   captured with.
 * accel_sync_status -- synchronize `stream`, return the word's value as the status of this
 *   call (with a message in accel_last_error()), and set it back to ACCEL_OK when `clear`
 *   is non-zero.  The word holds the errors of every call issued before this one on
 *   `stream` (and of calls on other streams that have completed).
 */
accel_status accel_set_device_status(int32_t* d_status);
accel_status accel_sync_status(int32_t* d_status, int32_t clear, void* stream);

/*
 * accel_set_watchdog_ns -- failure detection for the persistent single-CTA BF16 forward
 * (hmm_forward, ACCEL_HMM_BF16_SCALED, in the tuned configurations that run one CTA per
 * tile): a launch that has run longer than budget_ns stops at its next step boundary, after
 * the step's tensor-core work has completed, and reports ACCEL_ERR_TIMEOUT in its device
 * status word; its log-likelihoods are then incomplete.  0 (the default) means no limit.
 * Process-wide; read by each launch when it is issued (a captured graph keeps the value
 * it was captured with).  The cluster-pair configurations keep only their bounded waits.
 */
void accel_set_watchdog_ns(uint64_t budget_ns);
uint64_t accel_get_watchdog_ns(void);

/*
 * accel_set_sm_budget -- the most SMs the forward recursion of hmm_adjoint /
 * hmm_adjoint_forward may occupy (its persistent CTA-pair launch, K in {64, 128, 256} with
 * planned groups), so that it can run beside another stream's persistent kernel instead of
 * waiting for the whole GPU: the launch takes min(n, #SMs) / 2 pairs, but at least enough to
 * hold every sequence in two groups of 16.  0 (the default) means every SM.  The backward
 * rounds always use every SM.  Results do not depend on it (each sequence's forward
 * arithmetic is the same in any group).  Per host thread; read when a call is issued.
 */
void accel_set_sm_budget(int32_t n_sms);
int32_t accel_get_sm_budget(void);

/* =========================================================== marshaling (Sec. 3.3) */
/*
 * accel_marshal_ragged -- flatten a host list of S sequences (Appendix A `flatten`,
 * Sec. 3.3 marshaling of a [[T]] argument) into the backend format:
 *     d_offsets[0] = 0, d_offsets[s+1] = d_offsets[s] + h_lengths[s]   (int64, S+1)
 *     d_flat[d_offsets[s] + k] = h_ptrs[s][k]                           (k < h_lengths[s])
 *  h_ptrs    host array of S element pointers; each points to device memory or to
 *            page-locked host memory mapped for the device (UVA); may be NULL where the
 *            length is 0.
 *  h_lengths host array of S lengths >= 0 (read on the host too, for checks, in debug
 *            mode only).  When both tables are page-locked (mapped) host memory the kernels
 *            read them in place over the host link, when the stream reaches the call;
 *            otherwise they are copied to the workspace in stream order (a pageable table is
 *            staged before the call returns; pageable tables cannot be captured into a
 *            CUDA graph).  The tables and the pieces must stay unchanged until the stream
 *            has executed the call.
 *  dtype     element type of every sequence (4- or 8-byte).
 *  d_flat    device output, sum(lengths) elements; d_offsets device output, S+1 int64.
 *  d_ws      scratch of accel_marshal_ragged_workspace_size(S) bytes (pointer + length
 *            tables and scan partials).
 * Errors: INVALID_ARG (null/negative), DTYPE, WORKSPACE, CUDA.
 */
size_t accel_marshal_ragged_workspace_size(int64_t S);
accel_status accel_marshal_ragged(const void* const* h_ptrs, const int64_t* h_lengths, int64_t S,
                                  int32_t dtype, void* d_flat, int64_t* d_offsets,
                                  void* d_ws, size_t ws_bytes, void* stream);

/*
 * accel_marshal_nested -- [[[T]]] (App. A `flatten` applied twice; Sec. 3.3): G groups, group
 * g holding h_group_sizes[g] consecutive sequences of the S listed in h_ptrs / h_lengths
 * (as accel_marshal_ragged; sum of the group sizes must equal S, else ACCEL_ERR_SHAPE).
 * Writes d_flat and d_offsets[0..S] exactly as accel_marshal_ragged, and
 * d_group_offsets[0..G] (int64): group g's sequences are [d_group_offsets[g],
 * d_group_offsets[g+1]) of d_offsets.  A reduce of reduces is then two accel_segreduce calls
 * (inner segments by d_offsets, then the inner results by d_group_offsets).  Workspace:
 * accel_marshal_nested_workspace_size(S, G) bytes, 256-byte aligned.  Host tables are copied
 * in stream order as in accel_marshal_ragged; asynchronous on `stream`.
 */
size_t accel_marshal_nested_workspace_size(int64_t S, int64_t G);
accel_status accel_marshal_nested(const void* const* h_ptrs, const int64_t* h_lengths, int64_t S,
                                  const int64_t* h_group_sizes, int64_t G, int32_t dtype, void* d_flat,
                                  int64_t* d_offsets, int64_t* d_group_offsets, void* d_ws, size_t ws_bytes,
                                  void* stream);

/*
 * accel_unmarshal_ragged -- the inverse of accel_marshal_ragged (results converted back to
 * the host representation, Sec. 3.3): sequence s of the flat data (N elements of `dtype`,
 * device), elements [d_offsets[s], d_offsets[s+1]), is copied to h_dst_ptrs[s], a
 * caller-owned buffer with room for that many elements in device memory or in pinned host
 * memory (written by the kernel directly; one warp per sequence).  The pointer table is
 * copied in stream order as in accel_marshal_ragged; the copies are asynchronous on
 * `stream` (synchronize before reading host buffers).  Workspace: accel_unmarshal_ragged_workspace_size(S) bytes, 256-byte aligned.
 * Debug mode checks the offsets (monotone, offsets[S] == N).
 */
size_t accel_unmarshal_ragged_workspace_size(int64_t S);
accel_status accel_unmarshal_ragged(const void* d_flat, int64_t N, const int64_t* d_offsets, int64_t S,
                                    int32_t dtype, void* const* h_dst_ptrs, void* d_ws, size_t ws_bytes,
                                    void* stream);

/*
 * accel_marshal_records -- a sequence of n records {l_i = e_i} (Fig. mexpr-ast) stored as
 * an array of structures of `record_bytes` bytes each, converted to one array per field
 * (structure of arrays) (Sec. 3.3), or back when `inverse` != 0.
 *  d_aos            device, n * record_bytes bytes (input, or output when inverse).
 *  nfields          1..ACCEL_MAX_FIELDS; h_field_offsets[f] byte offset of field f inside
 *                   the record; h_field_dtypes[f] its element type (4- or 8-byte scalar,
 *                   naturally aligned).
 *  h_soa            host array of nfields device pointers, field f is n elements.
 *  With inverse, bytes of d_aos not covered by a field are left untouched.
 * Errors: INVALID_ARG, DTYPE (unaligned field or bad type), SHAPE (field outside record).
 */
accel_status accel_marshal_records(void* d_aos, int64_t n, int32_t record_bytes, int32_t nfields,
                                   const int32_t* h_field_offsets, const int32_t* h_field_dtypes,
                                   void* const* h_soa, int32_t inverse, void* stream);

/* ================================================== map / map2 (Appendix A, Fig. pmexpr) */
/*
 * accel_map -- d_out[k] = g(d_in[k])  or  g(d_in[k], d_in2[k]) for map2 operators, k < n.
 *  d_in2 must be non-NULL exactly for ACCEL_MAP_ADD2 / ACCEL_MAP_MUL2 and has in_dtype.
 *  Integer output: computed in int64, narrowed (two's complement) to out_dtype.
 *  Float output: computed in out_dtype.  Integer input with float output is converted.
 *  Float input with integer output is rejected (DTYPE).
 */
accel_status accel_map(int32_t op, int32_t in_dtype, const void* d_in, const void* d_in2,
                       int32_t out_dtype, void* d_out, int64_t n, double scalar, void* stream);

/* ============================================================ reduce (Appendix A) */
/*
 * accel_reduce -- *d_out = reduce f ne d_in[0..n)  (one element of `dtype`, device).
 *  Deterministic: one CTA for n <= 65,536, else two passes (per-CTA partials in d_ws, then
 *  one combining CTA).
 *  n == 0 gives ne.  Integer results are exact (wrapping), float results depend on the
 *  (fixed) combination order.
 */
size_t accel_reduce_workspace_size(int64_t n, int32_t dtype);
accel_status accel_reduce(int32_t op, int32_t dtype, const void* d_in, int64_t n, void* d_out,
                          void* d_ws, size_t ws_bytes, void* stream);

/*
 * accel_segreduce -- segmented reduce with a fused map, i.e. the nested pattern
 *     map (lam s. reduce f ne (map g s)) over a flattened [[T]] (Appendix A):
 *     d_out[s] = f-fold of g(d_data[k]) over k in [d_offsets[s], d_offsets[s+1]),
 *     ne for an empty segment.
 *  d_data     device, N elements of in_dtype (the flat data of accel_marshal_ragged).
 *  d_offsets  device, S+1 non-decreasing int64, d_offsets[0] = 0, d_offsets[S] = N.
 *  g          fused map (any single-operand ACCEL_MAP_*), applied in out_dtype
 *             (int64 for integer data: Sec. 5); `scalar` is used by ACCEL_MAP_SCALE.
 *  d_out      device, S elements of out_dtype.
 *  d_ws       accel_segreduce_workspace_size(N, S) bytes.
 * Errors: INVALID_ARG, DTYPE, WORKSPACE, SHAPE (debug mode: offsets not monotone / not
 * matching N), CUDA.
 */
size_t accel_segreduce_workspace_size(int64_t N, int64_t S);
accel_status accel_segreduce(int32_t op, int32_t fused_map, int32_t in_dtype, int32_t out_dtype,
                             const void* d_data, int64_t N, const int64_t* d_offsets, int64_t S,
                             double scalar, void* d_out, void* d_ws, size_t ws_bytes, void* stream);

/*
 * accel_segreduce_noalloc -- accel_segreduce for callers that cannot allocate device
 * memory (code that runs where cudaMalloc is unavailable or not allowed: inside an
 * allocator's own hooks, under a host framework that owns every allocation, or in a loop
 * that must never enter the allocator).  The paper has no counterpart: it is a property of
 * this library, not of expression acceleration.  Same arguments and results as
 * accel_segreduce, without (d_ws, ws_bytes): the scratch is a 2 MiB array inside the
 * library, created on each device when the library is loaded there and held until the
 * process exits.
 *  Limit: N <= 178,913,280 flat elements (any element type); larger N returns
 *  ACCEL_ERR_UNSUPPORTED before anything is launched.
 *  Sharing: every call in the process uses the same array; it keeps the last call's
 *  contents, and each call writes every byte it reads before reading it, so nothing needs
 *  clearing between calls.  Calls that overlap on the GPU (other streams, or other host
 *  threads without ordering) race on the array: order them.
 *  Set-up: the first call on a device looks up the array's device address with that device
 *  current and caches it; make that first call before any stream capture begins.  Resetting
 *  the device (cudaDeviceReset) after that first call is not supported: the cached address
 *  would belong to the destroyed context.
 *  The call itself allocates nothing and frees nothing.  Errors are those of accel_segreduce
 *  (messages name this entry point) and UNSUPPORTED for N beyond the limit.
 */
accel_status accel_segreduce_noalloc(int32_t op, int32_t fused_map, int32_t in_dtype, int32_t out_dtype,
                                     const void* d_data, int64_t N, const int64_t* d_offsets, int64_t S,
                                     double scalar, void* d_out, void* stream);

/* ============================================================== loop (Appendix A) */
/* A tensor argument (Tensor[Int] / Tensor[Float], rank <= 3, dense row-major). */
typedef struct accel_tensor {
    void*   data;                 /* device pointer                               */
    int32_t dtype;                /* ACCEL_I32 .. ACCEL_F64                        */
    int32_t rank;                 /* 0..ACCEL_MAX_RANK                             */
    int64_t dims[ACCEL_MAX_RANK]; /* dims[0..rank) used                            */
} accel_tensor;

/*
 * accel_loop -- `loop n f` with a fixed body over tensors args[0] (written) and args[1]
 * (read), both of the same dtype and with >= n elements; i in [0, n) in undefined order.
 *  ACCEL_LOOP_AXPY : t0[i] += scalar * t1[i];   ACCEL_LOOP_SCALE: t0[i] = scalar * t1[i].
 *  Integer tensors use (int64)scalar.
 * Errors: INVALID_ARG (nargs != 2, null), SHAPE (rank > 3 or fewer than n elements),
 * DTYPE (dtypes differ).
 */
accel_status accel_loop(int32_t body, int64_t n, const accel_tensor* args, int32_t nargs,
                        double scalar, void* stream);

/* ====================================================================== HMM */
/* Model parameters, float32 log-probabilities, device memory owned by the caller. */
typedef struct accel_hmm_model {
    int32_t K;             /* states, 1..ACCEL_HMM_MAX_K                                   */
    int32_t M;             /* observation symbols, 1..1024                                 */
    const float* log_A;    /* [K*K] row-major: log P(z_{t+1}=j | z_t=i) at i*K + j          */
    const float* log_B;    /* [K*M] row-major: log P(o_t=k | z_t=j)     at j*M + k          */
    const float* log_pi;   /* [K]:             log P(z_1=j)                                 */
} accel_hmm_model;

/*
 * hmm_forward -- per-sequence log-likelihood logL_s = log P(o_1..o_T_s) of S observation
 * sequences of uneven lengths, by the forward recursion: a map over states j of a reduce
 * over states i inside a sequential loop over t (Appendix A patterns; HMM arithmetic is
 * the textbook forward algorithm, which the paper does not discuss).
 *  precision  ACCEL_HMM_FP32_LOG: log-space recursion in FP32 (max-shifted sum of exp).
 *             ACCEL_HMM_BF16_SCALED: scaled recursion, alpha and A in BF16 on the tensor
 *             cores (tcgen05, FP32 accumulation in TMEM), per-step power-of-two rescaling,
 *             log-scale sum in FP64; one persistent launch for all sequences.
 *  d_obs      device int32 [total_T], symbols in [0, M); d_offsets device int64 [S+1].
 *  d_loglik   device float64 [S].
 *  d_ws       hmm_forward_workspace_size(...) bytes.
 * Every sequence must have length >= 1.  Errors: INVALID_ARG, SHAPE (debug mode: bad
 * offsets, symbol >= M, empty sequence), UNSUPPORTED (K or M beyond the limits of the
 * chosen precision), WORKSPACE, CUDA, TIMEOUT.
 */
size_t hmm_forward_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T,
                                  int32_t precision);
accel_status hmm_forward(const accel_hmm_model* m, int32_t precision, const int32_t* d_obs,
                         const int64_t* d_offsets, int64_t S, int64_t total_T, double* d_loglik,
                         void* d_ws, size_t ws_bytes, void* stream);

/*
 * hmm_adjoint -- gradients of L = sum_s w_s logL_s with respect to the log parameters,
 * treated as free parameters:
 *   d_grad_log_A[i*K+j]  = sum_s w_s sum_{t<T_s} P(z_t=i, z_{t+1}=j | o^s)  (expected transitions)
 *   d_grad_log_B[j*M+k]  = sum_s w_s sum_t P(z_t=j | o^s) [o^s_t = k]      (expected emissions)
 *   d_grad_log_pi[j]     = sum_s w_s P(z_1=j | o^s)
 * computed by a hand-written adjoint of the scaled forward recursion: a forward pass that
 * keeps alpha only every ceil(sqrt(T_s)) steps, then, segment by segment in reverse, a
 * recomputation of alpha from its checkpoint and the backward (beta) recursion.
 *  d_weights  device float64 [S] or NULL (all ones).
 *  d_loglik   device float64 [S] or NULL: the forward's logL_s.
 *  max_T      the largest sequence length (sizes the checkpoint storage; hmm_max_length
 *             computes it on the device).  A sequence longer than the checkpoints allow is
 *             skipped and reported as ACCEL_ERR_SHAPE: returned by the call in debug mode,
 *             else recorded in the device status word (accel_set_device_status).
 *  Outputs are overwritten (not accumulated); d_grad_log_pi may be NULL.
 *  Streams: the work is ordered after what `stream` already holds, and what `stream` enqueues
 *  next runs after it.  On K = 64, 128 or 256 the backward part runs on three streams the
 *  library creates once per host thread and device (the backward and recomputation passes at
 *  the highest stream priority, the count kernels at the lowest).  It forks from `stream`
 *  and joins it again through events, so a capture of `stream` into a CUDA graph takes the
 *  whole call.  Two host threads calling at once each use their own streams.
 */
size_t hmm_adjoint_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T, int64_t max_T);
accel_status hmm_adjoint(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets,
                         int64_t S, int64_t total_T, int64_t max_T, const double* d_weights,
                         double* d_loglik, float* d_grad_log_A, float* d_grad_log_B,
                         float* d_grad_log_pi, void* d_ws, size_t ws_bytes, void* stream);

/*
 * hmm_adjoint_forward / hmm_adjoint_backward -- hmm_adjoint in two calls, for a forward pass
 * whose gradient is taken later (e.g. an autograd function): the forward writes logL_s
 * (d_loglik, may be NULL) and leaves its saved state -- the ceil(sqrt(T_s)) checkpoints of
 * alpha, their exponents, the sequence order and grouping -- in d_ws; the backward then runs
 * the recomputation and the backward recursion from that state and writes the gradients as
 * hmm_adjoint does.  Both calls take the same model, observations, offsets, sizes and
 * workspace (hmm_adjoint_workspace_size bytes), and the model's log parameters must not change
 * in between; the forward does not depend on the weights, and the backward leaves the saved
 * state intact, so one forward may be followed by several backward calls (other weights).
 * Results equal hmm_adjoint's.  Errors as hmm_adjoint.
 */
accel_status hmm_adjoint_forward(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets,
                                 int64_t S, int64_t total_T, int64_t max_T, double* d_loglik, void* d_ws,
                                 size_t ws_bytes, void* stream);
accel_status hmm_adjoint_backward(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets,
                                  int64_t S, int64_t total_T, int64_t max_T, const double* d_weights,
                                  float* d_grad_log_A, float* d_grad_log_B, float* d_grad_log_pi, void* d_ws,
                                  size_t ws_bytes, void* stream);

/*
 * hmm_max_length -- *d_max_T = max_s (d_offsets[s+1] - d_offsets[s]) (device int64, caller
 * owned; 0 when S = 0): the max_T that hmm_adjoint and hmm_forward_long are sized with,
 * computed on the device (one CTA, asynchronous on `stream`) for callers that do not track
 * their sequences' lengths on the host.  Errors: INVALID_ARG.
 */
accel_status hmm_max_length(const int64_t* d_offsets, int64_t S, int64_t* d_max_T, void* stream);

/*
 * hmm_forward_long -- the same per-sequence log-likelihoods as hmm_forward, computed
 * parallel-in-T for few, very long sequences.  The forward recursion is the chain of
 * vector-matrix products alpha_T = (pi o b(o_1)) M_2 ... M_T with M_t = A diag(b(o_t));
 * because matrix products are associative (the reduce pattern of Appendix A applied to the
 * sequential loop of Listing 1), each sequence is cut into chunks whose products are formed
 * in parallel (one K x K x K product per step, FP32, rows rescaled by exact powers of two),
 * then folded into the vector chunk by chunk.  Depth T / chunks instead of T; work K^3 per
 * step instead of K^2.
 *  K <= 64 (UNSUPPORTED otherwise), S <= 65535, every T_s >= 1; max_T >= max_s T_s (it sets
 *  the number of chunks per sequence).  Arguments and layouts as hmm_forward; d_ws
 *  256-byte aligned, at least hmm_forward_long_workspace_size bytes (the chunk products:
 *  16 KB per chunk).  Asynchronous on `stream`.
 */
size_t hmm_forward_long_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T, int64_t max_T);
accel_status hmm_forward_long(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets,
                              int64_t S, int64_t total_T, int64_t max_T, double* d_loglik, void* d_ws,
                              size_t ws_bytes, void* stream);

/*
 * hmm_mstep -- re-estimation after hmm_adjoint (textbook HMM training step; the paper has no
 * HMM; its shape is a map over parameter rows of reductions over the row followed by a map,
 * Appendix A).  Each parameter is a set of probability rows: the K rows of A (over j), the K
 * rows of B (over k) and pi.  Inputs: the model (its log parameters, device) and the
 * gradients of L with respect to log A, log B, log pi read as free parameters, i.e. the
 * expected counts d_grad_log_* that hmm_adjoint writes (device FP32, same layouts as the
 * model; counts must be >= 0 for the M-step).  Outputs (device FP32, same layouts, caller
 * owned; any of the six pointers may be NULL to skip that output):
 *   d_grad_theta_*  gradient with respect to unconstrained row parameters theta with
 *                   P = softmax(theta) along each row, taken at theta = log P:
 *                   g_ij - P_ij sum_j' g_ij'  (each row sums to zero);
 *   d_new_log_*     Baum-Welch M-step: log(g_ij / sum_j' g_ij'); a row whose counts sum to
 *                   zero keeps its log P row.
 * Row reductions in FP64; one warp per row.  Every row of log P needs a finite entry.
 * Asynchronous on `stream`; errors: INVALID_ARG (null model or gradient), UNSUPPORTED (K, M).
 */
accel_status hmm_mstep(const accel_hmm_model* m, const float* d_grad_log_A, const float* d_grad_log_B,
                       const float* d_grad_log_pi, float* d_grad_theta_A, float* d_grad_theta_B,
                       float* d_grad_theta_pi, float* d_new_log_A, float* d_new_log_B,
                       float* d_new_log_pi, void* stream);

/*
 * hmm_autotune -- choose the launch configuration of the BF16 tensor-core forward (column
 * parts per row: 8 or 16 warps; sequence rows per tile: 128, 64 or 32; a tile on one CTA or
 * on a cluster of two or four CTAs that split the state columns) by timing each
 * candidate with CUDA events on these inputs, then the number of persistent work units of
 * the fastest (the fewest of all that fit, 3/4, 1/2, 3/8 and 1/4 of them within 1 % of its
 * time, so that a latency-bound forward leaves SMs free for other streams), and remember the
 * result for (device, K, M, floor(log2 S)); hmm_forward then launches with it.  `cache_path` (may be NULL) names a
 * file of JSON lines: an entry for the same key is reused without timing, a new result is
 * appended.  Arguments as hmm_forward (d_loglik receives the last timed run's result).
 * Synchronizes the stream.  h_best_ms (may be NULL) receives the best time (0 when taken from
 * the cache or when nothing is tunable, e.g. precision ACCEL_HMM_FP32_LOG).
 */
accel_status hmm_autotune(const accel_hmm_model* m, int32_t precision, const int32_t* d_obs,
                          const int64_t* d_offsets, int64_t S, int64_t total_T, double* d_loglik,
                          void* d_ws, size_t ws_bytes, const char* cache_path, float* h_best_ms,
                          void* stream);
/* The configuration hmm_forward(ACCEL_HMM_BF16_SCALED) uses for these sizes: column parts
 * per row, rows per tile, (h_pair, may be NULL) how a tile is split over a thread-block
 * cluster: 0 one CTA, 1 two CTAs, 2 four CTAs (each holding K/2 or K/4 state columns), and
 * (h_units, may be NULL) the persistent work units launched (CTAs or clusters; 0: all that
 * fit). */
accel_status hmm_tuned_config(int32_t K, int32_t M, int64_t S, int32_t* h_split, int32_t* h_rows,
                              int32_t* h_pair, int32_t* h_units);

/*
 * accel_pair_histogram -- all-pairs histogram of angular separations (the two-point angular
 * correlation, tpacf, that Table 1 lists among the paper's workloads): a map over point pairs
 * of a bin lookup, reduced into a histogram.  Points are unit vectors in three float32
 * arrays (device).  A pair's dot product d = (x_i x_j + y_i y_j) + z_i z_j is formed in FP32
 * with every product and sum rounded separately (no fused multiply-add); its bin is the
 * number of edges e_k >= d, for n_edges strictly decreasing float32 edges h_edges (host,
 * read before return; e.g. cosines of increasing angles): bin 0 holds pairs closer than
 * the first edge, bin n_edges those beyond the last.
 *  Self mode (B is A: d_bx == d_ax, d_by == d_ay, d_bz == d_az and NB == NA): the
 *  unordered pairs i < j of A.  Otherwise cross mode: all NA x NB pairs (i in A, j in B).
 *  d_hist  device int64 [n_edges + 1], overwritten.  1 <= n_edges <= 31.
 * Asynchronous on `stream`.  Errors: INVALID_ARG (null, negative, NaN edge), SHAPE (edges
 * not strictly decreasing), UNSUPPORTED (n_edges).
 */
accel_status accel_pair_histogram(const float* d_ax, const float* d_ay, const float* d_az, int64_t NA,
                                  const float* d_bx, const float* d_by, const float* d_bz, int64_t NB,
                                  const float* h_edges, int32_t n_edges, int64_t* d_hist, void* stream);

/* ========================================================================= graphs */
/*
 * Capture a sequence of library calls made on `stream` into an executable CUDA graph and
 * replay it (stream capture; e.g. the persistent batched HMM launch with its preparation
 * kernels).  Between accel_graph_begin and accel_graph_end only asynchronous library calls
 * may be made on the stream (debug mode off), with every buffer allocated beforehand: a
 * replay reuses the captured pointers and sizes.  `stream` must not be the legacy default
 * stream.  The graph owns only host-side CUDA objects; accel_graph_destroy frees them.
 */
typedef struct accel_graph_s* accel_graph;
accel_status accel_graph_begin(void* stream);
accel_status accel_graph_end(void* stream, accel_graph* out);
accel_status accel_graph_launch(accel_graph g, void* stream);
accel_status accel_graph_destroy(accel_graph g);
accel_status accel_graph_node_count(accel_graph g, int64_t* out);

/* =========================================================== all-pairs map-of-reduce */
/*
 * pairwise_mapreduce -- for every body i, a reduce over all bodies j (a map of a reduce,
 * Appendix A; the shape of the paper's tpacf / mri-q workloads, Table 1):
 *   ACCEL_PAIR_GRAVITY_SOFTENED:
 *     a_i = sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2)      (G = 1, FP32)
 *  d_x, d_y, d_z, d_m  device float32 [n] (structure of arrays, e.g. from
 *                      accel_marshal_records); outputs d_ax, d_ay, d_az float32 [n].
 *  eps                 softening length, > 0 and finite with eps^-3 <= FLT_MAX / 4
 *                      (eps >= about 1e-13); otherwise ACCEL_ERR_INVALID_ARG.  The j = i
 *                      term is 0 * m_i eps^-3: it is 0 while m_i eps^-3 is finite in FP32.
 *  Order of the sum (deterministic for a given n on a given device): the j range is split
 *  into P contiguous parts (P in {1, 2, 4, 8}, chosen from n and the device's SM count);
 *  within a part, the j's of each quarter of every 512-body tile are summed by parity, the
 *  two parities added, then the four quarters in order; then the P parts in order.
 *  One kernel launch (a thread-block cluster of P CTAs per 64 bodies).
 */
accel_status pairwise_mapreduce(int32_t op, const float* d_x, const float* d_y, const float* d_z,
                                const float* d_m, int64_t n, float eps, float* d_ax, float* d_ay,
                                float* d_az, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ACCEL_H */
