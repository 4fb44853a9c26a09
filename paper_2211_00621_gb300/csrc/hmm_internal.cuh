// Internal interfaces shared by the HMM kernels and the hmm_forward / hmm_adjoint entry
// points (not part of the C ABI).
#pragma once
#include "common.cuh"

namespace accel {
namespace hmm {

// Layout of the status block at the start of every HMM workspace.
constexpr size_t kDebugScratchOff = 0;   // 8 bytes for debug-mode checks
constexpr size_t kStatusOff = 8;         // int32 device status (ACCEL_OK or an error code)
constexpr size_t kQueueOff = 16;         // uint64 sequence-queue counter

// Sequence order by decreasing length (approximate: 1024 logarithmic length buckets), so
// that long sequences start first and groups of consecutive sequences have similar
// lengths.  order[q] = sequence index.  Scratch: order_ws_bytes(S) - S*4 bytes after order.
size_t order_ws_bytes(int64_t S);
accel_status order_by_length(const int64_t* d_off, int64_t S, int32_t* d_order, char* scratch, cudaStream_t st);

// FP32 log-space forward (k_hmm_plain.cu).
size_t plain_ws_bytes(int K, int M, int64_t S);
accel_status plain_forward(const accel_hmm_model* m, const int32_t* obs, const int64_t* off, int64_t S,
                           double* loglik, char* ws, int32_t* d_status, cudaStream_t st);

// Launch configuration of the BF16 tensor-core forward, chosen by the autotuner
// (hmm_autotune.cu): column parts per row (2: 8 warps, 4: 16 warps), sequence rows used per
// tile (<= 128; fewer rows spread the sequences over more SMs), and whether a tile runs on
// one CTA (pair = 0) or on a cluster that splits the state columns: two CTAs (pair = 1) or
// four (pair = 2).
struct TcConfig {
    int split;
    int rows;
    int pair;
    int units;      // persistent work units launched (CTAs, or clusters when pair > 0); 0: all that fit
};
bool tc_cl_supported(int K, int M, int rows, int split, int nc);
TcConfig tuned_config(int K, int M, int64_t S);

// BF16 tensor-core scaled forward (k_hmm_tc.cu).
accel_status tc_forward_cfg(const accel_hmm_model* m, const int32_t* obs, const int64_t* off, int64_t S,
                            double* loglik, char* ws, int32_t* d_status, TcConfig cfg, cudaStream_t st);
size_t tc_ws_bytes(int K, int M, int64_t S);
accel_status tc_forward(const accel_hmm_model* m, const int32_t* obs, const int64_t* off, int64_t S,
                        double* loglik, char* ws, int32_t* d_status, cudaStream_t st);
bool tc_supported(int K, int M);

// Tensor-core (TF32, hi/lo split) accumulation of the adjoint's transition and emission
// counts over the row buffers of one backward round (k_xi_tc.cu):
//   Upart[g] += P^T Q over rows [0, *rows_r), and, when cntp is not null,
//   cntp[g][i][k] += sum_rows G[row][i] [osym[row] == k].
// The rows are divided into xi_tc_splits(K) contiguous ranges; clusters of consecutive
// ranges add their sums together, so there are xi_tc_partials(K) partials g.
constexpr int kXiSplitMax = 160;
bool xi_tc_supported(int K);
bool xi_tc_counts_supported(int K, int M);
int xi_tc_splits(int K, int M, bool counts);
int xi_tc_partials(int K, int M, bool counts);   // partials the splits leave (one per cluster)
accel_status xi_tc_round(const float* P, const float* Q, const float* G, const int32_t* osym, const int32_t* rows_r,
                         int K, int M, float* Upart, float* cntp, int32_t* status, cudaStream_t st);

}  // namespace hmm
}  // namespace accel
