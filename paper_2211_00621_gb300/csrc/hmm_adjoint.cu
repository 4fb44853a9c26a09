// hmm_adjoint entry point (K9).
#include "hmm_internal.cuh"

using namespace accel;

extern "C" {

size_t hmm_adjoint_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T, int64_t max_T) {
    (void)m; (void)S; (void)total_T; (void)max_T;
    return kStatusBytes;
}

accel_status hmm_adjoint(const accel_hmm_model* m, const int32_t* d_obs, const int64_t* d_offsets, int64_t S,
                         int64_t total_T, int64_t max_T, const double* d_weights, double* d_loglik,
                         float* d_grad_log_A, float* d_grad_log_B, float* d_grad_log_pi, void* d_ws, size_t ws_bytes,
                         void* stream) {
    (void)m; (void)d_obs; (void)d_offsets; (void)S; (void)total_T; (void)max_T; (void)d_weights; (void)d_loglik;
    (void)d_grad_log_A; (void)d_grad_log_B; (void)d_grad_log_pi; (void)d_ws; (void)ws_bytes; (void)stream;
    return set_error(ACCEL_ERR_UNSUPPORTED, "hmm_adjoint: not built yet");
}

}  // extern "C"
