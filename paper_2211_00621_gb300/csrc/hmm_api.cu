// hmm_forward entry point: argument checks (debug mode: the paper's runtime checks,
// Sec. 3.2 / Appendix B), workspace sizing and dispatch to the FP32 log-space kernel or
// the BF16 tensor-core kernel.
#include "hmm_internal.cuh"

using namespace accel;
using namespace accel::hmm;

namespace accel {
namespace hmm {

accel_status check_model(const accel_hmm_model* m, const char* who) {
    ACCEL_REQUIRE(m, ACCEL_ERR_INVALID_ARG, "%s: null model", who);
    ACCEL_REQUIRE(m->K >= 1 && m->K <= ACCEL_HMM_MAX_K, ACCEL_ERR_UNSUPPORTED, "%s: K=%d outside [1, %d]", who, m->K, ACCEL_HMM_MAX_K);
    ACCEL_REQUIRE(m->M >= 1 && m->M <= 1024, ACCEL_ERR_UNSUPPORTED, "%s: M=%d outside [1, 1024]", who, m->M);
    ACCEL_REQUIRE(m->log_A && m->log_B && m->log_pi, ACCEL_ERR_INVALID_ARG, "%s: null parameter pointer", who);
    return ACCEL_OK;
}

accel_status read_device_status(const int32_t* d_status, cudaStream_t st) {
    int32_t h = 0;
    ACCEL_CUDA_TRY(cudaMemcpyAsync(&h, d_status, 4, cudaMemcpyDeviceToHost, st));
    ACCEL_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == ACCEL_ERR_TIMEOUT)
        return set_error(h, "device-side status TIMEOUT (a bounded wait gave up or the watchdog budget ran out)");
    if (h != ACCEL_OK) return set_error(h, "device-side status %d", h);
    return ACCEL_OK;
}

}  // namespace hmm
}  // namespace accel

extern "C" {

size_t hmm_forward_workspace_size(const accel_hmm_model* m, int64_t S, int64_t total_T, int32_t precision) {
    (void)total_T;
    if (!m || S < 0) return 0;
    size_t body = precision == ACCEL_HMM_BF16_SCALED ? tc_ws_bytes(m->K, m->M, S)
                                                      : kStatusBytes + plain_ws_bytes(m->K, m->M, S);
    return align_up(body, 256);
}

accel_status hmm_forward(const accel_hmm_model* m, int32_t precision, const int32_t* d_obs, const int64_t* d_offsets,
                         int64_t S, int64_t total_T, double* d_loglik, void* d_ws, size_t ws_bytes, void* stream) {
    accel_status r = check_model(m, "hmm_forward");
    if (r != ACCEL_OK) return r;
    ACCEL_REQUIRE(precision == ACCEL_HMM_FP32_LOG || precision == ACCEL_HMM_BF16_SCALED, ACCEL_ERR_INVALID_ARG,
                  "hmm_forward: bad precision %d", precision);
    ACCEL_REQUIRE(S >= 0 && total_T >= 0, ACCEL_ERR_INVALID_ARG, "hmm_forward: negative size");
    ACCEL_REQUIRE(d_offsets && d_ws && (S == 0 || d_loglik) && (total_T == 0 || d_obs), ACCEL_ERR_INVALID_ARG,
                  "hmm_forward: null pointer");
    ACCEL_REQUIRE(((uintptr_t)d_ws % 256) == 0, ACCEL_ERR_INVALID_ARG, "hmm_forward: d_ws must be 256-byte aligned");
    size_t need = hmm_forward_workspace_size(m, S, total_T, precision);
    ACCEL_REQUIRE(ws_bytes >= need, ACCEL_ERR_WORKSPACE, "hmm_forward: workspace %zu < %zu bytes", ws_bytes, need);
    if (S == 0) return ok();
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    if (debug_mode()) {
        r = debug_check_offsets(d_offsets, S, total_T, 1, ws + kDebugScratchOff, st);
        if (r != ACCEL_OK) return r;
        r = debug_check_symbols(d_obs, total_T, m->M, ws + kDebugScratchOff, st);
        if (r != ACCEL_OK) return r;
    }
    ACCEL_CUDA_TRY(cudaMemsetAsync(ws + kStatusOff, 0, 4, st));
    int32_t* dst = status_word((int32_t*)(ws + kStatusOff));
    if (precision == ACCEL_HMM_FP32_LOG) {
        r = plain_forward(m, d_obs, d_offsets, S, d_loglik, ws + kStatusBytes, dst, st);
    } else {
        r = tc_forward(m, d_obs, d_offsets, S, d_loglik, ws, dst, st);
    }
    if (r != ACCEL_OK) return r;
    if (debug_mode()) return read_device_status(dst, st);
    return ok();
}

}  // extern "C"
