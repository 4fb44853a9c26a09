// Housekeeping entry points of the C ABI (version, last error, debug mode) and the
// debug-mode validation kernels that stand in for the paper's debug-mode runtime checks
// (Sec. 3.2 "Recommended Workflow"; Appendix B "Dynamic Assumptions").
#include "common.cuh"

#include <atomic>
#include <string>

namespace accel {

static thread_local char g_last_error[512] = {0};
static std::atomic<int> g_debug{0};
static std::atomic<unsigned long long> g_launches{0};
static thread_local int32_t* g_status_word = nullptr;     // accel_set_device_status
static std::atomic<unsigned long long> g_watchdog_ns{0};  // accel_set_watchdog_ns

int32_t* status_word(int32_t* fallback) { return g_status_word ? g_status_word : fallback; }
uint64_t watchdog_ns() { return g_watchdog_ns.load(std::memory_order_relaxed); }
static thread_local int32_t g_sm_budget = 0;                 // accel_set_sm_budget
int32_t sm_budget() { return g_sm_budget; }

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

accel_status set_error(accel_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

accel_status ok() {
    g_last_error[0] = 0;
    return ACCEL_OK;
}

bool debug_mode() { return g_debug.load(std::memory_order_relaxed) != 0; }

accel_status after_launch(cudaStream_t stream, const char* what, int nkernels) {
    count_launches(nkernels);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ACCEL_ERR_CUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    if (debug_mode()) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return set_error(ACCEL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    return ok();
}

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int max_smem_optin() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return n;
}

// ------------------------------------------------------------- debug-mode validation
// d_bad[0] receives the smallest offending index (INT64_MAX when none).
__global__ void k_check_offsets(const int64_t* __restrict__ off, int64_t S, int64_t N, int64_t min_len,
                                unsigned long long* d_bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i <= S; i += stride) {
        bool bad = false;
        if (i == 0) bad = off[0] != 0;
        else bad = off[i] < off[i - 1] + min_len;
        if (i == S) bad = bad || off[S] != N;
        if (bad) atomicMin(d_bad, (unsigned long long)i);
    }
}

__global__ void k_check_symbols(const int32_t* __restrict__ obs, int64_t n, int32_t M,
                                unsigned long long* d_bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride)
        if (obs[i] < 0 || obs[i] >= M) atomicMin(d_bad, (unsigned long long)i);
}

static accel_status read_bad(void* d_scratch, cudaStream_t stream, unsigned long long* bad) {
    ACCEL_CUDA_TRY(cudaMemcpyAsync(bad, d_scratch, sizeof(*bad), cudaMemcpyDeviceToHost, stream));
    ACCEL_CUDA_TRY(cudaStreamSynchronize(stream));
    return ACCEL_OK;
}

accel_status debug_check_offsets(const int64_t* d_offsets, int64_t S, int64_t N, int64_t min_len,
                                 void* d_scratch, cudaStream_t stream) {
    ACCEL_CUDA_TRY(cudaMemsetAsync(d_scratch, 0xff, 8, stream));
    int blocks = (int)((S + 1 + 255) / 256);
    if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
    k_check_offsets<<<blocks, 256, 0, stream>>>(d_offsets, S, N, min_len, (unsigned long long*)d_scratch);
    count_launches(1);
    ACCEL_CUDA_TRY(cudaGetLastError());
    unsigned long long bad = 0;
    accel_status st = read_bad(d_scratch, stream, &bad);
    if (st != ACCEL_OK) return st;
    if (bad != ~0ull)
        return set_error(ACCEL_ERR_SHAPE,
                         "debug: offsets invalid at index %llu (need offsets[0]=0, offsets[s+1]-offsets[s] >= %lld, offsets[S]=N=%lld)",
                         bad, (long long)min_len, (long long)N);
    return ACCEL_OK;
}

accel_status debug_check_symbols(const int32_t* d_obs, int64_t n, int32_t M, void* d_scratch,
                                 cudaStream_t stream) {
    if (n == 0) return ACCEL_OK;
    ACCEL_CUDA_TRY(cudaMemsetAsync(d_scratch, 0xff, 8, stream));
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
    k_check_symbols<<<blocks, 256, 0, stream>>>(d_obs, n, M, (unsigned long long*)d_scratch);
    count_launches(1);
    ACCEL_CUDA_TRY(cudaGetLastError());
    unsigned long long bad = 0;
    accel_status st = read_bad(d_scratch, stream, &bad);
    if (st != ACCEL_OK) return st;
    if (bad != ~0ull) return set_error(ACCEL_ERR_SHAPE, "debug: symbol at index %llu outside [0, %d)", bad, M);
    return ACCEL_OK;
}

}  // namespace accel

extern "C" {

const char* accel_version(void) { return "libaccel 0.1 (sm_103a)"; }
const char* accel_last_error(void) { return accel::g_last_error; }
void accel_set_debug(int32_t on) { accel::g_debug.store(on ? 1 : 0); }
int32_t accel_get_debug(void) { return accel::g_debug.load(); }
uint64_t accel_launch_count(void) { return accel::g_launches.load(); }

accel_status accel_set_device_status(int32_t* d_status) {
    accel::g_status_word = d_status;
    return accel::ok();
}

accel_status accel_sync_status(int32_t* d_status, int32_t clear, void* stream) {
    using namespace accel;
    ACCEL_REQUIRE(d_status != nullptr, ACCEL_ERR_INVALID_ARG, "accel_sync_status: null status word");
    cudaStream_t st = as_stream(stream);
    int32_t h = 0;
    ACCEL_CUDA_TRY(cudaMemcpyAsync(&h, d_status, 4, cudaMemcpyDeviceToHost, st));
    if (clear) ACCEL_CUDA_TRY(cudaMemsetAsync(d_status, 0, 4, st));
    ACCEL_CUDA_TRY(cudaStreamSynchronize(st));
    switch (h) {
        case ACCEL_OK: return ok();
        case ACCEL_ERR_TIMEOUT:
            return set_error(h, "device-side status: TIMEOUT (a bounded wait gave up or the watchdog budget ran out)");
        case ACCEL_ERR_SHAPE:
            return set_error(h, "device-side status: SHAPE (a sequence longer than the max_T the call was sized for)");
        default: return set_error(h, "device-side status %d", h);
    }
}

void accel_set_watchdog_ns(uint64_t budget_ns) { accel::g_watchdog_ns.store(budget_ns); }
uint64_t accel_get_watchdog_ns(void) { return accel::g_watchdog_ns.load(); }
void accel_set_sm_budget(int32_t n_sms) { accel::g_sm_budget = n_sms < 0 ? 0 : n_sms; }
int32_t accel_get_sm_budget(void) { return accel::g_sm_budget; }

}  // extern "C"

// ------------------------------------------------------------------ CUDA graphs
// A captured sequence of library calls (stream capture -> instantiated executable graph).
struct accel_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

accel_status accel_graph_begin(void* stream) {
    using namespace accel;
    ACCEL_REQUIRE(stream != nullptr, ACCEL_ERR_INVALID_ARG, "accel_graph_begin: capture needs a non-default stream");
    ACCEL_REQUIRE(!debug_mode(), ACCEL_ERR_INVALID_ARG, "accel_graph_begin: debug mode synchronizes and cannot be captured");
    ACCEL_CUDA_TRY(cudaStreamBeginCapture(as_stream(stream), cudaStreamCaptureModeRelaxed));
    return ok();
}

accel_status accel_graph_end(void* stream, accel_graph* out) {
    using namespace accel;
    ACCEL_REQUIRE(stream != nullptr && out != nullptr, ACCEL_ERR_INVALID_ARG, "accel_graph_end: null argument");
    cudaGraph_t g = nullptr;
    ACCEL_CUDA_TRY(cudaStreamEndCapture(as_stream(stream), &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_error(ACCEL_ERR_CUDA, "accel_graph_end: instantiate failed: %s", cudaGetErrorString(e));
    }
    accel_graph_s* h = new accel_graph_s{g, ex};
    *out = h;
    return ok();
}

accel_status accel_graph_launch(accel_graph g, void* stream) {
    using namespace accel;
    ACCEL_REQUIRE(g != nullptr, ACCEL_ERR_INVALID_ARG, "accel_graph_launch: null graph");
    ACCEL_CUDA_TRY(cudaGraphLaunch(g->exec, as_stream(stream)));
    return after_launch(as_stream(stream), "accel_graph_launch", 0);
}

accel_status accel_graph_destroy(accel_graph g) {
    using namespace accel;
    if (!g) return ok();
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return ok();
}

accel_status accel_graph_node_count(accel_graph g, int64_t* out) {
    using namespace accel;
    ACCEL_REQUIRE(g && out, ACCEL_ERR_INVALID_ARG, "accel_graph_node_count: null argument");
    size_t n = 0;
    ACCEL_CUDA_TRY(cudaGraphGetNodes(g->graph, nullptr, &n));
    *out = (int64_t)n;
    return ok();
}

}  // extern "C"
