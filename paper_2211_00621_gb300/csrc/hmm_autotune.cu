// Autotuner for the BF16 tensor-core HMM forward: picks the launch configuration (column
// parts per row: 8 or 16 warps; sequence rows per tile: 128, 64 or 32; one CTA per tile or a
// cluster of two or four CTAs splitting the state columns) by timing every candidate on the caller's inputs
// with CUDA events, then the number of persistent work units of the winner: the fewest
// (of all that fit, 3/4, 1/2, 3/8 and 1/4 of them) within 1 % of its time.  The forward is
// bound by the step latency of its longest sequences, so on skewed length mixes a fraction
// of the GPU finishes it as fast as all of it, and the rest of the SMs stay free for work
// on other streams.  The winner is remembered per (device, K, M, floor(log2 S)) -- in this
// process, and optionally in a cache file of JSON lines so later processes skip the timing:
//   {"kernel": "hmm_forward_bf16", "device": "<name>", "K": 256, "M": 64, "S_log2": 12,
//    "split": 4, "rows": 128, "pair": 0, "units": 76, "ms": 17.21}
// (lines without "units" mean all units).  hmm_forward consults the table; without an entry
// it uses 16 warps, 128 rows, one CTA, all units.
#include "hmm_internal.cuh"

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace accel {
namespace hmm {

namespace {

using Key = std::tuple<std::string, int, int, int>;

std::mutex g_mu;
std::map<Key, TcConfig> g_table;

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    return prop.name;
}

int s_log2(int64_t S) {
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= S) ++b;
    return b;
}

TcConfig default_config(int K) { return TcConfig{(K / 4) % 32 == 0 ? 4 : 2, 128, 0, 0}; }

bool load_from_cache(const char* path, const Key& key, TcConfig* out) {
    if (!path || !path[0]) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char kern[64], dev[256];
        int K, M, sl, split, rows, pair, units = 0;
        float ms;
        int n = sscanf(line,
                       " {\"kernel\": \"%63[^\"]\", \"device\": \"%255[^\"]\", \"K\": %d, \"M\": %d, \"S_log2\": %d, "
                       "\"split\": %d, \"rows\": %d, \"pair\": %d, \"units\": %d, \"ms\": %f}",
                       kern, dev, &K, &M, &sl, &split, &rows, &pair, &units, &ms);
        if (n != 10) {
            units = 0;
            n = sscanf(line,
                       " {\"kernel\": \"%63[^\"]\", \"device\": \"%255[^\"]\", \"K\": %d, \"M\": %d, \"S_log2\": %d, "
                       "\"split\": %d, \"rows\": %d, \"pair\": %d, \"ms\": %f}",
                       kern, dev, &K, &M, &sl, &split, &rows, &pair, &ms);
            if (n != 9) continue;
        }
        if (strcmp(kern, "hmm_forward_bf16") != 0) continue;
        if (Key(dev, K, M, sl) == key) {
            *out = TcConfig{split, rows, pair < 0 ? 0 : (pair > 2 ? 2 : pair), units < 0 ? 0 : units};
            found = true;   // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

void append_to_cache(const char* path, const Key& key, TcConfig c, float ms) {
    if (!path || !path[0]) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"kernel\": \"hmm_forward_bf16\", \"device\": \"%s\", \"K\": %d, \"M\": %d, \"S_log2\": %d, "
            "\"split\": %d, \"rows\": %d, \"pair\": %d, \"units\": %d, \"ms\": %.4f}\n",
            std::get<0>(key).c_str(), std::get<1>(key), std::get<2>(key), std::get<3>(key), c.split, c.rows, c.pair,
            c.units, ms);
    fclose(f);
}

}  // namespace

TcConfig tuned_config(int K, int M, int64_t S) {
    Key key(device_name(), K, M, s_log2(S));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(key);
    return it != g_table.end() ? it->second : default_config(K);
}

accel_status check_model(const accel_hmm_model* m, const char* who);

}  // namespace hmm
}  // namespace accel

using namespace accel;
using namespace accel::hmm;

extern "C" {

accel_status hmm_autotune(const accel_hmm_model* m, int32_t precision, const int32_t* d_obs, const int64_t* d_offsets,
                          int64_t S, int64_t total_T, double* d_loglik, void* d_ws, size_t ws_bytes,
                          const char* cache_path, float* h_best_ms, void* stream) {
    accel_status r = check_model(m, "hmm_autotune");
    if (r != ACCEL_OK) return r;
    if (h_best_ms) *h_best_ms = 0.f;
    if (precision != ACCEL_HMM_BF16_SCALED || S == 0) return ok();   // nothing to tune
    ACCEL_REQUIRE(d_obs && d_offsets && d_loglik && d_ws, ACCEL_ERR_INVALID_ARG, "hmm_autotune: null pointer");
    ACCEL_REQUIRE(tc_supported(m->K, m->M), ACCEL_ERR_UNSUPPORTED, "hmm_autotune: shape not supported by the BF16 kernel");
    const size_t need = hmm_forward_workspace_size(m, S, total_T, precision);
    ACCEL_REQUIRE(ws_bytes >= need, ACCEL_ERR_WORKSPACE, "hmm_autotune: workspace %zu < %zu bytes", ws_bytes, need);
    ACCEL_REQUIRE(!debug_mode(), ACCEL_ERR_INVALID_ARG, "hmm_autotune: not available in debug mode");
    const Key key(device_name(), m->K, m->M, s_log2(S));
    TcConfig cached;
    if (load_from_cache(cache_path, key, &cached)) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_table[key] = cached;
        return ok();
    }
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    std::vector<TcConfig> cands;
    for (int pair : {0, 1, 2})
        for (int split : {4, 2})
            for (int rows : {128, 64, 32}) {
                if (split == 4 && (m->K / 4) % 32 != 0) continue;
                if (rows < 128 && (S + rows - 1) / rows <= (S + 127) / 128) continue;   // no more tiles than 128 rows
                if (pair && !tc_cl_supported(m->K, m->M, rows, split, pair == 1 ? 2 : 4)) continue;
                cands.push_back(TcConfig{split, rows, pair, 0});
            }
    cudaEvent_t e0, e1;
    ACCEL_CUDA_TRY(cudaEventCreate(&e0));
    ACCEL_CUDA_TRY(cudaEventCreate(&e1));
    // time one configuration: a warm-up run, then the mean of two (in *ms)
    auto time_cfg = [&](const TcConfig& c, float* ms) -> accel_status {
        ACCEL_CUDA_TRY(cudaMemsetAsync(ws + kStatusOff, 0, 4, st));
        accel_status q = tc_forward_cfg(m, d_obs, d_offsets, S, d_loglik, ws, (int32_t*)(ws + kStatusOff), c, st);
        if (q != ACCEL_OK) return q;
        float total = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            ACCEL_CUDA_TRY(cudaEventRecord(e0, st));
            q = tc_forward_cfg(m, d_obs, d_offsets, S, d_loglik, ws, (int32_t*)(ws + kStatusOff), c, st);
            if (q != ACCEL_OK) return q;
            ACCEL_CUDA_TRY(cudaEventRecord(e1, st));
            ACCEL_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            ACCEL_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            total += t;
        }
        int32_t dev_status = ACCEL_OK;      // a candidate that timed out on the device is an error
        ACCEL_CUDA_TRY(cudaMemcpy(&dev_status, ws + kStatusOff, 4, cudaMemcpyDeviceToHost));
        if (dev_status != ACCEL_OK)
            return set_error(dev_status, "hmm_autotune: device-side status %d while timing (split=%d, rows=%d, pair=%d, "
                             "units=%d)", dev_status, c.split, c.rows, c.pair, c.units);
        *ms = total / 2;
        return ACCEL_OK;
    };
    TcConfig best = default_config(m->K);
    float best_ms = INFINITY;
    for (const TcConfig& c : cands) {
        float ms = 0.f;
        r = time_cfg(c, &ms);
        if (r != ACCEL_OK) break;
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    if (r == ACCEL_OK && best_ms < INFINITY) {
        // fewer persistent work units: the smallest count within 1 % of the best time
        const int nc = best.pair == 2 ? 4 : (best.pair == 1 ? 2 : 1);
        const int64_t tiles = (S + best.rows - 1) / best.rows;
        const int64_t cap64 = tiles < num_sms() / nc ? tiles : num_sms() / nc;
        const int cap = (int)(cap64 < 1 ? 1 : cap64);
        const float limit = best_ms * 1.01f;
        for (int f8 : {6, 4, 3, 2}) {            // 3/4, 1/2, 3/8, 1/4 of the units
            TcConfig c = best;
            c.units = (cap * f8 + 7) / 8;
            if (c.units < 1 || c.units >= cap) continue;
            float ms = 0.f;
            r = time_cfg(c, &ms);
            if (r != ACCEL_OK) break;
            if (ms <= limit) {
                best = c;                        // keep the time of the full launch as the reference
                best_ms = ms < best_ms ? ms : best_ms;
            } else {
                break;                           // fewer units only get slower
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != ACCEL_OK) return r;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_table[key] = best;
    }
    append_to_cache(cache_path, key, best, best_ms);
    if (h_best_ms) *h_best_ms = best_ms;
    return ok();
}

// Configuration hmm_forward would use for these sizes (for tests and reports).
accel_status hmm_tuned_config(int32_t K, int32_t M, int64_t S, int32_t* h_split, int32_t* h_rows, int32_t* h_pair,
                              int32_t* h_units) {
    ACCEL_REQUIRE(h_split && h_rows, ACCEL_ERR_INVALID_ARG, "hmm_tuned_config: null pointer");
    TcConfig c = tuned_config(K, M, S);
    *h_split = c.split;
    *h_rows = c.rows;
    if (h_pair) *h_pair = c.pair;
    if (h_units) *h_units = c.units;
    return ok();
}

}  // extern "C"
