// Kernel launch statistics: launch counts per kernel and, when timing is on,
// CUDA-event durations with the algorithmic bytes and flops of every launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "stats.h"

namespace ptn {
namespace {
struct Rec {
    int kid;
    cudaEvent_t a, b;
    double bytes, flops;
    int block, step;
};
thread_local int t_block = -1, t_step = -1;
struct State {
    std::mutex mu;
    bool timing = false;
    int only = -1;               // time only this kernel class (-1: every class)
    int64_t launches[K_COUNT] = {};
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
};
State& st() {
    static State s;
    return s;
}
const char* kNames[K_COUNT] = {"contract_direct", "contract_gemm", "finalize", "presample", "logq",
                               "dedup", "var_ids", "scan", "alloc_shots", "sample_parents",
                               "emit_children", "gemm_pack", "expval", "misc", "harvest", "contract_small",
                               "cache_tables"};
cudaEvent_t take_event() {
    State& s = st();
    if (!s.pool.empty()) {
        cudaEvent_t e = s.pool.back();
        s.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void count_launches(int kid, int n) {
    State& g = st();
    std::lock_guard<std::mutex> lk(g.mu);
    g.launches[kid] += n;
}

void set_step_tag(int block, int step) {
    t_block = block;
    t_step = step;
}

StatScope::StatScope(int kid, cudaStream_t s, double bytes, double flops) : kid_(kid), s_(s) {
    block_ = t_block;
    step_ = t_step;
    State& g = st();
    std::lock_guard<std::mutex> lk(g.mu);
    g.launches[kid]++;
    timing_ = g.timing && (g.only < 0 || g.only == kid);
    if (timing_) {   // launches recorded into a CUDA graph are counted, not timed
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) timing_ = false;
    }
    if (timing_) {
        a_ = take_event();
        b_ = take_event();
        bytes_ = bytes;
        flops_ = flops;
        cudaEventRecord((cudaEvent_t)a_, s);
    }
}

StatScope::~StatScope() {
    if (!timing_) return;
    State& g = st();
    std::lock_guard<std::mutex> lk(g.mu);
    cudaEventRecord((cudaEvent_t)b_, s_);
    g.recs.push_back({kid_, (cudaEvent_t)a_, (cudaEvent_t)b_, bytes_, flops_, block_, step_});
}

}  // namespace ptn

using namespace ptn;

extern "C" ptn_status ptn_stats_enable(int32_t on) {
    State& g = st();
    std::lock_guard<std::mutex> lk(g.mu);
    g.timing = on != 0;
    g.only = -1;
    return PTN_OK;
}

extern "C" ptn_status ptn_stats_enable_only(const char* kernel) {
    if (!kernel || !*kernel) return ptn_stats_enable(1);
    int kid = -1;
    for (int k = 0; k < K_COUNT; k++)
        if (strcmp(kernel, kNames[k]) == 0) kid = k;
    if (kid < 0) return set_error(PTN_ERR_INVALID_ARG, "unknown kernel class '%s'", kernel);
    State& g = st();
    std::lock_guard<std::mutex> lk(g.mu);
    g.timing = true;
    g.only = kid;
    return PTN_OK;
}

extern "C" ptn_status ptn_stats_reset(void) {
    State& g = st();
    std::lock_guard<std::mutex> lk(g.mu);
    for (auto& r : g.recs) {
        g.pool.push_back(r.a);
        g.pool.push_back(r.b);
    }
    g.recs.clear();
    memset(g.launches, 0, sizeof g.launches);
    return PTN_OK;
}

extern "C" ptn_status ptn_stats_read(ptn_kernel_stat* out, int32_t cap, int32_t* n_out) {
    State& g = st();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "stats: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g.mu);
    ptn_kernel_stat acc[K_COUNT];
    memset(acc, 0, sizeof acc);
    for (int k = 0; k < K_COUNT; k++) {
        strncpy(acc[k].name, kNames[k], sizeof acc[k].name - 1);
        acc[k].launches = g.launches[k];
    }
    for (auto& r : g.recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        acc[r.kid].timed_launches++;
        acc[r.kid].ms += ms;
        acc[r.kid].alg_bytes += r.bytes;
        acc[r.kid].alg_flops += r.flops;
    }
    int n = 0;
    for (int k = 0; k < K_COUNT && n < cap; k++)
        if (acc[k].launches) out[n++] = acc[k];
    if (n_out) *n_out = n;
    return PTN_OK;
}

extern "C" ptn_status ptn_stats_read_steps(ptn_step_stat* out, int32_t cap, int32_t* n_out) {
    State& g = st();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "stats: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g.mu);
    std::map<std::tuple<int, int, int>, ptn_step_stat> acc;
    for (auto& r : g.recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        ptn_step_stat& x = acc[std::make_tuple(r.block, r.step, r.kid)];
        if (!x.launches) {
            x.block = r.block;
            x.step = r.step;
            strncpy(x.kernel, kNames[r.kid], sizeof x.kernel - 1);
        }
        x.launches++;
        x.ms += ms;
        x.alg_bytes += r.bytes;
        x.alg_flops += r.flops;
    }
    int n = 0;
    for (auto& kv : acc) {
        if (n >= cap) break;
        if (out) out[n] = kv.second;
        n++;
    }
    if (n_out) *n_out = n;
    return PTN_OK;
}
