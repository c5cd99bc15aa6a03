// Block-size autotuning (Sec. V-B, Fig. 7): the cost of a sampling run depends
// strongly on the qubit block size b (the paper measures 35.4 ms per block at
// b = 10 against 2176.8 ms at b = 24 on one circuit family), so the block
// size is chosen per circuit by measurement: every candidate b gets its own
// plan (blocks of b qubits, the last one taking the remainder) and a timed
// probe run (pre-sampling + proportional NBS on the GPU), and the fastest
// candidate wins.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kernels.cuh"

namespace ptn {
void clear_error();
}

using namespace ptn;

extern "C" ptn_status ptn_tune_block_sizes(const ptn_circuit* circuit, const ptn_noise* noise,
                                           const int32_t* candidates, int32_t n_cand, const ptn_plan_opts* opts,
                                           int64_t probe_traj, int64_t probe_shots, uint64_t seed, int32_t* best_b,
                                           double* seconds_out, ptn_stream stream) {
    clear_error();
    if (!circuit || !noise || !candidates || n_cand < 1 || !best_b || !seconds_out)
        return set_error(PTN_ERR_INVALID_ARG, "NULL argument or no candidates");
    if (probe_traj < 1 || probe_shots < 1) return set_error(PTN_ERR_INVALID_ARG, "probe sizes must be >= 1");
    const int n = circuit->n_qubits;
    for (int32_t i = 0; i < n_cand; i++)
        if (candidates[i] < 1 || candidates[i] > kMaxSampleBlock)
            return set_error(PTN_ERR_INVALID_ARG, "candidate block size %d outside 1..%d", candidates[i],
                             kMaxSampleBlock);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(PTN_ERR_CUDA, "event creation failed");
    int32_t best = -1;
    double best_s = INFINITY;
    ptn_status last = PTN_OK;
    for (int32_t i = 0; i < n_cand; i++) {
        seconds_out[i] = INFINITY;
        const int b = candidates[i];
        const int f = (n + b - 1) / b;
        std::vector<int32_t> bs(f, b);
        bs[f - 1] = n - b * (f - 1);
        ptn_plan* plan = nullptr;
        ptn_status st = ptn_plan_path(circuit, noise, bs.data(), f, opts, &plan);
        if (st != PTN_OK) {
            last = st;
            continue;
        }
        ptn_sample_opts so{};
        so.mode = PTN_PROPORTIONAL_TOTAL;
        so.total_shots = probe_shots;
        so.seed = seed;
        so.precision = PTN_PREC_FP32;
        double sec = INFINITY;
        for (int rep = 0; rep < 2 && st == PTN_OK; rep++) {   // the first run warms the workspace up
            ptn_traj* tr = nullptr;
            ptn_shots* sh = nullptr;
            cudaEventRecord(e0, s);
            st = ptn_presample_trajectories(plan, seed + (uint64_t)rep, 0, probe_traj, 0, &tr, stream);
            if (st == PTN_OK) st = ptn_sample_shots(plan, tr, &so, &sh, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = set_error(PTN_ERR_CUDA, "probe run failed");
            float ms = 0.f;
            if (st == PTN_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) sec = ms * 1e-3;
            ptn_shots_destroy(sh);
            ptn_traj_destroy(tr);
        }
        ptn_plan_destroy(plan);
        if (st != PTN_OK) {
            last = st;
            continue;
        }
        seconds_out[i] = sec;
        if (sec < best_s) {
            best_s = sec;
            best = b;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) return last != PTN_OK ? last : set_error(PTN_ERR_TOO_LARGE, "no candidate could run");
    *best_b = best;
    clear_error();
    return PTN_OK;
}
