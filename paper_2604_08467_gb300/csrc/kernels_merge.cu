// Merging the emitted shots across trajectories (the emit step's optional
// merge, Sec. III-B's final (bitstring, count) list): a stable LSD radix sort of
// the (bitstring, count) records by bitstring, 8 bits per pass, then one
// record per distinct bitstring with the summed count.
//
// Sort pass: the input is cut into segments of kSeg records, one thread per
// segment.  Each thread histograms its segment's digits; an exclusive scan of
// the digit-major histogram (digit, segment) gives every segment the first
// output slot of each digit, and the thread then scatters its records in
// order, which keeps the sort stable.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

constexpr int kSeg = 256;

__global__ void k_seg_hist(const uint64_t* __restrict__ key, int64_t n, int shift, int64_t n_seg,
                           int64_t* __restrict__ hist) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= n_seg) return;
    int32_t h[256];
    for (int d = 0; d < 256; d++) h[d] = 0;
    const int64_t i1 = (seg + 1) * kSeg < n ? (seg + 1) * kSeg : n;
    for (int64_t i = seg * kSeg; i < i1; i++) h[(key[i] >> shift) & 255u]++;
    for (int d = 0; d < 256; d++) hist[(int64_t)d * n_seg + seg] = h[d];
}

__global__ void k_seg_scatter(const uint64_t* __restrict__ key, const int64_t* __restrict__ val, int64_t n, int shift,
                              int64_t n_seg, const int64_t* __restrict__ off, uint64_t* __restrict__ key_out,
                              int64_t* __restrict__ val_out) {
    const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= n_seg) return;
    int64_t o[256];
    for (int d = 0; d < 256; d++) o[d] = off[(int64_t)d * n_seg + seg];
    const int64_t i1 = (seg + 1) * kSeg < n ? (seg + 1) * kSeg : n;
    for (int64_t i = seg * kSeg; i < i1; i++) {
        const uint64_t k = key[i];
        const int64_t p = o[(k >> shift) & 255u]++;
        key_out[p] = k;
        val_out[p] = val[i];
    }
}

__global__ void k_run_flags(const uint64_t* __restrict__ key, int64_t n, int64_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// run index of every run start: start[r] = i
__global__ void k_run_starts(const int64_t* __restrict__ flag, const int64_t* __restrict__ excl, int64_t n,
                             int64_t* __restrict__ start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) start[excl[i]] = i;
}

// one thread per run: its bitstring and the sum of its counts (in input order)
__global__ void k_run_sum(const uint64_t* __restrict__ key, const int64_t* __restrict__ val,
                          const int64_t* __restrict__ start, int64_t n_runs, int64_t n, int32_t* __restrict__ traj_out,
                          uint64_t* __restrict__ bits_out, int64_t* __restrict__ count_out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_runs; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = start[r], b = r + 1 < n_runs ? start[r + 1] : n;
        int64_t c = 0;
        for (int64_t i = a; i < b; i++) c += val[i];
        traj_out[r] = -1;
        bits_out[r] = key[a];
        count_out[r] = c;
    }
}

// Multi-word bitstrings (n_words > 1): records are sorted as indices, one
// word at a time from the least significant (LSD, every pass stable), so the
// final order is lexicographic by the whole string.
__global__ void k_gather_word(const uint64_t* __restrict__ bits, const int64_t* __restrict__ idx, int n_words, int w,
                              int64_t n, uint64_t* __restrict__ key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = bits[idx[i] * n_words + w];
}

__global__ void k_run_flags_words(const uint64_t* __restrict__ bits, const int64_t* __restrict__ idx, int n_words,
                                  int64_t n, int64_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t f = i == 0;
        if (i) {
            const uint64_t *a = bits + idx[i] * n_words, *b = bits + idx[i - 1] * n_words;
            for (int w = 0; w < n_words; w++) f |= a[w] != b[w];
        }
        flag[i] = f;
    }
}

// one thread per run: its bitstring and the sum of its counts (in input order)
__global__ void k_run_sum_words(const uint64_t* __restrict__ bits, const int64_t* __restrict__ count,
                                const int64_t* __restrict__ idx, int n_words, const int64_t* __restrict__ start,
                                int64_t n_runs, int64_t n, int32_t* __restrict__ traj_out,
                                uint64_t* __restrict__ bits_out, int64_t* __restrict__ count_out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_runs; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = start[r], b = r + 1 < n_runs ? start[r + 1] : n;
        int64_t c = 0;
        for (int64_t i = a; i < b; i++) c += count[idx[i]];
        traj_out[r] = -1;
        for (int w = 0; w < n_words; w++) bits_out[r * n_words + w] = bits[idx[a] * n_words + w];
        count_out[r] = c;
    }
}

unsigned blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

void launch_radix_pass(const uint64_t* key, const int64_t* val, int64_t n, int shift, int64_t* hist, int64_t* scan_tmp,
                       uint64_t* key_out, int64_t* val_out, cudaStream_t s) {
    const int64_t n_seg = (n + kSeg - 1) / kSeg;
    StatScope sc(K_MISC, s, 32.0 * (double)n, 0.0);
    count_launches(K_MISC);   // two kernels under one scope
    k_seg_hist<<<(unsigned)((n_seg + 127) / 128), 128, 0, s>>>(key, n, shift, n_seg, hist);
    launch_exclusive_scan(hist, hist, 256 * n_seg, scan_tmp, s);
    k_seg_scatter<<<(unsigned)((n_seg + 127) / 128), 128, 0, s>>>(key, val, n, shift, n_seg, hist, key_out, val_out);
}

int64_t radix_hist_elems(int64_t n) { return 256 * ((n + kSeg - 1) / kSeg); }

void launch_run_flags(const uint64_t* key, int64_t n, int64_t* flag, cudaStream_t s) {
    StatScope sc(K_MISC, s, 16.0 * (double)n, 0.0);
    k_run_flags<<<blocks_for(n, 256), 256, 0, s>>>(key, n, flag);
}

void launch_run_starts(const int64_t* flag, const int64_t* excl, int64_t n, int64_t* start, cudaStream_t s) {
    StatScope sc(K_MISC, s, 16.0 * (double)n, 0.0);
    k_run_starts<<<blocks_for(n, 256), 256, 0, s>>>(flag, excl, n, start);
}

void launch_run_sum(const uint64_t* key, const int64_t* val, const int64_t* start, int64_t n_runs, int64_t n,
                    int32_t* traj_out, uint64_t* bits_out, int64_t* count_out, cudaStream_t s) {
    if (n_runs <= 0) return;
    StatScope sc(K_MISC, s, 16.0 * (double)n + 20.0 * (double)n_runs, 0.0);
    k_run_sum<<<blocks_for(n_runs, 256), 256, 0, s>>>(key, val, start, n_runs, n, traj_out, bits_out, count_out);
}

void launch_gather_word(const uint64_t* bits, const int64_t* idx, int n_words, int w, int64_t n, uint64_t* key,
                        cudaStream_t s) {
    StatScope sc(K_MISC, s, 24.0 * (double)n, 0.0);
    k_gather_word<<<blocks_for(n, 256), 256, 0, s>>>(bits, idx, n_words, w, n, key);
}

void launch_run_flags_words(const uint64_t* bits, const int64_t* idx, int n_words, int64_t n, int64_t* flag,
                            cudaStream_t s) {
    StatScope sc(K_MISC, s, (16.0 * n_words + 16.0) * (double)n, 0.0);
    k_run_flags_words<<<blocks_for(n, 256), 256, 0, s>>>(bits, idx, n_words, n, flag);
}

void launch_run_sum_words(const uint64_t* bits, const int64_t* count, const int64_t* idx, int n_words,
                          const int64_t* start, int64_t n_runs, int64_t n, int32_t* traj_out, uint64_t* bits_out,
                          int64_t* count_out, cudaStream_t s) {
    if (n_runs <= 0) return;
    StatScope sc(K_MISC, s, 24.0 * (double)n + (12.0 + 8.0 * n_words) * (double)n_runs, 0.0);
    k_run_sum_words<<<blocks_for(n_runs, 256), 256, 0, s>>>(bits, count, idx, n_words, start, n_runs, n, traj_out,
                                                           bits_out, count_out);
}

}  // namespace ptn
