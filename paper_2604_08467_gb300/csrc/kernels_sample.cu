// Pre-trajectory sampling, error-set deduplication, UPV variant selection,
// proportional shot allocation and the conditional-marginal sampling of
// non-degenerate batched sampling (Sec. II-C, III-A, III-B).
//
// Bit-exactness rules shared with the CPU oracle:
//  * Kraus draw: u = ((x0 << 32 | x1) >> 11) * 2^-53 against the site's FP64
//    CDF table (smallest k with u < C[k]);
//  * a probability row is quantised to integers P_x = rint(max(p_x,0) 2^sigma)
//    held exactly in FP64 (sigma = 52 - bits - e, max p = f 2^e), so the
//    running sum C is exact in any summation order, and a draw picks the
//    smallest x with floor(a T / 2^64) < C[x], a = x0 << 32 | x1, T = C[last].
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

constexpr int kScanTile = 2048;   // elements per block in the scan (1024 threads x 2)

// ------------------------------------------------------------- presample --
__global__ void k_presample(const SiteTable* __restrict__ sites, int32_t S, int64_t n_traj, int64_t traj0, uint2 key,
                            uint32_t tagw, uint8_t* __restrict__ kraus) {
    const int64_t total = n_traj * S;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g / S;
        const int32_t s = (int32_t)(g - i * S);
        const uint4 x = philox4x32_10(make_uint4((uint32_t)s, 0u, (uint32_t)(traj0 + i), tagw), key);
        const double u = (double)(word64(x) >> 11) * 0x1p-53;
        const SiteTable& T = sites[s];
        int k = 0;
        while (k < T.n_kraus - 1 && !(u < T.cdf[k])) k++;
        kraus[g] = (uint8_t)k;
    }
}

__global__ void k_logq(const SiteTable* __restrict__ sites, int32_t S, int64_t n_traj,
                       const uint8_t* __restrict__ kraus, double* __restrict__ logq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_traj) return;
    double acc = 0.0;
    for (int32_t s = 0; s < S; s++) acc = acc + sites[s].logq[kraus[i * S + s]];
    logq[i] = acc;
}

// FNV-1a over a Kraus row
__global__ void k_row_hash(const uint8_t* __restrict__ kraus, int64_t n, int32_t S, uint64_t* __restrict__ h) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t v = 1469598103934665603ull;
    const uint8_t* r = kraus + i * S;
    for (int32_t s = 0; s < S; s++) v = (v ^ r[s]) * 1099511628211ull;
    h[i] = v;
}

// Rows with equal hashes are contiguous after a stable sort of (hash, index)
// pairs, in increasing index order: first[i] = smallest j whose row equals
// row i is the run's first index when the rows match (always, unless two
// different rows share a hash), else the first matching index further along
// the run (a hash collision: compared row by row).  p: position in the sorted
// order; run = inclusive count of run starts up to p, minus one.
__device__ __forceinline__ bool rows_equal(const uint8_t* __restrict__ kraus, int64_t a, int64_t b, int32_t S) {
    const uint8_t* ra = kraus + a * S;
    const uint8_t* rb = kraus + b * S;
    for (int32_t s = 0; s < S; s++)
        if (ra[s] != rb[s]) return false;
    return true;
}
__global__ void k_first_in_run(const uint8_t* __restrict__ kraus, int32_t S, const int64_t* __restrict__ idx,
                               const int64_t* __restrict__ flag, const int64_t* __restrict__ excl,
                               const int64_t* __restrict__ start, int64_t n, int64_t* __restrict__ first) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r0 = start[excl[p] + flag[p] - 1];
        const int64_t i = idx[p];
        int64_t f = i;
        for (int64_t q = r0; q < p; q++) {
            if (rows_equal(kraus, idx[q], i, S)) {
                f = idx[q];
                break;
            }
        }
        first[i] = f;
    }
}

__global__ void k_iota_i64(int64_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = i;
}

__global__ void k_flags_first(const int64_t* __restrict__ first, int64_t n, int64_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = first[i] == i ? 1 : 0;
}

__global__ void k_dedup_compact(const uint8_t* __restrict__ kraus, const double* __restrict__ logq,
                                const int64_t* __restrict__ first, const int64_t* __restrict__ uid, int64_t n,
                                int32_t S, uint8_t* __restrict__ kraus_u, double* __restrict__ logq_u,
                                unsigned long long* __restrict__ mult_u, int64_t* __restrict__ first_u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t f = first[i];
    const int64_t u = uid[f];
    atomicAdd(&mult_u[u], 1ull);
    if (f == i) {
        for (int32_t s = 0; s < S; s++) kraus_u[u * S + s] = kraus[i * S + s];
        logq_u[u] = logq[i];
        first_u[u] = i;
    }
}

// variant index of every multi-variant leaf: mixed radix over its sites
__global__ void k_var_ids(const uint8_t* __restrict__ kraus, int64_t n, int32_t S, const int32_t* __restrict__ ptr,
                          const int32_t* __restrict__ idx, const int32_t* __restrict__ mul, int32_t n_cols,
                          int32_t* __restrict__ var_ids) {
    const int64_t total = n * n_cols;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g / n_cols;
        const int32_t col = (int32_t)(g - i * n_cols);
        int32_t v = 0;
        for (int32_t e = ptr[col]; e < ptr[col + 1]; e++) v += (int32_t)kraus[i * S + idx[e]] * mul[e];
        var_ids[g] = v;
    }
}

// ----------------------------------------------------------------- scans --
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
    // sh: blockDim.x + 1 elements
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int64_t add = t >= off ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    const int64_t incl = sh[t];
    if (total) *total = sh[blockDim.x - 1];
    __syncthreads();
    return incl - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                     int64_t n, int64_t* __restrict__ tile_sums) {
    __shared__ int64_t sh[1025];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t i0 = base + 2 * threadIdx.x, i1 = i0 + 1;
    const int64_t a = i0 < n ? in[i0] : 0, b = i1 < n ? in[i1] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan(a + b, sh, &tot);
    if (i0 < n) out[i0] = ex;
    if (i1 < n) out[i1] = ex + a;
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tile_off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

// --------------------------------------------------------- allocation ----
// Quantise the weights into an exact-integer FP64 CDF (one block).
__global__ void __launch_bounds__(1024) k_quantise_cdf(const double* __restrict__ w, int64_t n, int bits,
                                                       double* __restrict__ C) {
    __shared__ double red[1024];
    __shared__ int64_t sh[1025];
    __shared__ double carry;
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, w[i] > 0.0 ? w[i] : 0.0);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    int e;
    frexp(red[0], &e);
    const int sigma = 52 - bits - e;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const double p = i < n ? rint(ldexp(w[i] > 0.0 ? w[i] : 0.0, sigma)) : 0.0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan((int64_t)p, sh, &tot);
        if (i < n) C[i] = carry + (double)(ex + (int64_t)p);
        __syncthreads();
        if (threadIdx.x == 0) carry += (double)tot;
        __syncthreads();
    }
}

// smallest x with r < C[x] (C non-decreasing, exact integers)
__device__ __forceinline__ int64_t cdf_search_u64(const uint64_t* C, int64_t n, uint64_t r) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (r < C[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int64_t cdf_search(const double* C, int64_t n, double r) {
    // smallest x with r < C[x]
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (r < C[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void k_alloc_draw(const double* __restrict__ C, int64_t n, int64_t total, uint2 key, uint32_t tagw,
                             unsigned long long* __restrict__ m) {
    const uint64_t T = (uint64_t)C[n - 1];
    if (T == 0) return;   // all weights zero: no shot is allocated
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint4 x = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)((uint64_t)t >> 32), 0u, tagw), key);
        const double r = (double)__umul64hi(word64(x), T);
        atomicAdd(&m[cdf_search(C, n, r)], 1ull);
    }
}

__global__ void k_mult_times_z(const int64_t* __restrict__ mult, const double* __restrict__ Z, int64_t n,
                               double* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = (double)mult[i] * Z[i];
}

__global__ void k_fill_i64(int64_t* p, int64_t v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_iota_i32(int32_t* p, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}
__global__ void k_scale_i64(const int64_t* a, int64_t k, int64_t n, int64_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * k;
}

// ------------------------------------------------------------ NBS step ----
__global__ void k_sample_prep(const int64_t* __restrict__ count, int64_t n, int b, const int32_t* __restrict__ traj,
                              int64_t* __restrict__ cap, unsigned long long* __restrict__ first) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c = count[i];
    const int64_t nb = (int64_t)1 << b;
    cap[i] = c < nb ? c : nb;
    atomicMin(&first[traj[i]], (unsigned long long)i);
}

__global__ void k_rank0(const int64_t* __restrict__ excl, const int32_t* __restrict__ traj,
                        const unsigned long long* __restrict__ first, int64_t n, int64_t* __restrict__ rank0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rank0[i] = excl[i] - excl[first[traj[i]]];
}

// One block per parent: quantised CDF, c draws, histogram, ordered compaction
// of the nonzero bins into the parent's slot of the temporary child list.
__global__ void __launch_bounds__(256) k_sample_parents(const float* __restrict__ marg, int b,
                                                        const int32_t* __restrict__ traj,
                                                        const int64_t* __restrict__ count,
                                                        const int64_t* __restrict__ rank0,
                                                        const int64_t* __restrict__ tmp_off, int64_t tmp_cap,
                                                        uint2 key, uint32_t tagw, int32_t* __restrict__ tmp_x,
                                                        int64_t* __restrict__ tmp_c, int64_t* __restrict__ ndist) {
    extern __shared__ unsigned char smem[];
    const int64_t nb = (int64_t)1 << b;
    uint64_t* C = reinterpret_cast<uint64_t*>(smem);                   // nb
    unsigned int* hist = reinterpret_cast<unsigned int*>(C + nb);      // nb
    __shared__ int64_t sh[257];
    __shared__ float fred[256];
    __shared__ uint64_t carry;
    __shared__ int64_t wpos;
    const int64_t n = blockIdx.x;
    const int64_t c = count[n];
    if (c <= 0) {
        if (threadIdx.x == 0) ndist[n] = 0;
        return;
    }
    const float* p = marg + n * nb;
    float m = 0.f;
    for (int64_t x = threadIdx.x; x < nb; x += blockDim.x) m = fmaxf(m, p[x] > 0.f ? p[x] : 0.f);
    fred[threadIdx.x] = m;
    for (int64_t x = threadIdx.x; x < nb; x += blockDim.x) hist[x] = 0u;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) fred[threadIdx.x] = fmaxf(fred[threadIdx.x], fred[threadIdx.x + s]);
        __syncthreads();
    }
    const int sigma = 52 - b - frexp_exp(fred[0]);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t x = base + threadIdx.x;
        const uint64_t v = x < nb ? quant_pow2(p[x], sigma) : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan((int64_t)v, sh, &tot);
        if (x < nb) C[x] = carry + (uint64_t)ex + v;
        __syncthreads();
        if (threadIdx.x == 0) carry += (uint64_t)tot;
        __syncthreads();
    }
    const uint64_t T = C[nb - 1];
    if (T == 0) {   // zero-norm network: its shots cannot be drawn and are dropped
        if (threadIdx.x == 0) ndist[n] = 0;
        return;
    }
    const uint32_t tr = (uint32_t)traj[n];
    const int64_t r0 = rank0[n];
    for (int64_t k = threadIdx.x; k < c; k += blockDim.x) {
        const uint64_t rank = (uint64_t)(r0 + k);
        const uint4 w = philox4x32_10(make_uint4((uint32_t)rank, (uint32_t)(rank >> 32), tr, tagw), key);
        atomicAdd(&hist[cdf_search_u64(C, nb, __umul64hi(word64(w), T))], 1u);
    }
    if (threadIdx.x == 0) wpos = 0;
    __syncthreads();
    const int64_t dst = tmp_off[n];
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t x = base + threadIdx.x;
        const unsigned int h = x < nb ? hist[x] : 0u;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(h ? 1 : 0, sh, &tot);
        // slots past tmp_cap are never written; the host reports the shortfall
        if (h && dst + wpos + ex < tmp_cap) {
            tmp_x[dst + wpos + ex] = (int32_t)x;
            tmp_c[dst + wpos + ex] = (int64_t)h;
        }
        __syncthreads();
        if (threadIdx.x == 0) wpos += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) ndist[n] = wpos;
}

// Blocks of up to 2^10 bins: one warp per parent, kSampWarps parents per CTA,
// no CTA-wide barrier.  The row is read in coalesced rounds of 32 bins (lane l
// holds bin 32 i + l of round i, kept in registers): the row maximum is a
// shuffle reduction; the exact-integer CDF is built round by round with a
// shuffle scan plus the running total in 64-bit integers (the values the FP64
// rule defines, computed without FP64 arithmetic); the draws
// search the warp's CDF in shared memory and count into its histogram; the
// nonzero bins are compacted in x order with one ballot per round.  Same
// arithmetic and results as k_sample_parents.
constexpr int kSampWarps = 4;
constexpr int kSampWarpMaxBits = 10;

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane) {
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}


__global__ void __launch_bounds__(kSampWarps * 32) k_sample_parents_warp(
    const float* __restrict__ marg, int b, int64_t n_parent, const int32_t* __restrict__ traj,
    const int64_t* __restrict__ count, const int64_t* __restrict__ rank0, const int64_t* __restrict__ tmp_off,
    int64_t tmp_cap, uint2 key, uint32_t tagw, int32_t* __restrict__ tmp_x, int64_t* __restrict__ tmp_c,
    int64_t* __restrict__ ndist) {
    extern __shared__ unsigned char smem[];
    constexpr int kMaxRounds = (1 << kSampWarpMaxBits) / 32;
    const int nb = 1 << b;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* C = reinterpret_cast<uint64_t*>(smem) + (int64_t)wib * nb;
    unsigned* hist = reinterpret_cast<unsigned*>(reinterpret_cast<uint64_t*>(smem) + (int64_t)kSampWarps * nb) +
                     (int64_t)wib * nb;
    const int64_t n = (int64_t)blockIdx.x * kSampWarps + wib;
    if (n >= n_parent) return;                 // the whole warp leaves together
    const int64_t c = count[n];
    if (c <= 0) {
        if (lane == 0) ndist[n] = 0;
        return;
    }
    const float* p = marg + n * (int64_t)nb;
    const int rounds = (nb + 31) >> 5;
    float v[kMaxRounds];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < kMaxRounds; i++) {
        const int x = 32 * i + lane;
        v[i] = 0.f;
        if (i < rounds && x < nb) {
            const float t = p[x];
            v[i] = t > 0.f ? t : 0.f;
        }
        m = fmaxf(m, v[i]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int sigma = 52 - b - frexp_exp(m);
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < kMaxRounds; i++) {
        if (i < rounds) {
            const int x = 32 * i + lane;
            const uint64_t inc = warp_incl_scan_u64(quant_pow2(v[i], sigma), lane);
            if (x < nb) {
                C[x] = carry + inc;
                hist[x] = 0u;
            }
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    __syncwarp();
    const uint64_t T = C[nb - 1];
    if (T == 0) {   // zero-norm network: its shots cannot be drawn and are dropped
        if (lane == 0) ndist[n] = 0;
        return;
    }
    const uint32_t tr = (uint32_t)traj[n];
    const int64_t r0 = rank0[n];
    for (int64_t k = lane; k < c; k += 32) {
        const uint64_t rank = (uint64_t)(r0 + k);
        const uint4 w = philox4x32_10(make_uint4((uint32_t)rank, (uint32_t)(rank >> 32), tr, tagw), key);
        atomicAdd(&hist[cdf_search_u64(C, nb, __umul64hi(word64(w), T))], 1u);
    }
    __syncwarp();
    int64_t pos = tmp_off[n];
    const unsigned below = (1u << lane) - 1u;
    for (int i = 0; i < rounds; i++) {
        const int x = 32 * i + lane;
        const unsigned h = x < nb ? hist[x] : 0u;
        const unsigned mask = __ballot_sync(0xffffffffu, h != 0u);
        if (h) {
            const int64_t q = pos + __popc(mask & below);
            // slots past tmp_cap are never written; the host reports the shortfall
            if (q < tmp_cap) {
                tmp_x[q] = x;
                tmp_c[q] = (int64_t)h;
            }
        }
        pos += __popc(mask);
    }
    if (lane == 0) ndist[n] = pos - tmp_off[n];
}

__global__ void k_emit_children(const int32_t* __restrict__ traj, const uint64_t* __restrict__ prefix,
                                const int64_t* __restrict__ tmp_off, const int64_t* __restrict__ ndist,
                                const int64_t* __restrict__ out_off, const int32_t* __restrict__ tmp_x,
                                const int64_t* __restrict__ tmp_c, int start, int64_t n, int n_words,
                                int32_t* __restrict__ ctraj, uint64_t* __restrict__ cprefix,
                                int64_t* __restrict__ ccount) {
    // one warp per parent
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int64_t nd = ndist[w], src = tmp_off[w], dst = out_off[w];
    const int32_t t = traj[w];
    if (n_words == 1) {
        const uint64_t pre = prefix[w];
        for (int64_t k = lane; k < nd; k += 32) {
            ctraj[dst + k] = t;
            cprefix[dst + k] = pre | ((uint64_t)tmp_x[src + k] << start);
            ccount[dst + k] = tmp_c[src + k];
        }
        return;
    }
    const uint64_t* pre = prefix + w * n_words;
    for (int64_t k = lane; k < nd; k += 32) {
        ctraj[dst + k] = t;
        bits_put(cprefix + (dst + k) * n_words, pre, n_words, (uint64_t)tmp_x[src + k], start);
        ccount[dst + k] = tmp_c[src + k];
    }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

void launch_presample(const SiteTable* sites, int32_t n_sites, int64_t n_traj, int64_t traj0, uint64_t seed,
                      int32_t circuit, uint8_t* kraus, double* logq, cudaStream_t s) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if (n_sites > 0) {
        StatScope sc(K_PRESAMPLE, s, (double)n_traj * n_sites, 0.0);
        k_presample<<<grid_for(n_traj * n_sites, 256), 256, 0, s>>>(sites, n_sites, n_traj, traj0, key,
                                                                    philox_tag(STREAM_KRAUS, circuit, 0), kraus);
    }
    StatScope sc2(K_LOGQ, s, (double)n_traj * (n_sites + 8), 0.0);
    k_logq<<<grid_for(n_traj, 128, 1 << 30), 128, 0, s>>>(sites, n_sites, n_traj, kraus, logq);
}

void launch_row_hash(const uint8_t* kraus, int64_t n, int32_t S, uint64_t* h, cudaStream_t s) {
    count_launches(K_DEDUP);
    k_row_hash<<<grid_for(n, 128, 1 << 30), 128, 0, s>>>(kraus, n, S, h);
}
void launch_first_in_run(const uint8_t* kraus, int32_t S, const int64_t* idx, const int64_t* flag, const int64_t* excl,
                         const int64_t* start, int64_t n, int64_t* first, cudaStream_t s) {
    if (n > 0) count_launches(K_DEDUP);
    if (n > 0) k_first_in_run<<<grid_for(n, 128, 1 << 30), 128, 0, s>>>(kraus, S, idx, flag, excl, start, n, first);
}
void launch_iota_i64(int64_t* p, int64_t n, cudaStream_t s) {
    if (n > 0) count_launches(K_MISC);
    if (n > 0) k_iota_i64<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(p, n);
}
void launch_flags_first(const int64_t* first, int64_t n, int64_t* flags, cudaStream_t s) {
    count_launches(K_DEDUP);
    k_flags_first<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(first, n, flags);
}
void launch_dedup_compact(const uint8_t* kraus, const double* logq, const int64_t* first, const int64_t* uid,
                          int64_t n, int32_t S, uint8_t* kraus_u, double* logq_u, int64_t* mult_u, int64_t* first_u,
                          cudaStream_t s) {
    count_launches(K_DEDUP);
    k_dedup_compact<<<grid_for(n, 128, 1 << 30), 128, 0, s>>>(kraus, logq, first, uid, n, S, kraus_u, logq_u,
                                                              reinterpret_cast<unsigned long long*>(mult_u), first_u);
}
void launch_var_ids(const uint8_t* kraus, int64_t n, int32_t S, const int32_t* ptr, const int32_t* idx,
                    const int32_t* mul, int32_t n_cols, int32_t* var_ids, cudaStream_t s) {
    if (n_cols <= 0) return;
    StatScope sc(K_VAR_IDS, s, (double)n * (S + 4.0 * n_cols), 0.0);
    k_var_ids<<<grid_for(n * n_cols, 256), 256, 0, s>>>(kraus, n, S, ptr, idx, mul, n_cols, var_ids);
}

int64_t scan_tmp_elems(int64_t n) {
    int64_t tot = 0;
    while (n > 1) {
        n = (n + kScanTile - 1) / kScanTile;
        tot += 2 * n + 2;
    }
    return tot + 2;
}

void launch_exclusive_scan(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    StatScope sc(K_SCAN, s, 16.0 * (double)n, 0.0);
    if (tiles == 1) {
        k_scan_tiles<<<1, 1024, 0, s>>>(in, out, n, nullptr);
        return;
    }
    int64_t* sums = tmp;
    int64_t* offs = tmp + tiles;
    count_launches(K_SCAN);   // the scope counts one of this level's two kernels
    k_scan_tiles<<<(unsigned)tiles, 1024, 0, s>>>(in, out, n, sums);
    launch_exclusive_scan(sums, offs, tiles, tmp + 2 * tiles + 2, s);
    k_scan_add<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(out, n, offs);
}

void launch_alloc_shots(const double* w, int64_t n, int64_t total, uint64_t seed, int32_t circuit, double* cdf_tmp,
                        int64_t* m, cudaStream_t s) {
    int bits = 0;
    while (((int64_t)1 << bits) < n) bits++;
    StatScope sc(K_ALLOC, s, (double)n * 16.0 + (double)total * 8.0, 0.0);
    k_quantise_cdf<<<1, 1024, 0, s>>>(w, n, bits, cdf_tmp);
    cudaMemsetAsync(m, 0, sizeof(int64_t) * n, s);
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if (total > 0) count_launches(K_ALLOC);
    if (total > 0)
        k_alloc_draw<<<grid_for(total, 256), 256, 0, s>>>(cdf_tmp, n, total, key,
                                                          philox_tag(STREAM_ALLOC, circuit, 0),
                                                          reinterpret_cast<unsigned long long*>(m));
}

void launch_mult_times_z(const int64_t* mult, const double* Z, int64_t n, double* w, cudaStream_t s) {
    count_launches(K_MISC);
    k_mult_times_z<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(mult, Z, n, w);
}
void launch_fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s) {
    if (n > 0) count_launches(K_MISC);
    if (n > 0) k_fill_i64<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(p, v, n);
}
void launch_iota_i32(int32_t* p, int64_t n, cudaStream_t s) {
    if (n > 0) count_launches(K_MISC);
    if (n > 0) k_iota_i32<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(p, n);
}
void launch_scale_i64(const int64_t* a, int64_t k, int64_t n, int64_t* out, cudaStream_t s) {
    if (n > 0) count_launches(K_MISC);
    if (n > 0) k_scale_i64<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(a, k, n, out);
}

int64_t run_sample_block(const float* marg, int b, int start, const int32_t* ptraj, const uint64_t* pprefix,
                         const int64_t* pcount, int64_t n_parent, int64_t n_traj_max, uint64_t seed, int circuit,
                         int block, int32_t* ctraj, uint64_t* cprefix, int64_t* ccount, int64_t child_cap,
                         const SampleScratch& sc, int64_t* host_tmp, cudaStream_t s, ptn_status* st, int n_words) {
    *st = PTN_OK;
    if (n_parent <= 0) return 0;
    cudaMemsetAsync(sc.first, 0xFF, sizeof(int64_t) * n_traj_max, s);
    count_launches(K_MISC, 2);   // k_sample_prep, k_rank0
    k_sample_prep<<<grid_for(n_parent, 256, 1 << 30), 256, 0, s>>>(pcount, n_parent, b, ptraj, sc.cap,
                                                                  reinterpret_cast<unsigned long long*>(sc.first));
    launch_exclusive_scan(sc.cap, sc.tmp_off, n_parent, sc.scan_tmp, s);
    launch_exclusive_scan(pcount, sc.excl, n_parent, sc.scan_tmp, s);
    k_rank0<<<grid_for(n_parent, 256, 1 << 30), 256, 0, s>>>(sc.excl, ptraj,
                                                            reinterpret_cast<const unsigned long long*>(sc.first),
                                                            n_parent, sc.rank0);
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    {
        StatScope st_sp(K_SAMPLE_PARENTS, s, (double)n_parent * ((double)((int64_t)1 << b) * 4.0 + 40.0), 0.0);
        if (b <= kSampWarpMaxBits) {
            // per warp: CDF (8 B) + histogram (4 B) per bin; 48 KB at 2^10 bins
            const size_t smem = (size_t)kSampWarps * (((size_t)1 << b) * (sizeof(uint64_t) + sizeof(unsigned)));
            k_sample_parents_warp<<<(unsigned)((n_parent + kSampWarps - 1) / kSampWarps), kSampWarps * 32, smem, s>>>(
                marg, b, n_parent, ptraj, pcount, sc.rank0, sc.tmp_off, child_cap, key,
                philox_tag(STREAM_SAMPLE, circuit, block), sc.tmp_x, sc.tmp_c, sc.ndist);
        } else {
            const size_t smem = (size_t)(((int64_t)1 << b) * (sizeof(uint64_t) + sizeof(unsigned int)));
            if (smem > 32 * 1024)
                cudaFuncSetAttribute(k_sample_parents, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_sample_parents<<<(unsigned)n_parent, 256, smem, s>>>(marg, b, ptraj, pcount, sc.rank0, sc.tmp_off,
                                                                   child_cap, key,
                                                                   philox_tag(STREAM_SAMPLE, circuit, block),
                                                                   sc.tmp_x, sc.tmp_c, sc.ndist);
        }
    }
    launch_exclusive_scan(sc.ndist, sc.out_off, n_parent, sc.scan_tmp, s);
    cudaMemcpyAsync(host_tmp, sc.out_off + n_parent - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(host_tmp + 1, sc.ndist + n_parent - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(host_tmp + 2, sc.tmp_off + n_parent - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(host_tmp + 3, sc.cap + n_parent - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        *st = set_error(PTN_ERR_CUDA, "sampling: %s", cudaGetErrorString(cudaGetLastError()));
        return -1;
    }
    // the temporary child slots (sum of min(count, 2^b)) share the caller's
    // capacity; the kernel skipped slots beyond it, so the result is incomplete
    const int64_t slots = host_tmp[2] + host_tmp[3];
    if (slots > child_cap) {
        *st = set_error(PTN_ERR_INVALID_ARG, "child capacity %lld < sum of min(count, 2^b) = %lld",
                        (long long)child_cap, (long long)slots);
        return -1;
    }
    const int64_t n_child = host_tmp[0] + host_tmp[1];
    StatScope st_em(K_EMIT, s, (double)n_child * 32.0, 0.0);
    k_emit_children<<<grid_for(n_parent * 32, 256, 1 << 30), 256, 0, s>>>(ptraj, pprefix, sc.tmp_off, sc.ndist,
                                                                          sc.out_off, sc.tmp_x, sc.tmp_c, start,
                                                                          n_parent, n_words, ctraj, cprefix, ccount);
    return n_child;
}

}  // namespace ptn
