// Intermediate caching across error sets (Sec. VI: regions of the network
// whose error choices do not change between error sets need not be
// recomputed).  A cached step's output depends only on the variants a
// trajectory takes at the step's columns (StepDesc.cache, BlockPlan.cache_bits).
// Per chunk and cache slot these kernels give every local trajectory tl its
// representative: the first trajectory of the chunk with the same variants on
// the slot's columns.  Keys are 128-bit: two independent sums, over the
// trajectory's non-baseline variant entries (column, variant) inside the
// slot's columns, of a 64-bit mixer; the first 64 bits index a first-occurrence
// hash table and the representative is taken only if the second 64 bits agree
// too (otherwise the trajectory is its own representative), so a wrong share
// needs a 128-bit collision.
#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

// The splitmix64 output function (Steele, Lea and Flood 2014, with the
// constants of Vigna's splitmix64): a bijective 64-bit mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
constexpr unsigned long long kEmptyKey = ~0ull;

// Non-baseline (non-zero) variant entries per trajectory: one warp per
// trajectory row of var_ids, lanes over consecutive columns.
__global__ void k_nz_count(const int32_t* __restrict__ var_ids, int64_t n, int32_t n_cols,
                           int64_t* __restrict__ cnt) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t > n) return;
    if (t == n) {   // the scan's last entry
        if (lane == 0) cnt[n] = 0;
        return;
    }
    const int32_t* row = var_ids + t * n_cols;
    int64_t c = 0;
    for (int32_t b = 0; b < n_cols; b += 32) {
        const bool nz = b + lane < n_cols && row[b + lane] != 0;
        c += __popc(__ballot_sync(0xffffffffu, nz));
    }
    if (lane == 0) cnt[t] = c;
}

__global__ void k_nz_fill(const int32_t* __restrict__ var_ids, int64_t n, int32_t n_cols,
                          const int64_t* __restrict__ ptr, int32_t* __restrict__ col, int32_t* __restrict__ val) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int32_t* row = var_ids + t * n_cols;
    int64_t o = ptr[t];
    for (int32_t b = 0; b < n_cols; b += 32) {
        const int32_t v = b + lane < n_cols ? row[b + lane] : 0;
        const unsigned m = __ballot_sync(0xffffffffu, v != 0);
        if (v != 0) {
            const int64_t at = o + __popc(m & ((1u << lane) - 1u));
            col[at] = b + lane;
            val[at] = v;
        }
        o += __popc(m);
    }
}

// Thread (k, tl): the two key halves of trajectory tl under slot k, and the
// insertion of the first half into slot k's table (the smallest tl wins).
__global__ void k_cache_keys(CacheArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.n_cache * a.n) return;
    const int64_t k = idx / a.n, tl = idx - k * a.n;
    const int64_t g = a.chunk_traj[tl];
    const uint32_t* bits = a.bits + k * a.words;
    uint64_t h1 = 0, h2 = 0;
    for (int64_t e = a.nz_ptr[g], e1 = a.nz_ptr[g + 1]; e < e1; e++) {
        const int32_t col = a.nz_col[e];
        if ((bits[col >> 5] >> (col & 31)) & 1u) {
            const uint64_t x = ((uint64_t)(uint32_t)col << 32) | (uint32_t)a.nz_val[e];
            h1 += mix64(x ^ 0x243f6a8885a308d3ull);
            h2 += mix64(x + 0x13198a2e03707344ull);
        }
    }
    if (h1 == kEmptyKey) h1 = kEmptyKey - 1;
    a.h[2 * idx] = h1;
    a.h[2 * idx + 1] = h2;
    unsigned long long* key = a.keys + k * a.P;
    int32_t* first = a.first + k * a.P;
    uint64_t slot = mix64(h1) & (uint64_t)(a.P - 1);
    for (int64_t it = 0; it < a.P; it++) {   // at most half the table is ever full
        const unsigned long long old = atomicCAS(key + slot, kEmptyKey, (unsigned long long)h1);
        if (old == kEmptyKey || old == h1) {
            atomicMin(first + slot, (int32_t)tl);
            break;
        }
        slot = (slot + 1) & (uint64_t)(a.P - 1);
    }
}

// Thread (k, tl): rep[k][tl] = the smallest trajectory inserted under tl's
// first key half if its second half agrees, else tl.
__global__ void k_cache_rep(CacheArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.n_cache * a.n) return;
    const int64_t k = idx / a.n, tl = idx - k * a.n;
    const uint64_t h1 = a.h[2 * idx], h2 = a.h[2 * idx + 1];
    const unsigned long long* key = a.keys + k * a.P;
    const int32_t* first = a.first + k * a.P;
    uint64_t slot = mix64(h1) & (uint64_t)(a.P - 1);
    int64_t r = tl;
    for (int64_t it = 0; it < a.P; it++) {
        const unsigned long long kk = key[slot];
        if (kk == h1) {
            const int64_t m = first[slot];
            if (m >= 0 && m < a.n && a.h[2 * (k * a.n + m) + 1] == h2) r = m;
            break;
        }
        if (kk == kEmptyKey) break;
        slot = (slot + 1) & (uint64_t)(a.P - 1);
    }
    a.rep[idx] = (int32_t)r;
}

// One CTA of 1024 threads per slot: the representatives (rep[k][tl] == tl) in
// increasing order, by ballot and a scan of the 32 warp counts.
constexpr int kListThreads = 1024;
__global__ void __launch_bounds__(kListThreads) k_cache_list(CacheArgs a) {
    __shared__ int32_t wsum[32];
    __shared__ int64_t base;
    const int64_t k = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < a.n; t0 += kListThreads) {
        const int64_t tl = t0 + threadIdx.x;
        const bool own = tl < a.n && a.rep[k * a.n + tl] == tl;
        const unsigned m = __ballot_sync(0xffffffffu, own);
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        if (w == 0) {
            int32_t v = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            wsum[lane] = v;   // inclusive
        }
        __syncthreads();
        if (own) a.list[k * a.n + base + (w ? wsum[w - 1] : 0) + __popc(m & ((1u << lane) - 1u))] = (int32_t)tl;
        __syncthreads();
        if (threadIdx.x == 0) base += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.cnt[k] = (int32_t)base;
}

}  // namespace

void launch_nz_count(const int32_t* var_ids, int64_t n, int32_t n_cols, int64_t* cnt, cudaStream_t s) {
    StatScope sc(K_MISC, s, 4.0 * (double)n * n_cols);
    const int64_t threads = 32 * (n + 1);
    k_nz_count<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(var_ids, n, n_cols, cnt);
}

void launch_nz_fill(const int32_t* var_ids, int64_t n, int32_t n_cols, const int64_t* ptr, int32_t* col,
                    int32_t* val, cudaStream_t s) {
    if (n <= 0) return;
    StatScope sc(K_MISC, s, 4.0 * (double)n * n_cols);
    const int64_t threads = 32 * n;
    k_nz_fill<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(var_ids, n, n_cols, ptr, col, val);
}

void launch_cache_tables(const CacheArgs& a, cudaStream_t s) {
    if (a.n_cache <= 0 || a.n <= 0) return;
    StatScope sc(K_CACHE, s, 16.0 * (double)a.n_cache * a.n);
    cudaMemsetAsync(a.keys, 0xFF, sizeof(unsigned long long) * (size_t)a.n_cache * (size_t)a.P, s);
    cudaMemsetAsync(a.first, 0x7F, sizeof(int32_t) * (size_t)a.n_cache * (size_t)a.P, s);
    const int64_t tot = (int64_t)a.n_cache * a.n;
    const unsigned grid = (unsigned)((tot + 255) / 256);
    k_cache_keys<<<grid, 256, 0, s>>>(a);
    k_cache_rep<<<grid, 256, 0, s>>>(a);
    k_cache_list<<<(unsigned)a.n_cache, kListThreads, 0, s>>>(a);
    count_launches(K_CACHE, 2);   // three kernels under one scope
}

}  // namespace ptn
