// Final-block harvest of non-proportional NBS (Sec. III-B): the last block's
// outcomes feed no later contraction, so its 2^{b_f} population vector is
// harvested in bulk, by direct sampling (many shots drawn from it) or
// exhaustively (every entry above a threshold, with its probability).
//
// Population vector of a network: P_x = rint(max(p_x, 0) 2^s) as 64-bit
// integers, s = 62 - b - e with max p = f 2^e, f in [0.5, 1); T = sum P_x <
// 2^62 is exact in any summation order (integer adds), so every decision
// below is bit-reproducible:
//  * exhaustive: keep x iff P_x > 0 and (double)P_x >= tau * (double)T, with
//    probability (double)P_x / (double)T;
//  * direct: shot rank r of the network's trajectory draws a = x0 << 32 | x1
//    from Philox4x32-10 counter (r_lo, r_hi, traj, (3 << 24)|(circuit << 8)|
//    block), r' = floor(a T / 2^64), x = smallest with r' < C[x] (C the
//    running sum of P).  The search is two-level: a binary search over the
//    running sums of 256-entry tiles, then one warp scans the tile (eight
//    entries per lane, a warp-shuffle scan of the lane sums and a ballot for
//    the first lane whose running sum exceeds r').
// Records are written in canonical order (networks in order, x increasing) by
// an ordered compaction: per 4096-entry tile a count, one exclusive scan, then
// a block-level scan of the per-thread counts for the write positions.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

constexpr int kHThreads = 256, kHPer = 16, kHTile = kHThreads * kHPer;   // compaction / sums tile
constexpr int kDTile = 256;                                              // CDF tile of direct draws

__device__ __forceinline__ int pop_shift(unsigned rowmax_bits, int b) {
    return 62 - b - frexp_exp(__uint_as_float(rowmax_bits));
}

// rint(max(p, 0) 2^s) in integer arithmetic (quant_pow2: the FP64 value, exactly)
__device__ __forceinline__ uint64_t pop_weight(float p, int s) { return quant_pow2(p, s); }

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ int64_t warp_incl_scan_i64(int64_t v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// rowmax[net] = largest entry (non-negative float bits order like unsigned ints)
__global__ void __launch_bounds__(kHThreads) k_row_max(const float* __restrict__ marg, int b, int64_t tiles,
                                                       unsigned* __restrict__ rowmax) {
    const int64_t net = blockIdx.x / tiles, tile = blockIdx.x - net * tiles;
    const int64_t nx = (int64_t)1 << b;
    const float* p = marg + net * nx;
    float m = 0.f;
    const int64_t x0 = tile * kHTile + (int64_t)threadIdx.x * kHPer;
    for (int k = 0; k < kHPer; k++)
        if (x0 + k < nx) m = fmaxf(m, p[x0 + k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&rowmax[net], __float_as_uint(m));
}

// T[net] += sum of P over the tile; with tsum, also the sums of the 256-entry
// CDF tiles (16 threads each)
__global__ void __launch_bounds__(kHThreads) k_pop_sums(const float* __restrict__ marg, int b, int64_t tiles,
                                                        const unsigned* __restrict__ rowmax,
                                                        unsigned long long* __restrict__ T, uint64_t* __restrict__ tsum,
                                                        int64_t tiles256) {
    const int64_t net = blockIdx.x / tiles, tile = blockIdx.x - net * tiles;
    const unsigned mb = rowmax[net];
    if (mb == 0u) return;                      // zero row: T stays 0
    const int s = pop_shift(mb, b);
    const int64_t nx = (int64_t)1 << b;
    const float* p = marg + net * nx;
    const int64_t x0 = tile * kHTile + (int64_t)threadIdx.x * kHPer;
    uint64_t acc = 0;
    for (int k = 0; k < kHPer; k++)
        if (x0 + k < nx) acc += pop_weight(p[x0 + k], s);
    if (tsum) {
        uint64_t t16 = acc;
        for (int o = 8; o > 0; o >>= 1) t16 += __shfl_xor_sync(0xffffffffu, t16, o);
        const int64_t t = x0 / kDTile;
        if ((threadIdx.x & 15) == 0 && x0 < nx) tsum[net * tiles256 + t] = t16;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&T[net], (unsigned long long)acc);
}

// in-place inclusive running sum of every network's 256-entry tile sums
__global__ void __launch_bounds__(1024) k_tile_cdf(uint64_t* __restrict__ tsum, int64_t tiles256) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t carry;
    uint64_t* t = tsum + (int64_t)blockIdx.x * tiles256;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < tiles256; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = i < tiles256 ? t[i] : 0;
        uint64_t inc = warp_incl_scan_u64(v);
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint64_t w = threadIdx.x < blockDim.x / 32 ? wsum[threadIdx.x] : 0;
            wsum[threadIdx.x] = warp_incl_scan_u64(w);
        }
        __syncthreads();
        const uint64_t before = (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0) + carry;
        if (i < tiles256) t[i] = before + inc;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[blockDim.x / 32 - 1];
        __syncthreads();
    }
}

// first[traj] = smallest network index of each trajectory (for shot ranks)
__global__ void k_first_net(const int32_t* __restrict__ traj, int64_t n, unsigned long long* __restrict__ first) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMin(&first[traj[i]], (unsigned long long)i);
}
__global__ void k_rank0_uniform(const int32_t* __restrict__ traj, const unsigned long long* __restrict__ first,
                                int64_t n, int64_t shots, int64_t* __restrict__ rank0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rank0[i] = (i - (int64_t)first[traj[i]]) * shots;
}

// one warp per draw: Philox word, two-level inverse CDF, histogram
__global__ void __launch_bounds__(256) k_direct_draws(const float* __restrict__ marg, int b, int64_t n_net,
                                                      const unsigned* __restrict__ rowmax,
                                                      const unsigned long long* __restrict__ T,
                                                      const uint64_t* __restrict__ tcdf, int64_t tiles256,
                                                      const int32_t* __restrict__ traj,
                                                      const int64_t* __restrict__ rank0, int64_t shots, uint2 key,
                                                      uint32_t tagw, unsigned* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nx = (int64_t)1 << b;
    const int64_t total = n_net * shots;
    for (int64_t d = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < total; d += warps) {
        const int64_t net = d / shots, k = d - net * shots;
        const uint64_t Tn = T[net];
        if (Tn == 0) continue;                 // zero-norm network: its shots cannot be drawn
        const uint64_t rank = (uint64_t)(rank0[net] + k);
        const uint4 w = philox4x32_10(make_uint4((uint32_t)rank, (uint32_t)(rank >> 32), (uint32_t)traj[net], tagw),
                                      key);
        const uint64_t r = __umul64hi(word64(w), Tn);
        const uint64_t* C = tcdf + net * tiles256;
        int64_t lo = 0, hi = tiles256 - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (r < C[mid]) hi = mid;
            else lo = mid + 1;
        }
        const uint64_t rr = r - (lo ? C[lo - 1] : 0);
        const int s = pop_shift(rowmax[net], b);
        const float* p = marg + net * nx + lo * kDTile + lane * 8;
        const int64_t xl = lo * kDTile + lane * 8;
        uint64_t P[8], ls = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            P[i] = xl + i < nx ? pop_weight(p[i], s) : 0;
            ls += P[i];
        }
        const uint64_t inc = warp_incl_scan_u64(ls);
        const unsigned hit = __ballot_sync(0xffffffffu, rr < inc);
        if (hit && lane == __ffs(hit) - 1) {
            uint64_t acc = inc - ls;
            int i = 0;
            for (; i < 7; i++) {
                acc += P[i];
                if (rr < acc) break;
            }
            atomicAdd(&cnt[net * nx + xl + i], 1u);
        }
    }
}

template <bool kDirect>
__device__ __forceinline__ bool keep_entry(const float* p, const unsigned* cnt, int64_t x, int s, double thr) {
    if (kDirect) return cnt[x] != 0u;
    const uint64_t P = pop_weight(p[x], s);
    return P != 0 && (double)P >= thr;
}

// records per 4096-entry tile
template <bool kDirect>
__global__ void __launch_bounds__(kHThreads) k_harvest_count(const float* __restrict__ marg, int b, int64_t tiles,
                                                             const unsigned* __restrict__ rowmax,
                                                             const unsigned long long* __restrict__ T, double tau,
                                                             const unsigned* __restrict__ cnt,
                                                             int64_t* __restrict__ tcnt) {
    __shared__ int64_t red[kHThreads / 32];
    const int64_t net = blockIdx.x / tiles, tile = blockIdx.x - net * tiles;
    const int64_t nx = (int64_t)1 << b;
    const unsigned mb = rowmax[net];
    int64_t c = 0;
    if (mb != 0u) {
        const int s = pop_shift(mb, b);
        const double thr = tau * (double)T[net];
        const int64_t x0 = tile * kHTile + (int64_t)threadIdx.x * kHPer;
        const float* p = marg + net * nx;
        const unsigned* cn = kDirect ? cnt + net * nx : nullptr;
        for (int k = 0; k < kHPer; k++)
            if (x0 + k < nx && keep_entry<kDirect>(p, cn, x0 + k, s, thr)) c++;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kHThreads / 32; w++) t += red[w];
        tcnt[blockIdx.x] = t;
    }
}

// ordered write of the kept entries: (traj, prefix | x << start, count, P / T)
template <bool kDirect>
__global__ void __launch_bounds__(kHThreads) k_harvest_write(const float* __restrict__ marg, int b, int start,
                                                             int64_t tiles, const unsigned* __restrict__ rowmax,
                                                             const unsigned long long* __restrict__ T, double tau,
                                                             const unsigned* __restrict__ cnt,
                                                             const int64_t* __restrict__ toff,
                                                             const int32_t* __restrict__ traj,
                                                             const uint64_t* __restrict__ prefix, int n_words,
                                                             int32_t* __restrict__ otraj, uint64_t* __restrict__ obits,
                                                             int64_t* __restrict__ ocount, double* __restrict__ oprob) {
    __shared__ int64_t wtot[kHThreads / 32];
    const int64_t net = blockIdx.x / tiles, tile = blockIdx.x - net * tiles;
    const int64_t nx = (int64_t)1 << b;
    const unsigned mb = rowmax[net];
    if (mb == 0u) return;
    const int s = pop_shift(mb, b);
    const double Td = (double)T[net];
    const double thr = tau * Td;
    const int64_t x0 = tile * kHTile + (int64_t)threadIdx.x * kHPer;
    const float* p = marg + net * nx;
    const unsigned* cn = kDirect ? cnt + net * nx : nullptr;
    unsigned mask = 0;
    for (int k = 0; k < kHPer; k++)
        if (x0 + k < nx && keep_entry<kDirect>(p, cn, x0 + k, s, thr)) mask |= 1u << k;
    const int64_t c = __popc(mask);
    const int64_t inc = warp_incl_scan_i64(c);
    if ((threadIdx.x & 31) == 31) wtot[threadIdx.x >> 5] = inc;
    __syncthreads();
    int64_t pos = toff[blockIdx.x] + inc - c;
    for (int w = 0; w < (int)(threadIdx.x >> 5); w++) pos += wtot[w];
    const int32_t t = traj[net];
    const uint64_t* pre = prefix + net * n_words;
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1;
        const int64_t x = x0 + k;
        otraj[pos] = t;
        if (n_words == 1) obits[pos] = pre[0] | ((uint64_t)x << start);
        else bits_put(obits + pos * n_words, pre, n_words, (uint64_t)x, start);
        ocount[pos] = kDirect ? (int64_t)cn[x] : 1;
        oprob[pos] = (double)pop_weight(p[x], s) / Td;
        pos++;
    }
}

inline unsigned grid1(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int64_t harvest_tiles(int b) { return (((int64_t)1 << b) + kHTile - 1) / kHTile; }
int64_t harvest_cdf_tiles(int b) { return (((int64_t)1 << b) + kDTile - 1) / kDTile; }

void launch_harvest_ranks(const int32_t* traj, int64_t n, int64_t n_traj_max, int64_t shots, unsigned long long* first,
                          int64_t* rank0, cudaStream_t s) {
    if (n <= 0) return;
    cudaMemsetAsync(first, 0xFF, sizeof(unsigned long long) * n_traj_max, s);
    count_launches(K_HARVEST, 2);
    k_first_net<<<grid1(n, 256), 256, 0, s>>>(traj, n, first);
    k_rank0_uniform<<<grid1(n, 256), 256, 0, s>>>(traj, first, n, shots, rank0);
}

int64_t run_harvest_count(const HarvestArgs& a, const HarvestScratch& h, int64_t* host_tmp, cudaStream_t s,
                          ptn_status* st) {
    *st = PTN_OK;
    const int64_t tiles = harvest_tiles(a.b), tiles256 = harvest_cdf_tiles(a.b);
    const int64_t nx = (int64_t)1 << a.b;
    const unsigned grid = (unsigned)(a.n_net * tiles);
    cudaMemsetAsync(h.rowmax, 0, sizeof(unsigned) * a.n_net, s);
    cudaMemsetAsync(h.T, 0, sizeof(unsigned long long) * a.n_net, s);
    {
        StatScope sc(K_HARVEST, s, 8.0 * (double)a.n_net * (double)nx, 0.0);
        count_launches(K_HARVEST);   // two kernels under one scope
        k_row_max<<<grid, kHThreads, 0, s>>>(a.marg, a.b, tiles, h.rowmax);
        k_pop_sums<<<grid, kHThreads, 0, s>>>(a.marg, a.b, tiles, h.rowmax, h.T, a.direct ? h.tcdf : nullptr,
                                               tiles256);
    }
    if (a.direct) {
        StatScope sc(K_HARVEST, s, 16.0 * (double)a.n_net * (double)tiles256 + 8.0 * (double)a.n_net * (double)nx +
                                       1024.0 * (double)a.n_net * (double)a.shots, 0.0);
        count_launches(K_HARVEST);
        k_tile_cdf<<<(unsigned)a.n_net, 1024, 0, s>>>(h.tcdf, tiles256);
        cudaMemsetAsync(h.cnt, 0, sizeof(unsigned) * a.n_net * nx, s);
        const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        int64_t blocks = (a.n_net * a.shots + 7) / 8;
        if (blocks > 152 * 32) blocks = 152 * 32;
        if (blocks < 1) blocks = 1;
        k_direct_draws<<<(unsigned)blocks, 256, 0, s>>>(a.marg, a.b, a.n_net, h.rowmax, h.T, h.tcdf, tiles256, a.traj,
                                                        a.rank0, a.shots, key,
                                                        philox_tag(STREAM_SAMPLE, a.circuit, a.block), h.cnt);
    }
    {
        StatScope sc(K_HARVEST, s, (a.direct ? 8.0 : 4.0) * (double)a.n_net * (double)nx, 0.0);
        if (a.direct)
            k_harvest_count<true><<<grid, kHThreads, 0, s>>>(a.marg, a.b, tiles, h.rowmax, h.T, a.tau, h.cnt, h.tcnt);
        else
            k_harvest_count<false><<<grid, kHThreads, 0, s>>>(a.marg, a.b, tiles, h.rowmax, h.T, a.tau, h.cnt,
                                                               h.tcnt);
    }
    launch_exclusive_scan(h.tcnt, h.toff, a.n_net * tiles, h.scan_tmp, s);
    cudaMemcpyAsync(host_tmp, h.toff + a.n_net * tiles - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(host_tmp + 1, h.tcnt + a.n_net * tiles - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *st = set_error(PTN_ERR_CUDA, "harvest: %s", cudaGetErrorString(e));
        return -1;
    }
    return host_tmp[0] + host_tmp[1];
}

void run_harvest_write(const HarvestArgs& a, const HarvestScratch& h, int32_t* otraj, uint64_t* obits, int64_t* ocount,
                       double* oprob, cudaStream_t s) {
    const int64_t tiles = harvest_tiles(a.b);
    const unsigned grid = (unsigned)(a.n_net * tiles);
    StatScope sc(K_HARVEST, s, (a.direct ? 8.0 : 4.0) * (double)a.n_net * (double)((int64_t)1 << a.b), 0.0);
    if (a.direct)
        k_harvest_write<true><<<grid, kHThreads, 0, s>>>(a.marg, a.b, a.start, tiles, h.rowmax, h.T, a.tau, h.cnt,
                                                         h.toff, a.traj, a.prefix, a.n_words, otraj, obits, ocount, oprob);
    else
        k_harvest_write<false><<<grid, kHThreads, 0, s>>>(a.marg, a.b, a.start, tiles, h.rowmax, h.T, a.tau, h.cnt,
                                                          h.toff, a.traj, a.prefix, a.n_words, otraj, obits, ocount, oprob);
}

}  // namespace ptn
