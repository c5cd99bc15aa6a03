// Batched pairwise contraction of block networks (the execution of one path
// step of P^j for every network of a chunk, Sec. III-A) and the marginal
// finalisation of the block's root tensor (Sec. II-B).
//
// k_contract_direct: each output element of one instance is one thread's
// accumulation; the element's operand addresses come from the step's per-bit
// stride tables, so any bit layout of either operand is read without a
// separate permutation pass.  The first operand read of a merged-gate leaf goes through the
// trajectory's variant index: the UPV merge happens as a gather fused into its
// first consumer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

__device__ __forceinline__ const float2* operand_ptr(const OperandDesc& d, int out_cls, int64_t inst,
                                                     const ChunkCtx& c) {
    int64_t tl = 0, net = 0;
    if (out_cls == CLS_NET) {
        net = inst;
        tl = c.net_tl[inst];
    } else if (out_cls == CLS_TRAJ) {
        tl = inst;
    }
    const float2* p;
    if (d.mode == OP_LEAF) {
        int64_t var = 0;
        if (d.leaf_col >= 0) {
            const int64_t g = c.chunk_traj[tl];
            var = c.var_ids[g * c.n_var_cols + d.leaf_col];
        }
        p = c.vtab + d.leaf_base + var * d.inst_size;
    } else {
        const int64_t oi = d.cls == CLS_CONST ? 0 : (d.cls == CLS_TRAJ ? rep_inst(d, tl, c) : net);
        p = c.arena[d.arena] + d.arena_off * c.arena_inst[d.arena] + oi * d.inst_size;
    }
    if (d.n_slice) {
        const uint64_t* pre = c.net_prefix + net * c.n_words;
        int64_t off = 0;
        for (int s = 0; s < d.n_slice; s++) off += (int64_t)bits_get(pre, d.slice_qubit[s]) * d.slice_stride[s];
        p += off;
    }
    return p;
}

// A warp takes tiles of 128 consecutive outputs (instance-major), four per
// lane (lane, lane + 32, ...): four independent accumulation chains, and each
// store instruction of the warp covers 32 consecutive outputs.  Offsets of the
// low 8 output bits and of the low 8 summed bits come from per-block tables;
// higher summed bits are walked in Gray-code order.  OffT is int32_t when
// every in-instance offset fits (the usual case), halving the address math.
constexpr int kDirThreads = 256;
constexpr int kDirU = 4;
template <typename OffT>
__global__ void __launch_bounds__(kDirThreads, 3) k_contract_direct(const StepDesc* __restrict__ gstep, const __grid_constant__ ChunkCtx c,
                                                                 int64_t n_inst) {
    __shared__ __align__(16) StepDesc s;
    {
        const int4* src = reinterpret_cast<const int4*>(gstep);
        int4* dst = reinterpret_cast<int4*>(&s);
        for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    __shared__ OffT otab[2][256];
    __shared__ OffT ktab[2][256];
    const int lowb = s.n_out < 8 ? s.n_out : 8;
    const int nk = s.n_sum;
    const int klo = nk < 8 ? nk : 8;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) {
        OffT a = 0, b = 0, ka = 0, kb = 0;
        for (int p = 0; p < lowb; p++)
            if ((t >> p) & 1) {
                a += (OffT)s.out_stride[0][p];
                b += (OffT)s.out_stride[1][p];
            }
        for (int p = 0; p < klo; p++)
            if ((t >> p) & 1) {
                ka += (OffT)s.sum_stride[0][p];
                kb += (OffT)s.sum_stride[1][p];
            }
        otab[0][t] = a;
        otab[1][t] = b;
        ktab[0][t] = ka;
        ktab[1][t] = kb;
    }
    __syncthreads();
    const int64_t total = n_inst << s.n_out;
    const int64_t mask = s.out_size - 1;
    const int lowmask = (1 << lowb) - 1;
    const int n_lo = 1 << klo;
    const int64_t n_hi = (int64_t)1 << (nk - klo);
    const float sa = s.op[0].conj ? -1.f : 1.f, sb = s.op[1].conj ? -1.f : 1.f;
    float2* outbase = c.arena[s.out_arena] + s.out_off * c.arena_inst[s.out_arena];
    const int lane = threadIdx.x & 31;
    const int64_t n_tiles = (total + 32 * kDirU - 1) / (32 * kDirU);
    const int64_t warps = (int64_t)gridDim.x * (kDirThreads / 32);
    // A cached step runs over the chunk's representatives: instance i writes
    // trajectory step_inst(i), odelta = (that - i) << n_out (cached steps have
    // n_out >= 7, so a tile of 128 outputs lies within one instance).
    int64_t cur_inst = -1, cur_hi = -1, odelta = 0;
    OffT hia = 0, hib = 0;
    const float2 *A = nullptr, *B = nullptr;
    for (int64_t tile = (int64_t)blockIdx.x * (kDirThreads / 32) + (threadIdx.x >> 5); tile < n_tiles; tile += warps) {
        const float2* pa[kDirU];
        const float2* pb[kDirU];
        float2 acc[kDirU];
#pragma unroll
        for (int u = 0; u < kDirU; u++) {
            acc[u] = make_float2(0.f, 0.f);
            const int64_t g = tile * (32 * kDirU) + u * 32 + lane;
            const int64_t gg = g < total ? g : total - 1;     // tail lanes compute a valid dummy
            const int64_t inst = gg >> s.n_out;
            const int64_t o = gg & mask;
            if (inst != cur_inst) {
                const int64_t tl = step_inst(s.cache, inst, c);
                odelta = (tl - inst) << s.n_out;
                A = operand_ptr(s.op[0], s.out_cls, tl, c);
                B = operand_ptr(s.op[1], s.out_cls, tl, c);
                cur_inst = inst;
            }
            const int64_t hi = o >> lowb;
            if (hi != cur_hi) {
                hia = hib = 0;
                for (int p = lowb; p < s.n_out; p++)
                    if ((o >> p) & 1) {
                        hia += (OffT)s.out_stride[0][p];
                        hib += (OffT)s.out_stride[1][p];
                    }
                cur_hi = hi;
            }
            pa[u] = A + (hia + otab[0][o & lowmask]);
            pb[u] = B + (hib + otab[1][o & lowmask]);
        }
        OffT ha = 0, hb = 0;
        for (int64_t th = 0; th < n_hi; th++) {
            if (th) {
                const int bit = __ffsll(th) - 1;
                const int64_t gray = th ^ (th >> 1);
                const OffT da = (OffT)s.sum_stride[0][klo + bit], db = (OffT)s.sum_stride[1][klo + bit];
                if ((gray >> bit) & 1) {
                    ha += da;
                    hb += db;
                } else {
                    ha -= da;
                    hb -= db;
                }
            }
            for (int tl = 0; tl < n_lo; tl++) {
                const OffT ka = ha + ktab[0][tl], kb = hb + ktab[1][tl];
#pragma unroll
                for (int u = 0; u < kDirU; u++) {
                    const float2 x = pa[u][ka], y = pb[u][kb];
                    const float xi = sa * x.y, yi = sb * y.y;
                    acc[u].x = fmaf(x.x, y.x, acc[u].x);
                    acc[u].x = fmaf(-xi, yi, acc[u].x);
                    acc[u].y = fmaf(x.x, yi, acc[u].y);
                    acc[u].y = fmaf(xi, y.x, acc[u].y);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kDirU; u++) {
            const int64_t g = tile * (32 * kDirU) + u * 32 + lane;
            if (g < total) outbase[g + odelta] = acc[u];
        }
    }
}

// Register-tiled variant: a thread computes a 2^RA x 2^RB micro-tile of
// outputs spanned by RA output bits along which only A varies and RB bits
// along which only B varies, so every term loads 2^RA + 2^RB operand values
// for 2^(RA+RB) complex multiply-adds.  The remaining output bits (the tile
// origin) run over the lanes, lowest first.
struct MicroBits {
    int32_t ta[2], tb[2];      // output bits of the micro-tile (A-only, B-only)
    int32_t ins[4];            // the same bits in ascending order (zero insertion)
    int32_t n_ins;
};
template <int RA, int RB>
__global__ void __launch_bounds__(kDirThreads, 2) k_contract_micro(const StepDesc* __restrict__ gstep, const __grid_constant__ ChunkCtx c,
                                                                   int64_t n_inst, const MicroBits mb) {
    __shared__ __align__(16) StepDesc s;
    {
        const int4* src = reinterpret_cast<const int4*>(gstep);
        int4* dst = reinterpret_cast<int4*>(&s);
        for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    __shared__ int32_t otab[2][256];
    __shared__ int32_t ktab[2][256];
    const int lowb = s.n_out < 8 ? s.n_out : 8;
    const int nk = s.n_sum;
    const int klo = nk < 8 ? nk : 8;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) {
        int32_t a = 0, b = 0, ka = 0, kb = 0;
        for (int p = 0; p < lowb; p++)
            if ((t >> p) & 1) {
                a += (int32_t)s.out_stride[0][p];
                b += (int32_t)s.out_stride[1][p];
            }
        for (int p = 0; p < klo; p++)
            if ((t >> p) & 1) {
                ka += (int32_t)s.sum_stride[0][p];
                kb += (int32_t)s.sum_stride[1][p];
            }
        otab[0][t] = a;
        otab[1][t] = b;
        ktab[0][t] = ka;
        ktab[1][t] = kb;
    }
    __syncthreads();
    constexpr int NA = 1 << RA, NB = 1 << RB;
    int32_t da[NA], db[NB];
    int64_t doa[NA], dob[NB];
#pragma unroll
    for (int i = 0; i < NA; i++) {
        da[i] = 0;
        doa[i] = 0;
#pragma unroll
        for (int j = 0; j < RA; j++)
            if ((i >> j) & 1) {
                da[i] += (int32_t)s.out_stride[0][mb.ta[j]];
                doa[i] += (int64_t)1 << mb.ta[j];
            }
    }
#pragma unroll
    for (int i = 0; i < NB; i++) {
        db[i] = 0;
        dob[i] = 0;
#pragma unroll
        for (int j = 0; j < RB; j++)
            if ((i >> j) & 1) {
                db[i] += (int32_t)s.out_stride[1][mb.tb[j]];
                dob[i] += (int64_t)1 << mb.tb[j];
            }
    }
    const int nq = s.n_out - RA - RB;
    const int64_t total = n_inst << nq;
    const int64_t qmask = ((int64_t)1 << nq) - 1;
    const int lowmask = (1 << lowb) - 1;
    const int n_lo = 1 << klo;
    const int64_t n_hi = (int64_t)1 << (nk - klo);
    const float sa = s.op[0].conj ? -1.f : 1.f, sb = s.op[1].conj ? -1.f : 1.f;
    float2* outbase = c.arena[s.out_arena] + s.out_off * c.arena_inst[s.out_arena];
    int64_t cur_inst = -1, cur_hi = -1, cur_tl = 0;
    int32_t hia = 0, hib = 0;
    const float2 *A = nullptr, *B = nullptr;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t inst = g >> nq;
        int64_t o = g & qmask;
        for (int z = 0; z < mb.n_ins; z++) {
            const int cbit = mb.ins[z];
            o = ((o >> cbit) << (cbit + 1)) | (o & (((int64_t)1 << cbit) - 1));
        }
        if (inst != cur_inst) {
            cur_tl = step_inst(s.cache, inst, c);   // a cached step runs over representatives
            A = operand_ptr(s.op[0], s.out_cls, cur_tl, c);
            B = operand_ptr(s.op[1], s.out_cls, cur_tl, c);
            cur_inst = inst;
        }
        const int64_t hi = o >> lowb;
        if (hi != cur_hi) {
            hia = hib = 0;
            for (int p = lowb; p < s.n_out; p++)
                if ((o >> p) & 1) {
                    hia += (int32_t)s.out_stride[0][p];
                    hib += (int32_t)s.out_stride[1][p];
                }
            cur_hi = hi;
        }
        const float2* pa = A + (hia + otab[0][o & lowmask]);
        const float2* pb = B + (hib + otab[1][o & lowmask]);
        float2 acc[NA][NB];
#pragma unroll
        for (int i = 0; i < NA; i++)
#pragma unroll
            for (int j = 0; j < NB; j++) acc[i][j] = make_float2(0.f, 0.f);
        int32_t ha = 0, hb = 0;
        for (int64_t th = 0; th < n_hi; th++) {
            if (th) {
                const int bit = __ffsll(th) - 1;
                const int64_t gray = th ^ (th >> 1);
                const int32_t dka = (int32_t)s.sum_stride[0][klo + bit], dkb = (int32_t)s.sum_stride[1][klo + bit];
                if ((gray >> bit) & 1) {
                    ha += dka;
                    hb += dkb;
                } else {
                    ha -= dka;
                    hb -= dkb;
                }
            }
            for (int tl = 0; tl < n_lo; tl++) {
                const int32_t ka = ha + ktab[0][tl], kb = hb + ktab[1][tl];
                float2 av[NA], bv[NB];
#pragma unroll
                for (int i = 0; i < NA; i++) {
                    av[i] = pa[da[i] + ka];
                    av[i].y *= sa;
                }
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    bv[j] = pb[db[j] + kb];
                    bv[j].y *= sb;
                }
#pragma unroll
                for (int i = 0; i < NA; i++)
#pragma unroll
                    for (int j = 0; j < NB; j++) {
                        acc[i][j].x = fmaf(av[i].x, bv[j].x, acc[i][j].x);
                        acc[i][j].x = fmaf(-av[i].y, bv[j].y, acc[i][j].x);
                        acc[i][j].y = fmaf(av[i].x, bv[j].y, acc[i][j].y);
                        acc[i][j].y = fmaf(av[i].y, bv[j].x, acc[i][j].y);
                    }
            }
        }
        float2* out = outbase + cur_tl * s.out_size + o;
#pragma unroll
        for (int i = 0; i < NA; i++)
#pragma unroll
            for (int j = 0; j < NB; j++) out[doa[i] + dob[j]] = acc[i][j];
    }
}

template <int RA, int RB>
static void launch_micro(const StepDesc* d_step, const ChunkCtx& ctx, int64_t n_inst, const MicroBits& mb,
                         int64_t total_q, cudaStream_t s) {
    int64_t blocks = (total_q + kDirThreads - 1) / kDirThreads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_contract_micro<RA, RB><<<(unsigned)blocks, kDirThreads, 0, s>>>(d_step, ctx, n_inst, mb);
}

// marg[n][x] = Re(root_n[x]) (the double-layer diagonal), Z[n] = sum_x in FP64.
// One block per (network, tile of kFinTile consecutive block outcomes x); a
// thread takes kFinPer consecutive x and steps its root offset from x to x + 1
// with delta[ctz(~x)] (delta[k] = stride[k] - sum of the strides below k).
// Z is the FP64 sum of the tile (written directly when the block has one tile,
// otherwise as a partial that k_finalize_sum adds in tile order).
constexpr int kFinThreads = 256, kFinPer = 16, kFinTile = kFinThreads * kFinPer;

__global__ void __launch_bounds__(kFinThreads) k_finalize(const RootRef* __restrict__ groot, const __grid_constant__ ChunkCtx c, int b,
                                                          int64_t tiles, float* __restrict__ marg,
                                                          double* __restrict__ Z, double* __restrict__ part) {
    __shared__ __align__(16) RootRef r;
    __shared__ int64_t delta[32];
    __shared__ double red[kFinThreads / 32];
    {
        const int4* src = reinterpret_cast<const int4*>(groot);
        int4* dst = reinterpret_cast<int4*>(&r);
        for (int i = threadIdx.x; i < (int)(sizeof(RootRef) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t below = 0;
        for (int t = 0; t < (int)threadIdx.x && t < b; t++) below += r.x_stride[t];
        delta[threadIdx.x] = (int)threadIdx.x < b ? r.x_stride[threadIdx.x] - below : 0;
    }
    __syncthreads();
    const int64_t net = blockIdx.x / tiles, tile = blockIdx.x - net * tiles;
    const float2* R = operand_ptr(r.op, CLS_NET, net, c);
    const int64_t nx = (int64_t)1 << b;
    int64_t x = tile * kFinTile + (int64_t)threadIdx.x * kFinPer;
    double acc = 0.0;
    if (x < nx) {
        int64_t off = 0;
        for (int t = 0; t < b; t++)
            if ((x >> t) & 1) off += r.x_stride[t];
        float* out = marg + net * nx;
        for (int k = 0; k < kFinPer && x < nx; k++, x++) {
            const float v = R[off].x;
            out[x] = v;
            acc += (double)v;
            off += delta[__ffsll(~x) - 1];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kFinThreads / 32; w++) t += red[w];
        if (tiles == 1) Z[net] = t;
        else part[blockIdx.x] = t;
    }
}

// Z[net] = sum of its tiles' partials, in tile order
__global__ void k_finalize_sum(const double* __restrict__ part, int64_t tiles, int64_t n_net, double* __restrict__ Z) {
    const int64_t net = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (net >= n_net) return;
    double t = 0.0;
    for (int64_t k = 0; k < tiles; k++) t += part[net * tiles + k];
    Z[net] = t;
}

// A run of consecutive small trajectory-class steps (the gate-level start of a
// block's path: outputs of at most 2^kSmallOutBits elements from operands of
// at most 2^kSmallOpBits) in one launch: one CTA per trajectory of the chunk
// walks the run in order, each step's descriptor staged in shared memory and
// its outputs written to the arena, with a CTA barrier between steps (the
// next step reads them back from L1/L2).  A CTA touches only its own
// trajectory's instances, and the planner admits a step into a run only if no
// other CTA's instances can share its output's addresses (small_step,
// fuse_prev), so the CTA barrier is the only ordering the run needs.  Every
// output is the same complex multiply-add chain over the summed bits as in
// k_contract_direct.
constexpr int kSmallThreads = 128;

__global__ void __launch_bounds__(kSmallThreads) k_small_steps(const StepDesc* __restrict__ steps, int n_steps,
                                                               const __grid_constant__ ChunkCtx c) {
    __shared__ __align__(16) StepDesc s;
    const int64_t inst = blockIdx.x;
    for (int k = 0; k < n_steps; k++) {
        {
            const int4* src = reinterpret_cast<const int4*>(steps + k);
            int4* dst = reinterpret_cast<int4*>(&s);
            for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();   // descriptor staged; the previous step's outputs are visible
        const float2* A = operand_ptr(s.op[0], CLS_TRAJ, inst, c);
        const float2* B = operand_ptr(s.op[1], CLS_TRAJ, inst, c);
        float2* out = c.arena[s.out_arena] + s.out_off * c.arena_inst[s.out_arena] + inst * s.out_size;
        const float sa = s.op[0].conj ? -1.f : 1.f, sb = s.op[1].conj ? -1.f : 1.f;
        const int nk = 1 << s.n_sum;
        for (int64_t o = threadIdx.x; o < s.out_size; o += blockDim.x) {
            int64_t oa = 0, ob = 0;
            for (int p = 0; p < s.n_out; p++)
                if ((o >> p) & 1) {
                    oa += s.out_stride[0][p];
                    ob += s.out_stride[1][p];
                }
            float2 acc = make_float2(0.f, 0.f);
            for (int kk = 0; kk < nk; kk++) {
                int64_t ka = oa, kb = ob;
                for (int q = 0; q < s.n_sum; q++)
                    if ((kk >> q) & 1) {
                        ka += s.sum_stride[0][q];
                        kb += s.sum_stride[1][q];
                    }
                const float2 x = A[ka], y = B[kb];
                const float xi = sa * x.y, yi = sb * y.y;
                acc.x = fmaf(x.x, y.x, acc.x);
                acc.x = fmaf(-xi, yi, acc.x);
                acc.y = fmaf(x.x, yi, acc.y);
                acc.y = fmaf(xi, y.x, acc.y);
            }
            out[o] = acc;
        }
        __syncthreads();   // outputs written before the descriptor is replaced
    }
}

}  // namespace

void launch_small_steps(const StepDesc* d_steps, const StepDesc* h_steps, int n_steps, const ChunkCtx& ctx,
                        int64_t n_traj, cudaStream_t s) {
    if (n_steps <= 0 || n_traj <= 0) return;
    double bytes = 0.0, flops = 0.0;
    for (int k = 0; k < n_steps; k++) {
        const StepDesc& h = h_steps[k];
        bytes += 8.0 * (double)n_traj * (double)(h.out_size + h.op[0].inst_size + h.op[1].inst_size);
        flops += 8.0 * (double)n_traj * (double)h.out_size * (double)(1ll << h.n_sum);
    }
    StatScope sc(K_CONTRACT_SMALL, s, bytes, flops);
    k_small_steps<<<(unsigned)n_traj, kSmallThreads, 0, s>>>(d_steps, n_steps, ctx);
}

void launch_contract_step(const StepDesc* d_step, const StepDesc& h, const ChunkCtx& ctx, int64_t n_inst,
                          cudaStream_t s) {
    const int64_t total = n_inst << h.n_out;
    if (total <= 0) return;
    const int64_t tiles = (total + 32 * kDirU - 1) / (32 * kDirU);
    int64_t blocks = (tiles + kDirThreads / 32 - 1) / (kDirThreads / 32);
    const int64_t cap = 152 * 16;
    if (blocks > cap) blocks = cap;
    // 32-bit in-instance offsets when both operands and the output fit
    const bool off32 = h.op[0].inst_size < (1ll << 31) && h.op[1].inst_size < (1ll << 31) &&
                       h.out_size < (1ll << 31);
    // algorithmic traffic: every distinct operand element once, the output once
    // (a cached step reads the operands of its n_inst representatives only)
    double bytes = 8.0 * (double)total;
    const double n_traj_read = (h.cache > 0 && ctx.cache_list) ? (double)n_inst : (double)ctx.arena_inst[CLS_TRAJ];
    for (int o = 0; o < 2; o++) {
        const OperandDesc& d = h.op[o];
        double inst = d.mode == OP_LEAF ? (d.leaf_col >= 0 ? n_traj_read : 1.0)
                                        : (d.cls == CLS_TRAJ ? n_traj_read : (double)ctx.arena_inst[d.cls]);
        bytes += 8.0 * inst * (double)d.inst_size;
    }
    const double flops = 8.0 * (double)total * (double)(1ll << h.n_sum);
    StatScope sc(K_CONTRACT_DIRECT, s, bytes, flops);
    // micro-tile bits: the highest output bits along which only one operand varies
    MicroBits mb;
    memset(&mb, 0, sizeof mb);
    int ra = 0, rb = 0;
    const int ra_max = h.tile ? (h.tile - 1) / 3 : 2, rb_max = h.tile ? (h.tile - 1) % 3 : 2;
    for (int p = h.n_out - 1; p >= 0; p--) {
        const bool va = h.out_stride[0][p] != 0, vb = h.out_stride[1][p] != 0;
        if (va && !vb && ra < ra_max) mb.ta[ra++] = p;
        else if (vb && !va && rb < rb_max) mb.tb[rb++] = p;
    }
    if (off32 && ra + rb > 0) {
        for (int j = 0; j < ra; j++) mb.ins[mb.n_ins++] = mb.ta[j];
        for (int j = 0; j < rb; j++) mb.ins[mb.n_ins++] = mb.tb[j];
        std::sort(mb.ins, mb.ins + mb.n_ins);
        const int64_t tq = n_inst << (h.n_out - ra - rb);
        switch (ra * 3 + rb) {
            case 1: launch_micro<0, 1>(d_step, ctx, n_inst, mb, tq, s); break;
            case 2: launch_micro<0, 2>(d_step, ctx, n_inst, mb, tq, s); break;
            case 3: launch_micro<1, 0>(d_step, ctx, n_inst, mb, tq, s); break;
            case 4: launch_micro<1, 1>(d_step, ctx, n_inst, mb, tq, s); break;
            case 5: launch_micro<1, 2>(d_step, ctx, n_inst, mb, tq, s); break;
            case 6: launch_micro<2, 0>(d_step, ctx, n_inst, mb, tq, s); break;
            case 7: launch_micro<2, 1>(d_step, ctx, n_inst, mb, tq, s); break;
            default: launch_micro<2, 2>(d_step, ctx, n_inst, mb, tq, s); break;
        }
        return;
    }
    if (off32)
        k_contract_direct<int32_t><<<(unsigned)blocks, kDirThreads, 0, s>>>(d_step, ctx, n_inst);
    else
        k_contract_direct<int64_t><<<(unsigned)blocks, kDirThreads, 0, s>>>(d_step, ctx, n_inst);
}

int64_t finalize_tiles(int b) { return (((int64_t)1 << b) + kFinTile - 1) / kFinTile; }

void launch_finalize(const RootRef* d_root, const ChunkCtx& ctx, int b, int64_t n_net, float* marg, double* Z,
                     double* part, cudaStream_t s) {
    if (n_net <= 0) return;
    const int64_t tiles = finalize_tiles(b);
    StatScope sc(K_FINALIZE, s, (double)n_net * (double)(1ll << b) * 12.0, 0.0);
    k_finalize<<<(unsigned)(n_net * tiles), kFinThreads, 0, s>>>(d_root, ctx, b, tiles, marg, Z, part);
    if (tiles > 1) count_launches(K_FINALIZE);
    if (tiles > 1) k_finalize_sum<<<(unsigned)((n_net + 127) / 128), 128, 0, s>>>(part, tiles, n_net, Z);
}

}  // namespace ptn
