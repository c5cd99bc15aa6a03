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
        const int64_t oi = d.cls == CLS_CONST ? 0 : (d.cls == CLS_TRAJ ? tl : net);
        p = c.arena[d.arena] + d.arena_off * c.arena_inst[d.arena] + oi * d.inst_size;
    }
    if (d.n_slice) {
        const uint64_t pre = c.net_prefix[net];
        int64_t off = 0;
        for (int s = 0; s < d.n_slice; s++) off += (int64_t)((pre >> d.slice_qubit[s]) & 1ull) * d.slice_stride[s];
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
__global__ void __launch_bounds__(kDirThreads, 3) k_contract_direct(const StepDesc* __restrict__ gstep, ChunkCtx c,
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
    int64_t cur_inst = -1, cur_hi = -1;
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
                A = operand_ptr(s.op[0], s.out_cls, inst, c);
                B = operand_ptr(s.op[1], s.out_cls, inst, c);
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
            if (g < total) outbase[g] = acc[u];
        }
    }
}

// marg[n][x] = Re(root_n[x]) (the double-layer diagonal), Z[n] = sum_x in FP64.
__global__ void __launch_bounds__(256) k_finalize(const RootRef* __restrict__ groot, ChunkCtx c, int b,
                                                  float* __restrict__ marg, double* __restrict__ Z) {
    __shared__ __align__(16) RootRef r;
    __shared__ double red[256];
    {
        const int4* src = reinterpret_cast<const int4*>(groot);
        int4* dst = reinterpret_cast<int4*>(&r);
        for (int i = threadIdx.x; i < (int)(sizeof(RootRef) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t net = blockIdx.x;
    const float2* R = operand_ptr(r.op, CLS_NET, net, c);
    const int64_t nx = (int64_t)1 << b;
    double acc = 0.0;
    for (int64_t x = threadIdx.x; x < nx; x += blockDim.x) {
        int64_t off = 0;
        for (int t = 0; t < b; t++)
            if ((x >> t) & 1) off += r.x_stride[t];
        const float v = R[off].x;
        marg[net * nx + x] = v;
        acc += (double)v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) Z[net] = red[0];
}

}  // namespace

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
    double bytes = 8.0 * (double)total;
    for (int o = 0; o < 2; o++) {
        const OperandDesc& d = h.op[o];
        double inst = d.mode == OP_LEAF ? (d.leaf_col >= 0 ? (double)ctx.arena_inst[CLS_TRAJ] : 1.0)
                                        : (double)ctx.arena_inst[d.cls];
        bytes += 8.0 * inst * (double)d.inst_size;
    }
    const double flops = 8.0 * (double)total * (double)(1ll << h.n_sum);
    StatScope sc(K_CONTRACT_DIRECT, s, bytes, flops);
    if (off32)
        k_contract_direct<int32_t><<<(unsigned)blocks, kDirThreads, 0, s>>>(d_step, ctx, n_inst);
    else
        k_contract_direct<int64_t><<<(unsigned)blocks, kDirThreads, 0, s>>>(d_step, ctx, n_inst);
}

void launch_finalize(const RootRef* d_root, const ChunkCtx& ctx, int b, int64_t n_net, float* marg, double* Z,
                     cudaStream_t s) {
    if (n_net <= 0) return;
    StatScope sc(K_FINALIZE, s, (double)n_net * (double)(1ll << b) * 12.0, 0.0);
    k_finalize<<<(unsigned)n_net, 256, 0, s>>>(d_root, ctx, b, marg, Z);
}

}  // namespace ptn
