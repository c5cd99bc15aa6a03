// Batched pairwise contraction of block networks (the execution of one path
// step of P^j for every network of a chunk, Sec. III-A) and the marginal
// finalisation of the block's root tensor (Sec. II-B).
//
// k_contract_direct: one thread per output element of one instance; the
// element's operand addresses come from the step's per-bit stride tables, so
// any bit layout of either operand is read without a separate permutation
// pass.  The summed bits are walked in Gray-code order so each term updates
// one stride.  The first operand read of a merged-gate leaf goes through the
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

__device__ __forceinline__ float2 cmul_acc(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

__global__ void __launch_bounds__(256) k_contract_direct(const StepDesc* __restrict__ gstep, ChunkCtx c,
                                                         int64_t n_inst) {
    __shared__ __align__(16) StepDesc s;
    {
        const int4* src = reinterpret_cast<const int4*>(gstep);
        int4* dst = reinterpret_cast<int4*>(&s);
        for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    // Operand offsets of the low (up to 8) output bits, shared by the block: a
    // block iteration covers 256 consecutive outputs, so each element adds one
    // table entry to the offsets of its remaining high bits.
    __shared__ int64_t tab[2][256];
    const int lowb = s.n_out < 8 ? s.n_out : 8;
    {
        const int t = threadIdx.x;
        int64_t a = 0, b = 0;
        for (int p = 0; p < lowb; p++)
            if ((t >> p) & 1) {
                a += s.out_stride[0][p];
                b += s.out_stride[1][p];
            }
        tab[0][t] = a;
        tab[1][t] = b;
    }
    __syncthreads();
    const int64_t total = n_inst << s.n_out;
    const int64_t mask = s.out_size - 1;
    const int64_t lowmask = (1ll << lowb) - 1;
    const int nk = s.n_sum;
    const bool ca = s.op[0].conj, cb = s.op[1].conj;
    float2* outbase = c.arena[s.out_arena] + s.out_off * c.arena_inst[s.out_arena];
    int64_t cur_inst = -1, cur_hi = -1, hia = 0, hib = 0;
    const float2 *A = nullptr, *B = nullptr;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t inst = g >> s.n_out;
        const int64_t o = g & mask;
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
                    hia += s.out_stride[0][p];
                    hib += s.out_stride[1][p];
                }
            cur_hi = hi;
        }
        const int64_t oa = hia + tab[0][o & lowmask], ob = hib + tab[1][o & lowmask];
        float2 acc = make_float2(0.f, 0.f);
        int64_t ka = 0, kb = 0;
        const int64_t nterm = (int64_t)1 << nk;
        for (int64_t t = 0; t < nterm; t++) {
            if (t) {
                const int bit = __ffsll(t) - 1;
                const int64_t gray = t ^ (t >> 1);
                if ((gray >> bit) & 1) {
                    ka += s.sum_stride[0][bit];
                    kb += s.sum_stride[1][bit];
                } else {
                    ka -= s.sum_stride[0][bit];
                    kb -= s.sum_stride[1][bit];
                }
            }
            float2 a = A[oa + ka], b = B[ob + kb];
            if (ca) a.y = -a.y;
            if (cb) b.y = -b.y;
            acc = cmul_acc(acc, a, b);
        }
        outbase[inst * s.out_size + o] = acc;
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
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = 152 * 16;
    if (blocks > cap) blocks = cap;
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
    k_contract_direct<<<(unsigned)blocks, 256, 0, s>>>(d_step, ctx, n_inst);
}

void launch_finalize(const RootRef* d_root, const ChunkCtx& ctx, int b, int64_t n_net, float* marg, double* Z,
                     cudaStream_t s) {
    if (n_net <= 0) return;
    StatScope sc(K_FINALIZE, s, (double)n_net * (double)(1ll << b) * 12.0, 0.0);
    k_finalize<<<(unsigned)n_net, 256, 0, s>>>(d_root, ctx, b, marg, Z);
}

}  // namespace ptn
