// Expectation values of diagonal Pauli sums on the trajectory states and the
// reductions of the adjoint (reverse-mode) pass into angle gradients.
//
// F_i = <psi_i| O |psi_i> = sum_x w(x) |psi_i(x)|^2 for O = sum_t c_t Z^{z_t},
// w(x) = sum_t c_t (-1)^{popcount(x & z_t)}.  Its holomorphic derivative with
// respect to psi_i(x) is w(x) conj(psi_i(x)): the adjoint the reversed path
// starts from.  With G_L the adjoint that reaches a parametrised merged gate
// tensor L(theta), dF_i/dtheta = 2 Re sum_e G_L[e] dL[e]/dtheta.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

// one block per trajectory of the chunk
__global__ void __launch_bounds__(256) k_observable(const RootRef* __restrict__ groot, const __grid_constant__ ChunkCtx c, int n,
                                                    const ObsTerm* __restrict__ terms, int n_terms,
                                                    int64_t root_adj_off, int64_t traj0, double* __restrict__ F) {
    __shared__ __align__(16) RootRef r;
    __shared__ double red[256];
    {
        const int4* src = reinterpret_cast<const int4*>(groot);
        int4* dst = reinterpret_cast<int4*>(&r);
        for (int i = threadIdx.x; i < (int)(sizeof(RootRef) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t t = blockIdx.x;
    const int64_t size = r.op.inst_size;
    // a circuit without multi-variant leaves has a trajectory-independent state
    const int64_t inst = r.op.cls == CLS_CONST ? 0 : t;
    const float2* psi = c.arena[r.op.arena] + r.op.arena_off * c.arena_inst[r.op.arena] + inst * size;
    float2* adj = c.arena[ARENA_ADJ] + root_adj_off * c.arena_inst[ARENA_ADJ] + t * size;
    const int64_t nx = (int64_t)1 << n;
    double acc = 0.0;
    for (int64_t x = threadIdx.x; x < nx; x += blockDim.x) {
        int64_t off = 0;
        for (int q = 0; q < n; q++)
            if ((x >> q) & 1) off += r.x_stride[q];
        double w = 0.0;
        for (int k = 0; k < n_terms; k++) w += (__popcll((uint64_t)x & terms[k].zmask) & 1) ? -terms[k].coeff : terms[k].coeff;
        const float2 v = psi[off];
        acc += w * ((double)v.x * v.x + (double)v.y * v.y);
        adj[off] = make_float2((float)(w * v.x), (float)(-w * v.y));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) F[traj0 + t] = red[0];
}

// one block per (trajectory of the chunk, parametrised leaf)
__global__ void __launch_bounds__(128) k_leaf_grad(const __grid_constant__ ChunkCtx c, const ParamLeaf* __restrict__ pl, int n_pl,
                                                   const float2* __restrict__ dvt, int64_t traj0, int n_params,
                                                   double* __restrict__ partial) {
    __shared__ double red[128];
    const int64_t t = blockIdx.x / n_pl;
    const int k = (int)(blockIdx.x - t * n_pl);
    const ParamLeaf p = pl[k];
    int64_t var = 0;
    if (p.var_col >= 0) var = c.var_ids[(int64_t)c.chunk_traj[t] * c.n_var_cols + p.var_col];
    // buffers are instance-major blocks: base + offset * instances + instance * size
    const float2* G = c.arena[ARENA_LGRAD] + p.lgrad_off * c.arena_inst[ARENA_LGRAD] + t * p.size;
    const float2* D = dvt + p.dvt_base + var * p.size;
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < p.size; e += blockDim.x) {
        const float2 g = G[e], d = D[e];
        acc += (double)g.x * d.x - (double)g.y * d.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&partial[(traj0 + t) * n_params + p.param_index], 2.0 * red[0]);
}

// one block per parameter (block 0 also reduces the value), fixed summation order
__global__ void __launch_bounds__(256) k_expval_reduce(const int64_t* __restrict__ mult, const double* __restrict__ F,
                                                       const double* __restrict__ partial, int64_t n_traj, int n_params,
                                                       double* __restrict__ value, double* __restrict__ grad) {
    __shared__ double red[256], redw[256];
    const int p = blockIdx.x;
    double acc = 0.0, wacc = 0.0, facc = 0.0;
    for (int64_t i = threadIdx.x; i < n_traj; i += blockDim.x) {
        const double w = (double)mult[i];
        wacc += w;
        if (p < n_params) acc += w * partial[i * n_params + p];
        if (p == 0) facc += w * F[i];
    }
    red[threadIdx.x] = acc;
    redw[threadIdx.x] = wacc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[threadIdx.x] += red[threadIdx.x + s];
            redw[threadIdx.x] += redw[threadIdx.x + s];
        }
        __syncthreads();
    }
    const double wsum = redw[0];
    if (threadIdx.x == 0 && p < n_params) grad[p] = red[0] / wsum;
    __syncthreads();
    if (p == 0) {
        red[threadIdx.x] = facc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) *value = red[0] / wsum;
    }
}

// amp[t][x] = psi_t(x) in qubit order (bit q of x = qubit q); one block per trajectory
__global__ void __launch_bounds__(256) k_amplitudes(const RootRef* __restrict__ groot, const __grid_constant__ ChunkCtx c, int n,
                                                    float2* __restrict__ amp) {
    __shared__ __align__(16) RootRef r;
    {
        const int4* src = reinterpret_cast<const int4*>(groot);
        int4* dst = reinterpret_cast<int4*>(&r);
        for (int i = threadIdx.x; i < (int)(sizeof(RootRef) / sizeof(int4)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t t = blockIdx.x;
    const int64_t size = r.op.inst_size;
    const int64_t inst = r.op.cls == CLS_CONST ? 0 : t;
    const float2* psi = c.arena[r.op.arena] + r.op.arena_off * c.arena_inst[r.op.arena] + inst * size;
    const int64_t nx = (int64_t)1 << n;
    for (int64_t x = threadIdx.x; x < nx; x += blockDim.x) {
        int64_t off = 0;
        for (int q = 0; q < n; q++)
            if ((x >> q) & 1) off += r.x_stride[q];
        amp[t * nx + x] = psi[off];
    }
}

}  // namespace

void launch_observable(const RootRef* d_root, const ChunkCtx& ctx, int n, const ObsTerm* terms, int n_terms,
                       int64_t root_adj_off, int64_t traj0, double* F, cudaStream_t s) {
    const int64_t nt = ctx.arena_inst[CLS_TRAJ];
    if (nt <= 0) return;
    StatScope sc(K_EXPVAL, s, (double)nt * (double)(1ll << n) * 16.0, 0.0);
    k_observable<<<(unsigned)nt, 256, 0, s>>>(d_root, ctx, n, terms, n_terms, root_adj_off, traj0, F);
}

void launch_amplitudes(const RootRef* d_root, const ChunkCtx& ctx, int n, int64_t n_traj, float2* amp, cudaStream_t s) {
    if (n_traj <= 0) return;
    StatScope sc(K_EXPVAL, s, (double)n_traj * (double)(1ll << n) * 16.0, 0.0);
    k_amplitudes<<<(unsigned)n_traj, 256, 0, s>>>(d_root, ctx, n, amp);
}

void launch_leaf_grad(const ChunkCtx& ctx, const ParamLeaf* d_pl, int n_pl, const float2* dvt, int64_t traj0,
                      int64_t n_traj, int n_params, double* partial, cudaStream_t s) {
    if (n_pl <= 0 || n_traj <= 0) return;
    StatScope sc(K_EXPVAL, s, 0.0, 0.0);
    k_leaf_grad<<<(unsigned)(n_traj * n_pl), 128, 0, s>>>(ctx, d_pl, n_pl, dvt, traj0, n_params, partial);
}

void launch_expval_reduce(const int64_t* mult, const double* F, const double* partial, int64_t n_traj, int n_params,
                          double* value, double* grad, cudaStream_t s) {
    const int blocks = n_params > 0 ? n_params : 1;
    StatScope sc(K_EXPVAL, s, 0.0, 0.0);
    k_expval_reduce<<<blocks, 256, 0, s>>>(mult, F, partial, n_traj, n_params, value, grad);
}

}  // namespace ptn
