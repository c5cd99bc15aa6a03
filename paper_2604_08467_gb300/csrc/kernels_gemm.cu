// Tensor-core execution of the large pairwise contractions of a path (the
// batched complex GEMMs of Sec. III-A's contraction, real and imaginary parts
// split into real GEMMs) on sm_103a: tcgen05.mma with the accumulator in
// tensor memory, operands staged by TMA into 128-byte-swizzled shared memory
// through an mbarrier pipeline.
//
// A step  C[inst][m, n] (h) = sum_k A[m, k] (h) * B[n, k] (h)  runs in two phases:
//  1. pack: each operand is gathered (any bit layout, merged-gate variant,
//     prefix slice) into row-major K-contiguous rows, each value split into a
//     high and a low part in the tensor-core input format F:
//       A rows:  [ hi(re0) hi(im0) hi(re1) ... | lo(re0) lo(im0) ... ]
//       B rows 2n, 2n+1 (the complex product as real dot products):
//         row 2n   = (re, -im) per k,  row 2n+1 = (im, re) per k, each [hi | lo];
//     so that  A_row . B_row(2n) = Re C[m, n]  and  A_row . B_row(2n+1) = Im C[m, n];
//  2. GEMM: D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T with FP32 accumulation
//     in TMEM (the lo*lo term is dropped) over segments of at most kSegKb
//     k-blocks, the segments added in FP32 by the epilogue; D[m][2n + c] ->
//     C[m, n], written through the step's output strides (any layout).
// Formats (the precision modes of the contraction):
//  - TF32 (PTN_PREC_FP32): hi = x rounded to TF32, lo = (x - hi) rounded to
//    TF32; |x - hi - lo| <= 2^-24 |x|, i.e. FP32-accurate products;
//  - BF16 (PTN_PREC_BF16X3): hi, lo rounded to BF16 (16 significant bits in
//    total, FP32 exponent range);
//  - FP16 (PTN_PREC_FP16X3): hi, lo rounded to FP16 (22 significant bits) after
//    scaling each packed row by a power of two that brings its largest
//    magnitude into [0.5, 1); the epilogue undoes the row and column scales
//    exactly.
// The GEMM kernel is persistent and warp-specialised (see k_gemm).
// Conjugated operands (bra layer) are conjugated while packing.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {

namespace {

constexpr int kBM = 128;          // UMMA M (cta_group::1)
constexpr int kBN = 128;          // UMMA N (realified B rows per tile)
constexpr int kRowBytes = 128;    // one swizzle row of every tile
constexpr int kStages = 3;        // pipeline depth (4 tiles of 16 KB per stage)
constexpr int kTileA = kBM * kRowBytes;
constexpr int kTileB = kBN * kRowBytes;
constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;
// epilogue staging for column-contiguous outputs: per epilogue warp a 32-row x
// 16-column complex fragment (rows padded to 17 slots) and its 32 row offsets
constexpr int kStgPitch = 17;
constexpr int kStgBytes = 4 * (32 * kStgPitch * 8 + 32 * 8);
constexpr int kTabBytes = 8192;   // barriers, TMEM slot, per-warp column offsets and FP16 column scales
constexpr int kGemmSmem = 1024 + kStages * kStageBytes + kTabBytes + kStgBytes;   // align slack + stages + tables + staging
constexpr int kMaxPackBits = 40;
constexpr int kSegKb = 16;        // longest run of k-blocks accumulated in TMEM before the epilogue adds it
// k-blocks are spread round-robin over kAcc TMEM accumulators that the
// epilogue adds in FP32: the tensor core's FP32 accumulation truncates, so
// shorter accumulation chains keep the contraction within FP32 accuracy.
constexpr int kAcc = 4;
constexpr uint32_t kTmemCols = kAcc * kBN;   // 512: the whole TMEM of the SM (one CTA per SM)

enum GemmFmt { FMT_TF32 = 0, FMT_BF16 = 1, FMT_FP16 = 2 };

template <int F>
struct Fmt;
template <>
struct Fmt<FMT_TF32> {
    using T = float;
    static constexpr int kBytes = 4;
    static constexpr uint32_t kAB = 2;   // TF32 in the instruction descriptor
};
template <>
struct Fmt<FMT_BF16> {
    using T = __nv_bfloat16;
    static constexpr int kBytes = 2;
    static constexpr uint32_t kAB = 1;   // BF16
};
template <>
struct Fmt<FMT_FP16> {
    using T = __half;
    static constexpr int kBytes = 2;
    static constexpr uint32_t kAB = 0;   // F16
};

struct PackArgs {
    OperandDesc op;
    int32_t pcls;            // instance class the packed operand is addressed by
    int32_t role;            // 0: rows (A), 1: realified (B)
    int32_t n_rb, n_hb, n_kb;
    int32_t Kh;              // elements per half row (hi or lo), a multiple of one swizzle row
    int64_t n_pinst;
    int64_t r_stride[kMaxPackBits];   // operand strides of the row bits
    int64_t h_stride[kMaxPackBits];
    int64_t k_stride[kMaxPackBits];
    void* dst;
    int8_t* row_exp;         // FP16: per packed row and K segment (row-major [row][segment]) the
                             // power-of-two exponent e of the segment's largest |component| (the
                             // segment is stored scaled by 2^-e), else null
    int32_t seg_slots;       // FP16: complex slots per K segment (the GEMM's kSegKb k-blocks)
    const int32_t* inst_map; // cached step: packed instance i is local trajectory inst_map[i] (else i)
    // Outer-product operand (StepDesc.prod): the element is op[o0] * op1[o1], and every
    // stride above holds o0 in its low and o1 in its high 32 bits (sums stay carry-free,
    // each factor having at most 2^31 elements per instance); xconj: conjugate the product
    int32_t prod, xconj;
    OperandDesc op1;
};

struct GemmArgs {
    int32_t M, N2, Kh, nkb;
    int32_t n_h;
    int32_t a_pcls, b_pcls, out_cls;
    int32_t n_mb, n_nb, n_hb;
    int32_t col_out;             // the lowest output bit is a column (N) bit: stores go column-contiguous
    int64_t tiles_m, tiles_n, n_inst, n_tiles;
    const int32_t* net_tl;
    // stacked mode: the rows of all networks of one trajectory form one GEMM
    // (rows = network-major (net, m)); tiles never cross trajectories
    int32_t stacked, m_bits;
    int64_t n_groups;
    const int32_t* grp_net0;     // [n_groups + 1] first network of each trajectory group
    const int64_t* grp_tile0;    // [n_groups + 1] first tile of each group
    float2* out;
    int64_t out_size;
    int* err;
    uint64_t wait_ns;            // limit of every pipeline wait (ptn_set_wait_limit)
    const int8_t* exp_a;         // FP16 row exponents of A and B (see PackArgs), else null
    const int8_t* exp_b;
    const int32_t* out_map;      // cached step: instance i writes local trajectory out_map[i] (else i)
    int64_t m_stride[kMaxOut];
    int64_t n_stride[kMaxOut];
    int64_t h_stride[kMaxOut];
};

// Round to the nearest TF32 value (ties away from zero): add half of the 13
// dropped mantissa bits, then clear them.
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <int F>
__device__ __forceinline__ void split(float x, typename Fmt<F>::T& hi, typename Fmt<F>::T& lo);
template <>
__device__ __forceinline__ void split<FMT_TF32>(float x, float& hi, float& lo) {
    hi = tf32_rn(x);
    lo = tf32_rn(x - hi);
}
template <>
__device__ __forceinline__ void split<FMT_BF16>(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
template <>
__device__ __forceinline__ void split<FMT_FP16>(float x, __half& hi, __half& lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

template <int F>
__device__ __forceinline__ void store_pair(typename Fmt<F>::T* d, typename Fmt<F>::T x, typename Fmt<F>::T y);
template <>
__device__ __forceinline__ void store_pair<FMT_TF32>(float* d, float x, float y) {
    *reinterpret_cast<float2*>(d) = make_float2(x, y);
}
template <>
__device__ __forceinline__ void store_pair<FMT_BF16>(__nv_bfloat16* d, __nv_bfloat16 x, __nv_bfloat16 y) {
    *reinterpret_cast<__nv_bfloat162*>(d) = __halves2bfloat162(x, y);
}
template <>
__device__ __forceinline__ void store_pair<FMT_FP16>(__half* d, __half x, __half y) {
    *reinterpret_cast<__half2*>(d) = __halves2half2(x, y);
}

__device__ __forceinline__ const float2* pack_operand_ptr(const OperandDesc& d, int pcls, int64_t inst,
                                                          const ChunkCtx& c) {
    int64_t tl = 0, net = 0;
    if (pcls == CLS_NET) {
        net = inst;
        tl = c.net_tl[inst];
    } else if (pcls == CLS_TRAJ) {
        tl = inst;
    }
    const float2* p;
    if (d.mode == OP_LEAF) {
        int64_t var = 0;
        if (d.leaf_col >= 0) var = c.var_ids[(int64_t)c.chunk_traj[tl] * c.n_var_cols + d.leaf_col];
        p = c.vtab + d.leaf_base + var * d.inst_size;
    } else {
        const int64_t oi = d.cls == CLS_CONST ? 0 : (d.cls == CLS_TRAJ ? rep_inst(d, tl, c) : net);
        p = c.arena[d.arena] + d.arena_off * c.arena_inst[d.arena] + oi * d.inst_size;
    }
    if (pcls == CLS_NET && d.n_slice) {
        const uint64_t* pre = c.net_prefix + net * c.n_words;
        int64_t off = 0;
        for (int s = 0; s < d.n_slice; s++) off += (int64_t)bits_get(pre, d.slice_qubit[s]) * d.slice_stride[s];
        p += off;
    }
    return p;
}

// Packing: one warp per packed row (instance, h, row) when a half row holds
// >= 32 complex slots, else 32 / slots rows per warp.  Every size is a power of
// two, so the row index is decoded with shifts.  The row's base offset is
// formed once per row; the K offsets come from a per-block shared table in two
// levels (bits 0-9 and 10-19; bit 20 and up, rarely used, by a loop), so a
// contiguous K axis turns into coalesced float2 loads.  Stores are float2 /
// 32-bit pairs, consecutive lanes on consecutive slots.  FP16 rows are scaled
// segment by segment: the GEMM accumulates K in segments of kSegKb k-blocks
// (512 complex slots in FP16) and adds them in FP32, so a scale needs to be
// uniform along one segment only.  Each (row, segment) is stored scaled by
// 2^-e, e the exponent of its largest |component|, in one pass: a warp keeps
// the segment in registers between the max and the store.
constexpr int kKTab = 1024;
constexpr int kPackRegRow = 512;   // longest FP16 K segment a warp holds in registers

__device__ __forceinline__ void build_ktab(const PackArgs& a, int64_t* ktab) {
    const int n_lo = a.n_kb < 10 ? a.n_kb : 10;
    const int n_mid = a.n_kb < 20 ? a.n_kb - n_lo : 10;
    for (int i = threadIdx.x; i < 2 * kKTab; i += blockDim.x) {
        const int lvl = i >= kKTab, v = i & (kKTab - 1);
        int64_t off = 0;
        const int nb = lvl ? n_mid : n_lo, b0 = lvl ? 10 : 0;
        for (int t = 0; t < nb; t++)
            if ((v >> t) & 1) off += a.k_stride[b0 + t];
        ktab[i] = off;
    }
}
__device__ __forceinline__ int64_t kofs(const PackArgs& a, const int64_t* ktab, int64_t kc) {
    int64_t off = ktab[kc & (kKTab - 1)] + ktab[kKTab + ((kc >> 10) & (kKTab - 1))];
    for (int t = 20; t < a.n_kb; t++)
        if ((kc >> t) & 1) off += a.k_stride[t];
    return off;
}
// Operand address of packed row jr = (pi * nh + h) * nrow + row; z = pi * nh + h.
// Row offsets from a two-level table like the K offsets (row bits 0-9 and
// 10-19; bit 20 and up by a loop): short rows would otherwise spend most of
// their time forming their base address.
__device__ __forceinline__ void build_rtab(const PackArgs& a, int64_t* rtab) {
    const int n_lo = a.n_rb < 10 ? a.n_rb : 10;
    const int n_mid = a.n_rb < 20 ? a.n_rb - n_lo : 10;
    for (int i = threadIdx.x; i < 2 * kKTab; i += blockDim.x) {
        const int lvl = i >= kKTab, v = i & (kKTab - 1);
        int64_t off = 0;
        const int nb = lvl ? n_mid : n_lo, b0 = lvl ? 10 : 0;
        for (int t = 0; t < nb; t++)
            if ((v >> t) & 1) off += a.r_stride[b0 + t];
        rtab[i] = off;
    }
}
struct PackSrc {
    const float2* b0;        // the operand's row (outer product: factor 0's)
    const float2* b1;        // outer product: factor 1's, else unused
};
constexpr int64_t kLo32 = 0xffffffffll;
__device__ __forceinline__ PackSrc pack_row_base(const PackArgs& a, const ChunkCtx& c, const int64_t* rtab,
                                                 int64_t jr, int64_t& z, int64_t& row) {
    row = jr & (((int64_t)1 << a.n_rb) - 1);
    z = jr >> a.n_rb;
    const int64_t h = z & (((int64_t)1 << a.n_hb) - 1);
    const int64_t pi = a.inst_map ? (int64_t)a.inst_map[z >> a.n_hb] : z >> a.n_hb;
    int64_t off = rtab[row & (kKTab - 1)] + rtab[kKTab + ((row >> 10) & (kKTab - 1))];
    for (int i = 20; i < a.n_rb; i++)
        if ((row >> i) & 1) off += a.r_stride[i];
    for (int i = 0; i < a.n_hb; i++)
        if ((h >> i) & 1) off += a.h_stride[i];
    PackSrc src;
    if (!a.prod) {
        src.b0 = pack_operand_ptr(a.op, a.pcls, pi, c) + off;
        src.b1 = nullptr;
    } else {
        src.b0 = pack_operand_ptr(a.op, a.pcls, pi, c) + (off & kLo32);
        src.b1 = pack_operand_ptr(a.op1, a.pcls, pi, c) + (off >> 32);
    }
    return src;
}
// Element at K offset koff of a row: a plain read, or the product of the two
// factors with the single-term multiply-add sequence of the SIMT contraction
// kernels (so the packed values equal those of the materialised product).
__device__ __forceinline__ float2 pack_load(const PackArgs& a, const PackSrc& src, int64_t koff) {
    if (!a.prod) return src.b0[koff];
    const float2 x = src.b0[koff & kLo32], y = src.b1[koff >> 32];
    const float xi = a.op.conj ? -x.y : x.y, yi = a.op1.conj ? -y.y : y.y;
    float2 r;
    r.x = fmaf(x.x, y.x, 0.f);
    r.x = fmaf(-xi, yi, r.x);
    r.y = fmaf(x.x, yi, 0.f);
    r.y = fmaf(xi, y.x, r.y);
    return r;
}
template <int F>
__device__ __forceinline__ void pack_store(const PackArgs& a, typename Fmt<F>::T* d0, int64_t rowlen, int64_t kc,
                                           float re, float im) {
    using T = typename Fmt<F>::T;
    T rh, rl, ih, il;
    split<F>(re, rh, rl);
    split<F>(im, ih, il);
    if (a.role == 0) {
        store_pair<F>(d0 + 2 * kc, rh, ih);
        store_pair<F>(d0 + a.Kh + 2 * kc, rl, il);
    } else {
        T nih, nil;
        split<F>(-im, nih, nil);
        store_pair<F>(d0 + 2 * kc, rh, nih);
        store_pair<F>(d0 + a.Kh + 2 * kc, rl, nil);
        store_pair<F>(d0 + rowlen + 2 * kc, ih, rh);
        store_pair<F>(d0 + rowlen + a.Kh + 2 * kc, il, rl);
    }
}
__device__ __forceinline__ int row_exponent(float mx) {
    int e = 0;
    if (mx > 0.f) {
        frexpf(mx, &e);
        e = e < -100 ? -100 : (e > 100 ? 100 : e);
    }
    return e;
}

template <int F>
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ PackArgs a, const __grid_constant__ ChunkCtx c) {
    using T = typename Fmt<F>::T;
    __shared__ int64_t ktab[2 * kKTab];
    __shared__ int64_t rtab[2 * kKTab];
    build_ktab(a, ktab);
    build_rtab(a, rtab);
    __syncthreads();
    T* dst = static_cast<T*>(a.dst);
    const int lk = 31 - __clz(a.Kh / 2);                // log2 complex slots per half row
    const int64_t kcp = (int64_t)1 << lk;
    const int64_t kc_real = (int64_t)1 << a.n_kb;
    const int64_t rowlen = 2 * (int64_t)a.Kh;
    const int rpw = lk >= 5 ? 1 : (32 >> lk);           // rows per warp
    const int lane = threadIdx.x & 31;
    const int sub = lk >= 5 ? 0 : (lane >> lk);         // row of this lane within the warp
    const int lstep = lk >= 5 ? 32 : (int)kcp;          // slots a lane advances by
    const int l0 = lk >= 5 ? lane : (lane & ((int)kcp - 1));
    const int64_t n_rows = a.n_pinst << (a.n_hb + a.n_rb);
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float csign = (a.prod ? a.xconj : a.op.conj) ? -1.f : 1.f;
    if (F == FMT_FP16 && kc_real < 32) {
        // short FP16 rows (fewer real slots than a warp, padded to 32): g =
        // kc_real lanes per row, 32 / g rows per warp, the row maximum
        // reduced within each lane group
        const int lg = a.n_kb, g = 1 << lg;
        const int sub_r = lane >> lg, l0r = lane & (g - 1);
        for (int64_t w = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); (w << (5 - lg)) < n_rows;
             w += warps) {
            const int64_t jr = (w << (5 - lg)) + sub_r;
            const bool act = jr < n_rows;
            float2 v = make_float2(0.f, 0.f);
            int64_t z = 0, row = 0;
            if (act) {
                const PackSrc src = pack_row_base(a, c, rtab, jr, z, row);
                v = pack_load(a, src, kofs(a, ktab, l0r));
            }
            float mx = fmaxf(fabsf(v.x), fabsf(v.y));
            for (int o = g >> 1; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (!act) continue;
            const int e = row_exponent(mx);
            const float sc = ldexpf(1.f, -e);
            if (l0r == 0) a.row_exp[jr] = (int8_t)e;
            T* d0 = a.role == 0 ? dst + jr * rowlen : dst + ((z << (a.n_rb + 1)) + 2 * row) * rowlen;
            pack_store<F>(a, d0, rowlen, l0r, v.x * sc, csign * v.y * sc);
            for (int64_t kc = l0r + g; kc < kcp; kc += g) pack_store<F>(a, d0, rowlen, kc, 0.f, 0.f);   // padding
        }
        return;
    }
    if constexpr (F == FMT_FP16) {
        // units of (row, K segment): a warp holds a segment of at most
        // kPackRegRow slots in registers, reduces its largest |component|,
        // and writes it scaled (rows span at least 32 slots: one unit per warp)
        const int64_t seg = kcp < a.seg_slots ? kcp : a.seg_slots;
        const int lseg = 63 - __clzll(seg);
        const int64_t nseg = kcp >> lseg;
        const int64_t units = n_rows << (lk - lseg);
        for (int64_t w = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < units; w += warps) {
            const int64_t jr = w >> (lk - lseg), sg = w & (nseg - 1);
            int64_t z, row;
            const PackSrc src = pack_row_base(a, c, rtab, jr, z, row);
            T* d0 = a.role == 0 ? dst + jr * rowlen : dst + ((z << (a.n_rb + 1)) + 2 * row) * rowlen;
            const int64_t kc0 = sg << lseg;
            float2 v[kPackRegRow / 32];
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < kPackRegRow / 32; i++) {
                const int64_t kc = kc0 + lane + 32 * i;
                v[i] = make_float2(0.f, 0.f);
                if (lane + 32 * i < seg && kc < kc_real) v[i] = pack_load(a, src, kofs(a, ktab, kc));
                mx = fmaxf(mx, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int e = row_exponent(mx);
            const float sc = ldexpf(1.f, -e);
            if (lane == 0) a.row_exp[jr * nseg + sg] = (int8_t)e;
#pragma unroll
            for (int i = 0; i < kPackRegRow / 32; i++)
                if (lane + 32 * i < seg)
                    pack_store<F>(a, d0, rowlen, kc0 + lane + 32 * i, v[i].x * sc, csign * v[i].y * sc);
        }
        return;
    }
    for (int64_t w = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); w * rpw < n_rows; w += warps) {
        const int64_t jr = w * rpw + sub;                // (pi, h, row), row fastest
        if (jr >= n_rows) continue;
        int64_t z, row;
        const PackSrc src = pack_row_base(a, c, rtab, jr, z, row);
        T* d0 = a.role == 0 ? dst + jr * rowlen : dst + ((z << (a.n_rb + 1)) + 2 * row) * rowlen;
        {
            for (int64_t kc = l0; kc < kcp; kc += lstep) {
                float re = 0.f, im = 0.f;
                if (kc < kc_real) {
                    const float2 v = pack_load(a, src, kofs(a, ktab, kc));
                    re = v.x;
                    im = csign * v.y;
                }
                pack_store<F>(a, d0, rowlen, kc, re, im);
            }
        }
    }
}

// ------------------------------------------------------------- PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait (limit_ns of wall time, 2 s by default); false when it gave up
// or another thread of the block aborted.  A limit of 0 gives up at the first
// poll that finds the phase incomplete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; i++) {
        if ((i & 255u) == 0u) {   // first after a failed poll, then every 256 polls
            if (*abort) return false;
            if (global_ns() - t0 >= limit_ns) return false;
        }
        if (mbar_try_wait(bar, parity)) return true;
    }
}
// Bounded wait that ignores the abort flag (used to drain own async work).
__device__ __forceinline__ bool mbar_wait_plain(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > 2000000000ull) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand tile in the 128-byte swizzle
// layout TMA writes (rows of 128 B, 8-row atoms 1024 B apart).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1u << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                   // descriptor version for tcgen05
    d |= (uint64_t)2u << 61;                   // SWIZZLE_128B
    return d;
}

// Instruction descriptor: D = F32, A = B = format F, both K-major, M = 128, N = kBN.
template <int F>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | (Fmt<F>::kAB << 7) | (Fmt<F>::kAB << 10) | ((uint32_t)(kBN >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

// One MMA over 32 bytes of K (8 TF32 or 16 BF16/FP16 elements).
template <int F>
__device__ __forceinline__ void umma(uint32_t taddr, uint64_t ad, uint64_t bd, uint32_t acc) {
    if constexpr (F == FMT_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc<F>()), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc<F>()), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Store 32 columns of this warp's 32 TMEM lanes (one register per column) and
// wait until the stores have completed.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Persistent warp-specialised GEMM: each CTA (one per SM) walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 0 lane 0 streams the K-blocks
// of all its tiles through the kStages shared-memory ring by TMA; warp 1
// lane 0 issues tcgen05.mma into the TMEM accumulators; warps 2-5 (one per
// TMEM lane quadrant) drain a finished item (a tile, or one K segment of a
// long tile) while the producer already loads the next one.  The MMA warp
// starts an item only after the epilogue has released that item's accumulator
// set (acc_empty), and the epilogue starts after the item's last MMA
// completes (acc_full).  Every wait is bounded.
constexpr int kGemmThreads = 320;   // producer, MMA, 8 epilogue warps
struct TileInfo {
    int64_t inst, h, row_end;
    int m0, n0, za, zb;
};
__device__ __forceinline__ TileInfo decode_tile(const GemmArgs& g, int64_t tile) {
    TileInfo t;
    if (!g.stacked) {
        const int64_t tiles = g.tiles_m * g.tiles_n;
        const int64_t zt = tile / tiles;
        const int64_t r = tile - zt * tiles;
        const int64_t tm = r % g.tiles_m, tn = r / g.tiles_m;
        t.inst = zt / g.n_h;
        t.h = zt - t.inst * g.n_h;
        t.m0 = (int)(tm * kBM);
        t.n0 = (int)(tn * kBN);
        t.row_end = g.M;
        const int64_t pa = g.a_pcls == g.out_cls ? t.inst : (g.a_pcls == CLS_TRAJ ? (int64_t)g.net_tl[t.inst] : 0);
        const int64_t pb = g.b_pcls == g.out_cls ? t.inst : (g.b_pcls == CLS_TRAJ ? (int64_t)g.net_tl[t.inst] : 0);
        t.za = (int)(pa * g.n_h + t.h);
        t.zb = (int)(pb * g.n_h + t.h);
    } else {
        // group (trajectory) of this tile: largest grp with grp_tile0[grp] <= tile
        int64_t lo = 0, hi = g.n_groups - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (g.grp_tile0[mid] <= tile) lo = mid;
            else hi = mid - 1;
        }
        const int64_t r = tile - g.grp_tile0[lo];
        const int64_t r0 = (int64_t)g.grp_net0[lo] << g.m_bits, r1 = (int64_t)g.grp_net0[lo + 1] << g.m_bits;
        const int64_t tmg = (r1 - r0 + kBM - 1) / kBM;
        t.m0 = (int)(r0 + (r % tmg) * kBM);
        t.n0 = (int)((r / tmg) * kBN);
        t.inst = lo;          // the trajectory (local index) supplies the B operand
        t.h = 0;
        t.row_end = r1;
        t.za = 0;
        t.zb = g.b_pcls == CLS_TRAJ ? (int)lo : 0;
    }
    return t;
}

template <int F>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          const __grid_constant__ GemmArgs g) {
    constexpr int kBK = kRowBytes / Fmt<F>::kBytes;   // elements per swizzle row
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* stage0 = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;   // per accumulator set
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    int64_t* noff_all = reinterpret_cast<int64_t*>(tslot + 4);   // 8 epilogue warps x kBN / 2 column offsets
    float* ucol_all = reinterpret_cast<float*>(noff_all + 8 * (kBN / 2));   // FP16: column scales 2^eb
    float2* stg_all = reinterpret_cast<float2*>(smem + kStages * kStageBytes + kTabBytes);   // column-contiguous staging
    int64_t* rbase_all = reinterpret_cast<int64_t*>(stg_all + 4 * 32 * kStgPitch);
    // Work items are (tile, K segment) pairs.  A tile's k-blocks run in
    // segments of at most kSegKb; the tensor core's accumulation truncates, so
    // long chains drift: every segment is accumulated on its own and the
    // epilogue adds the segments in FP32 (round to nearest), in order, into a
    // running sum kept in TMEM columns [2 kBN, 3 kBN), then writes the tile
    // once.  Segmented tiles use two accumulator sets of one accumulator, short
    // contractions (at most 8 k-blocks) two sets of kAcc / 2 (the epilogue of
    // one item overlaps the MMAs of the next); the others one set of kAcc.
    const int seg_kb = g.nkb > kSegKb ? kSegKb : g.nkb;
    const int n_seg = (g.nkb + seg_kb - 1) / seg_kb;
    const int n_sets = (g.nkb <= 8 || n_seg > 1) ? 2 : 1;
    const int acc_per = n_seg > 1 ? 1 : kAcc / n_sets;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 32) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int k = 0; k < 2; k++) {
            mbar_init(&acc_full[k], 1);
            mbar_init(&acc_empty[k], g.col_out ? 4 : 8);   // one arrival per working epilogue warp
        }
        mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int64_t n_tiles = g.n_tiles;

    if (warp == 0) {
        if (lane == 0) {
            int64_t it = 0;
            for (int64_t tile = blockIdx.x; tile < n_tiles && !*abort; tile += gridDim.x) {
                const TileInfo t = decode_tile(g, tile);
                for (int kb = 0; kb < g.nkb; kb++, it++) {
                    const int s = (int)(it % kStages);
                    if (it >= kStages && !mbar_wait(&empty[s], (uint32_t)((it / kStages) - 1) & 1u, abort, g.wait_ns)) {
                        atomicExch(g.err, 1);
                        *abort = 1;
                        break;
                    }
                    uint8_t* st = stage0 + s * kStageBytes;
                    mbar_expect_tx(&full[s], (uint32_t)kStageBytes);
                    tma_load_3d(st, &tmA, kb * kBK, t.m0, t.za, &full[s]);                          // A hi
                    tma_load_3d(st + kTileA, &tmA, g.Kh + kb * kBK, t.m0, t.za, &full[s]);          // A lo
                    tma_load_3d(st + 2 * kTileA, &tmB, kb * kBK, t.n0, t.zb, &full[s]);             // B hi
                    tma_load_3d(st + 2 * kTileA + kTileB, &tmB, g.Kh + kb * kBK, t.n0, t.zb, &full[s]);   // B lo
                }
            }
            // let this CTA's own copies land before it exits (on every path: the
            // MMA thread may have stopped early): the last load of every stage
            // is that stage's newest phase
            const int64_t first = it > kStages ? it - kStages : 0;
            for (int64_t j = first; j < it; j++) mbar_wait_plain(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int64_t it = 0, lt = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < n_tiles && !*abort && ok; tile += gridDim.x) {
                for (int sg = 0; sg < n_seg && ok; sg++, lt++) {
                    const int set = (int)(lt % n_sets);
                    // this set's previous item has been drained by the epilogue
                    if (lt >= n_sets &&
                        !mbar_wait(&acc_empty[set], (uint32_t)((lt / n_sets - 1) & 1), abort, g.wait_ns)) {
                        atomicExch(g.err, 4);
                        *abort = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int kb0 = sg * seg_kb, kb1 = kb0 + seg_kb < g.nkb ? kb0 + seg_kb : g.nkb;
                    for (int kb = kb0; kb < kb1; kb++, it++) {
                        const int s = (int)(it % kStages);
                        if (!mbar_wait(&full[s], (uint32_t)(it / kStages) & 1u, abort, g.wait_ns)) {
                            atomicExch(g.err, 2);
                            *abort = 1;
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(stage0 + s * kStageBytes);
                        const uint32_t sal = sa + kTileA, sb = sa + 2 * kTileA, sbl = sb + kTileB;
                        const int j = kb - kb0;
                        const uint32_t acc = tmem + (uint32_t)((set * acc_per + j % acc_per) * kBN);
                        const bool fresh = j < acc_per;
#pragma unroll
                        for (int kk = 0; kk < kRowBytes / 32; kk++) {   // 32 bytes of K per MMA
                            const uint32_t o = kk * 32;
                            umma<F>(acc, sdesc_sw128(sa + o), sdesc_sw128(sb + o), (fresh && kk == 0) ? 0u : 1u);
                            umma<F>(acc, sdesc_sw128(sa + o), sdesc_sw128(sbl + o), 1u);
                            umma<F>(acc, sdesc_sw128(sal + o), sdesc_sw128(sb + o), 1u);
                        }
                        umma_commit(&empty[s]);   // stage free once these MMAs have read it
                    }
                    if (!ok) break;
                    umma_commit(&acc_full[set]);  // accumulators complete for this item
                }
            }
            // MMAs still in flight finish before TMEM is freed (on every path: the
            // epilogue may have stopped early)
            umma_commit(drain);
            mbar_wait_plain(drain, 0u);
        }
        __syncwarp();
    } else {
        // epilogue warps 2..9: TMEM lane quadrant q = warp % 4 holds tile rows
        // 32q..32q+31; two warps per quadrant drain half of the tile's columns
        // each (one warp per SM sub-partition leaves its load and store
        // latencies exposed).  Column-contiguous outputs, which go through the
        // staging buffers, use warps 2..5 only, each over all columns.
        const int ew = warp - 2, q = warp & 3;
        const int n_epi = g.col_out ? 4 : 8;
        const int c_lo = g.col_out ? 0 : (ew >> 2) * (kBN / 2), c_hi = g.col_out ? kBN : c_lo + kBN / 2;
        int64_t* noff = noff_all + ew * (kBN / 2);
        float* ucol = ucol_all + ew * (kBN / 2);
        float2* stg = stg_all + (ew & 3) * 32 * kStgPitch;
        int64_t* rbase = rbase_all + (ew & 3) * 32;
        int64_t lt = 0;
        bool live = ew < n_epi;
        for (int64_t tile = blockIdx.x; tile < n_tiles && live; tile += gridDim.x) {
            if (__shfl_sync(0xffffffffu, *abort, 0)) break;   // warp-uniform stop
            const TileInfo t = decode_tile(g, tile);
            for (int c = c_lo / 2 + lane; c < c_hi / 2; c += 32) {   // output offsets of this warp's columns
                const int64_t n = (int64_t)(t.n0 / 2) + c;
                int64_t off = 0;
                for (int i = 0; i < g.n_nb; i++)
                    if ((n >> i) & 1) off += g.n_stride[i];
                noff[c] = off;
            }
            const int64_t row = (int64_t)t.m0 + q * 32 + lane;
            int64_t m = row, out_inst = g.out_map ? (int64_t)g.out_map[t.inst] : t.inst;
            if (g.stacked) {
                out_inst = row >> g.m_bits;
                m = row & (((int64_t)1 << g.m_bits) - 1);
            }
            int64_t moff = 0;
            for (int i = 0; i < g.n_mb; i++)
                if ((m >> i) & 1) moff += g.m_stride[i];
            for (int i = 0; i < g.n_hb; i++)
                if ((t.h >> i) & 1) moff += g.h_stride[i];
            const bool row_ok = row < t.row_end;
            float2* out = g.out + (row_ok ? out_inst : 0) * g.out_size + moff;
            if (g.col_out) rbase[lane] = row_ok ? out_inst * g.out_size + moff : -1;
            __syncwarp();
            for (int sg = 0; sg < n_seg; sg++, lt++) {
                const int set = (int)(lt % n_sets);
                const uint32_t acc0 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(set * acc_per * kBN);
                const int seg_len = (sg + 1) * seg_kb < g.nkb ? seg_kb : g.nkb - sg * seg_kb;
                const int n_acc = seg_len < acc_per ? seg_len : acc_per;
                const bool add = sg > 0;   // later segments add to the running sum
                // FP16: the segment's A row scale 2^ea (packed row za * M + row) and
                // column scales 2^eb; their product 2^(ea + eb) is exact
                float urow = 1.f;
                if (F == FMT_FP16) {
                    for (int c = c_lo / 2 + lane; c < c_hi / 2; c += 32) {
                        const int64_t n = (int64_t)(t.n0 / 2) + c;
                        ucol[c] = 2 * n < g.N2
                                      ? ldexpf(1.f, (int)g.exp_b[((int64_t)t.zb * (g.N2 >> 1) + n) * n_seg + sg])
                                      : 0.f;
                    }
                    if (row_ok) urow = ldexpf(1.f, (int)g.exp_a[((int64_t)t.za * g.M + row) * n_seg + sg]);
                    __syncwarp();
                }
                // one lane waits and the warp follows its outcome (lanes polling on
                // their own could disagree when a wait gives up)
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&acc_full[set], (uint32_t)((lt / n_sets) & 1), abort, g.wait_ns) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) {
                        atomicExch(g.err, 3);
                        *abort = 1;
                    }
                    live = false;
                    break;
                }
                __syncwarp();
                tc_fence_after();
                // one chunk of 32 columns of this thread's row: v[2j], v[2j+1] = complex
                // column (c0 / 2 + j), written through the output strides
                auto store_chunk = [&](int c0, const float* v) {
                    if (g.col_out) {
                        // column-contiguous output: the warp's 32 x 16 fragment goes
                        // through shared memory, then 16 lanes store 16 consecutive
                        // columns of one row (two rows per store instruction)
#pragma unroll
                        for (int j = 0; j < 16; j++) stg[lane * kStgPitch + j] = make_float2(v[2 * j], v[2 * j + 1]);
                        __syncwarp();
                        const int cc = lane & 15;
                        const bool col_ok = t.n0 + c0 + 2 * cc < g.N2;
                        const int64_t no = noff[(c0 >> 1) + cc];
#pragma unroll 4
                        for (int i = 0; i < 16; i++) {
                            const int rr = 2 * i + (lane >> 4);
                            const int64_t rb = rbase[rr];
                            if (rb >= 0 && col_ok) g.out[rb + no] = stg[rr * kStgPitch + cc];
                        }
                        __syncwarp();
                    } else if (row_ok) {
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const int col = t.n0 + c0 + 2 * j;
                            if (col < g.N2) out[noff[(c0 >> 1) + j]] = make_float2(v[2 * j], v[2 * j + 1]);
                        }
                    }
                };
                if (n_seg == 1) {
#pragma unroll 1
                    for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
                        float v[32];
                        uint32_t r[32];
                        tmem_ld32(acc0 + (uint32_t)c0, r);
#pragma unroll
                        for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
                        for (int a = 1; a < n_acc; a++) {
                            tmem_ld32(acc0 + (uint32_t)(a * kBN + c0), r);
#pragma unroll
                            for (int j = 0; j < 32; j++) v[j] += __uint_as_float(r[j]);
                        }
                        if (F == FMT_FP16) {
#pragma unroll
                            for (int j = 0; j < 16; j++) {
                                const float u = urow * ucol[(c0 >> 1) + j];
                                v[2 * j] *= u;
                                v[2 * j + 1] *= u;
                            }
                        }
                        store_chunk(c0, v);
                    }
                } else {
                    // segmented: add this segment to the running sum in TMEM; the
                    // last one writes the tile
#pragma unroll 1
                    for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
                        float v[32];
                        uint32_t r[32];
                        tmem_ld32(acc0 + (uint32_t)c0, r);
#pragma unroll
                        for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
                        if (F == FMT_FP16) {
#pragma unroll
                            for (int j = 0; j < 16; j++) {
                                const float u = urow * ucol[(c0 >> 1) + j];
                                v[2 * j] *= u;
                                v[2 * j + 1] *= u;
                            }
                        }
                        const uint32_t sa = tmem + ((uint32_t)(q * 32) << 16) + 2 * kBN + (uint32_t)c0;
                        if (add) {
                            tmem_ld32(sa, r);
#pragma unroll
                            for (int j = 0; j < 32; j++) v[j] += __uint_as_float(r[j]);
                        }
                        if (sg + 1 < n_seg) {
#pragma unroll
                            for (int j = 0; j < 32; j++) r[j] = __float_as_uint(v[j]);
                            tmem_st32(sa, r);
                        } else {
                            store_chunk(c0, v);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[set]);   // accumulators read: this set may take the next item
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Tiles of every trajectory group of a stacked GEMM (cnt[n_groups] = 0, so the
// exclusive scan of cnt ends with the total).
__global__ void k_group_tiles(const int32_t* __restrict__ net0, int64_t n_groups, int m_bits, int64_t tiles_n,
                              int64_t* __restrict__ cnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g > n_groups) return;
    if (g == n_groups) {
        cnt[g] = 0;
        return;
    }
    const int64_t r = (int64_t)(net0[g + 1] - net0[g]) << m_bits;
    cnt[g] = ((r + kBM - 1) / kBM) * tiles_n;
}

// ---------------------------------------------------------- host helpers --
std::atomic<uint64_t> g_wait_ns{2000000000ull};   // limit of the GEMM's pipeline waits

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    // thread-safe one-time lookup (function-local static initialisation)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    return fn;
}

// 3D map over packed rows: (elements of a row, rows, instances), boxes of one
// 128-byte swizzle row by box_rows rows.
ptn_status make_map(CUtensorMap* m, void* base, CUtensorMapDataType dt, int ebytes, int64_t row_elems, int64_t rows,
                    int64_t zs, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(PTN_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)row_elems, (cuuint64_t)rows, (cuuint64_t)zs};
    cuuint64_t strides[2] = {(cuuint64_t)row_elems * ebytes, (cuuint64_t)row_elems * ebytes * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / ebytes), (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PTN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PTN_OK;
}

int pack_class(const OperandDesc& d, int step_cls) {
    if (step_cls == CLS_NET && d.n_slice) return CLS_NET;
    if (d.mode == OP_LEAF) return d.leaf_col >= 0 ? CLS_TRAJ : CLS_CONST;
    return d.cls;
}

unsigned grid_of(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <int F>
ptn_status run_gemm(const StepDesc& st, const ChunkCtx& ctx, int64_t n_inst, void* pack_a, void* pack_b,
                    int* err, const GroupTable& grp, cudaStream_t s, const StepDesc* prod_src) {
    constexpr int kEB = Fmt<F>::kBytes;
    constexpr int kBK = kRowBytes / kEB;
    const CUtensorMapDataType dt = F == FMT_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : F == FMT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const bool stacked = st.kind == STEP_GEMM_STACKED;
    const int a = st.gemm_a, b = 1 - a;
    PackArgs pa, pb;
    memset(&pa, 0, sizeof pa);
    memset(&pb, 0, sizeof pb);
    GemmArgs ga;
    memset(&ga, 0, sizeof ga);
    int nm = 0, nn = 0, nh = 0;
    for (int p = 0; p < st.n_out; p++) {
        const int64_t sa = st.out_stride[a][p], sb = st.out_stride[b][p], so = (int64_t)1 << p;
        if (sa && sb) {
            pa.h_stride[nh] = sa;
            pb.h_stride[nh] = sb;
            ga.h_stride[nh] = so;
            nh++;
        } else if (sa) {
            pa.r_stride[nm] = sa;
            ga.m_stride[nm] = so;
            nm++;
        } else {
            pb.r_stride[nn] = sb;
            ga.n_stride[nn] = so;
            nn++;
        }
    }
    for (int q = 0; q < st.n_sum; q++) {
        pa.k_stride[q] = st.sum_stride[a][q];
        pb.k_stride[q] = st.sum_stride[b][q];
    }
    const int64_t M = (int64_t)1 << nm, N = (int64_t)1 << nn, Kc = (int64_t)1 << st.n_sum;
    const int64_t Kh = ((2 * Kc + kBK - 1) / kBK) * kBK;
    // A cached step (trajectory class, never stacked) runs over the chunk's
    // representatives of its slot: its trajectory-class operands are packed
    // for those instances only and its tiles write their trajectories' outputs.
    const int32_t* cmap = (st.cache > 0 && ctx.cache_list) ? ctx.cache_list + (int64_t)(st.cache - 1) * ctx.cache_n
                                                           : nullptr;
    const int64_t inst_of[3] = {1, cmap ? n_inst : ctx.arena_inst[CLS_TRAJ], ctx.arena_inst[CLS_NET]};
    pa.op = st.op[a];
    pb.op = st.op[b];
    pa.pcls = pack_class(st.op[a], st.out_cls);
    pb.pcls = pack_class(st.op[b], st.out_cls);
    if (st.prod) {
        // the operand st.prod - 1 is prod_src's outer product: bit p of it (stride
        // 2^p) is bit p of prod_src's output, at strides out_stride[0 / 1][p] of
        // the two factors, packed into one word (low / high 32 bits)
        if (!prod_src || st.prod < 1 || st.prod > 2)
            return set_error(PTN_ERR_INVALID_ARG, "internal: outer-product operand without its step");
        PackArgs& px = st.prod - 1 == a ? pa : pb;
        bool ok = true;
        auto packed = [&](int64_t v) -> int64_t {
            if (v <= 0 || (v & (v - 1))) {
                ok = false;
                return 0;
            }
            const int p = __builtin_ctzll((unsigned long long)v);
            if (p >= prod_src->n_out) {
                ok = false;
                return 0;
            }
            return prod_src->out_stride[0][p] | (prod_src->out_stride[1][p] << 32);
        };
        const int n_rb = st.prod - 1 == a ? nm : nn;
        for (int i = 0; i < n_rb; i++) px.r_stride[i] = packed(px.r_stride[i]);
        for (int i = 0; i < nh; i++) px.h_stride[i] = packed(px.h_stride[i]);
        for (int i = 0; i < st.n_sum; i++) px.k_stride[i] = packed(px.k_stride[i]);
        if (!ok) return set_error(PTN_ERR_INVALID_ARG, "internal: outer-product operand with a non-dense stride");
        px.prod = 1;
        px.xconj = st.op[st.prod - 1].conj;
        px.op = prod_src->op[0];
        px.op1 = prod_src->op[1];
    }
    pa.role = 0;
    pb.role = 1;
    pa.n_rb = nm;
    pb.n_rb = nn;
    pa.n_hb = pb.n_hb = nh;
    pa.n_kb = pb.n_kb = st.n_sum;
    pa.Kh = pb.Kh = (int32_t)Kh;
    pa.n_pinst = inst_of[pa.pcls];
    pb.n_pinst = inst_of[pb.pcls];
    pa.inst_map = pa.pcls == CLS_TRAJ ? cmap : nullptr;
    pb.inst_map = pb.pcls == CLS_TRAJ ? cmap : nullptr;
    pa.dst = pack_a;
    pb.dst = pack_b;
    ga.M = (int32_t)M;
    ga.N2 = (int32_t)(2 * N);
    ga.Kh = (int32_t)Kh;
    ga.nkb = (int32_t)(Kh / kBK);
    ga.n_h = 1 << nh;
    ga.a_pcls = pa.pcls;
    ga.b_pcls = pb.pcls;
    ga.out_cls = st.out_cls;
    ga.n_mb = nm;
    ga.n_nb = nn;
    ga.n_hb = nh;
    ga.col_out = (nn > 0 && ga.n_stride[0] == 1) ? 1 : 0;
    ga.tiles_m = (M + kBM - 1) / kBM;
    ga.tiles_n = (2 * N + kBN - 1) / kBN;
    ga.n_inst = n_inst;
    ga.net_tl = ctx.net_tl;
    ga.out = ctx.arena[st.out_arena] + st.out_off * ctx.arena_inst[st.out_arena];
    ga.out_size = st.out_size;
    ga.out_map = cmap;
    ga.err = err;
    ga.wait_ns = g_wait_ns.load(std::memory_order_relaxed);
    const int64_t tot_a = pa.n_pinst * (1ll << nh) * M * (Kh / 2);
    const int64_t tot_b = pb.n_pinst * (1ll << nh) * N * (Kh / 2);
    cudaError_t e;
    if (F == FMT_FP16) {
        // row exponents live after the packed rows (the pack buffers are sized for
        // 4-byte elements plus slack, FP16 rows use half of that)
        auto after = [&](void* base, int64_t rows) {
            const int64_t bytes = rows * 2 * Kh * kEB;
            return reinterpret_cast<int8_t*>(static_cast<uint8_t*>(base) + ((bytes + 255) & ~(int64_t)255));
        };
        pa.row_exp = after(pack_a, pa.n_pinst * (1ll << nh) * M);
        pb.row_exp = after(pack_b, pb.n_pinst * (1ll << nh) * 2 * N);   // B rows are realified pairs
        ga.exp_a = pa.row_exp;
        ga.exp_b = pb.row_exp;
        pa.seg_slots = pb.seg_slots = kSegKb * kBK / 2;
        if (Kh / 2 < 32) return set_error(PTN_ERR_INVALID_ARG, "internal: FP16 rows shorter than a warp");
    }
    {
        // algorithmic bytes: every operand element read once (an outer-product
        // operand: its two factors per instance), the hi/lo rows written once
        auto rd = [&](const PackArgs& pk, int64_t tot) {
            return pk.prod ? 8.0 * (double)pk.n_pinst * (double)(pk.op.inst_size + pk.op1.inst_size)
                           : 8.0 * (double)tot;
        };
        StatScope sc(K_PACK, s, rd(pa, tot_a) + rd(pb, tot_b) + 4.0 * kEB * (double)tot_a + 8.0 * kEB * (double)tot_b,
                     0.0);
        // (grid_of sizes by complex slots; the kernels stride over rows)
        for (PackArgs* pk : {&pa, &pb}) {
            const int64_t tot = pk == &pa ? tot_a : tot_b;
            k_pack<F><<<grid_of(tot), 256, 0, s>>>(*pk, ctx);
        }
        count_launches(K_PACK);   // two pack kernels under one scope
    }
    CUtensorMap mA, mB;
    int64_t blocks = ga.tiles_m * ga.tiles_n * n_inst * (1ll << nh);
    ptn_status ps;
    if (!stacked) {
        ps = make_map(&mA, pack_a, dt, kEB, 2 * Kh, M, pa.n_pinst * (1ll << nh), kBM);
    } else {
        // rows of all networks, network-major; groups (trajectories) tile separately.
        // The pack buffer holds at least one full tile of rows (planner), so a
        // chunk with fewer rows still spans the TMA box.
        const int64_t rows = pa.n_pinst * M;
        ps = make_map(&mA, pack_a, dt, kEB, 2 * Kh, rows < kBM ? kBM : rows, 1, kBM);
        ga.stacked = 1;
        ga.m_bits = nm;
        ga.n_groups = grp.n_groups;
        ga.grp_net0 = grp.d_net0;
        ga.grp_tile0 = grp.d_tile0;
        int64_t acc = 0;   // the same count the device tile table ends with
        for (int64_t gi = 0; gi < grp.n_groups; gi++) {
            const int64_t r = (int64_t)(grp.h_net0[gi + 1] - grp.h_net0[gi]) * M;
            acc += ((r + kBM - 1) / kBM) * ga.tiles_n;
        }
        blocks = acc;
        count_launches(K_MISC);
        k_group_tiles<<<(unsigned)((grp.n_groups + 256) / 256), 256, 0, s>>>(grp.d_net0, grp.n_groups, nm,
                                                                              ga.tiles_n, grp.d_cnt);
        launch_exclusive_scan(grp.d_cnt, grp.d_tile0, grp.n_groups + 1, grp.d_scan, s);
    }
    if (ps) return ps;
    ps = make_map(&mB, pack_b, dt, kEB, 2 * Kh, 2 * N, pb.n_pinst * (1ll << nh), kBN);
    if (ps) return ps;
    static const bool attr_set = [] {
        cudaFuncSetAttribute(k_gemm<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
        return true;
    }();
    (void)attr_set;
    if (blocks <= 0) return PTN_OK;
    const double flops = 8.0 * (double)n_inst * (double)(1ll << nh) * (double)M * (double)N * (double)Kc;
    const double bytes = 8.0 * ((double)n_inst * (1ll << nh) * M * N) +
                         (double)kEB * 2 * Kh * ((double)pa.n_pinst * M + (double)pb.n_pinst * 2 * N) * (1ll << nh);
    StatScope sc(K_CONTRACT_GEMM, s, bytes, flops);
    ga.n_tiles = blocks;
    static const int n_sm = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 148;
    }();
    const int64_t grid = blocks < n_sm ? blocks : n_sm;
    k_gemm<F><<<(unsigned)grid, kGemmThreads, kGemmSmem, s>>>(mA, mB, ga);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PTN_ERR_CUDA, "gemm launch: %s", cudaGetErrorString(e));
    return PTN_OK;
}

}  // namespace

ptn_status launch_gemm_step(const StepDesc& st, const ChunkCtx& ctx, int64_t n_inst, void* pack_a, void* pack_b,
                            int* err, const GroupTable& grp, int precision,
                            cudaStream_t s, const StepDesc* prod_src) {
    // Contractions of at most 16 complex terms run in TF32 hi/lo in every mode:
    // they fill one 128-byte K-block of TF32 exactly where a 16-bit K-block
    // would be half padding, and their time is the epilogue's (FP16 adds
    // per-row and per-column scales there); TF32 hi/lo is FP32-accurate.
    if (precision != PTN_PREC_FP32 && st.n_sum <= 4 &&
        (precision == PTN_PREC_BF16X3 || precision == PTN_PREC_FP16X3))
        precision = PTN_PREC_FP32;
    switch (precision) {
        case PTN_PREC_FP32: return run_gemm<FMT_TF32>(st, ctx, n_inst, pack_a, pack_b, err, grp, s, prod_src);
        case PTN_PREC_BF16X3: return run_gemm<FMT_BF16>(st, ctx, n_inst, pack_a, pack_b, err, grp, s, prod_src);
        case PTN_PREC_FP16X3: return run_gemm<FMT_FP16>(st, ctx, n_inst, pack_a, pack_b, err, grp, s, prod_src);
    }
    return set_error(PTN_ERR_UNSUPPORTED, "precision mode %d", precision);
}

}  // namespace ptn

extern "C" ptn_status ptn_set_wait_limit(double seconds) {
    if (!(seconds >= 0.0 && seconds <= 60.0))
        return ptn::set_error(PTN_ERR_INVALID_ARG, "wait limit %g s outside 0..60", seconds);
    ptn::g_wait_ns.store((uint64_t)(seconds * 1e9), std::memory_order_relaxed);
    return PTN_OK;
}
