// Device helpers and kernel launchers shared by the runtime's .cu files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ptn_internal.h"

namespace ptn {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies mixed with the key, the key bumped by the Weyl constants between
// rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint64_t word64(uint4 x) {
    return ((uint64_t)x.x << 32) | (uint64_t)x.y;
}

// Exact-integer quantisation of probabilities without FP64 arithmetic (the
// GB300's FP64 rate is a small fraction of its integer rate): for a float p,
// quant_pow2(p, s) = rint(max(p, 0) * 2^s) (rint: round half to even), the
// value the FP64 expression gives, since p * 2^s is exact in FP64.  The
// caller chooses s so that the result stays below 2^63.
__device__ __forceinline__ uint64_t quant_pow2(float p, int s) {
    if (!(p > 0.f)) return 0;
    const uint32_t bits = __float_as_uint(p);
    const int be = (int)((bits >> 23) & 0xFFu);
    uint64_t m = bits & 0x7FFFFFu;
    int E = -149;                      // subnormal: value = m * 2^-149
    if (be) {
        m |= 0x800000u;
        E = be - 150;                  // normal: value = m * 2^(be - 150)
    }
    const int sh = E + s;
    if (sh >= 0) return m << sh;
    const int d = -sh;
    if (d > 24) return 0;              // value < 0.5
    uint64_t q = m >> d;
    const uint64_t rem = m & ((1ull << d) - 1), half = 1ull << (d - 1);
    if (rem > half || (rem == half && (q & 1ull))) q++;
    return q;
}
// e with m = f * 2^e, f in [0.5, 1), as frexp((double)m) gives for a float m
// >= 0 (0 for m = 0).
__device__ __forceinline__ int frexp_exp(float m) {
    const uint32_t bits = __float_as_uint(m);
    const int be = (int)((bits >> 23) & 0xFFu);
    if (be) return be - 126;
    const uint32_t frac = bits & 0x7FFFFFu;
    return frac ? (31 - __clz((int)frac)) - 148 : 0;
}

// Counter word 3: (stream << 24) | (circuit << 8) | block.
enum { STREAM_KRAUS = 1, STREAM_ALLOC = 2, STREAM_SAMPLE = 3 };
__host__ __device__ __forceinline__ uint32_t philox_tag(int stream, int circuit, int block) {
    return ((uint32_t)(stream & 0xFF) << 24) | ((uint32_t)(circuit & 0xFFFF) << 8) | (uint32_t)(block & 0xFF);
}

// Bitstrings of n qubits are W = ceil(n / 64) little-endian 64-bit words (bit q
// of the string is bit q % 64 of word q / 64).
__device__ __forceinline__ uint64_t bits_get(const uint64_t* w, int q) { return (w[q >> 6] >> (q & 63)) & 1ull; }
// dst = src with the outcome x of a block placed at bit `start` (those bits of
// src are zero); x may straddle two words
__device__ __forceinline__ void bits_put(uint64_t* dst, const uint64_t* src, int n_words, uint64_t x, int start) {
    const int w0 = start >> 6, sh = start & 63;
    for (int w = 0; w < n_words; w++) {
        uint64_t v = src[w];
        if (w == w0) v |= x << sh;
        else if (w == w0 + 1 && sh) v |= x >> (64 - sh);
        dst[w] = v;
    }
}

// Per-chunk execution context of a block's step list.
struct ChunkCtx {
    const float2* vtab;         // merged-gate variant table
    const int32_t* var_ids;     // [traj][n_var_cols] variant of every multi-variant leaf
    int32_t n_var_cols;
    int32_t n_words;            // 64-bit words per prefix (ceil(n_qubits / 64))
    const int32_t* chunk_traj;  // local trajectory -> global (index into var_ids)
    const int32_t* net_tl;      // network -> local trajectory
    const uint64_t* net_prefix; // network -> prefix bits, n_words little-endian words each
    float2* arena[N_ARENAS];    // CONST, TRAJ, NET (+ ADJ, LGRAD for gradients) arenas
    int64_t arena_inst[N_ARENAS];   // instances of each arena in this chunk
    // intermediate caching (StepDesc.cache / OperandDesc.cache), null when off:
    // cache_rep[k * cache_n + tl] the representative of local trajectory tl for
    // cache slot k (the first trajectory of the chunk with the same variants on
    // the slot's columns), cache_list[k * cache_n + i] the i-th representative
    const int32_t* cache_rep = nullptr;
    const int32_t* cache_list = nullptr;
    int64_t cache_n = 0;
};

// Instance of a TRAJ-class buffer that local trajectory tl reads.
__device__ __forceinline__ int64_t rep_inst(const OperandDesc& d, int64_t tl, const ChunkCtx& c) {
    return (d.cache > 0 && c.cache_rep) ? (int64_t)c.cache_rep[(int64_t)(d.cache - 1) * c.cache_n + tl] : tl;
}
// Trajectory computed by the i-th instance of a launch of a step with cache id `cache`.
__device__ __forceinline__ int64_t step_inst(int32_t cache, int64_t i, const ChunkCtx& c) {
    return (cache > 0 && c.cache_list) ? (int64_t)c.cache_list[(int64_t)(cache - 1) * c.cache_n + i] : i;
}

// ---- intermediate caching (kernels_cache.cu)
// Per trajectory (of a ptn_traj) its non-zero variant entries, in column
// order: cnt holds n + 1 int64 (exclusive-scanned into the row pointers).
void launch_nz_count(const int32_t* var_ids, int64_t n, int32_t n_cols, int64_t* cnt, cudaStream_t s);
void launch_nz_fill(const int32_t* var_ids, int64_t n, int32_t n_cols, const int64_t* ptr, int32_t* col,
                    int32_t* val, cudaStream_t s);
struct CacheArgs {
    int32_t n_cache = 0, words = 0;   // cache slots of the block; 32-bit words per column bitmap
    int64_t n = 0;                    // trajectories of the chunk
    int64_t P = 0;                    // hash-table entries per slot (a power of two >= 2n)
    const int32_t* chunk_traj = nullptr;   // local -> global trajectory
    const int64_t* nz_ptr = nullptr;       // per global trajectory: its non-zero variant entries
    const int32_t* nz_col = nullptr;
    const int32_t* nz_val = nullptr;
    const uint32_t* bits = nullptr;        // [n_cache][words] column bitmaps
    uint64_t* h = nullptr;                 // [n_cache][n][2] key halves
    unsigned long long* keys = nullptr;    // [n_cache][P]
    int32_t* first = nullptr;              // [n_cache][P]
    int32_t* rep = nullptr;                // [n_cache][n] representative of every trajectory
    int32_t* list = nullptr;               // [n_cache][n] representatives in increasing order
    int32_t* cnt = nullptr;                // [n_cache] representatives per slot
};
void launch_cache_tables(const CacheArgs& a, cudaStream_t s);

// ---- launchers (kernels_contract.cu)
// a run of small trajectory-class steps (small_step, fuse_prev) in one launch
void launch_small_steps(const StepDesc* d_steps, const StepDesc* h_steps, int n_steps, const ChunkCtx& ctx,
                        int64_t n_traj, cudaStream_t s);
void launch_contract_step(const StepDesc* d_step, const StepDesc& h_step, const ChunkCtx& ctx,
                          int64_t n_inst, cudaStream_t s);
// marginal rows (real diagonal of the root) and their FP64 totals; part holds
// n_net * finalize_tiles(b) doubles when finalize_tiles(b) > 1 (else unused)
int64_t finalize_tiles(int b);
void launch_finalize(const RootRef* d_root, const ChunkCtx& ctx, int b, int64_t n_net, float* marg, double* Z,
                     double* part, cudaStream_t s);

// ---- tensor-core steps (kernels_gemm.cu); err: device word set on a timeout
// Networks of a chunk grouped by trajectory: group g holds networks
// [net0[g], net0[g+1]) (host and device copies); the rest is device scratch
// for the per-step tile table of stacked GEMMs.
struct GroupTable {
    int64_t n_groups = 0;
    const int32_t* h_net0 = nullptr;
    const int32_t* d_net0 = nullptr;
    int64_t* d_cnt = nullptr;     // n_groups + 1
    int64_t* d_tile0 = nullptr;   // n_groups + 1
    int64_t* d_scan = nullptr;    // scan_tmp_elems(n_groups + 1)
};
// precision: PTN_PREC_*.  pack_a / pack_b: packing scratch sized for 4-byte
// elements plus 1/64 slack (the FP16 mode keeps its per-row exponents there).
// prod_src: the (virt) outer-product step whose output is the operand st.prod - 1, formed
// in the pack from its two factors (st.prod != 0), else null.
ptn_status launch_gemm_step(const StepDesc& st, const ChunkCtx& ctx, int64_t n_inst, void* pack_a, void* pack_b,
                            int* err, const GroupTable& grp, int precision, cudaStream_t s,
                            const StepDesc* prod_src = nullptr);

// ---- expectation values and gradients (kernels_expval.cu)
struct ObsTerm {
    double coeff;
    uint64_t zmask;
};
// Per trajectory: F = sum_x w(x) |psi(x)|^2 and the root adjoint w(x) conj(psi(x)),
// w(x) = sum_t coeff_t (-1)^popc(x & zmask_t).
void launch_observable(const RootRef* d_root, const ChunkCtx& ctx, int n, const ObsTerm* terms, int n_terms,
                       int64_t root_adj_off, int64_t traj0, double* F, cudaStream_t s);
// amp[t][x] = psi_t(x), bit q of x = qubit q, for the n_traj trajectories of the chunk
void launch_amplitudes(const RootRef* d_root, const ChunkCtx& ctx, int n, int64_t n_traj, float2* amp, cudaStream_t s);
// partial[(traj0 + i) * n_params + param] += 2 Re sum_e G_leaf[e] dLeaf[e]
void launch_leaf_grad(const ChunkCtx& ctx, const ParamLeaf* d_pl, int n_pl, const float2* dvt, int64_t traj0,
                      int64_t n_traj, int n_params, double* partial, cudaStream_t s);
// value = sum_i c_i F_i / sum c_i, grad[p] = sum_i c_i partial[i][p] / sum c_i
void launch_expval_reduce(const int64_t* mult, const double* F, const double* partial, int64_t n_traj, int n_params,
                          double* value, double* grad, cudaStream_t s);

// ---- launchers (kernels_sample.cu)
// trajectory traj0 + i of the draw is row i (Philox counter word 2 = traj0 + i)
void launch_presample(const SiteTable* sites, int32_t n_sites, int64_t n_traj, int64_t traj0, uint64_t seed,
                      int32_t circuit, uint8_t* kraus, double* logq, cudaStream_t s);
void launch_row_hash(const uint8_t* kraus, int64_t n, int32_t S, uint64_t* h, cudaStream_t s);
// first[i] = smallest index whose Kraus row equals row i, from the (hash, index)
// pairs sorted stably by hash (idx: indices in sorted order) and the run
// flags / exclusive scan / run starts of the sorted hashes
void launch_first_in_run(const uint8_t* kraus, int32_t S, const int64_t* idx, const int64_t* flag, const int64_t* excl,
                         const int64_t* start, int64_t n, int64_t* first, cudaStream_t s);
void launch_iota_i64(int64_t* p, int64_t n, cudaStream_t s);
void launch_dedup_compact(const uint8_t* kraus, const double* logq, const int64_t* first,
                          const int64_t* uid, int64_t n, int32_t S, uint8_t* kraus_u,
                          double* logq_u, int64_t* mult_u, int64_t* first_u, cudaStream_t s);
void launch_var_ids(const uint8_t* kraus, int64_t n, int32_t S, const int32_t* ptr,
                    const int32_t* idx, const int32_t* mul, int32_t n_cols, int32_t* var_ids,
                    cudaStream_t s);
void launch_flags_first(const int64_t* first, int64_t n, int64_t* flags, cudaStream_t s);
// exclusive prefix sum of int64 (in may equal out); tmp must hold scan_tmp_elems(n) int64
int64_t scan_tmp_elems(int64_t n);
void launch_exclusive_scan(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);
void launch_alloc_shots(const double* w, int64_t n, int64_t total, uint64_t seed, int32_t circuit,
                        double* cdf_tmp, int64_t* m, cudaStream_t s);
void launch_mult_times_z(const int64_t* mult, const double* Z, int64_t n, double* w, cudaStream_t s);
void launch_fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s);
void launch_iota_i32(int32_t* p, int64_t n, cudaStream_t s);
void launch_scale_i64(const int64_t* a, int64_t k, int64_t n, int64_t* out, cudaStream_t s);

// ---- merging emitted shots across trajectories (kernels_merge.cu)
// one stable radix pass over 8 bits of key starting at `shift`; hist holds
// radix_hist_elems(n) int64, scan_tmp scan_tmp_elems(radix_hist_elems(n))
int64_t radix_hist_elems(int64_t n);
void launch_radix_pass(const uint64_t* key, const int64_t* val, int64_t n, int shift, int64_t* hist, int64_t* scan_tmp,
                       uint64_t* key_out, int64_t* val_out, cudaStream_t s);
void launch_run_flags(const uint64_t* key, int64_t n, int64_t* flag, cudaStream_t s);
// multi-word bitstrings ([n][n_words] records sorted as indices idx)
void launch_gather_word(const uint64_t* bits, const int64_t* idx, int n_words, int w, int64_t n, uint64_t* key,
                        cudaStream_t s);
void launch_run_flags_words(const uint64_t* bits, const int64_t* idx, int n_words, int64_t n, int64_t* flag,
                            cudaStream_t s);
void launch_run_sum_words(const uint64_t* bits, const int64_t* count, const int64_t* idx, int n_words,
                          const int64_t* start, int64_t n_runs, int64_t n, int32_t* traj_out, uint64_t* bits_out,
                          int64_t* count_out, cudaStream_t s);
void launch_run_starts(const int64_t* flag, const int64_t* excl, int64_t n, int64_t* start, cudaStream_t s);
void launch_run_sum(const uint64_t* key, const int64_t* val, const int64_t* start, int64_t n_runs, int64_t n,
                    int32_t* traj_out, uint64_t* bits_out, int64_t* count_out, cudaStream_t s);

// ---- final-block harvest of non-proportional sampling (kernels_harvest.cu)
struct HarvestArgs {
    const float* marg;          // [n_net][2^b] population vectors (unnormalised marginals)
    int b, start;
    int64_t n_net;
    bool direct;                // true: `shots` draws per network; false: threshold `tau`
    double tau;
    const int32_t* traj;        // [n_net]
    const uint64_t* prefix;     // [n_net][n_words]
    int n_words;                // 64-bit words per prefix and per output bitstring
    const int64_t* rank0;       // [n_net] first shot rank of each network (direct)
    int64_t shots;
    uint64_t seed;
    int circuit, block;
};
struct HarvestScratch {
    unsigned* rowmax;           // [n_net]
    unsigned long long* T;      // [n_net]
    uint64_t* tcdf;             // [n_net][harvest_cdf_tiles(b)] (direct)
    int64_t* tcnt;              // [n_net * harvest_tiles(b)]
    int64_t* toff;              // [n_net * harvest_tiles(b)]
    int64_t* scan_tmp;          // scan_tmp_elems(n_net * harvest_tiles(b))
    unsigned* cnt;              // [n_net][2^b] (direct)
};
int64_t harvest_tiles(int b);
int64_t harvest_cdf_tiles(int b);
// rank0[i] = (i - first network of traj[i]) * shots; first: n_traj_max scratch
void launch_harvest_ranks(const int32_t* traj, int64_t n, int64_t n_traj_max, int64_t shots,
                          unsigned long long* first, int64_t* rank0, cudaStream_t s);
// number of records of the networks (synchronises the stream), then the records
int64_t run_harvest_count(const HarvestArgs& a, const HarvestScratch& h, int64_t* host_tmp, cudaStream_t s,
                          ptn_status* st);
void run_harvest_write(const HarvestArgs& a, const HarvestScratch& h, int32_t* otraj, uint64_t* obits,
                       int64_t* ocount, double* oprob, cudaStream_t s);

struct SampleScratch {
    int64_t* cap;        // [n_parent] min(count, 2^b)
    int64_t* tmp_off;    // [n_parent]
    int64_t* rank0;      // [n_parent]
    int64_t* excl;       // [n_parent]
    int64_t* first;      // [n_traj_max]
    int64_t* ndist;      // [n_parent]
    int64_t* out_off;    // [n_parent]
    int32_t* tmp_x;      // [cap total]
    int64_t* tmp_c;      // [cap total]
    int64_t* scan_tmp;
};
// NBS sampling of one block; returns the number of children (synchronises).
int64_t run_sample_block(const float* marg, int b, int start, const int32_t* ptraj,
                         const uint64_t* pprefix, const int64_t* pcount, int64_t n_parent,
                         int64_t n_traj_max, uint64_t seed, int circuit, int block,
                         int32_t* ctraj, uint64_t* cprefix, int64_t* ccount, int64_t child_cap,
                         const SampleScratch& sc, int64_t* host_tmp, cudaStream_t s, ptn_status* st,
                         int n_words = 1);   // prefix words (pprefix / cprefix hold n_words per entry)

}  // namespace ptn
