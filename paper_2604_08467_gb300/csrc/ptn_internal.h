// Internal data structures shared by the host planner (planner.cpp) and the
// device runtime (runtime.cu, kernels_*.cu).  Not part of the public ABI.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ptn.h"

namespace ptn {

// Storage class of a tensor in a batch of block networks.
//   CONST: one copy for the whole batch;
//   TRAJ : one copy per distinct error set (trajectory) of the chunk;
//   NET  : one copy per network (trajectory, prefix) of the chunk.
enum Cls : int32_t { CLS_CONST = 0, CLS_TRAJ = 1, CLS_NET = 2 };
// Arenas a buffer can live in: the three storage classes, plus (expectation /
// gradient plans) the adjoints of intermediates and the adjoints of the
// parametrised gate tensors, both one copy per trajectory.
enum Arena : int32_t { ARENA_ADJ = 3, ARENA_LGRAD = 4, N_ARENAS = 5 };
enum OpMode : int32_t { OP_LEAF = 0, OP_BUF = 1 };

constexpr int kMaxOut = 40;     // output bits of one contraction step
constexpr int kMaxSum = 24;     // summed bits of one contraction step
constexpr int kMaxSlice = 64;   // prefix (projected) bits read by one operand
constexpr int kMaxBlocks = 64;
constexpr int kMaxQubits = 256;      // bitstrings of ceil(n / 64) 64-bit words (4 at most)
constexpr int kMaxSampleBlock = 14;   // blocks sampled by conditional draws (marginal CDF in shared memory)
constexpr int kMaxFinalBlock = 30;    // last block: harvested from its population vector in global memory
constexpr int kMaxKraus = 16;

// One operand of a batched pairwise contraction, as the kernels read it.
struct OperandDesc {
    int32_t mode;            // OP_LEAF: merged-gate variant table; OP_BUF: intermediate
    int32_t cls;             // storage class (CLS_*)
    int32_t conj;            // read the complex conjugate (bra layer)
    int32_t arena;           // OP_BUF: arena of the buffer (= its storage class)
    int64_t inst_size;       // elements per instance
    int64_t arena_off;       // OP_BUF: offset of the buffer in its arena, in elements per instance
    int64_t leaf_base;       // OP_LEAF: element offset of variant 0 in the variant table
    int32_t leaf_col;        // OP_LEAF: column of the variant index table, -1 = single variant
    int32_t n_slice;         // projected bits fixed from the network's prefix (NET steps)
    int32_t cache;           // OP_BUF of class TRAJ: 1 + cache slot of the step that wrote it (that
                             // step computed only representative trajectories: read instance
                             // rep[slot][tl]); 0 = every trajectory has its own instance
    int32_t reserved_c[3];
    int32_t slice_qubit[kMaxSlice];
    int64_t slice_stride[kMaxSlice];
};

// One batched pairwise contraction:
//   out[inst][o] = sum_k  A[inst'][addrA(o, k)] * B[inst''][addrB(o, k)]
// with o = sum_p bit_p << p over the n_out output bits and k over the n_sum
// summed bits; addr = sum_p bit_p(o) * out_stride[op][p] + sum_q bit_q(k) *
// sum_stride[op][q] + the operand's slice offset.
enum StepKind : int32_t { STEP_DIRECT = 0, STEP_GEMM = 1, STEP_GEMM_STACKED = 2 };

struct StepDesc {
    int32_t out_cls;
    int32_t n_out;
    int32_t n_sum;
    int32_t out_arena;
    int32_t kind;            // STEP_DIRECT or STEP_GEMM
    int32_t gemm_a;          // STEP_GEMM: which operand supplies the GEMM rows (the other is realified)
    int32_t fuse_prev;       // 1: may run in the same fused launch as the previous step (set by the planner)
    int32_t tile;            // SIMT micro-tile of a direct step (ptn_tune_tiles): 0 the default (up to
                             // 2 x 2 bits), else 1 + 3 ra + rb with ra, rb <= 2 the most tile bits taken
                             // from operand 0 / 1 (ra = rb = 0: the plain direct kernel)
    int32_t cache;           // 1 + cache slot of a trajectory-class step whose output is shared by
                             // the trajectories that agree on every variant column of its subtree
                             // (intermediate caching across error sets, Sec. VI): it runs over the
                             // chunk's representative trajectories only; 0 = not cached
    int32_t virt;            // 1: an outer product (no summed bits) read only by a tensor-core step
                             // that forms it in its operand pack; not launched
    int32_t prod;            // tensor-core steps: 1 + the operand (0 / 1) formed in the pack as the
                             // elementwise product of the factors of step prod_src (a virt step)
    int32_t prod_src;
    int64_t out_size;        // 2^n_out
    int64_t out_off;         // offset of the output buffer in its arena (elements per instance)
    OperandDesc op[2];
    int64_t out_stride[2][kMaxOut];
    int64_t sum_stride[2][kMaxSum];
};

// Small trajectory-class steps run fused, a run of consecutive ones per launch
// (one CTA per trajectory of the chunk walks the run): out <= 2^kSmallOutBits
// elements, summed bits <= kSmallSumBits, operands <= 2^kSmallOpBits.  In
// every arena the instances of one buffer are stored one after another
// (offset x instances + instance x size), so two buffers whose per-instance
// ranges overlap without coinciding share addresses across different
// instances, i.e. across CTAs of a fused launch.  The planner therefore keeps
// the buffers a run reads allocated until the run ends, and sets fuse_prev
// only where a step's output range meets no range touched earlier in its run
// other than itself.
constexpr int kSmallOutBits = 12, kSmallSumBits = 8, kSmallOpBits = 14;
inline bool small_step(const StepDesc& h) {
    return h.kind == STEP_DIRECT && h.out_cls == CLS_TRAJ && h.n_out <= kSmallOutBits && h.n_sum <= kSmallSumBits &&
           h.op[0].inst_size <= (1ll << kSmallOpBits) && h.op[1].inst_size <= (1ll << kSmallOpBits);
}

struct LeafInfo {
    int32_t gate;            // source gate, -1 for a |0> state
    int32_t part;            // 0 whole gate / |0>, 1 factor on q0, 2 factor on q1
    int32_t qubit0, qubit1;
    std::vector<int32_t> sites;   // sites selecting the variant (mixed radix, first fastest)
    std::vector<int32_t> radix;
    int64_t n_var = 1;
    int64_t size = 1;        // elements per variant
    int64_t var_base = 0;    // element offset in the variant table
    int32_t var_col = -1;    // column of var_ids, -1 if n_var == 1
    // legs in storage order (position 0 = stride 1): role codes, see planner.cpp
    std::vector<int32_t> legs;
    // parametrised one-qubit gates (RY / RZ): the noise operator N of every
    // variant (2x2 complex128, row-major) so the merged tensor N G(theta) and
    // its derivative can be rebuilt for any angle
    int32_t param_kind = PTN_PARAM_NONE;
    int32_t param_index = -1;
    std::vector<double> noise_ops;   // n_var * 8 doubles
};

// Ket network of the whole circuit with every qubit open (the trajectory
// state), its forward path with all intermediates kept, and the reversed
// (adjoint) path; used by ptn_expval_grad.
struct ParamLeaf {
    int32_t leaf;            // leaf id
    int32_t param_index;
    int32_t param_kind;
    int32_t var_col;         // variant column (-1: single variant)
    int64_t size;            // elements per variant
    int64_t n_var;
    int64_t lgrad_off;       // offset of its adjoint in the LGRAD arena (elements per trajectory)
    int64_t dvt_base;        // offset of its derivative variants in the derivative table
};

struct RootRef {             // where the block's final tensor lives
    OperandDesc op;          // read with NET addressing (slices applied)
    int64_t x_stride[32];    // stride of block bit t (or, for the whole-circuit state, qubit t) in the root
};
// The kernels copy descriptors into shared memory 16 bytes at a time.
static_assert(sizeof(OperandDesc) % 16 == 0, "OperandDesc must be a multiple of 16 bytes");
static_assert(sizeof(StepDesc) % 16 == 0, "StepDesc must be a multiple of 16 bytes");
static_assert(sizeof(RootRef) % 16 == 0, "RootRef must be a multiple of 16 bytes");

struct BlockPlan {
    int32_t start = 0, b = 0;
    int32_t ket_only = 0;                // sampling block lowered in the ket-only network form
    std::vector<StepDesc> steps;
    RootRef root;
    int64_t arena_peak[N_ARENAS] = {0, 0, 0, 0, 0};   // elements per instance, per arena
    int64_t pack_peak[2][3] = {{0, 0, 0}, {0, 0, 0}};   // GEMM packing floats per instance: [A/B][class]
    double est_macs[3] = {0, 0, 0};      // complex MACs per instance by output class
    double est_bytes[3] = {0, 0, 0};     // bytes moved per instance by output class
    double est_time = 0;                 // modelled seconds at the planning multiplicities
    double est_mult_traj = 0, est_mult_net = 0;
    int32_t n_leaves_used = 0;
    std::string path_summary;
    // intermediate caching (ptn_plan_opts.cache_intermediates): per cached step
    // (slot k = StepDesc.cache - 1) the variant columns its output depends on,
    // a bitmap of cache_words 32-bit words
    int32_t n_cache = 0, cache_words = 0;
    std::vector<uint32_t> cache_bits;
    uint32_t* d_cache_bits = nullptr;
    // device copy
    StepDesc* d_steps = nullptr;
    // expectation/gradient plans only: the reversed path and its targets
    std::vector<StepDesc> bwd;
    int64_t root_adj_off = 0;            // ADJ arena offset of the root adjoint
    std::vector<ParamLeaf> pleaves;
    int64_t dvt_size = 0;                // elements of the derivative variant table
    StepDesc* d_bwd = nullptr;
};

struct SiteTable {           // per site: Kraus CDF and log q (FP64), padded to kMaxKraus
    double cdf[kMaxKraus];
    double logq[kMaxKraus];
    int32_t n_kraus;
    int32_t pad;
};

}  // namespace ptn

struct ptn_plan {
    int32_t n_qubits = 0;
    int32_t n_sites = 0;
    std::vector<ptn::LeafInfo> leaves;
    int32_t n_var_cols = 0;
    std::vector<float> var_table;        // complex64 interleaved (re, im)
    std::vector<ptn::SiteTable> site_tables;
    std::vector<ptn::BlockPlan> blocks;
    ptn::BlockPlan* expval = nullptr;    // built on the first ptn_expval_grad call
    int32_t n_params = 0;                // 1 + largest parametrised gate index
    std::vector<int32_t> leaf_site_ptr;  // CSR over leaves with var_col >= 0 (by column)
    std::vector<int32_t> leaf_site_idx;
    std::vector<int32_t> leaf_site_mul;
    ptn_plan_opts opts{};
    double plan_seconds = 0;
    // device state (uploaded lazily)
    int device = -1;
    float* d_var_table = nullptr;
    ptn::SiteTable* d_site_tables = nullptr;
    int32_t* d_leaf_site_ptr = nullptr;
    int32_t* d_leaf_site_idx = nullptr;
    int32_t* d_leaf_site_mul = nullptr;
    ptn::RootRef* d_roots = nullptr;     // root descriptor of every block
    double mem_cap = 0;
};

namespace ptn {
// planner.cpp
ptn_status build_plan(const ptn_circuit* c, const ptn_noise* nz, const int32_t* block_sizes,
                      int32_t n_blocks, const ptn_plan_opts* o, ptn_plan* plan);
std::string describe_plan(const ptn_plan* plan, int detail);
void classify_step(StepDesc& st, int64_t pack_floats[2][3], bool allow_tc);   // planner.cpp
ptn_status build_expval_plan(ptn_plan* plan);                                   // planner.cpp
// merged tensor of a parametrised leaf at angle theta (and its derivative),
// written as complex64 into out[n_var * size] (out_d likewise)
void param_leaf_tables(const LeafInfo& L, double theta, float* out, float* out_d);
// errors.cpp
ptn_status set_error(ptn_status s, const char* fmt, ...);
}  // namespace ptn
