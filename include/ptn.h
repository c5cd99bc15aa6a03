/*
 * ptn.h — C ABI of the GB300-native tensor-network PTSBE hot path.
 *
 * The method (arxiv 2604.08467) samples shots of a noisy quantum circuit by
 *   1. pre-sampling E Kraus error sets K_i (pre-trajectory sampling, Sec. II-C),
 *   2. merging every sampled error operator into the gate it follows, so every
 *      error set yields a network with the structure of the error-free one and
 *      one contraction path per qubit block serves all of them (unified path
 *      variations, Sec. III-A, Fig. 2c),
 *   3. contracting, block by block, one network per (trajectory, distinct
 *      prefix of already-sampled bits) and drawing all shots that share a
 *      prefix from its conditional marginal, carrying repeated outcomes as
 *      counts (non-degenerate batched sampling, proportional case, Sec. III-B).
 *
 * Conventions used by every call:
 *   - qubit q is bit q of a bitstring; a bitstring (or prefix) of an n-qubit
 *     plan is W = ceil(n / 64) little-endian uint64 words, bit q being bit
 *     q % 64 of word q / 64 (n <= 256; W = 1 for n <= 64, a plain uint64);
 *     arrays of bitstrings hold W consecutive words per entry;
 *   - block j covers qubits [start_j, start_j + b_j), start_0 = 0, ascending;
 *     a block-local outcome x has bit t = qubit start_j + t;
 *   - complex numbers are (re, im) pairs; host inputs are complex128, device
 *     data is complex64 unless a precision mode says otherwise;
 *   - "device" pointers are CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary host memory;
 *   - every call returns a ptn_status and never aborts the process; the text
 *     of the last error of the calling thread is available from
 *     ptn_last_error();
 *   - calls that take a stream enqueue their GPU work on it; the ones that
 *     must read a size back to the host say so and synchronise that stream.
 *
 * Ownership: handles (ptn_plan, ptn_traj, ptn_shots) are created and owned by
 * the library and released only by the matching *_destroy call.  Host input
 * arrays are copied during the call.  Device output arrays named *_out are
 * allocated by the caller.
 */
#ifndef PTN_H
#define PTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PTN_OK = 0,
    PTN_ERR_INVALID_ARG = 1,   /* malformed argument (sizes, indices, null pointers) */
    PTN_ERR_NOT_CPTP = 2,      /* a channel fails sum_k K_k^dagger K_k = I to 1e-10 */
    PTN_ERR_TOO_LARGE = 3,     /* a plan or batch exceeds the memory cap (the failures counted in Sec. IV-D) */
    PTN_ERR_OOM = 4,           /* device or host allocation failed */
    PTN_ERR_CUDA = 5,          /* a CUDA runtime call failed (message has the CUDA error) */
    PTN_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
    PTN_ERR_UNSUPPORTED = 7    /* option or shape not supported by this build */
} ptn_status;

typedef struct ptn_plan ptn_plan;
typedef struct ptn_traj ptn_traj;
typedef struct ptn_shots ptn_shots;
typedef void* ptn_stream;      /* a cudaStream_t; NULL is the legacy default stream */

/* ---------------------------------------------------------------- inputs -- */

enum { PTN_PARAM_NONE = 0, PTN_PARAM_RY = 1, PTN_PARAM_RZ = 2 };

/* One coherent gate d_l (Sec. II-B: the deterministic gates D = {d_l}).
 * 1-qubit: mat[0..7] holds M[out][in] row-major as (re, im) pairs.
 * 2-qubit on (q0, q1): mat[0..31] holds the 4x4 matrix
 *   M[(o0 << 1) | o1][(i0 << 1) | i1], q0 being the high bit.
 * param_kind marks RY(angle) = exp(-i angle Y / 2) / RZ(angle) =
 * exp(-i angle Z / 2) gates whose angle theta[param_index] is differentiated
 * by ptn_expval_grad; mat must hold the gate at its current angle. */
typedef struct {
    int32_t arity;
    int32_t q0, q1;
    int32_t param_kind;
    int32_t param_index;
    int32_t reserved;
    double  mat[32];
} ptn_gate;

typedef struct {
    int32_t n_qubits;          /* 1 .. 256 */
    int32_t n_gates;
    const ptn_gate* gates;     /* host, n_gates entries, in circuit order */
} ptn_circuit;

/* A noise channel given by its Kraus operators (Sec. II-A): one-qubit
 * (n_qubits 0 or 1: n_kraus 2x2 complex128 matrices K[out][in], row-major
 * (re, im), 8 doubles each) or two-qubit (n_qubits 2: 4x4 matrices
 * K[(o_a o_b)][(i_a i_b)], 32 doubles each, a the first qubit of the gate the
 * site follows, as for ptn_gate; e.g. the two-qubit depolarizing channel of
 * the paper's benchmarks, Sec. IV-B). */
typedef struct {
    int32_t n_kraus;           /* 1 .. 16 */
    int32_t n_qubits;          /* 0 or 1: one-qubit channel; 2: two-qubit channel */
    const double* kraus;       /* host, n_kraus * 8 (or * 32) doubles */
} ptn_channel;

/* A noise site: channel `channel` acts on qubit `qubit` right after gate `gate`
 * (the paper couples channels to every coherent gate, Sec. IV-B); a two-qubit
 * channel acts on both qubits of its (two-qubit) gate and takes qubit = -1.
 * Sites are listed in application order: grouped by gate in circuit order;
 * within a gate, the sites act in list order.  Site s is column s of the
 * Kraus-index matrix. */
typedef struct {
    int32_t gate;
    int32_t qubit;             /* one of the gate's qubits; -1 for a two-qubit channel */
    int32_t channel;
} ptn_site;

typedef struct {
    int32_t n_channels;
    const ptn_channel* channels;
    int32_t n_sites;
    const ptn_site* sites;
} ptn_noise;

/* Path-planner options (Sec. III-A: one path set P^j found once for the
 * error-free network; Sec. IV-C: 100 hypersamples by default). */
typedef struct {
    int32_t  hypersamples;     /* randomised greedy restarts; 0 -> 100 */
    int32_t  split_gates;      /* 1: split 2-qubit gates by operator-Schmidt decomposition
                                  (bond padded to a power of two); 0: keep 4-leg tensors */
    uint64_t seed;             /* planner randomness */
    double   est_traj;         /* expected trajectories E for the cost model; 0 -> 1024 */
    double   est_shots;        /* expected shots for the cost model (bounds the number of
                                  distinct prefixes per block); 0 -> 1e6 */
    double   mem_cap_bytes;    /* device memory one execution chunk may use; 0 -> 40% of
                                  the device's free memory at first use */
    int32_t  simt_only;        /* 1: run every step on the SIMT kernel (no tensor cores) */
    int32_t  grad_checkpoint;  /* ptn_expval_grad: 0 keep every forward intermediate; 1 keep only
                                  those crossing segments of ~sqrt(steps) steps and recompute the
                                  rest segment by segment on the reversed path */
    int32_t  network_form;     /* sampling networks (PTN_FORM_*): AUTO (0) per block the cheaper
                                  (modelled) of the double layer and the ket-only form;
                                  DOUBLE_LAYER (1) <psi|P|psi> for every block; KET_ONLY (2) the
                                  amplitudes of the block and later qubits, then the marginal as
                                  the sum over later qubits of |a|^2, wherever it has a path */
    int32_t  fuse_max;         /* longest run of consecutive small trajectory-level steps (the
                                  gate-level start of a path) executed by one launch, one CTA per
                                  trajectory walking the run; 0 -> 1024, 1 -> one launch per step */
    int32_t  cache_intermediates; /* 1: intermediate caching across error sets (Sec. VI): every
                                  trajectory-level step outside the fused runs (at least 4096
                                  multiply-adds and 128 outputs per trajectory) is computed once
                                  per group of a
                                  chunk's trajectories that agree on every variant column of its
                                  subtree, and read through a per-chunk representative table;
                                  results are bit-identical to 0 (no caching) */
    int32_t  keep_products;    /* 0: an outer-product step (no summed bits) read only by a
                                  tensor-core step is not launched; that step's operand pack forms
                                  each element as the product of the two factors (the same
                                  rounding, so the same results); 1: materialise it */
    int32_t  search_threads;   /* 0: the restarts of the path search draw from one random stream,
                                  in order; n >= 1: restart h draws from its own stream (seeded
                                  from seed and h) and the restarts run on n host threads; the plan
                                  then does not depend on n (it differs from the one of 0) */
} ptn_plan_opts;

/* Network forms of the block marginals (Sec. II-B; the ket-only form gives the
 * same marginal, see ptn_plan_opts.network_form). */
enum { PTN_FORM_AUTO = 0, PTN_FORM_DOUBLE_LAYER = 1, PTN_FORM_KET_ONLY = 2 };

/* ------------------------------------------------------------- planning -- */

/* Build the plan: validates the channels (PTN_ERR_NOT_CPTP), builds the UPV
 * variant tables (every merged gate (N_a (x) N_b) d_l for every combination of
 * Kraus choices of its sites, N_q = product of K_k / sqrt(q_k), q_k =
 * Tr(K_k^dagger K_k) / d with d = 2 or 4; a gate with a two-qubit channel merges
 * every site's operator in application order and is not split by the
 * operator-Schmidt option), the double-layer marginal network of every block
 * (prefix qubits projected, block qubits open, later qubits traced), and one
 * contraction path per block (Sec. III-A), lowered to a list of batched
 * pairwise contractions.  Host only: needs no GPU (device tables are uploaded
 * on first use).  block_sizes may be NULL (then b = 10 blocks, the last one
 * taking the remainder); otherwise they must be in 1..14 (the last one in
 * 1..30, for the non-proportional final-block harvest) and sum to n_qubits. */
ptn_status ptn_plan_path(const ptn_circuit* circuit, const ptn_noise* noise,
                         const int32_t* block_sizes, int32_t n_blocks,
                         const ptn_plan_opts* opts, ptn_plan** plan_out);

/* JSON description of the plan: per block the number of steps by storage
 * class, arena sizes and modelled work.  detail = 1 adds every lowered step
 * (operand descriptors, stride tables), the block roots, the variant-selecting
 * sites of every merged-gate leaf and the complex64 variant table, so the
 * lowering can be inspected or replayed on the host.  Each step also carries
 * its cache slot ("cache", and per block "n_cache" and "cache_cols", the
 * variant columns of every slot) and its outer-product marks ("virt": formed
 * in its consumer's pack, "prod" / "prod_src": the operand formed and the
 * step it comes from).  detail = 2 adds the
 * expectation-value plan of ptn_expval_grad (ket network of the whole circuit,
 * its forward steps, the reversed adjoint steps and the parametrised leaves),
 * building it if needed.  Writes at most cap bytes
 * (NUL-terminated) to buf and the full length to *len (host). */
ptn_status ptn_plan_describe(const ptn_plan* plan, int32_t detail, char* buf, size_t cap, size_t* len);

void ptn_plan_destroy(ptn_plan* plan);

/* --------------------------------------------------------- pre-sampling -- */

/* Draw E Kraus error sets on the GPU (pre-trajectory sampling, Sec. II-C).
 * Site s of trajectory i takes the Philox4x32-10 counter
 * (s, 0, i, (1 << 24) | (circuit_id << 8)) with key (seed_lo, seed_hi); u =
 * ((x0 << 32 | x1) >> 11) * 2^-53; the Kraus index is the smallest k with
 * u < C_s[k], C_s the running sum of q_{s,.} (last entry 1.0).  log q_i, the
 * sum over sites in site order of log q_{s,k}, is kept in FP64.
 * dedup != 0 merges identical error sets (first-occurrence order) and keeps
 * their multiplicities; this synchronises the stream once to read the number
 * of distinct sets.  The first-occurrence search compares row hashes against
 * every earlier row (quadratic in n_traj: well under a second up to ~10^5
 * trajectories; use dedup = 0 beyond that).  Also computes, per trajectory, the variant index of every
 * merged tensor (the UPV merge as a table gather).  n_traj in 1 .. 2^24. */
ptn_status ptn_presample_trajectories(const ptn_plan* plan, uint64_t seed, int32_t circuit_id,
                                      int64_t n_traj, int32_t dedup, ptn_traj** traj_out,
                                      ptn_stream stream);

/* Trajectories traj0 .. traj0 + n_traj - 1 of the draw ptn_presample_trajectories
 * makes from the same seed (no dedup): trajectory traj0 + i uses the Philox
 * counter (s, 0, traj0 + i, (1 << 24) | (circuit_id << 8)) and is row i of the
 * result, whose `first` entries are traj0 + i.  Ranks that shard one job by
 * trajectory range draw their ranges with this call (Sec. III: the method
 * parallelises over error sets); their sampling calls then pass the global
 * trajectory index (traj0 + row) as parent_traj so that every Philox counter
 * is the one of the single-process run.  traj0 + n_traj <= 2^32. */
ptn_status ptn_presample_range(const ptn_plan* plan, uint64_t seed, int32_t circuit_id, int64_t traj0, int64_t n_traj,
                               ptn_traj** traj_out, ptn_stream stream);

/* Device views of a ptn_traj (valid until ptn_traj_destroy): kraus [n][S]
 * uint8 row-major, logq [n] double, mult [n] int64 (1 without dedup), first
 * [n] int64 (index of the error set in the original draw order). */
ptn_status ptn_traj_info(const ptn_traj* traj, int64_t* n_unique, int32_t* n_sites,
                         const uint8_t** kraus, const double** logq,
                         const int64_t** mult, const int64_t** first);

/* Copy the trajectory set into caller-allocated device arrays of n_unique
 * (x n_sites for kraus) entries; any pointer may be NULL. */
ptn_status ptn_traj_copy(const ptn_traj* traj, uint8_t* kraus_out, double* logq_out, int64_t* mult_out,
                         int64_t* first_out, ptn_stream stream);

void ptn_traj_destroy(ptn_traj* traj);

/* ---------------------------------------------------------- contraction -- */

/* Precision of the tensor-core contraction steps (the SIMT steps are FP32):
 * FP32: TF32 hi/lo operands, three MMAs per product, FP32-accurate;
 * BF16X3 / FP16X3: BF16 or FP16 hi/lo operands (FP16 scaled by a power of two
 * per row and K segment), three MMAs per product.  In every mode K is
 * accumulated in segments added in FP32, and a contraction over at most 16
 * complex terms runs with TF32 hi/lo operands (one 128-byte K-block without
 * padding). */
enum { PTN_PREC_FP32 = 0, PTN_PREC_BF16X3 = 1, PTN_PREC_FP16X3 = 2 };

/* Contract n_net block-`block` networks with the block's shared path
 * (Sec. III-A) and write their unnormalised marginals (Sec. II-B):
 *   marg_out[n][x] = <psi_i| P_s (x) |x><x| (x) I |psi_i>,  i = net_traj[n],
 *   s = the bits of prefix n below start_block (higher bits ignored); net_prefix
 *   holds W words per network (the plan's bitstring width, see the conventions),
 *   Z_out[n] = sum_x marg_out[n][x] accumulated in FP64.
 * net_traj (device int32, indices into the ptn_traj's distinct error sets) must
 * be non-decreasing.  marg_out: device float [n_net][2^b_block]; Z_out: device
 * double [n_net].  Copies net_traj to the host (one synchronisation) to split
 * the batch into chunks that fit the memory cap. */
ptn_status ptn_contract_batch(const ptn_plan* plan, const ptn_traj* traj, int32_t block,
                              const int32_t* net_traj, const uint64_t* net_prefix, int64_t n_net,
                              int32_t precision, float* marg_out, double* Z_out,
                              ptn_stream stream);

/* ------------------------------------------------------------- sampling -- */

/* One block of proportional NBS (Sec. III-B) for n_parent networks whose
 * marginals are given: parent n (trajectory parent_traj[n], prefix bits
 * parent_prefix[n], count parent_count[n] >= 0) draws its count shots from row
 * n of marg (device float [n_parent][2^b]) with the exact-integer FP64 CDF:
 * P_x = rint(max(p_x, 0) * 2^sigma), sigma = 52 - b - e, max p = f 2^e with f
 * in [0.5, 1); shot rank r (the ranks of a parent continue the ranks of the
 * trajectory's earlier parents) uses the Philox4x32-10 counter
 * (r_lo, r_hi, traj, (3 << 24) | (circuit_id << 8) | block), a = x0 << 32 | x1,
 * and picks the smallest x with floor(a T / 2^64) < C[x].  The distinct
 * outcomes are written, in canonical order (parents in order, x ascending), as
 * children (traj, prefix | x << start, count) to the device arrays child_*
 * (capacity child_cap >= sum_n min(count_n, 2^b); a smaller capacity returns
 * PTN_ERR_INVALID_ARG and writes no child).  Parents must be grouped by
 * trajectory.  Prefixes here are single uint64 words (start + b <= 64); plans
 * of more than 64 qubits sample through ptn_sample_shots.  Writes the number
 * of children to *n_child (host); synchronises the stream. */
ptn_status ptn_sample_block(const float* marg, int32_t b, int32_t start,
                            const int32_t* parent_traj, const uint64_t* parent_prefix,
                            const int64_t* parent_count, int64_t n_parent,
                            uint64_t seed, int32_t circuit_id, int32_t block,
                            int32_t* child_traj, uint64_t* child_prefix, int64_t* child_count,
                            int64_t child_cap, int64_t* n_child, ptn_stream stream);

/* ptn_sample_block without any run-time allocation (the paper has no
 * counterpart; this is a deployment variant).  Same arguments, results and
 * bit-exact output as ptn_sample_block, but its scratch memory is a fixed
 * 32 MiB array in the library's static device data instead of buffers the
 * library allocates, for callers that cannot call cudaMalloc while they run
 * (processes that reserve their whole GPU memory budget at start-up and
 * forbid later allocations, which would also synchronise the device, or code
 * that must stay inside a caching allocator).  Every GPU that loads the
 * library holds the array until the process exits.
 *  - Limits: the scratch holds 48 bytes per parent, 8 per trajectory index
 *    (up to the largest index used), 12 per child slot (child_cap) plus scan
 *    space; a call that needs more than 32 MiB returns PTN_ERR_TOO_LARGE with
 *    the sizes in the error text, before launching any sampling work.
 *  - The array used is the current device's; the stream must belong to that
 *    device (PTN_ERR_INVALID_ARG otherwise).
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - All calls share the array, whatever their stream: calls that overlap on
 *    the GPU race and corrupt each other's results; serialise them.  Each call
 *    clears what must start at zero, so stale contents of an earlier call do
 *    not leak into the next.
 *  - Synchronises the stream (it validates the parents and reads sizes back). */
ptn_status ptn_sample_block_noalloc(const float* marg, int32_t b, int32_t start,
                                    const int32_t* parent_traj, const uint64_t* parent_prefix,
                                    const int64_t* parent_count, int64_t n_parent,
                                    uint64_t seed, int32_t circuit_id, int32_t block,
                                    int32_t* child_traj, uint64_t* child_prefix, int64_t* child_count,
                                    int64_t child_cap, int64_t* n_child, ptn_stream stream);

/* Proportional shot allocation (Sec. II-C "shots m_i assigned by the rule"):
 * one multinomial draw of `total` shots over the device weights w[n] (FP64,
 * >= 0, not all zero), quantised like the marginals (b = ceil(log2 n)); shot t
 * uses the counter (t_lo, t_hi, 0, (2 << 24) | (circuit_id << 8)).  Writes
 * m_out (device int64 [n]). */
ptn_status ptn_allocate_shots(const double* weights, int64_t n, int64_t total, uint64_t seed,
                              int32_t circuit_id, int64_t* m_out, ptn_stream stream);

/* Sampling modes (Sec. III-B).  The proportional modes keep the circuit's
 * statistics; the non-proportional ones gather as much data as possible:
 * every non-final block draws branch_shots shots per distinct prefix (the
 * distinct outcomes become the next block's prefixes), and the final block,
 * whose outcomes feed no later contraction, is harvested from its population
 * vector, by direct sampling (final_shots draws per network) or exhaustively
 * (every outcome x with p(x | prefix) >= threshold, with that probability).
 * The final block of a plan may have up to 30 qubits for the non-proportional
 * modes; the proportional modes need every block <= 14. */
enum { PTN_PROPORTIONAL_FIXED = 0, PTN_PROPORTIONAL_TOTAL = 1, PTN_NONPROP_DIRECT = 2, PTN_NONPROP_EXHAUSTIVE = 3 };

typedef struct {
    int32_t  mode;               /* PTN_PROPORTIONAL_FIXED or PTN_PROPORTIONAL_TOTAL */
    int32_t  circuit_id;         /* goes into every Philox counter */
    int64_t  shots_per_traj;     /* FIXED: m_i = shots_per_traj * multiplicity_i */
    int64_t  total_shots;        /* TOTAL: M allocated over a_i = mult_i * w_i, w_i = Z of block 1 */
    uint64_t seed;               /* Philox key for allocation and sampling */
    int32_t  precision;          /* PTN_PREC_* */
    int32_t  max_traj_per_chunk; /* 0: as many as the memory cap allows; 1: the plain
                                    per-trajectory path (one trajectory per launch) */
    int32_t  use_graphs;         /* 1: every chunk's contraction (all steps of the block and the
                                    marginal finalisation) is recorded on a private stream and
                                    launched as one CUDA graph on the caller's stream; the
                                    block's executable graph stays in the plan's workspace and is
                                    updated in place for the next chunk or call, re-instantiated
                                    when the launch sequence changes shape.  Results equal those
                                    of 0; per-launch timing statistics are not taken inside
                                    graphs (launch counts are). */
    int32_t  reserved;
    int64_t  branch_shots;       /* NONPROP_*: shots drawn per prefix on every non-final block (>= 1) */
    int64_t  final_shots;        /* NONPROP_DIRECT: shots drawn from every final-block network (>= 1) */
    double   threshold;          /* NONPROP_EXHAUSTIVE: keep outcomes with p(x | prefix) >= threshold,
                                    in [0, 1] */
} ptn_sample_opts;

/* Full proportional NBS over all blocks (Sec. III-B): block 1 contracts one
 * network per distinct error set; every later block contracts one network per
 * distinct (trajectory, prefix) and draws all its shots from it.  The final
 * (trajectory, bitstring, count) list is in canonical order (trajectories in
 * order, then bitstrings lexicographic by block outcome, block 1 most
 * significant).  Synchronises the stream once per block to size the next
 * level. */
ptn_status ptn_sample_shots(const ptn_plan* plan, const ptn_traj* traj, const ptn_sample_opts* opts,
                            ptn_shots** shots_out, ptn_stream stream);

/* Non-proportional modes, final block: the population vector of a network
 * (trajectory i, prefix s) with b_f bits is quantised to 64-bit integers
 * P_x = rint(max(p_x, 0) 2^(62 - b_f - e)), max p = f 2^e with f in [0.5, 1),
 * T = sum P_x (exact).  Exhaustive: the records are the x with P_x > 0 and
 * (double)P_x >= threshold * (double)T, count 1.  Direct: shot rank r of the
 * trajectory (ranks continue over its final networks in order, final_shots
 * each) uses the Philox counter of ptn_sample_block and takes the smallest x
 * with floor(a T / 2^64) < sum_{y <= x} P_y; the records are the distinct x
 * with their counts.  Both give every record its probability
 * p(x | s) = (double)P_x / (double)T (ptn_shots_probs).  Records are in
 * canonical order (networks in order, x increasing); the final networks are
 * contracted and harvested in sub-batches that fit half the memory cap. */

/* Device views of the result (valid until ptn_shots_destroy) and, per block,
 * the number of networks contracted (host array of n_blocks, may be NULL).
 * bits holds W words per record (the plan's bitstring width). */
ptn_status ptn_shots_info(const ptn_shots* shots, int64_t* n_out, const int32_t** traj,
                          const uint64_t** bits, const int64_t** count,
                          int64_t* nets_per_block, int32_t cap_blocks);

/* Copy the result into caller-allocated device arrays of n_out entries
 * (bits_out: n_out x W words). */
ptn_status ptn_shots_copy(const ptn_shots* shots, int32_t* traj_out, uint64_t* bits_out, int64_t* count_out,
                          ptn_stream stream);

/* Per-record probabilities p(x | prefix) of a non-proportional result: device
 * view (NULL for proportional results) and a copy into a caller-allocated
 * device double array of n_out entries (PTN_ERR_INVALID_ARG without them). */
ptn_status ptn_shots_probs(const ptn_shots* shots, const double** prob);
ptn_status ptn_shots_copy_probs(const ptn_shots* shots, double* prob_out, ptn_stream stream);

void ptn_shots_destroy(ptn_shots* shots);

/* The emitted shots merged across trajectories: one record per distinct
 * bitstring with the summed count, in increasing bitstring order (traj = -1
 * in every record), built on the device by a stable radix sort of the
 * (bitstring, count) records followed by a reduction by key.  *merged_out is
 * a new handle (ptn_shots_destroy); nets_per_block is copied.  Synchronises
 * the stream once (to size the result). */
ptn_status ptn_shots_merge(const ptn_shots* shots, ptn_shots** merged_out, ptn_stream stream);

/* ------------------------------------------------ mixed-circuit batches -- */

/* One circuit of a heterogeneous batch: its plan, its pre-sampled error sets
 * and its sampling options (qubit counts, trajectory counts and shot budgets
 * may all differ between items). */
typedef struct {
    const ptn_plan*  plan;
    const ptn_traj*  traj;
    ptn_sample_opts  opts;
} ptn_batch_item;

typedef struct {
    int32_t n_workers;          /* circuits in flight at once (each on its own CUDA stream); 0: 4 */
    int32_t keep_workspaces;    /* 0: free each plan's device workspace when its items are done */
    double  mem_budget_bytes;   /* device memory shared by the workers; 0: 70% of free memory */
    double  max_est_seconds;    /* items whose plan's modelled time exceeds this are not run and
                                   get PTN_ERR_TOO_LARGE; 0: no limit */
} ptn_batch_opts;

/* Runs ptn_sample_shots for every item of a mixed-circuit batch (the
 * batching form of the method: many independent circuits, each with one
 * contraction path reused by all of its error sets).  Items are grouped by
 * plan (items sharing a plan run one after another), groups are taken in
 * decreasing modelled cost (longest first) by n_workers host threads, each
 * driving its own non-blocking stream that starts after the work already on
 * `stream`; `stream` waits for all of them before the call returns (the call
 * itself returns once every item has been issued and its level sizes read).
 * Each plan without an explicit memory cap gets mem_budget / n_workers for
 * the batch; an item that fails with PTN_ERR_OOM or PTN_ERR_CUDA while others
 * share the device runs once more alone with the whole budget.  A failing
 * item (e.g. PTN_ERR_TOO_LARGE: a circuit beyond the
 * memory cap, the failures the paper counts in Sec. IV-D) does not stop the
 * others: status_out[i] (host, n_items) holds each item's status and
 * shots_out[i] (host, n_items) its result or NULL.  Returns PTN_OK unless
 * the arguments are malformed.  Plans must have been made on the current
 * device; a plan must not be used by another call while the batch runs. */
ptn_status ptn_sample_shots_batch(const ptn_batch_item* items, int32_t n_items, const ptn_batch_opts* opts,
                                  ptn_shots** shots_out, ptn_status* status_out, ptn_stream stream);

/* ---------------------------------------------------------- gradients -- */

/* A real combination of Pauli strings, O = sum_t coeff[t] P_t, with
 * P_t = prod_q X_q^{x_mask bit q} Z_q^{z_mask bit q}.  This build evaluates
 * diagonal strings (x_mask = 0: products of Z) and rejects others with
 * PTN_ERR_UNSUPPORTED.  Host arrays of n_terms entries. */
typedef struct {
    int32_t n_terms;
    const double* coeff;
    const uint64_t* x_mask;
    const uint64_t* z_mask;
} ptn_pauli_sum;

/* Trajectory-averaged expectation value and its gradient with respect to the
 * angles of the parametrised gates (RY / RZ, ptn_gate.param_kind/param_index):
 *   F(theta) = sum_i c_i <psi_i(theta)| O |psi_i(theta)> / sum_i c_i,
 * psi_i the (unnormalised) state of error set i with every sampled Kraus
 * operator merged into its gate (the UPV merge, Sec. III-A), c_i its
 * multiplicity.  The state is the ket network with every qubit open,
 * contracted along one path found once for all error sets; the gradient is
 * reverse-mode differentiation of that contraction (adjoint contractions
 * along the reversed path, intermediates of the forward pass kept), then
 * dF/dtheta = 2 Re sum (adjoint of each merged gate) . d(merged gate)/dtheta.
 * theta: host double [n_theta] (n_theta >= the plan's largest parameter
 * index + 1); the plan's parametrised gates take these angles from now on.
 * value_out: device double [1]; grad_out: device double [n_theta].
 * Needs n_qubits <= 24.  Synchronises the stream. */
ptn_status ptn_expval_grad(const ptn_plan* plan, const ptn_traj* traj, const ptn_pauli_sum* obs,
                           const double* theta, int32_t n_theta, double* value_out, double* grad_out,
                           ptn_stream stream);

/* Amplitudes of the trajectory states psi_i (the ket network of the whole
 * circuit with every sampled Kraus operator merged into its gate, Sec. III-A,
 * contracted along the path ptn_expval_grad uses): for the distinct error sets
 * i = traj0 .. traj0 + n_traj - 1 of `traj`,
 *   amp_out[(i - traj0) * 2^n + x] = <x|psi_i>,  bit q of x = qubit q,
 * unnormalised (|psi_i|^2 = w_i, the trajectory weight).  amp_out: device
 * complex64 (re, im float pairs), n_traj * 2^n entries.  precision selects the
 * tensor-core operand split (PTN_PREC_*), as for the sampling contractions.
 * Needs n_qubits <= 24.  Synchronises the stream. */
ptn_status ptn_trajectory_amplitudes(const ptn_plan* plan, const ptn_traj* traj, int64_t traj0, int64_t n_traj,
                                     int32_t precision, float* amp_out, ptn_stream stream);

/* ----------------------------------------------------------- statistics -- */

/* Per-kernel launch statistics (instrumentation for roofline reporting).
 * Launch counts are always kept.  While timing is enabled every launch of the
 * library's kernels is bracketed by CUDA events on its stream and charged its
 * algorithmic bytes (distinct operand elements read + output written) and
 * flops (8 per complex multiply-add).  ptn_stats_read synchronises the device,
 * resolves the events and fills up to cap records; ptn_stats_reset clears. */
typedef struct {
    char    name[32];
    int64_t launches;
    int64_t timed_launches;
    double  ms;             /* summed event time of the timed launches */
    double  alg_bytes;      /* summed algorithmic bytes of the timed launches */
    double  alg_flops;
} ptn_kernel_stat;

ptn_status ptn_stats_enable(int32_t timing_on);
/* Timing of one kernel class only (a name as reported by ptn_stats_read, e.g.
 * "contract_gemm"): the other launches are only counted, so the timed class
 * can be measured inside an otherwise uninstrumented run.  NULL or "" times
 * every class; an unknown name returns PTN_ERR_INVALID_ARG.
 * ptn_stats_enable(0) turns timing off. */
ptn_status ptn_stats_enable_only(const char* kernel);
ptn_status ptn_stats_reset(void);
ptn_status ptn_stats_read(ptn_kernel_stat* out, int32_t cap, int32_t* n_out);

/* The same timings per path step: block (-1 for launches outside a block's
 * step list, -2 / -3 for the forward / adjoint steps of ptn_expval_grad), step
 * index within the block's lowered list, kernel.  Timing must have been
 * enabled.  Fills up to cap records (host array) ordered by block, step. */
typedef struct {
    int32_t block;
    int32_t step;
    char    kernel[32];
    int64_t launches;
    double  ms;
    double  alg_bytes;
    double  alg_flops;
} ptn_step_stat;

ptn_status ptn_stats_read_steps(ptn_step_stat* out, int32_t cap, int32_t* n_out);

/* ----------------------------------------------------- block-size tuning -- */

/* Block-size autotuning (Sec. V-B, Fig. 7: the contraction cost per block
 * changes by orders of magnitude with the block size, so b is a tuning
 * parameter of each circuit).  For every candidate b (1..14) the circuit is
 * planned with blocks of b qubits, the last taking the remainder, and a probe
 * run is timed on the stream with CUDA events: pre-sampling probe_traj error
 * sets (seed) and proportional NBS of probe_shots shots (FP32 mode), once to
 * warm up and once timed.  seconds_out[i] (host, n_cand) receives the timed
 * seconds of candidate i (+infinity if it could not be planned or run);
 * *best_b the fastest candidate.  opts as for ptn_plan_path.  Synchronises
 * the stream; returns the last failure if no candidate ran. */
ptn_status ptn_tune_block_sizes(const ptn_circuit* circuit, const ptn_noise* noise, const int32_t* candidates,
                                int32_t n_cand, const ptn_plan_opts* opts, int64_t probe_traj, int64_t probe_shots,
                                uint64_t seed, int32_t* best_b, double* seconds_out, ptn_stream stream);

/* Tile-shape autotuning of the SIMT contraction steps (the steps that do not
 * go to the tensor cores and do not run in a fused gate-level run): each such
 * step computes a micro-tile of up to 2^ra x 2^rb outputs per thread, spanned
 * by output bits along which only one operand varies (ra, rb <= 2, ra = rb = 0
 * the plain direct kernel).  Every block is contracted once on a probe of
 * min(n_probe, unique trajectories, what one chunk holds) networks (one per
 * trajectory, prefix 0) to fill its intermediates; then each step is launched
 * under every feasible (ra, rb), timed over `reps` launches with CUDA events
 * on the stream after one warm-up, and the fastest shape is stored in the
 * plan for later calls if it beats the default shape (the most tile bits) by
 * more than 5%.  The probe should be as large as the chunks of the intended
 * runs: a shape that wins on few instances can lose on many.
 * Timing does not depend on the data, and a step's output never aliases its
 * operands, so the repeated launches leave the intermediates intact.  The
 * arithmetic of each output (its multiply-add chain over the summed bits) is
 * the same for every shape.  *n_tuned_out (may be NULL): steps timed;
 * *n_changed_out (may be NULL): steps whose fastest shape differs from the
 * default.  Synchronises the stream.  n_probe >= 1, reps in 1..100. */
ptn_status ptn_tune_tiles(ptn_plan* plan, const ptn_traj* traj, int64_t n_probe, int32_t reps, int32_t* n_tuned_out,
                          int32_t* n_changed_out, ptn_stream stream);

/* ---------------------------------------------------------- bounded waits -- */

/* Wall-time limit of every pipeline wait inside the tensor-core contraction
 * kernel (mbarrier waits between its TMA, MMA and epilogue roles), 2 s by
 * default, for launches issued after the call (process-wide).  A wait that
 * runs out makes its CTA stop issuing work, let its own copies and MMAs in
 * flight finish, free its tensor memory and exit; the call then returns
 * PTN_ERR_TIMEOUT and the device stays usable.  seconds in [0, 60]. */
ptn_status ptn_set_wait_limit(double seconds);

/* ------------------------------------------------------------- utilities -- */

const char* ptn_status_string(ptn_status status);
const char* ptn_last_error(void);
const char* ptn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PTN_H */
