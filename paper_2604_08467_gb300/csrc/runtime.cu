// C-ABI entry points and the device runtime of the PTSBE hot path.
//
// Execution of a block (Sec. III-A/B): the networks of a level (one per
// distinct (trajectory, prefix), grouped by trajectory) are split into chunks
// that fit the memory cap; for every chunk the block's step list runs once,
// each step a single launch over all instances of its storage class (every
// distinct trajectory of the chunk for trajectory-only tensors, every network
// for prefix-dependent ones), then the root tensor is finalised into the
// networks' marginals.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "stats.h"

namespace ptn {
const char* last_error_text();
void clear_error();
}  // namespace ptn

using namespace ptn;

#define PTN_CUDA(call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return set_error(e_ == cudaErrorMemoryAllocation ? PTN_ERR_OOM : PTN_ERR_CUDA, "%s: %s (%s:%d)", \
                             #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

static_assert(sizeof(StepDesc) % 16 == 0, "StepDesc must be a multiple of 16 bytes");
static_assert(sizeof(RootRef) % 16 == 0, "RootRef must be a multiple of 16 bytes");

namespace {

// Stream on which workspace buffers are (re)allocated and freed by the calling
// thread: set by the batch executor's workers so that their allocations are
// stream-ordered (cudaMallocAsync / cudaFreeAsync) and never synchronise the
// device under other workers' work.  Unset: plain cudaMalloc / cudaFree.
thread_local bool t_async_alloc = false;
thread_local cudaStream_t t_alloc_stream = nullptr;
struct AsyncAllocScope {
    bool prev_on;
    cudaStream_t prev_s;
    explicit AsyncAllocScope(cudaStream_t s) : prev_on(t_async_alloc), prev_s(t_alloc_stream) {
        t_async_alloc = true;
        t_alloc_stream = s;
    }
    ~AsyncAllocScope() {
        t_async_alloc = prev_on;
        t_alloc_stream = prev_s;
    }
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    bool async = false;      // allocated by cudaMallocAsync
    ptn_status grow(size_t bytes) {
        if (bytes <= cap) return PTN_OK;
        release();
        size_t want = std::max(bytes, (size_t)256);
        async = t_async_alloc;
        cudaError_t e = async ? cudaMallocAsync(&p, want, t_alloc_stream) : cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            p = nullptr;
            return set_error(PTN_ERR_OOM, "device allocation of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        cap = want;
        return PTN_OK;
    }
    // stream-ordered free only for stream-ordered memory inside an async scope;
    // otherwise cudaFree (valid for both kinds, synchronising)
    void release() {
        if (p) {
            if (async && t_async_alloc)
                cudaFreeAsync(p, t_alloc_stream);
            else
                cudaFree(p);
        }
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

struct HostBuf {
    void* p = nullptr;
    size_t cap = 0;
    ptn_status grow(size_t bytes) {
        if (bytes <= cap) return PTN_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMallocHost(&p, std::max(bytes, (size_t)256));
        if (e != cudaSuccess) {
            p = nullptr;
            return set_error(PTN_ERR_OOM, "cudaMallocHost(%zu): %s", bytes, cudaGetErrorString(e));
        }
        cap = std::max(bytes, (size_t)256);
        return PTN_OK;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

}  // namespace

// Per-plan device workspace (calls that use the same plan must not overlap).
struct PlanWorkspace {
    DevBuf arena[3];
    DevBuf chunk_traj, net_tl;
    DevBuf marg, Z, w, cdf, m;
    DevBuf lvl_traj[2], lvl_prefix[2], lvl_count[2];
    DevBuf s_cap, s_tmp_off, s_rank0, s_excl, s_first, s_ndist, s_out_off, s_tmp_x, s_tmp_c, s_scan;
    DevBuf zero_prefix;
    DevBuf pack[2], err, grp, grp_cnt, grp_tile0, grp_scan;
    // expectation / gradient plans
    DevBuf arena_x[2];                    // ADJ, LGRAD arenas
    DevBuf ev_steps, ev_bwd, ev_root, ev_pl, ev_dvt, ev_terms, ev_F, ev_partial, ev_iota;
    DevBuf zpart;                         // per-tile partial totals of large marginal rows
    // final-block harvest of non-proportional sampling
    DevBuf h_rowmax, h_T, h_tcdf, h_tcnt, h_toff, h_scan, h_cnt, h_rank0, h_first;
    // intermediate caching: key halves, hash tables, representatives, lists, counts
    DevBuf c_h, c_keys, c_first, c_rep, c_list, c_cnt;
    HostBuf h_traj, h_chunk_traj, h_net_tl, h_small, h_grp, h_ccnt;
    // CUDA-graph execution of a block's chunk (ptn_sample_opts.use_graphs): the
    // capture stream and one executable graph per block, updated in place
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaGraphExec_t> gexec;
    void release_graphs() {
        for (auto& x : gexec)
            if (x) cudaGraphExecDestroy(x);
        gexec.clear();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cap_stream = nullptr;
    }
    void release() {
        release_graphs();
        DevBuf* all[] = {&arena[0], &arena[1], &arena[2], &chunk_traj, &net_tl, &marg, &Z, &w, &cdf, &m,
                         &lvl_traj[0], &lvl_traj[1], &lvl_prefix[0], &lvl_prefix[1], &lvl_count[0], &lvl_count[1],
                         &s_cap, &s_tmp_off, &s_rank0, &s_excl, &s_first, &s_ndist, &s_out_off, &s_tmp_x,
                         &s_tmp_c, &s_scan, &zero_prefix, &pack[0], &pack[1], &err, &grp, &grp_cnt,
                         &grp_tile0, &grp_scan, &arena_x[0], &arena_x[1], &ev_steps,
                         &ev_bwd, &ev_root, &ev_pl, &ev_dvt, &ev_terms, &ev_F, &ev_partial, &ev_iota, &zpart,
                         &h_rowmax, &h_T, &h_tcdf, &h_tcnt, &h_toff, &h_scan, &h_cnt, &h_rank0, &h_first,
                         &c_h, &c_keys, &c_first, &c_rep, &c_list, &c_cnt};
        for (DevBuf* b : all) b->release();
        h_grp.release();
        h_ccnt.release();
        h_traj.release();
        h_chunk_traj.release();
        h_net_tl.release();
        h_small.release();
    }
};

struct ptn_traj {
    int64_t n_orig = 0, n_unique = 0;
    int32_t n_sites = 0;
    int32_t n_var_cols = 0;
    uint8_t* kraus = nullptr;
    double* logq = nullptr;
    int64_t* mult = nullptr;
    int64_t* first = nullptr;
    int32_t* var_ids = nullptr;
    // non-zero variant entries per trajectory (intermediate caching), built on
    // first use: row pointers (n_unique + 1), columns, variants
    int64_t* nz_ptr = nullptr;
    int32_t* nz_col = nullptr;
    int32_t* nz_val = nullptr;
    const ptn_plan* plan = nullptr;
};

struct ptn_shots {
    int64_t n = 0;
    int32_t n_qubits = 64;
    int32_t n_words = 1;                 // 64-bit words per bitstring (ceil(n_qubits / 64))
    int32_t* traj = nullptr;
    uint64_t* bits = nullptr;            // [n][n_words]
    int64_t* count = nullptr;
    double* prob = nullptr;              // non-proportional final-block harvest: p(x | prefix) per record
    std::vector<int64_t> nets_per_block;
};

namespace {

PlanWorkspace* workspace(const ptn_plan* plan);

ptn_status ensure_device(const ptn_plan* cplan) {
    ptn_plan* plan = const_cast<ptn_plan*>(cplan);
    int dev = -1;
    PTN_CUDA(cudaGetDevice(&dev));
    if (plan->device == dev) return PTN_OK;
    if (plan->device >= 0) return set_error(PTN_ERR_INVALID_ARG, "plan was uploaded to device %d, current is %d", plan->device, dev);
    size_t vt_bytes = plan->var_table.size() * sizeof(float);
    PTN_CUDA(cudaMalloc(&plan->d_var_table, std::max(vt_bytes, (size_t)16)));
    PTN_CUDA(cudaMemcpy(plan->d_var_table, plan->var_table.data(), vt_bytes, cudaMemcpyHostToDevice));
    size_t st_bytes = plan->site_tables.size() * sizeof(SiteTable);
    PTN_CUDA(cudaMalloc(&plan->d_site_tables, std::max(st_bytes, (size_t)16)));
    if (st_bytes) PTN_CUDA(cudaMemcpy(plan->d_site_tables, plan->site_tables.data(), st_bytes, cudaMemcpyHostToDevice));
    auto up32 = [&](const std::vector<int32_t>& v, int32_t** d) -> ptn_status {
        size_t by = std::max(v.size() * sizeof(int32_t), (size_t)16);
        PTN_CUDA(cudaMalloc(d, by));
        if (!v.empty()) PTN_CUDA(cudaMemcpy(*d, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        return PTN_OK;
    };
    ptn_status e;
    if ((e = up32(plan->leaf_site_ptr, &plan->d_leaf_site_ptr))) return e;
    if ((e = up32(plan->leaf_site_idx, &plan->d_leaf_site_idx))) return e;
    if ((e = up32(plan->leaf_site_mul, &plan->d_leaf_site_mul))) return e;
    for (auto& bp : plan->blocks) {
        size_t by = bp.steps.size() * sizeof(StepDesc);
        PTN_CUDA(cudaMalloc(&bp.d_steps, std::max(by, (size_t)16)));
        if (by) PTN_CUDA(cudaMemcpy(bp.d_steps, bp.steps.data(), by, cudaMemcpyHostToDevice));
        if (!bp.cache_bits.empty()) {
            const size_t cb = bp.cache_bits.size() * sizeof(uint32_t);
            PTN_CUDA(cudaMalloc(&bp.d_cache_bits, cb));
            PTN_CUDA(cudaMemcpy(bp.d_cache_bits, bp.cache_bits.data(), cb, cudaMemcpyHostToDevice));
        }
    }
    std::vector<RootRef> roots;
    for (auto& bp : plan->blocks) roots.push_back(bp.root);
    PTN_CUDA(cudaMalloc(&plan->d_roots, sizeof(RootRef) * std::max<size_t>(roots.size(), 1)));
    PTN_CUDA(cudaMemcpy(plan->d_roots, roots.data(), sizeof(RootRef) * roots.size(), cudaMemcpyHostToDevice));
    if (plan->mem_cap <= 0) {
        size_t fr = 0, tot = 0;
        PTN_CUDA(cudaMemGetInfo(&fr, &tot));
        plan->mem_cap = 0.4 * (double)fr;
    }
    plan->device = dev;
    return PTN_OK;
}

// workspace storage keyed by plan (kept outside the public struct)
struct WsEntry {
    const ptn_plan* plan;
    PlanWorkspace* ws;
};
std::vector<WsEntry>& ws_table() {
    static std::vector<WsEntry> t;
    return t;
}
std::mutex& ws_mutex() {
    static std::mutex m;
    return m;
}
PlanWorkspace* workspace(const ptn_plan* plan) {
    std::lock_guard<std::mutex> lk(ws_mutex());
    for (auto& e : ws_table())
        if (e.plan == plan) return e.ws;
    PlanWorkspace* w = new PlanWorkspace();
    ws_table().push_back({plan, w});
    return w;
}
void drop_workspace(const ptn_plan* plan) {
    PlanWorkspace* w = nullptr;
    {
        std::lock_guard<std::mutex> lk(ws_mutex());
        auto& t = ws_table();
        for (size_t i = 0; i < t.size(); i++)
            if (t[i].plan == plan) {
                w = t[i].ws;
                t.erase(t.begin() + i);
                break;
            }
    }
    if (w) {
        w->release();
        delete w;
    }
}

struct Chunk {
    int64_t net0, n_net;     // networks [net0, net0 + n_net)
    int64_t traj0, n_traj;   // entries [traj0, traj0 + n_traj) of the chunk_traj list
};

// The non-zero variant entries of every trajectory (CSR over var_ids), made
// once per trajectory set on first use by a cached step.
ptn_status ensure_nz(const ptn_traj* ctr, cudaStream_t s) {
    ptn_traj* tr = const_cast<ptn_traj*>(ctr);
    if (tr->nz_ptr) return PTN_OK;
    const int64_t n = tr->n_unique;
    int64_t* ptr = nullptr;
    int64_t* tmp = nullptr;
    int32_t *col = nullptr, *val = nullptr;
    auto fail = [&](cudaError_t e) {
        cudaFree(ptr);
        cudaFree(tmp);
        cudaFree(col);
        cudaFree(val);
        return set_error(PTN_ERR_CUDA, "variant entry lists: %s", cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ptr, sizeof(int64_t) * (n + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&tmp, sizeof(int64_t) * scan_tmp_elems(n + 1))) != cudaSuccess) return fail(e);
    launch_nz_count(tr->var_ids, n, tr->n_var_cols, ptr, s);
    launch_exclusive_scan(ptr, ptr, n + 1, tmp, s);
    int64_t total = 0;
    if ((e = cudaMemcpyAsync(&total, ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMalloc(&col, sizeof(int32_t) * std::max<int64_t>(total, 1))) != cudaSuccess ||
        (e = cudaMalloc(&val, sizeof(int32_t) * std::max<int64_t>(total, 1))) != cudaSuccess)
        return fail(e);
    launch_nz_fill(tr->var_ids, n, tr->n_var_cols, ptr, col, val, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    cudaFree(tmp);
    tr->nz_ptr = ptr;
    tr->nz_col = col;
    tr->nz_val = val;
    return PTN_OK;
}

// Contract n_net networks of block j; marg/Z outputs are device arrays.
ptn_status contract_level(const ptn_plan* plan, const ptn_traj* tr, int j, const int32_t* d_net_traj,
                          const uint64_t* d_net_prefix, int64_t n_net, float* marg, double* Z, int max_traj_chunk,
                          int precision, cudaStream_t s, bool graphs = false) {
    if (n_net <= 0) return PTN_OK;
    if (precision != PTN_PREC_FP32 && precision != PTN_PREC_BF16X3 && precision != PTN_PREC_FP16X3)
        return set_error(PTN_ERR_INVALID_ARG, "unknown precision mode %d", precision);
    PlanWorkspace* ws = workspace(plan);
    const BlockPlan& bp = plan->blocks[j];
    ptn_status e;
    // host copy of the trajectory index of every network
    if ((e = ws->h_traj.grow(sizeof(int32_t) * n_net))) return e;
    PTN_CUDA(cudaMemcpyAsync(ws->h_traj.p, d_net_traj, sizeof(int32_t) * n_net, cudaMemcpyDeviceToHost, s));
    PTN_CUDA(cudaStreamSynchronize(s));
    const int32_t* ht = ws->h_traj.as<int32_t>();
    for (int64_t i = 0; i < n_net; i++) {
        if (ht[i] < 0 || ht[i] >= tr->n_unique)
            return set_error(PTN_ERR_INVALID_ARG, "net_traj[%lld] = %d out of range", (long long)i, ht[i]);
        if (i && ht[i] < ht[i - 1]) return set_error(PTN_ERR_INVALID_ARG, "net_traj must be non-decreasing");
    }
    // chunking against the memory cap (arenas + GEMM operand packing, per instance)
    auto pk = [&](int c) { return 4.0 * (double)(bp.pack_peak[0][c] + bp.pack_peak[1][c]); };
    const double bT = 8.0 * (double)bp.arena_peak[CLS_TRAJ] + pk(CLS_TRAJ);
    const double bN = 8.0 * (double)bp.arena_peak[CLS_NET] + 4.0 + 8.0 + pk(CLS_NET);
    const double bC = 8.0 * (double)bp.arena_peak[CLS_CONST] + pk(CLS_CONST);
    const double cap = plan->mem_cap;
    if (bC + bT + bN > cap)
        return set_error(PTN_ERR_TOO_LARGE, "block %d needs %.3g bytes for one network (cap %.3g)", j, bC + bT + bN, cap);
    std::vector<Chunk> chunks;
    if ((e = ws->h_chunk_traj.grow(sizeof(int32_t) * n_net))) return e;
    if ((e = ws->h_net_tl.grow(sizeof(int32_t) * n_net))) return e;
    int32_t* hct = ws->h_chunk_traj.as<int32_t>();
    int32_t* htl = ws->h_net_tl.as<int32_t>();
    int64_t n_ct = 0;
    {
        Chunk c{0, 0, 0, 0};
        int64_t i = 0;
        while (i < n_net) {
            int64_t k = i;
            while (k < n_net && ht[k] == ht[i]) k++;
            int64_t run = k - i;   // networks of trajectory ht[i]
            int64_t done = 0;
            while (done < run) {
                bool traj_limit = max_traj_chunk > 0 && c.n_traj >= max_traj_chunk;
                double room = cap - bC - bT * (double)(c.n_traj + 1) - bN * (double)c.n_net;
                int64_t fit = room > 0 ? (int64_t)(room / bN) : 0;
                if (traj_limit || fit <= 0) {
                    if (c.n_net == 0) return set_error(PTN_ERR_TOO_LARGE, "block %d: no room for one network", j);
                    chunks.push_back(c);
                    c = Chunk{c.net0 + c.n_net, 0, n_ct, 0};
                    continue;
                }
                int64_t take = std::min(fit, run - done);
                hct[n_ct] = ht[i];
                for (int64_t q = 0; q < take; q++) htl[c.net0 + c.n_net + q] = (int32_t)c.n_traj;
                n_ct++;
                c.n_traj++;
                c.n_net += take;
                done += take;
            }
            i = k;
        }
        if (c.n_net) chunks.push_back(c);
    }
    if ((e = ws->chunk_traj.grow(sizeof(int32_t) * n_ct))) return e;
    if ((e = ws->net_tl.grow(sizeof(int32_t) * n_net))) return e;
    PTN_CUDA(cudaMemcpyAsync(ws->chunk_traj.p, hct, sizeof(int32_t) * n_ct, cudaMemcpyHostToDevice, s));
    PTN_CUDA(cudaMemcpyAsync(ws->net_tl.p, htl, sizeof(int32_t) * n_net, cudaMemcpyHostToDevice, s));
    int64_t max_t = 0, max_n = 0;
    for (auto& c : chunks) {
        max_t = std::max(max_t, c.n_traj);
        max_n = std::max(max_n, c.n_net);
    }
    // per chunk, the first network of every trajectory group (n_traj + 1 entries)
    const int64_t n_grp_all = n_ct + (int64_t)chunks.size();
    if ((e = ws->h_grp.grow(sizeof(int32_t) * n_grp_all)) || (e = ws->grp.grow(sizeof(int32_t) * n_grp_all)) ||
        (e = ws->grp_cnt.grow(sizeof(int64_t) * (max_t + 1))) || (e = ws->grp_tile0.grow(sizeof(int64_t) * (max_t + 1))) ||
        (e = ws->grp_scan.grow(sizeof(int64_t) * scan_tmp_elems(max_t + 1))))
        return e;
    int32_t* hg = ws->h_grp.as<int32_t>();
    std::vector<int64_t> grp_off(chunks.size());
    {
        int64_t o = 0;
        for (size_t ci = 0; ci < chunks.size(); ci++) {
            const Chunk& c = chunks[ci];
            grp_off[ci] = o;
            int32_t t = -1;
            for (int64_t q = 0; q < c.n_net; q++)
                if (htl[c.net0 + q] != t) hg[o + (t = htl[c.net0 + q])] = (int32_t)q;
            hg[o + c.n_traj] = (int32_t)c.n_net;
            o += c.n_traj + 1;
        }
    }
    PTN_CUDA(cudaMemcpyAsync(ws->grp.p, hg, sizeof(int32_t) * n_grp_all, cudaMemcpyHostToDevice, s));
    if ((e = ws->arena[CLS_CONST].grow((size_t)(8.0 * bp.arena_peak[CLS_CONST] + 16)))) return e;
    if ((e = ws->arena[CLS_TRAJ].grow((size_t)(8.0 * bp.arena_peak[CLS_TRAJ] * max_t + 16)))) return e;
    if ((e = ws->arena[CLS_NET].grow((size_t)(8.0 * bp.arena_peak[CLS_NET] * max_n + 16)))) return e;
    for (int r = 0; r < 2; r++) {
        const double need = 4.0 * ((double)bp.pack_peak[r][CLS_CONST] + (double)bp.pack_peak[r][CLS_TRAJ] * max_t +
                                   (double)bp.pack_peak[r][CLS_NET] * max_n);
        if (need > 0 && (e = ws->pack[r].grow((size_t)(need + need / 64) + 4096))) return e;
    }
    if ((e = ws->err.grow(sizeof(int)))) return e;
    if ((e = ws->h_small.grow(64))) return e;
    if (finalize_tiles(bp.b) > 1 && (e = ws->zpart.grow(sizeof(double) * max_n * finalize_tiles(bp.b)))) return e;
    // intermediate caching: tables sized for the largest chunk
    const bool caching = plan->opts.cache_intermediates && bp.n_cache > 0 && max_t >= 2;
    auto table_size = [](int64_t n) {
        int64_t P = 1;
        while (P < 2 * n) P <<= 1;
        return P;
    };
    if (caching) {
        const int64_t nc = bp.n_cache, P = table_size(max_t);
        if ((e = ensure_nz(tr, s)) || (e = ws->c_h.grow(sizeof(uint64_t) * 2 * nc * max_t)) ||
            (e = ws->c_keys.grow(sizeof(unsigned long long) * nc * P)) || (e = ws->c_first.grow(sizeof(int32_t) * nc * P)) ||
            (e = ws->c_rep.grow(sizeof(int32_t) * nc * max_t)) || (e = ws->c_list.grow(sizeof(int32_t) * nc * max_t)) ||
            (e = ws->c_cnt.grow(sizeof(int32_t) * nc)) || (e = ws->h_ccnt.grow(sizeof(int32_t) * nc)))
            return e;
    }
    PTN_CUDA(cudaMemsetAsync(ws->err.p, 0, sizeof(int), s));
    const RootRef* d_root = plan->d_roots + j;
    if (graphs) {
        if (!ws->cap_stream) PTN_CUDA(cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking));
        if (ws->gexec.size() < plan->blocks.size()) ws->gexec.resize(plan->blocks.size(), nullptr);
    }
    for (size_t ci = 0; ci < chunks.size(); ci++) {
        const Chunk& c = chunks[ci];
        // Cached steps run over the chunk's representatives: their tables and
        // counts are made (and the counts read back) before the chunk's steps
        // are launched or recorded.
        const int32_t* ccnt = nullptr;
        if (caching && c.n_traj >= 2) {
            CacheArgs ca;
            ca.n_cache = bp.n_cache;
            ca.words = bp.cache_words;
            ca.n = c.n_traj;
            ca.P = table_size(c.n_traj);
            ca.chunk_traj = ws->chunk_traj.as<int32_t>() + c.traj0;
            ca.nz_ptr = tr->nz_ptr;
            ca.nz_col = tr->nz_col;
            ca.nz_val = tr->nz_val;
            ca.bits = bp.d_cache_bits;
            ca.h = ws->c_h.as<uint64_t>();
            ca.keys = ws->c_keys.as<unsigned long long>();
            ca.first = ws->c_first.as<int32_t>();
            ca.rep = ws->c_rep.as<int32_t>();
            ca.list = ws->c_list.as<int32_t>();
            ca.cnt = ws->c_cnt.as<int32_t>();
            launch_cache_tables(ca, s);
            int32_t* hc = ws->h_ccnt.as<int32_t>();
            PTN_CUDA(cudaMemcpyAsync(hc, ca.cnt, sizeof(int32_t) * bp.n_cache, cudaMemcpyDeviceToHost, s));
            PTN_CUDA(cudaStreamSynchronize(s));
            ccnt = hc;
        }
        // With graphs, the chunk's launches are recorded on the capture stream
        // (nothing runs while recording) and the graph is launched on s.
        cudaStream_t ls = s;
        if (graphs) {
            PTN_CUDA(cudaStreamBeginCapture(ws->cap_stream, cudaStreamCaptureModeRelaxed));
            ls = ws->cap_stream;
        }
        auto end_capture = [&]() {
            if (!graphs) return;
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(ws->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
        };
        GroupTable gt;
        gt.n_groups = c.n_traj;
        gt.h_net0 = hg + grp_off[ci];
        gt.d_net0 = ws->grp.as<int32_t>() + grp_off[ci];
        gt.d_cnt = ws->grp_cnt.as<int64_t>();
        gt.d_tile0 = ws->grp_tile0.as<int64_t>();
        gt.d_scan = ws->grp_scan.as<int64_t>();
        ChunkCtx ctx;
        ctx.vtab = reinterpret_cast<const float2*>(plan->d_var_table);
        ctx.var_ids = tr->var_ids;
        ctx.n_var_cols = tr->n_var_cols;
        ctx.n_words = (plan->n_qubits + 63) / 64;
        ctx.chunk_traj = ws->chunk_traj.as<int32_t>() + c.traj0;
        ctx.net_tl = ws->net_tl.as<int32_t>() + c.net0;
        ctx.net_prefix = d_net_prefix + c.net0;
        for (int a = 0; a < 3; a++) ctx.arena[a] = ws->arena[a].as<float2>();
        ctx.arena[ARENA_ADJ] = ctx.arena[ARENA_LGRAD] = nullptr;
        ctx.arena_inst[ARENA_ADJ] = ctx.arena_inst[ARENA_LGRAD] = 0;
        ctx.arena_inst[CLS_CONST] = 1;
        ctx.arena_inst[CLS_TRAJ] = c.n_traj;
        ctx.arena_inst[CLS_NET] = c.n_net;
        if (ccnt) {
            ctx.cache_rep = ws->c_rep.as<int32_t>();
            ctx.cache_list = ws->c_list.as<int32_t>();
            ctx.cache_n = c.n_traj;
        }
        for (size_t st = 0; st < bp.steps.size(); st++) {
            const StepDesc& h = bp.steps[st];
            if (h.virt) continue;   // formed inside its consumer's operand pack
            StepTag tag(j, (int)st);
            if (small_step(h)) {   // a run of small trajectory-class steps: one fused launch
                size_t en = st + 1;
                while (en < bp.steps.size() && en - st < (size_t)plan->opts.fuse_max && bp.steps[en].fuse_prev) en++;
                if (en - st >= 2) {
                    launch_small_steps(bp.d_steps + st, &bp.steps[st], (int)(en - st), ctx, c.n_traj, ls);
                    st = en - 1;
                    continue;
                }
            }
            int64_t ni = h.out_cls == CLS_CONST ? 1 : (h.out_cls == CLS_TRAJ ? c.n_traj : c.n_net);
            if (ccnt && h.cache > 0) ni = ccnt[h.cache - 1];
            if (h.kind == STEP_GEMM || h.kind == STEP_GEMM_STACKED) {
                e = launch_gemm_step(h, ctx, ni, ws->pack[0].p, ws->pack[1].p, ws->err.as<int>(), gt,
                                     precision, ls, h.prod ? &bp.steps[h.prod_src] : nullptr);
                if (e) {
                    end_capture();
                    return e;
                }
            } else {
                launch_contract_step(bp.d_steps + st, h, ctx, ni, ls);
            }
        }
        {
            StepTag tag(j, (int)bp.steps.size());
            launch_finalize(d_root, ctx, bp.b, c.n_net, marg + c.net0 * ((int64_t)1 << bp.b), Z + c.net0,
                            ws->zpart.as<double>(), ls);
        }
        if (graphs) {
            // the block's executable graph takes the new chunk's parameters in
            // place; a chunk whose launch sequence differs in shape (other
            // launch counts) gets a fresh executable
            cudaGraph_t g = nullptr;
            PTN_CUDA(cudaStreamEndCapture(ws->cap_stream, &g));
            cudaGraphExec_t& x = ws->gexec[j];
            if (x) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(x, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(x);
                    x = nullptr;
                }
            }
            cudaError_t ge = x ? cudaSuccess : cudaGraphInstantiate(&x, g, 0);
            cudaGraphDestroy(g);
            if (ge != cudaSuccess) {
                x = nullptr;
                return set_error(PTN_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ge));
            }
            PTN_CUDA(cudaGraphLaunch(x, s));
        }
    }
    PTN_CUDA(cudaGetLastError());
    // a tensor-core step that gave up a bounded wait reports it through the error word
    int* herr = reinterpret_cast<int*>(ws->h_small.as<int64_t>() + 4);
    PTN_CUDA(cudaMemcpyAsync(herr, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PTN_CUDA(cudaStreamSynchronize(s));
    if (*herr) return set_error(PTN_ERR_TIMEOUT, "block %d: a tensor-core step timed out (code %d)", j, *herr);
    return PTN_OK;
}

}  // namespace

// ====================================================================== API ==
extern "C" {

const char* ptn_version(void) { return "ptn 0.1 (sm_103a)"; }

const char* ptn_status_string(ptn_status s) {
    switch (s) {
        case PTN_OK: return "PTN_OK";
        case PTN_ERR_INVALID_ARG: return "PTN_ERR_INVALID_ARG";
        case PTN_ERR_NOT_CPTP: return "PTN_ERR_NOT_CPTP";
        case PTN_ERR_TOO_LARGE: return "PTN_ERR_TOO_LARGE";
        case PTN_ERR_OOM: return "PTN_ERR_OOM";
        case PTN_ERR_CUDA: return "PTN_ERR_CUDA";
        case PTN_ERR_TIMEOUT: return "PTN_ERR_TIMEOUT";
        case PTN_ERR_UNSUPPORTED: return "PTN_ERR_UNSUPPORTED";
    }
    return "PTN_UNKNOWN_STATUS";
}

const char* ptn_last_error(void) { return last_error_text(); }

ptn_status ptn_plan_path(const ptn_circuit* circuit, const ptn_noise* noise, const int32_t* block_sizes,
                         int32_t n_blocks, const ptn_plan_opts* opts, ptn_plan** plan_out) {
    clear_error();
    if (!plan_out) return set_error(PTN_ERR_INVALID_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    ptn_plan* p = new (std::nothrow) ptn_plan();
    if (!p) return set_error(PTN_ERR_OOM, "host allocation failed");
    ptn_status s;
    try {
        s = build_plan(circuit, noise, block_sizes, n_blocks, opts, p);
    } catch (const std::bad_alloc&) {
        s = set_error(PTN_ERR_OOM, "host allocation failed while planning");
    }
    if (s != PTN_OK) {
        delete p;
        return s;
    }
    *plan_out = p;
    return PTN_OK;
}

ptn_status ptn_plan_describe(const ptn_plan* plan, int32_t detail, char* buf, size_t cap, size_t* len) {
    if (!plan) return set_error(PTN_ERR_INVALID_ARG, "plan is NULL");
    if (detail >= 2) {
        ptn_status e = build_expval_plan(const_cast<ptn_plan*>(plan));
        if (e) return e;
    }
    std::string d = describe_plan(plan, detail);
    if (len) *len = d.size();
    if (buf && cap) {
        size_t n = std::min(cap - 1, d.size());
        memcpy(buf, d.data(), n);
        buf[n] = 0;
    }
    return PTN_OK;
}

void ptn_plan_destroy(ptn_plan* plan) {
    if (!plan) return;
    drop_workspace(plan);
    if (plan->device >= 0) {
        cudaFree(plan->d_var_table);
        cudaFree(plan->d_site_tables);
        cudaFree(plan->d_leaf_site_ptr);
        cudaFree(plan->d_leaf_site_idx);
        cudaFree(plan->d_leaf_site_mul);
        for (auto& b : plan->blocks) {
            cudaFree(b.d_steps);
            cudaFree(b.d_cache_bits);
        }
        cudaFree(plan->d_roots);
    }
    delete plan->expval;
    delete plan;
}

static ptn_status presample_impl(const ptn_plan* plan, uint64_t seed, int32_t circuit_id, int64_t traj0,
                                 int64_t n_traj, int32_t dedup, ptn_traj** traj_out, ptn_stream stream);

ptn_status ptn_presample_trajectories(const ptn_plan* plan, uint64_t seed, int32_t circuit_id, int64_t n_traj,
                                      int32_t dedup, ptn_traj** traj_out, ptn_stream stream) {
    clear_error();
    return presample_impl(plan, seed, circuit_id, 0, n_traj, dedup, traj_out, stream);
}

ptn_status ptn_presample_range(const ptn_plan* plan, uint64_t seed, int32_t circuit_id, int64_t traj0, int64_t n_traj,
                               ptn_traj** traj_out, ptn_stream stream) {
    clear_error();
    if (traj0 < 0 || traj0 + n_traj > ((int64_t)1 << 32))
        return set_error(PTN_ERR_INVALID_ARG, "trajectory range [%lld, %lld) outside 0..2^32", (long long)traj0,
                         (long long)(traj0 + n_traj));
    return presample_impl(plan, seed, circuit_id, traj0, n_traj, 0, traj_out, stream);
}

static ptn_status presample_impl(const ptn_plan* plan, uint64_t seed, int32_t circuit_id, int64_t traj0,
                                 int64_t n_traj, int32_t dedup, ptn_traj** traj_out, ptn_stream stream) {
    if (!plan || !traj_out) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    *traj_out = nullptr;
    if (n_traj < 1 || n_traj > (1 << 24)) return set_error(PTN_ERR_INVALID_ARG, "n_traj %lld out of 1..2^24", (long long)n_traj);
    ptn_status e = ensure_device(plan);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t S = plan->n_sites;
    ptn_traj* t = new ptn_traj();
    t->plan = plan;
    t->n_orig = n_traj;
    t->n_sites = S;
    t->n_var_cols = plan->n_var_cols;
    uint8_t* kraus = nullptr;
    double* logq = nullptr;
    auto fail = [&](ptn_status st) {
        cudaFree(kraus);
        cudaFree(logq);
        cudaFree(t->kraus);
        cudaFree(t->logq);
        cudaFree(t->mult);
        cudaFree(t->first);
        cudaFree(t->var_ids);
        delete t;
        return st;
    };
#define TRY_CUDA(call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(set_error(e_ == cudaErrorMemoryAllocation ? PTN_ERR_OOM : PTN_ERR_CUDA, "%s: %s", \
                                  #call, cudaGetErrorString(e_)));                                         \
    } while (0)
    TRY_CUDA(cudaMalloc(&kraus, std::max<size_t>((size_t)n_traj * S, 16)));
    TRY_CUDA(cudaMalloc(&logq, sizeof(double) * n_traj));
    launch_presample(plan->d_site_tables, S, n_traj, traj0, seed, circuit_id, kraus, logq, s);
    TRY_CUDA(cudaGetLastError());
    if (!dedup) {
        t->n_unique = n_traj;
        t->kraus = kraus;
        t->logq = logq;
        kraus = nullptr;
        logq = nullptr;
        TRY_CUDA(cudaMalloc(&t->mult, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&t->first, sizeof(int64_t) * n_traj));
        launch_fill_i64(t->mult, 1, n_traj, s);
        // first = the trajectory's index in the whole draw
        std::vector<int64_t> id(n_traj);
        for (int64_t i = 0; i < n_traj; i++) id[i] = traj0 + i;
        TRY_CUDA(cudaMemcpyAsync(t->first, id.data(), sizeof(int64_t) * n_traj, cudaMemcpyHostToDevice, s));
        TRY_CUDA(cudaStreamSynchronize(s));
    } else {
        // first occurrence of every Kraus row: rows hashed, (hash, index) pairs
        // sorted stably by hash (the radix sort of the shot merge), each row
        // compared with the first row of its run of equal hashes
        uint64_t *h = nullptr, *h2 = nullptr;
        int64_t *first = nullptr, *flags = nullptr, *uid = nullptr, *tmp = nullptr, *ix = nullptr, *ix2 = nullptr,
                *hist = nullptr, *excl = nullptr, *start = nullptr;
        int64_t n_u = 0;
        const int64_t nh = radix_hist_elems(n_traj);
        TRY_CUDA(cudaMalloc(&h, sizeof(uint64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&h2, sizeof(uint64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&ix, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&ix2, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&hist, sizeof(int64_t) * nh));
        TRY_CUDA(cudaMalloc(&excl, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&start, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&first, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&flags, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&uid, sizeof(int64_t) * n_traj));
        TRY_CUDA(cudaMalloc(&tmp, sizeof(int64_t) * std::max(scan_tmp_elems(n_traj), scan_tmp_elems(nh))));
        launch_row_hash(kraus, n_traj, S, h, s);
        launch_iota_i64(ix, n_traj, s);
        {
            uint64_t* k[2] = {h, h2};
            int64_t* v[2] = {ix, ix2};
            int cur = 0;
            for (int shift = 0; shift < 64; shift += 8) {
                launch_radix_pass(k[cur], v[cur], n_traj, shift, hist, tmp, k[1 - cur], v[1 - cur], s);
                cur = 1 - cur;
            }
            // 8 passes: the sorted pairs are back in (h, ix)
            launch_run_flags(h, n_traj, flags, s);
            launch_exclusive_scan(flags, excl, n_traj, tmp, s);
            launch_run_starts(flags, excl, n_traj, start, s);
            launch_first_in_run(kraus, S, ix, flags, excl, start, n_traj, first, s);
        }
        launch_flags_first(first, n_traj, flags, s);
        launch_exclusive_scan(flags, uid, n_traj, tmp, s);
        int64_t last[2];
        TRY_CUDA(cudaMemcpyAsync(&last[0], uid + n_traj - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaMemcpyAsync(&last[1], flags + n_traj - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        n_u = last[0] + last[1];
        t->n_unique = n_u;
        TRY_CUDA(cudaMalloc(&t->kraus, std::max<size_t>((size_t)n_u * S, 16)));
        TRY_CUDA(cudaMalloc(&t->logq, sizeof(double) * n_u));
        TRY_CUDA(cudaMalloc(&t->mult, sizeof(int64_t) * n_u));
        TRY_CUDA(cudaMalloc(&t->first, sizeof(int64_t) * n_u));
        TRY_CUDA(cudaMemsetAsync(t->mult, 0, sizeof(int64_t) * n_u, s));
        launch_dedup_compact(kraus, logq, first, uid, n_traj, S, t->kraus, t->logq, t->mult, t->first, s);
        TRY_CUDA(cudaStreamSynchronize(s));
        cudaFree(h);
        cudaFree(h2);
        cudaFree(ix);
        cudaFree(ix2);
        cudaFree(hist);
        cudaFree(excl);
        cudaFree(start);
        cudaFree(first);
        cudaFree(flags);
        cudaFree(uid);
        cudaFree(tmp);
        cudaFree(kraus);
        cudaFree(logq);
        kraus = nullptr;
        logq = nullptr;
    }
    TRY_CUDA(cudaMalloc(&t->var_ids, std::max<size_t>(sizeof(int32_t) * t->n_unique * std::max(1, plan->n_var_cols), 16)));
    launch_var_ids(t->kraus, t->n_unique, S, plan->d_leaf_site_ptr, plan->d_leaf_site_idx, plan->d_leaf_site_mul,
                   plan->n_var_cols, t->var_ids, s);
    TRY_CUDA(cudaGetLastError());
#undef TRY_CUDA
    *traj_out = t;
    return PTN_OK;
}

ptn_status ptn_traj_info(const ptn_traj* t, int64_t* n_unique, int32_t* n_sites, const uint8_t** kraus,
                         const double** logq, const int64_t** mult, const int64_t** first) {
    if (!t) return set_error(PTN_ERR_INVALID_ARG, "traj is NULL");
    if (n_unique) *n_unique = t->n_unique;
    if (n_sites) *n_sites = t->n_sites;
    if (kraus) *kraus = t->kraus;
    if (logq) *logq = t->logq;
    if (mult) *mult = t->mult;
    if (first) *first = t->first;
    return PTN_OK;
}

ptn_status ptn_traj_copy(const ptn_traj* t, uint8_t* kraus_out, double* logq_out, int64_t* mult_out,
                         int64_t* first_out, ptn_stream stream) {
    if (!t) return set_error(PTN_ERR_INVALID_ARG, "traj is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->n_unique;
    if (kraus_out && n * t->n_sites)
        PTN_CUDA(cudaMemcpyAsync(kraus_out, t->kraus, (size_t)n * t->n_sites, cudaMemcpyDeviceToDevice, s));
    if (logq_out) PTN_CUDA(cudaMemcpyAsync(logq_out, t->logq, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (mult_out) PTN_CUDA(cudaMemcpyAsync(mult_out, t->mult, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
    if (first_out) PTN_CUDA(cudaMemcpyAsync(first_out, t->first, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
    return PTN_OK;
}

void ptn_traj_destroy(ptn_traj* t) {
    if (!t) return;
    cudaFree(t->nz_ptr);
    cudaFree(t->nz_col);
    cudaFree(t->nz_val);
    cudaFree(t->kraus);
    cudaFree(t->logq);
    cudaFree(t->mult);
    cudaFree(t->first);
    cudaFree(t->var_ids);
    delete t;
}

ptn_status ptn_tune_tiles(ptn_plan* plan, const ptn_traj* traj, int64_t n_probe, int32_t reps, int32_t* n_tuned_out,
                          int32_t* n_changed_out, ptn_stream stream) {
    clear_error();
    if (!plan || !traj) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    if (traj->plan != plan) return set_error(PTN_ERR_INVALID_ARG, "trajectories belong to another plan");
    if (n_probe < 1 || reps < 1 || reps > 100) return set_error(PTN_ERR_INVALID_ARG, "n_probe >= 1, reps in 1..100");
    ptn_status e = ensure_device(plan);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)stream;
    PlanWorkspace* ws = workspace(plan);
    const int W = (plan->n_qubits + 63) / 64;
    int32_t* d_traj = nullptr;
    uint64_t* d_prefix = nullptr;
    float* marg = nullptr;
    double* Z = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release_probe = [&]() {
        cudaFree(d_traj);
        cudaFree(d_prefix);
        cudaFree(marg);
        cudaFree(Z);
        d_traj = nullptr;
        d_prefix = nullptr;
        marg = nullptr;
        Z = nullptr;
    };
    auto fail = [&](ptn_status st) {
        release_probe();
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return st;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(set_error(PTN_ERR_CUDA, "tile tuning events"));
    int32_t tuned = 0, changed = 0;
    for (size_t j = 0; j < plan->blocks.size(); j++) {
        BlockPlan& bp = plan->blocks[j];
        // probe in the shape of a real chunk: k networks per trajectory (the
        // plan's modelled networks per trajectory, distinct prefixes), as many
        // trajectories as n_probe and one chunk allow
        int64_t k = 1;
        if (bp.start > 0 && bp.est_mult_traj > 0) {
            const double r = bp.est_mult_net / bp.est_mult_traj;
            k = std::max<int64_t>(1, (int64_t)std::llround(r));
            if (bp.start < 40) k = std::min<int64_t>(k, (int64_t)1 << bp.start);
        }
        auto pk = [&](int c) { return 4.0 * (double)(bp.pack_peak[0][c] + bp.pack_peak[1][c]); };
        const double bT = 8.0 * (double)bp.arena_peak[CLS_TRAJ] + pk(CLS_TRAJ);
        const double bN = 8.0 * (double)bp.arena_peak[CLS_NET] + 4.0 + 8.0 + pk(CLS_NET);
        const double bC = 8.0 * (double)bp.arena_peak[CLS_CONST] + pk(CLS_CONST);
        const int64_t fit = (int64_t)((plan->mem_cap - bC) / (bT + (double)k * bN));
        const int64_t nt = std::min(std::min<int64_t>(n_probe, traj->n_unique), fit);
        if (nt < 1) continue;
        const int64_t nn = nt * k;
        std::vector<int32_t> ht(nn);
        std::vector<uint64_t> hp(nn * W, 0);
        for (int64_t t = 0; t < nt; t++)
            for (int64_t q = 0; q < k; q++) {
                ht[t * k + q] = (int32_t)t;
                hp[(t * k + q) * W] = (uint64_t)q;
            }
        if (cudaMalloc(&d_traj, sizeof(int32_t) * nn) != cudaSuccess ||
            cudaMalloc(&d_prefix, sizeof(uint64_t) * nn * W) != cudaSuccess ||
            cudaMalloc(&marg, sizeof(float) * nn * ((int64_t)1 << bp.b)) != cudaSuccess ||
            cudaMalloc(&Z, sizeof(double) * nn) != cudaSuccess)
            return fail(set_error(PTN_ERR_OOM, "tile tuning buffers"));
        if (cudaMemcpyAsync(d_traj, ht.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_prefix, hp.data(), sizeof(uint64_t) * nn * W, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(set_error(PTN_ERR_CUDA, "tile tuning setup"));
        if ((e = contract_level(plan, traj, (int)j, d_traj, d_prefix, nn, marg, Z, 0, PTN_PREC_FP32, s)))
            return fail(e);
        ChunkCtx ctx;
        memset(&ctx, 0, sizeof ctx);
        ctx.vtab = reinterpret_cast<const float2*>(plan->d_var_table);
        ctx.var_ids = traj->var_ids;
        ctx.n_var_cols = traj->n_var_cols;
        ctx.chunk_traj = ws->chunk_traj.as<int32_t>();
        ctx.net_tl = ws->net_tl.as<int32_t>();
        ctx.net_prefix = d_prefix;
        ctx.n_words = W;
        for (int a = 0; a < 3; a++) ctx.arena[a] = ws->arena[a].as<float2>();
        ctx.arena_inst[CLS_CONST] = 1;
        ctx.arena_inst[CLS_TRAJ] = nt;
        ctx.arena_inst[CLS_NET] = nn;
        for (size_t st = 0; st < bp.steps.size(); st++) {
            StepDesc& h = bp.steps[st];
            if (small_step(h)) {   // fused runs are not tuned (one launch walks the whole run)
                size_t en = st + 1;
                while (en < bp.steps.size() && en - st < (size_t)plan->opts.fuse_max && bp.steps[en].fuse_prev) en++;
                if (en - st >= 2) {
                    st = en - 1;
                    continue;
                }
            }
            if (h.kind != STEP_DIRECT || h.virt) continue;
            int ra_av = 0, rb_av = 0;
            for (int q = 0; q < h.n_out; q++) {
                const bool va = h.out_stride[0][q] != 0, vb = h.out_stride[1][q] != 0;
                if (va && !vb) ra_av++;
                else if (vb && !va) rb_av++;
            }
            ra_av = std::min(ra_av, 2);
            rb_av = std::min(rb_av, 2);
            const int64_t ni = h.out_cls == CLS_CONST ? 1 : (h.out_cls == CLS_TRAJ ? nt : nn);
            // the default shape first; another shape replaces it only if it is
            // more than 5% faster (timing noise does not move the choice)
            const int def = 1 + 3 * ra_av + rb_av;
            int best = def;
            float best_ms = INFINITY, def_ms = INFINITY;
            for (int cand = -1; cand < (ra_av + 1) * (rb_av + 1); cand++) {
                const int ra = cand < 0 ? ra_av : cand / (rb_av + 1), rb = cand < 0 ? rb_av : cand % (rb_av + 1);
                if (cand >= 0 && ra == ra_av && rb == rb_av) continue;
                StepDesc h2 = h;
                h2.tile = 1 + 3 * ra + rb;
                launch_contract_step(bp.d_steps + st, h2, ctx, ni, s);   // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps; r++) launch_contract_step(bp.d_steps + st, h2, ctx, ni, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess)
                    return fail(set_error(PTN_ERR_CUDA, "tile tuning: %s", cudaGetErrorString(cudaGetLastError())));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (cand < 0) def_ms = ms;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = h2.tile;
                }
            }
            if (best_ms > 0.95f * def_ms) best = def;
            tuned++;
            if (best != def) changed++;
            h.tile = best;
        }
        release_probe();
    }
    fail(PTN_OK);
    if (n_tuned_out) *n_tuned_out = tuned;
    if (n_changed_out) *n_changed_out = changed;
    return PTN_OK;
}

ptn_status ptn_contract_batch(const ptn_plan* plan, const ptn_traj* traj, int32_t block, const int32_t* net_traj,
                              const uint64_t* net_prefix, int64_t n_net, int32_t precision, float* marg_out,
                              double* Z_out, ptn_stream stream) {
    clear_error();
    if (!plan || !traj || (n_net > 0 && (!net_traj || !net_prefix || !marg_out || !Z_out)))
        return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    if (traj->plan != plan) return set_error(PTN_ERR_INVALID_ARG, "trajectories belong to another plan");
    if (block < 0 || block >= (int32_t)plan->blocks.size()) return set_error(PTN_ERR_INVALID_ARG, "bad block %d", block);
    if (n_net < 0) return set_error(PTN_ERR_INVALID_ARG, "n_net < 0");
    ptn_status e = ensure_device(plan);
    if (e) return e;
    return contract_level(plan, traj, block, net_traj, net_prefix, n_net, marg_out, Z_out, 0, precision,
                          (cudaStream_t)stream);
}

}  // extern "C"

namespace {
// Device copies of the whole-circuit ket plan (forward steps, reversed steps,
// root, parametrised leaves), made once per plan.
ptn_status upload_expval_plan(const BlockPlan& bp, PlanWorkspace* ws) {
    if (ws->ev_steps.p) return PTN_OK;
    ptn_status e;
    if ((e = ws->ev_steps.grow(sizeof(StepDesc) * std::max<size_t>(bp.steps.size(), 1))) ||
        (e = ws->ev_bwd.grow(sizeof(StepDesc) * std::max<size_t>(bp.bwd.size(), 1))) ||
        (e = ws->ev_root.grow(sizeof(RootRef))) ||
        (e = ws->ev_pl.grow(sizeof(ParamLeaf) * std::max<size_t>(bp.pleaves.size(), 1))) ||
        (e = ws->ev_dvt.grow(sizeof(float2) * std::max<int64_t>(bp.dvt_size, 1))))
        return e;
    PTN_CUDA(cudaMemcpy(ws->ev_steps.p, bp.steps.data(), sizeof(StepDesc) * bp.steps.size(), cudaMemcpyHostToDevice));
    if (!bp.bwd.empty())
        PTN_CUDA(cudaMemcpy(ws->ev_bwd.p, bp.bwd.data(), sizeof(StepDesc) * bp.bwd.size(), cudaMemcpyHostToDevice));
    PTN_CUDA(cudaMemcpy(ws->ev_root.p, &bp.root, sizeof(RootRef), cudaMemcpyHostToDevice));
    if (!bp.pleaves.empty())
        PTN_CUDA(cudaMemcpy(ws->ev_pl.p, bp.pleaves.data(), sizeof(ParamLeaf) * bp.pleaves.size(),
                            cudaMemcpyHostToDevice));
    return PTN_OK;
}
}  // namespace

extern "C" {

ptn_status ptn_trajectory_amplitudes(const ptn_plan* cplan, const ptn_traj* traj, int64_t traj0, int64_t n_traj,
                                     int32_t precision, float* amp_out, ptn_stream stream) {
    clear_error();
    if (!cplan || !traj || (n_traj > 0 && !amp_out)) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    if (traj->plan != cplan) return set_error(PTN_ERR_INVALID_ARG, "trajectories belong to another plan");
    if (traj0 < 0 || n_traj < 0 || traj0 + n_traj > traj->n_unique)
        return set_error(PTN_ERR_INVALID_ARG, "trajectory range [%lld, %lld) outside 0..%lld", (long long)traj0,
                         (long long)(traj0 + n_traj), (long long)traj->n_unique);
    if (precision != PTN_PREC_FP32 && precision != PTN_PREC_BF16X3 && precision != PTN_PREC_FP16X3)
        return set_error(PTN_ERR_INVALID_ARG, "unknown precision mode %d", precision);
    ptn_plan* plan = const_cast<ptn_plan*>(cplan);
    ptn_status e;
    try {
        e = build_expval_plan(plan);
    } catch (const std::bad_alloc&) {
        e = set_error(PTN_ERR_OOM, "host allocation failed while planning");
    }
    if (e) return e;
    if ((e = ensure_device(plan))) return e;
    if (n_traj == 0) return PTN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PlanWorkspace* ws = workspace(plan);
    const BlockPlan& bp = *plan->expval;
    if ((e = upload_expval_plan(bp, ws))) return e;
    const int64_t E = traj->n_unique;
    if ((e = ws->ev_iota.grow(sizeof(int32_t) * E))) return e;
    launch_iota_i32(ws->ev_iota.as<int32_t>(), E, s);
    // forward steps only: the arenas of the kept intermediates, no adjoints
    auto pk = [&](int c) { return 4.0 * (double)(bp.pack_peak[0][c] + bp.pack_peak[1][c]); };
    const double bT = 8.0 * (double)bp.arena_peak[CLS_TRAJ] + pk(CLS_TRAJ);
    const double bC = 8.0 * (double)bp.arena_peak[CLS_CONST] + pk(CLS_CONST);
    const int64_t per = (int64_t)((plan->mem_cap - bC) / std::max(bT, 1.0));
    if (per < 1) return set_error(PTN_ERR_TOO_LARGE, "one trajectory needs %.3g bytes (cap %.3g)", bT + bC, plan->mem_cap);
    const int64_t Ec = std::min<int64_t>(per, n_traj);
    if ((e = ws->arena[CLS_CONST].grow((size_t)(8.0 * bp.arena_peak[CLS_CONST] + 16))) ||
        (e = ws->arena[CLS_TRAJ].grow((size_t)(8.0 * bp.arena_peak[CLS_TRAJ] * Ec + 16))) ||
        (e = ws->err.grow(sizeof(int))) || (e = ws->h_small.grow(64)))
        return e;
    for (int r = 0; r < 2; r++) {
        const double need = 4.0 * ((double)bp.pack_peak[r][CLS_CONST] + (double)bp.pack_peak[r][CLS_TRAJ] * Ec);
        if (need > 0 && (e = ws->pack[r].grow((size_t)(need + need / 64) + 4096))) return e;
    }
    PTN_CUDA(cudaMemsetAsync(ws->err.p, 0, sizeof(int), s));
    GroupTable no_groups;
    const int n = plan->n_qubits;
    for (int64_t t0 = 0; t0 < n_traj; t0 += Ec) {
        const int64_t nt = std::min(Ec, n_traj - t0);
        ChunkCtx ctx;
        ctx.vtab = reinterpret_cast<const float2*>(plan->d_var_table);
        ctx.var_ids = traj->var_ids;
        ctx.n_var_cols = traj->n_var_cols;
        ctx.n_words = 1;
        ctx.chunk_traj = ws->ev_iota.as<int32_t>() + traj0 + t0;
        ctx.net_tl = nullptr;
        ctx.net_prefix = nullptr;
        ctx.arena[CLS_CONST] = ws->arena[CLS_CONST].as<float2>();
        ctx.arena[CLS_TRAJ] = ws->arena[CLS_TRAJ].as<float2>();
        ctx.arena[CLS_NET] = ctx.arena[ARENA_ADJ] = ctx.arena[ARENA_LGRAD] = nullptr;
        ctx.arena_inst[CLS_CONST] = 1;
        ctx.arena_inst[CLS_TRAJ] = nt;
        ctx.arena_inst[CLS_NET] = ctx.arena_inst[ARENA_ADJ] = ctx.arena_inst[ARENA_LGRAD] = 0;
        for (size_t k = 0; k < bp.steps.size(); k++) {
            const StepDesc& h = bp.steps[k];
            StepTag tag(-2, (int)k);
            if (small_step(h)) {   // a run of small trajectory-class steps: one fused launch
                size_t en = k + 1;
                while (en < bp.steps.size() && en - k < (size_t)plan->opts.fuse_max && bp.steps[en].fuse_prev) en++;
                if (en - k >= 2) {
                    launch_small_steps(ws->ev_steps.as<StepDesc>() + k, &bp.steps[k], (int)(en - k), ctx, nt, s);
                    k = en - 1;
                    continue;
                }
            }
            const int64_t ni = h.out_cls == CLS_CONST ? 1 : nt;
            if (h.kind != STEP_DIRECT) {
                if ((e = launch_gemm_step(h, ctx, ni, ws->pack[0].p, ws->pack[1].p, ws->err.as<int>(), no_groups,
                                          precision, s)))
                    return e;
            } else {
                launch_contract_step(ws->ev_steps.as<StepDesc>() + k, h, ctx, ni, s);
            }
        }
        launch_amplitudes(ws->ev_root.as<RootRef>(), ctx, n, nt, reinterpret_cast<float2*>(amp_out) + (t0 << n), s);
    }
    PTN_CUDA(cudaGetLastError());
    int* herr = reinterpret_cast<int*>(ws->h_small.as<int64_t>() + 4);
    PTN_CUDA(cudaMemcpyAsync(herr, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PTN_CUDA(cudaStreamSynchronize(s));
    if (*herr) return set_error(PTN_ERR_TIMEOUT, "amplitudes: a tensor-core step timed out (code %d)", *herr);
    return PTN_OK;
}

ptn_status ptn_expval_grad(const ptn_plan* cplan, const ptn_traj* traj, const ptn_pauli_sum* obs, const double* theta,
                           int32_t n_theta, double* value_out, double* grad_out, ptn_stream stream) {
    clear_error();
    if (!cplan || !traj || !obs || !value_out || (n_theta > 0 && (!theta || !grad_out)))
        return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    if (traj->plan != cplan) return set_error(PTN_ERR_INVALID_ARG, "trajectories belong to another plan");
    ptn_plan* plan = const_cast<ptn_plan*>(cplan);
    if (n_theta < plan->n_params)
        return set_error(PTN_ERR_INVALID_ARG, "n_theta = %d but the circuit uses %d parameters", n_theta, plan->n_params);
    if (obs->n_terms < 1 || obs->n_terms > 4096 || !obs->coeff || !obs->z_mask)
        return set_error(PTN_ERR_INVALID_ARG, "bad observable");
    std::vector<ObsTerm> terms(obs->n_terms);
    for (int t = 0; t < obs->n_terms; t++) {
        if (obs->x_mask && obs->x_mask[t]) return set_error(PTN_ERR_UNSUPPORTED, "non-diagonal Pauli strings");
        terms[t].coeff = obs->coeff[t];
        terms[t].zmask = obs->z_mask[t];
    }
    ptn_status e;
    try {
        e = build_expval_plan(plan);
    } catch (const std::bad_alloc&) {
        e = set_error(PTN_ERR_OOM, "host allocation failed while planning");
    }
    if (e) return e;
    if ((e = ensure_device(plan))) return e;
    cudaStream_t s = (cudaStream_t)stream;
    PlanWorkspace* ws = workspace(plan);
    const BlockPlan& bp = *plan->expval;
    const int n = plan->n_qubits;
    const int64_t E = traj->n_unique;
    const int np = std::max(n_theta, 1);
    if ((e = upload_expval_plan(bp, ws))) return e;
    // merged tensors of the parametrised gates at theta, and their derivatives
    {
        std::vector<float> dvt(2 * std::max<int64_t>(bp.dvt_size, 1));
        for (const ParamLeaf& p : bp.pleaves) {
            LeafInfo& L = plan->leaves[p.leaf];
            param_leaf_tables(L, theta[p.param_index], &plan->var_table[2 * L.var_base], &dvt[2 * p.dvt_base]);
        }
        for (const ParamLeaf& p : bp.pleaves) {
            const LeafInfo& L = plan->leaves[p.leaf];
            PTN_CUDA(cudaMemcpyAsync(plan->d_var_table + 2 * L.var_base, &plan->var_table[2 * L.var_base],
                                     sizeof(float) * 2 * L.n_var * L.size, cudaMemcpyHostToDevice, s));
        }
        if (bp.dvt_size)
            PTN_CUDA(cudaMemcpyAsync(ws->ev_dvt.p, dvt.data(), sizeof(float) * 2 * bp.dvt_size, cudaMemcpyHostToDevice, s));
        PTN_CUDA(cudaStreamSynchronize(s));
    }
    if ((e = ws->ev_terms.grow(sizeof(ObsTerm) * terms.size())) || (e = ws->ev_F.grow(sizeof(double) * E)) ||
        (e = ws->ev_partial.grow(sizeof(double) * E * np)) || (e = ws->ev_iota.grow(sizeof(int32_t) * E)))
        return e;
    PTN_CUDA(cudaMemcpyAsync(ws->ev_terms.p, terms.data(), sizeof(ObsTerm) * terms.size(), cudaMemcpyHostToDevice, s));
    PTN_CUDA(cudaMemsetAsync(ws->ev_partial.p, 0, sizeof(double) * E * np, s));
    launch_iota_i32(ws->ev_iota.as<int32_t>(), E, s);
    // chunks of trajectories that fit the memory cap
    auto pk = [&](int c) { return 4.0 * (double)(bp.pack_peak[0][c] + bp.pack_peak[1][c]); };
    const double bT = 8.0 * (double)(bp.arena_peak[CLS_TRAJ] + bp.arena_peak[ARENA_ADJ] + bp.arena_peak[ARENA_LGRAD]) +
                      pk(CLS_TRAJ);
    const double bC = 8.0 * (double)bp.arena_peak[CLS_CONST] + pk(CLS_CONST);
    const int64_t per = (int64_t)((plan->mem_cap - bC) / std::max(bT, 1.0));
    if (per < 1) return set_error(PTN_ERR_TOO_LARGE, "one trajectory needs %.3g bytes (cap %.3g)", bT + bC, plan->mem_cap);
    const int64_t Ec = std::min<int64_t>(per, E);
    if ((e = ws->arena[CLS_CONST].grow((size_t)(8.0 * bp.arena_peak[CLS_CONST] + 16))) ||
        (e = ws->arena[CLS_TRAJ].grow((size_t)(8.0 * bp.arena_peak[CLS_TRAJ] * Ec + 16))) ||
        (e = ws->arena_x[0].grow((size_t)(8.0 * bp.arena_peak[ARENA_ADJ] * Ec + 16))) ||
        (e = ws->arena_x[1].grow((size_t)(8.0 * bp.arena_peak[ARENA_LGRAD] * Ec + 16))) || (e = ws->err.grow(sizeof(int))) ||
        (e = ws->h_small.grow(64)))
        return e;
    for (int r = 0; r < 2; r++) {
        const double need = 4.0 * ((double)bp.pack_peak[r][CLS_CONST] + (double)bp.pack_peak[r][CLS_TRAJ] * Ec);
        if (need > 0 && (e = ws->pack[r].grow((size_t)(need + need / 64) + 4096))) return e;
    }
    PTN_CUDA(cudaMemsetAsync(ws->err.p, 0, sizeof(int), s));
    GroupTable no_groups;
    for (int64_t t0 = 0; t0 < E; t0 += Ec) {
        const int64_t nt = std::min(Ec, E - t0);
        ChunkCtx ctx;
        ctx.vtab = reinterpret_cast<const float2*>(plan->d_var_table);
        ctx.var_ids = traj->var_ids;
        ctx.n_var_cols = traj->n_var_cols;
        ctx.n_words = 1;
        ctx.chunk_traj = ws->ev_iota.as<int32_t>() + t0;
        ctx.net_tl = nullptr;
        ctx.net_prefix = nullptr;
        ctx.arena[CLS_CONST] = ws->arena[CLS_CONST].as<float2>();
        ctx.arena[CLS_TRAJ] = ws->arena[CLS_TRAJ].as<float2>();
        ctx.arena[CLS_NET] = nullptr;
        ctx.arena[ARENA_ADJ] = ws->arena_x[0].as<float2>();
        ctx.arena[ARENA_LGRAD] = ws->arena_x[1].as<float2>();
        ctx.arena_inst[CLS_CONST] = 1;
        ctx.arena_inst[CLS_TRAJ] = ctx.arena_inst[ARENA_ADJ] = ctx.arena_inst[ARENA_LGRAD] = nt;
        ctx.arena_inst[CLS_NET] = 0;
        auto run = [&](const std::vector<StepDesc>& steps, const StepDesc* d_steps, int tag_block) -> ptn_status {
            for (size_t k = 0; k < steps.size(); k++) {
                const StepDesc& h = steps[k];
                StepTag tag(tag_block, (int)k);
                if (small_step(h)) {   // a run of small trajectory-class steps: one fused launch
                    size_t en = k + 1;
                    while (en < steps.size() && en - k < (size_t)plan->opts.fuse_max && steps[en].fuse_prev) en++;
                    if (en - k >= 2) {
                        launch_small_steps(d_steps + k, &steps[k], (int)(en - k), ctx, nt, s);
                        k = en - 1;
                        continue;
                    }
                }
                const int64_t ni = h.out_cls == CLS_CONST ? 1 : nt;
                if (h.kind != STEP_DIRECT) {
                    ptn_status ee = launch_gemm_step(h, ctx, ni, ws->pack[0].p, ws->pack[1].p, ws->err.as<int>(),
                                                     no_groups, PTN_PREC_FP32, s);
                    if (ee) return ee;
                } else {
                    launch_contract_step(d_steps + k, h, ctx, ni, s);
                }
            }
            return PTN_OK;
        };
        if ((e = run(bp.steps, ws->ev_steps.as<StepDesc>(), -2))) return e;
        launch_observable(ws->ev_root.as<RootRef>(), ctx, n, ws->ev_terms.as<ObsTerm>(), (int)terms.size(),
                          bp.root_adj_off, t0, ws->ev_F.as<double>(), s);
        if ((e = run(bp.bwd, ws->ev_bwd.as<StepDesc>(), -3))) return e;
        launch_leaf_grad(ctx, ws->ev_pl.as<ParamLeaf>(), (int)bp.pleaves.size(), ws->ev_dvt.as<float2>(), t0, nt, np,
                         ws->ev_partial.as<double>(), s);
    }
    launch_expval_reduce(traj->mult, ws->ev_F.as<double>(), ws->ev_partial.as<double>(), E, n_theta, value_out,
                         grad_out, s);
    PTN_CUDA(cudaGetLastError());
    int* herr = reinterpret_cast<int*>(ws->h_small.as<int64_t>() + 4);
    PTN_CUDA(cudaMemcpyAsync(herr, ws->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PTN_CUDA(cudaStreamSynchronize(s));
    if (*herr) return set_error(PTN_ERR_TIMEOUT, "gradient: a tensor-core step timed out (code %d)", *herr);
    return PTN_OK;
}

ptn_status ptn_allocate_shots(const double* weights, int64_t n, int64_t total, uint64_t seed, int32_t circuit_id,
                              int64_t* m_out, ptn_stream stream) {
    clear_error();
    if (!weights || !m_out || n < 1 || total < 0) return set_error(PTN_ERR_INVALID_ARG, "bad allocation arguments");
    double* cdf = nullptr;
    PTN_CUDA(cudaMallocAsync((void**)&cdf, sizeof(double) * n, (cudaStream_t)stream));
    launch_alloc_shots(weights, n, total, seed, circuit_id, cdf, m_out, (cudaStream_t)stream);
    PTN_CUDA(cudaFreeAsync(cdf, (cudaStream_t)stream));
    PTN_CUDA(cudaGetLastError());
    return PTN_OK;
}

static ptn_status alloc_sample_scratch(PlanWorkspace* ws, int64_t n_parent, int64_t n_traj, int64_t child_cap,
                                       SampleScratch& sc) {
    ptn_status e;
    size_t np = sizeof(int64_t) * std::max<int64_t>(n_parent, 1);
    if ((e = ws->s_cap.grow(np)) || (e = ws->s_tmp_off.grow(np)) || (e = ws->s_rank0.grow(np)) ||
        (e = ws->s_excl.grow(np)) || (e = ws->s_ndist.grow(np)) || (e = ws->s_out_off.grow(np)) ||
        (e = ws->s_first.grow(sizeof(int64_t) * std::max<int64_t>(n_traj, 1))) ||
        (e = ws->s_tmp_x.grow(sizeof(int32_t) * std::max<int64_t>(child_cap, 1))) ||
        (e = ws->s_tmp_c.grow(sizeof(int64_t) * std::max<int64_t>(child_cap, 1))) ||
        (e = ws->s_scan.grow(sizeof(int64_t) * scan_tmp_elems(std::max<int64_t>(n_parent, 1)))))
        return e;
    sc.cap = ws->s_cap.as<int64_t>();
    sc.tmp_off = ws->s_tmp_off.as<int64_t>();
    sc.rank0 = ws->s_rank0.as<int64_t>();
    sc.excl = ws->s_excl.as<int64_t>();
    sc.first = ws->s_first.as<int64_t>();
    sc.ndist = ws->s_ndist.as<int64_t>();
    sc.out_off = ws->s_out_off.as<int64_t>();
    sc.tmp_x = ws->s_tmp_x.as<int32_t>();
    sc.tmp_c = ws->s_tmp_c.as<int64_t>();
    sc.scan_tmp = ws->s_scan.as<int64_t>();
    return PTN_OK;
}

// Scratch for the standalone sampling entry point (not tied to a plan).
static PlanWorkspace* standalone_ws() {
    static PlanWorkspace ws;
    return &ws;
}

ptn_status ptn_sample_block(const float* marg, int32_t b, int32_t start, const int32_t* parent_traj,
                            const uint64_t* parent_prefix, const int64_t* parent_count, int64_t n_parent,
                            uint64_t seed, int32_t circuit_id, int32_t block, int32_t* child_traj,
                            uint64_t* child_prefix, int64_t* child_count, int64_t child_cap, int64_t* n_child,
                            ptn_stream stream) {
    clear_error();
    if (!n_child || b < 1 || b > 14 || start < 0 || start + b > 64 || n_parent < 0)
        return set_error(PTN_ERR_INVALID_ARG, "bad sampling arguments (b must be 1..14)");
    *n_child = 0;
    if (n_parent == 0) return PTN_OK;
    if (!marg || !parent_traj || !parent_prefix || !parent_count || !child_traj || !child_prefix || !child_count)
        return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    // trajectory ids bound the "first parent" table
    std::vector<int32_t> ht(n_parent);
    PTN_CUDA(cudaMemcpyAsync(ht.data(), parent_traj, sizeof(int32_t) * n_parent, cudaMemcpyDeviceToHost, s));
    PTN_CUDA(cudaStreamSynchronize(s));
    int32_t tmax = 0;
    for (int64_t i = 0; i < n_parent; i++) {
        if (ht[i] < 0) return set_error(PTN_ERR_INVALID_ARG, "negative trajectory index");
        if (i && ht[i] < ht[i - 1]) return set_error(PTN_ERR_INVALID_ARG, "parents must be grouped by trajectory");
        tmax = std::max(tmax, ht[i]);
    }
    PlanWorkspace* ws = standalone_ws();
    SampleScratch sc;
    ptn_status e = alloc_sample_scratch(ws, n_parent, (int64_t)tmax + 1, child_cap, sc);
    if (e) return e;
    if ((e = ws->h_small.grow(64))) return e;
    ptn_status st;
    int64_t nc = run_sample_block(marg, b, start, parent_traj, parent_prefix, parent_count, n_parent,
                                  (int64_t)tmax + 1, seed, circuit_id, block, child_traj, child_prefix, child_count,
                                  child_cap, sc, ws->h_small.as<int64_t>(), s, &st);
    if (st != PTN_OK) return st;
    PTN_CUDA(cudaGetLastError());
    *n_child = nc;
    return PTN_OK;
}

// Non-proportional NBS (Sec. III-B): every non-final block draws branch_shots
// shots per distinct prefix (its distinct outcomes become the next block's
// prefixes); the final block's networks are contracted in sub-batches that fit
// half the memory cap and each sub-batch's population vectors are harvested
// at once (direct draws or threshold), the records appended in order.
static ptn_status sample_nonprop(const ptn_plan* plan, const ptn_traj* traj, const ptn_sample_opts* o,
                                 ptn_shots** shots_out, cudaStream_t s) {
    const bool direct = o->mode == PTN_NONPROP_DIRECT;
    if (o->branch_shots < 1) return set_error(PTN_ERR_INVALID_ARG, "branch_shots must be >= 1");
    if (direct && o->final_shots < 1) return set_error(PTN_ERR_INVALID_ARG, "final_shots must be >= 1");
    if (!direct && !(o->threshold >= 0.0 && o->threshold <= 1.0))
        return set_error(PTN_ERR_INVALID_ARG, "threshold must be in [0, 1]");
    ptn_status e = ensure_device(plan);
    if (e) return e;
    PlanWorkspace* ws = workspace(plan);
    const int W = (plan->n_qubits + 63) / 64;   // words per prefix
    const int64_t E = traj->n_unique;
    const int nblk = (int)plan->blocks.size();
    if ((e = ws->h_small.grow(64))) return e;
    auto grow_level = [&](int k, int64_t cap) -> ptn_status {
        ptn_status g;
        if ((g = ws->lvl_traj[k].grow(sizeof(int32_t) * cap)) || (g = ws->lvl_prefix[k].grow(sizeof(uint64_t) * cap * W)) ||
            (g = ws->lvl_count[k].grow(sizeof(int64_t) * cap)))
            return g;
        return PTN_OK;
    };
    int cur = 0;
    int64_t n = E;
    if ((e = grow_level(0, E))) return e;
    launch_iota_i32(ws->lvl_traj[0].as<int32_t>(), E, s);
    PTN_CUDA(cudaMemsetAsync(ws->lvl_prefix[0].p, 0, sizeof(uint64_t) * E * W, s));
    std::vector<int64_t> nets;
    for (int j = 0; j + 1 < nblk && n > 0; j++) {
        const BlockPlan& bp = plan->blocks[j];
        const int64_t nb = (int64_t)1 << bp.b;
        if ((e = ws->marg.grow(sizeof(float) * n * nb)) || (e = ws->Z.grow(sizeof(double) * n))) return e;
        e = contract_level(plan, traj, j, ws->lvl_traj[cur].as<int32_t>(), ws->lvl_prefix[cur].as<uint64_t>(), n,
                           ws->marg.as<float>(), ws->Z.as<double>(), o->max_traj_per_chunk, o->precision, s,
                           o->use_graphs != 0);
        if (e) return e;
        launch_fill_i64(ws->lvl_count[cur].as<int64_t>(), o->branch_shots, n, s);
        const int64_t child_cap = n * std::min<int64_t>(o->branch_shots, nb);
        if ((e = grow_level(1 - cur, child_cap))) return e;
        SampleScratch sc;
        if ((e = alloc_sample_scratch(ws, n, E, child_cap, sc))) return e;
        ptn_status st;
        const int64_t nc = run_sample_block(ws->marg.as<float>(), bp.b, bp.start, ws->lvl_traj[cur].as<int32_t>(),
                                            ws->lvl_prefix[cur].as<uint64_t>(), ws->lvl_count[cur].as<int64_t>(), n, E,
                                            o->seed, o->circuit_id, j, ws->lvl_traj[1 - cur].as<int32_t>(),
                                            ws->lvl_prefix[1 - cur].as<uint64_t>(), ws->lvl_count[1 - cur].as<int64_t>(),
                                            child_cap, sc, ws->h_small.as<int64_t>(), s, &st, W);
        if (st != PTN_OK) return st;
        nets.push_back(n);
        cur = 1 - cur;
        n = nc;
    }
    // ---- final block
    const int jf = nblk - 1;
    const BlockPlan& bf = plan->blocks[jf];
    const int64_t nx = (int64_t)1 << bf.b;
    nets.push_back(n);
    const int32_t* ftraj = ws->lvl_traj[cur].as<int32_t>();
    const uint64_t* fprefix = ws->lvl_prefix[cur].as<uint64_t>();
    if (direct && n > 0) {
        if ((e = ws->h_rank0.grow(sizeof(int64_t) * n)) || (e = ws->h_first.grow(sizeof(uint64_t) * E))) return e;
        launch_harvest_ranks(ftraj, n, E, o->final_shots, ws->h_first.as<unsigned long long>(),
                             ws->h_rank0.as<int64_t>(), s);
    }
    const int64_t tiles = harvest_tiles(bf.b), tiles256 = harvest_cdf_tiles(bf.b);
    const double per_net = 4.0 * nx + 8.0 + 8.0 * finalize_tiles(bf.b) + 12.0 + 16.0 * tiles + 8.0 * scan_tmp_elems(tiles) +
                           (direct ? 4.0 * nx + 8.0 * tiles256 : 0.0);
    const int64_t sub = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(0.5 * plan->mem_cap / per_net)));
    if (n > 0) {
        if ((e = ws->marg.grow(sizeof(float) * sub * nx)) || (e = ws->Z.grow(sizeof(double) * sub)) ||
            (e = ws->h_rowmax.grow(sizeof(unsigned) * sub)) || (e = ws->h_T.grow(sizeof(uint64_t) * sub)) ||
            (e = ws->h_tcnt.grow(sizeof(int64_t) * sub * tiles)) || (e = ws->h_toff.grow(sizeof(int64_t) * sub * tiles)) ||
            (e = ws->h_scan.grow(sizeof(int64_t) * scan_tmp_elems(sub * tiles))))
            return e;
        if (direct && ((e = ws->h_tcdf.grow(sizeof(uint64_t) * sub * tiles256)) ||
                       (e = ws->h_cnt.grow(sizeof(unsigned) * sub * nx))))
            return e;
    }
    HarvestScratch hs;
    hs.rowmax = ws->h_rowmax.as<unsigned>();
    hs.T = ws->h_T.as<unsigned long long>();
    hs.tcdf = ws->h_tcdf.as<uint64_t>();
    hs.tcnt = ws->h_tcnt.as<int64_t>();
    hs.toff = ws->h_toff.as<int64_t>();
    hs.scan_tmp = ws->h_scan.as<int64_t>();
    hs.cnt = ws->h_cnt.as<unsigned>();
    struct Part {
        int32_t* t;
        uint64_t* b;
        int64_t* c;
        double* p;
        int64_t n;
    };
    std::vector<Part> parts;
    auto free_parts = [&]() {
        for (Part& p : parts) {
            cudaFree(p.t);
            cudaFree(p.b);
            cudaFree(p.c);
            cudaFree(p.p);
        }
        parts.clear();
    };
    int64_t total = 0;
    for (int64_t a = 0; a < n; a += sub) {
        const int64_t m = std::min(sub, n - a);
        e = contract_level(plan, traj, jf, ftraj + a, fprefix + a * W, m, ws->marg.as<float>(), ws->Z.as<double>(),
                           o->max_traj_per_chunk, o->precision, s, o->use_graphs != 0);
        if (e) {
            free_parts();
            return e;
        }
        HarvestArgs ha;
        ha.marg = ws->marg.as<float>();
        ha.b = bf.b;
        ha.start = bf.start;
        ha.n_net = m;
        ha.direct = direct;
        ha.tau = o->threshold;
        ha.traj = ftraj + a;
        ha.prefix = fprefix + a * W;
        ha.n_words = W;
        ha.rank0 = direct ? ws->h_rank0.as<int64_t>() + a : nullptr;
        ha.shots = o->final_shots;
        ha.seed = o->seed;
        ha.circuit = o->circuit_id;
        ha.block = jf;
        ptn_status st;
        const int64_t nr = run_harvest_count(ha, hs, ws->h_small.as<int64_t>(), s, &st);
        if (st != PTN_OK) {
            free_parts();
            return st;
        }
        if (nr == 0) continue;
        Part p{nullptr, nullptr, nullptr, nullptr, nr};
        cudaError_t ce;
        if ((ce = cudaMalloc(&p.t, sizeof(int32_t) * nr)) != cudaSuccess ||
            (ce = cudaMalloc(&p.b, sizeof(uint64_t) * nr * W)) != cudaSuccess ||
            (ce = cudaMalloc(&p.c, sizeof(int64_t) * nr)) != cudaSuccess ||
            (ce = cudaMalloc(&p.p, sizeof(double) * nr)) != cudaSuccess) {
            parts.push_back(p);
            free_parts();
            return set_error(PTN_ERR_OOM, "harvest records (%lld): %s", (long long)nr, cudaGetErrorString(ce));
        }
        parts.push_back(p);
        run_harvest_write(ha, hs, p.t, p.b, p.c, p.p, s);
        total += nr;
    }
    ptn_shots* r = new ptn_shots();
    r->n = total;
    r->n_qubits = plan->n_qubits;
    r->n_words = W;
    r->nets_per_block = nets;
    const size_t mcap = std::max<int64_t>(total, 1);
    cudaError_t ce;
    if (parts.size() == 1) {
        r->traj = parts[0].t;
        r->bits = parts[0].b;
        r->count = parts[0].c;
        r->prob = parts[0].p;
        parts.clear();
    } else if ((ce = cudaMalloc(&r->traj, sizeof(int32_t) * mcap)) != cudaSuccess ||
               (ce = cudaMalloc(&r->bits, sizeof(uint64_t) * mcap * W)) != cudaSuccess ||
               (ce = cudaMalloc(&r->count, sizeof(int64_t) * mcap)) != cudaSuccess ||
               (ce = cudaMalloc(&r->prob, sizeof(double) * mcap)) != cudaSuccess) {
        free_parts();
        ptn_shots_destroy(r);
        return set_error(PTN_ERR_OOM, "result allocation: %s", cudaGetErrorString(ce));
    } else {
        int64_t o_ = 0;
        for (Part& p : parts) {
            cudaMemcpyAsync(r->traj + o_, p.t, sizeof(int32_t) * p.n, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(r->bits + o_ * W, p.b, sizeof(uint64_t) * p.n * W, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(r->count + o_, p.c, sizeof(int64_t) * p.n, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(r->prob + o_, p.p, sizeof(double) * p.n, cudaMemcpyDeviceToDevice, s);
            o_ += p.n;
        }
        cudaStreamSynchronize(s);
        free_parts();
    }
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        ptn_shots_destroy(r);
        return set_error(PTN_ERR_CUDA, "non-proportional sampling: %s", cudaGetErrorString(ce));
    }
    *shots_out = r;
    return PTN_OK;
}

ptn_status ptn_sample_shots(const ptn_plan* plan, const ptn_traj* traj, const ptn_sample_opts* o,
                            ptn_shots** shots_out, ptn_stream stream) {
    clear_error();
    if (!plan || !traj || !o || !shots_out) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    *shots_out = nullptr;
    if (traj->plan != plan) return set_error(PTN_ERR_INVALID_ARG, "trajectories belong to another plan");
    if (o->use_graphs != 0 && o->use_graphs != 1) return set_error(PTN_ERR_INVALID_ARG, "use_graphs must be 0 or 1");
    if (o->mode == PTN_NONPROP_DIRECT || o->mode == PTN_NONPROP_EXHAUSTIVE)
        return sample_nonprop(plan, traj, o, shots_out, (cudaStream_t)stream);
    if (o->mode != PTN_PROPORTIONAL_FIXED && o->mode != PTN_PROPORTIONAL_TOTAL)
        return set_error(PTN_ERR_UNSUPPORTED, "sampling mode %d", o->mode);
    for (size_t j = 0; j < plan->blocks.size(); j++)
        if (plan->blocks[j].b > kMaxSampleBlock)
            return set_error(PTN_ERR_UNSUPPORTED,
                             "block %zu has %d qubits; proportional sampling draws from blocks of at most %d "
                             "(larger final blocks are harvested by the non-proportional modes)",
                             j, plan->blocks[j].b, kMaxSampleBlock);
    int64_t total_cap;
    if (o->mode == PTN_PROPORTIONAL_FIXED) {
        if (o->shots_per_traj < 1) return set_error(PTN_ERR_INVALID_ARG, "shots_per_traj must be >= 1");
        total_cap = o->shots_per_traj * traj->n_orig;
    } else {
        if (o->total_shots < 1) return set_error(PTN_ERR_INVALID_ARG, "total_shots must be >= 1");
        total_cap = o->total_shots;
    }
    ptn_status e = ensure_device(plan);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)stream;
    PlanWorkspace* ws = workspace(plan);
    const int W = (plan->n_qubits + 63) / 64;   // words per prefix
    const int64_t E = traj->n_unique;
    const int64_t lvl_cap = std::max(E, total_cap);
    for (int k = 0; k < 2; k++) {
        if ((e = ws->lvl_traj[k].grow(sizeof(int32_t) * lvl_cap)) || (e = ws->lvl_prefix[k].grow(sizeof(uint64_t) * lvl_cap * W)) ||
            (e = ws->lvl_count[k].grow(sizeof(int64_t) * lvl_cap)))
            return e;
    }
    if ((e = ws->h_small.grow(64))) return e;
    int cur = 0;
    int64_t n = E;
    launch_iota_i32(ws->lvl_traj[0].as<int32_t>(), E, s);
    PTN_CUDA(cudaMemsetAsync(ws->lvl_prefix[0].p, 0, sizeof(uint64_t) * E * W, s));
    if (o->mode == PTN_PROPORTIONAL_FIXED) launch_scale_i64(traj->mult, o->shots_per_traj, E, ws->lvl_count[0].as<int64_t>(), s);
    std::vector<int64_t> nets;
    for (size_t j = 0; j < plan->blocks.size() && n > 0; j++) {
        const BlockPlan& bp = plan->blocks[j];
        const int64_t nb = (int64_t)1 << bp.b;
        if ((e = ws->marg.grow(sizeof(float) * n * nb)) || (e = ws->Z.grow(sizeof(double) * n))) return e;
        e = contract_level(plan, traj, (int)j, ws->lvl_traj[cur].as<int32_t>(), ws->lvl_prefix[cur].as<uint64_t>(), n,
                           ws->marg.as<float>(), ws->Z.as<double>(), o->max_traj_per_chunk, o->precision, s,
                           o->use_graphs != 0);
        if (e) return e;
        if (j == 0 && o->mode == PTN_PROPORTIONAL_TOTAL) {
            if ((e = ws->w.grow(sizeof(double) * E)) || (e = ws->cdf.grow(sizeof(double) * E))) return e;
            launch_mult_times_z(traj->mult, ws->Z.as<double>(), E, ws->w.as<double>(), s);
            launch_alloc_shots(ws->w.as<double>(), E, o->total_shots, o->seed, o->circuit_id, ws->cdf.as<double>(),
                               ws->lvl_count[cur].as<int64_t>(), s);
        }
        SampleScratch sc;
        if ((e = alloc_sample_scratch(ws, n, E, total_cap, sc))) return e;
        ptn_status st;
        int64_t nc = run_sample_block(ws->marg.as<float>(), bp.b, bp.start, ws->lvl_traj[cur].as<int32_t>(),
                                      ws->lvl_prefix[cur].as<uint64_t>(), ws->lvl_count[cur].as<int64_t>(), n, E,
                                      o->seed, o->circuit_id, (int)j, ws->lvl_traj[1 - cur].as<int32_t>(),
                                      ws->lvl_prefix[1 - cur].as<uint64_t>(), ws->lvl_count[1 - cur].as<int64_t>(),
                                      lvl_cap, sc, ws->h_small.as<int64_t>(), s, &st, W);
        if (st != PTN_OK) return st;
        nets.push_back(n);
        cur = 1 - cur;
        n = nc;
    }
    ptn_shots* r = new ptn_shots();
    r->n = n;
    r->n_qubits = plan->n_qubits;
    r->n_words = W;
    r->nets_per_block = nets;
    size_t m = std::max<int64_t>(n, 1);
    cudaError_t ce;
    if ((ce = cudaMalloc(&r->traj, sizeof(int32_t) * m)) != cudaSuccess || (ce = cudaMalloc(&r->bits, sizeof(uint64_t) * m * W)) != cudaSuccess ||
        (ce = cudaMalloc(&r->count, sizeof(int64_t) * m)) != cudaSuccess) {
        cudaFree(r->traj);
        cudaFree(r->bits);
        cudaFree(r->count);
        delete r;
        return set_error(PTN_ERR_OOM, "result allocation: %s", cudaGetErrorString(ce));
    }
    if (n > 0) {
        PTN_CUDA(cudaMemcpyAsync(r->traj, ws->lvl_traj[cur].p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        PTN_CUDA(cudaMemcpyAsync(r->bits, ws->lvl_prefix[cur].p, sizeof(uint64_t) * n * W, cudaMemcpyDeviceToDevice, s));
        PTN_CUDA(cudaMemcpyAsync(r->count, ws->lvl_count[cur].p, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    PTN_CUDA(cudaGetLastError());
    *shots_out = r;
    return PTN_OK;
}

ptn_status ptn_sample_shots_batch(const ptn_batch_item* items, int32_t n_items, const ptn_batch_opts* bo,
                                  ptn_shots** shots_out, ptn_status* status_out, ptn_stream stream) {
    clear_error();
    if (n_items < 0 || (n_items > 0 && (!items || !shots_out || !status_out)))
        return set_error(PTN_ERR_INVALID_ARG, "NULL argument or negative item count");
    for (int32_t i = 0; i < n_items; i++) {
        shots_out[i] = nullptr;
        status_out[i] = PTN_OK;
        if (!items[i].plan || !items[i].traj || items[i].traj->plan != items[i].plan)
            return set_error(PTN_ERR_INVALID_ARG, "item %d: missing plan/trajectories or trajectories of another plan", i);
    }
    if (n_items == 0) return PTN_OK;
    int dev = 0;
    PTN_CUDA(cudaGetDevice(&dev));
    const int n_workers = std::max(1, std::min(bo && bo->n_workers > 0 ? bo->n_workers : 4, 64));
    const bool keep = bo && bo->keep_workspaces;
    const double max_est = bo ? bo->max_est_seconds : 0.0;
    // groups of items sharing a plan, in first-appearance order
    struct Group {
        const ptn_plan* plan;
        std::vector<int32_t> items;
        double cost;
    };
    std::vector<Group> groups;
    for (int32_t i = 0; i < n_items; i++) {
        size_t g = 0;
        while (g < groups.size() && groups[g].plan != items[i].plan) g++;
        if (g == groups.size()) groups.push_back({items[i].plan, {}, 0.0});
        groups[g].items.push_back(i);
    }
    double budget = bo && bo->mem_budget_bytes > 0 ? bo->mem_budget_bytes : 0.0;
    for (auto& g : groups) {
        double est = 0;
        for (const auto& b : g.plan->blocks) est += b.est_time;
        g.cost = est * (double)g.items.size();
        if (max_est > 0 && est > max_est)
            for (int32_t i : g.items) status_out[i] = PTN_ERR_TOO_LARGE;
    }
    // longest first (ties by first appearance)
    std::vector<size_t> order(groups.size());
    for (size_t g = 0; g < order.size(); g++) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return groups[a].cost > groups[b].cost; });
    // upload plans and set their caps on this thread; earlier workspaces are
    // freed first so the workers allocate stream-ordered memory only
    std::vector<double> saved_cap(groups.size());
    for (auto& g : groups) {
        drop_workspace(g.plan);
        ptn_status e = ensure_device(g.plan);
        if (e) {
            for (int32_t i : g.items) status_out[i] = e;
        }
    }
    if (budget <= 0) {
        size_t fr = 0, tot = 0;
        PTN_CUDA(cudaMemGetInfo(&fr, &tot));
        budget = 0.7 * (double)fr;   // workspace beyond the arenas (packs, levels) comes on top
    }
    for (size_t g = 0; g < groups.size(); g++) {
        ptn_plan* pl = const_cast<ptn_plan*>(groups[g].plan);
        saved_cap[g] = pl->mem_cap;
        if (pl->opts.mem_cap_bytes <= 0) pl->mem_cap = budget / n_workers;
    }
    cudaStream_t s0 = (cudaStream_t)stream;
    cudaEvent_t ev0;
    PTN_CUDA(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
    PTN_CUDA(cudaEventRecord(ev0, s0));
    std::vector<cudaStream_t> ws_streams(n_workers, nullptr);
    std::vector<cudaEvent_t> ws_done(n_workers, nullptr);
    for (int w = 0; w < n_workers; w++) {
        PTN_CUDA(cudaStreamCreateWithFlags(&ws_streams[w], cudaStreamNonBlocking));
        PTN_CUDA(cudaEventCreateWithFlags(&ws_done[w], cudaEventDisableTiming));
        PTN_CUDA(cudaStreamWaitEvent(ws_streams[w], ev0, 0));
    }
    std::atomic<size_t> next{0};
    std::mutex msg_mu;
    std::string first_msg;
    bool first_strong = false;
    auto worker = [&](int w) {
        cudaSetDevice(dev);
        cudaStream_t s = ws_streams[w];
        AsyncAllocScope scope(s);
        for (;;) {
            const size_t k = next.fetch_add(1);
            if (k >= order.size()) break;
            const Group& g = groups[order[k]];
            for (int32_t i : g.items) {
                if (status_out[i] != PTN_OK) continue;
                ptn_status st;
                try {
                    st = ptn_sample_shots(items[i].plan, items[i].traj, &items[i].opts, &shots_out[i], s);
                } catch (const std::bad_alloc&) {
                    st = set_error(PTN_ERR_OOM, "host allocation failed");
                }
                status_out[i] = st;
                if (st != PTN_OK) {
                    // keep the first message, preferring a resource or CUDA failure over
                    // an over-budget circuit
                    std::lock_guard<std::mutex> lk(msg_mu);
                    const bool strong = st != PTN_ERR_TOO_LARGE;
                    if (first_msg.empty() || (strong && !first_strong)) {
                        char buf[64];
                        snprintf(buf, sizeof buf, "item %d: ", i);
                        first_msg = std::string(buf) + last_error_text();
                        first_strong = strong;
                    }
                }
            }
            if (!keep) drop_workspace(g.plan);
        }
        cudaEventRecord(ws_done[w], s);
    };
    std::vector<std::thread> threads;
    for (int w = 0; w < n_workers; w++) threads.emplace_back(worker, w);
    for (auto& t : threads) t.join();
    for (int w = 0; w < n_workers; w++) {
        cudaStreamWaitEvent(s0, ws_done[w], 0);
        cudaEventDestroy(ws_done[w]);
        cudaStreamDestroy(ws_streams[w]);
    }
    cudaEventDestroy(ev0);
    // Items that ran out of device memory (or hit a CUDA error) while sharing the
    // device with other workers run once more alone, with the whole budget.
    if (n_workers > 1) {
        AsyncAllocScope scope(s0);
        for (int32_t i = 0; i < n_items; i++) {
            if (status_out[i] != PTN_ERR_OOM && status_out[i] != PTN_ERR_CUDA) continue;
            ptn_plan* pl = const_cast<ptn_plan*>(items[i].plan);
            drop_workspace(pl);
            if (pl->opts.mem_cap_bytes <= 0) pl->mem_cap = budget;
            ptn_status st;
            try {
                st = ptn_sample_shots(items[i].plan, items[i].traj, &items[i].opts, &shots_out[i], s0);
            } catch (const std::bad_alloc&) {
                st = set_error(PTN_ERR_OOM, "host allocation failed");
            }
            status_out[i] = st;
            if (st != PTN_OK && first_msg.empty()) first_msg = std::string("retried item: ") + last_error_text();
            if (!keep) drop_workspace(pl);
        }
    }
    for (size_t g = 0; g < groups.size(); g++) const_cast<ptn_plan*>(groups[g].plan)->mem_cap = saved_cap[g];
    clear_error();
    if (!first_msg.empty()) set_error(PTN_OK, "%s", first_msg.c_str());
    PTN_CUDA(cudaGetLastError());
    return PTN_OK;
}

ptn_status ptn_shots_merge(const ptn_shots* in, ptn_shots** out, ptn_stream stream) {
    clear_error();
    if (!in || !out) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = in->n;
    ptn_shots* r = new ptn_shots();
    r->n_qubits = in->n_qubits;
    r->n_words = in->n_words;
    r->nets_per_block = in->nets_per_block;
    const int W = in->n_words;
    int64_t n_runs = 0;
    std::vector<void*> tmp;
    auto fail = [&](ptn_status st) {
        for (void* p : tmp) cudaFreeAsync(p, s);
        cudaFree(r->traj);
        cudaFree(r->bits);
        cudaFree(r->count);
        delete r;
        return st;
    };
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s) != cudaSuccess) return nullptr;
        tmp.push_back(p);
        return p;
    };
    if (n > 0) {
        const int64_t nh = radix_hist_elems(n);
        uint64_t* k[2] = {static_cast<uint64_t*>(alloc(8 * n)), static_cast<uint64_t*>(alloc(8 * n))};
        int64_t* v[2] = {static_cast<int64_t*>(alloc(8 * n)), static_cast<int64_t*>(alloc(8 * n))};
        int64_t* hist = static_cast<int64_t*>(alloc(8 * nh));
        int64_t* scan = static_cast<int64_t*>(alloc(8 * std::max(scan_tmp_elems(nh), scan_tmp_elems(n))));
        int64_t* flag = static_cast<int64_t*>(alloc(8 * n));
        int64_t* excl = static_cast<int64_t*>(alloc(8 * n));
        int64_t* start = static_cast<int64_t*>(alloc(8 * n));
        if (!k[0] || !k[1] || !v[0] || !v[1] || !hist || !scan || !flag || !excl || !start)
            return fail(set_error(PTN_ERR_OOM, "merge scratch"));
        cudaError_t ce = cudaSuccess;
        int cur = 0;
        if (W == 1) {
            ce = cudaMemcpyAsync(k[0], in->bits, 8 * n, cudaMemcpyDeviceToDevice, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(v[0], in->count, 8 * n, cudaMemcpyDeviceToDevice, s);
            if (ce != cudaSuccess) return fail(set_error(PTN_ERR_CUDA, "merge copy: %s", cudaGetErrorString(ce)));
            for (int shift = 0; shift < in->n_qubits; shift += 8) {
                launch_radix_pass(k[cur], v[cur], n, shift, hist, scan, k[1 - cur], v[1 - cur], s);
                cur = 1 - cur;
            }
            launch_run_flags(k[cur], n, flag, s);
        } else {
            // record indices sorted word by word, least significant word first
            launch_iota_i64(v[0], n, s);
            for (int w = 0; w < W; w++) {
                launch_gather_word(in->bits, v[cur], W, w, n, k[cur], s);
                const int top = std::min(64, in->n_qubits - 64 * w);
                for (int shift = 0; shift < top; shift += 8) {
                    launch_radix_pass(k[cur], v[cur], n, shift, hist, scan, k[1 - cur], v[1 - cur], s);
                    cur = 1 - cur;
                }
            }
            launch_run_flags_words(in->bits, v[cur], W, n, flag, s);
        }
        launch_exclusive_scan(flag, excl, n, scan, s);
        launch_run_starts(flag, excl, n, start, s);
        int64_t last[2];
        ce = cudaMemcpyAsync(&last[0], excl + n - 1, 8, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&last[1], flag + n - 1, 8, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return fail(set_error(PTN_ERR_CUDA, "merge: %s", cudaGetErrorString(ce)));
        n_runs = last[0] + last[1];
        size_t m = std::max<int64_t>(n_runs, 1);
        if ((ce = cudaMalloc(&r->traj, sizeof(int32_t) * m)) != cudaSuccess ||
            (ce = cudaMalloc(&r->bits, sizeof(uint64_t) * m * W)) != cudaSuccess ||
            (ce = cudaMalloc(&r->count, sizeof(int64_t) * m)) != cudaSuccess)
            return fail(set_error(PTN_ERR_OOM, "merge result: %s", cudaGetErrorString(ce)));
        if (W == 1) launch_run_sum(k[cur], v[cur], start, n_runs, n, r->traj, r->bits, r->count, s);
        else launch_run_sum_words(in->bits, in->count, v[cur], W, start, n_runs, n, r->traj, r->bits, r->count, s);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(set_error(PTN_ERR_CUDA, "merge: %s", cudaGetErrorString(ce)));
    } else {
        cudaError_t ce;
        if ((ce = cudaMalloc(&r->traj, 16)) != cudaSuccess || (ce = cudaMalloc(&r->bits, 16)) != cudaSuccess ||
            (ce = cudaMalloc(&r->count, 16)) != cudaSuccess)
            return fail(set_error(PTN_ERR_OOM, "merge result: %s", cudaGetErrorString(ce)));
    }
    for (void* p : tmp) cudaFreeAsync(p, s);
    r->n = n_runs;
    *out = r;
    return PTN_OK;
}

ptn_status ptn_shots_info(const ptn_shots* r, int64_t* n_out, const int32_t** traj, const uint64_t** bits,
                          const int64_t** count, int64_t* nets_per_block, int32_t cap_blocks) {
    if (!r) return set_error(PTN_ERR_INVALID_ARG, "shots is NULL");
    if (n_out) *n_out = r->n;
    if (traj) *traj = r->traj;
    if (bits) *bits = r->bits;
    if (count) *count = r->count;
    if (nets_per_block)
        for (int32_t j = 0; j < cap_blocks; j++) nets_per_block[j] = j < (int32_t)r->nets_per_block.size() ? r->nets_per_block[j] : 0;
    return PTN_OK;
}

ptn_status ptn_shots_copy(const ptn_shots* r, int32_t* traj_out, uint64_t* bits_out, int64_t* count_out,
                          ptn_stream stream) {
    if (!r) return set_error(PTN_ERR_INVALID_ARG, "shots is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (r->n > 0) {
        if (traj_out) PTN_CUDA(cudaMemcpyAsync(traj_out, r->traj, sizeof(int32_t) * r->n, cudaMemcpyDeviceToDevice, s));
        if (bits_out)
            PTN_CUDA(cudaMemcpyAsync(bits_out, r->bits, sizeof(uint64_t) * r->n * r->n_words, cudaMemcpyDeviceToDevice, s));
        if (count_out) PTN_CUDA(cudaMemcpyAsync(count_out, r->count, sizeof(int64_t) * r->n, cudaMemcpyDeviceToDevice, s));
    }
    return PTN_OK;
}

ptn_status ptn_shots_probs(const ptn_shots* r, const double** prob) {
    if (!r || !prob) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    *prob = r->prob;
    return PTN_OK;
}

ptn_status ptn_shots_copy_probs(const ptn_shots* r, double* prob_out, ptn_stream stream) {
    if (!r || !prob_out) return set_error(PTN_ERR_INVALID_ARG, "NULL argument");
    if (!r->prob) return set_error(PTN_ERR_INVALID_ARG, "these shots carry no probabilities");
    if (r->n > 0)
        PTN_CUDA(cudaMemcpyAsync(prob_out, r->prob, sizeof(double) * r->n, cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
    return PTN_OK;
}

void ptn_shots_destroy(ptn_shots* r) {
    if (!r) return;
    cudaFree(r->traj);
    cudaFree(r->bits);
    cudaFree(r->count);
    cudaFree(r->prob);
    delete r;
}

}  // extern "C"
