// Host planner: unified-path-variation networks, one contraction path per
// qubit block, lowered to batched pairwise contraction steps.
//
// Paper, Sec. III-A (UPV): every sampled error operator is merged into the
// gate it follows, so all error sets share the error-free network's structure
// and one path set P^j (one path per qubit block B_j) serves every error set
// and every shot.  Here the merge is precomputed for every combination of
// Kraus choices of a gate's sites ("variants"); executing a trajectory's
// network then only selects variants.
//
// Paper, Sec. II-B / III-B: the network of block j measures the block's qubits
// (open outputs), projects the earlier qubits onto the sampled prefix and
// traces the later ones.  It is built as a double layer <psi| . |psi>: the bra
// layer is the mirror image of the ket layer with conjugated tensors.
//
// Paper, Sec. IV-C: paths come from a randomised search with 100
// hypersamples.  The search here is a randomised greedy over pairwise
// contractions whose objective counts every step's work times the number of
// copies the batch needs: once per trajectory for tensors built from gates
// only, once per network (trajectory, prefix) for tensors that depend on
// projected prefix bits.  Projected bits are carried as open "slice" indices
// until a slice move fixes them from each network's prefix, so work shared by
// all prefixes of a trajectory is done once per trajectory.  Work on the ket
// layer is mirrored on the bra layer for free (its result is the complex
// conjugate), so mirrored pairs are contracted in lockstep.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <array>
#include <functional>
#include <map>
#include <thread>
#include <queue>
#include <random>
#include <unordered_map>

#include "ptn_internal.h"

namespace ptn {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors --
static thread_local std::string g_last_error;

ptn_status set_error(ptn_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}
const char* last_error_text() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

// --------------------------------------------------- small linear algebra --
using M2 = std::array<cd, 4>;    // row-major 2x2
using M4 = std::array<cd, 16>;   // row-major 4x4

static M2 mul2(const M2& a, const M2& b) {
    M2 r;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) r[i * 2 + j] = a[i * 2] * b[j] + a[i * 2 + 1] * b[2 + j];
    return r;
}
static M2 eye2() { return M2{cd(1), cd(0), cd(0), cd(1)}; }

// q_k = Tr(K^dagger K) / d (d = 2, or 4 for a two-qubit channel) with the
// entries summed as re*re + im*im in row-major order (a fixed order so every
// implementation gets the same bits).
static double kraus_prob(const double* k, int d = 2) {
    double acc = 0.0;
    for (int e = 0; e < d * d; e++) {
        double re = k[2 * e], im = k[2 * e + 1];
        double sq = re * re;
        sq = sq + im * im;
        acc = acc + sq;
    }
    return acc / (double)d;
}

// One-sided (Hestenes) Jacobi SVD of a complex 4x4 matrix X = sum_r u_r s_r v_r^H.
// Returns singular values (descending) with X*V columns and V.
static void svd4(const M4& x_in, double s[4], cd xv[4][4], cd v[4][4]) {
    cd x[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            x[i][j] = x_in[i * 4 + j];
            v[i][j] = (i == j) ? cd(1) : cd(0);
        }
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int p = 0; p < 3; p++)
            for (int q = p + 1; q < 4; q++) {
                double a = 0, b = 0;
                cd g = 0;
                for (int i = 0; i < 4; i++) {
                    a += std::norm(x[i][p]);
                    b += std::norm(x[i][q]);
                    g += std::conj(x[i][p]) * x[i][q];
                }
                double ag = std::abs(g);
                if (ag <= 1e-300 || ag <= 1e-16 * std::sqrt(a * b)) continue;
                off = std::max(off, ag / std::sqrt(a * b + 1e-300));
                cd ph = g / ag;   // rotate column q by conj(phase) to make <p,q> real
                double zeta = (b - a) / (2.0 * ag);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < 4; i++) {
                    cd xp = x[i][p], xq = x[i][q] * std::conj(ph);
                    x[i][p] = c * xp - sn * xq;
                    x[i][q] = sn * xp + c * xq;
                    cd vp = v[i][p], vq = v[i][q] * std::conj(ph);
                    v[i][p] = c * vp - sn * vq;
                    v[i][q] = sn * vp + c * vq;
                }
            }
        if (off < 1e-15) break;
    }
    int order[4] = {0, 1, 2, 3};
    double nrm[4];
    for (int j = 0; j < 4; j++) {
        double a = 0;
        for (int i = 0; i < 4; i++) a += std::norm(x[i][j]);
        nrm[j] = std::sqrt(a);
    }
    std::sort(order, order + 4, [&](int a, int b) { return nrm[a] > nrm[b]; });
    cd x2[4][4], v2[4][4];
    for (int j = 0; j < 4; j++) {
        s[j] = nrm[order[j]];
        for (int i = 0; i < 4; i++) {
            x2[i][j] = x[i][order[j]];
            v2[i][j] = v[i][order[j]];
        }
    }
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            xv[i][j] = x2[i][j];
            v[i][j] = v2[i][j];
        }
}

// ------------------------------------------------------------- leaf roles --
enum Role : int32_t { R_IN_A = 0, R_OUT_A = 1, R_IN_B = 2, R_OUT_B = 3, R_BOND = 4 };

// --------------------------------------------------------------- network --
// IX_REST: a later qubit of the ket-only sampling form, open in the ket network
// and summed only after |.|^2 (the closing step of the block)
enum IdxKind : int32_t { IX_INT = 0, IX_OPEN = 1, IX_TRACED = 2, IX_SLICE = 3, IX_REST = 4 };

struct NetIdx {
    int32_t kind;
    int32_t qubit;     // end indices and slices
    int32_t mirror;    // id on the other layer (itself for open / traced)
};

struct BlockNet {
    std::vector<NetIdx> idx;
    std::vector<std::vector<int32_t>> tidx;   // per tensor: index ids in leaf storage order
    std::vector<int32_t> tleaf;               // per tensor: leaf id
    std::vector<int32_t> tbra;                // per tensor: 1 for the bra layer
    std::vector<int32_t> tcls;
    int32_t n_leaf_tensors = 0;               // ket tensors; bra tensor i + n is the mirror of i
    bool ket_only = false;                    // no bra layer (the trajectory state itself)
};

// ------------------------------------------------------------ path search --
struct GT {
    std::vector<int32_t> idx;   // sorted index ids
    int32_t cls;
    int32_t side;               // 0 ket, 1 bra, 2 mixed
    int32_t mirror;             // live mirror partner or -1
    int32_t nslice;
    bool alive;
};

enum MoveType : int32_t { MV_CONTRACT = 0, MV_SLICE = 1 };
struct Move {
    int32_t type;
    int32_t a, b, c;            // operands and result (b = -1 for a slice)
    int32_t ma, mb, mc;         // lockstep mirror operands / result, -1 if none
};

struct CostModel {
    double mult[3];              // CONST, TRAJ, NET copies
    double tc_rate = 1.0e14;     // tensor-core steps, real flops/s (8 per complex MAC), FP32-accurate split
    double simt_rate = 2.5e12;   // SIMT contraction kernel, real flops/s
    double bw = 3.0e12;          // effective bytes/s of the memory-bound kernels
    double launch = 3.0e-6;      // per launch
    bool allow_tc = true;
};

struct Searcher {
    const BlockNet* net;
    const CostModel* cm;
    std::vector<GT> t;
    std::vector<std::vector<int32_t>> occ;   // index id -> live tensors holding it
    std::vector<Move> moves;
    double time = 0, macs[3] = {0, 0, 0}, bytes[3] = {0, 0, 0};
    int64_t max_rank = 0;
    int64_t max_sum = 0;     // most summed bits of a step, counted as the lowering counts them

    Searcher(const BlockNet& n, const CostModel& c) : net(&n), cm(&c) {}

    bool is_slice(int32_t i) const { return net->idx[i].kind == IX_SLICE; }
    bool is_open(int32_t i) const { return net->idx[i].kind == IX_OPEN || net->idx[i].kind == IX_REST; }

    void init() {
        t.clear();
        occ.assign(net->idx.size(), {});
        moves.clear();
        time = 0;
        for (int k = 0; k < 3; k++) macs[k] = bytes[k] = 0;
        max_rank = 0;
        max_sum = 0;
        int nl = net->n_leaf_tensors;
        for (size_t i = 0; i < net->tidx.size(); i++) {
            GT g;
            g.idx = net->tidx[i];
            std::sort(g.idx.begin(), g.idx.end());
            g.cls = net->tcls[i];
            g.side = net->tbra[i];
            g.mirror = net->ket_only ? -1 : (int32_t)((i < (size_t)nl) ? i + nl : i - nl);
            g.nslice = 0;
            for (int32_t x : g.idx) g.nslice += is_slice(x);
            g.alive = true;
            t.push_back(g);
            for (int32_t x : g.idx) occ[x].push_back((int32_t)i);
        }
    }

    // Result of contracting a and b (without applying it).
    void result(int32_t a, int32_t b, std::vector<int32_t>& out, int32_t& nsum, int32_t& cls,
                int32_t& nslice) const {
        const GT &A = t[a], &B = t[b];
        cls = std::max(A.cls, B.cls);
        out.clear();
        nsum = 0;
        nslice = 0;
        size_t i = 0, j = 0;
        auto keep = [&](int32_t x) {
            if (is_slice(x)) {
                if (cls == CLS_NET) return;   // fixed from the network's prefix
                nslice++;
            }
            out.push_back(x);
        };
        while (i < A.idx.size() || j < B.idx.size()) {
            if (j == B.idx.size() || (i < A.idx.size() && A.idx[i] < B.idx[j])) {
                keep(A.idx[i++]);
            } else if (i == A.idx.size() || B.idx[j] < A.idx[i]) {
                keep(B.idx[j++]);
            } else {
                int32_t x = A.idx[i];
                if (!is_open(x) && occ[x].size() == 2) nsum++;
                else keep(x);
                i++;
                j++;
            }
        }
    }

    double size_of(const GT& g, bool sliced) const {
        return std::ldexp(1.0, (int)g.idx.size() - (sliced ? g.nslice : 0));
    }

    // Cost of one step (count once for a lockstep mirror pair).
    // Modelled cost of one step on the kernel it will run on (the same
    // eligibility rules as classify_step): tensor-core GEMMs pay their MACs at
    // the tensor rate plus the operand packing traffic; other steps run on the
    // SIMT kernel.  A trajectory-level operand of a network step is read once
    // per trajectory.
    void account(int32_t cls, const std::vector<int32_t>& out, int32_t nsum, const GT& A, const GT& B) {
        const int64_t rank_out = (int64_t)out.size();
        const double m = cm->mult[cls];
        const double mac = std::ldexp(1.0, (int)(rank_out + nsum));
        double by = 8.0 * std::ldexp(1.0, (int)rank_out) * m;
        by += 8.0 * size_of(A, false) * cm->mult[A.cls];
        by += 8.0 * size_of(B, false) * cm->mult[B.cls];
        macs[cls] += mac * m;
        bytes[cls] += by;
        int fr[2] = {0, 0}, nh = 0;
        for (int32_t x : out) {
            const bool ia = std::binary_search(A.idx.begin(), A.idx.end(), x);
            const bool ib = std::binary_search(B.idx.begin(), B.idx.end(), x);
            if (ia && ib) nh++;
            else if (ia) fr[0]++;
            else fr[1]++;
        }
        auto pcls = [&](const GT& g) { return (cls == CLS_NET && g.cls != CLS_NET && g.nslice > 0) ? (int)CLS_NET : (int)g.cls; };
        const GT* op[2] = {&A, &B};
        int kind = 0, ra = 0;
        if (cm->allow_tc && nsum >= 3) {
            if (cls == CLS_NET && nh == 0)
                for (int a = 0; a < 2 && !kind; a++)
                    if (pcls(*op[a]) == CLS_NET && pcls(*op[1 - a]) != CLS_NET && fr[a] < 7 && fr[1 - a] >= 6 && fr[a] <= 16) {
                        kind = 2;
                        ra = a;
                    }
            if (!kind) {
                ra = fr[0] >= fr[1] ? 0 : 1;
                if (fr[ra] >= 7 && fr[1 - ra] >= 6 && nh <= 20) kind = 1;
            }
        }
        double t;
        const double flops = 8.0 * mac * m;
        if (kind) {
            const double kh = std::ceil(2.0 * std::ldexp(1.0, nsum) / 32.0) * 32.0;
            const double hh = std::ldexp(1.0, nh);
            const double fa = hh * std::ldexp(1.0, fr[ra]) * 2 * kh * cm->mult[pcls(*op[ra])];
            const double fb = hh * std::ldexp(2.0, fr[1 - ra]) * 2 * kh * cm->mult[pcls(*op[1 - ra])];
            const double pack_bytes = 4.0 * 2.0 * (fa + fb) + 8.0 * (size_of(A, false) * cm->mult[A.cls] + size_of(B, false) * cm->mult[B.cls]);
            t = flops / cm->tc_rate + (pack_bytes + 8.0 * std::ldexp(1.0, (int)rank_out) * m) / cm->bw + 3 * cm->launch;
        } else {
            t = std::max(flops / cm->simt_rate, by / cm->bw) + cm->launch;
        }
        time += t;
        max_rank = std::max<int64_t>(max_rank, rank_out);
    }

    int32_t add_tensor(GT&& g) {
        int32_t id = (int32_t)t.size();
        for (int32_t x : g.idx) occ[x].push_back(id);
        t.push_back(std::move(g));
        return id;
    }
    void kill(int32_t a) {
        t[a].alive = false;
        for (int32_t x : t[a].idx) {
            auto& v = occ[x];
            v.erase(std::find(v.begin(), v.end(), a));
        }
        if (t[a].mirror >= 0 && t[t[a].mirror].mirror == a) t[t[a].mirror].mirror = -1;
    }

    int32_t do_contract(int32_t a, int32_t b, bool count) {
        std::vector<int32_t> out;
        int32_t nsum, cls, nslice;
        result(a, b, out, nsum, cls, nslice);
        {
            // a prefix-projected index the two share is fixed per network, not
            // summed, when the step is lowered
            int32_t fixed = 0;
            const GT &A = t[a], &B = t[b];
            for (size_t i = 0, j = 0; i < A.idx.size() && j < B.idx.size();) {
                if (A.idx[i] < B.idx[j]) i++;
                else if (B.idx[j] < A.idx[i]) j++;
                else {
                    const int32_t x = A.idx[i];
                    if (is_slice(x) && occ[x].size() == 2) fixed++;
                    i++;
                    j++;
                }
            }
            max_sum = std::max<int64_t>(max_sum, nsum - fixed);
        }
        if (count) account(cls, out, nsum, t[a], t[b]);
        GT g;
        g.idx = std::move(out);
        g.cls = cls;
        g.side = (t[a].side == t[b].side) ? t[a].side : 2;
        g.mirror = -1;
        g.nslice = nslice;
        g.alive = true;
        int32_t keep_ma = t[a].mirror, keep_mb = t[b].mirror;
        (void)keep_ma;
        (void)keep_mb;
        kill(a);
        kill(b);
        return add_tensor(std::move(g));
    }

    int32_t do_slice(int32_t a, bool count) {
        GT g;
        for (int32_t x : t[a].idx)
            if (!is_slice(x)) g.idx.push_back(x);
        g.cls = CLS_NET;
        g.side = t[a].side;
        g.mirror = -1;
        g.nslice = 0;
        g.alive = true;
        (void)count;   // a slice is a view: no work
        kill(a);
        return add_tensor(std::move(g));
    }

    bool lockstep_pair(int32_t a, int32_t b) const {
        const GT &A = t[a], &B = t[b];
        return A.side == 0 && B.side == 0 && A.mirror >= 0 && B.mirror >= 0 &&
               t[A.mirror].alive && t[B.mirror].alive;
    }
    bool skip_pair(int32_t a, int32_t b) const {   // bra-side twin of a lockstep ket pair
        const GT &A = t[a], &B = t[b];
        return A.side == 1 && B.side == 1 && A.mirror >= 0 && B.mirror >= 0;
    }

    // Apply a contraction, with its mirror when in lockstep; returns result id.
    int32_t apply_contract(int32_t a, int32_t b) {
        Move mv{MV_CONTRACT, a, b, -1, -1, -1, -1};
        if (lockstep_pair(a, b)) {
            int32_t ma = t[a].mirror, mb = t[b].mirror;
            int32_t c = do_contract(a, b, true);
            int32_t mc = do_contract(ma, mb, false);
            t[c].mirror = mc;
            t[mc].mirror = c;
            mv.c = c;
            mv.ma = ma;
            mv.mb = mb;
            mv.mc = mc;
        } else {
            mv.c = do_contract(a, b, true);
        }
        moves.push_back(mv);
        return mv.c;
    }
    int32_t apply_slice(int32_t a) {
        Move mv{MV_SLICE, a, -1, -1, -1, -1, -1};
        int32_t m = t[a].mirror;
        bool lock = t[a].side == 0 && m >= 0 && t[m].alive && t[m].cls == CLS_TRAJ && t[m].nslice > 0;
        mv.c = do_slice(a, true);
        if (lock) {
            mv.ma = m;
            mv.mc = do_slice(m, false);
            t[mv.c].mirror = mv.mc;
            t[mv.mc].mirror = mv.c;
        }
        moves.push_back(mv);
        return mv.c;
    }

    struct Cand {
        double score;
        int32_t a, b;   // b = -1: slice move
        bool operator<(const Cand& o) const { return score > o.score; }   // min-heap
    };

    double pair_score(int32_t a, int32_t b, double costmod) const {
        std::vector<int32_t> out;
        int32_t nsum, cls, nslice;
        result(a, b, out, nsum, cls, nslice);
        double so = std::ldexp(1.0, (int)out.size()) * cm->mult[cls];
        double sa = size_of(t[a], false) * cm->mult[t[a].cls];
        double sb = size_of(t[b], false) * cm->mult[t[b].cls];
        return so - costmod * (sa + sb);
    }
    double slice_score(int32_t a, double costmod) const {
        double so = size_of(t[a], true) * cm->mult[CLS_NET];
        double sa = size_of(t[a], false) * cm->mult[t[a].cls];
        return so - costmod * sa;
    }

    void run(double temperature, double costmod, std::mt19937_64& rng) {
        init();
        std::priority_queue<Cand> heap;
        std::uniform_real_distribution<double> U(1e-12, 1.0);
        auto noisy = [&](double s) {
            double v = (s >= 0 ? 1.0 : -1.0) * std::log1p(std::fabs(s));
            if (temperature > 0) v -= temperature * (-std::log(-std::log(U(rng))));
            return v;
        };
        auto push_pairs = [&](int32_t a) {
            if (!t[a].alive) return;
            std::vector<int32_t> nb;
            for (int32_t x : t[a].idx)
                for (int32_t o : occ[x])
                    if (o != a) nb.push_back(o);
            std::sort(nb.begin(), nb.end());
            nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
            for (int32_t o : nb) {
                if (skip_pair(a, o)) continue;
                heap.push({noisy(pair_score(a, o, costmod)), std::min(a, o), std::max(a, o)});
            }
            if (t[a].cls == CLS_TRAJ && t[a].nslice > 0 && cm->mult[CLS_NET] > 0 &&
                !(t[a].side == 1 && t[a].mirror >= 0))
                heap.push({noisy(slice_score(a, costmod)), a, -1});
        };
        for (size_t i = 0; i < t.size(); i++) push_pairs((int32_t)i);
        while (!heap.empty()) {
            Cand c = heap.top();
            heap.pop();
            if (!t[c.a].alive || (c.b >= 0 && !t[c.b].alive)) continue;
            if (c.b >= 0 && skip_pair(c.a, c.b)) continue;
            if (c.b < 0 && !(t[c.a].cls == CLS_TRAJ && t[c.a].nslice > 0)) continue;
            int32_t r;
            if (c.b < 0) {
                int32_t m = t[c.a].mirror;
                r = apply_slice(c.a);
                push_pairs(r);
                if (t[r].mirror >= 0) push_pairs(t[r].mirror);
                (void)m;
            } else {
                r = apply_contract(c.a, c.b);
                push_pairs(r);
                if (t[r].mirror >= 0) push_pairs(t[r].mirror);
            }
        }
        // disconnected remainder: outer products, smallest first
        for (;;) {
            std::vector<int32_t> live;
            for (size_t i = 0; i < t.size(); i++)
                if (t[i].alive) live.push_back((int32_t)i);
            if (live.size() <= 1) break;
            std::sort(live.begin(), live.end(), [&](int32_t x, int32_t y) {
                return size_of(t[x], false) * cm->mult[t[x].cls] < size_of(t[y], false) * cm->mult[t[y].cls];
            });
            apply_contract(live[0], live[1]);
        }
        // the root must hold no unresolved slice index
        for (size_t i = 0; i < t.size(); i++)
            if (t[i].alive && t[i].cls == CLS_TRAJ && t[i].nslice > 0) apply_slice((int32_t)i);
    }

    int32_t root() const {
        for (size_t i = 0; i < t.size(); i++)
            if (t[i].alive) return (int32_t)i;
        return -1;
    }
};

// -------------------------------------------------------------- lowering --
struct TRef {
    int32_t mode;               // OP_LEAF / OP_BUF
    int32_t id;                 // leaf id / buffer id
    int32_t conj;
    int32_t cls;                // storage class
    std::vector<int32_t> layout;   // index ids, position = log2(stride)
};

struct ArenaAlloc {   // first-fit offsets of live buffers in one arena
    std::vector<std::pair<int64_t, int64_t>> live;   // (offset, size)
    int64_t peak = 0;
    int64_t alloc(int64_t size) {
        std::sort(live.begin(), live.end());
        int64_t off = 0;
        for (auto& b : live) {
            if (b.first - off >= size) break;
            off = std::max(off, b.first + b.second);
        }
        live.push_back({off, size});
        peak = std::max(peak, off + size);
        return off;
    }
    void release(int64_t off) {
        for (size_t i = 0; i < live.size(); i++)
            if (live[i].first == off) {
                live.erase(live.begin() + i);
                return;
            }
    }
};

// Set fuse_prev on the steps of a list that may join the fused launch of the
// step before them: a run is a maximal sequence of small steps, cut wherever a
// step's output range overlaps, without coinciding with it, a range of the
// same arena read or written earlier in the run, or one of its operands
// overlaps, without coinciding, an output written earlier in the run.  A
// coinciding range holds the same instance at the same addresses, which only
// the CTA of that instance touches, in order.
static void mark_fusable_runs(std::vector<StepDesc>& steps) {
    struct Rng {
        int32_t arena;
        int64_t off, size;
        bool wrote;
    };
    std::vector<Rng> touched;
    auto clash = [&](const Rng& r, bool writes) {
        for (const Rng& t : touched) {
            if (t.arena != r.arena || (!writes && !t.wrote)) continue;
            const bool same = t.off == r.off && t.size == r.size;
            if (!same && t.off < r.off + r.size && r.off < t.off + t.size) return true;
        }
        return false;
    };
    for (size_t i = 0; i < steps.size(); i++) {
        StepDesc& st = steps[i];
        st.fuse_prev = 0;
        if (!small_step(st)) {
            touched.clear();
            continue;
        }
        const Rng out{st.out_arena, st.out_off, st.out_size, true};
        std::vector<Rng> ins;
        for (const OperandDesc& d : st.op)
            if (d.mode == OP_BUF) ins.push_back({d.arena, d.arena_off, d.inst_size, false});
        bool join = i > 0 && small_step(steps[i - 1]) && !clash(out, true);
        for (const Rng& r : ins) join = join && !clash(r, false);
        if (!join) touched.clear();
        st.fuse_prev = join ? 1 : 0;
        touched.insert(touched.end(), ins.begin(), ins.end());
        touched.push_back(out);
    }
}

// Intermediate caching across error sets (Sec. VI).  A trajectory-class
// step's output depends only on the variants its subtree's leaves take, i.e.
// on the trajectory's entries in the variant columns of those leaves, so all
// trajectories that agree on these columns share one output.  Walking the
// steps in order, a step's column set is the union of its operands' sets: a
// leaf contributes its own column, a buffer the set of the step that wrote it
// (found by its arena address, which no other live buffer shares).  A
// trajectory-class step outside the fused runs of small steps (a CTA of a run
// computes every step of the run for its own trajectory) with at least kCacheMinWork
// multiply-adds and 2^kCacheMinOutBits outputs per instance (a SIMT tile of
// 128 outputs then lies within one instance) gets a cache slot and its column
// bitmap; every later read of its buffer, the root's included, records the slot.
constexpr double kCacheMinWork = 4096.0;
constexpr int kCacheMinOutBits = 7;
static void assign_cache(const ptn_plan* plan, BlockPlan& bp) {
    const int words = (plan->n_var_cols + 31) / 32;
    using Bits = std::vector<uint32_t>;
    std::map<std::pair<int32_t, int64_t>, std::pair<Bits, int32_t>> written;   // (arena, offset) -> (columns, cache)
    bp.n_cache = 0;
    bp.cache_words = words;
    bp.cache_bits.clear();
    auto read = [&](OperandDesc& d, Bits& acc) {
        d.cache = 0;
        if (d.mode == OP_LEAF) {
            if (d.leaf_col >= 0) acc[d.leaf_col >> 5] |= 1u << (d.leaf_col & 31);
            return;
        }
        auto it = written.find({d.arena, d.arena_off});
        if (it == written.end()) return;
        if (d.cls == CLS_TRAJ) d.cache = it->second.second;
        for (int w = 0; w < words; w++) acc[w] |= it->second.first[w];
    };
    for (size_t i = 0; i < bp.steps.size(); i++) {
        StepDesc& st = bp.steps[i];
        Bits acc(words, 0u);
        for (OperandDesc& d : st.op) read(d, acc);
        st.cache = 0;
        const bool varies = std::any_of(acc.begin(), acc.end(), [](uint32_t w) { return w != 0; });
        // a small step joins a fused run if it is marked fuse_prev or the next one
        // is (fuse_max = 1: every step is launched on its own)
        const bool fused = plan->opts.fuse_max > 1 && small_step(st) &&
                           (st.fuse_prev || (i + 1 < bp.steps.size() && bp.steps[i + 1].fuse_prev));
        if (st.out_cls == CLS_TRAJ && st.kind != STEP_GEMM_STACKED && !fused && varies &&
            st.n_out >= kCacheMinOutBits && std::ldexp(1.0, st.n_out + st.n_sum) >= kCacheMinWork) {
            st.cache = ++bp.n_cache;
            bp.cache_bits.insert(bp.cache_bits.end(), acc.begin(), acc.end());
        }
        written[{st.out_arena, st.out_off}] = {std::move(acc), st.cache};
    }
    Bits root(words, 0u);
    read(bp.root.op, root);
}

// Outer products formed in the operand pack.  A direct step P with no summed
// bits writes out[o] = f0[a0(o)] f1[a1(o)]; when its only reader is an operand
// X of a tensor-core step G, G's pack can form each element of X from the two
// factors instead of reading P's output, and P is not launched.  X reads P's
// dense output bit by bit (stride 2^p for bit p), so every stride of X maps to
// one stride per factor.  Conditions: P outside the fused runs, X without
// projected bits, factors of at most 2^31 elements per instance (the pack keeps
// both 32-bit offsets in one 64-bit word), and no step between P and G writing
// into an arena range of either factor (their buffers were released after P).
static void mark_pack_products(BlockPlan& bp, int fuse_max) {
    const size_t n = bp.steps.size();
    std::map<std::pair<int32_t, int64_t>, size_t> writer;
    std::vector<std::array<int64_t, 2>> prod_of(n, {-1, -1});   // producer of each operand
    for (size_t i = 0; i < n; i++) {
        StepDesc& st = bp.steps[i];
        st.virt = st.prod = st.prod_src = 0;
        for (int x = 0; x < 2; x++) {
            const OperandDesc& d = st.op[x];
            if (d.mode != OP_BUF) continue;
            auto it = writer.find({d.arena, d.arena_off});
            if (it != writer.end()) prod_of[i][x] = (int64_t)it->second;
        }
        writer[{st.out_arena, st.out_off}] = i;
    }
    for (size_t g = 0; g < n; g++) {
        StepDesc& G = bp.steps[g];
        if (G.kind == STEP_DIRECT) continue;
        for (int x = 0; x < 2 && !G.prod; x++) {
            if (prod_of[g][x] < 0 || G.op[x].n_slice) continue;
            const size_t k = (size_t)prod_of[g][x];
            StepDesc& P = bp.steps[k];
            const bool fused = fuse_max > 1 && small_step(P) && (P.fuse_prev || (k + 1 < n && bp.steps[k + 1].fuse_prev));
            if (P.kind != STEP_DIRECT || P.n_sum != 0 || P.virt || fused) continue;
            if (P.op[0].inst_size > (1ll << 31) || P.op[1].inst_size > (1ll << 31)) continue;
            bool clash = false;
            for (size_t s = k + 1; s < g && !clash; s++) {
                const StepDesc& S = bp.steps[s];
                for (const OperandDesc& f : P.op)
                    if (f.mode == OP_BUF && f.arena == S.out_arena && f.arena_off < S.out_off + S.out_size &&
                        S.out_off < f.arena_off + f.inst_size)
                        clash = true;
            }
            if (clash) continue;
            P.virt = 1;
            G.prod = 1 + x;
            G.prod_src = (int32_t)k;
        }
    }
}

// Lower a searched path to step descriptors.  expval: the network is the ket
// state with every qubit open; the forward intermediates are kept (all of
// them, or with checkpointing those crossing a segment boundary) and the
// reversed (adjoint) path is lowered too, see the end.
static ptn_status lower_block(const ptn_plan* plan, const BlockNet& net, const Searcher& s,
                              int32_t start, int32_t b, BlockPlan& bp, bool expval = false) {
    struct Rec {
        TRef a, b, c;
    };
    std::vector<Rec> recs;
    const auto& idx = net.idx;
    std::vector<TRef> ref(s.t.size());
    int nl = net.n_leaf_tensors;
    for (size_t i = 0; i < net.tidx.size(); i++) {
        const LeafInfo& L = plan->leaves[net.tleaf[i]];
        TRef r;
        r.mode = OP_LEAF;
        r.id = net.tleaf[i];
        r.conj = net.tbra[i];
        r.cls = L.n_var > 1 ? CLS_TRAJ : CLS_CONST;
        r.layout = net.tidx[i];
        ref[i] = r;
    }
    (void)nl;
    struct BufInfo {
        int32_t arena;
        int64_t off;
        int32_t refs;
    };
    std::vector<BufInfo> bufs;
    ArenaAlloc arenas[3];
    auto pos_in = [](const std::vector<int32_t>& lay, int32_t x) -> int {
        for (size_t p = 0; p < lay.size(); p++)
            if (lay[p] == x) return (int)p;
        return -1;
    };
    auto make_op = [&](const TRef& r, int32_t step_cls, OperandDesc& d) -> ptn_status {
        memset(&d, 0, sizeof d);
        d.mode = r.mode;
        d.cls = r.cls;
        d.conj = r.conj;
        d.inst_size = (int64_t)1 << r.layout.size();
        if (r.mode == OP_LEAF) {
            const LeafInfo& L = plan->leaves[r.id];
            d.leaf_base = L.var_base;
            d.leaf_col = L.var_col;
            d.arena = -1;
        } else {
            d.arena = bufs[r.id].arena;
            d.arena_off = bufs[r.id].off;
            d.leaf_col = -1;
        }
        d.n_slice = 0;
        if (step_cls == CLS_NET && r.cls != CLS_NET) {
            for (size_t p = 0; p < r.layout.size(); p++) {
                const NetIdx& x = idx[r.layout[p]];
                if (x.kind != IX_SLICE) continue;
                if (d.n_slice >= kMaxSlice)
                    return set_error(PTN_ERR_UNSUPPORTED, "too many projected bits on one operand");
                d.slice_qubit[d.n_slice] = x.qubit;
                d.slice_stride[d.n_slice] = (int64_t)1 << p;
                d.n_slice++;
            }
        }
        return PTN_OK;
    };
    // Gradient plans keep every forward intermediate, or with checkpointing only
    // those that cross a segment boundary of the step list (segments of about
    // sqrt(steps) steps); the others are recomputed segment by segment on the
    // reversed path.
    const bool ckpt = expval && plan->opts.grad_checkpoint;
    // segments by produced size: with T elements produced in all and tensors of
    // at most m elements, segments of about sqrt(T m) elements keep about
    // 2 sqrt(T m) elements live instead of T
    std::vector<int32_t> step_seg;
    {
        std::vector<double> sz;
        for (const Move& mv : s.moves)
            if (mv.type == MV_CONTRACT) sz.push_back(std::ldexp(1.0, (int)s.t[mv.c].idx.size()));
        double tot = 0, mx = 1;
        for (double v : sz) tot += v, mx = std::max(mx, v);
        const double seg = std::max(mx, std::sqrt(tot * mx));
        double cum = 0;
        for (double v : sz) {
            step_seg.push_back((int32_t)(cum / seg));
            cum += v;
        }
    }
    int cur_step = 0;
    std::vector<int32_t> buf_step;   // producing step of every buffer
    // Inside a run of small steps (one fused launch, one CTA per trajectory)
    // a released slot is not reused before the run ends: the slot's other
    // instances may still be read by other CTAs (mark_fusable_runs).
    bool in_run = false;
    std::vector<std::pair<int32_t, int64_t>> deferred;
    auto release = [&](int32_t arena, int64_t off) {
        if (in_run) deferred.push_back({arena, off});
        else arenas[arena].release(off);
    };
    auto end_run = [&]() {
        for (const auto& d : deferred) arenas[d.first].release(d.second);
        deferred.clear();
        in_run = false;
    };
    auto consume = [&](const TRef& r) {
        if (r.mode != OP_BUF) return;
        BufInfo& bi = bufs[r.id];
        if (--bi.refs != 0) return;
        if (!expval) {
            release(bi.arena, bi.off);
            return;
        }
        if (ckpt && step_seg[buf_step[r.id]] == step_seg[cur_step]) release(bi.arena, bi.off);
    };

    int32_t root_id = s.root();
    // find the move that produces the root (or the tensor the root is a slice of)
    int32_t root_src = root_id;
    for (auto it = s.moves.rbegin(); it != s.moves.rend(); ++it)
        if (it->c == root_src && it->type == MV_SLICE) root_src = it->a;

    // The contraction that consumes every tensor (through slice views), and the
    // bits it sums.  A producer writes those bits innermost, in increasing id
    // order of the consumer's view, and every step lists its summed bits in
    // increasing id order: the consumer then reads its operands' summed bits
    // contiguously (coalesced packing for tensor-core steps).
    std::vector<int32_t> cons(s.t.size(), -1);
    for (size_t i = 0; i < s.moves.size(); i++) {
        const Move& mv = s.moves[i];
        if (mv.type != MV_CONTRACT) continue;
        cons[mv.a] = cons[mv.b] = (int32_t)i;
    }
    for (auto it = s.moves.rbegin(); it != s.moves.rend(); ++it) {
        if (it->type != MV_SLICE) continue;
        cons[it->a] = cons[it->c];
        if (it->ma >= 0) cons[it->ma] = cons[it->mc];
    }
    auto summed_by = [&](int32_t k) {
        std::vector<int32_t> S;
        const Move& m = s.moves[k];
        const auto &ia = s.t[m.a].idx, &ib = s.t[m.b].idx, &ic = s.t[m.c].idx;
        for (int32_t x : ia)
            if (std::binary_search(ib.begin(), ib.end(), x) && !std::binary_search(ic.begin(), ic.end(), x) &&
                idx[x].kind != IX_SLICE)
                S.push_back(x);
        return S;   // sorted (ia is sorted)
    };

    std::string summary;
    for (const Move& mv : s.moves) {
        if (mv.type == MV_SLICE) {
            ref[mv.c] = ref[mv.a];       // a view: same storage, NET addressing when consumed
            if (mv.mc >= 0) ref[mv.mc] = ref[mv.ma];
            continue;
        }
        const GT& C = s.t[mv.c];
        const TRef& A = ref[mv.a];
        const TRef& B = ref[mv.b];
        StepDesc st;
        memset(&st, 0, sizeof st);
        st.out_cls = C.cls;
        // output layout: A's kept bits in A's order, then B's
        std::vector<int32_t> out;
        auto keep_from = [&](const TRef& r) {
            for (int32_t x : r.layout)
                if (std::binary_search(C.idx.begin(), C.idx.end(), x) &&
                    std::find(out.begin(), out.end(), x) == out.end())
                    out.push_back(x);
        };
        if (mv.c == root_src) {
            // canonical: open bits by qubit (block bit t = qubit start + t), then the rest
            std::vector<int32_t> open, rest;
            for (int32_t x : C.idx) (idx[x].kind == IX_OPEN ? open : rest).push_back(x);
            std::sort(open.begin(), open.end(), [&](int32_t u, int32_t v) { return idx[u].qubit < idx[v].qubit; });
            out = open;
            out.insert(out.end(), rest.begin(), rest.end());
        } else {
            std::vector<int32_t> lead;
            if (cons[mv.c] >= 0) {
                lead = summed_by(cons[mv.c]);
            } else if (mv.mc >= 0 && cons[mv.mc] >= 0) {
                for (int32_t x : summed_by(cons[mv.mc])) lead.push_back(idx[x].mirror);
            }
            for (int32_t x : lead)
                if (std::binary_search(C.idx.begin(), C.idx.end(), x) && std::find(out.begin(), out.end(), x) == out.end())
                    out.push_back(x);
            keep_from(A);
            keep_from(B);
        }
        if (out.size() != C.idx.size())
            return set_error(PTN_ERR_INVALID_ARG, "internal: output layout mismatch");
        if ((int)out.size() > kMaxOut)
            return set_error(PTN_ERR_TOO_LARGE, "a contraction step has %d output bits (max %d)",
                             (int)out.size(), kMaxOut);
        // summed bits: in both operands' layouts, not in the output, not a slice
        std::vector<int32_t> sum;
        for (int32_t x : A.layout)
            if (pos_in(B.layout, x) >= 0 && pos_in(out, x) < 0 && idx[x].kind != IX_SLICE) sum.push_back(x);
        std::sort(sum.begin(), sum.end());
        if ((int)sum.size() > kMaxSum)
            return set_error(PTN_ERR_TOO_LARGE, "a contraction step sums %d bits (max %d)",
                             (int)sum.size(), kMaxSum);
        st.n_out = (int32_t)out.size();
        st.n_sum = (int32_t)sum.size();
        st.out_size = (int64_t)1 << out.size();
        ptn_status e = make_op(A, C.cls, st.op[0]);
        if (e) return e;
        e = make_op(B, C.cls, st.op[1]);
        if (e) return e;
        const TRef* ops[2] = {&A, &B};
        for (int o = 0; o < 2; o++) {
            for (size_t p = 0; p < out.size(); p++) {
                int q = pos_in(ops[o]->layout, out[p]);
                st.out_stride[o][p] = q >= 0 ? ((int64_t)1 << q) : 0;
            }
            for (size_t p = 0; p < sum.size(); p++) {
                int q = pos_in(ops[o]->layout, sum[p]);
                st.sum_stride[o][p] = (int64_t)1 << q;
            }
        }
        int64_t pf[2][3];
        classify_step(st, pf, !plan->opts.simt_only);
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) bp.pack_peak[r][k] = std::max(bp.pack_peak[r][k], pf[r][k]);
        if (!small_step(st)) end_run();
        // output buffer: allocate before releasing the operands
        BufInfo bi;
        bi.arena = C.cls;
        bi.off = arenas[C.cls].alloc(st.out_size);
        in_run = small_step(st);
        bi.refs = mv.mc >= 0 ? 2 : 1;
        int32_t bid = (int32_t)bufs.size();
        bufs.push_back(bi);
        buf_step.push_back(cur_step);
        st.out_arena = C.cls;
        st.out_off = bi.off;
        consume(A);
        consume(B);
        if (mv.ma >= 0) {
            consume(ref[mv.ma]);
            consume(ref[mv.mb]);
        }
        TRef rc;
        rc.mode = OP_BUF;
        rc.id = bid;
        rc.conj = 0;
        rc.cls = C.cls;
        rc.layout = out;
        ref[mv.c] = rc;
        if (mv.mc >= 0) {
            TRef rm = rc;
            rm.conj = 1;
            for (auto& x : rm.layout) x = idx[x].mirror;
            ref[mv.mc] = rm;
        }
        bp.steps.push_back(st);
        if (expval) recs.push_back({A, B, rc});
        cur_step++;
    }
    // root descriptor
    TRef R = ref[root_id];
    if (R.mode != OP_BUF) return set_error(PTN_ERR_UNSUPPORTED, "degenerate block network");
    if (net.ket_only && !expval) {
        // Ket-only form: the network's result is the amplitude a(x, rest) of the
        // block bits and the later qubits; the closing step forms the marginal
        // sum_rest a(x, rest) conj(a(x, rest)) (real; the finalisation reads its
        // real part), one pairwise contraction of the tensor with its conjugate.
        std::vector<int32_t> xs, rs;
        bool sliced = false;
        for (int32_t x : R.layout) {
            const int32_t k = idx[x].kind;
            if (k == IX_OPEN) xs.push_back(x);
            else if (k == IX_REST) rs.push_back(x);
            else if (k == IX_SLICE) sliced = true;
            else return set_error(PTN_ERR_INVALID_ARG, "internal: unexpected bit in a ket-only root");
        }
        std::sort(xs.begin(), xs.end(), [&](int32_t u, int32_t v) { return idx[u].qubit < idx[v].qubit; });
        if ((int)rs.size() > kMaxSum)
            return set_error(PTN_ERR_TOO_LARGE, "ket-only block sums %d later qubits (max %d)", (int)rs.size(), kMaxSum);
        const int32_t cls = (R.cls == CLS_NET || sliced) ? (int32_t)CLS_NET : R.cls;
        StepDesc st;
        memset(&st, 0, sizeof st);
        st.out_cls = cls;
        st.n_out = (int32_t)xs.size();
        st.n_sum = (int32_t)rs.size();
        st.out_size = (int64_t)1 << xs.size();
        TRef Rc = R;
        Rc.conj = 1;
        ptn_status e0 = make_op(R, cls, st.op[0]);
        if (e0) return e0;
        e0 = make_op(Rc, cls, st.op[1]);
        if (e0) return e0;
        for (size_t p = 0; p < xs.size(); p++)
            st.out_stride[0][p] = st.out_stride[1][p] = (int64_t)1 << pos_in(R.layout, xs[p]);
        for (size_t q = 0; q < rs.size(); q++)
            st.sum_stride[0][q] = st.sum_stride[1][q] = (int64_t)1 << pos_in(R.layout, rs[q]);
        int64_t pf[2][3];
        classify_step(st, pf, !plan->opts.simt_only);
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) bp.pack_peak[r][k] = std::max(bp.pack_peak[r][k], pf[r][k]);
        if (!small_step(st)) end_run();
        BufInfo bi;
        bi.arena = cls;
        bi.off = arenas[cls].alloc(st.out_size);
        in_run = small_step(st);
        bi.refs = 1;
        const int32_t bid = (int32_t)bufs.size();
        bufs.push_back(bi);
        buf_step.push_back(cur_step);
        st.out_arena = cls;
        st.out_off = bi.off;
        consume(R);
        bp.steps.push_back(st);
        cur_step++;
        {   // modelled cost of the closing step (the search did not see it)
            const double inst = cls == CLS_NET ? bp.est_mult_net : bp.est_mult_traj;
            const double macs = std::ldexp(1.0, st.n_out + st.n_sum) * inst;
            bp.est_macs[cls] += macs;
            bp.est_time += std::max(8.0 * macs / 2.5e12, 8.0 * (2.0 * std::ldexp(1.0, st.n_out + st.n_sum) +
                                                              std::ldexp(1.0, st.n_out)) * inst / 3.0e12);
        }
        TRef rn;
        rn.mode = OP_BUF;
        rn.id = bid;
        rn.conj = 0;
        rn.cls = cls;
        rn.layout = xs;
        R = rn;
    }
    end_run();
    mark_fusable_runs(bp.steps);
    ptn_status e = make_op(R, CLS_NET, bp.root.op);
    if (e) return e;
    for (int tb = 0; tb < b; tb++) bp.root.x_stride[tb] = -1;
    for (size_t p = 0; p < R.layout.size(); p++) {
        const NetIdx& x = idx[R.layout[p]];
        if (x.kind == IX_OPEN) bp.root.x_stride[x.qubit - start] = (int64_t)1 << p;
    }
    for (int tb = 0; tb < b; tb++)
        if (bp.root.x_stride[tb] < 0) return set_error(PTN_ERR_INVALID_ARG, "internal: root misses an open bit");
    for (int k = 0; k < 3; k++) bp.arena_peak[k] = arenas[k].peak;
    if (!expval) {
        if (plan->opts.cache_intermediates) assign_cache(plan, bp);
        if (!plan->opts.keep_products) mark_pack_products(bp, plan->opts.fuse_max);
        return PTN_OK;
    }

    // ---- reversed path (reverse-mode differentiation of the contraction tree).
    // The ket network is holomorphic in its tensors, so for a step
    // C = sum_k A B the adjoint of A is  G_A = sum_n G_C B  over the bits of C
    // that come from B alone (again a pairwise contraction, written in A's
    // layout), and likewise for B.  Only tensors that contain a parametrised
    // gate get adjoints; a parametrised leaf's adjoint goes to its own slot.
    auto leaf_param = [&](const TRef& r) {
        return r.mode == OP_LEAF && plan->leaves[r.id].param_kind != PTN_PARAM_NONE;
    };
    std::vector<char> buf_need(bufs.size(), 0);
    auto need = [&](const TRef& r) { return r.mode == OP_LEAF ? leaf_param(r) : buf_need[r.id] != 0; };
    for (auto& rc : recs) buf_need[rc.c.id] = need(rc.a) || need(rc.b);
    ArenaAlloc adj, lg;
    std::vector<int64_t> adj_off(bufs.size(), -1);
    adj_off[R.id] = adj.alloc((int64_t)1 << R.layout.size());
    bp.root_adj_off = adj_off[R.id];
    std::unordered_map<int32_t, int64_t> leaf_slot;
    for (auto& rc : recs)
        for (const TRef* x : {&rc.a, &rc.b})
            if (leaf_param(*x) && !leaf_slot.count(x->id)) {
                const LeafInfo& L = plan->leaves[x->id];
                ParamLeaf p;
                p.leaf = x->id;
                p.param_index = L.param_index;
                p.param_kind = L.param_kind;
                p.var_col = L.var_col;
                p.size = L.size;
                p.n_var = L.n_var;
                p.lgrad_off = lg.alloc(L.size);
                p.dvt_base = bp.dvt_size;
                bp.dvt_size += L.n_var * L.size;
                bp.pleaves.push_back(p);
                leaf_slot[x->id] = p.lgrad_off;
            }
    // which forward outputs stayed allocated (the others get recomputed)
    std::vector<char> kept(bufs.size(), 1);
    if (ckpt) {
        std::vector<int32_t> last_use(bufs.size(), -1);
        for (size_t t = 0; t < recs.size(); t++)
            for (const TRef* x : {&recs[t].a, &recs[t].b})
                if (x->mode == OP_BUF) last_use[x->id] = (int32_t)t;
        for (size_t i = 0; i < bufs.size(); i++)
            kept[i] = (int32_t)i == R.id || last_use[i] < 0 || step_seg[buf_step[i]] != step_seg[last_use[i]];
    }
    std::vector<std::pair<int32_t, int64_t>> recomputed;   // (arena, offset) of this segment's recomputed buffers
    int cur_seg = -1;
    for (auto it = recs.rbegin(); it != recs.rend(); ++it) {
        const TRef& C = it->c;
        const int t = (int)(recs.rend() - it) - 1;
        if (ckpt && step_seg[t] != cur_seg) {
            // leave the previous segment: free its recomputed buffers; enter this
            // one: replay its forward steps whose outputs were not kept
            for (const auto& ro : recomputed) arenas[ro.first].release(ro.second);
            recomputed.clear();
            cur_seg = step_seg[t];
            int t0 = t;
            while (t0 > 0 && step_seg[t0 - 1] == cur_seg) t0--;
            for (int u = t0; u <= t; u++) {
                const int32_t id = recs[u].c.id;
                if (kept[id]) continue;
                StepDesc st = bp.steps[u];
                const int32_t cls = bufs[id].arena;
                bufs[id].off = arenas[cls].alloc(st.out_size);
                recomputed.push_back({cls, bufs[id].off});
                ptn_status ee = make_op(recs[u].a, st.out_cls, st.op[0]);
                if (ee) return ee;
                ee = make_op(recs[u].b, st.out_cls, st.op[1]);
                if (ee) return ee;
                st.out_off = bufs[id].off;
                bp.bwd.push_back(st);
            }
        }
        if (!buf_need[C.id]) continue;
        for (int side = 0; side < 2; side++) {
            const TRef& X = side ? it->b : it->a;
            const TRef& Y = side ? it->a : it->b;
            if (!need(X)) continue;
            StepDesc st;
            memset(&st, 0, sizeof st);
            st.out_cls = CLS_TRAJ;
            const std::vector<int32_t>& out = X.layout;
            std::vector<int32_t> sum;
            for (int32_t x : C.layout)
                if (pos_in(Y.layout, x) >= 0 && pos_in(out, x) < 0) sum.push_back(x);
            std::sort(sum.begin(), sum.end());
            for (int32_t x : out)
                if (pos_in(C.layout, x) < 0 && pos_in(Y.layout, x) < 0)
                    return set_error(PTN_ERR_INVALID_ARG, "internal: adjoint output bit not reachable");
            if ((int)out.size() > kMaxOut || (int)sum.size() > kMaxSum)
                return set_error(PTN_ERR_TOO_LARGE, "an adjoint step exceeds the kernel limits");
            st.n_out = (int32_t)out.size();
            st.n_sum = (int32_t)sum.size();
            st.out_size = (int64_t)1 << out.size();
            OperandDesc& g = st.op[0];
            g.mode = OP_BUF;
            g.cls = CLS_TRAJ;
            g.conj = 0;
            g.arena = ARENA_ADJ;
            g.inst_size = (int64_t)1 << C.layout.size();
            g.arena_off = adj_off[C.id];
            g.leaf_col = -1;
            g.n_slice = 0;
            ptn_status ee = make_op(Y, CLS_TRAJ, st.op[1]);
            if (ee) return ee;
            for (size_t p = 0; p < out.size(); p++) {
                const int qc = pos_in(C.layout, out[p]), qy = pos_in(Y.layout, out[p]);
                st.out_stride[0][p] = qc >= 0 ? ((int64_t)1 << qc) : 0;
                st.out_stride[1][p] = qy >= 0 ? ((int64_t)1 << qy) : 0;
            }
            for (size_t p = 0; p < sum.size(); p++) {
                st.sum_stride[0][p] = (int64_t)1 << pos_in(C.layout, sum[p]);
                st.sum_stride[1][p] = (int64_t)1 << pos_in(Y.layout, sum[p]);
            }
            if (X.mode == OP_BUF) {
                adj_off[X.id] = adj.alloc(st.out_size);
                st.out_arena = ARENA_ADJ;
                st.out_off = adj_off[X.id];
            } else {
                st.out_arena = ARENA_LGRAD;
                st.out_off = leaf_slot[X.id];
            }
            int64_t pf[2][3];
            classify_step(st, pf, !plan->opts.simt_only);
            for (int r = 0; r < 2; r++)
                for (int k = 0; k < 3; k++) bp.pack_peak[r][k] = std::max(bp.pack_peak[r][k], pf[r][k]);
            bp.bwd.push_back(st);
        }
        adj.release(adj_off[C.id]);
    }
    mark_fusable_runs(bp.bwd);
    bp.arena_peak[ARENA_ADJ] = adj.peak;
    bp.arena_peak[ARENA_LGRAD] = lg.peak;
    for (int k = 0; k < 3; k++) bp.arena_peak[k] = arenas[k].peak;   // recomputed buffers included
    return PTN_OK;
}

// Choose the kernel of a step.  Tensor cores (tcgen05) when the step is a
// real matrix product worth a 128-row tile:
//  - STEP_GEMM: both free sides fill tiles (realified B counts twice) and the
//    contraction is deep enough; one GEMM per (instance, hyper index);
//  - STEP_GEMM_STACKED: a network-level step whose network operand has few
//    rows per network while the other operand is shared by all networks of a
//    trajectory: the rows of all networks of a trajectory are stacked into one
//    GEMM against the trajectory's operand;
// else the direct SIMT kernel.  pack_floats[r][c]: floats per instance of
// class c that packing operand r (0 = GEMM rows, 1 = realified) needs.
void classify_step(StepDesc& st, int64_t pack_floats[2][3], bool allow_tc) {
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++) pack_floats[r][k] = 0;
    st.kind = STEP_DIRECT;
    st.gemm_a = 0;
    if (!allow_tc) return;
    int free_[2] = {0, 0}, nh = 0;
    for (int p = 0; p < st.n_out; p++) {
        const bool i0 = st.out_stride[0][p] != 0, i1 = st.out_stride[1][p] != 0;
        if (i0 && i1) nh++;
        else if (i0) free_[0]++;
        else free_[1]++;
    }
    auto pcls = [&](const OperandDesc& d) {
        if (st.out_cls == CLS_NET && d.n_slice) return (int)CLS_NET;
        if (d.mode == OP_LEAF) return d.leaf_col >= 0 ? (int)CLS_TRAJ : (int)CLS_CONST;
        return (int)d.cls;
    };
    const int64_t kc = (int64_t)1 << st.n_sum;
    const int64_t kh = ((2 * kc + 31) / 32) * 32;
    if (st.n_sum < 3) return;
    // stacked: network operand (rows) x trajectory-level operand (realified)
    if (st.out_cls == CLS_NET && nh == 0) {
        for (int a = 0; a < 2; a++) {
            const int b = 1 - a;
            if (pcls(st.op[a]) != CLS_NET || pcls(st.op[b]) == CLS_NET) continue;
            if (free_[a] >= 7 || free_[b] < 6 || free_[a] > 16) continue;
            st.kind = STEP_GEMM_STACKED;
            st.gemm_a = a;
            pack_floats[0][CLS_NET] = ((int64_t)1 << free_[a]) * 2 * kh;
            pack_floats[0][CLS_CONST] = 128 * 2 * kh;   // one full tile of rows for small chunks
            pack_floats[1][pcls(st.op[b])] = ((int64_t)2 << free_[b]) * 2 * kh;
            return;
        }
    }
    const int a = free_[0] >= free_[1] ? 0 : 1, b = 1 - a;
    if (free_[a] < 7 || free_[b] < 6 || nh > 20) return;
    st.kind = STEP_GEMM;
    st.gemm_a = a;
    pack_floats[0][pcls(st.op[a])] = ((int64_t)1 << nh) * ((int64_t)1 << free_[a]) * 2 * kh;
    pack_floats[1][pcls(st.op[b])] = ((int64_t)1 << nh) * ((int64_t)2 << free_[b]) * 2 * kh;
}

// ------------------------------------------------------ block networks --
// The ket layer in circuit order; end indices per block: prefix qubits
// projected (slice), block qubits open, later qubits traced.  ket_only: no
// bra layer, every qubit open (start = 0, b = n): the trajectory state.
static void build_block_net(const ptn_plan* plan, int n, int start, int b, bool ket_only, BlockNet& net) {
    std::vector<int32_t> cur(n, -1);
    auto new_idx = [&](int32_t kind, int32_t q) {
        net.idx.push_back({kind, q, -1});
        return (int32_t)net.idx.size() - 1;
    };
    std::vector<std::vector<int32_t>> ket_idx;
    std::vector<int32_t> ket_leaf;
    int32_t bond = -1;
    for (size_t li = 0; li < plan->leaves.size(); li++) {
        const LeafInfo& L = plan->leaves[li];
        std::vector<int32_t> ids;
        int qa = L.qubit0, qb = L.qubit1;
        int qA = (L.part == 2) ? qb : qa;   // the factor's own qubit
        if (L.part == 1) bond = -1;
        int32_t in_a = cur[qA], in_b = (L.part == 0 && L.qubit1 >= 0) ? cur[qb] : -1;
        int32_t out_a = new_idx(IX_INT, qA), out_b = (L.part == 0 && L.qubit1 >= 0) ? new_idx(IX_INT, qb) : -1;
        for (int32_t role : L.legs) {
            switch (role) {
                case R_IN_A: ids.push_back(in_a); break;
                case R_OUT_A: ids.push_back(out_a); break;
                case R_IN_B: ids.push_back(in_b); break;
                case R_OUT_B: ids.push_back(out_b); break;
                case R_BOND:
                    if (bond < 0) bond = new_idx(IX_INT, -1);
                    ids.push_back(bond);
                    break;
            }
        }
        cur[qA] = out_a;
        if (out_b >= 0) cur[qb] = out_b;
        ket_idx.push_back(ids);
        ket_leaf.push_back((int32_t)li);
    }
    for (int q = 0; q < n; q++) {
        NetIdx& x = net.idx[cur[q]];
        x.qubit = q;
        x.kind = q < start ? IX_SLICE : (q < start + b ? IX_OPEN : (ket_only ? IX_REST : IX_TRACED));
    }
    int nl = (int)ket_idx.size();
    net.n_leaf_tensors = nl;
    net.ket_only = ket_only;
    if (!ket_only) {
        size_t n_ket_idx = net.idx.size();
        for (size_t i = 0; i < n_ket_idx; i++) {
            NetIdx& x = net.idx[i];
            if (x.kind == IX_OPEN || x.kind == IX_TRACED) {
                x.mirror = (int32_t)i;
            } else {
                NetIdx m{x.kind, x.qubit, (int32_t)i};
                net.idx.push_back(m);
                net.idx[i].mirror = (int32_t)net.idx.size() - 1;
            }
        }
    }
    for (int side = 0; side < (ket_only ? 1 : 2); side++)
        for (int i = 0; i < nl; i++) {
            std::vector<int32_t> ids = ket_idx[i];
            if (side)
                for (auto& x : ids) x = net.idx[x].mirror;
            net.tidx.push_back(ids);
            net.tleaf.push_back(ket_leaf[i]);
            net.tbra.push_back(side);
            net.tcls.push_back(plan->leaves[ket_leaf[i]].n_var > 1 ? CLS_TRAJ : CLS_CONST);
        }
}

// Randomised greedy path search (hypersamples) under the step-cost model, then
// lowering of the best path.
static ptn_status search_and_lower(ptn_plan* plan, BlockNet& net, int j, int start, int b, double E, double D,
                                   std::mt19937_64& rng, BlockPlan& bp, bool expval) {
    const ptn_plan_opts& opts = plan->opts;
    CostModel cm;
    cm.mult[CLS_CONST] = 1.0;
    cm.mult[CLS_TRAJ] = E;
    cm.mult[CLS_NET] = D;
    cm.allow_tc = !opts.simt_only;
    Searcher best(net, cm), cur_s(net, cm);
    double best_time = INFINITY;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    if (opts.search_threads <= 0) {
        // one random stream for all restarts, in order
        for (int h = 0; h < opts.hypersamples; h++) {
            double temp = h == 0 ? 0.0 : 0.02 + 1.0 * U(rng);
            double costmod = h == 0 ? 1.0 : 0.5 + 1.5 * U(rng);
            cur_s.run(temp, costmod, rng);
            if (cur_s.root() < 0) continue;
            if (cur_s.max_rank > kMaxOut || cur_s.max_sum > kMaxSum) continue;
            if (cur_s.time < best_time) {
                best_time = cur_s.time;
                best = cur_s;
            }
        }
    } else {
        // restart h draws from its own stream (seeded from one draw of the plan's
        // stream and h); the best restart, ties to the lowest h, does not depend
        // on how the restarts are spread over the threads
        const uint64_t base = rng();
        const int T = std::max(1, std::min(opts.search_threads, opts.hypersamples));
        std::vector<Searcher> wbest(T, Searcher(net, cm));
        std::vector<double> wtime(T, INFINITY);
        std::vector<int> wh(T, -1);
        std::vector<int> wfail(T, 0);
        auto work = [&](int w) {
            try {
                Searcher cur(net, cm);
                for (int h = w; h < opts.hypersamples; h += T) {
                    uint64_t z = base + 0x9E3779B97F4A7C15ull * (uint64_t)(h + 1);   // splitmix64 step
                    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
                    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
                    std::mt19937_64 r(z ^ (z >> 31));
                    std::uniform_real_distribution<double> Uw(0.0, 1.0);
                    const double temp = h == 0 ? 0.0 : 0.02 + 1.0 * Uw(r);
                    const double costmod = h == 0 ? 1.0 : 0.5 + 1.5 * Uw(r);
                    cur.run(temp, costmod, r);
                    if (cur.root() < 0 || cur.max_rank > kMaxOut || cur.max_sum > kMaxSum) continue;
                    if (cur.time < wtime[w]) {   // h increases within a thread: ties keep the lower h
                        wtime[w] = cur.time;
                        wh[w] = h;
                        wbest[w] = cur;
                    }
                }
            } catch (...) {
                wfail[w] = 1;
            }
        };
        std::vector<std::thread> pool;
        for (int w = 1; w < T; w++) pool.emplace_back(work, w);
        work(0);
        for (auto& t : pool) t.join();
        int pick = -1;
        for (int w = 0; w < T; w++) {
            if (wfail[w]) return set_error(PTN_ERR_OOM, "block %d: path search thread failed", j);
            if (wh[w] < 0) continue;
            if (pick < 0 || wtime[w] < wtime[pick] || (wtime[w] == wtime[pick] && wh[w] < wh[pick])) pick = w;
        }
        if (pick >= 0) {
            best_time = wtime[pick];
            best = wbest[pick];
        }
    }
    if (!std::isfinite(best_time))
        return set_error(PTN_ERR_TOO_LARGE, "block %d: no path with at most %d open and %d summed bits per step", j,
                         kMaxOut, kMaxSum);
    bp.start = start;
    bp.b = b;
    for (int k = 0; k < 3; k++) {
        bp.est_macs[k] = best.macs[k];
        bp.est_bytes[k] = best.bytes[k];
    }
    bp.est_time = best.time;
    bp.est_mult_traj = E;
    bp.est_mult_net = D;
    ptn_status e = lower_block(plan, net, best, start, b, bp, expval);
    if (e) return e;
    char buf[256];
    snprintf(buf, sizeof buf, "steps=%zu max_rank=%lld est_time=%.3es", bp.steps.size(), (long long)best.max_rank,
             best.time);
    bp.path_summary = buf;
    return PTN_OK;
}

ptn_status build_expval_plan(ptn_plan* plan) {
    if (plan->expval) return PTN_OK;
    if (plan->n_qubits > 24) return set_error(PTN_ERR_UNSUPPORTED, "expectation values need n_qubits <= 24");
    BlockNet net;
    build_block_net(plan, plan->n_qubits, 0, plan->n_qubits, true, net);
    std::mt19937_64 rng(plan->opts.seed ^ 0xA5A5A5A5A5A5A5A5ull);
    BlockPlan* bp = new BlockPlan();
    ptn_status e = search_and_lower(plan, net, -1, 0, plan->n_qubits, plan->opts.est_traj, plan->opts.est_traj, rng,
                                    *bp, true);
    if (e) {
        delete bp;
        return e;
    }
    plan->expval = bp;
    return PTN_OK;
}

// N G(theta) and N dG/dtheta for every variant of a parametrised leaf, in the
// leaf's storage order (legs); RY(t) = exp(-i t Y / 2), RZ(t) = exp(-i t Z / 2).
void param_leaf_tables(const LeafInfo& L, double theta, float* out, float* out_d) {
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    M2 G, dG;
    if (L.param_kind == PTN_PARAM_RY) {
        G = M2{cd(c), cd(-s), cd(s), cd(c)};
        dG = M2{cd(-s / 2), cd(-c / 2), cd(c / 2), cd(-s / 2)};
    } else {
        const cd e0 = std::exp(cd(0, -theta / 2)), e1 = std::exp(cd(0, theta / 2));
        G = M2{e0, cd(0), cd(0), e1};
        dG = M2{cd(0, -0.5) * e0, cd(0), cd(0), cd(0, 0.5) * e1};
    }
    for (int64_t v = 0; v < L.n_var; v++) {
        M2 N;
        for (int e = 0; e < 4; e++) N[e] = cd(L.noise_ops[8 * v + 2 * e], L.noise_ops[8 * v + 2 * e + 1]);
        const M2 NG = mul2(N, G), NdG = mul2(N, dG);
        for (int64_t el = 0; el < L.size; el++) {
            int32_t rb[5] = {0, 0, 0, 0, 0};
            for (size_t p = 0; p < L.legs.size(); p++) rb[L.legs[p]] = (int32_t)((el >> p) & 1);
            const int k = rb[R_OUT_A] * 2 + rb[R_IN_A];
            const int64_t o = 2 * (v * L.size + el);
            out[o] = (float)NG[k].real();
            out[o + 1] = (float)NG[k].imag();
            out_d[o] = (float)NdG[k].real();
            out_d[o + 1] = (float)NdG[k].imag();
        }
    }
}

// ------------------------------------------------------------ build plan --
static void cd_from(const double* p, cd* out, int n) {
    for (int i = 0; i < n; i++) out[i] = cd(p[2 * i], p[2 * i + 1]);
}

ptn_status build_plan(const ptn_circuit* c, const ptn_noise* nz, const int32_t* block_sizes,
                      int32_t n_blocks, const ptn_plan_opts* o, ptn_plan* plan) {
    auto t0 = std::chrono::steady_clock::now();
    if (!c || !c->gates || c->n_qubits < 1 || c->n_qubits > kMaxQubits || c->n_gates < 0)
        return set_error(PTN_ERR_INVALID_ARG, "invalid circuit");
    const int n = c->n_qubits;
    plan->n_qubits = n;
    ptn_plan_opts opts{};
    if (o) opts = *o;
    if (opts.hypersamples <= 0) opts.hypersamples = 100;
    if (opts.est_traj <= 0) opts.est_traj = 1024;
    if (opts.est_shots <= 0) opts.est_shots = 1e6;
    if (opts.network_form < 0 || opts.network_form > 2)
        return set_error(PTN_ERR_INVALID_ARG, "network_form must be 0, 1 or 2");
    if (opts.fuse_max < 0) return set_error(PTN_ERR_INVALID_ARG, "fuse_max must be >= 0");
    if (opts.fuse_max == 0) opts.fuse_max = 1024;
    if (opts.cache_intermediates < 0 || opts.cache_intermediates > 1)
        return set_error(PTN_ERR_INVALID_ARG, "cache_intermediates must be 0 or 1");
    if (opts.keep_products < 0 || opts.keep_products > 1)
        return set_error(PTN_ERR_INVALID_ARG, "keep_products must be 0 or 1");
    if (opts.search_threads < 0 || opts.search_threads > 1024)
        return set_error(PTN_ERR_INVALID_ARG, "search_threads must be in 0..1024");
    plan->opts = opts;
    plan->mem_cap = opts.mem_cap_bytes;

    // ---- validate gates and noise
    for (int l = 0; l < c->n_gates; l++) {
        const ptn_gate& g = c->gates[l];
        if (g.arity != 1 && g.arity != 2) return set_error(PTN_ERR_INVALID_ARG, "gate %d: arity %d", l, g.arity);
        if (g.q0 < 0 || g.q0 >= n || (g.arity == 2 && (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)))
            return set_error(PTN_ERR_INVALID_ARG, "gate %d: bad qubits", l);
    }
    int n_sites = nz ? nz->n_sites : 0;
    int n_ch = nz ? nz->n_channels : 0;
    plan->n_sites = n_sites;
    auto ch_dim = [&](int k) { return nz->channels[k].n_qubits == 2 ? 4 : 2; };
    for (int k = 0; k < n_ch; k++) {
        const ptn_channel& ch = nz->channels[k];
        if (ch.n_kraus < 1 || ch.n_kraus > kMaxKraus || !ch.kraus)
            return set_error(PTN_ERR_INVALID_ARG, "channel %d: n_kraus %d", k, ch.n_kraus);
        if (ch.n_qubits < 0 || ch.n_qubits > 2)
            return set_error(PTN_ERR_INVALID_ARG, "channel %d: n_qubits %d", k, ch.n_qubits);
        const int d = ch_dim(k);
        std::vector<cd> s(d * d, cd(0)), m(d * d);
        for (int a = 0; a < ch.n_kraus; a++) {
            cd_from(ch.kraus + 2 * d * d * a, m.data(), d * d);
            for (int i = 0; i < d; i++)
                for (int j = 0; j < d; j++)
                    for (int r = 0; r < d; r++) s[i * d + j] += std::conj(m[r * d + i]) * m[r * d + j];
        }
        double err = 0.0;
        for (int i = 0; i < d; i++)
            for (int j = 0; j < d; j++) err = std::max(err, std::abs(s[i * d + j] - (i == j ? 1.0 : 0.0)));
        if (err > 1e-10) return set_error(PTN_ERR_NOT_CPTP, "channel %d: |sum K^dag K - I| = %.3g", k, err);
    }
    int prev_gate = -1;
    for (int s = 0; s < n_sites; s++) {
        const ptn_site& st = nz->sites[s];
        if (st.gate < 0 || st.gate >= c->n_gates || st.channel < 0 || st.channel >= n_ch)
            return set_error(PTN_ERR_INVALID_ARG, "site %d: bad gate or channel", s);
        const ptn_gate& g = c->gates[st.gate];
        if (ch_dim(st.channel) == 4) {
            if (g.arity != 2 || st.qubit != -1)
                return set_error(PTN_ERR_INVALID_ARG, "site %d: a two-qubit channel needs a two-qubit gate and qubit -1",
                                 s);
        } else if (st.qubit != g.q0 && !(g.arity == 2 && st.qubit == g.q1)) {
            return set_error(PTN_ERR_INVALID_ARG, "site %d: qubit not on its gate", s);
        }
        if (st.gate < prev_gate) return set_error(PTN_ERR_INVALID_ARG, "sites must be grouped by gate in order");
        prev_gate = st.gate;
    }

    // ---- site tables (Kraus CDF and log q)
    plan->site_tables.assign(n_sites, SiteTable{});
    std::vector<std::vector<double>> qtab(n_ch);
    for (int k = 0; k < n_ch; k++) {
        const ptn_channel& ch = nz->channels[k];
        const int d = ch_dim(k);
        for (int a = 0; a < ch.n_kraus; a++) qtab[k].push_back(kraus_prob(ch.kraus + 2 * d * d * a, d));
    }
    for (int s = 0; s < n_sites; s++) {
        SiteTable& T = plan->site_tables[s];
        const auto& q = qtab[nz->sites[s].channel];
        T.n_kraus = (int32_t)q.size();
        double acc = 0.0;
        for (int a = 0; a < kMaxKraus; a++) {
            if (a < T.n_kraus) {
                acc = acc + q[a];
                T.cdf[a] = acc;
                T.logq[a] = q[a] > 0 ? std::log(q[a]) : -INFINITY;
            } else {
                T.cdf[a] = 2.0;
                T.logq[a] = 0.0;
            }
        }
        T.cdf[T.n_kraus - 1] = 1.0;
    }
    std::vector<std::vector<int32_t>> gsites(c->n_gates);
    for (int s = 0; s < n_sites; s++) gsites[nz->sites[s].gate].push_back(s);

    // scaled Kraus operator K_k / sqrt(q_k) of a site
    auto scaled_kraus = [&](int s, int k) {
        const ptn_channel& ch = nz->channels[nz->sites[s].channel];
        cd m[4];
        cd_from(ch.kraus + 8 * k, m, 4);
        double q = qtab[nz->sites[s].channel][k];
        double sc = q > 0 ? 1.0 / std::sqrt(q) : 0.0;
        M2 r;
        for (int i = 0; i < 4; i++) r[i] = m[i] * sc;
        return r;
    };

    // scaled operator of site s as a 4x4 on its two-qubit gate's (a, b) = (q0, q1)
    // (a one-qubit operator embedded on its qubit, a the high bit)
    auto scaled_kraus4 = [&](int s, int k, const ptn_gate& g) {
        const ptn_site& st = nz->sites[s];
        const ptn_channel& ch = nz->channels[st.channel];
        double q = qtab[st.channel][k];
        double sc = q > 0 ? 1.0 / std::sqrt(q) : 0.0;
        M4 r{};
        if (ch_dim(st.channel) == 4) {
            cd m[16];
            cd_from(ch.kraus + 32 * k, m, 16);
            for (int i = 0; i < 16; i++) r[i] = m[i] * sc;
        } else {
            const M2 N = scaled_kraus(s, k);
            const bool on_a = st.qubit == g.q0;
            for (int oa = 0; oa < 2; oa++)
                for (int ob = 0; ob < 2; ob++)
                    for (int ia = 0; ia < 2; ia++)
                        for (int ib = 0; ib < 2; ib++) {
                            cd v = on_a ? (ob == ib ? N[oa * 2 + ia] : cd(0)) : (oa == ia ? N[ob * 2 + ib] : cd(0));
                            r[(oa * 2 + ob) * 4 + ia * 2 + ib] = v;
                        }
        }
        return r;
    };
    auto mul4 = [](const M4& a, const M4& b) {
        M4 r{};
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) {
                cd z = 0;
                for (int k = 0; k < 4; k++) z += a[i * 4 + k] * b[k * 4 + j];
                r[i * 4 + j] = z;
            }
        return r;
    };

    // ---- leaves and their variant tables
    std::vector<bool> touched(n, false);
    plan->leaves.clear();
    std::vector<float>& vt = plan->var_table;
    vt.clear();
    auto finish_leaf = [&](LeafInfo& L, const std::function<cd(int64_t var, const int32_t* role_bits)>& val) {
        L.size = (int64_t)1 << L.legs.size();
        L.n_var = 1;
        for (int32_t r : L.radix) L.n_var *= r;
        L.var_base = (int64_t)vt.size() / 2;
        for (int64_t v = 0; v < L.n_var; v++)
            for (int64_t e = 0; e < L.size; e++) {
                int32_t rb[5] = {0, 0, 0, 0, 0};
                for (size_t p = 0; p < L.legs.size(); p++) rb[L.legs[p]] = (int32_t)((e >> p) & 1);
                cd z = val(v, rb);
                vt.push_back((float)z.real());
                vt.push_back((float)z.imag());
            }
        L.var_col = L.n_var > 1 ? plan->n_var_cols++ : -1;
        plan->leaves.push_back(L);
    };
    // decode the Kraus choices of a variant and build N_q for one qubit
    auto noise_op = [&](const LeafInfo& L, int64_t var, int qubit) {
        M2 N = eye2();
        int64_t v = var;
        for (size_t i = 0; i < L.sites.size(); i++) {
            int k = (int)(v % L.radix[i]);
            v /= L.radix[i];
            if (nz->sites[L.sites[i]].qubit == qubit) N = mul2(scaled_kraus(L.sites[i], k), N);
        }
        return N;
    };
    plan->n_var_cols = 0;
    for (int l = 0; l < c->n_gates; l++) {
        const ptn_gate& g = c->gates[l];
        if (g.arity == 1) {
            LeafInfo L;
            L.gate = l;
            L.part = 0;
            L.qubit0 = g.q0;
            L.qubit1 = -1;
            for (int32_t s : gsites[l]) {
                L.sites.push_back(s);
                L.radix.push_back((int32_t)qtab[nz->sites[s].channel].size());
            }
            bool fixed = !touched[g.q0];
            touched[g.q0] = true;
            if (!fixed) L.legs.push_back(R_IN_A);
            L.legs.push_back(R_OUT_A);
            if (g.param_kind == PTN_PARAM_RY || g.param_kind == PTN_PARAM_RZ) {
                if (g.param_index < 0) return set_error(PTN_ERR_INVALID_ARG, "gate %d: parametrised without index", l);
                L.param_kind = g.param_kind;
                L.param_index = g.param_index;
                plan->n_params = std::max(plan->n_params, g.param_index + 1);
                int64_t nv = 1;
                for (int32_t r : L.radix) nv *= r;
                for (int64_t v = 0; v < nv; v++) {
                    M2 N = noise_op(L, v, g.q0);
                    for (int e = 0; e < 4; e++) {
                        L.noise_ops.push_back(N[e].real());
                        L.noise_ops.push_back(N[e].imag());
                    }
                }
            }
            M2 M;
            cd_from(g.mat, M.data(), 4);
            finish_leaf(L, [&](int64_t v, const int32_t* rb) {
                M2 NM = mul2(noise_op(L, v, g.q0), M);
                return NM[rb[R_OUT_A] * 2 + rb[R_IN_A]];
            });
        } else {
            M4 M;
            cd_from(g.mat, M.data(), 16);
            bool fa = !touched[g.q0], fb = !touched[g.q1];
            touched[g.q0] = touched[g.q1] = true;
            // operator-Schmidt rank: X[(oa ia)][(ob ib)] = M[(oa ob)][(ia ib)]
            M4 X;
            for (int oa = 0; oa < 2; oa++)
                for (int ob = 0; ob < 2; ob++)
                    for (int ia = 0; ia < 2; ia++)
                        for (int ib = 0; ib < 2; ib++)
                            X[(oa * 2 + ia) * 4 + ob * 2 + ib] = M[(oa * 2 + ob) * 4 + ia * 2 + ib];
            double sv[4];
            cd xv[4][4], vv[4][4];
            svd4(X, sv, xv, vv);
            int rank = 0;
            for (int r = 0; r < 4; r++)
                if (sv[r] > 1e-12 * std::max(sv[0], 1e-300)) rank++;
            bool two_qubit_noise = false;
            for (int32_t s2 : gsites[l]) two_qubit_noise |= ch_dim(nz->sites[s2].channel) == 4;
            if (opts.split_gates && rank <= 2 && !two_qubit_noise) {
                int bond_bits = rank == 2 ? 1 : 0;
                // left factor A_r[oa][ia] = (X V)[(oa ia), r] / sqrt(s_r); right B_r[ob][ib] = sqrt(s_r) conj(V[(ob ib), r])
                for (int part = 1; part <= 2; part++) {
                    LeafInfo L;
                    L.gate = l;
                    L.part = part;
                    L.qubit0 = g.q0;
                    L.qubit1 = g.q1;
                    int q = part == 1 ? g.q0 : g.q1;
                    for (int32_t s : gsites[l])
                        if (nz->sites[s].qubit == q) {
                            L.sites.push_back(s);
                            L.radix.push_back((int32_t)qtab[nz->sites[s].channel].size());
                        }
                    bool fixed = part == 1 ? fa : fb;
                    if (!fixed) L.legs.push_back(R_IN_A);
                    L.legs.push_back(R_OUT_A);
                    if (bond_bits) L.legs.push_back(R_BOND);
                    finish_leaf(L, [&, part, q](int64_t v, const int32_t* rb) {
                        int r = rb[R_BOND];
                        M2 F;
                        for (int oo = 0; oo < 2; oo++)
                            for (int ii = 0; ii < 2; ii++) {
                                double sr = std::sqrt(sv[r]);
                                F[oo * 2 + ii] = part == 1 ? xv[oo * 2 + ii][r] / sr : sr * std::conj(vv[oo * 2 + ii][r]);
                            }
                        M2 NF = mul2(noise_op(L, v, q), F);
                        return NF[rb[R_OUT_A] * 2 + rb[R_IN_A]];
                    });
                }
            } else {
                LeafInfo L;
                L.gate = l;
                L.part = 0;
                L.qubit0 = g.q0;
                L.qubit1 = g.q1;
                for (int32_t s : gsites[l]) {
                    L.sites.push_back(s);
                    L.radix.push_back((int32_t)qtab[nz->sites[s].channel].size());
                }
                if (!fb) L.legs.push_back(R_IN_B);
                if (!fa) L.legs.push_back(R_IN_A);
                L.legs.push_back(R_OUT_B);
                L.legs.push_back(R_OUT_A);
                finish_leaf(L, [&](int64_t v, const int32_t* rb) {
                    if (two_qubit_noise) {   // every site's operator in application order, then the gate
                        M4 T{};
                        for (int i = 0; i < 4; i++) T[i * 4 + i] = 1.0;
                        int64_t vv = v;
                        for (size_t i = 0; i < L.sites.size(); i++) {
                            const int k = (int)(vv % L.radix[i]);
                            vv /= L.radix[i];
                            T = mul4(scaled_kraus4(L.sites[i], k, g), T);
                        }
                        const M4 TM = mul4(T, M);
                        return TM[(rb[R_OUT_A] * 2 + rb[R_OUT_B]) * 4 + rb[R_IN_A] * 2 + rb[R_IN_B]];
                    }
                    M2 Na = noise_op(L, v, g.q0), Nb = noise_op(L, v, g.q1);
                    int ro = rb[R_OUT_A] * 2 + rb[R_OUT_B];
                    int ci = rb[R_IN_A] * 2 + rb[R_IN_B];
                    // ((Na (x) Nb) M)[ro][ci] = sum_{a,b} Na[oa][a] Nb[ob][b] M[(a b)][ci]
                    cd z = 0;
                    for (int a = 0; a < 2; a++)
                        for (int bb = 0; bb < 2; bb++)
                            z += Na[rb[R_OUT_A] * 2 + a] * Nb[rb[R_OUT_B] * 2 + bb] * M[(a * 2 + bb) * 4 + ci];
                    (void)ro;
                    return z;
                });
            }
        }
    }
    for (int q = 0; q < n; q++)
        if (!touched[q]) {
            LeafInfo L;
            L.gate = -1;
            L.part = 0;
            L.qubit0 = q;
            L.qubit1 = -1;
            L.legs.push_back(R_OUT_A);
            finish_leaf(L, [](int64_t, const int32_t* rb) { return rb[R_OUT_A] ? cd(0) : cd(1); });
        }
    // CSR of variant-selecting sites per var column
    plan->leaf_site_ptr.assign(plan->n_var_cols + 1, 0);
    plan->leaf_site_idx.clear();
    plan->leaf_site_mul.clear();
    {
        std::vector<const LeafInfo*> bycol(plan->n_var_cols, nullptr);
        for (auto& L : plan->leaves)
            if (L.var_col >= 0) bycol[L.var_col] = &L;
        for (int col = 0; col < plan->n_var_cols; col++) {
            const LeafInfo& L = *bycol[col];
            int64_t mul = 1;
            for (size_t i = 0; i < L.sites.size(); i++) {
                plan->leaf_site_idx.push_back(L.sites[i]);
                plan->leaf_site_mul.push_back((int32_t)mul);
                mul *= L.radix[i];
            }
            plan->leaf_site_ptr[col + 1] = (int32_t)plan->leaf_site_idx.size();
        }
    }

    // ---- blocks
    std::vector<int32_t> bs;
    if (block_sizes && n_blocks > 0) {
        bs.assign(block_sizes, block_sizes + n_blocks);
    } else {
        int f = (n + 9) / 10;
        for (int j = 0; j < f - 1; j++) bs.push_back(10);
        bs.push_back(n - 10 * (f - 1));
    }
    if ((int)bs.size() > kMaxBlocks) return set_error(PTN_ERR_INVALID_ARG, "too many blocks");
    int tot = 0;
    for (size_t j = 0; j < bs.size(); j++) {
        const int32_t v = bs[j];
        const int32_t vmax = j + 1 == bs.size() ? kMaxFinalBlock : kMaxSampleBlock;
        if (v < 1 || v > vmax)
            return set_error(PTN_ERR_INVALID_ARG, "block sizes must be in 1..%d (the last block 1..%d)", kMaxSampleBlock,
                             kMaxFinalBlock);
        tot += v;
    }
    if (tot != n) return set_error(PTN_ERR_INVALID_ARG, "block sizes sum to %d, circuit has %d qubits", tot, n);

    std::mt19937_64 rng(opts.seed ^ 0x9E3779B97F4A7C15ull);
    int start = 0;
    plan->blocks.clear();
    for (size_t j = 0; j < bs.size(); j++) {
        int b = bs[j];
        BlockNet net;
        build_block_net(plan, n, start, b, false, net);
        double E = opts.est_traj;
        double D = j == 0 ? E : std::min(E * std::ldexp(1.0, start), opts.est_shots);
        D = std::max(D, E);
        BlockPlan bp;
        ptn_status e = PTN_OK;
        if (opts.network_form == PTN_FORM_DOUBLE_LAYER) {
            e = search_and_lower(plan, net, (int)j, start, b, E, j == 0 ? E : D, rng, bp, false);
        } else {
            // ket-only form (amplitudes of the block and later qubits, closing |.|^2
            // step), alone (KET_ONLY) or against the double layer (AUTO) by
            // modelled time; either falls back to the double layer without a path
            // (the ket-only search draws from its own stream, so the double-layer
            // path is the one DOUBLE_LAYER finds)
            BlockNet knet;
            build_block_net(plan, n, start, b, true, knet);
            BlockPlan bk, bd;
            std::mt19937_64 krng(rng);   // a copy: rng itself is not advanced
            const ptn_status ek = search_and_lower(plan, knet, (int)j, start, b, E, j == 0 ? E : D, krng, bk, false);
            ptn_status ed = PTN_ERR_TOO_LARGE;
            if (opts.network_form == PTN_FORM_AUTO || ek != PTN_OK)
                ed = search_and_lower(plan, net, (int)j, start, b, E, j == 0 ? E : D, rng, bd, false);
            if (ek == PTN_OK && (ed != PTN_OK || bk.est_time <= bd.est_time)) {
                bp = std::move(bk);
                bp.ket_only = 1;
            } else if (ed == PTN_OK) {
                bp = std::move(bd);
            }
            else e = ed;
            if (!e) clear_error();
        }
        if (e) return e;
        plan->blocks.push_back(std::move(bp));
        start += b;
    }
    plan->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return PTN_OK;
}

static void json_op(std::string& s, const OperandDesc& d) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "{\"mode\":%d,\"cls\":%d,\"conj\":%d,\"arena\":%d,\"inst_size\":%lld,\"arena_off\":%lld,"
             "\"leaf_base\":%lld,\"leaf_col\":%d,\"cache\":%d,\"slices\":[",
             d.mode, d.cls, d.conj, d.arena, (long long)d.inst_size, (long long)d.arena_off, (long long)d.leaf_base,
             d.leaf_col, d.cache);
    s += buf;
    for (int k = 0; k < d.n_slice; k++) {
        snprintf(buf, sizeof buf, "%s[%d,%lld]", k ? "," : "", d.slice_qubit[k], (long long)d.slice_stride[k]);
        s += buf;
    }
    s += "]}";
}

static void json_i64(std::string& s, const int64_t* v, int n) {
    char buf[32];
    s += "[";
    for (int k = 0; k < n; k++) {
        snprintf(buf, sizeof buf, "%s%lld", k ? "," : "", (long long)v[k]);
        s += buf;
    }
    s += "]";
}

static void json_steps(std::string& s, const std::vector<StepDesc>& steps) {
    char buf[512];
    s += "[";
    for (size_t i = 0; i < steps.size(); i++) {
        const StepDesc& st = steps[i];
        snprintf(buf, sizeof buf,
                 "%s{\"out_cls\":%d,\"n_out\":%d,\"n_sum\":%d,\"kind\":%d,\"gemm_a\":%d,\"out_arena\":%d,"
                 "\"out_off\":%lld,\"fuse_prev\":%d,\"cache\":%d,\"virt\":%d,\"prod\":%d,\"prod_src\":%d,"
                 "\"ops\":[",
                 i ? "," : "", st.out_cls, st.n_out, st.n_sum, st.kind, st.gemm_a, st.out_arena, (long long)st.out_off,
                 st.fuse_prev, st.cache, st.virt, st.prod, st.prod_src);
        s += buf;
        json_op(s, st.op[0]);
        s += ",";
        json_op(s, st.op[1]);
        s += "],\"out_stride\":[";
        json_i64(s, st.out_stride[0], st.n_out);
        s += ",";
        json_i64(s, st.out_stride[1], st.n_out);
        s += "],\"sum_stride\":[";
        json_i64(s, st.sum_stride[0], st.n_sum);
        s += ",";
        json_i64(s, st.sum_stride[1], st.n_sum);
        s += "]}";
    }
    s += "]";
}

std::string describe_plan(const ptn_plan* p, int detail) {
    std::string s = "{";
    char buf[768];
    snprintf(buf, sizeof buf,
             "\"n_qubits\":%d,\"n_sites\":%d,\"n_leaves\":%zu,\"n_var_cols\":%d,\"plan_seconds\":%.6f,\"blocks\":[",
             p->n_qubits, p->n_sites, p->leaves.size(), p->n_var_cols, p->plan_seconds);
    s += buf;
    for (size_t j = 0; j < p->blocks.size(); j++) {
        const BlockPlan& b = p->blocks[j];
        int cnt[3] = {0, 0, 0}, n_gemm = 0;
        int64_t maxout = 0;
        for (auto& st : b.steps) {
            cnt[st.out_cls]++;
            n_gemm += st.kind != STEP_DIRECT;
            maxout = std::max<int64_t>(maxout, st.n_out);
        }
        snprintf(buf, sizeof buf,
                 "%s{\"start\":%d,\"b\":%d,\"ket_only\":%d,\"n_gemm\":%d,\"n_steps\":%zu,\"steps_const\":%d,\"steps_traj\":%d,\"steps_net\":%d,"
                 "\"max_out_bits\":%lld,\"arena_const\":%lld,\"arena_traj\":%lld,\"arena_net\":%lld,"
                 "\"macs_const\":%.6e,\"macs_traj\":%.6e,\"macs_net\":%.6e,\"bytes_traj\":%.6e,\"bytes_net\":%.6e,"
                 "\"est_time\":%.6e,\"mult_traj\":%.1f,\"mult_net\":%.1f,\"n_cache\":%d",
                 j ? "," : "", b.start, b.b, b.ket_only, n_gemm, b.steps.size(), cnt[0], cnt[1], cnt[2], (long long)maxout,
                 (long long)b.arena_peak[0], (long long)b.arena_peak[1], (long long)b.arena_peak[2], b.est_macs[0],
                 b.est_macs[1], b.est_macs[2], b.est_bytes[1], b.est_bytes[2], b.est_time, b.est_mult_traj,
                 b.est_mult_net, b.n_cache);
        s += buf;
        if (detail) {
            s += ",\"cache_cols\":[";
            for (int k = 0; k < b.n_cache; k++) {
                s += k ? ",[" : "[";
                bool first = true;
                for (int c = 0; c < p->n_var_cols; c++)
                    if ((b.cache_bits[(size_t)k * b.cache_words + (c >> 5)] >> (c & 31)) & 1u) {
                        snprintf(buf, sizeof buf, "%s%d", first ? "" : ",", c);
                        s += buf;
                        first = false;
                    }
                s += "]";
            }
            s += "]";
            s += ",\"steps\":";
            json_steps(s, b.steps);
            s += ",\"root\":{\"op\":";
            json_op(s, b.root.op);
            s += ",\"x_stride\":";
            json_i64(s, b.root.x_stride, b.b);
            s += "}";
        }
        s += "}";
    }
    s += "]";
    if (detail) {
        s += ",\"var_cols\":[";
        for (int c = 0; c < p->n_var_cols; c++) {
            s += c ? ",[" : "[";
            for (int e = p->leaf_site_ptr[c]; e < p->leaf_site_ptr[c + 1]; e++) {
                snprintf(buf, sizeof buf, "%s[%d,%d]", e > p->leaf_site_ptr[c] ? "," : "", p->leaf_site_idx[e],
                         p->leaf_site_mul[e]);
                s += buf;
            }
            s += "]";
        }
        s += "],\"var_table\":[";
        for (size_t k = 0; k < p->var_table.size(); k++) {
            snprintf(buf, sizeof buf, "%s%.9g", k ? "," : "", p->var_table[k]);
            s += buf;
        }
        s += "],\"site_cdf\":[";
        for (size_t k = 0; k < p->site_tables.size(); k++) {
            const SiteTable& T = p->site_tables[k];
            s += k ? ",[" : "[";
            for (int a = 0; a < T.n_kraus; a++) {
                snprintf(buf, sizeof buf, "%s%.17g", a ? "," : "", T.cdf[a]);
                s += buf;
            }
            s += "]";
        }
        s += "]";
    }
    if (detail >= 2 && p->expval) {
        const BlockPlan& e = *p->expval;
        snprintf(buf, sizeof buf,
                 ",\"expval\":{\"n_params\":%d,\"arena\":[%lld,%lld,%lld,%lld,%lld],\"root_adj_off\":%lld,"
                 "\"dvt_size\":%lld,\"steps\":",
                 p->n_params, (long long)e.arena_peak[0], (long long)e.arena_peak[1], (long long)e.arena_peak[2],
                 (long long)e.arena_peak[3], (long long)e.arena_peak[4], (long long)e.root_adj_off,
                 (long long)e.dvt_size);
        s += buf;
        json_steps(s, e.steps);
        s += ",\"bwd\":";
        json_steps(s, e.bwd);
        s += ",\"root\":{\"op\":";
        json_op(s, e.root.op);
        s += ",\"x_stride\":";
        json_i64(s, e.root.x_stride, p->n_qubits);
        s += "},\"pleaves\":[";
        for (size_t k = 0; k < e.pleaves.size(); k++) {
            const ParamLeaf& q = e.pleaves[k];
            snprintf(buf, sizeof buf,
                     "%s{\"leaf\":%d,\"param_index\":%d,\"param_kind\":%d,\"var_col\":%d,\"size\":%lld,"
                     "\"n_var\":%lld,\"lgrad_off\":%lld,\"dvt_base\":%lld,\"var_base\":%lld}",
                     k ? "," : "", q.leaf, q.param_index, q.param_kind, q.var_col, (long long)q.size,
                     (long long)q.n_var, (long long)q.lgrad_off, (long long)q.dvt_base,
                     (long long)p->leaves[q.leaf].var_base);
            s += buf;
        }
        s += "]}";
    }
    s += "}";
    return s;
}

}  // namespace ptn
