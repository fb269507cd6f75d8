// hierarchy.cu -- setup driver (Algorithm 1), Sparse Galerkin sparsify
// (Algorithm 4 with Algorithm 3b), cycle preparation and autotuning, the
// V-cycle (Algorithm 2), PCG and the adaptive solve (Algorithm 5).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <exception>
#include <map>
#include <mutex>
#include <thread>

#include "common.cuh"
#include "cycle_ops.cuh"
#include "hierarchy.cuh"
#include "setup_ops.cuh"

namespace amg {

Hierarchy::~Hierarchy() {
    // one wait for the device, then every buffer goes back to the pool
    // (on another current device the buffers fall back to one wait each)
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur == device && cudaDeviceSynchronize() == cudaSuccess) idle_release.enter();
    if (g_update) cudaGraphExecDestroy(g_update);
    if (g_precond) cudaGraphExecDestroy(g_precond);
    if (graph_stream) cudaStreamDestroy(graph_stream);
    for (auto &p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : event_pool) cudaEventDestroy(e);
    if (h_scal) cudaFreeHost(h_scal);
    if (g_gmres) cudaGraphExecDestroy(g_gmres);
    if (h_gsc) cudaFreeHost(h_gsc);
}

// ---------------------------------------------------------------------------
// Algorithm 1 (sparsify off): strength, PMIS, direct interpolation, Galerkin
// product, and the minimal-pattern flags of each coarse operator.
// Stop: n_l <= max_size, max_levels reached, or |C| = 0 or |C| > 0.9 n_l.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// per-kernel timing with events on the launching stream
// ---------------------------------------------------------------------------
static cudaEvent_t get_event(Hierarchy &h) {
    if (!h.event_pool.empty()) {
        cudaEvent_t e = h.event_pool.back();
        h.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    AMG_CUDA(cudaEventCreate(&e));
    return e;
}

template <class F> static void timed(Hierarchy &h, int kind, int level, double bytes, cudaStream_t s, F &&f) {
    if (!h.timing) { f(); return; }
    PendingEvent pe{kind, level, bytes, get_event(h), get_event(h)};
    AMG_CUDA(cudaEventRecord(pe.a, s));
    f();
    AMG_CUDA(cudaEventRecord(pe.b, s));
    h.pending.push_back(pe);
}

void timing_collect(Hierarchy &h) {
    for (auto &pe : h.pending) {
        AMG_CUDA(cudaEventSynchronize(pe.b));
        float ms = 0.f;
        AMG_CUDA(cudaEventElapsedTime(&ms, pe.a, pe.b));
        if (pe.kind >= 0 && pe.kind < kTimingKinds && pe.level >= 0 && pe.level < kMaxLevels) {
            Timing &t = h.timers[pe.kind][pe.level];
            t.launches++;
            t.ms += ms;
            t.bytes += pe.bytes;
        }
        h.event_pool.push_back(pe.a);
        h.event_pool.push_back(pe.b);
    }
    h.pending.clear();
}

static void init_level_maps(Level &V, cudaStream_t s, bool check = true) {
    V.diagpos.alloc(sizeof(int32_t) * (V.A.nrows + 1));
    V.tpos.alloc(sizeof(int32_t) * (V.A.nnz + 1));
    setup::level_maps(V.A, V.diagpos.as<int32_t>(), V.tpos.as<int32_t>(), s, check);
    V.keep.alloc(V.A.nnz + kPad);
}

// Non-Galerkin step of Algorithm 1: the coarse operator just formed is
// thinned and replaces the Galerkin product (its maps are rebuilt, M and the
// Galerkin values are dropped).
static void nongalerkin_thin(Hierarchy &h, Level &C, double g, cudaStream_t s) {
    C.gamma = g;
    if (g == 0.0) return;
    TmpBuf S;
    if (h.opt.lump == AMG_LUMP_STRONG) {
        S.alloc(C.A.nnz + kPad, s);
        setup::strength(C.A, h.opt.theta, S.as<uint8_t>(), s);
    }
    DevCSR H;
    setup::sparsify(C.A, C.inM.as<uint8_t>(), C.tpos.as<int32_t>(), C.diagpos.as<int32_t>(), g,
                    C.keep.as<uint8_t>(), H, s, S.as<uint8_t>());
    C.A = std::move(H);
    C.inM.release();
    try {
        init_level_maps(C, s);  // validates the thinned operator (diagonal positive)
    } catch (const Error &e) {
        if (e.status != AMG_ERR_INVALID) throw;
        throw Error(AMG_BREAKDOWN, "non-Galerkin: a thinned coarse operator has a non-positive diagonal entry "
                                   "(lower gamma on that level, or use full lumping)");
    }
}

// Setup pipeline (plain Sparse Galerkin setups that are not timed per
// phase): a level's sparsification (Algorithm 4) and cycle preparation need
// only that level and its interpolation, so a second host thread issues them
// on a second stream while the coarsening goes on to the next levels -- the
// coarsening's host round trips and short launches leave the device idle,
// and the second stream's kernels fill those gaps.  Relaxation and transfer
// variants whose decision would need timed trials are left for the calling
// thread, which times them once both streams have drained.
class SetupPipeline {
  public:
    SetupPipeline(Hierarchy &h, cudaStream_t main, const double *gamma, int n_gamma);
    ~SetupPipeline();
    void level_ready(int l);      // level l and its P_l, R_l are formed (on the main stream)
    void coarsening_done(int nlev);
    void finish();                // joins; the main stream then waits for the second one
    // R = P^T on a third stream (of the main stream's priority), beside A P
    // on the main stream; wait_beside() orders the main stream after it
    void transpose_beside(const DevCSR &P, DevCSR &R);
    void wait_beside();
    // the minimal pattern of the new level C on the third stream; A P's
    // buffers are released there once it is done
    void minimal_pattern_beside(Level &C, setup::SlotProduct &AP, const int32_t *cpts);

  private:
    void run();
    void cancel();
    Hierarchy &h_;
    cudaStream_t main_, side_ = nullptr;
    int device_ = 0;
    std::vector<double> gamma_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::vector<cudaEvent_t> ev_;  // ev_[l]: level l is ready; the last one also marks the end of coarsening
    std::vector<cudaEvent_t> evx_;  // evx_[l]: the third stream's work up to level l's readiness
    int nready_ = 0, nlev_ = -1;
    bool stop_ = false;
    std::exception_ptr err_;
    std::vector<int> defer_relax_, defer_transfer_;
    cudaEvent_t done_ = nullptr;
    cudaStream_t aux_ = nullptr;
    cudaEvent_t ev_p_ = nullptr, ev_r_ = nullptr;
    std::thread th_;
};

void build_galerkin(Hierarchy &h, const DevCSR &A0in, cudaStream_t s, const double *gamma, int n_gamma,
                   SetupPipeline *pipe) {
    (void)A0in;
    const amg_options &o = h.opt;
    h.lev.reserve(kMaxLevels + 1);  // the pipeline thread holds references into it while levels are added
    const bool nongal = o.method == AMG_METHOD_NONGALERKIN;
    for (int l = 0;; ++l) {
        Level &V = *h.lev[l];
        if (l == 0) timed(h, 12, 0, 0.0, s, [&] { init_level_maps(V, s); });
        int32_t n = V.A.nrows;
        if (n <= o.max_size || l + 1 >= o.max_levels) break;
        V.strong.alloc(V.A.nnz + kPad);
        V.cf.alloc(n + kPad);
        V.cmap.alloc(sizeof(int32_t) * (n + 1));
        timed(h, 8, l, 0.0, s, [&] { setup::strength(V.A, o.theta, V.strong.as<uint8_t>(), s); });
        int64_t nc = 0;
        timed(h, 9, l, 0.0, s, [&] {
            nc = setup::pmis(V.A, V.strong.as<uint8_t>(), V.tpos.as<int32_t>(), o.seed, o.level_offset + l,
                             V.cf.as<int8_t>(), V.cmap.as<int32_t>(), s);
        });
        if (nc == 0 || (double)nc > 0.9 * (double)n) {
            V.strong.release();
            V.cf.release();
            V.cmap.release();
            break;
        }
        V.cpts.alloc(sizeof(int32_t) * (nc + 1));
        timed(h, 9, l, 0.0, s, [&] {
            setup::coarse_points(V.cf.as<int8_t>(), n, V.cmap.as<int32_t>(), V.cpts.as<int32_t>(), s);
        });
        timed(h, 10, l, 0.0, s, [&] {
            setup::direct_interp(V.A, V.strong.as<uint8_t>(), V.cf.as<int8_t>(), V.cmap.as<int32_t>(),
                                 (int32_t)nc, V.P, s);
            if (pipe) pipe->transpose_beside(V.P, V.R);  // R forms while A P does
            else setup::transpose(V.P, V.R, s);
        });
        // A P is read twice (by R (A P) and the minimal pattern) and then
        // dropped: it stays in the product slots of its one-pass SpGEMM
        setup::SlotProduct AP;
        auto C = std::make_unique<Level>();
        timed(h, 11, l, 0.0, s, [&] {
            setup::spgemm_slots(V.A, V.P, AP, s);
            if (pipe) pipe->wait_beside();
            setup::spgemm(V.R, AP.rows, C->A, s);
        });
        timed(h, 12, l, 0.0, s, [&] {
            init_level_maps(*C, s, false);  // R (A P) of a checked A_l
            C->inM.alloc(C->A.nnz + kPad);
            if (pipe) {  // only the sparsification reads M: off the coarsening's path, with A P freed there
                pipe->minimal_pattern_beside(*C, AP, V.cpts.as<int32_t>());
            } else {
                setup::minimal_pattern(C->A, AP.rows, V.cpts.as<int32_t>(), C->inM.as<uint8_t>(), s,
                                       C->tpos.as<int32_t>());
            }
        });
        if (nongal) {
            const double g = (n_gamma > 0 && gamma) ? gamma[std::min(l + 1, n_gamma - 1)] : 0.0;
            timed(h, 13, l + 1, 0.0, s, [&] { nongalerkin_thin(h, *C, g, s); });
        }
        h.lev.push_back(std::move(C));
        if (pipe) pipe->level_ready(l);
    }
    if (pipe) pipe->coarsening_done(h.nlev());
}

// Levels given by the caller (amg_hierarchy_assemble / load).
void assemble_levels(Hierarchy &h, std::vector<DevCSR> &A, std::vector<DevCSR> &P,
                     const std::vector<std::vector<int8_t>> &cf,
                     const std::vector<std::vector<uint8_t>> &inM, cudaStream_t s) {
    int L = (int)A.size();
    for (int l = 0; l < L; ++l) {
        auto V = std::make_unique<Level>();
        V->A = std::move(A[l]);
        init_level_maps(*V, s);
        if (l + 1 < L) {
            require(P[l].nrows == V->A.nrows && P[l].ncols == A[l + 1].nrows,
                    "assemble: P_l must be n_l x n_{l+1}");
            V->P = std::move(P[l]);
            setup::validate_rect(V->P, "interpolation operator", s);
            setup::transpose(V->P, V->R, s);
            require((int64_t)cf[l].size() == V->A.nrows, "assemble: cf_l has the wrong length");
            V->cf.alloc(V->A.nrows + kPad);
            AMG_CUDA(cudaMemcpyAsync(V->cf.ptr, cf[l].data(), cf[l].size(), cudaMemcpyHostToDevice, s));
        }
        if (l > 0) {
            require((int64_t)inM[l].size() == V->A.nnz, "assemble: inM_l has the wrong length");
            V->inM.alloc(V->A.nnz + kPad);
            AMG_CUDA(cudaMemcpyAsync(V->inM.ptr, inM[l].data(), inM[l].size(), cudaMemcpyHostToDevice, s));
        }
        h.lev.push_back(std::move(V));
    }
    AMG_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// Algorithm 4 (Sparse Galerkin), Algorithm 3 / 3b per level
// ---------------------------------------------------------------------------
// Hybrid Galerkin (Algorithm 4, hybrid line): the minimal pattern of level l
// comes from Phat^T Ahat_{l-1} P + P^T Ahat_{l-1} Phat with the *sparsified*
// operator of level l-1, i.e. the C rows of Ahat_{l-1} P_{l-1} and their
// transpose.  For l = 1, Ahat_0 = A_0 and the Sparse Galerkin flags apply.
static const uint8_t *hybrid_pattern(Hierarchy &h, int l, cudaStream_t s) {
    Level &F = *h.lev[l - 1];
    Level &V = *h.lev[l];
    if (!F.cpts.ptr) {  // assembled hierarchies carry C/F markers only
        require(F.cf.ptr != nullptr, "hybrid sparsify needs the C/F markers of level l-1");
        int64_t nc = F.P.ncols;
        F.cmap.alloc(sizeof(int32_t) * (F.n() + 1));
        F.cpts.alloc(sizeof(int32_t) * (nc + 1));
        setup::coarse_map(F.cf.as<int8_t>(), F.n(), F.cmap.as<int32_t>(), F.cpts.as<int32_t>(), nc, s);
    }
    DevCSR APh;
    setup::spgemm(F.op(), F.P, APh, s);
    V.inM_hybrid.alloc(V.A.nnz + kPad);
    setup::minimal_pattern(V.A, setup::rows_of(APh), F.cpts.as<int32_t>(), V.inM_hybrid.as<uint8_t>(), s,
                           V.tpos.as<int32_t>());
    return V.inM_hybrid.as<uint8_t>();
}

static void resparsify_one(Hierarchy &h, Level &V, int l, cudaStream_t s) {
    if (l == 0 || V.gamma == 0.0) {
        V.H = DevCSR();
        V.h_alias = true;
        AMG_CUDA(cudaMemsetAsync(V.keep.ptr, 1, V.A.nnz, s));
        return;
    }
    const uint8_t *inM = V.inM.as<uint8_t>();
    if (h.opt.method == AMG_METHOD_HYBRID && l >= 2) inM = hybrid_pattern(h, l, s);
    DevCSR H;
    TmpBuf S;
    if (h.opt.lump == AMG_LUMP_STRONG) {  // Algorithm 3's S: strength of A_l itself
        S.alloc(V.A.nnz + kPad, s);
        setup::strength(V.A, h.opt.theta, S.as<uint8_t>(), s);
    }
    setup::sparsify(V.A, inM, V.tpos.as<int32_t>(), V.diagpos.as<int32_t>(), V.gamma, V.keep.as<uint8_t>(), H, s,
                    S.as<uint8_t>());
    V.H = std::move(H);
    V.h_alias = false;
}

void resparsify_level(Hierarchy &h, int l, cudaStream_t s) { resparsify_one(h, *h.lev[l], l, s); }

static double level_gamma(const double *gamma, int n_gamma, int l) {
    return (l > 0 && n_gamma > 0 && gamma) ? gamma[std::min(l, n_gamma - 1)] : 0.0;
}

void apply_gammas(Hierarchy &h, const double *gamma, int n_gamma, cudaStream_t s) {
    if (h.opt.method == AMG_METHOD_NONGALERKIN) {  // thinned during the setup: every level is final
        for (int l = 0; l < h.nlev(); ++l) {
            Level &V = *h.lev[l];
            V.H = DevCSR();
            V.h_alias = true;
            AMG_CUDA(cudaMemsetAsync(V.keep.ptr, 1, V.A.nnz, s));
        }
        return;
    }
    for (int l = 0; l < h.nlev(); ++l) {
        h.lev[l]->gamma = level_gamma(gamma, n_gamma, l);
        timed(h, 13, l, 0.0, s, [&] { resparsify_level(h, l, s); });
    }
}

// Algorithm 5 drop-tolerance update (finest level >= 1 with gamma > 0, s
// levels, gamma/10 or 0 below gamma_min) and re-sparsify from the retained
// Galerkin operators.  Returns the number of levels changed.
int reintroduce(Hierarchy &h, int s_levels, cudaStream_t s) {
    int L = h.nlev();
    int lstart = -1;
    for (int l = 1; l < L; ++l)
        if (h.lev[l]->gamma > 0.0) { lstart = l; break; }
    if (lstart < 0) return 0;
    std::vector<int> changed;
    for (int l = lstart; l < lstart + s_levels && l < L; ++l) {
        double g = h.lev[l]->gamma / 10.0;
        h.lev[l]->gamma = (g >= h.opt.gamma_min * (1.0 - 1e-12)) ? g : 0.0;
        timed(h, 13, l, 0.0, s, [&] { resparsify_level(h, l, s); });
        changed.push_back(l);
    }
    prepare_cycle(h, s, changed);
    return (int)changed.size();
}

// ---------------------------------------------------------------------------
// cycle preparation: ell1 diagonals, precision copies, SELL, autotuning
// ---------------------------------------------------------------------------
static int heuristic_variant(const DevCSR &M) {
    double mean = M.nrows > 0 ? (double)M.nnz / M.nrows : 0.0;
    if (mean <= 3.0) return AMG_SPMV_CSR2;
    if (mean <= 8.0) return AMG_SPMV_CSR4;
    if (mean <= 20.0) return AMG_SPMV_CSR8;
    if (mean <= 48.0) return AMG_SPMV_CSR16;
    return AMG_SPMV_CSR32;
}

// SELL-C copy (C = 32, 16 or 8 rows per slice) of M with values vals.  If
// slices of consecutive rows would pad the matrix by more than 3%, rows are
// sorted by length inside windows of kSellSigma rows (SELL-C-sigma) and
// kernels write through the permutation.
template <typename VT>
static void build_sell_copy(const DevCSR &M, const VT *vals, SellCopy &S, cudaStream_t s, int C = 32) {
    const int32_t nsl = (M.nrows + C - 1) / C;
    S.c = C;
    S.soff.alloc(sizeof(int32_t) * (nsl + 1));
    S.sw.alloc(sizeof(int32_t) * (nsl + 1));
    S.perm.release();
    S.entries = cyc::sell_layout(M.nrows, M.rp(), nullptr, S.soff.as<int32_t>(), S.sw.as<int32_t>(), s, C);
    if ((double)S.entries > 1.03 * (double)M.nnz) {
        S.perm.alloc(sizeof(int32_t) * (M.nrows + kPad));
        S.entries = cyc::sell_layout(M.nrows, M.rp(), S.perm.as<int32_t>(), S.soff.as<int32_t>(),
                                     S.sw.as<int32_t>(), s, C);
    }
    S.sci.alloc(sizeof(int32_t) * (S.entries + kPad));
    S.sv.alloc(sizeof(VT) * (S.entries + kPad));
    cyc::sell_fill<VT>(M.nrows, M.rp(), M.ci(), vals, S.perm.ptr ? S.perm.as<int32_t>() : nullptr,
                       S.soff.as<int32_t>(), S.sw.as<int32_t>(), S.sci.as<int32_t>(), S.sv.as<VT>(), s, nullptr, C);
}

// SELL-C copy of the relaxed operator of V (C = 32, 16 or 8)
template <typename VT> static void build_sell(Level &V, cudaStream_t s, int C = 32) {
    const DevCSR &M = V.op();
    int32_t nsl = (M.nrows + C - 1) / C;
    V.sell_c = C;
    V.soff.alloc(sizeof(int32_t) * (nsl + 1));
    V.sw.alloc(sizeof(int32_t) * (nsl + 1));
    V.sperm.release();
    V.sell_entries = cyc::sell_layout(M.nrows, M.rp(), nullptr, V.soff.as<int32_t>(), V.sw.as<int32_t>(), s, C);
    if ((double)V.sell_entries > 1.03 * (double)M.nnz) {
        V.sperm.alloc(sizeof(int32_t) * (M.nrows + kPad));
        V.sell_entries = cyc::sell_layout(M.nrows, M.rp(), V.sperm.as<int32_t>(), V.soff.as<int32_t>(),
                                          V.sw.as<int32_t>(), s, C);
    }
    // columns as int16 offsets from the row when every one fits (2 bytes less per entry)
    V.sci.release();
    V.sd.release();
    V.max_row = 0;
    const bool d16 = M.nrows == M.ncols && cyc::max_col_offset(M.nrows, M.rp(), M.ci(), s, &V.max_row) <= 32767;
    if (d16) V.sd.alloc(sizeof(int16_t) * (V.sell_entries + kPad));
    else V.sci.alloc(sizeof(int32_t) * (V.sell_entries + kPad));
    V.sv.alloc(sizeof(VT) * (V.sell_entries + kPad));
    CycMat<VT> m = op_mat<VT>(V);
    cyc::sell_fill<VT>(M.nrows, M.rp(), M.ci(), m.v, V.sperm.ptr ? V.sperm.as<int32_t>() : nullptr,
                       V.soff.as<int32_t>(), V.sw.as<int32_t>(), d16 ? nullptr : V.sci.as<int32_t>(),
                       V.sv.as<VT>(), s, d16 ? V.sd.as<int16_t>() : nullptr, C);
}


static void free_sell(Level &V) {
    V.soff.release(); V.sw.release(); V.sci.release(); V.sd.release(); V.sv.release(); V.sperm.release();
    V.sv64.release();
    V.sell_entries = 0;
}

// Autotuner: time the post-smoothing kernel of one level under each plausible
// variant (vector-CSR with T lanes covering between a quarter and four times
// the mean row, and SELL-32), keep the fastest.  Decisions are cached per
// (rows, entries, value bytes) so setting up the same operator shape again
// costs no trials.
struct TuneKey {
    int64_t n, nnz;
    int vbytes;
    bool operator<(const TuneKey &o) const {
        return n != o.n ? n < o.n : (nnz != o.nnz ? nnz < o.nnz : vbytes < o.vbytes);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune_cache;
static bool g_tune_loaded = false;

// Decisions persist across processes when AMG_TUNE_CACHE names a file: it is
// read on first use and every new decision is appended ("n nnz kind variant").
static void tune_cache_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("AMG_TUNE_CACHE");
    if (!path || !*path) return;
    std::FILE *f = std::fopen(path, "r");
    if (!f) return;
    long long n, z;
    int kind, var;
    while (std::fscanf(f, "%lld %lld %d %d", &n, &z, &kind, &var) == 4) g_tune_cache[TuneKey{n, z, kind}] = var;
    std::fclose(f);
}

static void tune_cache_store_locked(const TuneKey &k, int variant) {
    g_tune_cache[k] = variant;
    const char *path = std::getenv("AMG_TUNE_CACHE");
    if (!path || !*path) return;
    if (std::FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "%lld %lld %d %d\n", (long long)k.n, (long long)k.nnz, k.vbytes, variant);
        std::fclose(f);
    }
}

// fine: level 0, whose SELL copy also serves the outer PCG's fused SELL-32
// kernels, keeps one lane per row; the coarse levels' longer rows may split
// over 2 or 4 lanes (SELL-16, SELL-8)
static std::vector<int> tune_candidates(const DevCSR &M, int vbytes, bool fine) {
    double mean = M.nrows > 0 ? (double)M.nnz / M.nrows : 0.0;
    int V = 16 / vbytes;  // entries per 16-byte load
    std::vector<int> c;
    const int vars[] = {AMG_SPMV_CSR2, AMG_SPMV_CSR4, AMG_SPMV_CSR8, AMG_SPMV_CSR16, AMG_SPMV_CSR32};
    for (int v : vars) {
        double cover = (double)cyc::threads_per_row(v) * V;
        if (cover >= mean / 4.0 && cover <= std::max(4.0 * mean, (double)V * 2)) c.push_back(v);
    }
    if (c.empty()) c.push_back(AMG_SPMV_CSR4);
    c.push_back(AMG_SPMV_SELL32);
    if (!fine && mean >= 4.0) c.push_back(AMG_SPMV_SELL16);
    if (!fine && mean >= 8.0) c.push_back(AMG_SPMV_SELL8);
    return c;
}

// Evicts the L2 cache before a timed trial: in the V-cycle a level's
// operator is re-read after the finer levels' traffic has passed through L2,
// so a trial on an L2-resident operator would favour the wrong variant.
struct L2Flush {
    TmpBuf buf;
    void run(cudaStream_t s) {
        if (!buf.ptr) {
            int dev = 0, l2 = 0;
            AMG_CUDA(cudaGetDevice(&dev));
            AMG_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
            buf.alloc((size_t)std::max(l2, 1 << 20) * 3 / 2, s);
        }
        AMG_CUDA(cudaMemsetAsync(buf.ptr, 0, buf.bytes, s));
    }
};

template <typename VT, typename XT> static void autotune_level(Hierarchy &h, Level &V, cudaStream_t s, bool fine) {
    const std::vector<int> cands = tune_candidates(V.op(), V.vbytes, fine);
    L2Flush flush;
    cudaEvent_t e0, e1;
    AMG_CUDA(cudaEventCreate(&e0));
    AMG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_v = V.variant;
    const XT *dinv = sizeof(XT) == 8 ? reinterpret_cast<const XT *>(V.dinv.ptr) : V.dinv32.as<XT>();
    for (int c : cands) {
        V.variant = c;
        const int C = sell_height(c);
        if (C && V.sell_c != C) build_sell<VT>(V, s, C);
        CycMat<VT> m = op_mat<VT>(V);
        cyc::post_smooth<VT, XT>(m, V.x.as<XT>(), V.b.as<XT>(), dinv, V.xo.as<XT>(), s);  // warm-up
        float tmin = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            flush.run(s);
            AMG_CUDA(cudaEventRecord(e0, s));
            cyc::post_smooth<VT, XT>(m, V.x.as<XT>(), V.b.as<XT>(), dinv, V.xo.as<XT>(), s);
            AMG_CUDA(cudaEventRecord(e1, s));
            AMG_CUDA(cudaEventSynchronize(e1));
            float ms;
            AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            tmin = std::min(tmin, ms);
        }
        if (tmin < best * 0.98f) { best = tmin; best_v = c; }
    }
    V.variant = best_v;
    const int C = sell_height(best_v);
    if (C && V.sell_c != C) build_sell<VT>(V, s, C);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)h;
}

template <typename T> static void alloc_zero(DevBuf &b, int64_t n, cudaStream_t s) {
    b.alloc(sizeof(T) * (size_t)(n + kPad));
    AMG_CUDA(cudaMemsetAsync(b.ptr, 0, b.bytes, s));
}

// Cycle data of level V (= level l; has_p: it has a coarser level).  Without
// allow_tune a relaxation variant that would need timed trials is left to the
// caller (returns true): trials are timed only with the device to themselves.
static bool prepare_level_at(Hierarchy &h, Level &V, int l, bool has_p, cudaStream_t s, bool allow_tune) {
    const DevCSR &M = V.op();
    int32_t n = V.n();
    int prec = h.opt.precision;
    V.l1.alloc(sizeof(double) * (n + kPad));
    V.dinv.alloc(sizeof(double) * (n + kPad));
    setup::l1_diag(M, V.l1.as<double>(), V.dinv.as<double>(), s);
    V.vbytes = prec == AMG_PREC_FP64 ? 8 : (prec == AMG_PREC_FP32_BF16 && l >= 2 ? 2 : 4);
    V.hv32.release();
    V.hv16.release();
    V.dinv32.release();
    free_sell(V);
    if (prec == AMG_PREC_FP64) {
        alloc_zero<double>(V.b, n, s); alloc_zero<double>(V.x, n, s);
        alloc_zero<double>(V.r, n, s); alloc_zero<double>(V.xo, n, s);
    } else {
        alloc_zero<float>(V.b, n, s); alloc_zero<float>(V.x, n, s);
        alloc_zero<float>(V.r, n, s); alloc_zero<float>(V.xo, n, s);
        V.dinv32.alloc(sizeof(float) * (n + kPad));
        cyc::convert_values<float>(V.dinv.as<double>(), V.dinv32.as<float>(), n, s);
        if (V.vbytes == 4) {
            V.hv32.alloc(sizeof(float) * (M.nnz + kPad));
            AMG_CUDA(cudaMemsetAsync(V.hv32.ptr, 0, V.hv32.bytes, s));
            cyc::convert_values<float>(M.v(), V.hv32.as<float>(), M.nnz, s);
        } else {
            V.hv16.alloc(sizeof(__nv_bfloat16) * (M.nnz + kPad));
            AMG_CUDA(cudaMemsetAsync(V.hv16.ptr, 0, V.hv16.bytes, s));
            cyc::convert_values<__nv_bfloat16>(M.v(), V.hv16.as<__nv_bfloat16>(), M.nnz, s);
        }
        if (has_p && !V.pv32.ptr) {
            V.pv32.alloc(sizeof(float) * (V.P.nnz + kPad));
            V.rv32.alloc(sizeof(float) * (V.R.nnz + kPad));
            AMG_CUDA(cudaMemsetAsync(V.pv32.ptr, 0, V.pv32.bytes, s));
            AMG_CUDA(cudaMemsetAsync(V.rv32.ptr, 0, V.rv32.bytes, s));
            cyc::convert_values<float>(V.P.v(), V.pv32.as<float>(), V.P.nnz, s);
            cyc::convert_values<float>(V.R.v(), V.rv32.as<float>(), V.R.nnz, s);
        }
    }
    if (has_p && !V.pr_tuned) {
        V.variant_p = heuristic_variant(V.P);
        V.variant_r = heuristic_variant(V.R);
    }
    // relaxation SpMV variant
    int forced = h.opt.spmv_variant;
    bool tune = forced == AMG_SPMV_AUTO && M.nnz >= 20000 && has_p;
    V.variant = forced == AMG_SPMV_AUTO ? heuristic_variant(M) : forced;
    TuneKey key{M.nrows, M.nnz, V.vbytes};
    if (tune) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load_locked();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            V.variant = it->second;
            tune = false;
        }
    }
    if (tune && !allow_tune) return true;
    if (tune || sell_height(V.variant)) {
        const int C = tune ? 32 : sell_height(V.variant);
        if (V.vbytes == 8) build_sell<double>(V, s, C);
        else if (V.vbytes == 4) build_sell<float>(V, s, C);
        else build_sell<__nv_bfloat16>(V, s, C);
    }
    if (tune) {
        if (V.vbytes == 8) autotune_level<double, double>(h, V, s, l == 0);
        else if (V.vbytes == 4) autotune_level<float, float>(h, V, s, l == 0);
        else autotune_level<__nv_bfloat16, float>(h, V, s, l == 0);
        if (!sell_height(V.variant)) free_sell(V);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_store_locked(key, V.variant);
    }
    // FP32 cycles: the outer PCG multiplies by A_0 in FP64 -- give it the same
    // SELL layout with FP64 values when level 0 relaxes through SELL
    if (l == 0 && V.vbytes != 8 && V.variant == AMG_SPMV_SELL32 && V.sv.ptr) {
        // the index array is the one already filled (same layout); only the values are written again
        V.sv64.alloc(sizeof(double) * (V.sell_entries + kPad));
        TmpBuf junk_idx(V.sd.ptr ? sizeof(int16_t) * (V.sell_entries + kPad) : sizeof(int32_t) * (V.sell_entries + kPad), s);
        cyc::sell_fill<double>(M.nrows, M.rp(), M.ci(), M.v(), V.sperm.ptr ? V.sperm.as<int32_t>() : nullptr,
                               V.soff.as<int32_t>(), V.sw.as<int32_t>(), V.sd.ptr ? nullptr : junk_idx.as<int32_t>(),
                               V.sv64.as<double>(), s, V.sd.ptr ? junk_idx.as<int16_t>() : nullptr);
    }
    return false;
}

static void prepare_level(Hierarchy &h, int l, cudaStream_t s) {
    prepare_level_at(h, *h.lev[l], l, l + 1 < h.nlev(), s, true);
}

static void prepare_coarse_at(Hierarchy &h, Level &V, cudaStream_t s) {
    const DevCSR &M = V.op();
    int32_t n = V.n();
    h.coarse_n = n;
    h.coarse_inv.alloc(sizeof(double) * ((size_t)n * n + kPad));
    setup::cholesky_inverse(M, h.coarse_inv.as<double>(), s);
}

static void prepare_coarse(Hierarchy &h, cudaStream_t s) { prepare_coarse_at(h, *h.lev[h.nlev() - 1], s); }

// Transfer operators: time prolongation (x += P x_c) and restriction
// (b_c = R r, x_c = d_c b_c) under the vector-CSR widths that fit their mean
// row, keep the fastest (cached per shape like the relaxation).
// Without allow_tune, an operator whose decision is not cached is left to the
// caller (returns true) instead of being timed.
template <typename XT> static bool autotune_transfers_at(Level &V, Level &C, cudaStream_t s, bool allow_tune) {
    int vb = sizeof(XT);
    bool deferred = false;
    L2Flush flush;
    cudaEvent_t e0, e1;
    AMG_CUDA(cudaEventCreate(&e0));
    AMG_CUDA(cudaEventCreate(&e1));
    auto tune = [&](const DevCSR &M, const XT *vals, SellCopy &S, int kind, int &variant, auto run) {
        TuneKey key{M.nrows, M.nnz, 100 * kind + vb};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            tune_cache_load_locked();
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                variant = it->second;
                if (sell_height(variant)) build_sell_copy<XT>(M, vals, S, s, sell_height(variant));
                return;
            }
        }
        S.release();  // a copy of an earlier operator must not stand in for this one
        if (!allow_tune) {
            deferred = true;
            return;
        }
        double mean = M.nrows > 0 ? (double)M.nnz / M.nrows : 0.0;
        int V16 = 16 / vb;
        float best = 1e30f;
        int best_v = variant;
        const int vars[] = {AMG_SPMV_CSR1, AMG_SPMV_CSR2, AMG_SPMV_CSR4, AMG_SPMV_CSR8, AMG_SPMV_CSR16,
                            AMG_SPMV_SELL32, AMG_SPMV_SELL16, AMG_SPMV_SELL8};
        for (int v : vars) {
            const int C = sell_height(v);
            double cover = (double)cyc::threads_per_row(v) * V16;
            if (!C && v != AMG_SPMV_CSR1 &&
                !(cover >= mean / 4.0 && cover <= std::max(4.0 * mean, (double)V16 * 2)))
                continue;
            if ((C == 16 && mean < 4.0) || (C == 8 && mean < 8.0)) continue;
            if (C && (!S.sv.ptr || S.c != C)) build_sell_copy<XT>(M, vals, S, s, C);
            variant = v;
            run();
            float tmin = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                flush.run(s);
                AMG_CUDA(cudaEventRecord(e0, s));
                run();
                AMG_CUDA(cudaEventRecord(e1, s));
                AMG_CUDA(cudaEventSynchronize(e1));
                float ms;
                AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                tmin = std::min(tmin, ms);
            }
            if (tmin < best * 0.98f) { best = tmin; best_v = v; }
        }
        variant = best_v;
        const int C = sell_height(variant);
        if (!C) S.release();
        else if (S.c != C) build_sell_copy<XT>(M, vals, S, s, C);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_store_locked(key, best_v);
    };
    if (V.P.nnz >= 20000) {
        const XT *pv, *rv;
        if constexpr (sizeof(XT) == 8) {
            pv = reinterpret_cast<const XT *>(V.P.v());
            rv = reinterpret_cast<const XT *>(V.R.v());
        } else {
            pv = V.pv32.as<XT>();
            rv = V.rv32.as<XT>();
        }
        tune(V.P, pv, V.psell, 1, V.variant_p,
             [&] { cyc::spmv<XT, XT>(p_mat<XT>(V), C.xo.as<XT>(), V.x.as<XT>(), true, s); });
        tune(V.R, rv, V.rsell, 2, V.variant_r, [&] {
            cyc::spmv_scaled<XT, XT>(r_mat<XT>(V), V.r.as<XT>(), dinv_of<XT>(C), C.b.as<XT>(), C.x.as<XT>(), s);
        });
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return deferred;
}

template <typename XT> static void autotune_transfers(Hierarchy &h, int l, cudaStream_t s) {
    autotune_transfers_at<XT>(*h.lev[l], *h.lev[l + 1], s, true);
}

void prepare_cycle(Hierarchy &h, cudaStream_t s, const std::vector<int> &levels) {
    for (int l : levels) {
        timed(h, 14, l, 0.0, s, [&] { prepare_level(h, l, s); });
        if (l == h.nlev() - 1) timed(h, 15, l, 0.0, s, [&] { prepare_coarse(h, s); });
        if (h.parts > 1) replan_relaxation(h, l, s);
    }
    if (h.opt.transfer_variant != AMG_SPMV_AUTO) {  // forced for P and R
        const int tv = h.opt.transfer_variant, C = sell_height(tv);
        for (int l : levels) {
            if (l + 1 >= h.nlev() || h.lev[l]->pr_tuned) continue;
            Level &V = *h.lev[l];
            V.variant_p = V.variant_r = tv;
            if (C && h.opt.precision == AMG_PREC_FP64) {
                build_sell_copy<double>(V.P, V.P.v(), V.psell, s, C);
                build_sell_copy<double>(V.R, V.R.v(), V.rsell, s, C);
            } else if (C) {
                build_sell_copy<float>(V.P, V.pv32.as<float>(), V.psell, s, C);
                build_sell_copy<float>(V.R, V.rv32.as<float>(), V.rsell, s, C);
            }
            V.pr_tuned = true;
        }
    } else if (h.opt.spmv_variant == AMG_SPMV_AUTO) {
        for (int l : levels) {
            if (l + 1 >= h.nlev() || h.lev[l]->pr_tuned) continue;
            timed(h, 14, l, 0.0, s, [&] {
                if (h.opt.precision == AMG_PREC_FP64) autotune_transfers<double>(h, l, s);
                else autotune_transfers<float>(h, l, s);
            });
            h.lev[l]->pr_tuned = true;
        }
    }
    h.graph_dirty = true;
    h.version++;
    AMG_CUDA(cudaStreamSynchronize(s));
}

// A non-blocking stream of a given priority and an event, released on scope
// exit (after the stream's work is done).
struct StreamGuard {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    explicit StreamGuard(int priority) {
        AMG_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, priority));
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamDestroy(s);
            throw Error(AMG_ERR_CUDA, "cudaEventCreate failed");
        }
    }
    StreamGuard() {
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            throw Error(AMG_ERR_CUDA, "cudaEventCreate failed");
        }
    }
    ~StreamGuard() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        cudaEventDestroy(ev);
        cudaGetLastError();
    }
    StreamGuard(const StreamGuard &) = delete;
    StreamGuard &operator=(const StreamGuard &) = delete;
};

// ---------------------------------------------------------------------------
// SetupPipeline
// ---------------------------------------------------------------------------
SetupPipeline::SetupPipeline(Hierarchy &h, cudaStream_t main, const double *gamma, int n_gamma)
    : h_(h), main_(main), gamma_(gamma && n_gamma > 0 ? std::vector<double>(gamma, gamma + n_gamma)
                                                      : std::vector<double>()) {
    AMG_CUDA(cudaGetDevice(&device_));
    int prio = 0;
    AMG_CUDA(cudaStreamGetPriority(main_, &prio));
    // every handle is released by the destructor, also when a later one fails
    struct Undo {
        SetupPipeline *p;
        bool ok = false;
        ~Undo() {
            if (ok) return;
            if (p->side_) cudaStreamDestroy(p->side_);
            if (p->aux_) cudaStreamDestroy(p->aux_);
            if (p->done_) cudaEventDestroy(p->done_);
            if (p->ev_p_) cudaEventDestroy(p->ev_p_);
            if (p->ev_r_) cudaEventDestroy(p->ev_r_);
            cudaGetLastError();
        }
    } undo{this};
    AMG_CUDA(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking));
    AMG_CUDA(cudaStreamCreateWithPriority(&aux_, cudaStreamNonBlocking, prio));
    AMG_CUDA(cudaEventCreateWithFlags(&done_, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreateWithFlags(&ev_p_, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreateWithFlags(&ev_r_, cudaEventDisableTiming));
    th_ = std::thread([this] { run(); });
    undo.ok = true;
}

void SetupPipeline::transpose_beside(const DevCSR &P, DevCSR &R) {
    AMG_CUDA(cudaEventRecord(ev_p_, main_));
    AMG_CUDA(cudaStreamWaitEvent(aux_, ev_p_, 0));
    {
        AllocOn alloc_scope(aux_);  // R's buffers are ordered on the stream that fills them
        setup::transpose(P, R, aux_);
    }
    AMG_CUDA(cudaEventRecord(ev_r_, aux_));
}

void SetupPipeline::wait_beside() { AMG_CUDA(cudaStreamWaitEvent(main_, ev_r_, 0)); }

void SetupPipeline::minimal_pattern_beside(Level &C, setup::SlotProduct &AP, const int32_t *cpts) {
    AMG_CUDA(cudaEventRecord(ev_p_, main_));  // R (A P), the level maps and M's buffer
    AMG_CUDA(cudaStreamWaitEvent(aux_, ev_p_, 0));
    setup::minimal_pattern(C.A, AP.rows, cpts, C.inM.as<uint8_t>(), aux_, C.tpos.as<int32_t>());
    // A P's slot buffers go back to the pool in the third stream's order, after M has read them
    for (TmpBuf *b : {&AP.ci, &AP.v, &AP.beg, &AP.end}) b->stream = aux_;
}

SetupPipeline::~SetupPipeline() {
    cancel();
    // work already issued on the second stream finishes before the levels it
    // writes can be released
    cudaStreamSynchronize(side_);
    cudaStreamSynchronize(aux_);
    cudaGetLastError();
    for (cudaEvent_t e : ev_) cudaEventDestroy(e);
    for (cudaEvent_t e : evx_) cudaEventDestroy(e);
    cudaEventDestroy(done_);
    cudaEventDestroy(ev_p_);
    cudaEventDestroy(ev_r_);
    cudaStreamDestroy(side_);
    cudaStreamDestroy(aux_);
}

void SetupPipeline::cancel() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    if (th_.joinable()) th_.join();
}

// An event recorded now on stream s (appended to `to` under the lock by the caller).
static cudaEvent_t record_now(cudaStream_t s) {
    cudaEvent_t e;
    AMG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (cudaEventRecord(e, s) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e);
        throw Error(AMG_ERR_CUDA, "setup pipeline: cudaEventRecord failed");
    }
    return e;
}

void SetupPipeline::level_ready(int l) {
    cudaEvent_t e = record_now(main_), x = nullptr;
    try {
        x = record_now(aux_);
    } catch (...) {
        cudaEventDestroy(e);
        throw;
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        ev_.push_back(e);
        evx_.push_back(x);
        nready_ = l + 1;
    }
    cv_.notify_all();
}

void SetupPipeline::coarsening_done(int nlev) {
    cudaEvent_t e = record_now(main_), x = nullptr;
    try {
        x = record_now(aux_);
    } catch (...) {
        cudaEventDestroy(e);
        throw;
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        ev_.push_back(e);
        evx_.push_back(x);
        nlev_ = nlev;
    }
    cv_.notify_all();
}

void SetupPipeline::run() {
    try {
        AMG_CUDA(cudaSetDevice(device_));
        AllocOn alloc_scope(side_);
        const amg_options &o = h_.opt;
        const bool fp64 = o.precision == AMG_PREC_FP64;
        const bool tune_transfers = o.transfer_variant == AMG_SPMV_AUTO && o.spmv_variant == AMG_SPMV_AUTO;
        for (int l = 0;; ++l) {
            bool has_p = false, last = false;
            cudaEvent_t e = nullptr, x = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || nready_ > l || nlev_ >= 0; });
                if (stop_) return;
                if (nready_ > l) {
                    has_p = true;
                    e = ev_[l];
                    x = evx_[l];
                } else {
                    if (l >= nlev_) break;
                    last = l == nlev_ - 1;
                    has_p = !last;
                    e = ev_.back();
                    x = evx_.back();
                }
            }
            AMG_CUDA(cudaStreamWaitEvent(side_, e, 0));
            AMG_CUDA(cudaStreamWaitEvent(side_, x, 0));  // the level's minimal pattern
            Level &V = *h_.lev[l];
            V.gamma = level_gamma(gamma_.data(), (int)gamma_.size(), l);
            resparsify_one(h_, V, l, side_);
            if (prepare_level_at(h_, V, l, has_p, side_, false)) defer_relax_.push_back(l);
            if (last) prepare_coarse_at(h_, V, side_);
            if (l > 0) {  // the transfers of level l-1 run on level l's vectors
                Level &F = *h_.lev[l - 1];
                if (o.transfer_variant != AMG_SPMV_AUTO) {
                    const int tv = o.transfer_variant, C = sell_height(tv);
                    F.variant_p = F.variant_r = tv;
                    if (C && fp64) {
                        build_sell_copy<double>(F.P, F.P.v(), F.psell, side_, C);
                        build_sell_copy<double>(F.R, F.R.v(), F.rsell, side_, C);
                    } else if (C) {
                        build_sell_copy<float>(F.P, F.pv32.as<float>(), F.psell, side_, C);
                        build_sell_copy<float>(F.R, F.rv32.as<float>(), F.rsell, side_, C);
                    }
                    F.pr_tuned = true;
                } else if (tune_transfers) {
                    const bool d = fp64 ? autotune_transfers_at<double>(F, V, side_, false)
                                        : autotune_transfers_at<float>(F, V, side_, false);
                    if (d) defer_transfer_.push_back(l - 1);
                    else F.pr_tuned = true;
                }
            }
        }
        AMG_CUDA(cudaEventRecord(done_, side_));
    } catch (...) {
        err_ = std::current_exception();
        cudaEventRecord(done_, side_);
        cudaGetLastError();
    }
}

void SetupPipeline::finish() {
    if (th_.joinable()) th_.join();
    if (err_) std::rethrow_exception(err_);
    AMG_CUDA(cudaStreamWaitEvent(main_, done_, 0));
    // the trials left over, timed on the main stream with the device to themselves
    AMG_CUDA(cudaStreamSynchronize(side_));
    for (int l : defer_relax_) prepare_level(h_, l, main_);
    const bool fp64 = h_.opt.precision == AMG_PREC_FP64;
    for (int l : defer_transfer_) {
        if (fp64) autotune_transfers<double>(h_, l, main_);
        else autotune_transfers<float>(h_, l, main_);
        h_.lev[l]->pr_tuned = true;
    }
    h_.graph_dirty = true;
    h_.version++;
}

// Algorithm 1 and the cycle preparation of every level (amg_setup).
void setup_hierarchy(Hierarchy &h, cudaStream_t s, const double *gamma, int n_gamma) {
    const bool pipelined = !h.timing && h.opt.method == AMG_METHOD_SPARSE && h.parts <= 1;
    if (!pipelined) {
        build_galerkin(h, h.lev[0]->A, s, gamma, n_gamma);
        apply_gammas(h, gamma, n_gamma, s);
        std::vector<int> all;
        for (int l = 0; l < h.nlev(); ++l) all.push_back(l);
        prepare_cycle(h, s, all);
        return;
    }
    // the coarsening -- the longer chain -- runs on a stream of the highest
    // priority, so the second stream's blocks fill the gaps it leaves instead
    // of delaying it
    int lo = 0, hi = 0;
    AMG_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    StreamGuard sc(hi), join;
    AMG_CUDA(cudaEventRecord(join.ev, s));  // the uploaded operator
    AMG_CUDA(cudaStreamWaitEvent(sc.s, join.ev, 0));
    {
        AllocOn alloc_scope(sc.s);
        SetupPipeline pipe(h, sc.s, gamma, n_gamma);
        build_galerkin(h, h.lev[0]->A, sc.s, gamma, n_gamma, &pipe);
        pipe.finish();
    }
    AMG_CUDA(cudaEventRecord(join.ev, sc.s));
    AMG_CUDA(cudaStreamWaitEvent(s, join.ev, 0));
    AMG_CUDA(cudaStreamSynchronize(s));
}

void ensure_workspace(Hierarchy &h, cudaStream_t s) {
    int64_t n = h.lev[0]->n();
    if (h.ws_n == n) return;
    alloc_zero<double>(h.pb, n, s); alloc_zero<double>(h.px, n, s);
    alloc_zero<double>(h.pr, n, s); alloc_zero<double>(h.pz, n, s);
    alloc_zero<double>(h.pp, n, s); alloc_zero<double>(h.pq, n, s);
    alloc_zero<double>(h.pt, n, s); alloc_zero<double>(h.pxs, n, s);
    if (h.opt.precision != AMG_PREC_FP64) {
        alloc_zero<float>(h.r32, n, s);
        alloc_zero<float>(h.z32, n, s);
    }
    h.scal.alloc(sizeof(PcgScalars));
    AMG_CUDA(cudaMemsetAsync(h.scal.ptr, 0, sizeof(PcgScalars), s));
    h.partials.alloc(sizeof(double) * (4 * kMaxReduceBlocks + 4 * 256));
    h.counter.alloc(sizeof(unsigned) * 512);
    AMG_CUDA(cudaMemsetAsync(h.counter.ptr, 0, h.counter.bytes, s));
    if (!h.h_scal) AMG_CUDA(cudaMallocHost(&h.h_scal, sizeof(PcgScalars)));
    h.ws_n = n;
}

// ---------------------------------------------------------------------------
// algorithmic bytes (compulsory HBM traffic) per kernel launch
// ---------------------------------------------------------------------------
static double bytes_pre(int64_t n, int64_t nnz, int vb, int xb) { return (double)nnz * (vb + 4) + 4.0 * (n + 1) + 4.0 * n * xb; }
// levels >= 1: x = D^{-1} b was written by the restriction; read b, x, write r
static double bytes_pre_x(int64_t n, int64_t nnz, int vb, int xb) { return (double)nnz * (vb + 4) + 4.0 * (n + 1) + 3.0 * n * xb; }
// restriction that also writes the coarse pre-smooth x_c = d_c .* b_c
static double bytes_restrict_x(int64_t nc, int64_t n, int64_t nnz, int vb, int xb) { return (double)nnz * (vb + 4) + 4.0 * (nc + 1) + (double)(n + 3 * nc) * xb; }
static double bytes_post(int64_t n, int64_t nnz, int vb, int xb) { return (double)nnz * (vb + 4) + 4.0 * (n + 1) + 4.0 * n * xb; }
static double bytes_restrict(int64_t nc, int64_t n, int64_t nnz, int vb, int xb) { return (double)nnz * (vb + 4) + 4.0 * (nc + 1) + (double)(n + nc) * xb; }
static double bytes_prolong(int64_t n, int64_t nc, int64_t nnz, int vb, int xb) { return (double)nnz * (vb + 4) + 4.0 * (n + 1) + (double)(nc + 2 * n) * xb; }

double level_cycle_bytes(const Hierarchy &h, int l) {
    const Level &V = *h.lev[l];
    int xb = h.opt.precision == AMG_PREC_FP64 ? 8 : 4;
    int64_t n = V.n(), nnz = V.op().nnz;
    if (l == h.nlev() - 1) return (double)n * n * 8 + 2.0 * n * xb;
    double b = (l == 0 ? bytes_pre(n, nnz, V.vbytes, xb) : bytes_pre_x(n, nnz, V.vbytes, xb)) +
               bytes_post(n, nnz, V.vbytes, xb);
    b += (l + 2 < h.nlev() ? bytes_restrict_x(V.R.nrows, n, V.R.nnz, xb, xb) : bytes_restrict(V.R.nrows, n, V.R.nnz, xb, xb)) +
         bytes_prolong(n, V.P.ncols, V.P.nnz, xb, xb);
    return b;
}

// ---------------------------------------------------------------------------
// Algorithm 2: V(1,1) on the residual equation, zero initial guess per level
// ---------------------------------------------------------------------------
// Pre-smooth from zero and residual.  Level 0 forms x = D^{-1} b here (one
// pass, gathering b and d); on coarser levels the restriction already wrote
// x = D^{-1} b, so the pass gathers x alone.
template <typename XT>
static void relax_pre(Hierarchy &h, int l, const XT *b, cudaStream_t s, bool x_ready) {
    Level &V = *h.lev[l];
    int xb = sizeof(XT);
    if (!x_ready) {
        timed(h, 0, l, bytes_pre(V.n(), V.op().nnz, V.vbytes, xb), s, [&] {
            if constexpr (sizeof(XT) == 8) {
                cyc::pre_smooth_residual<double, double>(op_mat<double>(V), b, dinv_of<XT>(V), V.x.as<XT>(), V.r.as<XT>(), s);
            } else {
                if (V.vbytes == 2)
                    cyc::pre_smooth_residual<__nv_bfloat16, float>(op_mat<__nv_bfloat16>(V), b, dinv_of<XT>(V), V.x.as<XT>(), V.r.as<XT>(), s);
                else
                    cyc::pre_smooth_residual<float, float>(op_mat<float>(V), b, dinv_of<XT>(V), V.x.as<XT>(), V.r.as<XT>(), s);
            }
        });
        return;
    }
    timed(h, 0, l, bytes_pre_x(V.n(), V.op().nnz, V.vbytes, xb), s, [&] {
        if constexpr (sizeof(XT) == 8) {
            cyc::residual_from_x<double, double>(op_mat<double>(V), b, V.x.as<XT>(), V.r.as<XT>(), s);
        } else {
            if (V.vbytes == 2)
                cyc::residual_from_x<__nv_bfloat16, float>(op_mat<__nv_bfloat16>(V), b, V.x.as<XT>(), V.r.as<XT>(), s);
            else
                cyc::residual_from_x<float, float>(op_mat<float>(V), b, V.x.as<XT>(), V.r.as<XT>(), s);
        }
    });
}

template <typename XT>
static void relax_post(Hierarchy &h, int l, const XT *b, XT *out, cudaStream_t s) {
    Level &V = *h.lev[l];
    int xb = sizeof(XT);
    timed(h, 3, l, bytes_post(V.n(), V.op().nnz, V.vbytes, xb), s, [&] {
        if constexpr (sizeof(XT) == 8) {
            cyc::post_smooth<double, double>(op_mat<double>(V), V.x.as<XT>(), b, dinv_of<XT>(V), out, s);
        } else {
            if (V.vbytes == 2)
                cyc::post_smooth<__nv_bfloat16, float>(op_mat<__nv_bfloat16>(V), V.x.as<XT>(), b, dinv_of<XT>(V), out, s);
            else
                cyc::post_smooth<float, float>(op_mat<float>(V), V.x.as<XT>(), b, dinv_of<XT>(V), out, s);
        }
    });
}

template <typename XT>
static bool vcycle_impl(Hierarchy &h, const XT *b0, XT *z0, cudaStream_t s, const CycleCtl &ctl) {
    int L = h.nlev();
    int xb = sizeof(XT);
    bool fused = false;
    if (L == 1) {
        timed(h, 4, 0, (double)h.coarse_n * h.coarse_n * 8 + 2.0 * h.coarse_n * xb, s,
              [&] { cyc::coarse_solve<XT>(h.coarse_n, h.coarse_inv.as<double>(), b0, z0, s); });
        return false;
    }
    for (int l = 0; l + 1 < L; ++l) {
        Level &V = *h.lev[l];
        const XT *b = l == 0 ? b0 : V.b.as<XT>();
        relax_pre<XT>(h, l, b, s, l > 0 || ctl.x0_ready);
        Level &C = *h.lev[l + 1];
        if (l + 2 < L) {  // the coarse level relaxes: fold its x = D^{-1} b into the restriction
            timed(h, 1, l, bytes_restrict_x(V.R.nrows, V.n(), V.R.nnz, xb, xb), s, [&] {
                cyc::spmv_scaled<XT, XT>(r_mat<XT>(V), V.r.as<XT>(), dinv_of<XT>(C), C.b.as<XT>(), C.x.as<XT>(), s);
            });
        } else {
            timed(h, 1, l, bytes_restrict(V.R.nrows, V.n(), V.R.nnz, xb, xb), s,
                  [&] { cyc::spmv<XT, XT>(r_mat<XT>(V), V.r.as<XT>(), C.b.as<XT>(), false, s); });
        }
    }
    Level &Cl = *h.lev[L - 1];
    timed(h, 4, L - 1, (double)h.coarse_n * h.coarse_n * 8 + 2.0 * h.coarse_n * xb, s,
          [&] { cyc::coarse_solve<XT>(h.coarse_n, h.coarse_inv.as<double>(), Cl.b.as<XT>(), Cl.xo.as<XT>(), s); });
    for (int l = L - 2; l >= 0; --l) {
        Level &V = *h.lev[l];
        Level &C = *h.lev[l + 1];
        timed(h, 2, l, bytes_prolong(V.n(), V.P.ncols, V.P.nnz, xb, xb), s,
              [&] { cyc::spmv<XT, XT>(p_mat<XT>(V), C.xo.as<XT>(), V.x.as<XT>(), true, s); });
        const XT *b = l == 0 ? b0 : V.b.as<XT>();
        if constexpr (sizeof(XT) == 8) {
            if (l == 0 && ctl.fuse_rz && V.vbytes == 8) {
                // z.q only for flexible CG (plain CG's beta is r.z / rho)
                const double *q = h.opt.precision != AMG_PREC_FP64 ? ctl.q : nullptr;
                timed(h, 3, 0, bytes_post(V.n(), V.op().nnz, V.vbytes, xb) + (q ? 8.0 * V.n() : 0.0), s, [&] {
                    fused = cyc::post_smooth_rz(op_mat<double>(V), V.x.as<double>(), b, dinv_of<double>(V), z0, q,
                                                h.dscal(), h.reduce(), s);
                });
                if (fused) continue;
            }
        }
        relax_post<XT>(h, l, b, l == 0 ? z0 : V.xo.as<XT>(), s);
    }
    return fused;
}

bool vcycle_f64(Hierarchy &h, const double *r, double *z, cudaStream_t s, const CycleCtl &ctl) {
    if (h.opt.precision == AMG_PREC_FP64) return vcycle_impl<double>(h, r, z, s, ctl);
    int64_t n = h.lev[0]->n();
    Level &V0 = *h.lev[0];
    CycleCtl c32 = ctl;
    if (h.nlev() > 1) {
        // FP32 input and its level-0 pre-smooth in one pass
        cyc::to_f32_scaled(n, r, V0.dinv32.as<float>(), h.r32.as<float>(), V0.x.as<float>(), s);
        c32.x0_ready = true;
    } else {
        cyc::convert_vec_from_f64<float>(r, h.r32.as<float>(), n, s);
    }
    vcycle_impl<float>(h, h.r32.as<float>(), h.z32.as<float>(), s, c32);
    if (ctl.fuse_rz) {
        timed(h, 6, 0, 28.0 * n, s, [&] {
            cyc::to_f64_rz((int32_t)n, h.z32.as<float>(), z, r, ctl.q, h.dscal(), h.reduce(), s);
        });
        return true;
    }
    cyc::convert_vec_to_f64<float>(h.z32.as<float>(), z, n, s);
    return false;
}

// ---------------------------------------------------------------------------
// PCG (FP64 recurrences; flexible CG when the cycle is FP32)
//
// One CG step is the body [z = M r; rho, beta; p = z + beta p; q = A_0 p,
// alpha; x += alpha p, r -= alpha q, rr].  With graphs on (and per-kernel
// timing off) the body is captured once into the child graph of a CUDA WHILE
// node whose condition the last kernel sets on the device -- the whole run up
// to the recurrence stop test is one graph launch.  The host then confirms
// convergence with the true residual, exactly as in the eager path.
// ---------------------------------------------------------------------------
namespace {
struct Run {
    int steps = 0, replacements = 0;
    bool converged = false, breakdown = false, diverged = false;
    double rnorm = 0.0;
};

// A_0 in FP64 for the outer PCG: shares level 0's SELL copy when the cycle is
// FP64 and the autotuner chose SELL there
CycMat<double> a0_mat(Hierarchy &h) {
    Level &V = *h.lev[0];
    if (V.vbytes == 8) {
        CycMat<double> m = op_mat<double>(V);
        if (m.variant == AMG_SPMV_SELL32 && !m.sv) m.variant = heuristic_variant(V.A);
        return m;
    }
    CycMat<double> m = make_mat<double>(V.A, V.A.v());
    if (V.variant == AMG_SPMV_SELL32 && V.sv64.ptr) {
        m.variant = AMG_SPMV_SELL32;
        m.nslices = (V.A.nrows + 31) / 32;
        m.soff = V.soff.as<int32_t>();
        m.sw = V.sw.as<int32_t>();
        m.sci = V.sci.ptr ? V.sci.as<int32_t>() : nullptr;
        m.sd = V.sd.ptr ? V.sd.as<int16_t>() : nullptr;
        m.sv = V.sv64.as<double>();
        m.perm = V.sperm.ptr ? V.sperm.as<int32_t>() : nullptr;
        m.max_row = V.max_row;
    } else {
        m.variant = V.variant == AMG_SPMV_SELL32 ? heuristic_variant(V.A) : V.variant;
    }
    return m;
}

void read_scalars(Hierarchy &h, cudaStream_t s) {
    AMG_CUDA(cudaMemcpyAsync(h.h_scal, h.dscal(), sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
}

// the device is idle here (every caller synchronised after its last launch)
void write_scalars(Hierarchy &h, cudaStream_t s) {
    AMG_CUDA(cudaMemcpyAsync(h.dscal(), h.h_scal, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
}

double true_resnorm(Hierarchy &h, const double *b, const double *x, cudaStream_t s) {
    CycMat<double> A0 = a0_mat(h);
    cyc::true_residual(A0, b, x, h.pt.as<double>(), h.dscal(), h.reduce(), s);
    read_scalars(h, s);
    return std::sqrt(h.h_scal->tt);
}

// In FP64 the level-0 pre-smooth x0 = D0^-1 r of the next cycle is written by
// the x, r update; after r is set any other way it is formed here.
void refresh_x0(Hierarchy &h, cudaStream_t s) {
    if (h.opt.precision != AMG_PREC_FP64 || h.nlev() < 2) return;
    Level &V0 = *h.lev[0];
    cyc::scale<double>(V0.n(), h.pr.as<double>(), V0.dinv.as<double>(), V0.x.as<double>(), s);
}

// r = b - A x, p = 0, start = 1 (the next body sets beta = 0); returns ||r||
double pcg_start(Hierarchy &h, const double *b, const double *x, cudaStream_t s) {
    int64_t n = h.lev[0]->n();
    double rn = true_resnorm(h, b, x, s);
    AMG_CUDA(cudaMemcpyAsync(h.pr.ptr, h.pt.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    refresh_x0(h, s);
    AMG_CUDA(cudaMemsetAsync(h.pp.ptr, 0, sizeof(double) * n, s));
    h.h_scal->start = 1;
    h.h_scal->breakdown = 0;
    write_scalars(h, s);
    return rn;
}

// one CG step on the internal x (h.px)
void pcg_body(Hierarchy &h, cudaStream_t s, cudaGraphConditionalHandle handle, bool use_handle) {
    int32_t n = h.lev[0]->n();
    CycMat<double> A0 = a0_mat(h);
    double ap_bytes = (double)A0.nnz * 12 + 4.0 * (n + 1) + 16.0 * n;
    CycleCtl ctl;
    ctl.x0_ready = true;  // pcg_start / replacement / the previous x, r update formed it
    ctl.fuse_rz = true;
    ctl.q = h.pq.as<double>();
    bool fused = vcycle_f64(h, h.pr.as<double>(), h.pz.as<double>(), s, ctl);
    if (!fused)
        timed(h, 6, 0, 24.0 * n, s, [&] {
            cyc::pcg_rz(n, h.pr.as<double>(), h.pz.as<double>(), h.pq.as<double>(), h.dscal(), h.reduce(), s);
        });
    timed(h, 6, 0, 24.0 * n, s, [&] { cyc::pcg_p_update(n, h.pz.as<double>(), h.pp.as<double>(), h.dscal(), s); });
    timed(h, 5, 0, ap_bytes, s, [&] { cyc::pcg_ap(A0, h.pp.as<double>(), h.pq.as<double>(), h.dscal(), h.reduce(), s); });
    bool fp64 = h.opt.precision == AMG_PREC_FP64 && h.nlev() > 1;
    Level &V0 = *h.lev[0];
    timed(h, 6, 0, fp64 ? 64.0 * n : 48.0 * n, s, [&] {
        cyc::pcg_xr_update(n, h.pp.as<double>(), h.pq.as<double>(), h.px.as<double>(), h.pr.as<double>(), h.dscal(),
                           h.reduce(), handle, use_handle, fp64 ? V0.dinv.as<double>() : nullptr,
                           fp64 ? V0.x.as<double>() : nullptr, h.pxs.as<double>(), s);
    });
}

void destroy_graph(Hierarchy &h) {
    if (h.g_update) cudaGraphExecDestroy(h.g_update);
    h.g_update = nullptr;
}

void ensure_graph(Hierarchy &h) {
    if (h.g_update && !h.graph_dirty) return;
    destroy_graph(h);
    if (!h.graph_stream) AMG_CUDA(cudaStreamCreateWithFlags(&h.graph_stream, cudaStreamNonBlocking));
    cudaGraph_t g;
    AMG_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle handle;
    AMG_CUDA(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        AMG_CUDA(e);
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    AMG_CUDA(cudaStreamBeginCaptureToGraph(h.graph_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    bool was = h.timing;
    h.timing = false;
    try {
        pcg_body(h, h.graph_stream, handle, true);
    } catch (...) {
        cudaGraph_t junk;
        cudaStreamEndCapture(h.graph_stream, &junk);
        h.timing = was;
        cudaGraphDestroy(g);
        throw;
    }
    h.timing = was;
    cudaGraph_t captured;
    AMG_CUDA(cudaStreamEndCapture(h.graph_stream, &captured));
    e = cudaGraphInstantiate(&h.g_update, g, 0);
    cudaGraphDestroy(g);
    AMG_CUDA(e);
    h.graph_dirty = false;
}

// Runs up to max_steps CG steps (stopping at the recurrence test, then
// confirming with the true residual; a failed confirmation replaces r).
// divf > 0 adds the divergence test (Section 6: with too many entries
// dropped the method stops converging): windows of k_check steps, counted
// from the run's start and from every replacement; a window whose recurrence
// residual grew by more than divf, or a non-finite residual, stops the run
// with x back at the window's start.
void pcg_iterate(Hierarchy &h, const double *b, double bnorm, double tol, int max_steps, double rnorm_now,
                 double divf, cudaStream_t s, Run &run) {
    run = Run();
    run.rnorm = rnorm_now;
    if (rnorm_now <= tol * bnorm) { run.converged = true; return; }
    bool graph = h.opt.use_graph && !h.timing;
    if (graph) ensure_graph(h);
    double thresh2 = (tol * bnorm) * (tol * bnorm);
    int32_t n = h.lev[0]->n();
    double rn_ws = rnorm_now;
    while (run.steps < max_steps) {
        h.h_scal->its = 0;
        h.h_scal->max_its = max_steps - run.steps;
        h.h_scal->thresh2 = thresh2;
        h.h_scal->divf = divf;
        h.h_scal->kwin = std::max(1, h.opt.k_check);
        h.h_scal->rn_ws = rn_ws;
        h.h_scal->diverged = 0;
        write_scalars(h, s);
        if (graph) {
            AMG_CUDA(cudaGraphLaunch(h.g_update, s));
            read_scalars(h, s);
        } else {
            while (true) {
                pcg_body(h, s, cudaGraphConditionalHandle{}, false);
                read_scalars(h, s);
                const PcgScalars &c = *h.h_scal;
                if (!(c.rr > c.thresh2 && c.its < c.max_its && !c.breakdown && !c.diverged && std::isfinite(c.rr)))
                    break;
            }
        }
        const PcgScalars &sc = *h.h_scal;
        run.steps += sc.its;
        if (sc.diverged) {
            AMG_CUDA(cudaMemcpyAsync(h.px.ptr, h.pxs.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            run.rnorm = sc.rn_ws;
            run.diverged = true;
            return;
        }
        if (sc.breakdown || !std::isfinite(sc.rr)) { run.breakdown = true; return; }
        run.rnorm = std::sqrt(sc.rr);
        if (sc.rr > thresh2) return;  // step budget used up
        double tn = true_resnorm(h, b, h.px.as<double>(), s);
        run.rnorm = tn;
        if (tn <= tol * bnorm) { run.converged = true; return; }
        AMG_CUDA(cudaMemcpyAsync(h.pr.ptr, h.pt.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        refresh_x0(h, s);
        run.replacements++;
        rn_ws = tn;  // the window count restarts with the replaced residual
    }
}
// ---------------------------------------------------------------------------
// Restarted flexible GMRES (FGMRES(m)) with the V-cycle as right
// preconditioner, FP64 recurrences.  Each Arnoldi step is the fixed sequence
// [z = M v_j, store z_j, w = A_0 z, two classical Gram-Schmidt passes,
// Givens rotation, v_{j+1} = w / h_{j+1,j}]; with graphs on, a cycle runs as
// one WHILE-node graph launch whose condition the rotation kernel sets.  The
// host forms x = x0 + Z y at the end of a cycle (or of an Algorithm 5
// window), confirms convergence with the true residual and restarts.
// ---------------------------------------------------------------------------
struct GmRun {
    int steps = 0, replacements = 0;
    bool converged = false, breakdown = false;
    double rnorm = 0.0;
};

GmresArrays gm_arrays(Hierarchy &h) { return gmres_arrays(h.garr.as<double>(), h.gm_m); }
GmresScalars *gm_dsc(Hierarchy &h) { return h.gsc.as<GmresScalars>(); }

void gm_read(Hierarchy &h, cudaStream_t s) {
    AMG_CUDA(cudaMemcpyAsync(h.h_gsc, gm_dsc(h), sizeof(GmresScalars), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
}
void gm_write(Hierarchy &h, cudaStream_t s) {
    AMG_CUDA(cudaMemcpyAsync(gm_dsc(h), h.h_gsc, sizeof(GmresScalars), cudaMemcpyHostToDevice, s));
}

void gm_workspace(Hierarchy &h, cudaStream_t s) {
    const int m = h.opt.restart;
    const int64_t n = h.lev[0]->n();
    if (h.gm_m == m && h.gm_n == n) return;
    h.gV.alloc(sizeof(double) * ((size_t)(m + 1) * n + kPad));
    h.gZ.alloc(sizeof(double) * ((size_t)m * n + kPad));
    h.gx0.alloc(sizeof(double) * (n + kPad));
    h.garr.alloc(sizeof(double) * gmres_array_doubles(m));
    h.gsc.alloc(sizeof(GmresScalars));
    AMG_CUDA(cudaMemsetAsync(h.garr.ptr, 0, h.garr.bytes, s));
    AMG_CUDA(cudaMemsetAsync(h.gsc.ptr, 0, sizeof(GmresScalars), s));
    if (!h.h_gsc) AMG_CUDA(cudaMallocHost(&h.h_gsc, sizeof(GmresScalars)));
    std::memset(h.h_gsc, 0, sizeof(GmresScalars));
    h.gm_m = m;
    h.gm_n = n;
    h.g_gmres_version = -1;
}

void gm_step(Hierarchy &h, cudaStream_t s, cudaGraphConditionalHandle handle, bool use_handle) {
    const int64_t n = h.lev[0]->n();
    const int m = h.gm_m;
    GmresArrays ar = gm_arrays(h);
    GmresScalars *sc = gm_dsc(h);
    double *V = h.gV.as<double>(), *Z = h.gZ.as<double>(), *w = h.pq.as<double>();
    vcycle_f64(h, h.pr.as<double>(), h.pz.as<double>(), s);
    timed(h, 6, 0, 16.0 * n, s, [&] { gm::store_z(n, h.pz.as<double>(), Z, sc, s); });
    CycMat<double> A0 = a0_mat(h);
    const double ap_bytes = (double)A0.nnz * 12 + 4.0 * (n + 1) + 16.0 * n;
    timed(h, 5, 0, ap_bytes, s, [&] { cyc::spmv<double, double>(A0, h.pz.as<double>(), w, false, s); });
    timed(h, 6, 0, 0.0, s, [&] {
        gm::mdot(n, m, V, w, sc, ar, false, s);
        gm::mupdate(n, m, V, w, sc, ar, false, handle, false, s);
        gm::mdot(n, m, V, w, sc, ar, true, s);
        gm::mupdate(n, m, V, w, sc, ar, true, handle, use_handle, s);
        gm::normalize(n, w, V, h.pr.as<double>(), sc, s);
    });
}

void gm_ensure_graph(Hierarchy &h) {
    if (h.g_gmres && h.g_gmres_version == h.version) return;
    if (h.g_gmres) cudaGraphExecDestroy(h.g_gmres);
    h.g_gmres = nullptr;
    if (!h.graph_stream) AMG_CUDA(cudaStreamCreateWithFlags(&h.graph_stream, cudaStreamNonBlocking));
    cudaGraph_t g;
    AMG_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle handle;
    AMG_CUDA(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        AMG_CUDA(e);
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    AMG_CUDA(cudaStreamBeginCaptureToGraph(h.graph_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    bool was = h.timing;
    h.timing = false;
    try {
        gm_step(h, h.graph_stream, handle, true);
    } catch (...) {
        cudaGraph_t junk;
        cudaStreamEndCapture(h.graph_stream, &junk);
        h.timing = was;
        cudaGraphDestroy(g);
        throw;
    }
    h.timing = was;
    cudaGraph_t captured;
    AMG_CUDA(cudaStreamEndCapture(h.graph_stream, &captured));
    e = cudaGraphInstantiate(&h.g_gmres, g, 0);
    cudaGraphDestroy(g);
    AMG_CUDA(e);
    h.g_gmres_version = h.version;
}

// new cycle from the internal x (h.px): r = b - A x, v_0 = r / ||r||,
// g = ||r|| e_1, x0 = x; returns ||r||
double gm_start(Hierarchy &h, const double *b, double thresh, cudaStream_t s) {
    const int64_t n = h.lev[0]->n();
    double rn = true_resnorm(h, b, h.px.as<double>(), s);
    AMG_CUDA(cudaMemcpyAsync(h.gx0.ptr, h.px.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    GmresScalars &c = *h.h_gsc;
    c.m = h.gm_m;
    c.thresh = thresh;
    c.tt = rn * rn;
    gm_write(h, s);
    gm::start(n, h.pt.as<double>(), h.gV.as<double>(), h.pr.as<double>(), gm_dsc(h), gm_arrays(h), s);
    gm_read(h, s);
    return rn;
}

void gm_form_x(Hierarchy &h, cudaStream_t s) {
    const int64_t n = h.lev[0]->n();
    timed(h, 6, 0, 0.0, s, [&] {
        gm::form_x(n, h.gm_m, h.gZ.as<double>(), h.gx0.as<double>(), h.px.as<double>(), gm_dsc(h), gm_arrays(h), s);
    });
}

// Up to max_steps Arnoldi steps from the current cycle; x (h.px) holds the
// iterate on return, the cycle itself goes on unless it converged, broke
// down or was restarted.
void gm_iterate(Hierarchy &h, const double *b, double bnorm, double tol, int max_steps, cudaStream_t s,
                GmRun &run) {
    run = GmRun();
    const double thresh = tol * bnorm;
    GmresScalars &c = *h.h_gsc;
    run.rnorm = c.est;
    if (c.est <= thresh) { run.converged = true; return; }
    const bool graph = h.opt.use_graph && !h.timing;
    if (graph) gm_ensure_graph(h);
    while (run.steps < max_steps) {
        if (c.j == h.gm_m) {  // restart
            gm_form_x(h, s);
            gm_start(h, b, thresh, s);
        }
        const int before = c.its;
        c.max_its = c.its + (max_steps - run.steps);
        gm_write(h, s);
        if (graph) {
            AMG_CUDA(cudaGraphLaunch(h.g_gmres, s));
            gm_read(h, s);
        } else {
            while (true) {
                gm_step(h, s, cudaGraphConditionalHandle{}, false);
                gm_read(h, s);
                if (!(c.est > c.thresh && c.hn > 0.0 && c.j < c.m && c.its < c.max_its && !c.breakdown)) break;
            }
        }
        run.steps += c.its - before;
        if (c.breakdown) {
            gm_form_x(h, s);
            run.breakdown = true;
            return;
        }
        run.rnorm = c.est;
        if (c.est <= thresh || c.happy) {
            gm_form_x(h, s);
            const double tn = gm_start(h, b, thresh, s);
            run.rnorm = tn;
            if (tn <= thresh) { run.converged = true; return; }
            run.replacements++;
        }
    }
    gm_form_x(h, s);
}

amg_status solve_gmres(Hierarchy &h, const double *b, double bnorm, double tol, int max_it, bool adaptive,
                       cudaStream_t s, amg_solve_info *info) {
    gm_workspace(h, s);
    const int64_t n = h.lev[0]->n();
    double *x = h.px.as<double>();
    const double thresh = tol * bnorm;
    h.h_gsc->its = 0;
    if (!adaptive) {
        const double r0 = gm_start(h, b, thresh, s);
        GmRun run;
        gm_iterate(h, b, bnorm, tol, max_it, s, run);
        info->iterations = run.steps;
        info->replacements = run.replacements;
        info->conv_factor = run.steps > 0 ? std::pow(run.rnorm / r0, 1.0 / run.steps) : 0.0;
        return run.converged ? AMG_OK : (run.breakdown ? AMG_BREAKDOWN : AMG_NOT_CONVERGED);
    }
    // Algorithm 5 around GMRES: every k steps the iterate is formed (the
    // cycle goes on) and checked; a reintroduction restarts GMRES with the
    // new preconditioner
    const int k = std::max(1, h.opt.k_check), sl = std::max(1, h.opt.s_levels);
    TmpBuf xs(sizeof(double) * (n + kPad), s);
    double rstart = bnorm;
    gm_start(h, b, thresh, s);
    int total = 0;
    bool converged = false, breakdown = false;
    while (total < max_it) {
        AMG_CUDA(cudaMemcpyAsync(xs.ptr, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        GmRun run;
        gm_iterate(h, b, bnorm, tol, std::min(k, max_it - total), s, run);
        total += run.steps;
        info->replacements += run.replacements;
        double rend = true_resnorm(h, b, x, s);
        if (run.converged || rend <= thresh) { converged = true; break; }
        breakdown = run.breakdown;
        const double factor = run.steps > 0 ? std::pow(rend / rstart, 1.0 / run.steps) : 1.0;
        if (factor > h.opt.rho_max || breakdown) {
            const int cnt = reintroduce(h, sl, s);
            const bool back = !(rend <= rstart);
            if (cnt == 0 && breakdown) {
                if (back) AMG_CUDA(cudaMemcpyAsync(x, xs.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                break;
            }
            if (cnt > 0) {
                info->resets++;
                breakdown = false;
                if (back) {
                    AMG_CUDA(cudaMemcpyAsync(x, xs.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                    rend = rstart;
                }
                gm_start(h, b, thresh, s);
            }
        }
        rstart = rend;
    }
    info->iterations = total;
    return converged ? AMG_OK : (breakdown ? AMG_BREAKDOWN : AMG_NOT_CONVERGED);
}
}  // namespace

amg_status solve(Hierarchy &h, const double *b, double *x_out, double tol, int max_it, bool adaptive,
                 cudaStream_t s, amg_solve_info *info) {
    ensure_workspace(h, s);
    int64_t n = h.lev[0]->n();
    double *x = h.px.as<double>();
    std::memset(info, 0, sizeof(*info));
    std::memset(h.h_scal, 0, sizeof(PcgScalars));
    h.h_scal->flexible = h.opt.precision != AMG_PREC_FP64;
    write_scalars(h, s);
    AMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    double bnorm = true_resnorm(h, b, x, s);
    if (!std::isfinite(bnorm)) throw Error(AMG_ERR_INVALID, "b has a non-finite value");
    amg_status st = AMG_OK;
    if (bnorm == 0.0) {
        info->status = AMG_OK;
    } else if (h.opt.krylov == AMG_KRYLOV_GMRES) {
        st = solve_gmres(h, b, bnorm, tol, max_it, adaptive, s, info);
    } else if (!adaptive) {
        double r0 = pcg_start(h, b, x, s);
        Run run;
        pcg_iterate(h, b, bnorm, tol, max_it, r0, h.opt.div_factor, s, run);
        info->iterations = run.steps;
        info->replacements = run.replacements;
        info->conv_factor = run.steps > 0 ? std::pow(run.rnorm / r0, 1.0 / run.steps) : 0.0;
        st = run.converged ? AMG_OK
           : run.diverged  ? AMG_DIVERGED
           : (run.breakdown ? AMG_BREAKDOWN : AMG_NOT_CONVERGED);
    } else {
        // Algorithm 5: check every k steps; reintroduce on slow convergence
        int k = std::max(1, h.opt.k_check), sl = std::max(1, h.opt.s_levels);
        TmpBuf xs(sizeof(double) * (n + kPad), s);
        double rstart = bnorm;
        double rnow = pcg_start(h, b, x, s);
        int total = 0;
        bool converged = false, breakdown = false, diverged = false;
        const double divf = h.opt.div_factor;
        while (total < max_it) {
            AMG_CUDA(cudaMemcpyAsync(xs.ptr, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            Run run;
            pcg_iterate(h, b, bnorm, tol, std::min(k, max_it - total), rnow, 0.0, s, run);
            total += run.steps;
            info->replacements += run.replacements;
            double rend = true_resnorm(h, b, x, s);
            if (run.converged || rend <= tol * bnorm) { converged = true; break; }
            breakdown = run.breakdown;
            rnow = run.rnorm;
            double factor = run.steps > 0 ? std::pow(rend / rstart, 1.0 / run.steps) : 1.0;
            // grew by more than divf over the window (a non-finite residual included)
            const bool growing = divf > 0.0 && !(rend <= divf * rstart);
            if (factor > h.opt.rho_max || breakdown || growing) {
                int cnt = reintroduce(h, sl, s);
                // back to the checkpoint whenever the residual did not
                // decrease (a non-finite residual included)
                const bool back = !(rend <= rstart);
                if (cnt == 0 && breakdown) {
                    if (back) AMG_CUDA(cudaMemcpyAsync(x, xs.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                    break;
                }
                if (cnt == 0 && growing) {  // diverged, nothing left to reintroduce
                    AMG_CUDA(cudaMemcpyAsync(x, xs.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                    diverged = true;
                    break;
                }
                if (cnt > 0) {
                    info->resets++;
                    breakdown = false;
                    if (back) {
                        AMG_CUDA(cudaMemcpyAsync(x, xs.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                        rend = rstart;
                    }
                    rnow = pcg_start(h, b, x, s);
                }
            }
            rstart = rend;
        }
        info->iterations = total;
        st = converged ? AMG_OK : diverged ? AMG_DIVERGED : (breakdown ? AMG_BREAKDOWN : AMG_NOT_CONVERGED);
    }
    if (bnorm > 0.0) {
        double fin = true_resnorm(h, b, x, s);
        info->final_relres = fin / bnorm;
        if (adaptive) info->conv_factor = info->iterations > 0 ? std::pow(info->final_relres, 1.0 / info->iterations) : 0.0;
    }
    info->status = st;
    if (x_out != x) AMG_CUDA(cudaMemcpyAsync(x_out, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    timing_collect(h);
    return st;
}

}  // namespace amg
