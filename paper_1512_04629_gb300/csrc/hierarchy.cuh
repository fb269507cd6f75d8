// hierarchy.cuh -- the device-resident AMG hierarchy and its drivers.
#pragma once

#include <memory>
#include <vector>

#include <map>

#include "batch_ops.cuh"
#include "common.cuh"
#include "cycle_ops.cuh"
#include "gmres_ops.cuh"

namespace amg {

// SELL-32 copy of a CSR operator (slices of 32 rows stored column-major;
// rows length-sorted within windows when that cuts the padding).
struct SellCopy {
    DevBuf soff, sw, sci, sv, perm;
    int64_t entries = 0;
    int c = 32;  // slice height
    void release() {
        soff.release(); sw.release(); sci.release(); sv.release(); perm.release();
        entries = 0;
    }
};

// One operator split into row blocks (amg_partition): the device copy of its
// halo plan and its ghost buffer; recv (parts x parts, values block p
// receives from block q) stays on the host for the statistics.
struct PartOp {
    DevBuf cext, gcol, bounds, gbuf;  // bounds: int32 row0 | col0 | goff, parts + 1 each
    int parts = 0;
    int64_t nghost = 0;
    std::vector<int64_t> recv;
    PartView view() const {
        PartView v;
        v.parts = parts;
        v.cext = cext.as<int32_t>();
        v.row0 = bounds.as<int32_t>();
        v.col0 = v.row0 + parts + 1;
        v.goff = v.col0 + parts + 1;
        v.gcol = gcol.as<int32_t>();
        v.gbuf = gbuf.as<double>();
        v.nghost = nghost;
        return v;
    }
};

// One level l of the hierarchy.  A is the retained Galerkin operator
// (Algorithm 4 keeps it so Algorithm 5 can reintroduce entries); H is the
// relaxed operator Ahat_l (an alias of A where nothing is dropped).
struct Level {
    DevCSR A;
    DevBuf diagpos, tpos;  // int32 per row / per entry of A
    DevBuf strong;         // uint8 per entry of A (levels that were coarsened)
    DevBuf inM, keep;      // uint8 per entry of A
    DevBuf inM_hybrid;     // Hybrid Galerkin: M from the sparsified operator of level l-1
    DevBuf cf;             // int8 per row (coarsened levels)
    DevBuf cmap, cpts;     // int32
    DevCSR P, R;           // interpolation and restriction (not on the coarsest level)
    DevCSR H;              // sparsified operator when it differs from A
    bool h_alias = true;
    double gamma = 0.0;
    DevBuf l1, dinv;       // FP64 ell1 diagonal and its inverse

    // cycle representation (precision-dependent copies)
    int vbytes = 8;        // bytes per value of the relaxed operator in the cycle
    DevBuf hv32, hv16;     // FP32 / BF16 values of the relaxed operator
    DevBuf pv32, rv32;     // FP32 values of P and R
    DevBuf dinv32;
    DevBuf soff, sw, sci, sv;  // SELL-C copy of the relaxed operator (C = sell_c)
    DevBuf sd;                 // its columns as int16 offsets from the row (instead of sci) when they fit
    DevBuf sperm;              // SELL position -> row when rows are length-sorted
    DevBuf sv64;               // level 0 in FP32 modes: FP64 values in the same SELL layout (outer PCG)
    int64_t sell_entries = 0;
    int sell_c = 32;
    int32_t max_row = 0;       // longest row of the relaxed operator (kernel choice)
    SellCopy psell, rsell;     // SELL copies of P and R (cycle precision) when they win the trial
    int variant = AMG_SPMV_CSR4, variant_p = AMG_SPMV_CSR2, variant_r = AMG_SPMV_CSR8;
    bool pr_tuned = false;  // transfer-operator variants chosen by timed trials
    // row-partitioned execution (amg_partition): block boundaries of this
    // level's rows, the plans of the relaxed operator, P and R, and the
    // receive counts of the Galerkin A_l (statistics only)
    std::vector<int64_t> prow0;
    std::unique_ptr<PartOp> part_h, part_p, part_r;
    std::vector<int64_t> recv_galerkin;

    // work vectors in the cycle precision (b, x, r, post-smoothed output)
    DevBuf b, x, r, xo;

    const DevCSR &op() const { return h_alias ? A : H; }
    int32_t n() const { return A.nrows; }
};

struct Timing {
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
};
constexpr int kTimingKinds = 16;
constexpr int kMaxLevels = 64;

struct PendingEvent {
    int kind, level;
    double bytes;
    cudaEvent_t a, b;
};

// Workspace of a K-column (multi-right-hand-side) solve: per-level cycle
// vectors (n_l x K, cycle precision), FP64 PCG blocks (n_0 x K) and the
// per-column scalars.
struct BatchWS {
    int K = 0;
    std::vector<DevBuf> b, x, r, xo;
    DevBuf B, X, R, Z, P, Q, T;
    DevBuf R32, Z32;
    DevBuf sc_buf, partials, mask;
    bat::ColScalars sc{};
    double *h_d = nullptr;  // pinned: rho, pq, alpha, beta, rr, zq, tt (K each)
    int *h_i = nullptr;     // pinned: active, start, mask (K each)
    cudaGraphExec_t graph = nullptr;  // one captured iteration
    int graph_version = -1;
    ~BatchWS();
    double *h_rho() { return h_d; }
    double *h_pq() { return h_d + K; }
    double *h_rr() { return h_d + 4 * K; }
    double *h_tt() { return h_d + 6 * K; }
    int *h_active() { return h_i; }
    int *h_start() { return h_i + K; }
    int *h_mask() { return h_i + 2 * K; }
};

struct Hierarchy {
    IdleRelease idle_release;  // first member: destroyed after every buffer below
    amg_options opt{};
    int device = 0;
    int parts = 1;  // row blocks of every level (amg_partition); 1 = not partitioned
    std::vector<std::unique_ptr<Level>> lev;
    DevBuf coarse_inv;  // FP64 dense inverse of the coarsest relaxed operator
    int32_t coarse_n = 0;

    // FP64 PCG workspace
    DevBuf pb, px, pr, pz, pp, pq, pt;
    DevBuf pxs;  // x at the start of the current divergence-test window
    DevBuf scal;          // PcgScalars
    DevBuf partials, counter;
    PcgScalars *h_scal = nullptr;  // pinned
    DevBuf z32, r32;      // FP32 V-cycle input/output in the FP32 modes
    int64_t ws_n = -1;

    // per-kernel timing
    bool timing = false;
    Timing timers[kTimingKinds][kMaxLevels];
    std::vector<PendingEvent> pending;
    std::vector<cudaEvent_t> event_pool;

    // CUDA graphs of the PCG iteration halves (captured per stream)
    cudaGraphExec_t g_update = nullptr, g_precond = nullptr;
    cudaStream_t graph_stream = nullptr;
    bool graph_dirty = true;
    int version = 0;  // bumped whenever the cycle's buffers or operators change

    std::map<int, std::unique_ptr<BatchWS>> batch;

    // GMRES workspace (the first GMRES solve allocates it): basis V
    // ((m + 1) x n), preconditioned vectors Z (m x n), the cycle's starting
    // x, the Hessenberg arrays and the device scalars
    DevBuf gV, gZ, gx0, garr, gsc;
    int gm_m = 0;
    int64_t gm_n = -1;
    GmresScalars *h_gsc = nullptr;  // pinned
    cudaGraphExec_t g_gmres = nullptr;  // one captured Arnoldi step in a WHILE loop
    int g_gmres_version = -1;

    ~Hierarchy();
    int nlev() const { return (int)lev.size(); }
    Reduce reduce() {
        return Reduce{partials.as<double>(), counter.as<unsigned>(), partials.as<double>() + 4 * kMaxReduceBlocks};
    }
    PcgScalars *dscal() { return scal.as<PcgScalars>(); }
};

// views of a level in the cycle precision
template <typename VT> inline CycMat<VT> make_mat(const DevCSR &M, const VT *vals) {
    CycMat<VT> m;
    m.nrows = M.nrows;
    m.ncols = M.ncols;
    m.nnz = M.nnz;
    m.rp = M.rp();
    m.ci = M.ci();
    m.v = vals;
    m.stream = M.nnz * (int64_t)(sizeof(VT) + sizeof(int32_t)) > kStreamBytes;
    return m;
}

template <typename VT> inline CycMat<VT> op_mat(const Level &V) {
    const DevCSR &M = V.op();
    const VT *vals;
    if constexpr (sizeof(VT) == 8) vals = reinterpret_cast<const VT *>(M.v());
    else if constexpr (sizeof(VT) == 4) vals = V.hv32.as<VT>();
    else vals = V.hv16.as<VT>();
    CycMat<VT> m = make_mat<VT>(M, vals);
    if (V.sv.ptr) {
        m.sell_c = V.sell_c;
        m.nslices = (M.nrows + V.sell_c - 1) / V.sell_c;
        m.soff = V.soff.as<int32_t>();
        m.sw = V.sw.as<int32_t>();
        m.sci = V.sci.ptr ? V.sci.as<int32_t>() : nullptr;
        m.sd = V.sd.ptr ? V.sd.as<int16_t>() : nullptr;
        m.sv = V.sv.as<VT>();
        m.perm = V.sperm.ptr ? V.sperm.as<int32_t>() : nullptr;
    }
    m.max_row = V.max_row;
    m.variant = V.variant;
    if constexpr (sizeof(VT) == 8)
        if (V.part_h) m.part = V.part_h->view();
    return m;
}

template <typename VT> inline void attach_sell(CycMat<VT> &m, const SellCopy &S) {
    if (!S.sv.ptr) return;
    m.sell_c = S.c;
    m.nslices = (m.nrows + S.c - 1) / S.c;
    m.soff = S.soff.as<int32_t>();
    m.sw = S.sw.as<int32_t>();
    m.sci = S.sci.as<int32_t>();
    m.sv = S.sv.as<VT>();
    m.perm = S.perm.ptr ? S.perm.as<int32_t>() : nullptr;
}

template <typename XT> inline CycMat<XT> p_mat(const Level &V) {
    const XT *vals;
    if constexpr (sizeof(XT) == 8) vals = reinterpret_cast<const XT *>(V.P.v());
    else vals = V.pv32.as<XT>();
    CycMat<XT> m = make_mat<XT>(V.P, vals);
    attach_sell<XT>(m, V.psell);
    m.variant = V.variant_p;
    if constexpr (sizeof(XT) == 8)
        if (V.part_p) m.part = V.part_p->view();
    return m;
}

template <typename XT> inline CycMat<XT> r_mat(const Level &V) {
    const XT *vals;
    if constexpr (sizeof(XT) == 8) vals = reinterpret_cast<const XT *>(V.R.v());
    else vals = V.rv32.as<XT>();
    CycMat<XT> m = make_mat<XT>(V.R, vals);
    attach_sell<XT>(m, V.rsell);
    m.variant = V.variant_r;
    if constexpr (sizeof(XT) == 8)
        if (V.part_r) m.part = V.part_r->view();
    return m;
}

template <typename XT> inline const XT *dinv_of(const Level &V) {
    if constexpr (sizeof(XT) == 8) return reinterpret_cast<const XT *>(V.dinv.ptr);
    else return V.dinv32.as<XT>();
}

// row-partitioned execution (partition.cu): re-plan the relaxed operator of
// level l after it changed (sparsify / reintroduce)
void replan_relaxation(Hierarchy &h, int l, cudaStream_t s);

// drivers (hierarchy.cu)
// Algorithm 1; with method AMG_METHOD_NONGALERKIN each new coarse operator is
// thinned (gamma convention of amg_setup) before it is coarsened further.
class SetupPipeline;
void build_galerkin(Hierarchy &h, const DevCSR &A0in, cudaStream_t s, const double *gamma = nullptr,
                    int n_gamma = 0, SetupPipeline *pipe = nullptr);
// build_galerkin, the sparsification of every level and its cycle data; plain
// Sparse Galerkin setups overlap the last two with the coarsening
void setup_hierarchy(Hierarchy &h, cudaStream_t s, const double *gamma, int n_gamma);
void assemble_levels(Hierarchy &h, std::vector<DevCSR> &A, std::vector<DevCSR> &P,
                     const std::vector<std::vector<int8_t>> &cf,
                     const std::vector<std::vector<uint8_t>> &inM, cudaStream_t s);
void apply_gammas(Hierarchy &h, const double *gamma, int n_gamma, cudaStream_t s);
void resparsify_level(Hierarchy &h, int l, cudaStream_t s);
void prepare_cycle(Hierarchy &h, cudaStream_t s, const std::vector<int> &levels);
void ensure_workspace(Hierarchy &h, cudaStream_t s);
int reintroduce(Hierarchy &h, int s_levels, cudaStream_t s);
// V-cycle options: x0_ready -- level 0's x already holds D0^-1 r (FP64);
// fuse_rz -- the last pass also forms rho = r.z and z.q (q given) and beta.
struct CycleCtl {
    bool x0_ready = false;
    bool fuse_rz = false;
    const double *q = nullptr;
};
// z = M r; returns true when rho / beta were formed in the cycle (fuse_rz)
bool vcycle_f64(Hierarchy &h, const double *r, double *z, cudaStream_t s, const CycleCtl &ctl = CycleCtl());
amg_status solve(Hierarchy &h, const double *b_dev, double *x_dev, double tol, int max_it, bool adaptive,
                 cudaStream_t s, amg_solve_info *info);
void timing_collect(Hierarchy &h);

// multi-right-hand-side solves (batch_driver.cu)
BatchWS &batch_workspace(Hierarchy &h, int K, cudaStream_t s);
void batch_vcycle(Hierarchy &h, BatchWS &w, cudaStream_t s);
void batch_iteration(Hierarchy &h, BatchWS &w, cudaStream_t s);  // async; scalars copied to w.h_d
void batch_true_residual(Hierarchy &h, BatchWS &w, cudaStream_t s);  // async; tt copied to w.h_d
void batch_push_flags(BatchWS &w, cudaStream_t s);
amg_status solve_batch(Hierarchy &h, int k, const double *B, double *X, bool on_device, double tol, int max_it,
                       cudaStream_t s, amg_solve_info *infos);
double level_cycle_bytes(const Hierarchy &h, int l);

}  // namespace amg

// the opaque handle of the C ABI
struct amg_hierarchy {
    amg::Hierarchy h;
};
