// cycle_ops.cuh -- solve-phase kernels (cycle.cu): SpMV-based relaxation,
// restriction, interpolation, coarse solve, PCG vector kernels.
#pragma once
#include "common.cuh"

namespace amg {

// SELL slice height of an SpMV variant (32, 16, 8), 0 for the CSR variants.
// A slice of C rows is read by one warp with 32 / C lanes per row.
inline int sell_height(int variant) {
    return variant == AMG_SPMV_SELL32 ? 32 : variant == AMG_SPMV_SELL16 ? 16 : variant == AMG_SPMV_SELL8 ? 8 : 0;
}

// A row-partitioned operator (amg_partition): its columns in block-local
// numbering, and where each block's ghost values come from.
struct PartView {
    int parts = 0;                  // 0: not partitioned
    const int32_t *cext = nullptr;  // per stored entry: owned column j - col0[p], or nloc + ghost index
    const int32_t *row0 = nullptr;  // parts + 1: first row of each block
    const int32_t *col0 = nullptr;  // parts + 1: first owned column of each block
    const int32_t *goff = nullptr;  // parts + 1: first ghost of each block in gbuf
    const int32_t *gcol = nullptr;  // global column of each ghost
    double *gbuf = nullptr;         // ghost values, written by the exchange
    int64_t nghost = 0;
};

// A matrix as the cycle kernels read it: CSR in value type VT, plus an
// optional SELL-C copy (slices of C rows, column-major inside a slice).
template <typename VT> struct CycMat {
    int32_t nrows = 0, ncols = 0;
    int64_t nnz = 0;
    const int32_t *rp = nullptr, *ci = nullptr;
    const VT *v = nullptr;
    int32_t nslices = 0;
    const int32_t *soff = nullptr, *sw = nullptr, *sci = nullptr;
    const int16_t *sd = nullptr;    // SELL column as int16 offset from the row (replaces sci when set)
    const int32_t *perm = nullptr;  // SELL position -> row (null: identity)
    const VT *sv = nullptr;
    int32_t max_row = 0;  // most stored entries of a row (0: not known)
    int variant = AMG_SPMV_CSR4;
    int sell_c = 32;      // slice height of the SELL copy
    bool stream = false;  // stored entries larger than kStreamBytes: the SELL kernels load them
                          // with the evict-first policy (read once per pass, they would only
                          // push the vectors and the smaller levels out of L1 and L2)
    PartView part;        // set when the hierarchy runs row-partitioned (FP64 only)
};
constexpr int64_t kStreamBytes = 48ll << 20;

// Device-side scalars of one PCG run.
struct PcgScalars {
    double rho;      // r . z
    double pq;       // p . A p
    double alpha, beta;
    double rr;       // r . r after the update
    double zq;       // z . q (flexible CG)
    double tt;       // ||b - A x||^2 of the last true-residual check
    double thresh2;  // (tol ||b||)^2: the recurrence stop test
    int flexible;
    int start;       // 1: next r.z starts a (re)started run (beta = 0)
    int its;         // CG steps taken
    int max_its;     // the graph loop stops at this count
    int breakdown;   // p.Ap <= 0 or r.z <= 0 was met
    int diverged;    // the residual grew by more than divf over a window
    // divergence test (off when divf == 0): windows of kwin steps counted
    // by `its`; at a window's end sqrt(rr) is compared with rn_ws, the norm
    // at its start, and x at the window's start is kept in the checkpoint
    double divf;
    double rn_ws;
    int kwin;
    int pad;
};

// Deterministic reduction workspace: per-block partials + arrival counter.
struct Reduce {
    double *partials = nullptr;   // 4 * kMaxReduceBlocks (per block)
    unsigned *counter = nullptr;  // [0]: groups done; [1 + g]: blocks done in group g (257 used)
    double *gpartials = nullptr;  // 4 * 256 (per group of 256 blocks)
};
constexpr int kMaxReduceBlocks = 65536;

namespace cyc {

int threads_per_row(int variant);

// relaxation and transfers (XT = vector type, VT = matrix value type)
template <typename VT, typename XT>
void pre_smooth_residual(const CycMat<VT> &A, const XT *b, const XT *dinv, XT *x, XT *r, cudaStream_t s);
template <typename VT, typename XT>
void post_smooth(const CycMat<VT> &A, const XT *x, const XT *b, const XT *dinv, XT *xo, cudaStream_t s);
template <typename VT, typename XT>
void spmv(const CycMat<VT> &A, const XT *x, XT *y, bool accumulate, cudaStream_t s);
// restriction with the coarse pre-smooth folded in: y = A x, xs = d .* y
template <typename VT, typename XT>
void spmv_scaled(const CycMat<VT> &A, const XT *x, const XT *d, XT *y, XT *xs, cudaStream_t s);
// pre-smooth residual when x = D^{-1} b is already stored: r = b - A x
template <typename VT, typename XT>
void residual_from_x(const CycMat<VT> &A, const XT *b, const XT *x, XT *r, cudaStream_t s);

// coarsest level: x = inv * b (dense, FP64 inverse)
template <typename XT>
void coarse_solve(int32_t n, const double *inv, const XT *b, XT *x, cudaStream_t s);

// PCG (FP64)
void pcg_p_update(int32_t n, const double *z, double *p, const PcgScalars *sc, cudaStream_t s);
void pcg_ap(const CycMat<double> &A, const double *p, double *q, PcgScalars *sc, Reduce red, cudaStream_t s);
// x += alpha p, r -= alpha q, rr, its += 1; with a graph handle, the WHILE
// condition is set to continue while rr > thresh2, its < max_its, no
// breakdown and no divergence.  With the divergence test on (sc->divf > 0),
// a step that starts a window first copies x to xs.
void pcg_xr_update(int32_t n, const double *p, const double *q, double *x, double *r, PcgScalars *sc,
                   Reduce red, cudaGraphConditionalHandle handle, bool use_handle, const double *dinv0,
                   double *x0, double *xs, cudaStream_t s);
// level-0 post-smoothing that also forms rho = r.z and, when q is given
// (flexible CG), z.q, and beta: z is the output, r = b the cycle input.
// Returns false (nothing launched) for an empty level.
bool post_smooth_rz(const CycMat<double> &A, const double *x, const double *b, const double *dinv, double *z,
                    const double *q, PcgScalars *sc, Reduce red, cudaStream_t s);
// z = (double) z32 and rho = r.z, z.q (FP32 cycles)
void to_f64_rz(int32_t n, const float *z32, double *z, const double *r, const double *q, PcgScalars *sc, Reduce red,
               cudaStream_t s);
// out = a .* d (pre-smooth from zero)
template <typename XT> void scale(int64_t n, const XT *a, const XT *d, XT *out, cudaStream_t s);
// dst = (float) src and xdst = dst .* d (FP32 cycle input with its pre-smooth)
void to_f32_scaled(int64_t n, const double *src, const float *d, float *dst, float *xdst, cudaStream_t s);
void pcg_rz(int32_t n, const double *r, const double *z, const double *q, PcgScalars *sc, Reduce red,
            cudaStream_t s);
// t = b - A x, sc->tt = ||t||^2; if `replace`, r = t
void true_residual(const CycMat<double> &A, const double *b, const double *x, double *t, PcgScalars *sc,
                   Reduce red, cudaStream_t s);

// precision conversion and SELL construction
template <typename VT> void convert_values(const double *src, VT *dst, int64_t n, cudaStream_t s);
template <typename XT> void convert_vec_from_f64(const double *src, XT *dst, int64_t n, cudaStream_t s);
template <typename XT> void convert_vec_to_f64(const XT *src, double *dst, int64_t n, cudaStream_t s);
// SELL-C layout (C = 32, 16 or 8 rows per slice): slice widths (a multiple
// of 32 / C, the lanes that share a row) and offsets, optionally over rows
// sorted by length (descending) inside windows of kSellSigma rows (perm:
// position -> row); returns the padded entry count.  sw and soff hold
// ceil(n / C) + 1 entries.
constexpr int kSellSigma = 1024;
int64_t sell_layout(int32_t n, const int32_t *rp, int32_t *perm, int32_t *soff, int32_t *sw, cudaStream_t s,
                    int C = 32);
template <typename VT>
void sell_fill(int32_t n, const int32_t *rp, const int32_t *ci, const VT *v, const int32_t *perm,
               const int32_t *soff, const int32_t *sw, int32_t *sci, VT *sv, cudaStream_t s, int16_t *sd = nullptr,
               int C = 32);
// max over stored entries of |column - row| (square operators), for the int16 SELL offsets;
// *max_row (if given) receives the longest row
int32_t max_col_offset(int32_t n, const int32_t *rp, const int32_t *ci, cudaStream_t s, int32_t *max_row = nullptr);

}  // namespace cyc
}  // namespace amg
