// batch_ops.cuh -- multi-right-hand-side kernels (batch.cu).
//
// K right-hand sides are stored row-major, n x K (entry (i, c) at i*K + c), so
// one matrix entry a_ij is loaded once and applied to the K contiguous values
// of row j.  Every column's arithmetic is the same sequence of operations
// whatever the other columns hold, so a result does not depend on the batch
// it was solved in.
#pragma once
#include "common.cuh"
#include "cycle_ops.cuh"

namespace amg {
namespace bat {

// widths the kernels are compiled for; a batch of k columns uses the
// smallest width >= k (extra columns stay zero and inactive)
int batch_width(int k);

template <typename VT, typename XT>
void pre_smooth_residual(const CycMat<VT> &A, int K, const XT *B, const XT *dinv, XT *X, XT *R, cudaStream_t s);
// OT: type of the output -- XT, or double for the FP32 cycle's finest level,
// which writes the FP64 correction Z directly
template <typename VT, typename XT, typename OT = XT>
void post_smooth(const CycMat<VT> &A, int K, const XT *X, const XT *B, const XT *dinv, OT *XO, cudaStream_t s);
template <typename VT, typename XT>
void spmm(const CycMat<VT> &A, int K, const XT *X, XT *Y, bool accumulate, cudaStream_t s);
template <typename XT>
void coarse_solve(int32_t n, int K, const double *inv, const XT *B, XT *X, cudaStream_t s);

// per-column PCG state on the device
struct ColScalars {
    double *rho, *pq, *alpha, *beta, *rr, *zq, *tt;
    int *active;  // 1: column iterates; 0: frozen (done or empty)
    int *start;   // 1: first iteration after (re)start: beta = 0
};

// Z = M R done by the caller; then:
void rz(int32_t n, int K, const double *R, const double *Z, const double *Q, ColScalars sc, int flexible,
        double *partials, cudaStream_t s);
void p_update(int32_t n, int K, const double *Z, double *P, ColScalars sc, cudaStream_t s);
void ap(const CycMat<double> &A, int K, const double *P, double *Q, ColScalars sc, double *partials,
        cudaStream_t s);
// R32 (FP32 cycles; else nullptr): also written with every column's new
// residual, which the next V-cycle reads -- no separate conversion pass
void xr_update(int32_t n, int K, const double *P, const double *Q, double *X, double *R, float *R32, ColScalars sc,
               double *partials, cudaStream_t s);
// T = B - A X, tt[c] = ||T_c||^2
void residual(const CycMat<double> &A, int K, const double *B, const double *X, double *T, ColScalars sc,
              double *partials, cudaStream_t s);
// column c of an n x K block <- / -> a contiguous n-vector
// (M32: when given, column c of the FP32 copy of M too)
void scatter_column(int32_t n, int K, int c, const double *v, double *M, cudaStream_t s, float *M32 = nullptr);
void gather_column(int32_t n, int K, int c, const double *M, double *v, cudaStream_t s);
void zero_column(int32_t n, int K, int c, double *M, cudaStream_t s);
// R = T for the columns flagged in mask (residual replacement)
void copy_masked_columns(int32_t n, int K, const double *T, double *R, const int *mask, cudaStream_t s,
                         float *R32 = nullptr);

template <typename XT> void to_cycle(const double *src, XT *dst, int64_t n, cudaStream_t s);
template <typename XT> void from_cycle(const XT *src, double *dst, int64_t n, cudaStream_t s);

constexpr int kMaxCols = 64;
constexpr int kBatchReduceBlocks = 8192;

}  // namespace bat
}  // namespace amg
