// tail_ops.cuh -- the coarse end of the V-cycle in one cooperative launch
// (tail.cu).
#pragma once
#include "common.cuh"

namespace amg {

// One level of the fused coarse end, as the kernel reads it.  Matrix values
// of the relaxed operator in VT, transfer values and vectors in XT; P and R
// lead to the next level of the array (absent on the last, coarsest entry).
template <typename VT, typename XT> struct TailLevel {
    int32_t n;
    const int32_t *rp, *ci;
    const VT *v;                       // relaxed operator A_hat_l
    const int32_t *prp, *pci;          // P_l (n x n_{l+1})
    const XT *pv;
    const int32_t *rrp, *rci;          // R_l (n_{l+1} x n)
    const XT *rv;
    const XT *dinv;
    XT *b, *x, *r, *xo;
};

// Grid-barrier state (zeroed once): arrival count, generation, error flag.
struct TailSync {
    unsigned *count;
    unsigned *gen;
    int *err;  // set when a barrier wait ran out (the cycle's result is then invalid)
};

namespace cyc {

// Runs, for the levels in lv[0 .. nl-1] (the last one the coarsest):
// pre-smooth residuals and restrictions down, the dense coarse solve, then
// prolongations and post-smoothing up -- the same steps as the per-level
// kernels, separated by grid barriers.  On entry lv[0].x = D^{-1} b; on exit
// lv[0].xo holds the post-smoothed result.  grid = resident blocks.
template <typename VT, typename XT>
void tail_cycle(const TailLevel<VT, XT> *lv_dev, int nl, const double *coarse_inv, int32_t n_coarse,
                TailSync sync, int grid, cudaStream_t s);
// blocks of the tail kernel that fit on the device at once (cooperative limit)
template <typename VT, typename XT> int tail_grid();

}  // namespace cyc
}  // namespace amg
