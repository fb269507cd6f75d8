// gmres_ops.cuh -- kernels of the restarted, right-preconditioned (flexible)
// GMRES outer solver (gmres.cu).  The paper solves with GMRES where full
// lumping (Algorithm 3) can cost the preconditioner its definiteness.
#pragma once
#include "common.cuh"

namespace amg {

// Device-side state of one GMRES run.  The basis size of the current cycle
// (j) lives here, so one captured Arnoldi step serves every j.
struct GmresScalars {
    int j;          // Arnoldi steps in the current cycle (basis v_0..v_j)
    int its;        // steps in this run
    int max_its;    // the graph loop stops at this count
    int m;          // restart length
    int breakdown;  // a non-finite or singular Hessenberg column
    int happy;      // ||w|| = 0: the Krylov space is invariant
    int reorth;     // the step's second Gram-Schmidt pass runs
    int pad;
    double thresh;  // tol ||b||: stop when the residual estimate reaches it
    double est;     // |g_j|, the residual norm of the cycle's current iterate
    double hn;      // ||w|| of the last step (h_{j+1,j})
    double tt;      // ||b - A x||^2 of the last true residual
    double ww;      // ||w||^2 before orthogonalisation
    double wn2;     // ||w||^2 after the first pass
};

// Device arrays of the Hessenberg least-squares problem (doubles).
struct GmresArrays {
    double *H;    // (m + 1) x m, H[i * m + c]
    double *cs, *sn;  // Givens rotations, m each
    double *g;    // rotated right-hand side, m + 1
    double *y;    // solution of R y = g, m
    double *hc, *hc2;  // the two Gram-Schmidt coefficient passes, m + 1 each
    double *part;      // per-block partials, (m + 2) x kGmresMaxBlocks (row m + 1: ||w||^2)
};
constexpr int kGmresMaxBlocks = 2048;
// doubles needed for GmresArrays with restart length m
inline size_t gmres_array_doubles(int m) {
    return (size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + m + 2 * (size_t)(m + 1) +
           (size_t)(m + 2) * kGmresMaxBlocks;
}
GmresArrays gmres_arrays(double *base, int m);

namespace gm {

// blocks of the column-parallel kernels (a resident wave, capped)
int dot_blocks(int64_t n);
// hc[i] = V_i . w for i = 0..j (device j) and ww = w . w; second pass (only
// when sc->reorth): hc2[i] = V_i . w
void mdot(int64_t n, int m, const double *V, const double *w, GmresScalars *sc, GmresArrays ar, bool second,
          cudaStream_t s);
// First pass: w -= sum_{i<=j} hc[i] V_i with ||w||^2, then the decision of
// the second pass ("twice is enough": reorthogonalise only when the pass
// removed more than half of ||w||^2, i.e. ||w'|| < ||w|| / sqrt 2).  Second
// pass (when sc->reorth): w -= sum hc2[i] V_i with ||w||^2; then the step
// finisher: H column j = hc + hc2, Givens rotation, residual estimate,
// j += 1, and the WHILE condition when `use_handle`.
void mupdate(int64_t n, int m, const double *V, double *w, GmresScalars *sc, GmresArrays ar, bool second,
             cudaGraphConditionalHandle handle, bool use_handle, cudaStream_t s);
// v_j = w / hn into V (row j) and into `next` (the next cycle input)
void normalize(int64_t n, const double *w, double *V, double *next, const GmresScalars *sc, cudaStream_t s);
// Z row j = z (before the step finisher increments j)
void store_z(int64_t n, const double *z, double *Z, const GmresScalars *sc, cudaStream_t s);
// new cycle: v_0 = r / beta into V and next, g = beta e_1, j = 0 (beta from sc->tt)
void start(int64_t n, const double *r, double *V, double *next, GmresScalars *sc, GmresArrays ar, cudaStream_t s);
// x = x0 + Z y with R y = g over the cycle's j columns
void form_x(int64_t n, int m, const double *Z, const double *x0, double *x, GmresScalars *sc, GmresArrays ar,
            cudaStream_t s);

}  // namespace gm
}  // namespace amg
