/*
 * amg_oracle.h -- plain FP64 CPU oracle of the sparsified-AMG hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * It follows, in order and notation, Bienz, Falgout, Gropp, Olson, Schroder,
 * "Reducing Parallel Communication in Algebraic Multigrid through
 * Sparsification" (arXiv:1512.04629):
 *   Algorithm 1 (amg_setup), Algorithm 2 (amg_solve, the V-cycle),
 *   Algorithm 3 (sparsify: minimal pattern M, drop test, symmetric N) with its
 *   own loop (full lumping to strong neighbours) and the diagonal-lumping loop
 *   of Algorithm 3b, Algorithm 4 (Sparse and Hybrid Galerkin), Algorithm 1's
 *   non-Galerkin option, Algorithm 5 (adaptive_solve), PCG (Section 5.5 /
 *   Section 6) and restarted GMRES (Section 5.3).
 * Where the paper leaves a choice open (strength formula, PMIS details, direct
 * interpolation, stop rule, ell1-Jacobi, the garbled lines of Algorithms 4 and
 * 5) the reading taken is stated at the function that implements it.
 *
 * Floating point: every sum runs sequentially in increasing column order and
 * the file is compiled with -ffp-contract=off, so each result is the plain
 * IEEE-754 double evaluation of the formula as written.
 *
 * Parity status: every function here is pinned by a CPU test against closed
 * forms, dense brute force or the paper's worked example (Example 1); the
 * iteration counts of PCG are pinned only through those parts ("parity
 * unpinned" against the paper, whose convergence plots are not printed).
 */
#ifndef AMG_ORACLE_H
#define AMG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* CSR matrix: nrows x ncols, int32 indices, columns increasing in each row. */
typedef struct {
    int32_t nrows, ncols, nnz;
    int32_t *rowptr; /* nrows + 1 */
    int32_t *col;    /* nnz */
    double *val;     /* nnz */
} orc_csr;

typedef struct {
    int32_t iterations;   /* number of products with A_0 p */
    int32_t status;       /* 0 converged, 4 not converged, 5 diverged, 6 breakdown */
    int32_t resets;       /* adaptive: number of reintroductions (PCG restarts) */
    int32_t replacements; /* residual replacements after a failed true-residual check */
    double final_relres;  /* ||b - A x|| / ||b|| at exit (true residual) */
    double conv_factor;   /* (||r_end|| / ||r_0||)^(1 / iterations) */
} orc_info;

typedef struct orc_hier orc_hier;

/* One check window of Algorithm 5 (orc_adaptive_solve_ex's trace). */
typedef struct {
    int32_t steps;  /* PCG steps taken in the window */
    int32_t action; /* ORC_WIN_* below */
    double rstart;  /* true residual norm at the window's start */
    double rend;    /* true residual norm at its end (a restart from the
                       window's start then begins from rstart again) */
    double factor;  /* (rend / rstart)^(1 / steps), before any restart */
} orc_window;
enum {
    ORC_WIN_CONTINUE = 0,       /* factor <= rho_max: the Krylov run goes on */
    ORC_WIN_RESTART_HERE = 1,   /* reintroduced; PCG restarts from the current x */
    ORC_WIN_RESTART_BACK = 2,   /* reintroduced; the residual grew: restart from the window's x */
    ORC_WIN_CONVERGED = 3,      /* tolerance reached */
    ORC_WIN_NOTHING_LEFT = 4,   /* slow, but every gamma is 0 already: the run goes on */
    ORC_WIN_BREAKDOWN_STOP = 5, /* breakdown with nothing to reintroduce; x kept */
    ORC_WIN_BREAKDOWN_BACK = 6, /* the same, x back to the window's start */
    ORC_WIN_DIVERGED = 7        /* grew by more than divf, nothing to reintroduce */
};

/* ---- building blocks (Section 2, Algorithm 1) ---- */
void orc_strength(const orc_csr *A, double theta, uint8_t *strong);
int orc_pmis(const orc_csr *A, const uint8_t *strong, uint64_t seed, int32_t level, int8_t *cf);
orc_csr *orc_direct_interp(const orc_csr *A, const uint8_t *strong, const int8_t *cf);
orc_csr *orc_transpose(const orc_csr *M);
orc_csr *orc_spgemm(const orc_csr *A, const orc_csr *B);
int orc_minimal_pattern(const orc_csr *Ac, const orc_csr *AP, const int8_t *cf, uint8_t *inM);
orc_csr *orc_sparsify_diag(const orc_csr *Ac, const uint8_t *inM, double gamma, uint8_t *keep);
orc_csr *orc_sparsify_full(const orc_csr *Ac, const uint8_t *inM, double gamma, double theta,
                           uint8_t *keep);
void orc_l1_diag(const orc_csr *A, double *d);
int orc_cholesky(int32_t n, double *a);
void orc_chol_solve(int32_t n, const double *L, const double *b, double *x);
int orc_lu(int32_t n, double *a, int32_t *piv);
void orc_lu_solve(int32_t n, const double *LU, const int32_t *piv, const double *b, double *x);
void orc_spmv(const orc_csr *A, const double *x, double *y);
double orc_uniform_weight(uint64_t seed, int32_t level, int64_t i);
int orc_gamma_schedule(double *gamma, int32_t nlev, int32_t s, double gamma_min, int32_t *changed);

/* ---- hierarchy (Algorithms 1, 2, 4, 5) ---- */
orc_hier *orc_setup(const orc_csr *A0, double theta, int32_t max_size, int32_t max_levels,
                    uint64_t seed, int32_t *status);
/* Algorithm 1 with the non-Galerkin sparsify inside the loop (the paper's
 * comparator): gamma[l] thins the operator of level l as soon as it is formed
 * (gamma[0] = 0); lump as orc_sparsify_opts.  Nothing Galerkin is retained:
 * orc_sparsify* and orc_reintroduce refuse such a hierarchy. */
orc_hier *orc_setup_nongalerkin(const orc_csr *A0, double theta, int32_t max_size, int32_t max_levels,
                                uint64_t seed, const double *gamma, int32_t ngamma, int32_t lump,
                                int32_t *status);
int orc_sparsify(orc_hier *h, const double *gamma, int32_t ngamma);
/* method 0: Sparse Galerkin (M from the Galerkin A_{l-1}); 1: Hybrid Galerkin
 * (M from the sparsified Ahat_{l-1}, levels processed in order). */
int orc_sparsify_method(orc_hier *h, const double *gamma, int32_t ngamma, int32_t method);
/* the same with lump 0: diagonal lumping (Algorithm 3b), 1: full lumping to
 * strong neighbours (Algorithm 3's own loop) */
int orc_sparsify_opts(orc_hier *h, const double *gamma, int32_t ngamma, int32_t method, int32_t lump);
int orc_reintroduce(orc_hier *h, int32_t s, double gamma_min, int32_t *changed);
int orc_vcycle(orc_hier *h, const double *b, double *x);
int orc_pcg(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, orc_info *info);
/* PCG with the divergence test made explicit: windows of kwin steps, growth
 * factor divf (0: off, else >= 1); orc_pcg uses kwin = 3, divf = 1e3. */
int orc_pcg_ex(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, int32_t kwin,
               double divf, orc_info *info);
int orc_adaptive_solve(orc_hier *h, const double *b, double *x, double tol, int32_t max_it,
                       int32_t k, int32_t s, double gamma_min, double rho_max, orc_info *info);
/* Algorithm 5 with its divergence factor (orc_adaptive_solve: 1e3) and an
 * optional trace of the check windows: *ntrace receives the number of
 * windows, of which the first cap are written to trace. */
int orc_adaptive_solve_ex(orc_hier *h, const double *b, double *x, double tol, int32_t max_it,
                          int32_t k, int32_t s, double gamma_min, double rho_max, double divf,
                          orc_window *trace, int32_t cap, int32_t *ntrace, orc_info *info);
/* restarted right-preconditioned (flexible) GMRES with M = one V-cycle, the
 * same unpreconditioned on a plain CSR matrix, and Algorithm 5 around it */
int orc_gmres(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, int32_t restart,
              orc_info *info);
int orc_gmres_plain(const orc_csr *A, const double *b, double *x, double tol, int32_t max_it, int32_t restart,
                    orc_info *info);
int orc_adaptive_gmres(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, int32_t restart,
                       int32_t k, int32_t s, double gamma_min, double rho_max, orc_info *info);
void orc_free(orc_hier *h);
void orc_csr_free(orc_csr *m);

/* accessors for the tests (borrowed pointers, valid until orc_free) */
int32_t orc_num_levels(const orc_hier *h);
const orc_csr *orc_level_matrix(const orc_hier *h, int32_t l, int32_t which);
const void *orc_level_array(const orc_hier *h, int32_t l, int32_t which);
double orc_level_gamma(const orc_hier *h, int32_t l);

#ifdef __cplusplus
}
#endif
#endif
