/*
 * amg.h -- C ABI of the GB300 sparsified algebraic-multigrid library (libamg.so).
 *
 * The library solves SPD systems A x = b (Bienz, Falgout, Gropp, Olson,
 * Schroder, "Reducing Parallel Communication in Algebraic Multigrid through
 * Sparsification", arXiv:1512.04629, Section 1) with preconditioned CG whose
 * preconditioner is one AMG V-cycle (Algorithm 2) over a classical Galerkin
 * hierarchy (Algorithm 1) whose coarse operators are thinned by Sparse
 * Galerkin sparsification with diagonal lumping (Algorithm 4 with the loop of
 * Algorithm 3b), and whose dropped entries can be reintroduced when
 * convergence is slow (Algorithm 5).  Every step runs in the library's own
 * CUDA kernels on one GPU (sm_103a).
 *
 * Conventions shared by every call:
 *  - Matrices are CSR with int32 row pointers and column indices, columns
 *    strictly increasing within a row, the diagonal stored, fewer than 2^31
 *    stored entries, FP64 values.
 *  - Pointers are host pointers unless an argument or struct field says they
 *    are device pointers.  "Device pointer" means memory of the current CUDA
 *    device (e.g. the data pointer of a CUDA torch tensor).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work of a call is ordered on that stream; a call that
 *    returns host data synchronises it.
 *  - The caller owns every buffer it passes; the library only reads inputs
 *    and writes outputs during the call and keeps no pointer to them.  The
 *    library owns every hierarchy, its device memory, and every server.
 *  - No C++ exception crosses the ABI.  Every call returns an amg_status; on
 *    failure amg_last_error() holds a thread-local message.  Invalid input is
 *    rejected with AMG_ERR_INVALID before any kernel is launched.
 *  - A hierarchy may be used by one thread at a time (the server serialises
 *    its own use).
 */
#ifndef AMG_H
#define AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMG_OK = 0,
    AMG_ERR_INVALID = 1,   /* bad argument or matrix; nothing was launched */
    AMG_ERR_OOM = 2,       /* device or host allocation failed */
    AMG_ERR_CUDA = 3,      /* a CUDA call failed; see amg_last_error() */
    AMG_NOT_CONVERGED = 4, /* max_it reached; x and info are still filled */
    AMG_DIVERGED = 5,      /* residual grew by more than div_factor (1e3) over a
                              check window; x is the window's starting iterate */
    AMG_BREAKDOWN = 6,     /* CG lost positive definiteness (rho or p.Ap <= 0) */
    AMG_TIMEOUT = 7,       /* a wait ran past its time limit */
    AMG_REJECTED = 8       /* admission refused (server: memory budget / queue) */
} amg_status;

/* A square (or, with ncols > 0, rectangular) CSR matrix, caller-owned and
 * read-only.  on_device != 0: rowptr, col, val are device pointers. */
typedef struct {
    int64_t n;             /* rows */
    int64_t nnz;           /* stored entries = rowptr[n] */
    const int32_t *rowptr; /* n + 1 */
    const int32_t *col;    /* nnz, increasing within each row */
    const double *val;     /* nnz */
    int on_device;
    int64_t ncols;         /* 0 means ncols = n */
} amg_csr;

/* AMG_METHOD_SPARSE / AMG_METHOD_HYBRID: Algorithm 4 on a retained Galerkin
 * hierarchy (minimal pattern M from the Galerkin, resp. the sparsified, level
 * above).  AMG_METHOD_NONGALERKIN: Algorithm 1's optional step, the paper's
 * comparator -- each coarse operator is thinned as soon as the Galerkin
 * product forms it and replaces it for the rest of the setup; nothing
 * Galerkin is retained, so amg_sparsify, amg_reintroduce, adaptive solves,
 * amg_hierarchy_save and amg_hierarchy_assemble reject such a hierarchy /
 * method (AMG_ERR_INVALID), and amg_level_stats reports the thinned operator
 * as nnz_galerkin. */
enum { AMG_METHOD_SPARSE = 0, AMG_METHOD_HYBRID = 1, AMG_METHOD_NONGALERKIN = 2 };
/* How sparsify treats a dropped entry: AMG_LUMP_DIAG adds it to the diagonal
 * of its row (Algorithm 3b; keeps an SPD diagonally dominant operator SPD,
 * Theorem 1); AMG_LUMP_STRONG spreads it symmetrically over the strong
 * neighbours that the row keeps (Algorithm 3's own loop: symmetry and row
 * sums are kept, definiteness is not -- solve with GMRES). */
enum { AMG_LUMP_DIAG = 0, AMG_LUMP_STRONG = 1 };
/* Outer Krylov method of amg_solve: preconditioned CG, or restarted GMRES
 * right-preconditioned by the V-cycle (the paper's solver where full lumping
 * can cost positive definiteness, Section 5).  amg_solve_batch and the server
 * run per-column CG whatever this says; a column that meets an indefinite
 * preconditioner ends with AMG_BREAKDOWN in its own info. */
enum { AMG_KRYLOV_CG = 0, AMG_KRYLOV_GMRES = 1 };
enum { AMG_PREC_FP64 = 0, AMG_PREC_FP32 = 1, AMG_PREC_FP32_BF16 = 2 };
/* SpMV kernel variants: CSR with T threads per row, or SELL-C slices (C rows
 * per slice, column-major inside it, read by one warp with 32 / C lanes per
 * row: SELL32 one lane per row, SELL16 two, SELL8 four). */
enum {
    AMG_SPMV_AUTO = -1,
    AMG_SPMV_CSR2 = 1, AMG_SPMV_CSR4 = 2, AMG_SPMV_CSR8 = 3, AMG_SPMV_CSR16 = 4,
    AMG_SPMV_CSR32 = 5, AMG_SPMV_SELL32 = 6, AMG_SPMV_CSR1 = 7, AMG_SPMV_SELL16 = 8, AMG_SPMV_SELL8 = 9
};

typedef struct {
    double theta;        /* strength threshold (classical rule), default 0.25 */
    int max_size;        /* stop coarsening at n <= max_size, default 100 */
    int max_levels;      /* default 25 */
    uint64_t seed;       /* PMIS random weights, default 0 */
    int method;          /* AMG_METHOD_SPARSE (default), _HYBRID or _NONGALERKIN */
    int precision;       /* AMG_PREC_*: storage/arithmetic of the V-cycle */
    int k_check;         /* Algorithm 5: PCG steps between checks, default 3 */
    int s_levels;        /* Algorithm 5: levels updated per step, default 1 */
    double gamma_min;    /* Algorithm 5: smaller tolerances become 0, default 0.01 */
    double rho_max;      /* Algorithm 5: reintroduce above this factor, default 0.5 */
    int level_offset;    /* PMIS level index of the first level, default 0 */
    int spmv_variant;    /* AMG_SPMV_AUTO (autotuned per level) or forced */
    int use_graph;       /* capture the PCG iteration in a CUDA graph, default 1 */
    int check_every;     /* reserved, must be >= 1 (default 1): the recurrence
                            stop test runs on the device after every step */
    int setup_timing;    /* 1: time the setup phases with events (amg_timing_get
                            kinds 8..15), default 0 */
    int lump;            /* AMG_LUMP_DIAG (default) or AMG_LUMP_STRONG */
    int krylov;          /* AMG_KRYLOV_CG (default) or AMG_KRYLOV_GMRES */
    int restart;         /* GMRES restart length m (Krylov vectors kept), default 30 */
    double div_factor;   /* AMG_DIVERGED when the residual grows by more than this
                            factor over a check window of k_check CG steps,
                            default 1e3; 0 turns the test off, else >= 1 */
    int transfer_variant; /* AMG_SPMV_AUTO (default: P and R timed per level
                            when spmv_variant is AUTO, else the mean-row
                            heuristic) or an AMG_SPMV_* forced for P and R */
} amg_options;

typedef struct {
    int iterations;      /* products with A_0 (CG steps) */
    int status;          /* amg_status of the solve */
    int resets;          /* adaptive: reintroductions (PCG restarts) */
    int replacements;    /* true-residual replacements */
    double final_relres; /* ||b - A x||_2 / ||b||_2, FP64, at exit */
    double conv_factor;  /* (||r_end|| / ||r_0||)^(1/iterations) */
    double solve_ms;     /* wall time of the call (host clock) */
} amg_solve_info;

typedef struct {
    int64_t n;              /* rows of A_l */
    int64_t nnz_galerkin;   /* stored entries of the Galerkin A_l */
    int64_t nnz_operator;   /* stored entries of the relaxed operator Ahat_l */
    int64_t nnz_p;          /* entries of P_l (0 on the coarsest level) */
    int64_t n_coarse;       /* columns of P_l */
    double gamma;           /* drop tolerance of the level */
    int spmv_variant;       /* AMG_SPMV_* used by the level's relaxation */
    int value_bytes;        /* bytes per stored value in the cycle (8, 4, 2) */
    double bytes_per_cycle; /* algorithmic HBM bytes of the level per V(1,1) cycle */
    int spmv_variant_p;     /* AMG_SPMV_* of the interpolation x += P x_c (0 on the coarsest) */
    int spmv_variant_r;     /* AMG_SPMV_* of the restriction b_c = R r (0 on the coarsest) */
} amg_level_info;

typedef struct amg_hierarchy amg_hierarchy;
typedef struct amg_server amg_server;

/* Fill *opt with the defaults listed above. */
void amg_options_default(amg_options *opt);

/*
 * amg_setup -- Algorithm 1 (Galerkin hierarchy: classical strength, PMIS
 * C/F splitting, direct interpolation, A_{l+1} = P_l^T A_l P_l), then
 * Algorithm 4 (Sparse Galerkin sparsify with diagonal lumping, Algorithm 3b)
 * with gamma_per_level, then the ell1-Jacobi diagonals and the coarsest-level
 * Cholesky factor.  gamma_per_level[l] applies to level l; levels past
 * n_gamma - 1 use the last value; gamma_per_level[0] must be 0 (level 0 is
 * never sparsified); n_gamma = 0 (or NULL) means no sparsification.  `theta`
 * overrides opt->theta.  A is copied (host or device); the hierarchy, owned
 * by the library, is returned in *out and freed with amg_free.
 * Errors: AMG_ERR_INVALID for a non-square, unsorted, non-symmetric-pattern
 * matrix, a missing or non-positive diagonal, non-finite values or bad
 * options; AMG_ERR_OOM; AMG_ERR_CUDA.
 */
amg_status amg_setup(const amg_csr *A, double theta, const double *gamma_per_level, int n_gamma,
                     const amg_options *opt, void *stream, amg_hierarchy **out);

/*
 * amg_hierarchy_assemble -- build a hierarchy from given Galerkin operators
 * A_0..A_{L-1}, interpolations P_0..P_{L-2} (ncols = n_{l+1}), C/F markers
 * cf_0..cf_{L-2} (1 = C, -1 = F, host int8) and minimal-pattern flags
 * inM_1..inM_{L-1} (host uint8 per stored entry of A_l; inM[0] is ignored),
 * e.g. a hierarchy saved earlier or built by another code.  Then as
 * amg_setup: sparsify, ell1 diagonals, Cholesky.  Errors as amg_setup.
 */
amg_status amg_hierarchy_assemble(int levels, const amg_csr *A, const amg_csr *P,
                                  const int8_t *const *cf, const uint8_t *const *inM,
                                  const double *gamma_per_level, int n_gamma,
                                  const amg_options *opt, void *stream, amg_hierarchy **out);

/* amg_sparsify -- re-run Algorithm 4 on the retained Galerkin operators with
 * new drop tolerances (same gamma convention as amg_setup). */
amg_status amg_sparsify(amg_hierarchy *h, const double *gamma_per_level, int n_gamma);

/* amg_reintroduce -- one drop-tolerance update of Algorithm 5: from the
 * finest level l >= 1 with gamma_l > 0, on s_levels levels, gamma <- gamma/10
 * (0 below gamma_min), and those levels are re-sparsified from the retained
 * Galerkin A_l.  *levels_changed (may be NULL) receives the number of levels
 * changed (0: every gamma is already 0). */
amg_status amg_reintroduce(amg_hierarchy *h, int s_levels, int *levels_changed);

/*
 * amg_solve -- PCG (FP64 recurrences, x0 = 0) preconditioned by one V(1,1)
 * cycle (Algorithm 2) to ||b - A_0 x|| / ||b|| <= tol, at most max_it steps.
 * adaptive != 0 runs Algorithm 5 around it (k_check, s_levels, gamma_min,
 * rho_max from the options given at setup).  b and x are n-vectors, both host
 * or both device: on_device says which.  In the FP32 precision modes the
 * outer loop is flexible CG.  Returns the solve status (also in info->status).
 * Divergence (Section 6: with too many entries dropped the method stops
 * converging): a plain CG solve is cut into windows of k_check steps (counted
 * again after each true-residual replacement); when the recurrence residual
 * at a window's end exceeds div_factor times the one at its start, or is not
 * finite, the solve stops with AMG_DIVERGED and x is the iterate at the
 * window's start.  An adaptive solve applies the same factor to the true
 * residual of its Algorithm 5 windows, and first tries to recover by
 * reintroduction; it returns AMG_DIVERGED (x at the window's start) only
 * when every gamma is already 0.  GMRES minimises the residual, so it never
 * reports AMG_DIVERGED; neither do batched or served solves.
 */
amg_status amg_solve(amg_hierarchy *h, const double *b, double *x, double tol, int max_it,
                     int adaptive, int on_device, void *stream, amg_solve_info *info);

/*
 * amg_solve_batch -- k independent solves sharing one hierarchy; B and X are
 * row-major n x k (column j = right-hand side j), host or device per
 * on_device.  The V-cycle runs as a multi-right-hand-side SpMM; each column
 * keeps its own CG scalars and stops on its own (always CG: amg_options.krylov
 * applies to amg_solve only).  info_k has k entries.
 */
amg_status amg_solve_batch(amg_hierarchy *h, int k, const double *B, double *X, double tol,
                           int max_it, int on_device, void *stream, amg_solve_info *info_k);

/* amg_precond_apply -- z = M r, one V(1,1) cycle; r, z: device n-vectors. */
amg_status amg_precond_apply(amg_hierarchy *h, const double *r, double *z, void *stream);

/* amg_num_levels / amg_level_stats -- hierarchy shape and per-level figures. */
int amg_num_levels(const amg_hierarchy *h);
amg_status amg_level_stats(const amg_hierarchy *h, int level, amg_level_info *out);

/*
 * amg_level_export -- copy one matrix of a level to host buffers.
 * which: 0 Galerkin A_l, 1 relaxed operator Ahat_l, 2 P_l, 3 R_l = P_l^T.
 * With rowptr == NULL only *nrows, *ncols, *nnz are returned (size query);
 * otherwise rowptr (nrows+1), col and val (nnz) are filled.
 */
amg_status amg_level_export(const amg_hierarchy *h, int level, int which, int32_t *rowptr,
                            int32_t *col, double *val, int64_t *nrows, int64_t *ncols,
                            int64_t *nnz);

/*
 * amg_level_array -- copy a per-level array to a host buffer `out`:
 * which 0: cf (int8, n; 1 = C, -1 = F), 1: keep mask (uint8 per entry of A_l),
 * 2: inM (uint8 per entry of A_l), 3: ell1 diagonal (double, n),
 * 4: strength flags (uint8 per entry of A_l).  *count receives the length.
 */
amg_status amg_level_array(const amg_hierarchy *h, int level, int which, void *out,
                           int64_t *count);

/* Per-kernel timing with CUDA events on the solve stream (off by default).
 * amg_timing_get returns, for kernel class `kind` (0 fused pre-smooth +
 * residual, 1 restrict, 2 prolong, 3 post-smooth, 4 coarse solve, 5 PCG
 * A p + dot, 6 PCG vector update) on `level`, the number of timed launches,
 * their total milliseconds and their algorithmic bytes.  With
 * amg_options.setup_timing, or while timing is enabled during amg_sparsify /
 * amg_reintroduce, the setup phases are recorded too (bytes 0): 8 strength,
 * 9 C/F splitting (PMIS and the coarse numbering), 10 interpolation P and
 * R = P^T, 11 Galerkin products A P and R (A P), 12 level maps of the new
 * level (diagonal and transpose positions) and its minimal pattern M,
 * 13 sparsification (Algorithm 3 / 3b), 14 cycle preparation (ell1
 * diagonal, precision copies, SELL layout, autotuning), 15 coarsest-level
 * Cholesky inverse.  Kinds 8..12 are filed under the fine level l of the
 * step that builds level l + 1. */
amg_status amg_timing_enable(amg_hierarchy *h, int on);
amg_status amg_timing_get(const amg_hierarchy *h, int kind, int level, int64_t *launches,
                          double *total_ms, double *bytes);
amg_status amg_timing_reset(amg_hierarchy *h);

/* Save / load the Galerkin hierarchy, C/F markers, minimal-pattern flags and
 * drop tolerances to a file.  The file is little-endian binary:
 *   char magic[4] = "AMGH"; u32 version = 1; u32 L (levels, 1..25);
 *   then for each level l = 0 .. L-1:
 *     i64 n, i64 nnz; i32 rowptr[n+1]; i32 col[nnz]; f64 val[nnz]
 *       (the retained Galerkin operator A_l, rows sorted by column);
 *     f64 gamma_l (the drop tolerance of level l; level 0's is ignored);
 *     if l > 0:     u8 inM[nnz] (1 = entry of A_l in the minimal pattern M);
 *     if l < L - 1: i8 cf[n] (1 = C point, -1 = F point);
 *                   i64 n_coarse, i64 nnz_P; i32 rowptr[n+1]; i32 col[nnz_P];
 *                   f64 val[nnz_P] (the interpolation P_l, n x n_coarse).
 * Load rebuilds everything else (R, sparsified operators, smoother
 * diagonals, the coarsest inverse) on the device from these arrays with the
 * given options.  A non-Galerkin hierarchy retains no Galerkin operator and
 * cannot be saved (AMG_ERR_INVALID); a short or foreign file gives
 * AMG_ERR_INVALID. */
amg_status amg_hierarchy_save(const amg_hierarchy *h, const char *path);
amg_status amg_hierarchy_load(const char *path, const amg_options *opt, void *stream,
                              amg_hierarchy **out);

void amg_free(amg_hierarchy *h);
const char *amg_status_str(amg_status s);
const char *amg_last_error(void);

/*
 * amg_residual_noalloc -- r = b - A_0 x and rnorm[0] = ||r||_2 for the
 * finest operator of h, for callers that cannot allocate device memory at
 * the moment they call: a framework or real-time loop whose device memory is
 * handed out only by its own pool (a cudaMalloc there would bypass its
 * accounting or stall the loop), or a process whose memory budget is already
 * fully committed, where an allocation would fail.  The paper has no
 * counterpart: it is a service of this library, not a step of the method.
 * b, x, r, rnorm: device pointers on h's device (b, x, r of length n; rnorm
 * one double, written on the device -- the call does not synchronise).  The
 * call must be made with h's device current; another current device, or
 * pointers that are host memory or belong to another device, give
 * AMG_ERR_INVALID and launch nothing.  The call allocates nothing: its
 * reduction scratch is a fixed array of about 530 KB in the library image,
 * held by every GPU that loads the library until the process exits.  n is
 * limited to 67,108,864 rows (AMG_ERR_INVALID beyond).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress, once
 * per device).  All calls share the scratch and its counters are cleared at
 * the start of each call, so calls that overlap on the GPU race: order them
 * (e.g. one stream).
 */
amg_status amg_residual_noalloc(const amg_hierarchy *h, const double *b, const double *x, double *r,
                                double *rnorm, void *stream);

/*
 * Row-partitioned execution (the paper's parallel SpMV, Section 2, and its
 * communication model, Section 4).  Each level's rows are split into `parts`
 * contiguous blocks, one per process of a distributed solve: the finest
 * level in blocks of n / parts rows, every coarser level so that each block
 * keeps its own C points (coarse point c belongs to the block of the fine
 * point it came from).  A block's columns split into the ones it owns (the
 * diagonal block) and ghosts owned by other blocks (the off-diagonal block),
 * whose values it receives before each product; a message is one ordered
 * pair of blocks that exchange at least one value.
 *
 * amg_halo_plan -- the plan of one operator, on the host (no GPU): rows
 * [row0[p], row0[p+1]) form block p, which owns columns [col0[p], col0[p+1]).
 * Caller-allocated outputs: cext[nnz] (each entry's column in its block's
 * numbering: owned columns j - col0[p], then ghost g as (col0[p+1] - col0[p])
 * + g), goff[parts + 1] (block p's ghosts are gcol[goff[p] .. goff[p+1]),
 * increasing), gcol[nnz] (room for the worst case), recv[parts * parts]
 * (values block p receives from block q, at p * parts + q).  1 <= parts <= 64.
 * AMG_ERR_INVALID for inconsistent bounds or columns out of range.
 */
amg_status amg_halo_plan(int64_t nrows, int64_t ncols, const int32_t *rowptr, const int32_t *col, int parts,
                         const int64_t *row0, const int64_t *col0, int32_t *cext, int64_t *goff,
                         int32_t *gcol, int64_t *recv);

/*
 * amg_partition -- split every level of h into `parts` blocks (1 <= parts <=
 * 64; 1 removes the split) and plan each operator of the solve: the relaxed
 * operator Ahat_l (A_0 on level 0), P_l and R_l; the Galerkin A_l is planned
 * for its statistics.  Solves (amg_solve, CG or GMRES, FP64 precision only;
 * AMG_ERR_INVALID otherwise) then run block by block on this GPU: before each
 * product every block gathers its ghost values -- the exchange a distributed
 * run performs by messages -- and multiplies its rows by its own columns and
 * its ghosts.  Rows are summed in stored order, so a partitioned solve equals
 * an unpartitioned one whose relaxation and transfers run one lane per row
 * (spmv_variant = transfer_variant = AMG_SPMV_CSR1) bit for bit.  amg_sparsify
 * and amg_reintroduce re-plan the levels they change.  Batched and served
 * solves ignore the split.
 */
amg_status amg_partition(amg_hierarchy *h, int parts);

/* Communication of one level per product (SpMV) under the current split. */
typedef struct {
    int parts;
    int64_t messages;           /* ordered block pairs exchanging values, relaxed operator */
    int64_t halo_values;        /* ghost values received, summed over blocks */
    int64_t max_messages;       /* most messages one block receives */
    int64_t max_halo;           /* most ghost values one block receives */
    int64_t messages_galerkin;  /* the same two for the Galerkin A_l */
    int64_t halo_galerkin;
    int64_t messages_p, halo_p; /* interpolation x += P x_c (0 on the coarsest level) */
    int64_t messages_r, halo_r; /* restriction b_c = R r */
} amg_comm_info;
amg_status amg_comm_stats(const amg_hierarchy *h, int level, amg_comm_info *out);
/* row0[0 .. parts]: the block boundaries of level `level` (parts + 1 values). */
amg_status amg_partition_rows(const amg_hierarchy *h, int level, int64_t *row0);

/* Number of CUDA kernels this process has launched through the library so
 * far (a diagnostic counter, e.g. to count the launches of one solve). */
int64_t amg_kernel_launches(void);

/* Host-side fault injection for tests of the out-of-memory paths: the device
 * allocation that comes `after` allocations from now (0: the next one) fails
 * as if the device had no memory left -- the entry point that made it returns
 * AMG_ERR_OOM and releases what it had allocated, and the library stays
 * usable.  One failure per arming; after < 0 disarms.  No GPU fault is
 * involved: the allocation is refused on the host before CUDA is asked. */
void amg_debug_fail_allocation(int64_t after);

/* Device memory the library currently holds for hierarchies (bytes). */
int64_t amg_device_bytes(const amg_hierarchy *h);

/*
 * Serving: a host thread owns a queue of solve requests against registered
 * hierarchies.  Requests on one hierarchy are solved together as columns of
 * one multi-right-hand-side solve; new requests join the running batch at the
 * next iteration boundary when a column slot and device memory are free
 * (continuous batching).  Each column's CG scalars are its own, so a result
 * does not depend on what else is in the batch.
 *
 * Each registered hierarchy runs on its own stream, and submit/wait copy on
 * one more.  CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware
 * queues (8 unless set), and streams sharing a queue wait on one another: a
 * caller serving more than a handful of hierarchies should set it (up to 32)
 * before the process creates its CUDA context.  The Python package sets 32
 * on import unless the variable is already set.
 */
typedef struct {
    int max_batch;          /* column slots per hierarchy, default 32 */
    int64_t hbm_budget;     /* bytes the server may allocate for batch workspaces;
                               0 = 70% of the HBM free at create */
    int max_queue;          /* pending requests before submits are rejected, default 4096 */
    int max_it;             /* per request, default 500 */
    int64_t stage_budget;   /* bytes of device memory, on top of hbm_budget, for requests
                               held on the device: right-hand sides from submit to
                               admission, results from retirement to wait.  0 (default)
                               = a quarter of the workspace budget; -1 = none.  A request
                               that finds no room is staged through host memory by the
                               worker thread instead (same result, slower). */
    int64_t wait_limit_ms;  /* longest the worker waits for one piece of device work (a
                               batch iteration, a residual check, a host staging copy),
                               default 120000; must be >= 1.  Every such wait is a poll
                               of an event.  When one runs out, the worker stops: every
                               request not yet finished ends with AMG_TIMEOUT (wait
                               returns it and the ticket is consumed), and later
                               submits return AMG_TIMEOUT.  The copies of b in submit
                               and of x in wait always run to completion before those
                               calls return (the device reads or writes the caller's
                               memory). */
} amg_server_opts;

void amg_server_opts_default(amg_server_opts *o);
amg_status amg_server_create(const amg_server_opts *o, amg_server **out);
/* The hierarchy stays owned by the caller and must outlive the server. */
amg_status amg_server_register(amg_server *s, amg_hierarchy *h, int *hid);
/* b: host n-vector, copied at submit (uploaded to the device when the
 * staging budget has room; b is free for reuse when the call returns).
 * Returns a ticket. */
amg_status amg_server_submit(amg_server *s, int hid, const double *b, double tol,
                             uint64_t *ticket);
/* Waits up to timeout_ms for the ticket; x: host n-vector, written on the
 * calling thread (the download of a device-staged result runs here, not on
 * the worker).  AMG_TIMEOUT if not finished in time (the request stays
 * queued and can be waited again). */
amg_status amg_server_wait(amg_server *s, uint64_t ticket, double *x, int timeout_ms,
                           amg_solve_info *info);
/* Stops the worker after the running batches finish; frees the server. */
void amg_server_destroy(amg_server *s);

#ifdef __cplusplus
}
#endif
#endif
