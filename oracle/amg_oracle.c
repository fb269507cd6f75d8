/*
 * amg_oracle.c -- plain FP64 CPU oracle of the sparsified-AMG hot path.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).
 * Single-threaded, no blocking, no fusion: each function is the step of the
 * paper it cites, written out.  Compile with -ffp-contract=off.
 * See amg_oracle.h for the paper reference and the floating-point contract.
 */
#include "amg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_OOM 2
#define ORC_NOT_CONVERGED 4
#define ORC_DIVERGED 5
#define ORC_BREAKDOWN 6

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static orc_csr *csr_alloc(int32_t nrows, int32_t ncols, int64_t nnz) {
    if (nnz < 0 || nnz >= ((int64_t)1 << 31)) return NULL;
    orc_csr *m = (orc_csr *)calloc(1, sizeof(orc_csr));
    if (!m) return NULL;
    m->nrows = nrows;
    m->ncols = ncols;
    m->nnz = (int32_t)nnz;
    m->rowptr = (int32_t *)calloc((size_t)nrows + 1, sizeof(int32_t));
    m->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    m->val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!m->rowptr || !m->col || !m->val) {
        orc_csr_free(m);
        return NULL;
    }
    return m;
}

void orc_csr_free(orc_csr *m) {
    if (!m) return;
    free(m->rowptr);
    free(m->col);
    free(m->val);
    free(m);
}

static orc_csr *csr_copy(const orc_csr *a) {
    orc_csr *m = csr_alloc(a->nrows, a->ncols, a->nnz);
    if (!m) return NULL;
    memcpy(m->rowptr, a->rowptr, sizeof(int32_t) * ((size_t)a->nrows + 1));
    memcpy(m->col, a->col, sizeof(int32_t) * (size_t)a->nnz);
    memcpy(m->val, a->val, sizeof(double) * (size_t)a->nnz);
    return m;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* The all-core timing build (compiled with -fopenmp) splits the row loops
 * of the solve phase -- SpMV, vector updates, dot products -- over the host's
 * threads; the setup stays sequential.  Without -fopenmp these pragmas are
 * ignored and every loop runs in order: that build is the parity reference.
 * Only the dot products' summation order differs between the two. */
#define ORC_PRAGMA(x) _Pragma(#x)
#define ORC_PAR_FOR(n) ORC_PRAGMA(omp parallel for schedule(static) if ((n) > 16384))
#define ORC_PAR_SUM(n, v) ORC_PRAGMA(omp parallel for schedule(static) reduction(+ : v) if ((n) > 16384))

static double dot(int32_t n, const double *a, const double *b) {
    double s = 0.0;
    ORC_PAR_SUM(n, s)
    for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double norm2(int32_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* y = A x, each row summed in column order. */
void orc_spmv(const orc_csr *A, const double *x, double *y) {
    ORC_PAR_FOR(A->nrows)
    for (int32_t i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) s += A->val[p] * x[A->col[p]];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* strength (Section 2, Algorithm 1 "strength"; the paper describes it only   */
/* in words).  Reading: the classical Ruge-Stueben rule on negative couplings */
/*   j in S_i  <=>  j != i  and  -a_ij >= theta * max_{k != i}(-a_ik),          */
/* and a row whose largest negative coupling is <= 0 has no strong entries.   */
/* ------------------------------------------------------------------------ */
void orc_strength(const orc_csr *A, double theta, uint8_t *strong) {
    for (int32_t i = 0; i < A->nrows; ++i) {
        int32_t p0 = A->rowptr[i], p1 = A->rowptr[i + 1];
        double m = 0.0;
        int any = 0;
        for (int32_t p = p0; p < p1; ++p) {
            if (A->col[p] == i) continue;
            double v = -A->val[p];
            if (!any || v > m) {
                m = v;
                any = 1;
            }
        }
        double t = theta * m;
        for (int32_t p = p0; p < p1; ++p)
            strong[p] = (uint8_t)(any && m > 0.0 && A->col[p] != i && -A->val[p] >= t);
    }
}

/* ------------------------------------------------------------------------ */
/* PMIS C/F splitting (Section 1 cites PMIS as aggressive coarsening; Section */
/* 2 defines the split C u F and n_{l+1} = |C|).  Reading:                    */
/*   w_i = |S^T_i| + u_i,  u_i = top 53 bits of SplitMix64(seed ^ (l<<40) ^ i) */
/*   * 2^-53  (SplitMix64: Steele, Lea, Flood 2014);                           */
/*   points with |S^T_i| = 0 (w_i < 1) start as F;                             */
/*   each round, an undecided i becomes C if (w_i, i) > (w_j, j) for every     */
/*   undecided j in S_i u S^T_i (rounds are synchronous); then every undecided */
/*   j that has a C point in S_j becomes F.                                    */
/* cf[i] = 1 for C, -1 for F.                                                 */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64_oracle(uint64_t key) {
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform_weight(uint64_t seed, int32_t level, int64_t i) {
    uint64_t key = seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)i;
    return (double)(splitmix64_oracle(key) >> 11) * (1.0 / 9007199254740992.0);
}

int orc_pmis(const orc_csr *A, const uint8_t *strong, uint64_t seed, int32_t level, int8_t *cf) {
    int32_t n = A->nrows;
    /* S^T as explicit lists: st_ptr/st_idx hold, for each i, the rows j with i in S_j. */
    int32_t *st_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *st_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int8_t *state = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *newc = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!st_ptr || !st_idx || !fill || !w || !state || !newc) {
        free(st_ptr); free(st_idx); free(fill); free(w); free(state); free(newc);
        return ORC_OOM;
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
            if (strong[p]) st_ptr[A->col[p] + 1]++;
    for (int32_t i = 0; i < n; ++i) st_ptr[i + 1] += st_ptr[i];
    for (int32_t i = 0; i < n; ++i) fill[i] = st_ptr[i];
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
            if (strong[p]) st_idx[fill[A->col[p]]++] = i;

    enum { U = 0, C = 1, F = -1 };
    int64_t undecided = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t cnt = st_ptr[i + 1] - st_ptr[i];
        w[i] = (double)cnt + orc_uniform_weight(seed, level, i);
        state[i] = (cnt == 0) ? F : U;
        if (state[i] == U) undecided++;
    }
    while (undecided > 0) {
        /* select: undecided local maxima of (w, index) over S_i u S^T_i */
        for (int32_t i = 0; i < n; ++i) {
            newc[i] = 0;
            if (state[i] != U) continue;
            int wins = 1;
            for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1] && wins; ++p) {
                if (!strong[p]) continue;
                int32_t j = A->col[p];
                if (state[j] == U && (w[j] > w[i] || (w[j] == w[i] && j > i))) wins = 0;
            }
            for (int32_t q = st_ptr[i]; q < st_ptr[i + 1] && wins; ++q) {
                int32_t j = st_idx[q];
                if (state[j] == U && (w[j] > w[i] || (w[j] == w[i] && j > i))) wins = 0;
            }
            newc[i] = (uint8_t)wins;
        }
        for (int32_t i = 0; i < n; ++i)
            if (newc[i]) {
                state[i] = C;
                undecided--;
            }
        /* every undecided j with a C point in S_j becomes F */
        for (int32_t j = 0; j < n; ++j) {
            if (state[j] != U) continue;
            for (int32_t p = A->rowptr[j]; p < A->rowptr[j + 1]; ++p)
                if (strong[p] && state[A->col[p]] == C) {
                    state[j] = F;
                    undecided--;
                    break;
                }
        }
    }
    for (int32_t i = 0; i < n; ++i) cf[i] = state[i];
    free(st_ptr); free(st_idx); free(fill); free(w); free(state); free(newc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* direct interpolation P: R^{n_c} -> R^{n} (Section 2, "interpolation").    */
/* Reading: Stueben's direct interpolation with the sign split.  For an F    */
/* point i with strong C neighbours C_i:                                     */
/*   alpha = sum_{k != i} a_ik^- / sum_{k in C_i} a_ik^-                      */
/*   beta  = sum_{k != i} a_ik^+ / sum_{k in C_i} a_ik^+   (if the latter != 0,*/
/*           otherwise the positive sum is added to the diagonal, beta = 0)  */
/*   w_ij  = -alpha a_ij / a_ii  (a_ij < 0),  -beta a_ij / a_ii  (a_ij > 0).   */
/* C points get a unit row; an F point with C_i empty gets an empty row.     */
/* Coarse index of a C point = number of C points before it.                 */
/* ------------------------------------------------------------------------ */
orc_csr *orc_direct_interp(const orc_csr *A, const uint8_t *strong, const int8_t *cf) {
    int32_t n = A->nrows;
    int32_t *cmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!cmap) return NULL;
    int32_t nc = 0;
    for (int32_t i = 0; i < n; ++i) cmap[i] = (cf[i] == 1) ? nc++ : -1;
    int64_t nnz = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (cf[i] == 1) {
            nnz += 1;
            continue;
        }
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
            if (strong[p] && cf[A->col[p]] == 1) nnz++;
    }
    orc_csr *P = csr_alloc(n, nc, nnz);
    if (!P) {
        free(cmap);
        return NULL;
    }
    int32_t pos = 0;
    for (int32_t i = 0; i < n; ++i) {
        P->rowptr[i] = pos;
        if (cf[i] == 1) {
            P->col[pos] = cmap[i];
            P->val[pos] = 1.0;
            pos++;
            continue;
        }
        double diag = 0.0, sum_neg = 0.0, sum_pos = 0.0, sum_neg_c = 0.0, sum_pos_c = 0.0;
        int has_c = 0;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            int32_t j = A->col[p];
            double v = A->val[p];
            if (j == i) {
                diag = v;
                continue;
            }
            if (v < 0.0) sum_neg += v;
            if (v > 0.0) sum_pos += v;
            if (strong[p] && cf[j] == 1) {
                has_c = 1;
                if (v < 0.0) sum_neg_c += v;
                if (v > 0.0) sum_pos_c += v;
            }
        }
        if (!has_c) continue;
        double alpha = (sum_neg_c != 0.0) ? sum_neg / sum_neg_c : 0.0;
        double beta = 0.0;
        if (sum_pos_c != 0.0)
            beta = sum_pos / sum_pos_c;
        else
            diag = diag + sum_pos;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            int32_t j = A->col[p];
            if (j == i || !strong[p] || cf[j] != 1) continue;
            double v = A->val[p];
            double wgt = (v < 0.0) ? (-alpha * v) / diag : (-beta * v) / diag;
            P->col[pos] = cmap[j];
            P->val[pos] = wgt;
            pos++;
        }
    }
    P->rowptr[n] = pos;
    P->nnz = pos;
    free(cmap);
    return P;
}

/* Transpose by counting; rows of the result list sources in increasing order. */
orc_csr *orc_transpose(const orc_csr *M) {
    orc_csr *T = csr_alloc(M->ncols, M->nrows, M->nnz);
    if (!T) return NULL;
    for (int32_t p = 0; p < M->nnz; ++p) T->rowptr[M->col[p] + 1]++;
    for (int32_t j = 0; j < M->ncols; ++j) T->rowptr[j + 1] += T->rowptr[j];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M->ncols > 0 ? M->ncols : 1));
    if (!fill) {
        orc_csr_free(T);
        return NULL;
    }
    for (int32_t j = 0; j < M->ncols; ++j) fill[j] = T->rowptr[j];
    for (int32_t i = 0; i < M->nrows; ++i)
        for (int32_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) {
            int32_t q = fill[M->col[p]]++;
            T->col[q] = i;
            T->val[q] = M->val[p];
        }
    free(fill);
    return T;
}

/* ------------------------------------------------------------------------ */
/* C = A B, row by row with a dense accumulator (Gustavson).  Structural:    */
/* every product creates an entry, exact zeros are kept.  Each entry starts  */
/* at 0.0 and gains a_ik b_kj in the order (k over row i of A, increasing;   */
/* j over row k of B).  Output rows are sorted by column.                    */
/* Used for the Galerkin product A_{l+1} = P^T (A_l P_l) (Section 2, Alg 1). */
/* ------------------------------------------------------------------------ */
orc_csr *orc_spgemm(const orc_csr *A, const orc_csr *B) {
    int32_t n = A->nrows, m = B->ncols;
    int32_t *marker = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    double *acc = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!marker || !acc || !list) {
        free(marker); free(acc); free(list);
        return NULL;
    }
    for (int32_t j = 0; j < m; ++j) marker[j] = -1;
    /* symbolic pass: count */
    int64_t nnz = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            int32_t k = A->col[p];
            for (int32_t q = B->rowptr[k]; q < B->rowptr[k + 1]; ++q) {
                int32_t j = B->col[q];
                if (marker[j] != i) {
                    marker[j] = i;
                    nnz++;
                }
            }
        }
    }
    orc_csr *Cm = csr_alloc(n, m, nnz);
    if (!Cm) {
        free(marker); free(acc); free(list);
        return NULL;
    }
    for (int32_t j = 0; j < m; ++j) marker[j] = -1;
    int32_t pos = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t len = 0;
        Cm->rowptr[i] = pos;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
            int32_t k = A->col[p];
            double a = A->val[p];
            for (int32_t q = B->rowptr[k]; q < B->rowptr[k + 1]; ++q) {
                int32_t j = B->col[q];
                if (marker[j] != i) {
                    marker[j] = i;
                    acc[j] = 0.0;
                    list[len++] = j;
                }
                acc[j] += a * B->val[q];
            }
        }
        qsort(list, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int32_t t = 0; t < len; ++t) {
            Cm->col[pos] = list[t];
            Cm->val[pos] = acc[list[t]];
            pos++;
        }
    }
    Cm->rowptr[n] = pos;
    free(marker); free(acc); free(list);
    return Cm;
}

/* ------------------------------------------------------------------------ */
/* Minimal sparsity pattern (Section 2.1, Algorithm 3):                      */
/*   M = edges(Phat^T A P + P^T A Phat),  Phat = injection at the C points.   */
/* Phat^T A P is the block of rows of AP at the C points (coarse-indexed),   */
/* X; P^T A Phat = (Phat^T A^T P)^T = X^T because A is symmetric.  Edges are */
/* read structurally (stored entries).  inM[p] flags entry p of Ac.          */
/* ------------------------------------------------------------------------ */
int orc_minimal_pattern(const orc_csr *Ac, const orc_csr *AP, const int8_t *cf, uint8_t *inM) {
    int32_t nc = Ac->nrows;
    /* X: rows of AP at C points, in coarse order */
    int64_t xnnz = 0;
    int32_t ci = 0;
    for (int32_t f = 0; f < AP->nrows; ++f)
        if (cf[f] == 1) {
            xnnz += AP->rowptr[f + 1] - AP->rowptr[f];
            ci++;
        }
    if (ci != nc) return ORC_INVALID;
    orc_csr *X = csr_alloc(nc, AP->ncols, xnnz);
    if (!X) return ORC_OOM;
    int32_t pos = 0;
    ci = 0;
    for (int32_t f = 0; f < AP->nrows; ++f) {
        if (cf[f] != 1) continue;
        X->rowptr[ci] = pos;
        for (int32_t p = AP->rowptr[f]; p < AP->rowptr[f + 1]; ++p) {
            X->col[pos] = AP->col[p];
            X->val[pos] = AP->val[p];
            pos++;
        }
        ci++;
    }
    X->rowptr[nc] = pos;
    orc_csr *XT = orc_transpose(X);
    int32_t *marker = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    if (!XT || !marker) {
        orc_csr_free(X); orc_csr_free(XT); free(marker);
        return ORC_OOM;
    }
    for (int32_t j = 0; j < nc; ++j) marker[j] = -1;
    for (int32_t i = 0; i < nc; ++i) {
        for (int32_t p = X->rowptr[i]; p < X->rowptr[i + 1]; ++p) marker[X->col[p]] = i;
        for (int32_t p = XT->rowptr[i]; p < XT->rowptr[i + 1]; ++p) marker[XT->col[p]] = i;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) inM[p] = (uint8_t)(marker[Ac->col[p]] == i);
    }
    orc_csr_free(X); orc_csr_free(XT); free(marker);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* sparsify with diagonal lumping (Algorithm 3's first loop + Algorithm 3b). */
/*   first loop: (i,j) enters N, with (j,i), if (i,j) in M or                 */
/*     |a_ij| >= gamma max_{k != i} |a_ik|;                                   */
/*   3b loop: an entry in N (or the ismax guard) is kept, every other         */
/*     off-diagonal a_ij is added to the diagonal of row i.                   */
/* Readings: the diagonal is always kept and is the lumping target; max over */
/* k != i excludes the diagonal; the ismax guard (garbled in the paper)      */
/* keeps the entries equal to the row maximum of a zero-row-sum row none of  */
/* whose off-diagonals is in N (|row sum| <= 1e-12 sum |a_ij|), and adds the  */
/* mirrored entries to N too so that N stays symmetric.  With gamma <= 1 it  */
/* never fires.  Dropped entries are added in increasing column order to    */
/* the diagonal value.  keep[p] flags the kept entries of Ac.                */
/* ------------------------------------------------------------------------ */
static int32_t find_entry(const orc_csr *A, int32_t i, int32_t j) {
    for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p)
        if (A->col[p] == j) return p;
    return -1;
}

orc_csr *orc_sparsify_diag(const orc_csr *Ac, const uint8_t *inM, double gamma, uint8_t *keep) {
    int32_t n = Ac->nrows;
    int32_t nnz = Ac->nnz;
    uint8_t *flag = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    uint8_t *guard = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    double *rowmax = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!flag || !guard || !rowmax) {
        free(flag); free(guard); free(rowmax);
        return NULL;
    }
    /* first loop of Algorithm 3: entries passing the test */
    for (int32_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p)
            if (Ac->col[p] != i && fabs(Ac->val[p]) > m) m = fabs(Ac->val[p]);
        rowmax[i] = m;
        double t = gamma * m;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p)
            flag[p] = (uint8_t)(Ac->col[p] != i && (inM[p] || fabs(Ac->val[p]) >= t));
    }
    /* N = flagged entries and their mirrors; the diagonal is always kept */
    for (int32_t p = 0; p < nnz; ++p) keep[p] = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
            int32_t j = Ac->col[p];
            if (j == i) {
                keep[p] = 1;
                continue;
            }
            if (flag[p]) {
                keep[p] = 1;
                int32_t q = find_entry(Ac, j, i);
                if (q >= 0) keep[q] = 1;
            }
        }
    /* ismax guard (Algorithm 3b) */
    for (int32_t i = 0; i < n; ++i) {
        int any_off = 0;
        double rs = 0.0, ra = 0.0;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
            rs += Ac->val[p];
            ra += fabs(Ac->val[p]);
            if (Ac->col[p] != i && keep[p]) any_off = 1;
        }
        guard[i] = (uint8_t)(!any_off && rowmax[i] > 0.0 && fabs(rs) <= 1e-12 * ra);
    }
    for (int32_t i = 0; i < n; ++i) {
        if (!guard[i]) continue;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
            int32_t j = Ac->col[p];
            if (j != i && fabs(Ac->val[p]) == rowmax[i]) {
                keep[p] = 1;
                int32_t q = find_entry(Ac, j, i);
                if (q >= 0) keep[q] = 1;
            }
        }
    }
    /* 3b loop: kept entries are copied, dropped ones are lumped to the diagonal */
    int64_t knnz = 0;
    for (int32_t p = 0; p < nnz; ++p) knnz += keep[p];
    orc_csr *H = csr_alloc(n, Ac->ncols, knnz);
    if (!H) {
        free(flag); free(guard); free(rowmax);
        return NULL;
    }
    int32_t pos = 0;
    for (int32_t i = 0; i < n; ++i) {
        H->rowptr[i] = pos;
        int32_t dpos = -1;
        double d = 0.0;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p)
            if (Ac->col[p] == i) d = Ac->val[p];
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p)
            if (!keep[p]) d += Ac->val[p];
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
            if (!keep[p]) continue;
            H->col[pos] = Ac->col[p];
            H->val[pos] = Ac->val[p];
            if (Ac->col[p] == i) dpos = pos;
            pos++;
        }
        if (dpos >= 0) H->val[dpos] = d;
    }
    H->rowptr[n] = pos;
    free(flag); free(guard); free(rowmax);
    return H;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 with its own second loop (full lumping to strong neighbours, */
/* the non-Galerkin sparsify of Falgout and Schroder).  The first loop and  */
/* N are those of orc_sparsify_diag (the diagonal always kept, no ismax     */
/* guard: Algorithm 3 has none).  Readings:                                 */
/*  - S is the classical strength matrix of Ac itself (the indices j, k of  */
/*    W are coarse points), with the rule of orc_strength and the setup's   */
/*    theta; S_{j,k} = (Ac)_{j,k} on strong entries, 0 elsewhere;           */
/*  - the loop over "omega" runs over W (the set just built);               */
/*  - "(Ahat_c)_{i,j} = (A_c)_{i,j}" for (i,j) in N is the starting value   */
/*    of Ahat_c, not an assignment that could overwrite lumped values       */
/*    added earlier in the loop: Ahat_c starts as Ac restricted to N and    */
/*    every update below accumulates on it;                                 */
/*  - a dropped entry whose W is empty (or whose strong weights sum to 0)   */
/*    has no neighbour to take it: it is lumped to the diagonal of its row, */
/*    as in Algorithm 3b, so row sums stay exact;                           */
/*  - dropped entries are processed in CSR order (row by row, increasing    */
/*    column), each k of W in increasing column order, and the three        */
/*    updates of one k in the order written: (i,k), (k,i), (k,k).           */
/* Each update is symmetric and leaves every row sum unchanged, so Ahat_c   */
/* is symmetric with the row sums of Ac -- but it can lose definiteness.    */
/* ------------------------------------------------------------------------ */
orc_csr *orc_sparsify_full(const orc_csr *Ac, const uint8_t *inM, double gamma, double theta,
                           uint8_t *keep) {
    int32_t n = Ac->nrows;
    int32_t nnz = Ac->nnz;
    uint8_t *flag = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    uint8_t *S = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    double *val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!flag || !S || !val) {
        free(flag); free(S); free(val);
        return NULL;
    }
    /* first loop: entries passing the drop test or in M */
    for (int32_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p)
            if (Ac->col[p] != i && fabs(Ac->val[p]) > m) m = fabs(Ac->val[p]);
        double t = gamma * m;
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p)
            flag[p] = (uint8_t)(Ac->col[p] != i && (inM[p] || fabs(Ac->val[p]) >= t));
    }
    /* N: flagged entries, their mirrors and the diagonal */
    for (int32_t p = 0; p < nnz; ++p) keep[p] = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
            int32_t j = Ac->col[p];
            if (j == i) {
                keep[p] = 1;
            } else if (flag[p]) {
                keep[p] = 1;
                int32_t q = find_entry(Ac, j, i);
                if (q >= 0) keep[q] = 1;
            }
        }
    orc_strength(Ac, theta, S);
    /* Ahat_c starts as Ac on N */
    for (int32_t p = 0; p < nnz; ++p) val[p] = keep[p] ? Ac->val[p] : 0.0;
    /* second loop: lump every dropped entry to the strong neighbours of j */
    /* that row i keeps                                                     */
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
            if (keep[p]) continue;
            int32_t j = Ac->col[p];
            double a = Ac->val[p];
            /* sum over W of |S_{j,m}| */
            double denom = 0.0;
            for (int32_t q = Ac->rowptr[j]; q < Ac->rowptr[j + 1]; ++q) {
                if (!S[q]) continue;
                int32_t pik = find_entry(Ac, i, Ac->col[q]);
                if (pik >= 0 && keep[pik]) denom += fabs(Ac->val[q]);
            }
            if (!(denom > 0.0)) {
                int32_t pii = find_entry(Ac, i, i);
                if (pii >= 0) val[pii] += a;
                continue;
            }
            for (int32_t q = Ac->rowptr[j]; q < Ac->rowptr[j + 1]; ++q) {
                if (!S[q]) continue;
                int32_t k = Ac->col[q];
                int32_t pik = find_entry(Ac, i, k);
                if (pik < 0 || !keep[pik]) continue;
                double alpha = fabs(Ac->val[q]) / denom;
                double t = alpha * a;
                val[pik] += t;
                int32_t pki = find_entry(Ac, k, i);
                if (pki >= 0) val[pki] += t;
                int32_t pkk = find_entry(Ac, k, k);
                if (pkk >= 0) val[pkk] -= t;
            }
        }
    int64_t knnz = 0;
    for (int32_t p = 0; p < nnz; ++p) knnz += keep[p];
    orc_csr *H = csr_alloc(n, Ac->ncols, knnz);
    if (H) {
        int32_t pos = 0;
        for (int32_t i = 0; i < n; ++i) {
            H->rowptr[i] = pos;
            for (int32_t p = Ac->rowptr[i]; p < Ac->rowptr[i + 1]; ++p) {
                if (!keep[p]) continue;
                H->col[pos] = Ac->col[p];
                H->val[pos] = val[p];
                pos++;
            }
        }
        H->rowptr[n] = pos;
    }
    free(flag); free(S); free(val);
    return H;
}

/* ell1 diagonal d_i = sum_j |a_ij| of the relaxed operator (reading: the    */
/* paper's "relax" is e.g. Jacobi; ell1-Jacobi without damping is used).    */
void orc_l1_diag(const orc_csr *A, double *d) {
    for (int32_t i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int32_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) s += fabs(A->val[p]);
        d[i] = s;
    }
}

/* Dense Cholesky A = L L^T in place (row-major n x n, lower triangle used), */
/* for the coarsest-level direct solve of Algorithm 2.                      */
int orc_cholesky(int32_t n, double *a) {
    for (int32_t j = 0; j < n; ++j) {
        double s = a[(size_t)j * n + j];
        for (int32_t k = 0; k < j; ++k) s -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(s > 0.0)) return ORC_BREAKDOWN;
        double ljj = sqrt(s);
        a[(size_t)j * n + j] = ljj;
        for (int32_t i = j + 1; i < n; ++i) {
            double t = a[(size_t)i * n + j];
            for (int32_t k = 0; k < j; ++k) t -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = t / ljj;
        }
        for (int32_t i = 0; i < j; ++i) a[(size_t)i * n + j] = 0.0;
    }
    return ORC_OK;
}

void orc_chol_solve(int32_t n, const double *L, const double *b, double *x) {
    for (int32_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int32_t k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int32_t k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

/* Dense LU with partial pivoting, P A = L U in place (row-major; unit L    */
/* below the diagonal).  piv[j] is the row swapped with row j at step j (the */
/* first row of largest |a_ij|, i >= j).  ORC_BREAKDOWN if a pivot is 0.    */
int orc_lu(int32_t n, double *a, int32_t *piv) {
    for (int32_t j = 0; j < n; ++j) {
        int32_t r = j;
        for (int32_t i = j + 1; i < n; ++i)
            if (fabs(a[(size_t)i * n + j]) > fabs(a[(size_t)r * n + j])) r = i;
        piv[j] = r;
        if (!(a[(size_t)r * n + j] != 0.0)) return ORC_BREAKDOWN;
        if (r != j)
            for (int32_t c = 0; c < n; ++c) {
                double t = a[(size_t)j * n + c];
                a[(size_t)j * n + c] = a[(size_t)r * n + c];
                a[(size_t)r * n + c] = t;
            }
        for (int32_t i = j + 1; i < n; ++i) {
            double l = a[(size_t)i * n + j] / a[(size_t)j * n + j];
            a[(size_t)i * n + j] = l;
            for (int32_t c = j + 1; c < n; ++c) a[(size_t)i * n + c] -= l * a[(size_t)j * n + c];
        }
    }
    return ORC_OK;
}

void orc_lu_solve(int32_t n, const double *LU, const int32_t *piv, const double *b, double *x) {
    for (int32_t i = 0; i < n; ++i) x[i] = b[i];
    for (int32_t j = 0; j < n; ++j) {
        double t = x[j];
        x[j] = x[piv[j]];
        x[piv[j]] = t;
    }
    for (int32_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int32_t k = 0; k < i; ++k) s -= LU[(size_t)i * n + k] * x[k];
        x[i] = s;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int32_t k = i + 1; k < n; ++k) s -= LU[(size_t)i * n + k] * x[k];
        x[i] = s / LU[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 5's drop-tolerance update.  Readings of the garbled lines:      */
/* l_start = the finest level l >= 1 with gamma_l > 0; the levels            */
/* l_start .. l_start + s - 1 (clamped to the hierarchy) get                  */
/* gamma <- gamma / 10 if gamma / 10 >= gamma_min (relative slack 1e-12),     */
/* else 0 (Example 1 maps 0.1 to 0.01 and 0.01 to 0).  Level 0 is never      */
/* sparsified.  changed[l] is set to 1 for the updated levels; the return    */
/* value is their count (0: nothing left to reintroduce).                    */
/* ------------------------------------------------------------------------ */
int orc_gamma_schedule(double *gamma, int32_t nlev, int32_t s, double gamma_min, int32_t *changed) {
    int32_t lstart = -1;
    for (int32_t l = 0; l < nlev; ++l) changed[l] = 0;
    for (int32_t l = 1; l < nlev; ++l)
        if (gamma[l] > 0.0) {
            lstart = l;
            break;
        }
    if (lstart < 0) return 0;
    int cnt = 0;
    for (int32_t l = lstart; l < lstart + s && l < nlev; ++l) {
        double g = gamma[l] / 10.0;
        gamma[l] = (g >= gamma_min * (1.0 - 1e-12)) ? g : 0.0;
        changed[l] = 1;
        cnt++;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* hierarchy                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_csr *A;      /* Galerkin A_l, retained (Section 3: store A_c and Ahat_c) */
    orc_csr *Ahat;   /* relaxed operator; for l = 0 and gamma = 0 a copy of A */
    uint8_t *strong; /* per entry of A (levels that were coarsened) */
    uint8_t *inM;    /* per entry of A (l >= 1) */
    uint8_t *keep;   /* per entry of A */
    int8_t *cf;
    orc_csr *P, *R, *AP;
    double *d;       /* ell1 diagonal of Ahat */
    double gamma;
    double *b, *x, *r;
} orc_level;

struct orc_hier {
    int32_t nlev;
    int32_t method; /* 0 Sparse Galerkin, 1 Hybrid Galerkin (set by orc_sparsify_method), 2 non-Galerkin */
    int32_t lump;   /* 0 diagonal lumping (Algorithm 3b), 1 full lumping (Algorithm 3) */
    double theta;   /* strength threshold of the setup (full lumping's S) */
    orc_level lev[64];
    double *chol;   /* dense factor of Ahat of the coarsest level: Cholesky, or LU */
    int32_t *piv;   /* row permutation of the LU factor (NULL: Cholesky) */
};

static void level_free(orc_level *L) {
    if (L->Ahat != L->A) orc_csr_free(L->Ahat);
    orc_csr_free(L->A);
    orc_csr_free(L->P);
    orc_csr_free(L->R);
    orc_csr_free(L->AP);
    free(L->strong); free(L->inM); free(L->keep); free(L->cf); free(L->d);
    free(L->b); free(L->x); free(L->r);
    memset(L, 0, sizeof(*L));
}

void orc_free(orc_hier *h) {
    if (!h) return;
    for (int32_t l = 0; l < h->nlev; ++l) level_free(&h->lev[l]);
    free(h->chol);
    free(h->piv);
    free(h);
}

static int level_workspace(orc_level *L) {
    int32_t n = L->A->nrows;
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    L->d = (double *)malloc(sz);
    L->b = (double *)calloc(1, sz);
    L->x = (double *)calloc(1, sz);
    L->r = (double *)calloc(1, sz);
    L->keep = (uint8_t *)malloc((size_t)(L->A->nnz > 0 ? L->A->nnz : 1));
    if (!L->d || !L->b || !L->x || !L->r || !L->keep) return ORC_OOM;
    for (int32_t p = 0; p < L->A->nnz; ++p) L->keep[p] = 1;
    return ORC_OK;
}

/* Coarsest-level direct solve of Algorithm 2 (the paper does not name the  */
/* factorization).  Reading: Cholesky; when the coarsest relaxed operator is */
/* not positive definite (full lumping can make it indefinite) an LU        */
/* factorization with partial pivoting takes its place.                     */
static void densify_coarsest(const orc_level *L, double *a) {
    int32_t n = L->A->nrows;
    for (size_t t = 0; t < (size_t)n * (size_t)n; ++t) a[t] = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = L->Ahat->rowptr[i]; p < L->Ahat->rowptr[i + 1]; ++p)
            a[(size_t)i * n + L->Ahat->col[p]] = L->Ahat->val[p];
}

static int factor_coarsest(orc_hier *h) {
    orc_level *L = &h->lev[h->nlev - 1];
    int32_t n = L->A->nrows;
    free(h->chol);
    free(h->piv);
    h->piv = NULL;
    h->chol = (double *)calloc((size_t)n * (size_t)n + 1, sizeof(double));
    if (!h->chol) return ORC_OOM;
    densify_coarsest(L, h->chol);
    if (orc_cholesky(n, h->chol) == ORC_OK) return ORC_OK;
    h->piv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!h->piv) return ORC_OOM;
    densify_coarsest(L, h->chol);
    return orc_lu(n, h->chol, h->piv);
}

/* Algorithm 1 with sparsify off (the Galerkin hierarchy of Algorithm 4's   */
/* first line).  Stop rule (the paper leaves max_size unvalued): stop when  */
/* n_l <= max_size, at max_levels levels, or when the coarse grid would be  */
/* empty or larger than 0.9 n_l; the last level is the coarsest.            */
static orc_hier *setup_core(const orc_csr *A0, double theta, int32_t max_size, int32_t max_levels,
                            uint64_t seed, const double *gamma, int32_t ngamma, int32_t lump,
                            int32_t *status);

orc_hier *orc_setup(const orc_csr *A0, double theta, int32_t max_size, int32_t max_levels,
                    uint64_t seed, int32_t *status) {
    return setup_core(A0, theta, max_size, max_levels, seed, NULL, 0, 0, status);
}

/* Algorithm 1 with its optional non-Galerkin step (Section 2.1, the       */
/* method of Falgout and Schroder the paper compares against): each coarse */
/* operator is sparsified as soon as the Galerkin product forms it, and    */
/* the sparsified operator replaces it -- strength, C/F splitting,         */
/* interpolation and the next Galerkin product all use it.  Readings: the  */
/* call's garbled tolerance index is the per-level convention of           */
/* Algorithm 4 (gamma[l] thins the operator of level l, levels past        */
/* ngamma - 1 use the last value, gamma[0] = 0); M is formed from the      */
/* current (already sparsified) A_l; S of full lumping is the strength of  */
/* the coarse operator being thinned.  No Galerkin operator is retained,   */
/* so Algorithm 5 does not apply (orc_sparsify / orc_reintroduce refuse).  */
/* A thinned operator with a non-positive diagonal entry ends the setup    */
/* with ORC_BREAKDOWN (lumping can push a diagonal to or below zero when   */
/* the coarse operator is not diagonally dominant).                        */
orc_hier *orc_setup_nongalerkin(const orc_csr *A0, double theta, int32_t max_size, int32_t max_levels,
                                uint64_t seed, const double *gamma, int32_t ngamma, int32_t lump,
                                int32_t *status) {
    if (ngamma < 1 || gamma[0] != 0.0 || lump < 0 || lump > 1) {
        *status = ORC_INVALID;
        return NULL;
    }
    for (int32_t l = 0; l < ngamma; ++l)
        if (!(gamma[l] >= 0.0) || !isfinite(gamma[l])) {
            *status = ORC_INVALID;
            return NULL;
        }
    return setup_core(A0, theta, max_size, max_levels, seed, gamma, ngamma, lump, status);
}

static orc_hier *setup_core(const orc_csr *A0, double theta, int32_t max_size, int32_t max_levels,
                            uint64_t seed, const double *gamma, int32_t ngamma, int32_t lump,
                            int32_t *status) {
    *status = ORC_OK;
    if (max_levels < 1 || max_levels > 64) {
        *status = ORC_INVALID;
        return NULL;
    }
    orc_hier *h = (orc_hier *)calloc(1, sizeof(orc_hier));
    if (!h) {
        *status = ORC_OOM;
        return NULL;
    }
    h->lev[0].A = csr_copy(A0);
    h->nlev = 1;
    h->theta = theta;
    if (!h->lev[0].A) goto oom;
    for (int32_t l = 0; l + 1 < max_levels; ++l) {
        orc_level *L = &h->lev[l];
        int32_t n = L->A->nrows;
        if (n <= max_size) break;
        L->strong = (uint8_t *)malloc((size_t)(L->A->nnz > 0 ? L->A->nnz : 1));
        L->cf = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
        if (!L->strong || !L->cf) goto oom;
        orc_strength(L->A, theta, L->strong);
        if (orc_pmis(L->A, L->strong, seed, l, L->cf) != ORC_OK) goto oom;
        int32_t nc = 0;
        for (int32_t i = 0; i < n; ++i) nc += (L->cf[i] == 1);
        if (nc == 0 || (double)nc > 0.9 * (double)n) {
            free(L->strong); free(L->cf);
            L->strong = NULL;
            L->cf = NULL;
            break;
        }
        L->P = orc_direct_interp(L->A, L->strong, L->cf);
        if (!L->P) goto oom;
        L->R = orc_transpose(L->P);
        L->AP = orc_spgemm(L->A, L->P);
        if (!L->R || !L->AP) goto oom;
        orc_level *Lc = &h->lev[l + 1];
        Lc->A = orc_spgemm(L->R, L->AP);
        if (!Lc->A) goto oom;
        Lc->inM = (uint8_t *)malloc((size_t)(Lc->A->nnz > 0 ? Lc->A->nnz : 1));
        if (!Lc->inM) goto oom;
        if (orc_minimal_pattern(Lc->A, L->AP, L->cf, Lc->inM) != ORC_OK) goto oom;
        h->nlev = l + 2;
        if (gamma) {  /* non-Galerkin: the thinned operator replaces A_{l+1} */
            double g = gamma[(l + 1) < ngamma ? (l + 1) : ngamma - 1];
            Lc->gamma = g;
            if (g > 0.0) {
                uint8_t *keep = (uint8_t *)malloc((size_t)(Lc->A->nnz > 0 ? Lc->A->nnz : 1));
                if (!keep) goto oom;
                orc_csr *H = lump ? orc_sparsify_full(Lc->A, Lc->inM, g, theta, keep)
                                  : orc_sparsify_diag(Lc->A, Lc->inM, g, keep);
                free(keep);
                if (!H) goto oom;
                orc_csr_free(Lc->A);
                Lc->A = H;
                free(Lc->inM);   /* M belonged to the Galerkin pattern */
                Lc->inM = NULL;
                /* a thinned operator whose diagonal is no longer positive   */
                /* cannot be coarsened or relaxed: the setup breaks down      */
                for (int32_t i = 0; i < H->nrows; ++i) {
                    int32_t pd = find_entry(H, i, i);
                    if (pd < 0 || !(H->val[pd] > 0.0)) {
                        *status = ORC_BREAKDOWN;
                        orc_free(h);
                        return NULL;
                    }
                }
            }
        }
    }
    if (gamma) {
        h->method = 2;
        h->lump = lump;
    }
    for (int32_t l = 0; l < h->nlev; ++l) {
        orc_level *L = &h->lev[l];
        L->Ahat = L->A;
        if (!gamma) L->gamma = 0.0;
        if (level_workspace(L) != ORC_OK) goto oom;
        orc_l1_diag(L->Ahat, L->d);
    }
    if (h->lev[h->nlev - 1].A->nrows > 8192) {
        *status = ORC_INVALID;
        orc_free(h);
        return NULL;
    }
    {
        int st = factor_coarsest(h);
        if (st != ORC_OK) {
            *status = st;
            orc_free(h);
            return NULL;
        }
    }
    return h;
oom:
    *status = ORC_OOM;
    orc_free(h);
    return NULL;
}

/* Minimal pattern of level l for Hybrid Galerkin (Section 3, Algorithm 4,
 * hybrid line): M = edges(Phat^T Ahat P + P^T Ahat Phat) with Ahat the
 * sparsified operator of level l-1 (for l = 1, Ahat_0 = A_0). */
static int hybrid_pattern(orc_hier *h, int32_t l, uint8_t *inM) {
    orc_level *F = &h->lev[l - 1];
    orc_csr *AP = orc_spgemm(F->Ahat, F->P);
    if (!AP) return ORC_OOM;
    int st = orc_minimal_pattern(h->lev[l].A, AP, F->cf, inM);
    orc_csr_free(AP);
    return st;
}

/* (Re)build Ahat_l from the retained A_l at the level's gamma; method 1
 * (Hybrid) takes M from the current Ahat_{l-1}. */
static int resparsify_level_m(orc_hier *h, int32_t l, int32_t method);

static int resparsify_level_m(orc_hier *h, int32_t l, int32_t method) {
    orc_level *L = &h->lev[l];
    if (L->Ahat != L->A) orc_csr_free(L->Ahat);
    L->Ahat = L->A;
    if (l == 0 || L->gamma == 0.0) {
        for (int32_t p = 0; p < L->A->nnz; ++p) L->keep[p] = 1;
    } else {
        const uint8_t *inM = L->inM;
        uint8_t *hyb = NULL;
        if (method == 1) {
            hyb = (uint8_t *)malloc((size_t)(L->A->nnz > 0 ? L->A->nnz : 1));
            if (!hyb) return ORC_OOM;
            int st = hybrid_pattern(h, l, hyb);
            if (st != ORC_OK) {
                free(hyb);
                return st;
            }
            inM = hyb;
        }
        orc_csr *H = h->lump ? orc_sparsify_full(L->A, inM, L->gamma, h->theta, L->keep)
                             : orc_sparsify_diag(L->A, inM, L->gamma, L->keep);
        free(hyb);
        if (!H) return ORC_OOM;
        L->Ahat = H;
    }
    orc_l1_diag(L->Ahat, L->d);
    if (l == h->nlev - 1) return factor_coarsest(h);
    return ORC_OK;
}

/* Algorithm 4, Sparse Galerkin: Ahat_l = sparsify(A_l, A_{l-1}, P_{l-1},   */
/* S_{l-1}, gamma_l) for l = 1 .. L-1 (reading of the garbled indices: the  */
/* loop writes Ahat_l; Ahat_0 = A_0).  gamma[l] applies to level l, levels  */
/* past ngamma - 1 use gamma[ngamma - 1]; gamma[0] must be 0.               */
int orc_sparsify_method(orc_hier *h, const double *gamma, int32_t ngamma, int32_t method) {
    return orc_sparsify_opts(h, gamma, ngamma, method, 0);
}

/* lump 0: the loop of Algorithm 3b (diagonal lumping); 1: Algorithm 3's own */
/* loop (full lumping to strong neighbours). */
int orc_sparsify_opts(orc_hier *h, const double *gamma, int32_t ngamma, int32_t method, int32_t lump) {
    if (ngamma < 1 || gamma[0] != 0.0 || method < 0 || method > 1 || lump < 0 || lump > 1 || h->method == 2)
        return ORC_INVALID;
    for (int32_t l = 0; l < ngamma; ++l)
        if (!(gamma[l] >= 0.0) || !isfinite(gamma[l])) return ORC_INVALID;
    h->method = method;
    h->lump = lump;
    for (int32_t l = 1; l < h->nlev; ++l) {  /* in order: Hybrid reads Ahat_{l-1} */
        h->lev[l].gamma = gamma[l < ngamma ? l : ngamma - 1];
        int st = resparsify_level_m(h, l, method);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

int orc_sparsify(orc_hier *h, const double *gamma, int32_t ngamma) {
    return orc_sparsify_method(h, gamma, ngamma, 0);
}

/* One reintroduction step of Algorithm 5: new gammas on s levels, then    */
/* re-sparsify those levels from the retained Galerkin A_l.               */
/* Algorithm 5 re-sparsifies only the levels whose gamma changed; with the
 * Hybrid method their M comes from the current Ahat_{l-1}. */
int orc_reintroduce(orc_hier *h, int32_t s, double gamma_min, int32_t *changed) {
    if (h->method == 2) return -ORC_INVALID;  /* non-Galerkin: nothing retained to reintroduce */
    double g[64];
    for (int32_t l = 0; l < h->nlev; ++l) g[l] = h->lev[l].gamma;
    int cnt = orc_gamma_schedule(g, h->nlev, s, gamma_min, changed);
    for (int32_t l = 0; l < h->nlev; ++l) {
        if (!changed[l]) continue;
        h->lev[l].gamma = g[l];
        int st = resparsify_level_m(h, l, h->method);
        if (st != ORC_OK) return -st;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, V(1,1) cycle applied to the residual equation (zero initial  */
/* guess on every level) with ell1-Jacobi relax: x <- x + D^{-1}(b - Ahat x).  */
/* The pre-smooth from zero is x = D^{-1} b.  Level 0 relaxes with A_0.      */
/* ------------------------------------------------------------------------ */
int orc_vcycle(orc_hier *h, const double *b, double *x) {
    int32_t L = h->nlev;
    memcpy(h->lev[0].b, b, sizeof(double) * (size_t)h->lev[0].A->nrows);
    for (int32_t l = 0; l + 1 < L; ++l) {
        orc_level *V = &h->lev[l];
        int32_t n = V->A->nrows;
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) V->x[i] = V->b[i] / V->d[i];   /* pre-smooth */
        orc_spmv(V->Ahat, V->x, V->r);
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) V->r[i] = V->b[i] - V->r[i];    /* residual */
        orc_spmv(V->R, V->r, h->lev[l + 1].b);                          /* restrict */
    }
    orc_level *Cl = &h->lev[L - 1];
    if (h->piv) orc_lu_solve(Cl->A->nrows, h->chol, h->piv, Cl->b, Cl->x);  /* coarse solve */
    else orc_chol_solve(Cl->A->nrows, h->chol, Cl->b, Cl->x);
    for (int32_t l = L - 2; l >= 0; --l) {
        orc_level *V = &h->lev[l];
        int32_t n = V->A->nrows;
        orc_spmv(V->P, h->lev[l + 1].x, V->r);
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) V->x[i] += V->r[i];             /* interpolate, correct */
        orc_spmv(V->Ahat, V->x, V->r);
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) V->r[i] = V->x[i] + (V->b[i] - V->r[i]) / V->d[i];
        memcpy(V->x, V->r, sizeof(double) * (size_t)n);                  /* post-smooth */
    }
    memcpy(x, h->lev[0].x, sizeof(double) * (size_t)h->lev[0].A->nrows);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* PCG with M = one V-cycle (Section 5.5 solves with PCG).  The state is    */
/* resumable so that Algorithm 5 can continue the Krylov run between checks */
/* and restart it only after the preconditioner changed.  Convergence: the  */
/* recurrence residual reaches tol ||b|| and the true residual b - A_0 x     */
/* confirms it; otherwise the true residual replaces r and the run goes on. */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    double *r, *z, *p, *q, *xs;
    double rho;
} pcg_state;

typedef struct {
    int32_t steps, converged, breakdown, replacements, diverged;
    double rnorm; /* residual norm at the end of the run */
} pcg_run;

static void pcg_free(pcg_state *s) {
    free(s->r); free(s->z); free(s->p); free(s->q); free(s->xs);
    memset(s, 0, sizeof(*s));
}

static int pcg_alloc(pcg_state *s, int32_t n) {
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    s->n = n;
    s->r = (double *)malloc(sz);
    s->z = (double *)malloc(sz);
    s->p = (double *)malloc(sz);
    s->q = (double *)malloc(sz);
    s->xs = (double *)malloc(sz);
    if (!s->r || !s->z || !s->p || !s->q || !s->xs) {
        pcg_free(s);
        return ORC_OOM;
    }
    return ORC_OK;
}

/* (re)start: r = b - A_0 x, z = M r, p = z, rho = r.z; returns ||r|| */
static double pcg_start(orc_hier *h, pcg_state *s, const double *b, const double *x) {
    int32_t n = s->n;
    orc_spmv(h->lev[0].A, x, s->q);
    ORC_PAR_FOR(n)
    for (int32_t i = 0; i < n; ++i) s->r[i] = b[i] - s->q[i];
    orc_vcycle(h, s->r, s->z);
    memcpy(s->p, s->z, sizeof(double) * (size_t)n);
    s->rho = dot(n, s->r, s->z);
    return norm2(n, s->r);
}

/* Divergence, the failure Algorithm 5 exists to recover from (Section 6:  */
/* with too many entries dropped the method stops converging).  Reading:    */
/* with divf > 0 the run is cut into windows of kwin steps, counted from    */
/* its start and again from every residual replacement; at the end of a     */
/* window the recurrence residual norm is compared with the one at the      */
/* window's start, and if it grew by more than the factor divf -- or if it  */
/* is non-finite after any step -- x goes back to the window's starting     */
/* iterate and the run stops as diverged.  divf = 0 turns the test off.     */
static void pcg_iterate(orc_hier *h, pcg_state *s, const double *b, double *x, double bnorm,
                        double tol, int32_t max_steps, int32_t kwin, double divf, pcg_run *run) {
    const orc_csr *A = h->lev[0].A;
    int32_t n = s->n;
    memset(run, 0, sizeof(*run));
    run->rnorm = norm2(n, s->r);
    if (run->rnorm <= tol * bnorm) {
        run->converged = 1;
        return;
    }
    int32_t w = 0;            /* steps since the window count (re)started */
    double rws = run->rnorm;  /* residual norm at the current window's start */
    while (run->steps < max_steps) {
        if (divf > 0.0 && w % kwin == 0) memcpy(s->xs, x, sizeof(double) * (size_t)n);
        orc_spmv(A, s->p, s->q);
        double pq = dot(n, s->p, s->q);
        run->steps++;
        if (!(pq > 0.0) || !(s->rho > 0.0)) {
            run->breakdown = 1;
            return;
        }
        double alpha = s->rho / pq;
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) x[i] += alpha * s->p[i];
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) s->r[i] -= alpha * s->q[i];
        run->rnorm = norm2(n, s->r);
        w++;
        if (divf > 0.0) {
            if (!isfinite(run->rnorm) || (w % kwin == 0 && run->rnorm > divf * rws)) {
                memcpy(x, s->xs, sizeof(double) * (size_t)n);
                run->rnorm = rws;
                run->diverged = 1;
                return;
            }
            if (w % kwin == 0) rws = run->rnorm;
        }
        if (run->rnorm <= tol * bnorm) {
            orc_spmv(A, x, s->q);
            ORC_PAR_FOR(n)
            for (int32_t i = 0; i < n; ++i) s->q[i] = b[i] - s->q[i];
            double tn = norm2(n, s->q);
            run->rnorm = tn;
            if (tn <= tol * bnorm) {
                run->converged = 1;
                return;
            }
            memcpy(s->r, s->q, sizeof(double) * (size_t)n);
            run->replacements++;
            w = 0;
            rws = tn;
        }
        orc_vcycle(h, s->r, s->z);
        double rho_new = dot(n, s->r, s->z);
        double beta = rho_new / s->rho;
        s->rho = rho_new;
        ORC_PAR_FOR(n)
        for (int32_t i = 0; i < n; ++i) s->p[i] = s->z[i] + beta * s->p[i];
    }
}

static double true_resnorm(orc_hier *h, const double *b, const double *x, double *work) {
    const orc_csr *A = h->lev[0].A;
    int32_t n = A->nrows;
    orc_spmv(A, x, work);
    double s = 0.0;
    ORC_PAR_SUM(n, s)
    for (int32_t i = 0; i < n; ++i) {
        double e = b[i] - work[i];
        s += e * e;
    }
    return sqrt(s);
}

/* PCG from x0 = 0 to ||b - A x|| / ||b|| <= tol (at most max_it steps),  */
/* stopping as diverged when the residual grows by more than divf over a    */
/* window of kwin steps (see pcg_iterate; divf = 0: no such test).          */
int orc_pcg_ex(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, int32_t kwin,
               double divf, orc_info *info) {
    int32_t n = h->lev[0].A->nrows;
    memset(info, 0, sizeof(*info));
    if (kwin < 1 || !(divf == 0.0 || divf >= 1.0)) return ORC_INVALID;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    double bnorm = norm2(n, b);
    if (bnorm == 0.0) return ORC_OK;
    pcg_state s;
    if (pcg_alloc(&s, n) != ORC_OK) return ORC_OOM;
    double r0 = pcg_start(h, &s, b, x);
    pcg_run run;
    pcg_iterate(h, &s, b, x, bnorm, tol, max_it, kwin, divf, &run);
    info->iterations = run.steps;
    info->replacements = run.replacements;
    info->final_relres = true_resnorm(h, b, x, s.q) / bnorm;
    info->conv_factor = run.steps > 0 ? pow(run.rnorm / r0, 1.0 / run.steps) : 0.0;
    info->status = run.converged ? ORC_OK
                 : run.diverged  ? ORC_DIVERGED
                 : (run.breakdown ? ORC_BREAKDOWN : ORC_NOT_CONVERGED);
    pcg_free(&s);
    return info->status;
}

/* the defaults of the library: windows of 3 steps, growth factor 1e3 */
int orc_pcg(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, orc_info *info) {
    return orc_pcg_ex(h, b, x, tol, max_it, 3, 1e3, info);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 5, adaptive_solve.  Readings of its garbled lines: the loop    */
/* runs while ||r|| / ||r_0|| > tol; every k PCG steps the true residual    */
/* r = b - A x is formed, and the per-iteration factor                      */
/* (||r_end|| / ||r_start||)^(1/k) over the window is compared with rho_max. */
/* Above it (or on a breakdown), while some coarse gamma is > 0, one        */
/* reintroduction step is taken and PCG restarts, from the current x unless */
/* the residual grew over the window, then from the window's starting x.    */
/* Otherwise the Krylov run continues unchanged.  Divergence (Section 6):   */
/* when the residual grew by more than divf over the window (or is          */
/* non-finite) and nothing is left to reintroduce, x goes back to the       */
/* window's starting iterate and the solve stops as diverged (divf = 0:     */
/* never).  With trace != NULL each window is recorded (at most cap).       */
/* ------------------------------------------------------------------------ */
static void record(orc_window *trace, int32_t cap, int32_t *ntrace, int32_t steps, double rstart, double rend,
                   double factor, int32_t action) {
    if (!trace || !ntrace) return;
    if (*ntrace < cap) {
        orc_window *w = &trace[*ntrace];
        w->steps = steps;
        w->action = action;
        w->rstart = rstart;
        w->rend = rend;
        w->factor = factor;
    }
    (*ntrace)++;
}

int orc_adaptive_solve_ex(orc_hier *h, const double *b, double *x, double tol, int32_t max_it,
                          int32_t k, int32_t s, double gamma_min, double rho_max, double divf,
                          orc_window *trace, int32_t cap, int32_t *ntrace, orc_info *info) {
    int32_t n = h->lev[0].A->nrows;
    memset(info, 0, sizeof(*info));
    if (ntrace) *ntrace = 0;
    if (k < 1 || s < 1 || !(divf == 0.0 || divf >= 1.0)) return ORC_INVALID;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    double bnorm = norm2(n, b);
    if (bnorm == 0.0) return ORC_OK;
    double *xs = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *work = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    pcg_state st;
    if (!xs || !work || pcg_alloc(&st, n) != ORC_OK) {
        free(xs); free(work);
        return ORC_OOM;
    }
    pcg_start(h, &st, b, x);
    double rstart = bnorm, rend = bnorm;
    int32_t total = 0;
    int converged = 0, breakdown = 0, diverged = 0, status = ORC_OK;
    int32_t changed[64];
    while (total < max_it) {
        memcpy(xs, x, sizeof(double) * (size_t)n);
        pcg_run run;
        int32_t steps = (max_it - total < k) ? max_it - total : k;
        pcg_iterate(h, &st, b, x, bnorm, tol, steps, k, 0.0, &run);
        total += run.steps;
        info->replacements += run.replacements;
        rend = true_resnorm(h, b, x, work);
        double factor = (run.steps > 0) ? pow(rend / rstart, 1.0 / run.steps) : 1.0;
        if (run.converged || rend <= tol * bnorm) {
            converged = 1;
            record(trace, cap, ntrace, run.steps, rstart, rend, factor, ORC_WIN_CONVERGED);
            break;
        }
        breakdown = run.breakdown;
        /* grew by more than divf, a non-finite residual included */
        int growing = divf > 0.0 && !(rend <= divf * rstart);
        int action = ORC_WIN_CONTINUE;
        if (factor > rho_max || breakdown || growing) {
            int cnt = orc_reintroduce(h, s, gamma_min, changed);
            if (cnt < 0) {
                status = -cnt;
                break;
            }
            /* a restart, or a final breakdown, goes back to the checkpoint
               whenever the residual did not decrease -- a non-finite residual
               included (!(rend <= rstart) holds for NaN) */
            int back = !(rend <= rstart);
            if (cnt == 0 && breakdown) {
                if (back) memcpy(x, xs, sizeof(double) * (size_t)n);
                record(trace, cap, ntrace, run.steps, rstart, rend, factor,
                       back ? ORC_WIN_BREAKDOWN_BACK : ORC_WIN_BREAKDOWN_STOP);
                break;
            }
            if (cnt == 0 && growing) {
                memcpy(x, xs, sizeof(double) * (size_t)n);
                diverged = 1;
                record(trace, cap, ntrace, run.steps, rstart, rend, factor, ORC_WIN_DIVERGED);
                break;
            }
            if (cnt > 0) {
                info->resets++;
                breakdown = 0;
                action = back ? ORC_WIN_RESTART_BACK : ORC_WIN_RESTART_HERE;
            } else {
                action = ORC_WIN_NOTHING_LEFT;
            }
        }
        record(trace, cap, ntrace, run.steps, rstart, rend, factor, action);
        if (action == ORC_WIN_RESTART_BACK) {
            memcpy(x, xs, sizeof(double) * (size_t)n);
            rend = rstart;
        }
        if (action == ORC_WIN_RESTART_HERE || action == ORC_WIN_RESTART_BACK) pcg_start(h, &st, b, x);
        rstart = rend;
    }
    info->iterations = total;
    info->final_relres = true_resnorm(h, b, x, work) / bnorm;
    info->conv_factor = total > 0 ? pow(info->final_relres, 1.0 / total) : 0.0;
    if (status == ORC_OK)
        status = converged ? ORC_OK
               : diverged  ? ORC_DIVERGED
               : (breakdown ? ORC_BREAKDOWN : ORC_NOT_CONVERGED);
    info->status = status;
    free(xs); free(work);
    pcg_free(&st);
    return status;
}

int orc_adaptive_solve(orc_hier *h, const double *b, double *x, double tol, int32_t max_it,
                       int32_t k, int32_t s, double gamma_min, double rho_max, orc_info *info) {
    return orc_adaptive_solve_ex(h, b, x, tol, max_it, k, s, gamma_min, rho_max, 1e3, NULL, 0, NULL, info);
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES, right-preconditioned in the flexible form (FGMRES,      */
/* Saad 1993): z_j = M v_j is kept and x = x0 + Z y.  The paper solves with */
/* GMRES where full lumping (Algorithm 3) can cost positive definiteness.   */
/* Readings: x0 = 0; Arnoldi by modified Gram-Schmidt; Givens rotations     */
/* reduce the Hessenberg matrix column by column, so |g_{j+1}| is the       */
/* residual norm of the j-step iterate; a run stops when that estimate      */
/* reaches tol ||b|| and the true residual b - A_0 x confirms it (else the  */
/* cycle restarts from x, a residual replacement), restarts after `restart` */
/* steps, and ends at max_it steps.  M is one V-cycle, or the identity in   */
/* the unpreconditioned variant.  The state is resumable: Algorithm 5 reads */
/* the iterate between checks without ending the cycle.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_csr *A;
    orc_hier *h;        /* preconditioner: V-cycle of h, or NULL = identity */
    int32_t n, m, j;    /* size, restart length, steps in the current cycle */
    double *V, *Z;      /* (m + 1) x n and m x n, row j = vector j */
    double *H;          /* (m + 1) x m, H[i * m + c] */
    double *cs, *sn, *g, *y, *x0, *w;
} gm_state;

typedef struct {
    int32_t steps, converged, breakdown, replacements;
    double rnorm; /* residual estimate (or true residual at convergence) */
} gm_run;

static void gm_free(gm_state *s) {
    free(s->V); free(s->Z); free(s->H); free(s->cs); free(s->sn); free(s->g); free(s->y);
    free(s->x0); free(s->w);
    memset(s, 0, sizeof(*s));
}

static int gm_alloc(gm_state *s, const orc_csr *A, orc_hier *h, int32_t m) {
    memset(s, 0, sizeof(*s));
    s->A = A;
    s->h = h;
    s->n = A->nrows;
    s->m = m;
    size_t n = (size_t)(s->n > 0 ? s->n : 1);
    s->V = (double *)calloc(n * (size_t)(m + 1), sizeof(double));
    s->Z = (double *)calloc(n * (size_t)m, sizeof(double));
    s->H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    s->cs = (double *)calloc((size_t)m, sizeof(double));
    s->sn = (double *)calloc((size_t)m, sizeof(double));
    s->g = (double *)calloc((size_t)m + 1, sizeof(double));
    s->y = (double *)calloc((size_t)m, sizeof(double));
    s->x0 = (double *)calloc(n, sizeof(double));
    s->w = (double *)calloc(n, sizeof(double));
    if (!s->V || !s->Z || !s->H || !s->cs || !s->sn || !s->g || !s->y || !s->x0 || !s->w) {
        gm_free(s);
        return ORC_OOM;
    }
    return ORC_OK;
}

/* new cycle from x: v_0 = r / ||r||, g = ||r|| e_1; returns ||r|| */
static double gm_start(gm_state *s, const double *b, const double *x) {
    int32_t n = s->n;
    orc_spmv(s->A, x, s->w);
    for (int32_t i = 0; i < n; ++i) s->w[i] = b[i] - s->w[i];
    double beta = norm2(n, s->w);
    for (int32_t i = 0; i < n; ++i) s->V[i] = (beta > 0.0) ? s->w[i] / beta : 0.0;
    memcpy(s->x0, x, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i <= s->m; ++i) s->g[i] = 0.0;
    s->g[0] = beta;
    s->j = 0;
    return beta;
}

/* x = x0 + Z y with R y = g over the cycle's first j steps (back substitution) */
static void gm_form_x(gm_state *s, double *x) {
    int32_t n = s->n, m = s->m, j = s->j;
    for (int32_t i = j - 1; i >= 0; --i) {
        double t = s->g[i];
        for (int32_t c = i + 1; c < j; ++c) t -= s->H[(size_t)i * m + c] * s->y[c];
        s->y[i] = t / s->H[(size_t)i * m + i];
    }
    for (int32_t e = 0; e < n; ++e) {
        double t = s->x0[e];
        for (int32_t i = 0; i < j; ++i) t += s->y[i] * s->Z[(size_t)i * n + e];
        x[e] = t;
    }
}

static void gm_iterate(gm_state *s, const double *b, double *x, double bnorm, double tol, int32_t max_steps,
                       gm_run *run) {
    int32_t n = s->n, m = s->m;
    memset(run, 0, sizeof(*run));
    run->rnorm = fabs(s->g[s->j]);
    if (run->rnorm <= tol * bnorm) {
        run->converged = 1;
        return;
    }
    while (run->steps < max_steps) {
        if (s->j == m) {                        /* restart */
            gm_form_x(s, x);
            gm_start(s, b, x);
        }
        int32_t j = s->j;
        double *vj = s->V + (size_t)j * n, *zj = s->Z + (size_t)j * n, *w = s->w;
        if (s->h) orc_vcycle(s->h, vj, zj);
        else memcpy(zj, vj, sizeof(double) * (size_t)n);
        orc_spmv(s->A, zj, w);
        run->steps++;
        for (int32_t i = 0; i <= j; ++i) {      /* modified Gram-Schmidt */
            const double *vi = s->V + (size_t)i * n;
            double hij = dot(n, w, vi);
            s->H[(size_t)i * m + j] = hij;
            for (int32_t e = 0; e < n; ++e) w[e] -= hij * vi[e];
        }
        double hn = norm2(n, w);
        if (!isfinite(hn)) {                    /* the step is lost: keep the iterate of j steps */
            run->breakdown = 1;
            gm_form_x(s, x);
            return;
        }
        s->H[(size_t)(j + 1) * m + j] = hn;
        double *vn = s->V + (size_t)(j + 1) * n;
        for (int32_t e = 0; e < n; ++e) vn[e] = (hn > 0.0) ? w[e] / hn : 0.0;
        for (int32_t i = 0; i < j; ++i) {       /* earlier rotations on column j */
            double a = s->H[(size_t)i * m + j], c = s->H[(size_t)(i + 1) * m + j];
            s->H[(size_t)i * m + j] = s->cs[i] * a + s->sn[i] * c;
            s->H[(size_t)(i + 1) * m + j] = -s->sn[i] * a + s->cs[i] * c;
        }
        double a = s->H[(size_t)j * m + j], c = hn;
        double r = sqrt(a * a + c * c);
        s->cs[j] = (r > 0.0) ? a / r : 1.0;
        s->sn[j] = (r > 0.0) ? c / r : 0.0;
        s->H[(size_t)j * m + j] = r;
        s->H[(size_t)(j + 1) * m + j] = 0.0;
        s->g[j + 1] = -s->sn[j] * s->g[j];
        s->g[j] = s->cs[j] * s->g[j];
        s->j = j + 1;
        run->rnorm = fabs(s->g[j + 1]);
        if (!(r > 0.0)) {                       /* singular Hessenberg column */
            run->breakdown = 1;
            s->j = j;
            gm_form_x(s, x);
            return;
        }
        if (run->rnorm <= tol * bnorm || hn == 0.0) {
            gm_form_x(s, x);
            double tn = gm_start(s, b, x);
            run->rnorm = tn;
            if (tn <= tol * bnorm) {
                run->converged = 1;
                return;
            }
            run->replacements++;
        }
    }
    gm_form_x(s, x);
}

static int gmres_solve(const orc_csr *A, orc_hier *h, const double *b, double *x, double tol, int32_t max_it,
                       int32_t restart, orc_info *info) {
    int32_t n = A->nrows;
    memset(info, 0, sizeof(*info));
    if (restart < 1 || max_it < 0) return ORC_INVALID;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    double bnorm = norm2(n, b);
    if (bnorm == 0.0) return ORC_OK;
    gm_state s;
    if (gm_alloc(&s, A, h, restart) != ORC_OK) return ORC_OOM;
    double r0 = gm_start(&s, b, x);
    gm_run run;
    gm_iterate(&s, b, x, bnorm, tol, max_it, &run);
    orc_spmv(A, x, s.w);
    double t = 0.0;
    for (int32_t i = 0; i < n; ++i) t += (b[i] - s.w[i]) * (b[i] - s.w[i]);
    info->iterations = run.steps;
    info->replacements = run.replacements;
    info->final_relres = sqrt(t) / bnorm;
    info->conv_factor = run.steps > 0 ? pow(run.rnorm / r0, 1.0 / run.steps) : 0.0;
    info->status = run.converged ? ORC_OK : (run.breakdown ? ORC_BREAKDOWN : ORC_NOT_CONVERGED);
    gm_free(&s);
    return info->status;
}

int orc_gmres(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, int32_t restart,
              orc_info *info) {
    return gmres_solve(h->lev[0].A, h, b, x, tol, max_it, restart, info);
}

int orc_gmres_plain(const orc_csr *A, const double *b, double *x, double tol, int32_t max_it, int32_t restart,
                    orc_info *info) {
    return gmres_solve(A, NULL, b, x, tol, max_it, restart, info);
}

/* Algorithm 5 around GMRES: as orc_adaptive_solve, every k steps the       */
/* iterate is formed (the cycle goes on) and its true residual checked; a  */
/* reintroduction ends the cycle and GMRES restarts with the new M.         */
int orc_adaptive_gmres(orc_hier *h, const double *b, double *x, double tol, int32_t max_it, int32_t restart,
                       int32_t k, int32_t s, double gamma_min, double rho_max, orc_info *info) {
    int32_t n = h->lev[0].A->nrows;
    memset(info, 0, sizeof(*info));
    if (k < 1 || s < 1 || restart < 1) return ORC_INVALID;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    double bnorm = norm2(n, b);
    if (bnorm == 0.0) return ORC_OK;
    double *xs = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *work = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    gm_state st;
    if (!xs || !work || gm_alloc(&st, h->lev[0].A, h, restart) != ORC_OK) {
        free(xs); free(work);
        return ORC_OOM;
    }
    gm_start(&st, b, x);
    double rstart = bnorm, rend = bnorm;
    int32_t total = 0;
    int converged = 0, breakdown = 0, status = ORC_OK;
    int32_t changed[64];
    while (total < max_it) {
        memcpy(xs, x, sizeof(double) * (size_t)n);
        gm_run run;
        int32_t steps = (max_it - total < k) ? max_it - total : k;
        gm_iterate(&st, b, x, bnorm, tol, steps, &run);
        total += run.steps;
        info->replacements += run.replacements;
        rend = true_resnorm(h, b, x, work);
        if (run.converged || rend <= tol * bnorm) {
            converged = 1;
            break;
        }
        breakdown = run.breakdown;
        double factor = (run.steps > 0) ? pow(rend / rstart, 1.0 / run.steps) : 1.0;
        if (factor > rho_max || breakdown) {
            int cnt = orc_reintroduce(h, s, gamma_min, changed);
            if (cnt < 0) {
                status = -cnt;
                break;
            }
            if (cnt == 0 && breakdown) {
                if (!(rend <= rstart)) memcpy(x, xs, sizeof(double) * (size_t)n);
                break;
            }
            if (cnt > 0) {
                info->resets++;
                breakdown = 0;
                if (!(rend <= rstart)) {
                    memcpy(x, xs, sizeof(double) * (size_t)n);
                    rend = rstart;
                }
                gm_start(&st, b, x);
            }
        }
        rstart = rend;
    }
    info->iterations = total;
    info->final_relres = true_resnorm(h, b, x, work) / bnorm;
    info->conv_factor = total > 0 ? pow(info->final_relres, 1.0 / total) : 0.0;
    if (status == ORC_OK)
        status = converged ? ORC_OK : (breakdown ? ORC_BREAKDOWN : ORC_NOT_CONVERGED);
    info->status = status;
    free(xs); free(work);
    gm_free(&st);
    return status;
}

/* ------------------------------------------------------------------------ */
/* accessors                                                                 */
/* ------------------------------------------------------------------------ */
int32_t orc_num_levels(const orc_hier *h) { return h->nlev; }

/* which: 0 A (Galerkin), 1 Ahat, 2 P, 3 R, 4 AP */
const orc_csr *orc_level_matrix(const orc_hier *h, int32_t l, int32_t which) {
    if (l < 0 || l >= h->nlev) return NULL;
    const orc_level *L = &h->lev[l];
    switch (which) {
        case 0: return L->A;
        case 1: return L->Ahat;
        case 2: return L->P;
        case 3: return L->R;
        case 4: return L->AP;
        default: return NULL;
    }
}

/* which: 0 strong (u8/nnz A), 1 cf (i8/n), 2 inM (u8/nnz A), 3 keep (u8/nnz A), 4 d (f64/n), 5 chol */
const void *orc_level_array(const orc_hier *h, int32_t l, int32_t which) {
    if (l < 0 || l >= h->nlev) return NULL;
    const orc_level *L = &h->lev[l];
    switch (which) {
        case 0: return L->strong;
        case 1: return L->cf;
        case 2: return L->inM;
        case 3: return L->keep;
        case 4: return L->d;
        case 5: return (l == h->nlev - 1) ? h->chol : NULL;
        default: return NULL;
    }
}

double orc_level_gamma(const orc_hier *h, int32_t l) {
    return (l >= 0 && l < h->nlev) ? h->lev[l].gamma : -1.0;
}
