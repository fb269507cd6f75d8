// setup_ops.cuh -- host entry points of the setup kernels (setup.cu).
#pragma once
#include "common.cuh"

namespace amg {
namespace setup {

// Checks squareness, sortedness, column range, finite values, a stored
// positive diagonal and a symmetric pattern; writes the diagonal position of
// every row and the position of the mirrored entry (j,i) of every stored
// (i,j).  Throws AMG_ERR_INVALID naming every failed check.  check = false
// skips the read-back of the checks (a Galerkin product this library formed:
// sorted rows and a symmetric pattern by construction).
void level_maps(const DevCSR &A, int32_t *diagpos, int32_t *tpos, cudaStream_t s, bool check = true);
// Row pointers, column range, strictly increasing columns and finite values of
// a rectangular operator; throws AMG_ERR_INVALID naming `what`.
void validate_rect(const DevCSR &M, const char *what, cudaStream_t s);
// Classical strength flags (one byte per stored entry).
void strength(const DevCSR &A, double theta, uint8_t *strong, cudaStream_t s);
// PMIS C/F splitting; cf[i] = 1 (C) / -1 (F); cmap (n + 1 entries) receives
// the exclusive scan of the C flags (the coarse number of every C point);
// returns |C|.
int64_t pmis(const DevCSR &A, const uint8_t *strong, const int32_t *tpos, uint64_t seed,
             int32_t level, int8_t *cf, int32_t *cmap, cudaStream_t s);
// cpts[c] = fine index of coarse point c, from cf and the scanned cmap;
// cmap[i] becomes -1 at F points.
void coarse_points(const int8_t *cf, int32_t n, int32_t *cmap, int32_t *cpts, cudaStream_t s);
// Coarse numbering from cf alone: the scan into cmap, then coarse_points;
// throws AMG_ERR_INVALID unless cf marks exactly nc C points (cpts holds nc).
void coarse_map(const int8_t *cf, int32_t n, int32_t *cmap, int32_t *cpts, int64_t nc, cudaStream_t s);
// Direct interpolation P (n x nc).
void direct_interp(const DevCSR &A, const uint8_t *strong, const int8_t *cf, const int32_t *cmap,
                   int32_t nc, DevCSR &P, cudaStream_t s);
// R = P^T with sorted rows.
void transpose(const DevCSR &P, DevCSR &R, cudaStream_t s);
// Rows of a sparse operand: row i holds ci / v[beg[i] .. end[i]), sorted by
// column; a CSR matrix is beg = rowptr, end = rowptr + 1.
struct SpRows {
    const int32_t *beg = nullptr, *end = nullptr, *ci = nullptr;
    const double *v = nullptr;
    int32_t nrows = 0, ncols = 0;
};
inline SpRows rows_of(const DevCSR &M) { return SpRows{M.rp(), M.rp() + 1, M.ci(), M.v(), M.nrows, M.ncols}; }
// A product kept where the one-pass SpGEMM wrote it: row i's sorted entries
// at the start of its slot (sized by the row's product count), with no
// compaction; when the products would not fit in memory the product is
// formed as a CSR matrix instead.  `rows` views either form.
struct SlotProduct {
    DevCSR csr;
    TmpBuf ci, v, beg, end;
    SpRows rows;
};
// C = A B (structural, deterministic, sorted rows).
void spgemm(const DevCSR &A, const SpRows &B, DevCSR &C, cudaStream_t s);
inline void spgemm(const DevCSR &A, const DevCSR &B, DevCSR &C, cudaStream_t s) { spgemm(A, rows_of(B), C, s); }
// A B left in its product slots (for an operand that is read, not kept).
void spgemm_slots(const DevCSR &A, const DevCSR &B, SlotProduct &C, cudaStream_t s);
// Minimal-pattern flags of Ac's entries from the C rows of AP; tpos (the
// mirrored-entry positions of Ac's symmetric pattern), when given, lets each
// entry be tested in its own row only.
void minimal_pattern(const DevCSR &Ac, const SpRows &AP, const int32_t *cpts, uint8_t *inM, cudaStream_t s,
                     const int32_t *tpos = nullptr);
// Hybrid variant: pattern of Phat^T Ahat P (+ transpose) with Ahat the
// sparsified fine operator.  Recomputes AP from Ahat.
// Sparsify (Algorithm 3's drop test and symmetric N); fills keep[] and Ahat;
// returns nnz(Ahat).  S == nullptr: diagonal lumping (Algorithm 3b, with its
// ismax guard); otherwise full lumping to the strong neighbours given by the
// strength flags S of A (Algorithm 3's own loop).
int64_t sparsify(const DevCSR &A, const uint8_t *inM, const int32_t *tpos, const int32_t *diagpos,
                 double gamma, uint8_t *keep, DevCSR &Ahat, cudaStream_t s, const uint8_t *S = nullptr);
// Copy of A (Ahat = A when gamma = 0) with keep[] = 1.
void copy_all(const DevCSR &A, uint8_t *keep, DevCSR &Ahat, cudaStream_t s);
// ell1 diagonal d_i = sum_j |a_ij| and its inverse.
void l1_diag(const DevCSR &A, double *d, double *dinv, cudaStream_t s);
// Dense inverse of the coarsest operator through its Cholesky factor; when a
// Cholesky pivot is not positive, by Gauss-Jordan elimination with partial
// pivoting.  Throws AMG_BREAKDOWN if the operator is singular.
void cholesky_inverse(const DevCSR &A, double *inv, cudaStream_t s);

}  // namespace setup
}  // namespace amg
