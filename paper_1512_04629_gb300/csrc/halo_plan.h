// halo_plan.h -- host-side communication plan of a row-partitioned operator
// (halo_plan.cpp); used by amg_halo_plan and amg_partition.
#pragma once
#include <cstdint>
#include <vector>

namespace amg {

constexpr int kMaxParts = 64;

// Rows [row0[p], row0[p+1]) belong to block p, which owns columns
// [col0[p], col0[p+1]).  Fills cext (one per stored entry: the column in
// block-local numbering -- owned columns 0 .. nloc-1, then ghosts), goff
// (parts + 1: block p's ghosts are gcol[goff[p] .. goff[p+1]), increasing
// global columns) and recv (parts x parts: values block p receives from q).
// Throws std::invalid_argument on inconsistent input.
void halo_plan(int64_t nrows, int64_t ncols, const int32_t *rowptr, const int32_t *col, int parts,
               const int64_t *row0, const int64_t *col0, int32_t *cext, std::vector<int64_t> &goff,
               std::vector<int32_t> &gcol, std::vector<int64_t> &recv);

}  // namespace amg
