// halo_plan.cpp -- communication plan of a row-partitioned sparse operator.
//
// The paper's parallel SpMV (Section 2) splits a matrix by contiguous row
// blocks, one per process: the columns a block owns form its diagonal block,
// every other column is off-diagonal, and the values of those columns --
// ghosts -- must be received from their owners before each product.  Its
// cost model (Section 4) counts, per product, the messages (process pairs
// that exchange values) and the values sent.  This file builds that plan on
// the host, as a distributed solver builds its communication package: no GPU
// is involved, so the plan can be computed and checked on any machine.
#include <algorithm>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "amg.h"
#include "halo_plan.h"

namespace amg {

void set_last_error(const std::string &msg);

void halo_plan(int64_t nrows, int64_t ncols, const int32_t *rowptr, const int32_t *col, int parts,
               const int64_t *row0, const int64_t *col0, int32_t *cext, std::vector<int64_t> &goff,
               std::vector<int32_t> &gcol, std::vector<int64_t> &recv) {
    auto bad = [](const std::string &m) { throw std::invalid_argument("halo plan: " + m); };
    if (parts < 1 || parts > kMaxParts) bad("parts must be in [1, " + std::to_string(kMaxParts) + "]");
    if (nrows < 0 || ncols < 0 || !rowptr || (!col && rowptr[nrows] > 0)) bad("bad matrix");
    if (!row0 || !col0) bad("NULL partition bounds");
    if (row0[0] != 0 || row0[parts] != nrows || col0[0] != 0 || col0[parts] != ncols)
        bad("partition bounds must run from 0 to the row / column count");
    for (int p = 0; p < parts; ++p)
        if (row0[p + 1] < row0[p] || col0[p + 1] < col0[p]) bad("partition bounds must not decrease");
    goff.assign(parts + 1, 0);
    gcol.clear();
    recv.assign((size_t)parts * parts, 0);
    std::vector<int32_t> ghosts;
    for (int p = 0; p < parts; ++p) {
        const int64_t c0 = col0[p], c1 = col0[p + 1];
        const int32_t nloc = (int32_t)(c1 - c0);
        ghosts.clear();
        for (int64_t i = row0[p]; i < row0[p + 1]; ++i)
            for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                const int32_t j = col[q];
                if (j < 0 || j >= ncols) bad("column out of range");
                if (j < c0 || j >= c1) ghosts.push_back(j);
            }
        std::sort(ghosts.begin(), ghosts.end());
        ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
        // each entry in the block's local numbering: owned columns first, then ghosts
        for (int64_t i = row0[p]; i < row0[p + 1]; ++i)
            for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                const int32_t j = col[q];
                if (j >= c0 && j < c1) {
                    cext[q] = j - (int32_t)c0;
                } else {
                    auto it = std::lower_bound(ghosts.begin(), ghosts.end(), j);
                    cext[q] = nloc + (int32_t)(it - ghosts.begin());
                }
            }
        // the owner of each ghost: ghosts are increasing, owners' ranges contiguous
        int owner = 0;
        for (int32_t j : ghosts) {
            while (owner + 1 < parts && col0[owner + 1] <= j) ++owner;
            recv[(size_t)p * parts + owner]++;
        }
        gcol.insert(gcol.end(), ghosts.begin(), ghosts.end());
        goff[p + 1] = (int64_t)gcol.size();
    }
}

}  // namespace amg

extern "C" amg_status amg_halo_plan(int64_t nrows, int64_t ncols, const int32_t *rowptr, const int32_t *col,
                                    int parts, const int64_t *row0, const int64_t *col0, int32_t *cext,
                                    int64_t *goff, int32_t *gcol, int64_t *recv) {
    try {
        amg::set_last_error("");
        if (!cext || !goff || !gcol || !recv) throw std::invalid_argument("halo plan: NULL output");
        std::vector<int64_t> go, rv;
        std::vector<int32_t> gc;
        amg::halo_plan(nrows, ncols, rowptr, col, parts, row0, col0, cext, go, gc, rv);
        std::copy(go.begin(), go.end(), goff);
        std::copy(gc.begin(), gc.end(), gcol);
        std::copy(rv.begin(), rv.end(), recv);
        return AMG_OK;
    } catch (const std::invalid_argument &e) {
        amg::set_last_error(e.what());
        return AMG_ERR_INVALID;
    } catch (const std::bad_alloc &) {
        amg::set_last_error("halo plan: host allocation failed");
        return AMG_ERR_OOM;
    }
}
