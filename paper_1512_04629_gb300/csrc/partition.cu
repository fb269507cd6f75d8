// partition.cu -- row-partitioned execution of a hierarchy (amg_partition).
//
// The paper solves on many processes, each owning a contiguous block of rows
// of every level (Section 2, parallel SpMV), and measures what sparsification
// saves in communication (Section 4: messages and values per product).  Here
// the blocks of one process group run on one GPU: every level's rows are
// split into `parts` blocks -- the finest in blocks of n / parts rows, each
// coarser one so that every block keeps the C points of its fine rows, as
// distributed AMG keeps coarse points on their owners -- and each operator of
// the solve gets its halo plan (halo_plan.cpp).  Before a product the
// exchange kernel fills every block's ghost buffer from the global vector
// (the values a distributed run would receive in messages), then the block's
// rows multiply its own columns and its ghosts.
#include <algorithm>
#include <cstring>
#include <stdexcept>
#include <string>

#include "halo_plan.h"
#include "hierarchy.cuh"

namespace amg {

void set_last_error(const std::string &msg);

namespace {

// Plans M (rows split at row0, columns owned as split at col0) and returns
// its receive counts; with P given, also uploads the plan into P.
void plan_operator(const DevCSR &M, int parts, const std::vector<int64_t> &row0, const std::vector<int64_t> &col0,
                   PartOp *P, std::vector<int64_t> &recv, cudaStream_t s) {
    const int64_t n = M.nrows, nnz = M.nnz;
    std::vector<int32_t> rp(n + 1), ci(nnz > 0 ? nnz : 1), cext(nnz > 0 ? nnz : 1);
    AMG_CUDA(cudaMemcpyAsync(rp.data(), M.rp(), sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    if (nnz) AMG_CUDA(cudaMemcpyAsync(ci.data(), M.ci(), sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> goff;
    std::vector<int32_t> gcol;
    try {
        halo_plan(n, M.ncols, rp.data(), ci.data(), parts, row0.data(), col0.data(), cext.data(), goff, gcol, recv);
    } catch (const std::invalid_argument &e) {
        throw Error(AMG_ERR_INVALID, e.what());
    }
    if (!P) return;
    P->parts = parts;
    P->nghost = (int64_t)gcol.size();
    P->recv = recv;
    P->cext.alloc(sizeof(int32_t) * (nnz + kPad));
    P->gcol.alloc(sizeof(int32_t) * (P->nghost + kPad));
    P->gbuf.alloc(sizeof(double) * (P->nghost + kPad));
    std::vector<int32_t> bounds(3 * (parts + 1));
    for (int p = 0; p <= parts; ++p) {
        bounds[p] = (int32_t)row0[p];
        bounds[parts + 1 + p] = (int32_t)col0[p];
        bounds[2 * (parts + 1) + p] = (int32_t)goff[p];
    }
    P->bounds.alloc(sizeof(int32_t) * bounds.size());
    if (nnz) AMG_CUDA(cudaMemcpyAsync(P->cext.ptr, cext.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
    if (P->nghost)
        AMG_CUDA(cudaMemcpyAsync(P->gcol.ptr, gcol.data(), sizeof(int32_t) * P->nghost, cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(P->bounds.ptr, bounds.data(), sizeof(int32_t) * bounds.size(), cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
}

void clear_partition(Hierarchy &h) {
    for (auto &L : h.lev) {
        L->part_h.reset();
        L->part_p.reset();
        L->part_r.reset();
        L->prow0.clear();
        L->recv_galerkin.clear();
    }
    h.parts = 1;
}

// row blocks of every level: balanced on the finest, C points kept with
// their fine rows below (C points are numbered in fine-row order, so the
// coarse block p is the run of C points among the fine block p's rows)
void split_rows(Hierarchy &h, int parts, cudaStream_t s) {
    const int L = h.nlev();
    Level &V0 = *h.lev[0];
    V0.prow0.assign(parts + 1, 0);
    for (int p = 0; p <= parts; ++p) V0.prow0[p] = (int64_t)p * V0.n() / parts;
    for (int l = 0; l + 1 < L; ++l) {
        Level &V = *h.lev[l];
        require(V.cf.ptr != nullptr, "amg_partition: level " + std::to_string(l) + " lacks its C/F split");
        std::vector<int8_t> cf(V.n() > 0 ? V.n() : 1);
        AMG_CUDA(cudaMemcpyAsync(cf.data(), V.cf.ptr, V.n(), cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> &c0 = h.lev[l + 1]->prow0;
        c0.assign(parts + 1, 0);
        int64_t count = 0, i = 0;
        for (int p = 0; p <= parts; ++p) {
            for (; i < V.prow0[p]; ++i) count += cf[i] == 1;
            c0[p] = count;
        }
        require(c0[parts] == h.lev[l + 1]->n(), "amg_partition: C points do not match the coarse level");
    }
}

void plan_level(Hierarchy &h, int l, cudaStream_t s) {
    const int parts = h.parts;
    Level &V = *h.lev[l];
    std::vector<int64_t> recv;
    V.part_h = std::make_unique<PartOp>();
    plan_operator(V.op(), parts, V.prow0, V.prow0, V.part_h.get(), recv, s);
    plan_operator(V.A, parts, V.prow0, V.prow0, nullptr, V.recv_galerkin, s);
    if (l + 1 < h.nlev()) {
        const std::vector<int64_t> &c0 = h.lev[l + 1]->prow0;
        V.part_p = std::make_unique<PartOp>();
        plan_operator(V.P, parts, V.prow0, c0, V.part_p.get(), recv, s);
        V.part_r = std::make_unique<PartOp>();
        plan_operator(V.R, parts, c0, V.prow0, V.part_r.get(), recv, s);
    }
}

// messages (ordered pairs p <- q, p != q, with values) and values of a
// parts x parts receive matrix; the largest of each over receiving blocks
void summarise(const std::vector<int64_t> &recv, int parts, int64_t &msgs, int64_t &vals, int64_t *max_msgs,
               int64_t *max_vals) {
    msgs = vals = 0;
    int64_t mm = 0, mv = 0;
    for (int p = 0; p < parts && !recv.empty(); ++p) {
        int64_t m = 0, v = 0;
        for (int q = 0; q < parts; ++q) {
            const int64_t r = recv[(size_t)p * parts + q];
            if (q != p && r > 0) { m++; v += r; }
        }
        msgs += m;
        vals += v;
        mm = std::max(mm, m);
        mv = std::max(mv, v);
    }
    if (max_msgs) *max_msgs = mm;
    if (max_vals) *max_vals = mv;
}

template <class F> amg_status guarded_call(F &&f) {
    try {
        set_last_error("");
        return f();
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return AMG_ERR_OOM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return AMG_ERR_CUDA;
    }
}

}  // namespace

void replan_relaxation(Hierarchy &h, int l, cudaStream_t s) {
    if (h.parts <= 1 || l < 0 || l >= h.nlev()) return;
    Level &V = *h.lev[l];
    std::vector<int64_t> recv;
    V.part_h = std::make_unique<PartOp>();
    plan_operator(V.op(), h.parts, V.prow0, V.prow0, V.part_h.get(), recv, s);
}

}  // namespace amg

using namespace amg;

extern "C" amg_status amg_partition(amg_hierarchy *H, int parts) {
    return guarded_call([&] {
        require(H != nullptr, "hierarchy is NULL");
        require(parts >= 1 && parts <= kMaxParts, "parts must be in [1, 64]");
        Hierarchy &h = H->h;
        require(h.opt.precision == AMG_PREC_FP64, "row-partitioned solves run in FP64 precision only");
        cudaStream_t s = nullptr;
        AllocOn alloc_scope(s);
        try {
            clear_partition(h);
            if (parts > 1) {
                h.parts = parts;
                split_rows(h, parts, s);
                for (int l = 0; l < h.nlev(); ++l) plan_level(h, l, s);
            }
        } catch (...) {
            clear_partition(h);
            h.graph_dirty = true;
            h.version++;
            throw;
        }
        h.graph_dirty = true;  // the captured iterations launch other kernels now
        h.version++;
        AMG_CUDA(cudaStreamSynchronize(s));
        return AMG_OK;
    });
}

extern "C" amg_status amg_comm_stats(const amg_hierarchy *H, int level, amg_comm_info *out) {
    return guarded_call([&] {
        require(H != nullptr && out != nullptr, "NULL argument");
        const Hierarchy &h = H->h;
        require(level >= 0 && level < h.nlev(), "level out of range");
        const Level &V = *h.lev[level];
        std::memset(out, 0, sizeof(*out));
        out->parts = h.parts;
        if (h.parts <= 1 || !V.part_h) return AMG_OK;
        summarise(V.part_h->recv, h.parts, out->messages, out->halo_values, &out->max_messages, &out->max_halo);
        summarise(V.recv_galerkin, h.parts, out->messages_galerkin, out->halo_galerkin, nullptr, nullptr);
        if (V.part_p) summarise(V.part_p->recv, h.parts, out->messages_p, out->halo_p, nullptr, nullptr);
        if (V.part_r) summarise(V.part_r->recv, h.parts, out->messages_r, out->halo_r, nullptr, nullptr);
        return AMG_OK;
    });
}

extern "C" amg_status amg_partition_rows(const amg_hierarchy *H, int level, int64_t *row0) {
    return guarded_call([&] {
        require(H != nullptr && row0 != nullptr, "NULL argument");
        const Hierarchy &h = H->h;
        require(level >= 0 && level < h.nlev(), "level out of range");
        const Level &V = *h.lev[level];
        if (h.parts <= 1) {
            row0[0] = 0;
            row0[1] = V.n();
            return AMG_OK;
        }
        std::copy(V.prow0.begin(), V.prow0.end(), row0);
        return AMG_OK;
    });
}
