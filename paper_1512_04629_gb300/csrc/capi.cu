// capi.cu -- the extern "C" boundary of libamg.so (declared in include/amg.h).
// Each call validates its arguments before any launch, converts internal
// errors to amg_status and leaves a thread-local message in amg_last_error().
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>

#include "common.cuh"
#include "hierarchy.cuh"

namespace amg {
const char *last_error_cstr();
extern std::atomic<int64_t> g_device_bytes;
extern std::atomic<int64_t> g_launches;
}  // namespace amg

using namespace amg;

namespace {

template <class F> amg_status guarded(F &&f) {
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
    } catch (...) {
        set_last_error("unknown error");
        return AMG_ERR_CUDA;
    }
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void check_csr_header(const amg_csr *A, bool square) {
    require(A != nullptr, "matrix is NULL");
    require(A->n > 0 && A->n < ((int64_t)1 << 31), "matrix rows must be in [1, 2^31)");
    require(A->nnz >= 0 && A->nnz < ((int64_t)1 << 31), "matrix must have fewer than 2^31 entries");
    int64_t nc = A->ncols > 0 ? A->ncols : A->n;
    require(nc < ((int64_t)1 << 31), "matrix columns must be < 2^31");
    if (square) require(nc == A->n, "matrix must be square");
    require(A->rowptr && (A->nnz == 0 || (A->col && A->val)), "matrix arrays are NULL");
    if (A->on_device)
        require(is_device_ptr(A->rowptr) && (A->nnz == 0 || (is_device_ptr(A->col) && is_device_ptr(A->val))),
                "on_device = 1 but the matrix arrays are not device memory");
}

// Upload (or copy on device) a caller CSR; checks rowptr consistency.
void upload_csr(const amg_csr *A, DevCSR &M, cudaStream_t s) {
    int64_t nc = A->ncols > 0 ? A->ncols : A->n;
    M.allocate((int32_t)A->n, (int32_t)nc, A->nnz);
    cudaMemcpyKind k = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // the row pointers' order and ends (rowptr[0] = 0, rowptr[n] = nnz), the
    // column range and finite values are checked on the device (level_maps /
    // validate_rect) before any kernel follows them; host arrays are checked
    // here as well, for the message
    if (!A->on_device)
        require(A->rowptr[0] == 0 && A->rowptr[A->n] == A->nnz, "rowptr[0] must be 0 and rowptr[n] = nnz");
    require(A->n > 0 || A->nnz == 0, "a matrix without rows holds no entries (rowptr[n] = nnz)");
    AMG_CUDA(cudaMemcpyAsync(M.rowptr.ptr, A->rowptr, sizeof(int32_t) * (A->n + 1), k, s));
    // only the padding past nnz needs zeros: the copies fill the rest
    AMG_CUDA(cudaMemsetAsync(M.ci() + A->nnz, 0, M.col.bytes - sizeof(int32_t) * A->nnz, s));
    AMG_CUDA(cudaMemsetAsync(M.v() + A->nnz, 0, M.val.bytes - sizeof(double) * A->nnz, s));
    if (A->nnz > 0) {
        AMG_CUDA(cudaMemcpyAsync(M.col.ptr, A->col, sizeof(int32_t) * A->nnz, k, s));
        AMG_CUDA(cudaMemcpyAsync(M.val.ptr, A->val, sizeof(double) * A->nnz, k, s));
    }
}

void check_options(const amg_options &o) {
    require(std::isfinite(o.theta) && o.theta >= 0.0 && o.theta <= 1.0, "theta must be in [0, 1]");
    require(o.max_size >= 1, "max_size must be >= 1");
    require(o.max_levels >= 1 && o.max_levels <= kMaxLevels, "max_levels must be in [1, 64]");
    require(o.method == AMG_METHOD_SPARSE || o.method == AMG_METHOD_HYBRID || o.method == AMG_METHOD_NONGALERKIN,
            "unknown method");
    require(o.precision >= AMG_PREC_FP64 && o.precision <= AMG_PREC_FP32_BF16, "unknown precision");
    require(o.k_check >= 1 && o.s_levels >= 1, "k_check and s_levels must be >= 1");
    require(o.gamma_min >= 0.0 && std::isfinite(o.rho_max), "bad gamma_min / rho_max");
    require(o.spmv_variant == AMG_SPMV_AUTO || (o.spmv_variant >= AMG_SPMV_CSR2 && o.spmv_variant <= AMG_SPMV_SELL8),
            "unknown spmv_variant");
    require(o.check_every >= 1, "check_every must be >= 1");
    require(o.lump == AMG_LUMP_DIAG || o.lump == AMG_LUMP_STRONG, "unknown lump");
    require(o.krylov == AMG_KRYLOV_CG || o.krylov == AMG_KRYLOV_GMRES, "unknown krylov");
    require(o.restart >= 1 && o.restart <= 512, "restart must be in [1, 512]");
    require(o.div_factor == 0.0 || (std::isfinite(o.div_factor) && o.div_factor >= 1.0),
            "div_factor must be 0 (off) or a finite value >= 1");
    require(o.transfer_variant == AMG_SPMV_AUTO ||
                (o.transfer_variant >= AMG_SPMV_CSR2 && o.transfer_variant <= AMG_SPMV_SELL8),
            "unknown transfer_variant");
}

void check_gammas(const double *g, int n) {
    require(n >= 0, "n_gamma must be >= 0");
    if (n > 0) {
        require(g != nullptr, "gamma_per_level is NULL");
        require(g[0] == 0.0, "gamma_per_level[0] must be 0: level 0 is never sparsified");
        for (int i = 0; i < n; ++i) require(std::isfinite(g[i]) && g[i] >= 0.0, "gamma must be finite and >= 0");
    }
}

void finish_setup(Hierarchy &h, const double *gamma, int n_gamma, cudaStream_t s) {
    apply_gammas(h, gamma, n_gamma, s);
    std::vector<int> all;
    for (int l = 0; l < h.nlev(); ++l) all.push_back(l);
    prepare_cycle(h, s, all);
    ensure_workspace(h, s);
    AMG_CUDA(cudaStreamSynchronize(s));
    if (h.opt.setup_timing) {  // setup phases were timed; the solve timing stays opt-in
        timing_collect(h);
        h.timing = false;
    }
}

}  // namespace

extern "C" {

void amg_options_default(amg_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->theta = 0.25;
    o->max_size = 100;
    o->max_levels = 25;
    o->seed = 0;
    o->method = AMG_METHOD_SPARSE;
    o->precision = AMG_PREC_FP64;
    o->k_check = 3;
    o->s_levels = 1;
    o->gamma_min = 0.01;
    o->rho_max = 0.5;
    o->level_offset = 0;
    o->spmv_variant = AMG_SPMV_AUTO;
    o->use_graph = 1;
    o->check_every = 1;
    o->lump = AMG_LUMP_DIAG;
    o->krylov = AMG_KRYLOV_CG;
    o->restart = 30;
    o->div_factor = 1e3;
    o->transfer_variant = AMG_SPMV_AUTO;
}

amg_status amg_setup(const amg_csr *A, double theta, const double *gamma, int n_gamma, const amg_options *opt,
                     void *stream, amg_hierarchy **out) {
    return guarded([&] {
        require(out != nullptr, "out is NULL");
        *out = nullptr;
        amg_options o;
        if (opt) o = *opt; else amg_options_default(&o);
        o.theta = theta;
        check_options(o);
        check_csr_header(A, true);
        check_gammas(gamma, n_gamma);
        cudaStream_t s = as_stream(stream);
        AllocOn alloc_scope(s);
        auto H = std::make_unique<amg_hierarchy>();
        Hierarchy &h = H->h;
        h.opt = o;
        AMG_CUDA(cudaGetDevice(&h.device));
        h.timing = o.setup_timing != 0;
        h.lev.push_back(std::make_unique<Level>());
        upload_csr(A, h.lev[0]->A, s);
        setup_hierarchy(h, s, gamma, n_gamma);
        ensure_workspace(h, s);
        AMG_CUDA(cudaStreamSynchronize(s));
        if (h.opt.setup_timing) {  // setup phases were timed; the solve timing stays opt-in
            timing_collect(h);
            h.timing = false;
        }
        *out = H.release();
        return AMG_OK;
    });
}

amg_status amg_hierarchy_assemble(int levels, const amg_csr *A, const amg_csr *P, const int8_t *const *cf,
                                  const uint8_t *const *inM, const double *gamma, int n_gamma,
                                  const amg_options *opt, void *stream, amg_hierarchy **out) {
    return guarded([&] {
        require(out != nullptr, "out is NULL");
        *out = nullptr;
        require(levels >= 1 && levels <= kMaxLevels, "levels must be in [1, 64]");
        require(A != nullptr && (levels == 1 || (P && cf)) && (levels == 1 || inM), "NULL level arrays");
        amg_options o;
        if (opt) o = *opt; else amg_options_default(&o);
        check_options(o);
        require(o.method != AMG_METHOD_NONGALERKIN,
                "non-Galerkin coarse operators are formed during the setup; assemble takes Galerkin levels");
        check_gammas(gamma, n_gamma);
        cudaStream_t s = as_stream(stream);
        AllocOn alloc_scope(s);
        std::vector<DevCSR> dA(levels), dP(levels > 1 ? levels - 1 : 0);
        std::vector<std::vector<int8_t>> hcf(levels);
        std::vector<std::vector<uint8_t>> hinM(levels);
        for (int l = 0; l < levels; ++l) {
            check_csr_header(&A[l], true);
            upload_csr(&A[l], dA[l], s);
            if (l + 1 < levels) {
                check_csr_header(&P[l], false);
                upload_csr(&P[l], dP[l], s);
                require(cf[l] != nullptr, "cf_l is NULL");
                hcf[l].assign(cf[l], cf[l] + A[l].n);
            }
            if (l > 0) {
                require(inM[l] != nullptr, "inM_l is NULL");
                hinM[l].assign(inM[l], inM[l] + A[l].nnz);
            }
        }
        auto H = std::make_unique<amg_hierarchy>();
        Hierarchy &h = H->h;
        h.opt = o;
        AMG_CUDA(cudaGetDevice(&h.device));
        assemble_levels(h, dA, dP, hcf, hinM, s);
        finish_setup(h, gamma, n_gamma, s);
        *out = H.release();
        return AMG_OK;
    });
}

amg_status amg_sparsify(amg_hierarchy *H, const double *gamma, int n_gamma) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        check_gammas(gamma, n_gamma);
        Hierarchy &h = H->h;
        require(h.opt.method != AMG_METHOD_NONGALERKIN, "a non-Galerkin hierarchy retains no Galerkin operator");
        cudaStream_t s = nullptr;
        AllocOn alloc_scope(s);
        apply_gammas(h, gamma, n_gamma, s);
        std::vector<int> all;
        for (int l = 0; l < h.nlev(); ++l) all.push_back(l);
        prepare_cycle(h, s, all);
        return AMG_OK;
    });
}

amg_status amg_reintroduce(amg_hierarchy *H, int s_levels, int *changed) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        require(s_levels >= 1, "s_levels must be >= 1");
        require(H->h.opt.method != AMG_METHOD_NONGALERKIN, "a non-Galerkin hierarchy retains no Galerkin operator");
        AllocOn alloc_scope(nullptr);
        int c = reintroduce(H->h, s_levels, nullptr);
        if (changed) *changed = c;
        return AMG_OK;
    });
}

amg_status amg_solve(amg_hierarchy *H, const double *b, double *x, double tol, int max_it, int adaptive,
                     int on_device, void *stream, amg_solve_info *info) {
    amg_solve_info local;
    if (!info) info = &local;
    std::memset(info, 0, sizeof(*info));
    return guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        require(H != nullptr && b != nullptr && x != nullptr, "NULL argument");
        require(std::isfinite(tol) && tol > 0.0, "tol must be > 0");
        require(max_it >= 1, "max_it must be >= 1");
        Hierarchy &h = H->h;
        require(!adaptive || h.opt.method != AMG_METHOD_NONGALERKIN,
                "adaptive solves reintroduce from retained Galerkin operators; a non-Galerkin hierarchy has none");
        cudaStream_t s = as_stream(stream);
        AllocOn alloc_scope(s);
        ensure_workspace(h, s);
        int64_t n = h.lev[0]->n();
        const double *bd = b;
        double *xd = x;
        if (on_device) {
            require(is_device_ptr(b) && is_device_ptr(x), "on_device = 1 but b or x is not device memory");
        } else {  // b's values are checked through its norm on the device
            AMG_CUDA(cudaMemcpyAsync(h.pb.ptr, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
            bd = h.pb.as<double>();
            xd = h.px.as<double>();
        }
        amg_status st = solve(h, bd, xd, tol, max_it, adaptive != 0, s, info);
        if (!on_device) {
            AMG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        }
        AMG_CUDA(cudaStreamSynchronize(s));
        info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return st;
    });
}

amg_status amg_solve_batch(amg_hierarchy *H, int k, const double *B, double *X, double tol, int max_it,
                           int on_device, void *stream, amg_solve_info *info_k) {
    return guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        require(H != nullptr && B != nullptr && X != nullptr && info_k != nullptr, "NULL argument");
        require(k >= 1 && k <= 64, "k must be in [1, 64]");
        require(std::isfinite(tol) && tol > 0.0, "tol must be > 0");
        require(max_it >= 1, "max_it must be >= 1");
        Hierarchy &h = H->h;
        int64_t n = h.lev[0]->n();
        if (on_device) {
            require(is_device_ptr(B) && is_device_ptr(X), "on_device = 1 but B or X is not device memory");
        }  // B's values are checked through its column norms on the device
        AllocOn alloc_scope(as_stream(stream));
        amg_status st = solve_batch(h, k, B, X, on_device != 0, tol, max_it, as_stream(stream), info_k);
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        for (int c = 0; c < k; ++c) info_k[c].solve_ms = ms;
        return st;
    });
}

amg_status amg_precond_apply(amg_hierarchy *H, const double *r, double *z, void *stream) {
    return guarded([&] {
        require(H != nullptr && r != nullptr && z != nullptr, "NULL argument");
        require(is_device_ptr(r) && is_device_ptr(z), "r and z must be device memory");
        Hierarchy &h = H->h;
        cudaStream_t s = as_stream(stream);
        AllocOn alloc_scope(s);
        ensure_workspace(h, s);
        vcycle_f64(h, r, z, s);
        timing_collect(h);
        AMG_CUDA(cudaStreamSynchronize(s));
        return AMG_OK;
    });
}

int amg_num_levels(const amg_hierarchy *H) { return H ? H->h.nlev() : 0; }

amg_status amg_level_stats(const amg_hierarchy *H, int level, amg_level_info *out) {
    return guarded([&] {
        require(H != nullptr && out != nullptr, "NULL argument");
        const Hierarchy &h = H->h;
        require(level >= 0 && level < h.nlev(), "level out of range");
        const Level &V = *h.lev[level];
        std::memset(out, 0, sizeof(*out));
        out->n = V.n();
        out->nnz_galerkin = V.A.nnz;
        out->nnz_operator = V.op().nnz;
        out->nnz_p = level + 1 < h.nlev() ? V.P.nnz : 0;
        out->n_coarse = level + 1 < h.nlev() ? V.P.ncols : 0;
        out->gamma = V.gamma;
        out->spmv_variant = V.variant;
        out->value_bytes = V.vbytes;
        out->bytes_per_cycle = level_cycle_bytes(h, level);
        out->spmv_variant_p = level + 1 < h.nlev() ? V.variant_p : 0;
        out->spmv_variant_r = level + 1 < h.nlev() ? V.variant_r : 0;
        return AMG_OK;
    });
}

amg_status amg_level_export(const amg_hierarchy *H, int level, int which, int32_t *rowptr, int32_t *col,
                            double *val, int64_t *nrows, int64_t *ncols, int64_t *nnz) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        const Hierarchy &h = H->h;
        require(level >= 0 && level < h.nlev(), "level out of range");
        const Level &V = *h.lev[level];
        const DevCSR *M = nullptr;
        switch (which) {
            case 0: M = &V.A; break;
            case 1: M = &V.op(); break;
            case 2: M = &V.P; break;
            case 3: M = &V.R; break;
            default: require(false, "which must be 0..3");
        }
        require(which < 2 || level + 1 < h.nlev(), "the coarsest level has no P / R");
        if (nrows) *nrows = M->nrows;
        if (ncols) *ncols = M->ncols;
        if (nnz) *nnz = M->nnz;
        if (!rowptr) return AMG_OK;
        require(col && val, "col / val are NULL");
        AMG_CUDA(cudaMemcpy(rowptr, M->rp(), sizeof(int32_t) * (M->nrows + 1), cudaMemcpyDeviceToHost));
        if (M->nnz > 0) {
            AMG_CUDA(cudaMemcpy(col, M->ci(), sizeof(int32_t) * M->nnz, cudaMemcpyDeviceToHost));
            AMG_CUDA(cudaMemcpy(val, M->v(), sizeof(double) * M->nnz, cudaMemcpyDeviceToHost));
        }
        return AMG_OK;
    });
}

amg_status amg_level_array(const amg_hierarchy *H, int level, int which, void *out, int64_t *count) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        const Hierarchy &h = H->h;
        require(level >= 0 && level < h.nlev(), "level out of range");
        const Level &V = *h.lev[level];
        const DevBuf *b = nullptr;
        int64_t cnt = 0;
        size_t esz = 1;
        switch (which) {
            case 0: b = &V.cf; cnt = V.cf.ptr ? V.n() : 0; break;
            case 1: b = &V.keep; cnt = V.A.nnz; break;
            case 2: b = &V.inM; cnt = V.inM.ptr ? V.A.nnz : 0; break;
            case 3: b = &V.l1; cnt = V.n(); esz = 8; break;
            case 4: b = &V.strong; cnt = V.strong.ptr ? V.A.nnz : 0; break;
            default: require(false, "which must be 0..4");
        }
        if (count) *count = cnt;
        if (out && cnt > 0) AMG_CUDA(cudaMemcpy(out, b->ptr, esz * cnt, cudaMemcpyDeviceToHost));
        return AMG_OK;
    });
}

amg_status amg_timing_enable(amg_hierarchy *H, int on) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        H->h.timing = on != 0;
        return AMG_OK;
    });
}

amg_status amg_timing_reset(amg_hierarchy *H) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        timing_collect(H->h);
        for (auto &row : H->h.timers)
            for (auto &t : row) t = Timing();
        return AMG_OK;
    });
}

amg_status amg_timing_get(const amg_hierarchy *H, int kind, int level, int64_t *launches, double *total_ms,
                          double *bytes) {
    return guarded([&] {
        require(H != nullptr, "hierarchy is NULL");
        require(kind >= 0 && kind < kTimingKinds && level >= 0 && level < kMaxLevels, "kind / level out of range");
        const Timing &t = H->h.timers[kind][level];
        if (launches) *launches = t.launches;
        if (total_ms) *total_ms = t.ms;
        if (bytes) *bytes = t.bytes;
        return AMG_OK;
    });
}

// File layout (little-endian): "AMGH", u32 version = 1, u32 levels, then per
// level l: i64 n, i64 nnz, i32 rowptr[n+1], i32 col[nnz], f64 val[nnz]
// (Galerkin A_l), f64 gamma_l; for l > 0: u8 inM[nnz]; for l < L-1: i8 cf[n],
// i64 n_coarse, i64 nnz_p, i32 rowptr[n+1], i32 col[nnz_p], f64 val[nnz_p].
amg_status amg_hierarchy_save(const amg_hierarchy *H, const char *path) {
    return guarded([&] {
        require(H != nullptr && path != nullptr, "NULL argument");
        const Hierarchy &h = H->h;
        require(h.opt.method != AMG_METHOD_NONGALERKIN,
                "a non-Galerkin hierarchy retains no Galerkin operator to save (rebuild it from A_0)");
        std::ofstream f(path, std::ios::binary);
        require((bool)f, std::string("cannot open ") + path);
        auto put = [&](const void *p, size_t n) { f.write(reinterpret_cast<const char *>(p), (std::streamsize)n); };
        auto put_dev = [&](const void *d, size_t n) {
            std::vector<char> tmp(n);
            if (n) AMG_CUDA(cudaMemcpy(tmp.data(), d, n, cudaMemcpyDeviceToHost));
            put(tmp.data(), n);
        };
        uint32_t hdr[2] = {1u, (uint32_t)h.nlev()};
        put("AMGH", 4);
        put(hdr, sizeof(hdr));
        for (int l = 0; l < h.nlev(); ++l) {
            const Level &V = *h.lev[l];
            int64_t n = V.A.nrows, nnz = V.A.nnz;
            put(&n, 8);
            put(&nnz, 8);
            put_dev(V.A.rp(), sizeof(int32_t) * (n + 1));
            put_dev(V.A.ci(), sizeof(int32_t) * nnz);
            put_dev(V.A.v(), sizeof(double) * nnz);
            put(&V.gamma, 8);
            if (l > 0) put_dev(V.inM.ptr, nnz);
            if (l + 1 < h.nlev()) {
                require(V.cf.ptr != nullptr, "hierarchy lacks C/F markers");
                put_dev(V.cf.ptr, n);
                int64_t nc = V.P.ncols, np = V.P.nnz;
                put(&nc, 8);
                put(&np, 8);
                put_dev(V.P.rp(), sizeof(int32_t) * (n + 1));
                put_dev(V.P.ci(), sizeof(int32_t) * np);
                put_dev(V.P.v(), sizeof(double) * np);
            }
        }
        require((bool)f, "write failed");
        return AMG_OK;
    });
}

amg_status amg_hierarchy_load(const char *path, const amg_options *opt, void *stream, amg_hierarchy **out) {
    return guarded([&] {
        require(path != nullptr && out != nullptr, "NULL argument");
        *out = nullptr;
        std::ifstream f(path, std::ios::binary);
        require((bool)f, std::string("cannot open ") + path);
        auto get = [&](void *p, size_t n) {
            f.read(reinterpret_cast<char *>(p), (std::streamsize)n);
            require((bool)f, "truncated hierarchy file");
        };
        char magic[4];
        uint32_t hdr[2];
        get(magic, 4);
        get(hdr, sizeof(hdr));
        require(std::memcmp(magic, "AMGH", 4) == 0 && hdr[0] == 1u, "not a version-1 hierarchy file");
        int L = (int)hdr[1];
        require(L >= 1 && L <= kMaxLevels, "bad level count");
        std::vector<std::vector<int32_t>> arp(L), aci(L), prp(L), pci(L);
        std::vector<std::vector<double>> av(L), pv(L);
        std::vector<std::vector<int8_t>> cf(L);
        std::vector<std::vector<uint8_t>> inM(L);
        std::vector<double> gamma(L, 0.0);
        std::vector<amg_csr> A(L), P(L > 1 ? L - 1 : 0);
        for (int l = 0; l < L; ++l) {
            int64_t n, nnz;
            get(&n, 8);
            get(&nnz, 8);
            require(n > 0 && n < ((int64_t)1 << 31) && nnz >= 0 && nnz < ((int64_t)1 << 31), "bad level size");
            arp[l].resize(n + 1); aci[l].resize(nnz); av[l].resize(nnz);
            get(arp[l].data(), sizeof(int32_t) * (n + 1));
            get(aci[l].data(), sizeof(int32_t) * nnz);
            get(av[l].data(), sizeof(double) * nnz);
            get(&gamma[l], 8);
            A[l] = amg_csr{n, nnz, arp[l].data(), aci[l].data(), av[l].data(), 0, 0};
            if (l > 0) { inM[l].resize(nnz); get(inM[l].data(), nnz); }
            if (l + 1 < L) {
                cf[l].resize(n);
                get(cf[l].data(), n);
                int64_t nc, np;
                get(&nc, 8);
                get(&np, 8);
                require(nc > 0 && nc < ((int64_t)1 << 31) && np >= 0 && np < ((int64_t)1 << 31), "bad P size");
                prp[l].resize(n + 1); pci[l].resize(np); pv[l].resize(np);
                get(prp[l].data(), sizeof(int32_t) * (n + 1));
                get(pci[l].data(), sizeof(int32_t) * np);
                get(pv[l].data(), sizeof(double) * np);
                P[l] = amg_csr{n, np, prp[l].data(), pci[l].data(), pv[l].data(), 0, nc};
            }
        }
        std::vector<const int8_t *> cfp(L);
        std::vector<const uint8_t *> inMp(L);
        for (int l = 0; l < L; ++l) {
            cfp[l] = cf[l].empty() ? nullptr : cf[l].data();
            inMp[l] = inM[l].empty() ? nullptr : inM[l].data();
        }
        gamma[0] = 0.0;
        return amg_hierarchy_assemble(L, A.data(), P.empty() ? nullptr : P.data(), cfp.data(), inMp.data(),
                                      gamma.data(), L, opt, stream, out);
    });
}

void amg_free(amg_hierarchy *H) {
    try {
        delete H;
    } catch (...) {
    }
}

const char *amg_status_str(amg_status s) {
    switch (s) {
        case AMG_OK: return "AMG_OK";
        case AMG_ERR_INVALID: return "AMG_ERR_INVALID";
        case AMG_ERR_OOM: return "AMG_ERR_OOM";
        case AMG_ERR_CUDA: return "AMG_ERR_CUDA";
        case AMG_NOT_CONVERGED: return "AMG_NOT_CONVERGED";
        case AMG_DIVERGED: return "AMG_DIVERGED";
        case AMG_BREAKDOWN: return "AMG_BREAKDOWN";
        case AMG_TIMEOUT: return "AMG_TIMEOUT";
        case AMG_REJECTED: return "AMG_REJECTED";
        default: return "AMG_UNKNOWN_STATUS";
    }
}

const char *amg_last_error(void) { return amg::last_error_cstr(); }

int64_t amg_kernel_launches(void) { return amg::g_launches.load(); }

void amg_debug_fail_allocation(int64_t after) { amg::arm_allocation_failure(after); }

int64_t amg_device_bytes(const amg_hierarchy *H) {
    (void)H;
    return amg::g_device_bytes.load();
}

}  // extern "C"
