// batch_driver.cu -- K-column PCG with one SpMM V-cycle per iteration.
//
// Each column keeps its own CG scalars (rho, alpha, beta, ...), stops on its
// own, and is frozen (active = 0) once converged; a frozen or empty column
// holds zeros and costs bandwidth but changes nothing.  The iteration body is
// uniform over columns -- a column that (re)starts only has beta forced to 0
// -- which is what lets the server admit a request into a free column
// between two iterations of a running batch.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "batch_ops.cuh"
#include "hierarchy.cuh"

namespace amg {

BatchWS::~BatchWS() {
    if (graph) cudaGraphExecDestroy(graph);
    if (h_d) cudaFreeHost(h_d);
    if (h_i) cudaFreeHost(h_i);
}

BatchWS &batch_workspace(Hierarchy &h, int K, cudaStream_t s) {
    auto it = h.batch.find(K);
    if (it != h.batch.end()) return *it->second;
    auto w = std::make_unique<BatchWS>();
    w->K = K;
    int L = h.nlev();
    size_t xb = h.opt.precision == AMG_PREC_FP64 ? 8 : 4;
    w->b.resize(L); w->x.resize(L); w->r.resize(L); w->xo.resize(L);
    for (int l = 0; l < L; ++l) {
        size_t bytes = xb * ((size_t)h.lev[l]->n() * K + kPad);
        for (DevBuf *d : {&w->b[l], &w->x[l], &w->r[l], &w->xo[l]}) {
            d->alloc(bytes);
            AMG_CUDA(cudaMemsetAsync(d->ptr, 0, bytes, s));
        }
    }
    size_t nb = sizeof(double) * ((size_t)h.lev[0]->n() * K + kPad);
    for (DevBuf *d : {&w->B, &w->X, &w->R, &w->Z, &w->P, &w->Q, &w->T}) {
        d->alloc(nb);
        AMG_CUDA(cudaMemsetAsync(d->ptr, 0, nb, s));
    }
    if (h.opt.precision != AMG_PREC_FP64) {
        size_t fb = sizeof(float) * ((size_t)h.lev[0]->n() * K + kPad);
        w->R32.alloc(fb);
        AMG_CUDA(cudaMemsetAsync(w->R32.ptr, 0, fb, s));  // kept equal to (float) R by every writer of R
        if (L == 1) w->Z32.alloc(fb);  // deeper cycles write Z themselves
    }
    w->sc_buf.alloc(sizeof(double) * 7 * K + sizeof(int) * 3 * K);
    AMG_CUDA(cudaMemsetAsync(w->sc_buf.ptr, 0, w->sc_buf.bytes, s));
    double *d = w->sc_buf.as<double>();
    int *iv = reinterpret_cast<int *>(d + 7 * K);
    w->sc = bat::ColScalars{d, d + K, d + 2 * K, d + 3 * K, d + 4 * K, d + 5 * K, d + 6 * K, iv, iv + K};
    w->mask.alloc(sizeof(int) * K);
    w->partials.alloc(sizeof(double) * 3 * bat::kMaxCols * bat::kBatchReduceBlocks);
    AMG_CUDA(cudaMallocHost(&w->h_d, sizeof(double) * 7 * K));
    AMG_CUDA(cudaMallocHost(&w->h_i, sizeof(int) * 3 * K));
    std::memset(w->h_d, 0, sizeof(double) * 7 * K);
    std::memset(w->h_i, 0, sizeof(int) * 3 * K);
    BatchWS &ref = *w;
    h.batch[K] = std::move(w);
    return ref;
}

// active / start flags host -> device
void batch_push_flags(BatchWS &w, cudaStream_t s) {
    AMG_CUDA(cudaMemcpyAsync(w.sc.active, w.h_i, sizeof(int) * 2 * w.K, cudaMemcpyHostToDevice, s));
}

// level l's smoothers; the finest post-smoothing writes Z0 of type OT0
// (double on the FP32 cycle: no separate conversion pass back)
template <typename XT>
static void pre_level(Level &V, int K, const XT *b, XT *x, XT *r, cudaStream_t s) {
    if constexpr (sizeof(XT) == 8) {
        bat::pre_smooth_residual<double, double>(op_mat<double>(V), K, b, dinv_of<XT>(V), x, r, s);
    } else if (V.vbytes == 2) {
        bat::pre_smooth_residual<__nv_bfloat16, float>(op_mat<__nv_bfloat16>(V), K, b, dinv_of<XT>(V), x, r, s);
    } else {
        bat::pre_smooth_residual<float, float>(op_mat<float>(V), K, b, dinv_of<XT>(V), x, r, s);
    }
}
template <typename XT, typename OT>
static void post_level(Level &V, int K, const XT *x, const XT *b, OT *out, cudaStream_t s) {
    if constexpr (sizeof(XT) == 8) {
        bat::post_smooth<double, double, OT>(op_mat<double>(V), K, x, b, dinv_of<XT>(V), out, s);
    } else if (V.vbytes == 2) {
        bat::post_smooth<__nv_bfloat16, float, OT>(op_mat<__nv_bfloat16>(V), K, x, b, dinv_of<XT>(V), out, s);
    } else {
        bat::post_smooth<float, float, OT>(op_mat<float>(V), K, x, b, dinv_of<XT>(V), out, s);
    }
}

// Z0 = M B0 over the hierarchy's levels (at least two)
template <typename XT, typename OT0>
static void batch_vcycle_impl(Hierarchy &h, BatchWS &w, const XT *B0, OT0 *Z0, cudaStream_t s) {
    int L = h.nlev(), K = w.K;
    for (int l = 0; l + 1 < L; ++l) {
        Level &V = *h.lev[l];
        XT *x = w.x[l].as<XT>(), *r = w.r[l].as<XT>();
        pre_level<XT>(V, K, l == 0 ? B0 : w.b[l].as<XT>(), x, r, s);
        bat::spmm<XT, XT>(r_mat<XT>(V), K, r, w.b[l + 1].as<XT>(), false, s);
    }
    bat::coarse_solve<XT>(h.coarse_n, K, h.coarse_inv.as<double>(), w.b[L - 1].as<XT>(), w.xo[L - 1].as<XT>(), s);
    for (int l = L - 2; l >= 0; --l) {
        Level &V = *h.lev[l];
        XT *x = w.x[l].as<XT>();
        bat::spmm<XT, XT>(p_mat<XT>(V), K, w.xo[l + 1].as<XT>(), x, true, s);
        if (l == 0) post_level<XT, OT0>(V, K, x, B0, Z0, s);
        else post_level<XT, XT>(V, K, x, w.b[l].as<XT>(), w.xo[l].as<XT>(), s);
    }
}

// Z = M R for all K columns
void batch_vcycle(Hierarchy &h, BatchWS &w, cudaStream_t s) {
    int64_t nk = (int64_t)h.lev[0]->n() * w.K;
    const bool fp64 = h.opt.precision == AMG_PREC_FP64;
    if (fp64) {
        if (h.nlev() == 1)
            bat::coarse_solve<double>(h.coarse_n, w.K, h.coarse_inv.as<double>(), w.R.as<double>(), w.Z.as<double>(), s);
        else
            batch_vcycle_impl<double, double>(h, w, w.R.as<double>(), w.Z.as<double>(), s);
        return;
    }
    // R32 = (float) R already: written with R by the x, r update, admission
    // and residual replacement
    if (h.nlev() == 1) {  // the coarse solve alone, in FP32 vectors
        bat::coarse_solve<float>(h.coarse_n, w.K, h.coarse_inv.as<double>(), w.R32.as<float>(), w.Z32.as<float>(), s);
        bat::from_cycle<float>(w.Z32.as<float>(), w.Z.as<double>(), nk, s);
    } else {
        batch_vcycle_impl<float, double>(h, w, w.R32.as<float>(), w.Z.as<double>(), s);
    }
}

static CycMat<double> a0(Hierarchy &h) {
    Level &V = *h.lev[0];
    return make_mat<double>(V.A, V.A.v());
}

// One CG step for every active column: Z = M R; rho, beta; P = Z + beta P;
// Q = A P, alpha; X += alpha P, R -= alpha Q, rr.  Scalars are copied to the
// pinned host mirror; the caller synchronises the stream before reading.
static void batch_iteration_body(Hierarchy &h, BatchWS &w, cudaStream_t s) {
    int32_t n = h.lev[0]->n();
    int K = w.K;
    int flexible = h.opt.precision != AMG_PREC_FP64;
    batch_vcycle(h, w, s);
    bat::rz(n, K, w.R.as<double>(), w.Z.as<double>(), w.Q.as<double>(), w.sc, flexible, w.partials.as<double>(), s);
    bat::p_update(n, K, w.Z.as<double>(), w.P.as<double>(), w.sc, s);
    bat::ap(a0(h), K, w.P.as<double>(), w.Q.as<double>(), w.sc, w.partials.as<double>(), s);
    bat::xr_update(n, K, w.P.as<double>(), w.Q.as<double>(), w.X.as<double>(), w.R.as<double>(), w.R32.as<float>(), w.sc,
                   w.partials.as<double>(), s);
    AMG_CUDA(cudaMemcpyAsync(w.h_d, w.sc_buf.ptr, sizeof(double) * 6 * K, cudaMemcpyDeviceToHost, s));
}

// The iteration is captured once per (workspace, hierarchy version) and then
// launched as one graph: ~4 L + 8 kernels and a copy per launch.
void batch_iteration(Hierarchy &h, BatchWS &w, cudaStream_t s) {
    if (!h.opt.use_graph) {
        batch_iteration_body(h, w, s);
        return;
    }
    if (!w.graph || w.graph_version != h.version) {
        if (w.graph) cudaGraphExecDestroy(w.graph);
        w.graph = nullptr;
        cudaStream_t cs;
        AMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        AMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            batch_iteration_body(h, w, cs);
        } catch (...) {
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            throw;
        }
        AMG_CUDA(cudaStreamEndCapture(cs, &g));
        cudaError_t e = cudaGraphInstantiate(&w.graph, g, 0);
        cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        AMG_CUDA(e);
        w.graph_version = h.version;
    }
    AMG_CUDA(cudaGraphLaunch(w.graph, s));
}

// T = B - A X and tt per column
void batch_true_residual(Hierarchy &h, BatchWS &w, cudaStream_t s) {
    bat::residual(a0(h), w.K, w.B.as<double>(), w.X.as<double>(), w.T.as<double>(), w.sc, w.partials.as<double>(), s);
    AMG_CUDA(cudaMemcpyAsync(w.h_tt(), w.sc.tt, sizeof(double) * w.K, cudaMemcpyDeviceToHost, s));
}

namespace {
__global__ void repack_kernel(int64_t n, int k, int K, const double *src, double *dst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    int64_t i = e / K;
    int c = (int)(e % K);
    dst[e] = c < k ? src[i * k + c] : 0.0;
}
__global__ void unpack_kernel(int64_t n, int k, int K, const double *src, double *dst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    int64_t i = e / k;
    int c = (int)(e % k);
    dst[e] = src[i * K + c];
}
}  // namespace

amg_status solve_batch(Hierarchy &h, int k, const double *B, double *X, bool on_device, double tol, int max_it,
                       cudaStream_t s, amg_solve_info *infos) {
    ensure_workspace(h, s);
    int K = bat::batch_width(k);
    BatchWS &w = batch_workspace(h, K, s);
    int32_t n = h.lev[0]->n();
    // stage B (n x k, caller layout) into the n x K block
    TmpBuf staged;
    const double *Bk = B;
    if (!on_device) {
        staged.alloc(sizeof(double) * (size_t)n * k, s);
        AMG_CUDA(cudaMemcpyAsync(staged.ptr, B, sizeof(double) * (size_t)n * k, cudaMemcpyHostToDevice, s));
        Bk = staged.as<double>();
    }
    { repack_kernel<<<div_up((int64_t)n * K, 256), 256, 0, s>>>(n, k, K, Bk, w.B.as<double>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    size_t nb = sizeof(double) * (size_t)n * K;
    AMG_CUDA(cudaMemsetAsync(w.X.ptr, 0, nb, s));
    AMG_CUDA(cudaMemsetAsync(w.P.ptr, 0, nb, s));
    AMG_CUDA(cudaMemsetAsync(w.Q.ptr, 0, nb, s));
    AMG_CUDA(cudaMemcpyAsync(w.R.ptr, w.B.ptr, nb, cudaMemcpyDeviceToDevice, s));
    if (w.R32.ptr) bat::to_cycle<float>(w.R.as<double>(), w.R32.as<float>(), (int64_t)n * K, s);
    // ||b_c|| through the true residual at X = 0
    batch_true_residual(h, w, s);
    AMG_CUDA(cudaStreamSynchronize(s));
    std::vector<double> bnorm(K), rnorm(K);
    std::vector<int> its(K, 0), reps(K, 0), status(K, AMG_NOT_CONVERGED);
    for (int c = 0; c < K; ++c) {
        bnorm[c] = std::sqrt(w.h_tt()[c]);
        if (c < k && !std::isfinite(bnorm[c])) throw Error(AMG_ERR_INVALID, "B has a non-finite value");
        rnorm[c] = bnorm[c];
        bool live = c < k && bnorm[c] > 0.0;
        w.h_active()[c] = live ? 1 : 0;
        w.h_start()[c] = 1;
        if (c < k && !live) status[c] = AMG_OK;
    }
    batch_push_flags(w, s);
    int live = 0;
    for (int c = 0; c < K; ++c) live += w.h_active()[c];
    for (int it = 0; it < max_it && live > 0; ++it) {
        batch_iteration(h, w, s);
        AMG_CUDA(cudaStreamSynchronize(s));
        bool any_candidate = false, changed = false;
        for (int c = 0; c < K; ++c) {
            if (!w.h_active()[c]) continue;
            its[c]++;
            double pq = w.h_pq()[c], rho = w.h_rho()[c], rr = w.h_rr()[c];
            if (!(pq > 0.0) || !(rho > 0.0) || !std::isfinite(rr)) {
                status[c] = AMG_BREAKDOWN;
                w.h_active()[c] = 0;
                changed = true;
                continue;
            }
            rnorm[c] = std::sqrt(rr);
            w.h_mask()[c] = rnorm[c] <= tol * bnorm[c];
            any_candidate |= w.h_mask()[c] != 0;
        }
        if (any_candidate) {
            batch_true_residual(h, w, s);
            AMG_CUDA(cudaStreamSynchronize(s));
            bool replace = false;
            for (int c = 0; c < K; ++c) {
                if (!w.h_active()[c] || !w.h_mask()[c]) continue;
                double tn = std::sqrt(w.h_tt()[c]);
                rnorm[c] = tn;
                if (tn <= tol * bnorm[c]) {
                    status[c] = AMG_OK;
                    w.h_active()[c] = 0;
                    w.h_mask()[c] = 0;
                    changed = true;
                } else {
                    reps[c]++;
                    replace = true;
                }
            }
            if (replace) {
                AMG_CUDA(cudaMemcpyAsync(w.mask.ptr, w.h_mask(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
                bat::copy_masked_columns(n, K, w.T.as<double>(), w.R.as<double>(), w.mask.as<int>(), s,
                                         w.R32.as<float>());
            }
            for (int c = 0; c < K; ++c) w.h_mask()[c] = 0;
        }
        if (changed) {
            // start flags are cleared on the device by rz; keep the host copy in step
            for (int c = 0; c < K; ++c) w.h_start()[c] = 0;
            batch_push_flags(w, s);
        }
        live = 0;
        for (int c = 0; c < K; ++c) live += w.h_active()[c];
    }
    // final true residuals and results
    batch_true_residual(h, w, s);
    if (on_device) {
        { unpack_kernel<<<div_up((int64_t)n * k, 256), 256, 0, s>>>(n, k, K, w.X.as<double>(), X); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
    } else {
        { unpack_kernel<<<div_up((int64_t)n * k, 256), 256, 0, s>>>(n, k, K, w.X.as<double>(), staged.as<double>()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        AMG_CUDA(cudaMemcpyAsync(X, staged.ptr, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToHost, s));
    }
    AMG_CUDA(cudaStreamSynchronize(s));
    amg_status worst = AMG_OK;
    for (int c = 0; c < k; ++c) {
        amg_solve_info &inf = infos[c];
        std::memset(&inf, 0, sizeof(inf));
        inf.iterations = its[c];
        inf.replacements = reps[c];
        inf.final_relres = bnorm[c] > 0 ? std::sqrt(w.h_tt()[c]) / bnorm[c] : 0.0;
        inf.conv_factor = its[c] > 0 && bnorm[c] > 0 ? std::pow(rnorm[c] / bnorm[c], 1.0 / its[c]) : 0.0;
        inf.status = status[c];
        if (status[c] != AMG_OK && worst == AMG_OK) worst = (amg_status)status[c];
    }
    for (int c = 0; c < K; ++c) w.h_active()[c] = 0;
    batch_push_flags(w, s);
    AMG_CUDA(cudaStreamSynchronize(s));
    return worst;
}

}  // namespace amg
