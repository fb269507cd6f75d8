// batch.cu -- multi-right-hand-side (SpMM) V-cycle kernels and batched PCG.
//
// SpMM layout: a group of G lanes owns a row; the lanes load G consecutive
// (column index, value) pairs of the row with one coalesced access, then
// broadcast them with shuffles; lane t applies each entry to its CPL columns
// t, t+G, ... of the K-wide row block.  The matrix is read once per block of
// K right-hand sides instead of K times.
#include <cuda_bf16.h>

#include "batch_ops.cuh"
#include "common.cuh"

namespace amg {
namespace bat {

namespace {

constexpr int kThreads = 256;

template <typename VT, typename XT> __device__ __forceinline__ XT cvt(VT v) { return (XT)v; }

// lanes of this thread's G-lane group (groups never straddle a warp); the
// groups of one warp own different rows and run different trip counts, so
// their shuffles name only their own lanes
template <int G> __device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}
template <> __device__ __forceinline__ float cvt<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }

enum Op { kPre = 0, kPost = 1, kSpmv = 2, kSpmvAdd = 3 };

template <typename VT, typename XT, int G, int CPL, int OP>
__global__ void __launch_bounds__(kThreads)
spmm_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const VT *__restrict__ v,
            const XT *__restrict__ B, const XT *__restrict__ dinv, const XT *__restrict__ X,
            XT *__restrict__ O1, XT *__restrict__ O2) {
    constexpr int K = G * CPL;
    int64_t g = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / G;
    int t = threadIdx.x % G;
    int32_t i = (int32_t)g;
    int32_t p0 = 0, p1 = 0;
    if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
    XT acc[CPL];
#pragma unroll
    for (int u = 0; u < CPL; ++u) acc[u] = XT(0);
    const unsigned gm = group_mask<G>();
    for (int32_t e0 = p0; e0 < p1; e0 += G) {
        int32_t my_j = 0;
        XT my_a = XT(0);
        if (e0 + t < p1) { my_j = __ldg(ci + e0 + t); my_a = cvt<VT, XT>(__ldg(v + e0 + t)); }
        int cnt = min(G, p1 - e0);
        for (int e = 0; e < cnt; ++e) {
            int32_t j = __shfl_sync(gm, my_j, e, G);
            XT a = __shfl_sync(gm, my_a, e, G);
            const XT *src = (OP == kPre ? B : X) + (int64_t)j * K + t;
            if (OP == kPre) {
                XT dj = __ldg(dinv + j);
#pragma unroll
                for (int u = 0; u < CPL; ++u) acc[u] += a * (__ldg(src + u * G) * dj);
            } else {
#pragma unroll
                for (int u = 0; u < CPL; ++u) acc[u] += a * __ldg(src + u * G);
            }
        }
    }
    if (i >= n) return;
    int64_t base = (int64_t)i * K + t;
    if (OP == kPre) {
        XT di = dinv[i];
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            XT bi = B[base + u * G];
            O1[base + u * G] = bi * di;
            O2[base + u * G] = bi - acc[u];
        }
    } else if (OP == kPost) {
        XT di = dinv[i];
#pragma unroll
        for (int u = 0; u < CPL; ++u) O1[base + u * G] = X[base + u * G] + di * (B[base + u * G] - acc[u]);
    } else if (OP == kSpmv) {
#pragma unroll
        for (int u = 0; u < CPL; ++u) O1[base + u * G] = acc[u];
    } else {
#pragma unroll
        for (int u = 0; u < CPL; ++u) O1[base + u * G] += acc[u];
    }
}

template <typename VT, typename XT, int OP>
void dispatch(const CycMat<VT> &A, int K, const XT *B, const XT *dinv, const XT *X, XT *O1, XT *O2, cudaStream_t s) {
    int32_t n = A.nrows;
    if (n == 0) return;
    auto blocks = [&](int G) { return div_up((int64_t)n * G, kThreads); };
    switch (K) {
        case 8: { spmm_kernel<VT, XT, 8, 1, OP><<<blocks(8), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        case 16: { spmm_kernel<VT, XT, 16, 1, OP><<<blocks(16), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        case 32: { spmm_kernel<VT, XT, 32, 1, OP><<<blocks(32), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        case 64: { spmm_kernel<VT, XT, 32, 2, OP><<<blocks(32), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        default: throw Error(AMG_ERR_INVALID, "batch width must be 8, 16, 32 or 64");
    }
    AMG_CHECK_LAUNCH();
}

template <typename XT>
__global__ void coarse_kernel(int32_t n, int K, const double *__restrict__ inv, const XT *__restrict__ B, XT *__restrict__ X) {
    int32_t row = blockIdx.x;
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        double s = 0.0;
        for (int32_t j = 0; j < n; ++j) s += inv[(size_t)row * n + j] * (double)B[(int64_t)j * K + c];
        X[(int64_t)row * K + c] = (XT)s;
    }
}

// ---------------------------------------------------------------------------
// per-column deterministic reductions.  A thread's slot is its column; each
// block sums its slots in thread order and stores one partial per column; a
// finisher kernel (one block per column) sums the partials in block order
// and updates that column's scalars.  No atomics, no fences.
template <int NV>
__device__ void col_partials(double (&v)[NV], int K, double *partials) {
    __shared__ double sh[NV][kThreads];
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int r = threadIdx.x; r < kThreads; r += K) s += sh[k][r];
            partials[((size_t)k * kMaxCols + threadIdx.x) * kBatchReduceBlocks + blockIdx.x] = s;
        }
    }
}

enum ColFin { kColRz = 0, kColAp = 1, kColXr = 2, kColTt = 3 };

template <int NV, int FIN>
__global__ void __launch_bounds__(kThreads)
col_finish_kernel(int nblocks, const double *partials, ColScalars sc, int flexible) {
    const int c = blockIdx.x;
    __shared__ double sh[NV][kThreads / 32];
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        t[k] = 0.0;
        const double *p = partials + ((size_t)k * kMaxCols + c) * kBatchReduceBlocks;
        for (int b = threadIdx.x; b < nblocks; b += kThreads) t[k] += p[b];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = t[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double out[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        out[k] = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) out[k] += sh[k][i];
    }
    if (FIN == kColRz) {
        if (sc.active[c]) {
            double rho_new = out[0];
            if (sc.start[c]) sc.beta[c] = 0.0;
            else sc.beta[c] = flexible ? (-sc.alpha[c] * out[NV - 1]) / sc.rho[c] : rho_new / sc.rho[c];
            sc.zq[c] = out[NV - 1];
            sc.rho[c] = rho_new;
            sc.start[c] = 0;
        }
    } else if (FIN == kColAp) {
        sc.pq[c] = out[0];
        sc.alpha[c] = (sc.active[c] && out[0] > 0.0) ? sc.rho[c] / out[0] : 0.0;
    } else if (FIN == kColXr) {
        sc.rr[c] = out[0];
    } else {
        sc.tt[c] = out[0];
    }
}

// at least four rows per thread and at most one resident wave of blocks
int grid_for(int64_t n, int K) {
    int64_t rows_per_block = kThreads / K;
    int64_t b = (n + rows_per_block - 1) / rows_per_block;
    b = (b + 3) / 4;
    int64_t cap = std::min<int64_t>(kBatchReduceBlocks, ::amg::resident_blocks(kThreads));
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// thread -> (row, column) with column = threadIdx % K (K divides 256)
__global__ void __launch_bounds__(kThreads)
rz_kernel(int32_t n, int K, const double *__restrict__ R, const double *__restrict__ Z, const double *__restrict__ Q,
          double *partials) {
    int c = threadIdx.x % K;
    int rpb = kThreads / K;
    double v[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * rpb + threadIdx.x / K; i < n; i += (int64_t)gridDim.x * rpb) {
        double z = Z[i * K + c];
        v[0] += R[i * K + c] * z;
        v[1] += z * Q[i * K + c];
    }
    col_partials<2>(v, K, partials);
}

__global__ void p_update_kernel(int64_t total, int K, const double *__restrict__ Z, double *__restrict__ P, ColScalars sc) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int c = (int)(e % K);
    if (!sc.active[c]) return;
    P[e] = Z[e] + sc.beta[c] * P[e];
}

template <int G, int CPL, bool RESID>
__global__ void __launch_bounds__(kThreads)
ap_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
          const double *__restrict__ Pin, const double *__restrict__ Bin, double *__restrict__ Qout,
          double *partials) {
    constexpr int K = G * CPL;
    int t = threadIdx.x % G;
    double part[CPL];
#pragma unroll
    for (int u = 0; u < CPL; ++u) part[u] = 0.0;
    int rpb = kThreads / G;
    for (int64_t i = (int64_t)blockIdx.x * rpb + threadIdx.x / G; i < ((n + rpb - 1) / rpb) * (int64_t)rpb;
         i += (int64_t)gridDim.x * rpb) {
        int32_t p0 = 0, p1 = 0;
        if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
        double acc[CPL];
#pragma unroll
        for (int u = 0; u < CPL; ++u) acc[u] = 0.0;
        const unsigned gm = group_mask<G>();
        for (int32_t e0 = p0; e0 < p1; e0 += G) {
            int32_t my_j = 0;
            double my_a = 0.0;
            if (e0 + t < p1) { my_j = __ldg(ci + e0 + t); my_a = __ldg(v + e0 + t); }
            int cnt = min(G, p1 - e0);
            for (int e = 0; e < cnt; ++e) {
                int32_t j = __shfl_sync(gm, my_j, e, G);
                double a = __shfl_sync(gm, my_a, e, G);
#pragma unroll
                for (int u = 0; u < CPL; ++u) acc[u] += a * __ldg(Pin + (int64_t)j * K + t + u * G);
            }
        }
        if (i < n) {
#pragma unroll
            for (int u = 0; u < CPL; ++u) {
                int64_t e = i * K + t + u * G;
                if (RESID) {
                    double r = Bin[e] - acc[u];
                    Qout[e] = r;
                    part[u] += r * r;
                } else {
                    Qout[e] = acc[u];
                    part[u] += Pin[e] * acc[u];
                }
            }
        }
    }
    // per-column partial: slot of thread t, value u -> column t + u*G
    __shared__ double sh[CPL][kThreads];
#pragma unroll
    for (int u = 0; u < CPL; ++u) sh[u][threadIdx.x] = part[u];
    __syncthreads();
    if (threadIdx.x < K) {
        int col = threadIdx.x, u = col / G, tt = col % G;
        double s = 0.0;
        for (int r = tt; r < kThreads; r += G) s += sh[u][r];
        partials[(size_t)col * kBatchReduceBlocks + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads)
xr_kernel(int32_t n, int K, const double *__restrict__ P, const double *__restrict__ Q, double *__restrict__ X,
          double *__restrict__ R, ColScalars sc, double *partials) {
    int c = threadIdx.x % K;
    int rpb = kThreads / K;
    double alpha = sc.active[c] ? sc.alpha[c] : 0.0;
    double v[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * rpb + threadIdx.x / K; i < n; i += (int64_t)gridDim.x * rpb) {
        int64_t e = i * K + c;
        double r = R[e];
        if (alpha != 0.0) {
            X[e] += alpha * P[e];
            r -= alpha * Q[e];
            R[e] = r;
        }
        v[0] += r * r;
    }
    col_partials<1>(v, K, partials);
}

__global__ void scatter_kernel(int32_t n, int K, int c, const double *v, double *M) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) M[i * K + c] = v[i];
}
__global__ void gather_kernel(int32_t n, int K, int c, const double *M, double *v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = M[i * K + c];
}
__global__ void zero_col_kernel(int32_t n, int K, int c, double *M) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) M[i * K + c] = 0.0;
}
__global__ void copy_masked_kernel(int64_t total, int K, const double *T, double *R, const int *mask) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total && mask[e % K]) R[e] = T[e];
}

template <typename XT> __global__ void to_cycle_kernel(const double *src, XT *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (XT)src[i];
}
template <typename XT> __global__ void from_cycle_kernel(const XT *src, double *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

}  // namespace

int batch_width(int k) {
    if (k <= 8) return 8;
    if (k <= 16) return 16;
    if (k <= 32) return 32;
    if (k <= 64) return 64;
    throw Error(AMG_ERR_INVALID, "at most 64 right-hand sides per batch");
}

template <typename VT, typename XT>
void pre_smooth_residual(const CycMat<VT> &A, int K, const XT *B, const XT *dinv, XT *X, XT *R, cudaStream_t s) {
    dispatch<VT, XT, kPre>(A, K, B, dinv, nullptr, X, R, s);
}
template <typename VT, typename XT>
void post_smooth(const CycMat<VT> &A, int K, const XT *X, const XT *B, const XT *dinv, XT *XO, cudaStream_t s) {
    dispatch<VT, XT, kPost>(A, K, B, dinv, X, XO, nullptr, s);
}
template <typename VT, typename XT>
void spmm(const CycMat<VT> &A, int K, const XT *X, XT *Y, bool accumulate, cudaStream_t s) {
    if (accumulate) dispatch<VT, XT, kSpmvAdd>(A, K, nullptr, nullptr, X, Y, nullptr, s);
    else dispatch<VT, XT, kSpmv>(A, K, nullptr, nullptr, X, Y, nullptr, s);
}
template <typename XT>
void coarse_solve(int32_t n, int K, const double *inv, const XT *B, XT *X, cudaStream_t s) {
    if (n == 0) return;
    { coarse_kernel<XT><<<n, 64, 0, s>>>(n, K, inv, B, X); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void rz(int32_t n, int K, const double *R, const double *Z, const double *Q, ColScalars sc, int flexible,
        double *partials, unsigned *counter, cudaStream_t s) {
    int blocks = grid_for(n, K);
    { rz_kernel<<<blocks, kThreads, 0, s>>>(n, K, R, Z, Q, partials); ::amg::count_launch(); }
    { col_finish_kernel<2, kColRz><<<K, kThreads, 0, s>>>(blocks, partials, sc, flexible); ::amg::count_launch(); }
    (void)counter;
    AMG_CHECK_LAUNCH();
}

void p_update(int32_t n, int K, const double *Z, double *P, ColScalars sc, cudaStream_t s) {
    int64_t total = (int64_t)n * K;
    { p_update_kernel<<<div_up(total, kThreads), kThreads, 0, s>>>(total, K, Z, P, sc); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

template <bool RESID>
static void launch_ap(const CycMat<double> &A, int K, const double *P, const double *B, double *Q, ColScalars sc,
                      double *partials, unsigned *counter, cudaStream_t s) {
    int32_t n = A.nrows;
    auto grid = [&](int G) {
        int64_t rpb = kThreads / G;
        int64_t b = ((n + rpb - 1) / rpb + 3) / 4;
        int64_t cap = std::min<int64_t>(kBatchReduceBlocks, ::amg::resident_blocks(kThreads));
        return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
    };
    (void)counter;
    int blocks = 0;
    switch (K) {
        case 8: blocks = grid(8); { ap_kernel<8, 1, RESID><<<blocks, kThreads, 0, s>>>(n, A.rp, A.ci, A.v, P, B, Q, partials); ::amg::count_launch(); } break;
        case 16: blocks = grid(16); { ap_kernel<16, 1, RESID><<<blocks, kThreads, 0, s>>>(n, A.rp, A.ci, A.v, P, B, Q, partials); ::amg::count_launch(); } break;
        case 32: blocks = grid(32); { ap_kernel<32, 1, RESID><<<blocks, kThreads, 0, s>>>(n, A.rp, A.ci, A.v, P, B, Q, partials); ::amg::count_launch(); } break;
        case 64: blocks = grid(32); { ap_kernel<32, 2, RESID><<<blocks, kThreads, 0, s>>>(n, A.rp, A.ci, A.v, P, B, Q, partials); ::amg::count_launch(); } break;
        default: throw Error(AMG_ERR_INVALID, "batch width must be 8, 16, 32 or 64");
    }
    if (RESID) { col_finish_kernel<1, kColTt><<<K, kThreads, 0, s>>>(blocks, partials, sc, 0); ::amg::count_launch(); }
    else { col_finish_kernel<1, kColAp><<<K, kThreads, 0, s>>>(blocks, partials, sc, 0); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void ap(const CycMat<double> &A, int K, const double *P, double *Q, ColScalars sc, double *partials,
        unsigned *counter, cudaStream_t s) {
    launch_ap<false>(A, K, P, nullptr, Q, sc, partials, counter, s);
}

void residual(const CycMat<double> &A, int K, const double *B, const double *X, double *T, ColScalars sc,
              double *partials, unsigned *counter, cudaStream_t s) {
    launch_ap<true>(A, K, X, B, T, sc, partials, counter, s);
}

void xr_update(int32_t n, int K, const double *P, const double *Q, double *X, double *R, ColScalars sc,
               double *partials, unsigned *counter, cudaStream_t s) {
    int blocks = grid_for(n, K);
    { xr_kernel<<<blocks, kThreads, 0, s>>>(n, K, P, Q, X, R, sc, partials); ::amg::count_launch(); }
    { col_finish_kernel<1, kColXr><<<K, kThreads, 0, s>>>(blocks, partials, sc, 0); ::amg::count_launch(); }
    (void)counter;
    AMG_CHECK_LAUNCH();
}

void scatter_column(int32_t n, int K, int c, const double *v, double *M, cudaStream_t s) {
    { scatter_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, K, c, v, M); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}
void gather_column(int32_t n, int K, int c, const double *M, double *v, cudaStream_t s) {
    { gather_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, K, c, M, v); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}
void zero_column(int32_t n, int K, int c, double *M, cudaStream_t s) {
    { zero_col_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, K, c, M); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}
void copy_masked_columns(int32_t n, int K, const double *T, double *R, const int *mask, cudaStream_t s) {
    int64_t total = (int64_t)n * K;
    { copy_masked_kernel<<<div_up(total, kThreads), kThreads, 0, s>>>(total, K, T, R, mask); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

template <typename XT> void to_cycle(const double *src, XT *dst, int64_t n, cudaStream_t s) {
    { to_cycle_kernel<XT><<<div_up(n, kThreads), kThreads, 0, s>>>(src, dst, n); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}
template <typename XT> void from_cycle(const XT *src, double *dst, int64_t n, cudaStream_t s) {
    { from_cycle_kernel<XT><<<div_up(n, kThreads), kThreads, 0, s>>>(src, dst, n); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

#define AMG_BINST(VT, XT)                                                                                       \
    template void pre_smooth_residual<VT, XT>(const CycMat<VT> &, int, const XT *, const XT *, XT *, XT *, cudaStream_t); \
    template void post_smooth<VT, XT>(const CycMat<VT> &, int, const XT *, const XT *, const XT *, XT *, cudaStream_t); \
    template void spmm<VT, XT>(const CycMat<VT> &, int, const XT *, XT *, bool, cudaStream_t);
AMG_BINST(double, double)
AMG_BINST(float, float)
AMG_BINST(__nv_bfloat16, float)
#undef AMG_BINST
template void coarse_solve<double>(int32_t, int, const double *, const double *, double *, cudaStream_t);
template void coarse_solve<float>(int32_t, int, const double *, const float *, float *, cudaStream_t);
template void to_cycle<float>(const double *, float *, int64_t, cudaStream_t);
template void from_cycle<float>(const float *, double *, int64_t, cudaStream_t);

}  // namespace bat
}  // namespace amg
