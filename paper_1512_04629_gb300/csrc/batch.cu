// batch.cu -- multi-right-hand-side (SpMM) V-cycle kernels and batched PCG.
//
// SpMM layout: the K right-hand sides of a row are contiguous (row-major
// n x K).  A group of G = K / W lanes owns a row, and lane t owns the W
// consecutive columns W t .. W t + W - 1, moved as one 16-byte vector (W = 4
// floats or 2 doubles).  Every lane of the group reads the row's (column,
// value) pairs itself -- the same address across the group, served as one
// broadcast -- and keeps the vector loads of kAhead entries in flight before
// it uses them; each column still sums its entries in row order.  The matrix
// is read once per block of K right-hand sides instead of K times.
#include <cuda_bf16.h>

#include "batch_ops.cuh"
#include "common.cuh"

namespace amg {
namespace bat {

namespace {

constexpr int kThreads = 256;

template <typename VT, typename XT> __device__ __forceinline__ XT cvt(VT v) { return (XT)v; }

template <> __device__ __forceinline__ float cvt<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }

enum Op { kPre = 0, kPost = 1, kSpmv = 2, kSpmvAdd = 3 };

constexpr int kAhead = 4;  // entries whose vector loads are in flight together

// 16-byte vectors of a row block (the block's base is 16-byte aligned: K is a
// multiple of 8 and every n x K buffer starts on an allocation boundary)
__device__ __forceinline__ void vload(const float *p, float (&x)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
}
__device__ __forceinline__ void vload(const double *p, double (&x)[2]) {
    const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    x[0] = q.x; x[1] = q.y;
}
// for a buffer the same kernel writes (its own row only)
__device__ __forceinline__ void vload_rw(const float *p, float (&x)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
}
__device__ __forceinline__ void vload_rw(const double *p, double (&x)[2]) {
    const double2 q = *reinterpret_cast<const double2 *>(p);
    x[0] = q.x; x[1] = q.y;
}
__device__ __forceinline__ void vstore(float *p, const float (&x)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void vstore(double *p, const double (&x)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]);
}
// the FP32 cycle's finest post-smoothing writes the FP64 correction itself
// (4 floats widened exactly into 32 bytes of doubles) instead of a separate
// conversion pass.  Its input stays the FP32 copy of the residual: a gather
// that rounded FP64 neighbours on load would convert every value once per
// row that uses it, on GB300's narrow FP64 pipe.
__device__ __forceinline__ void vstore(double *p, const float (&x)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2((double)x[0], (double)x[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2((double)x[2], (double)x[3]);
}

// acc[w] += sum over the row's entries, in entry order, of a_ij * src_j[c0 + w]
// (times dinv_j when SCALE: the pre-smoothing's x_j = dinv_j b_j)
template <typename VT, typename XT, typename ST, int K, bool SCALE>
__device__ __forceinline__ void row_block_sum(int32_t p0, int32_t p1, const int32_t *__restrict__ ci,
                                              const VT *__restrict__ v, const ST *__restrict__ src,
                                              const XT *__restrict__ dinv, int c0, XT (&acc)[16 / sizeof(XT)]) {
    constexpr int W = 16 / sizeof(XT);
    int32_t e = p0;
    for (; e + kAhead <= p1; e += kAhead) {
        int32_t j[kAhead];
        XT a[kAhead], d[kAhead], x[kAhead][W];
#pragma unroll
        for (int q = 0; q < kAhead; ++q) {
            j[q] = __ldg(ci + e + q);
            a[q] = cvt<VT, XT>(__ldg(v + e + q));
        }
#pragma unroll
        for (int q = 0; q < kAhead; ++q) {
            vload(src + (int64_t)j[q] * K + c0, x[q]);
            if (SCALE) d[q] = __ldg(dinv + j[q]);
        }
#pragma unroll
        for (int q = 0; q < kAhead; ++q) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (SCALE) acc[w] += a[q] * (x[q][w] * d[q]);
                else acc[w] += a[q] * x[q][w];
            }
        }
    }
    for (; e < p1; ++e) {
        const int32_t j = __ldg(ci + e);
        const XT a = cvt<VT, XT>(__ldg(v + e));
        XT x[W];
        vload(src + (int64_t)j * K + c0, x);
        if (SCALE) {
            const XT d = __ldg(dinv + j);
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] += a * (x[w] * d);
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] += a * x[w];
        }
    }
}

// BT: type of B (the right-hand side); OT: type of O1 for the
// post-smoothing (double on the FP32 cycle's level 0, else XT)
template <typename VT, typename XT, typename BT, typename OT, int K, int OP>
__global__ void __launch_bounds__(kThreads)
spmm_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const VT *__restrict__ v,
            const BT *__restrict__ B, const XT *__restrict__ dinv, const XT *__restrict__ X,
            OT *__restrict__ O1, XT *__restrict__ O2) {
    constexpr int W = 16 / sizeof(XT), G = K / W;
    const int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int32_t i = (int32_t)(g / G);
    if (i >= n) return;
    const int c0 = (int)(g % G) * W;
    XT acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = XT(0);
    if constexpr (OP == kPre) row_block_sum<VT, XT, BT, K, true>(__ldg(rp + i), __ldg(rp + i + 1), ci, v, B, dinv, c0, acc);
    else row_block_sum<VT, XT, XT, K, false>(__ldg(rp + i), __ldg(rp + i + 1), ci, v, X, dinv, c0, acc);
    const int64_t base = (int64_t)i * K + c0;
    XT o[W];
    if constexpr (OP == kPre) {
        const XT di = dinv[i];
        XT bi[W], r[W];
        vload(B + base, bi);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            o[w] = bi[w] * di;
            r[w] = bi[w] - acc[w];
        }
        vstore(O1 + base, o);
        vstore(O2 + base, r);
    } else if constexpr (OP == kPost) {
        const XT di = dinv[i];
        XT xi[W], bi[W];
        vload(X + base, xi);
        vload(B + base, bi);
#pragma unroll
        for (int w = 0; w < W; ++w) o[w] = xi[w] + di * (bi[w] - acc[w]);
        vstore(O1 + base, o);
    } else if constexpr (OP == kSpmv) {
        vstore(O1 + base, acc);
    } else {
        vload_rw(O1 + base, o);
#pragma unroll
        for (int w = 0; w < W; ++w) o[w] += acc[w];
        vstore(O1 + base, o);
    }
}

template <typename VT, typename XT, int OP, typename BT = XT, typename OT = XT>
void dispatch(const CycMat<VT> &A, int K, const BT *B, const XT *dinv, const XT *X, OT *O1, XT *O2, cudaStream_t s) {
    int32_t n = A.nrows;
    if (n == 0) return;
    constexpr int W = 16 / sizeof(XT);
    auto blocks = [&](int k) { return div_up((int64_t)n * (k / W), kThreads); };
    switch (K) {
        case 8: { spmm_kernel<VT, XT, BT, OT, 8, OP><<<blocks(8), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        case 16: { spmm_kernel<VT, XT, BT, OT, 16, OP><<<blocks(16), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        case 32: { spmm_kernel<VT, XT, BT, OT, 32, OP><<<blocks(32), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
        case 64: { spmm_kernel<VT, XT, BT, OT, 64, OP><<<blocks(64), kThreads, 0, s>>>(n, A.rp, A.ci, A.v, B, dinv, X, O1, O2); ::amg::count_launch(); } break;
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

// Q = A P (or T = B - A X when RESID) on the FP64 n x K blocks, with the
// per-column partials of p . Ap (or ||t||^2); the row-block mapping of
// spmm_kernel with W = 2, rows taken grid-stride
template <int K, bool RESID>
__global__ void __launch_bounds__(kThreads)
ap_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
          const double *__restrict__ Pin, const double *__restrict__ Bin, double *__restrict__ Qout,
          double *partials) {
    constexpr int W = 2, G = K / W, RPB = kThreads / G;
    const int t = threadIdx.x % G, c0 = t * W;
    double part[W] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * RPB + threadIdx.x / G; i < n; i += (int64_t)gridDim.x * RPB) {
        double acc[W] = {0.0, 0.0};
        row_block_sum<double, double, double, K, false>(__ldg(rp + i), __ldg(rp + i + 1), ci, v, Pin, nullptr, c0, acc);
        const int64_t base = i * K + c0;
        if (RESID) {
            double b[W], r[W];
            vload(Bin + base, b);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                r[w] = b[w] - acc[w];
                part[w] += r[w] * r[w];
            }
            vstore(Qout + base, r);
        } else {
            double p[W];
            vload(Pin + base, p);
            vstore(Qout + base, acc);
#pragma unroll
            for (int w = 0; w < W; ++w) part[w] += p[w] * acc[w];
        }
    }
    // per-column partial: column W t + w sums slot w of the threads with lane t, in thread order
    __shared__ double sh[W][kThreads];
#pragma unroll
    for (int w = 0; w < W; ++w) sh[w][threadIdx.x] = part[w];
    __syncthreads();
    if (threadIdx.x < K) {
        const int col = threadIdx.x, tt = col / W, w = col % W;
        double sum = 0.0;
        for (int r = tt; r < kThreads; r += G) sum += sh[w][r];
        partials[(size_t)col * kBatchReduceBlocks + blockIdx.x] = sum;
    }
}

__global__ void __launch_bounds__(kThreads)
xr_kernel(int32_t n, int K, const double *__restrict__ P, const double *__restrict__ Q, double *__restrict__ X,
          double *__restrict__ R, float *__restrict__ R32, ColScalars sc, double *partials) {
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
        if (R32) R32[e] = (float)r;  // the next FP32 cycle's input, every column
        v[0] += r * r;
    }
    col_partials<1>(v, K, partials);
}

__global__ void scatter_kernel(int32_t n, int K, int c, const double *v, double *M, float *M32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    M[i * K + c] = v[i];
    if (M32) M32[i * K + c] = (float)v[i];
}
__global__ void gather_kernel(int32_t n, int K, int c, const double *M, double *v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = M[i * K + c];
}
__global__ void zero_col_kernel(int32_t n, int K, int c, double *M) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) M[i * K + c] = 0.0;
}
__global__ void copy_masked_kernel(int64_t total, int K, const double *T, double *R, float *R32, const int *mask) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total || !mask[e % K]) return;
    R[e] = T[e];
    if (R32) R32[e] = (float)T[e];
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
    dispatch<VT, XT, kPre, XT, XT>(A, K, B, dinv, nullptr, X, R, s);
}
template <typename VT, typename XT, typename OT>
void post_smooth(const CycMat<VT> &A, int K, const XT *X, const XT *B, const XT *dinv, OT *XO, cudaStream_t s) {
    dispatch<VT, XT, kPost, XT, OT>(A, K, B, dinv, X, XO, nullptr, s);
}
template <typename VT, typename XT>
void spmm(const CycMat<VT> &A, int K, const XT *X, XT *Y, bool accumulate, cudaStream_t s) {
    if (accumulate) dispatch<VT, XT, kSpmvAdd, XT, XT>(A, K, nullptr, nullptr, X, Y, nullptr, s);
    else dispatch<VT, XT, kSpmv, XT, XT>(A, K, nullptr, nullptr, X, Y, nullptr, s);
}
template <typename XT>
void coarse_solve(int32_t n, int K, const double *inv, const XT *B, XT *X, cudaStream_t s) {
    if (n == 0) return;
    { coarse_kernel<XT><<<n, 64, 0, s>>>(n, K, inv, B, X); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void rz(int32_t n, int K, const double *R, const double *Z, const double *Q, ColScalars sc, int flexible,
        double *partials, cudaStream_t s) {
    int blocks = grid_for(n, K);
    { rz_kernel<<<blocks, kThreads, 0, s>>>(n, K, R, Z, Q, partials); ::amg::count_launch(); }
    { col_finish_kernel<2, kColRz><<<K, kThreads, 0, s>>>(blocks, partials, sc, flexible); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void p_update(int32_t n, int K, const double *Z, double *P, ColScalars sc, cudaStream_t s) {
    int64_t total = (int64_t)n * K;
    { p_update_kernel<<<div_up(total, kThreads), kThreads, 0, s>>>(total, K, Z, P, sc); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

// one resident wave of ap_kernel blocks (at least four rows per thread group)
template <int K, bool RESID>
static int ap_grid(int32_t n) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ap_kernel<K, RESID>, kThreads, 0));
        per_sm = std::max(b, 1);
    }
    const int64_t rpb = kThreads / (K / 2);
    const int64_t want = ((n + rpb - 1) / rpb + 3) / 4;
    const int64_t cap = std::min<int64_t>(kBatchReduceBlocks, (int64_t)per_sm * ::amg::resident_blocks(2048));
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

template <int K, bool RESID>
static void launch_ap_k(const CycMat<double> &A, const double *P, const double *B, double *Q, ColScalars sc,
                        double *partials, cudaStream_t s) {
    const int blocks = ap_grid<K, RESID>(A.nrows);
    { ap_kernel<K, RESID><<<blocks, kThreads, 0, s>>>(A.nrows, A.rp, A.ci, A.v, P, B, Q, partials); ::amg::count_launch(); }
    if (RESID) { col_finish_kernel<1, kColTt><<<K, kThreads, 0, s>>>(blocks, partials, sc, 0); ::amg::count_launch(); }
    else { col_finish_kernel<1, kColAp><<<K, kThreads, 0, s>>>(blocks, partials, sc, 0); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

template <bool RESID>
static void launch_ap(const CycMat<double> &A, int K, const double *P, const double *B, double *Q, ColScalars sc,
                      double *partials, cudaStream_t s) {
    switch (K) {
        case 8: launch_ap_k<8, RESID>(A, P, B, Q, sc, partials, s); break;
        case 16: launch_ap_k<16, RESID>(A, P, B, Q, sc, partials, s); break;
        case 32: launch_ap_k<32, RESID>(A, P, B, Q, sc, partials, s); break;
        case 64: launch_ap_k<64, RESID>(A, P, B, Q, sc, partials, s); break;
        default: throw Error(AMG_ERR_INVALID, "batch width must be 8, 16, 32 or 64");
    }
}

void ap(const CycMat<double> &A, int K, const double *P, double *Q, ColScalars sc, double *partials,
        cudaStream_t s) {
    launch_ap<false>(A, K, P, nullptr, Q, sc, partials, s);
}

void residual(const CycMat<double> &A, int K, const double *B, const double *X, double *T, ColScalars sc,
              double *partials, cudaStream_t s) {
    launch_ap<true>(A, K, X, B, T, sc, partials, s);
}

void xr_update(int32_t n, int K, const double *P, const double *Q, double *X, double *R, float *R32, ColScalars sc,
               double *partials, cudaStream_t s) {
    int blocks = grid_for(n, K);
    { xr_kernel<<<blocks, kThreads, 0, s>>>(n, K, P, Q, X, R, R32, sc, partials); ::amg::count_launch(); }
    { col_finish_kernel<1, kColXr><<<K, kThreads, 0, s>>>(blocks, partials, sc, 0); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void scatter_column(int32_t n, int K, int c, const double *v, double *M, cudaStream_t s, float *M32) {
    { scatter_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, K, c, v, M, M32); ::amg::count_launch(); }
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
void copy_masked_columns(int32_t n, int K, const double *T, double *R, const int *mask, cudaStream_t s, float *R32) {
    int64_t total = (int64_t)n * K;
    { copy_masked_kernel<<<div_up(total, kThreads), kThreads, 0, s>>>(total, K, T, R, R32, mask); ::amg::count_launch(); }
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

#define AMG_PINST(VT, XT) \
    template void pre_smooth_residual<VT, XT>(const CycMat<VT> &, int, const XT *, const XT *, XT *, XT *, cudaStream_t);
AMG_PINST(double, double)
AMG_PINST(float, float)
AMG_PINST(__nv_bfloat16, float)
#undef AMG_PINST
#define AMG_QINST(VT, XT, OT) \
    template void post_smooth<VT, XT, OT>(const CycMat<VT> &, int, const XT *, const XT *, const XT *, OT *, cudaStream_t);
AMG_QINST(double, double, double)
AMG_QINST(float, float, float)
AMG_QINST(__nv_bfloat16, float, float)
AMG_QINST(float, float, double)
AMG_QINST(__nv_bfloat16, float, double)
#undef AMG_QINST
#define AMG_SINST(VT, XT) template void spmm<VT, XT>(const CycMat<VT> &, int, const XT *, XT *, bool, cudaStream_t);
AMG_SINST(double, double)
AMG_SINST(float, float)
AMG_SINST(__nv_bfloat16, float)
#undef AMG_SINST
template void coarse_solve<double>(int32_t, int, const double *, const double *, double *, cudaStream_t);
template void coarse_solve<float>(int32_t, int, const double *, const float *, float *, cudaStream_t);
template void to_cycle<float>(const double *, float *, int64_t, cudaStream_t);
template void from_cycle<float>(const float *, double *, int64_t, cudaStream_t);

}  // namespace bat
}  // namespace amg
