// gmres.cu -- kernels of the restarted flexible GMRES outer solver.
//
// One Arnoldi step of FGMRES(m) (Saad 1993) with the V-cycle as right
// preconditioner: z_j = M v_j, w = A_0 z_j, classical Gram-Schmidt
// (h = V^T w, w -= V h: each pass is one streaming read of the basis instead
// of j + 1 dependent reductions) with a second pass only when the first
// removed more than half of ||w||^2 (Daniel, Gragg, Kaufman, Stewart 1976:
// "twice is enough"), h_{j+1,j} = ||w||, the Givens rotations of the
// Hessenberg column, v_{j+1} = w / h_{j+1,j}.  On this part the FP64 FMAs
// of the passes cost as much as their HBM traffic, so the skipped pass
// halves the orthogonalisation.
// The basis size j is a device scalar, so the step is one fixed launch
// sequence and a restart cycle runs as one CUDA-graph WHILE loop.  Every
// reduction is deterministic: per-block partials in a fixed layout, summed
// in block order by a finisher.
#include "gmres_ops.cuh"

namespace amg {

GmresArrays gmres_arrays(double *base, int m) {
    GmresArrays a;
    double *p = base;
    a.H = p; p += (size_t)(m + 1) * m;
    a.cs = p; p += m;
    a.sn = p; p += m;
    a.g = p; p += m + 1;
    a.y = p; p += m;
    a.hc = p; p += m + 1;
    a.hc2 = p; p += m + 1;
    a.part = p;
    return a;
}

namespace gm {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;       // basis vectors per block row of the dot kernel
constexpr int kMaxCoef = 513;   // restart length <= 512

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < kThreads / 32 ? sh[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            v[k] = x;
        }
    }
}

// Block sums of NV values through shared memory: each of NV x 8 threads adds
// 32 values in a fixed order, then NV threads add the 8 results.  A shuffle
// tree costs five warp-wide FP64 adds per value and warp, and on this part
// each occupies the FP64 pipe for 16 clocks: with a few elements per thread
// those trees took more FP64 issue than the dot products themselves; this
// takes about a quarter of it.  Result in v[] of thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_smem(double (&v)[NV]) {
    constexpr int kPadRow = kThreads + 4;
    __shared__ double sh[NV][kPadRow];
    __shared__ double sh2[NV][8];
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int t = threadIdx.x; t < NV * 8; t += blockDim.x) {
        const int k = t >> 3, s = t & 7;
        double x = 0.0;
        for (int u = 0; u < kThreads / 8; ++u) x += sh[k][u * 8 + s];
        sh2[k][s] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
            for (int s = 0; s < 8; ++s) x += sh2[k][s];
            v[k] = x;
        }
    }
}

// partial dot products of w with NV basis vectors from i0, and w . w (WW)
template <int NV, bool WW>
__device__ __forceinline__ void mdot_loop(int64_t n, const double *__restrict__ V, const double *__restrict__ w,
                                          int i0, double (&acc)[kGroup + 1]) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const double we = w[e];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += V[(size_t)(i0 + q) * n + e] * we;
        if (WW) acc[kGroup] += we * we;
    }
}

// partial dot products of w with basis vectors 8 y .. 8 y + 7 (y = blockIdx.y):
// eight independent loads per element keep enough requests in flight, and a
// loop specialised on the block's vector count issues no predicated-off FP64
// FMAs (they would still occupy the FP64 pipe);
// WW: the y = 0 blocks also sum w . w into part row m + 1
template <bool WW>
__global__ void __launch_bounds__(kThreads)
mdot_kernel(int64_t n, int m, const double *__restrict__ V, const double *__restrict__ w, const GmresScalars *sc,
            double *part) {
    if (!WW && !sc->reorth) return;  // second pass skipped (uniform)
    const int j = sc->j;
    const int i0 = blockIdx.y * kGroup;
    if (i0 > j) return;  // uniform over the block
    const int nv = min(kGroup, j + 1 - i0);
    double acc[kGroup + 1];
#pragma unroll
    for (int q = 0; q <= kGroup; ++q) acc[q] = 0.0;
    const bool ww = WW && blockIdx.y == 0;
    switch (nv) {
        case 1: ww ? mdot_loop<1, true>(n, V, w, i0, acc) : mdot_loop<1, false>(n, V, w, i0, acc); break;
        case 2: ww ? mdot_loop<2, true>(n, V, w, i0, acc) : mdot_loop<2, false>(n, V, w, i0, acc); break;
        case 3: ww ? mdot_loop<3, true>(n, V, w, i0, acc) : mdot_loop<3, false>(n, V, w, i0, acc); break;
        case 4: ww ? mdot_loop<4, true>(n, V, w, i0, acc) : mdot_loop<4, false>(n, V, w, i0, acc); break;
        case 5: ww ? mdot_loop<5, true>(n, V, w, i0, acc) : mdot_loop<5, false>(n, V, w, i0, acc); break;
        case 6: ww ? mdot_loop<6, true>(n, V, w, i0, acc) : mdot_loop<6, false>(n, V, w, i0, acc); break;
        case 7: ww ? mdot_loop<7, true>(n, V, w, i0, acc) : mdot_loop<7, false>(n, V, w, i0, acc); break;
        default: ww ? mdot_loop<8, true>(n, V, w, i0, acc) : mdot_loop<8, false>(n, V, w, i0, acc); break;
    }
    block_sum_smem<kGroup + 1>(acc);
    if (threadIdx.x == 0) {
        for (int q = 0; q < nv; ++q) part[(size_t)(i0 + q) * kGmresMaxBlocks + blockIdx.x] = acc[q];
        if (ww) part[(size_t)(m + 1) * kGmresMaxBlocks + blockIdx.x] = acc[kGroup];
    }
}

// out[i] = sum over blocks of part row i, i = 0..j (and, WW, sc->ww from
// row m + 1): one warp per vector
template <bool WW>
__global__ void mdot_finish_kernel(int nblocks, int m, GmresScalars *sc, const double *part, double *out) {
    if (!WW && !sc->reorth) return;
    const int j = sc->j;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rows = WW ? j + 2 : j + 1;
    for (int q = wid; q < rows; q += nw) {
        const int i = q <= j ? q : m + 1;
        double t = 0.0;
        for (int b = lane; b < nblocks; b += 32) t += part[(size_t)i * kGmresMaxBlocks + b];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            if (q <= j) out[i] = t;
            else sc->ww = t;
        }
    }
}

// second pass or not: ||w'||^2 from the first update's partials
__global__ void decide_kernel(int nblocks, GmresScalars *sc, GmresArrays ar) {
    const int lane = threadIdx.x;
    double t = 0.0;
    for (int b = lane; b < nblocks; b += 32) t += ar.part[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const bool again = !(t >= 0.5 * sc->ww);  // also on a non-finite norm
    const int j = sc->j;
    if (!again)
        for (int i = lane; i <= j; i += 32) ar.hc2[i] = 0.0;
    if (lane == 0) {
        sc->wn2 = t;
        sc->reorth = again ? 1 : 0;
    }
}

// out = base + sign * sum_{i < cnt} coef[i] V_i, cnt = j + 1 (update) or j
// (forming x); NORM: ||out||^2 block partials into part row 0; IFREORTH:
// only when the second pass runs
template <bool NORM, bool IFREORTH>
__global__ void __launch_bounds__(kThreads)
combo_kernel(int64_t n, const double *base, double *out, const double *__restrict__ V, const double *coef,
             const GmresScalars *sc, int cnt_plus, double sign, double *part) {
    if (IFREORTH && !sc->reorth) return;
    __shared__ double c[kMaxCoef];
    const int cnt = sc->j + cnt_plus;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) c[i] = sign * coef[i];
    __syncthreads();
    double nrm[1] = {0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        double t = base[e];
        for (int i = 0; i < cnt; ++i) t += c[i] * V[(size_t)i * n + e];
        out[e] = t;
        if (NORM) nrm[0] += t * t;
    }
    if (NORM) {
        block_sum<1>(nrm);
        if (threadIdx.x == 0) part[blockIdx.x] = nrm[0];
    }
}

// ||w||, the Hessenberg column j, its Givens rotation and the stop test
__global__ void step_finish_kernel(int nblocks, GmresScalars *sc, GmresArrays ar,
                                   cudaGraphConditionalHandle handle, int use_handle) {
    const int lane = threadIdx.x;
    double t = 0.0;
    if (sc->reorth) {
        for (int b = lane; b < nblocks; b += 32) t += ar.part[b];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    } else {
        t = sc->wn2;
    }
    if (lane != 0) return;
    const int j = sc->j, m = sc->m;
    const double hn = sqrt(t);
    bool finite = isfinite(hn);
    for (int i = 0; i <= j; ++i) {
        const double h = ar.hc[i] + ar.hc2[i];
        ar.H[(size_t)i * m + j] = h;
        finite = finite && isfinite(h);
    }
    sc->its += 1;
    if (!finite) {  // the step is lost: the cycle keeps its j columns
        sc->breakdown = 1;
        if (use_handle) cudaGraphSetConditional(handle, 0u);
        return;
    }
    ar.H[(size_t)(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = ar.H[(size_t)i * m + j], c = ar.H[(size_t)(i + 1) * m + j];
        ar.H[(size_t)i * m + j] = ar.cs[i] * a + ar.sn[i] * c;
        ar.H[(size_t)(i + 1) * m + j] = -ar.sn[i] * a + ar.cs[i] * c;
    }
    const double a = ar.H[(size_t)j * m + j];
    const double r = sqrt(a * a + hn * hn);
    const bool ok = r > 0.0;
    ar.cs[j] = ok ? a / r : 1.0;
    ar.sn[j] = ok ? hn / r : 0.0;
    ar.H[(size_t)j * m + j] = r;
    ar.H[(size_t)(j + 1) * m + j] = 0.0;
    ar.g[j + 1] = -ar.sn[j] * ar.g[j];
    ar.g[j] = ar.cs[j] * ar.g[j];
    const double est = fabs(ar.g[j + 1]);
    sc->est = est;
    sc->hn = hn;
    sc->happy = hn == 0.0;
    if (!ok) {  // singular Hessenberg column
        sc->breakdown = 1;
        if (use_handle) cudaGraphSetConditional(handle, 0u);
        return;
    }
    sc->j = j + 1;
    if (use_handle) {
        const bool go = est > sc->thresh && hn > 0.0 && j + 1 < m && sc->its < sc->max_its;
        cudaGraphSetConditional(handle, go ? 1u : 0u);
    }
}

__global__ void normalize_kernel(int64_t n, const double *w, double *V, double *next, const GmresScalars *sc) {
    if (sc->breakdown) return;
    const int j = sc->j;
    const double hn = sc->hn;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const double v = hn > 0.0 ? w[e] / hn : 0.0;
        V[(size_t)j * n + e] = v;
        next[e] = v;
    }
}

__global__ void store_z_kernel(int64_t n, const double *z, double *Z, const GmresScalars *sc) {
    const int j = sc->j;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
        Z[(size_t)j * n + e] = z[e];
}

__global__ void start_kernel(int64_t n, const double *r, double *V, double *next, GmresScalars *sc,
                             GmresArrays ar) {
    const double beta = sqrt(sc->tt);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const double v = beta > 0.0 ? r[e] / beta : 0.0;
        V[e] = v;
        next[e] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i <= sc->m; ++i) ar.g[i] = 0.0;
        ar.g[0] = beta;
        sc->j = 0;
        sc->est = beta;
        sc->hn = 0.0;
        sc->breakdown = 0;
        sc->happy = 0;
    }
}

// back substitution R y = g over the cycle's j columns (one thread: j <= 512)
__global__ void solve_y_kernel(GmresScalars *sc, GmresArrays ar) {
    const int j = sc->j, m = sc->m;
    for (int i = j - 1; i >= 0; --i) {
        double t = ar.g[i];
        for (int c = i + 1; c < j; ++c) t -= ar.H[(size_t)i * m + c] * ar.y[c];
        ar.y[i] = t / ar.H[(size_t)i * m + i];
    }
}

int stream_blocks(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    int64_t cap = ::amg::resident_blocks(kThreads);
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace

int dot_blocks(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    int64_t cap = std::min<int64_t>(::amg::resident_blocks(kThreads), kGmresMaxBlocks);
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

namespace {
// the dot kernel's block columns: at least 8 elements per thread, so the
// per-block sums stay small next to the streaming FMAs
int mdot_blocks(int64_t n) {
    int64_t b = (n + kThreads * 8 - 1) / (kThreads * 8);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, dot_blocks(n)));
}
}  // namespace

void mdot(int64_t n, int m, const double *V, const double *w, GmresScalars *sc, GmresArrays ar, bool second,
          cudaStream_t s) {
    const int bx = mdot_blocks(n);
    const dim3 grid(bx, (m + 1 + kGroup - 1) / kGroup);
    if (second) {
        { mdot_kernel<false><<<grid, kThreads, 0, s>>>(n, m, V, w, sc, ar.part); ::amg::count_launch(); }
        { mdot_finish_kernel<false><<<1, 1024, 0, s>>>(bx, m, sc, ar.part, ar.hc2); ::amg::count_launch(); }
    } else {
        { mdot_kernel<true><<<grid, kThreads, 0, s>>>(n, m, V, w, sc, ar.part); ::amg::count_launch(); }
        { mdot_finish_kernel<true><<<1, 1024, 0, s>>>(bx, m, sc, ar.part, ar.hc); ::amg::count_launch(); }
    }
    AMG_CHECK_LAUNCH();
}

void mupdate(int64_t n, int m, const double *V, double *w, GmresScalars *sc, GmresArrays ar, bool second,
             cudaGraphConditionalHandle handle, bool use_handle, cudaStream_t s) {
    (void)m;
    const int bx = dot_blocks(n);
    if (second) {
        { combo_kernel<true, true><<<bx, kThreads, 0, s>>>(n, w, w, V, ar.hc2, sc, 1, -1.0, ar.part); ::amg::count_launch(); }
        { step_finish_kernel<<<1, 32, 0, s>>>(bx, sc, ar, handle, use_handle ? 1 : 0); ::amg::count_launch(); }
    } else {
        { combo_kernel<true, false><<<bx, kThreads, 0, s>>>(n, w, w, V, ar.hc, sc, 1, -1.0, ar.part); ::amg::count_launch(); }
        { decide_kernel<<<1, 32, 0, s>>>(bx, sc, ar); ::amg::count_launch(); }
    }
    AMG_CHECK_LAUNCH();
}

void normalize(int64_t n, const double *w, double *V, double *next, const GmresScalars *sc, cudaStream_t s) {
    { normalize_kernel<<<stream_blocks(n), kThreads, 0, s>>>(n, w, V, next, sc); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void store_z(int64_t n, const double *z, double *Z, const GmresScalars *sc, cudaStream_t s) {
    { store_z_kernel<<<stream_blocks(n), kThreads, 0, s>>>(n, z, Z, sc); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void start(int64_t n, const double *r, double *V, double *next, GmresScalars *sc, GmresArrays ar, cudaStream_t s) {
    { start_kernel<<<stream_blocks(n), kThreads, 0, s>>>(n, r, V, next, sc, ar); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void form_x(int64_t n, int m, const double *Z, const double *x0, double *x, GmresScalars *sc, GmresArrays ar,
            cudaStream_t s) {
    (void)m;
    { solve_y_kernel<<<1, 1, 0, s>>>(sc, ar); ::amg::count_launch(); }
    { combo_kernel<false, false><<<dot_blocks(n), kThreads, 0, s>>>(n, x0, x, Z, ar.y, sc, 0, 1.0, ar.part); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

}  // namespace gm
}  // namespace amg
