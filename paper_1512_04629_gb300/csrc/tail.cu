// tail.cu -- the coarse end of the V-cycle in one cooperative launch.
//
// On the coarse levels of a hierarchy every relaxation, restriction and
// prolongation is a few microseconds of launch and dependency latency around
// a few microseconds of work.  This kernel runs all of them for the levels
// from the first one with at most kTailRows rows down to the coarsest, phases
// separated by a grid barrier, so the cycle pays one launch for the whole
// coarse end.  The arithmetic per row is that of the per-level kernels
// (vector-CSR sums in the cycle precision, FP64 dense coarse solve).
//
// The barrier waits are bounded: a wait that runs out sets the error flag,
// every later barrier returns at once, and the host reports the failure.
#include <cuda_bf16.h>

#include "common.cuh"
#include "cycle_ops.cuh"
#include "tail_ops.cuh"

namespace amg {
namespace cyc {

namespace {

constexpr int kTailThreads = 256;
constexpr int kLanes = 8;                          // lanes per row
constexpr long long kBarrierCycles = 2000000000ll;  // about one second at 2 GHz

template <typename VT, typename XT> __device__ __forceinline__ XT val_as(VT v) { return (XT)v; }
template <> __device__ __forceinline__ float val_as<__nv_bfloat16, float>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// Vectors are written by other blocks inside this launch: read them through
// L2 only (L1 is not coherent across SMs).
template <typename T> __device__ __forceinline__ T ldv(const T *p) { return __ldcg(p); }

// Returns false, in every thread of the block alike, once any block's wait
// has run out (the decision goes through shared memory so the block never
// splits between returning and waiting at the next barrier).
__device__ bool grid_barrier(const TailSync &sync) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = sync.gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(sync.count, 1u) == gridDim.x - 1) {
            atomicExch(sync.count, 0u);
            __threadfence();
            atomicAdd(sync.gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > kBarrierCycles) {
                    atomicExch(sync.err, 1);
                    break;
                }
            }
        }
        __threadfence();
        ok = *(volatile int *)sync.err == 0;
    }
    __syncthreads();
    return ok != 0;
}

// Every row of a CSR matrix with values MV: s_i = sum_j m_ij x_j, handed to
// f(i, s) by the row's first lane.  Groups of kLanes lanes per row; the loop
// bounds are the same for every thread of the grid (shuffles stay full-warp).
template <typename MV, typename XT, class F>
__device__ __forceinline__ void rows_apply(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                           const MV *__restrict__ v, const XT *x, F f) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / kLanes;
    const int64_t g = gtid / kLanes;
    const int t = (int)(gtid % kLanes);
    for (int64_t base = 0; base < n; base += ngroups) {
        const int64_t i = base + g;
        XT acc = XT(0);
        if (i < n) {
            const int32_t p1 = __ldg(rp + i + 1);
            for (int32_t p = __ldg(rp + i) + t; p < p1; p += kLanes)
                acc += val_as<MV, XT>(__ldg(v + p)) * ldv(x + __ldg(ci + p));
        }
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, kLanes);
        if (i < n && t == 0) f((int32_t)i, acc);
    }
}

template <typename VT, typename XT>
__global__ void __launch_bounds__(kTailThreads)
tail_kernel(const TailLevel<VT, XT> *__restrict__ lv, int nl, const double *__restrict__ inv, int32_t nL,
            TailSync sync) {
    // down: residual of the pre-smoothed x = D^{-1} b, restriction (with the
    // next level's pre-smooth folded in unless it is the coarsest)
    for (int k = 0; k + 1 < nl; ++k) {
        const TailLevel<VT, XT> V = lv[k];
        rows_apply<VT, XT>(V.n, V.rp, V.ci, V.v, V.x, [&](int32_t i, XT s) { V.r[i] = ldv(V.b + i) - s; });
        if (!grid_barrier(sync)) return;
        const TailLevel<VT, XT> C = lv[k + 1];
        const bool relax_c = k + 2 < nl;
        rows_apply<XT, XT>(C.n, V.rrp, V.rci, V.rv, V.r, [&](int32_t c, XT s) {
            C.b[c] = s;
            if (relax_c) C.x[c] = s * C.dinv[c];
        });
        if (!grid_barrier(sync)) return;
    }
    // coarsest level: xo = inv b, FP64 sums, one warp per row
    {
        const TailLevel<VT, XT> C = lv[nl - 1];
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
        const int lane = threadIdx.x & 31;
        for (int64_t row = gtid / 32; row < nL; row += nwarps) {
            double acc = 0.0;
            for (int32_t j = lane; j < nL; j += 32) acc += __ldg(inv + row * nL + j) * (double)ldv(C.b + j);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) C.xo[row] = (XT)acc;
        }
        if (!grid_barrier(sync)) return;
    }
    // up: prolongation, then post-smoothing into xo
    for (int k = nl - 2; k >= 0; --k) {
        const TailLevel<VT, XT> V = lv[k];
        const TailLevel<VT, XT> C = lv[k + 1];
        rows_apply<XT, XT>(V.n, V.prp, V.pci, V.pv, C.xo, [&](int32_t i, XT s) { V.x[i] = ldv(V.x + i) + s; });
        if (!grid_barrier(sync)) return;
        rows_apply<VT, XT>(V.n, V.rp, V.ci, V.v, V.x, [&](int32_t i, XT s) {
            V.xo[i] = ldv(V.x + i) + V.dinv[i] * (ldv(V.b + i) - s);
        });
        if (k > 0 && !grid_barrier(sync)) return;
    }
}

}  // namespace

template <typename VT, typename XT> int tail_grid() {
    static int cached[64] = {};
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && cached[dev]) return cached[dev];
    int per_sm = 0, sms = 0;
    AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_kernel<VT, XT>, kTailThreads, 0));
    AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int g = std::max(1, std::min(per_sm, 2)) * sms;
    if (dev < 64) cached[dev] = g;
    return g;
}

template <typename VT, typename XT>
void tail_cycle(const TailLevel<VT, XT> *lv_dev, int nl, const double *coarse_inv, int32_t n_coarse,
                TailSync sync, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident at once, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, tail_kernel<VT, XT>, lv_dev, nl, coarse_inv, n_coarse, sync));
    ::amg::count_launch();
}

template void tail_cycle<double, double>(const TailLevel<double, double> *, int, const double *, int32_t, TailSync, int,
                                         cudaStream_t);
template void tail_cycle<float, float>(const TailLevel<float, float> *, int, const double *, int32_t, TailSync, int,
                                       cudaStream_t);
template void tail_cycle<__nv_bfloat16, float>(const TailLevel<__nv_bfloat16, float> *, int, const double *, int32_t,
                                               TailSync, int, cudaStream_t);
template int tail_grid<double, double>();
template int tail_grid<float, float>();
template int tail_grid<__nv_bfloat16, float>();

}  // namespace cyc
}  // namespace amg
