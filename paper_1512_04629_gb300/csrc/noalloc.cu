// noalloc.cu -- residual and its norm for callers that cannot allocate.
//
// Some callers must not allocate device memory at the moment they call: code
// that runs under a framework or real-time loop whose device memory is handed
// out only by its own pool (a cudaMalloc there would bypass the pool's
// accounting, or stall the loop while the driver maps memory), and callers
// whose memory budget is already fully committed, where an allocation would
// fail.  For them, amg_residual_noalloc computes r = b - A_0 x and ||r||_2
// (the quantity an outer iteration checks for convergence) with its
// reduction scratch in a fixed array that the library image carries in
// device memory, so the call allocates nothing.
//
// The scratch: one FP64 partial per block (at most kBlocks blocks of
// kRowsPerBlock rows), the partials of each group of 256 blocks, and arrival
// counters -- about 530 KB, held by every GPU that loads the library until
// the process exits.  Every call shares it and it keeps the last call's
// contents; the counters are cleared (an asynchronous memset, not an
// allocation) at the start of each call.  Calls whose kernels overlap on the
// GPU race on the scratch: issue them on one stream, or order them.
#include <mutex>

#include "hierarchy.cuh"

namespace amg {
void set_last_error(const std::string &msg);
}

using namespace amg;

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 65536;
constexpr int kRowsPerBlock = 1024;
constexpr int64_t kMaxRows = (int64_t)kBlocks * kRowsPerBlock;  // 67,108,864
constexpr int kMaxDevices = 64;

struct Scratch {
    double partials[kBlocks];
    double gpartials[256];
    unsigned counters[512];  // [0]: groups done; [1 + g]: blocks done in group g
};

static __device__ __align__(256) Scratch g_noalloc_scratch;

std::mutex g_mu;
Scratch *g_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device.  In host code the symbol is only a stand-in for the device array,
// so the address must come from cudaGetSymbolAddress.
Scratch *scratch_for_current_device() {
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    require(dev >= 0 && dev < kMaxDevices, "device ordinal out of range for the no-alloc scratch");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(AMG_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        }
        g_ptr[dev] = static_cast<Scratch *>(p);
    }
    return g_ptr[dev];
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = lane < kThreads / 32 ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;  // valid in thread 0
}

// r = b - A x on kRowsPerBlock rows per block (4 lanes per row), ||r||^2 by a
// fixed two-level tree: per block, per group of 256 blocks, over the groups.
__global__ void __launch_bounds__(kThreads)
residual_noalloc_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                        const double *__restrict__ v, const double *__restrict__ b, const double *__restrict__ x,
                        double *__restrict__ r, double *__restrict__ norm_out, Scratch *sc) {
    constexpr int T = 4;
    double part = 0.0;
    int64_t row0 = (int64_t)blockIdx.x * kRowsPerBlock;
    for (int64_t base = row0; base < row0 + kRowsPerBlock; base += kThreads / T) {
        int64_t i = base + threadIdx.x / T;
        int t = threadIdx.x % T;
        double s = 0.0;
        if (i < n) {
            for (int32_t p = __ldg(rp + i) + t; p < __ldg(rp + i + 1); p += T) s += __ldg(v + p) * __ldg(x + __ldg(ci + p));
        }
        for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, T);
        if (i < n && t == 0) {
            double e = b[i] - s;
            r[i] = e;
            part += e * e;
        }
    }
    __shared__ bool last;
    const int g = blockIdx.x >> 8;
    const int gsize = min(256, (int)gridDim.x - g * 256);
    const int ngroups = ((int)gridDim.x + 255) >> 8;
    double tot = block_sum(part);
    if (threadIdx.x == 0) {
        sc->partials[blockIdx.x] = tot;
        __threadfence();
        last = atomicAdd(&sc->counters[1 + g], 1u) == (unsigned)gsize - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    tot = block_sum((int)threadIdx.x < gsize ? ((volatile double *)sc->partials)[g * 256 + threadIdx.x] : 0.0);
    if (threadIdx.x == 0) {
        sc->gpartials[g] = tot;
        __threadfence();
        last = atomicAdd(&sc->counters[0], 1u) == (unsigned)ngroups - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    tot = block_sum((int)threadIdx.x < ngroups ? ((volatile double *)sc->gpartials)[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) *norm_out = sqrt(tot);
}

// True for device (or managed) memory that belongs to device `dev`.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" amg_status amg_residual_noalloc(const amg_hierarchy *H, const double *b, const double *x, double *r,
                                           double *rnorm, void *stream) {
    try {
        set_last_error("");
        require(H != nullptr && b != nullptr && x != nullptr && r != nullptr && rnorm != nullptr, "NULL argument");
        const Level &L0 = *H->h.lev[0];
        int64_t n = L0.A.nrows;
        require(n <= kMaxRows, "amg_residual_noalloc: n = " + std::to_string(n) +
                                   " exceeds the fixed scratch capacity of 67,108,864 rows");
        int dev = -1;
        AMG_CUDA(cudaGetDevice(&dev));
        require(dev == H->h.device, "amg_residual_noalloc: the current device (" + std::to_string(dev) +
                                        ") is not the hierarchy's device (" + std::to_string(H->h.device) + ")");
        require(on_device(b, dev) && on_device(x, dev) && on_device(r, dev) && on_device(rnorm, dev),
                "amg_residual_noalloc: b, x, r and rnorm must be device memory of the hierarchy's device");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        Scratch *sc = scratch_for_current_device();
        AMG_CUDA(cudaMemsetAsync(sc->counters, 0, sizeof(sc->counters), s));
        int blocks = (int)((n + kRowsPerBlock - 1) / kRowsPerBlock);
        if (blocks < 1) blocks = 1;
        { residual_noalloc_kernel<<<blocks, kThreads, 0, s>>>((int32_t)n, L0.A.rp(), L0.A.ci(), L0.A.v(), b, x, r, rnorm, sc); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        return AMG_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return AMG_ERR_CUDA;
    }
}
