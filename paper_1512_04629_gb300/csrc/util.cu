// util.cu -- device buffers, thread-local error text, exclusive scans.
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>

#include "common.cuh"

namespace amg {

static thread_local std::string g_last_error;
std::atomic<int64_t> g_device_bytes{0};

std::atomic<int64_t> g_launches{0};

void set_last_error(const std::string &msg) { g_last_error = msg; }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Host-side fault injection (amg_debug_fail_allocation): while the count is
// >= 0, every device allocation decrements it, and the one that finds it at
// 0 fails as out of memory (which disarms it).  No CUDA call is involved.
static std::atomic<int64_t> g_fail_after{-1};
void arm_allocation_failure(int64_t after) { g_fail_after.store(after < 0 ? -1 : after); }
bool injected_allocation_failure() {
    int64_t v = g_fail_after.load();
    while (v >= 0)
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

int resident_blocks(int threads_per_block) {
    static std::atomic<int> sm_count[64];
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    int sms = dev < 64 ? sm_count[dev].load(std::memory_order_relaxed) : 0;
    if (sms == 0) {
        AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (dev < 64) sm_count[dev].store(sms, std::memory_order_relaxed);
    }
    int per_sm = 2048 / threads_per_block;
    return sms * (per_sm > 0 ? per_sm : 1);
}
const char *last_error_cstr() { return g_last_error.c_str(); }

namespace {
__global__ void read_back_kernel(const unsigned char *__restrict__ src, unsigned char *__restrict__ dst, int bytes) {
    for (int i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = src[i];
}
// one mapped pinned buffer per thread and device, kept for the thread's life
struct MappedBuf {
    unsigned char *host = nullptr, *dev = nullptr;
};
constexpr int kMaxDevices = 64;
thread_local MappedBuf g_mapped[kMaxDevices];
}  // namespace

void read_back(void *dst, const void *dsrc, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    if (bytes > kReadBackMax) throw Error(AMG_ERR_INVALID, "read_back: more than kReadBackMax bytes");
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error(AMG_ERR_INVALID, "read_back: device index out of range");
    MappedBuf &m = g_mapped[dev];
    if (!m.host) {
        void *h = nullptr, *d = nullptr;
        AMG_CUDA(cudaHostAlloc(&h, kReadBackMax, cudaHostAllocMapped));
        AMG_CUDA(cudaHostGetDevicePointer(&d, h, 0));
        m.host = static_cast<unsigned char *>(h);
        m.dev = static_cast<unsigned char *>(d);
    }
    { read_back_kernel<<<1, 32, 0, s>>>(static_cast<const unsigned char *>(dsrc), m.dev, (int)bytes); count_launch(); }
    AMG_CHECK_LAUNCH();
    AMG_CUDA(cudaStreamSynchronize(s));
    std::memcpy(dst, m.host, bytes);
}

namespace {
thread_local int g_idle_depth = 0;
thread_local cudaStream_t g_alloc_stream = nullptr;
thread_local bool g_alloc_scoped = false;

// one non-blocking stream per device for pool allocations and bulk frees
cudaStream_t pool_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    if (dev >= 64) throw Error(AMG_ERR_CUDA, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev]) AMG_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    return streams[dev];
}
}  // namespace

AllocOn::AllocOn(cudaStream_t s) : prev(g_alloc_stream), prev_scoped(g_alloc_scoped) {
    g_alloc_stream = s;
    g_alloc_scoped = true;
}
AllocOn::~AllocOn() {
    g_alloc_stream = prev;
    g_alloc_scoped = prev_scoped;
}

void IdleRelease::enter() {
    if (!active) { ++g_idle_depth; active = true; }
}
IdleRelease::~IdleRelease() {
    if (active) --g_idle_depth;
}

static void keep_pool_warm();

void DevBuf::alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    if (injected_allocation_failure())
        throw Error(AMG_ERR_OOM, "device allocation of " + std::to_string(b) + " bytes failed (injected)");
    keep_pool_warm();
    cudaError_t e;
    if (g_alloc_scoped) {
        // ordered on the entry point's stream: usable by the work that follows there
        e = cudaMallocAsync(&ptr, b, g_alloc_stream);
    } else {
        cudaStream_t ps = pool_stream();
        e = cudaMallocAsync(&ptr, b, ps);
        // the pool may order the allocation after frees still pending on other
        // streams: wait for it, so the memory is usable from any stream at once
        if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        throw Error(e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA,
                    std::string("cudaMallocAsync(") + std::to_string(b) + "): " + cudaGetErrorString(e));
    }
    bytes = b;
    g_device_bytes += (int64_t)b;
}
void DevBuf::release() {
    if (ptr) {
        cudaStream_t ps = nullptr;
        if (g_idle_depth > 0) {
            try { ps = pool_stream(); } catch (...) { ps = nullptr; }
        }
        if (ps) cudaFreeAsync(ptr, ps);  // the owner synchronized the device
        else cudaFree(ptr);              // waits for the device first
        g_device_bytes -= (int64_t)bytes;
    }
    ptr = nullptr;
    bytes = 0;
}

// the default pool keeps freed blocks (no release back to the driver) so
// stream-ordered temporaries are recycled without synchronisation
static void keep_pool_warm() {
    static thread_local int done_for = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (done_for == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done_for = dev;
}

void TmpBuf::alloc(size_t b, cudaStream_t s) {
    release();
    keep_pool_warm();
    if (b == 0) b = 16;
    if (injected_allocation_failure())
        throw Error(AMG_ERR_OOM, "device allocation of " + std::to_string(b) + " bytes failed (injected)");
    cudaError_t e = cudaMallocAsync(&ptr, b, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        throw Error(e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA,
                    std::string("cudaMallocAsync(") + std::to_string(b) + "): " + cudaGetErrorString(e));
    }
    bytes = b;
    stream = s;
}

void TmpBuf::release() {
    if (ptr) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
    bytes = 0;
}

void DevCSR::allocate(int32_t r, int32_t c, int64_t z) {
    nrows = r;
    ncols = c;
    nnz = z;
    rowptr.alloc(sizeof(int32_t) * ((size_t)r + 1));
    col.alloc(sizeof(int32_t) * (size_t)(z + kPad));
    val.alloc(sizeof(double) * (size_t)(z + kPad));
}

// ---------------------------------------------------------------------------
// exclusive scan: out[i] = sum_{k<i} in[k], out[n] = total (three passes:
// per-tile sums, a single-block scan of the tile sums, tile-local scans)
// ---------------------------------------------------------------------------
namespace {
constexpr int kScanThreads = 256, kScanItems = 4, kTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *total) {
    __shared__ T warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    T base = w > 0 ? warp_sums[w - 1] : T(0);
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

template <typename TI>
__global__ void tile_sum_kernel(const TI *in, int64_t n, int64_t *sums) {
    int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    int64_t tot;
    block_exclusive_scan<int64_t>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename TO>
__global__ void scan_sums_kernel(int64_t *sums, int64_t m, int64_t *total, TO *out_n) {
    int64_t carry = 0;
    for (int64_t b = 0; b < m; b += kScanThreads) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < m ? sums[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan<int64_t>(v, &tot);
        if (i < m) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *total = carry;
        *out_n = (TO)carry;  // checked against the int32 range by the host reader
    }
}

template <typename TI, typename TO>
__global__ void tile_scan_kernel(const TI *in, int64_t n, const int64_t *sums, TO *out) {
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan<int64_t>(s, &tot) + sums[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = (TO)ex;
        ex += v[k];
    }
}

// all on the stream, nothing read back: out[0..n] and *total on the device
// Short arrays: the whole scan in one block (one launch instead of three);
// each thread scans a contiguous chunk, the block scans the chunk sums.
constexpr int64_t kOneBlockScan = 16 * 1024;

template <typename TI, typename TO>
__global__ void one_block_scan_kernel(const TI *in, int64_t n, TO *out, int64_t *total) {
    const int64_t chunk = (n + kScanThreads - 1) / kScanThreads;
    const int64_t b0 = (int64_t)threadIdx.x * chunk, b1 = b0 + chunk < n ? b0 + chunk : n;
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += (int64_t)in[i];
    int64_t tot;
    int64_t ex = block_exclusive_scan<int64_t>(s, &tot);
    for (int64_t i = b0; i < b1; ++i) {
        const int64_t v = (int64_t)in[i];
        out[i] = (TO)ex;
        ex += v;
    }
    if (threadIdx.x == 0) {
        *total = tot;
        out[n] = (TO)tot;  // checked against the int32 range by the host reader
    }
}

template <typename TI, typename TO>
void scan_launch(const TI *in, TO *out, int64_t n, int64_t *total, cudaStream_t s) {
    int64_t tiles = (n + kTile - 1) / kTile;
    if (n > 0 && n <= kOneBlockScan) {
        { one_block_scan_kernel<TI, TO><<<1, kScanThreads, 0, s>>>(in, n, out, total); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        return;
    }
    if (n > 0) {
        TmpBuf sums(sizeof(int64_t) * (tiles + 1), s);
        { tile_sum_kernel<TI><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums.as<int64_t>()); ::amg::count_launch(); }
        { scan_sums_kernel<TO><<<1, kScanThreads, 0, s>>>(sums.as<int64_t>(), tiles, total, out + n); ::amg::count_launch(); }
        { tile_scan_kernel<TI, TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums.as<int64_t>(), out); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
    } else {
        AMG_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        AMG_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), s));
    }
}

template <typename TI, typename TO>
int64_t scan_impl(const TI *in, TO *out, int64_t n, cudaStream_t s) {
    TmpBuf total(sizeof(int64_t), s);
    scan_launch<TI, TO>(in, out, n, total.as<int64_t>(), s);
    int64_t t = read_scalar(total.as<int64_t>(), s);
    if (sizeof(TO) == 4 && t >= ((int64_t)1 << 31))
        throw Error(AMG_ERR_INVALID, "scan: total exceeds the int32 index range");
    return t;
}
}  // namespace

int64_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t, int32_t>(in, out, n, s);
}
int64_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t, int64_t>(in, out, n, s);
}
int64_t exclusive_scan_i64_from_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t, int64_t>(in, out, n, s);
}
void exclusive_scan_i64_async(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s) {
    scan_launch<int64_t, int64_t>(in, out, n, total, s);
}
void exclusive_scan_i32_known(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    TmpBuf total(sizeof(int64_t), s);
    scan_launch<int32_t, int32_t>(in, out, n, total.as<int64_t>(), s);
}

}  // namespace amg
