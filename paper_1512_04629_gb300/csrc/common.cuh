// common.cuh -- internal definitions shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/amg.h"

namespace amg {

// ---------------------------------------------------------------------------
// errors: internal code throws amg::Error; the C ABI turns it into a status.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
    amg_status status;
    Error(amg_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

void set_last_error(const std::string &msg);

// number of kernels the library has launched (diagnostic counter)
void count_launch();
// host-side fault injection: the allocation `after` device allocations from
// now fails as out of memory (-1: off); injected_allocation_failure() is
// asked by every device allocation and answers true for the one that fails
void arm_allocation_failure(int64_t after);
bool injected_allocation_failure();
// thread blocks of the given size that fit on the current device at once
// (SM count x resident blocks per SM at full thread occupancy), cached
int resident_blocks(int threads_per_block);

#define AMG_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            if (e_ == cudaErrorMemoryAllocation) {                                         \
                cudaGetLastError();                                                        \
                throw ::amg::Error(AMG_ERR_OOM, std::string("device allocation: ") +      \
                                                     cudaGetErrorString(e_));              \
            }                                                                              \
            throw ::amg::Error(AMG_ERR_CUDA, std::string(#call) + ": " +                   \
                                                 cudaGetErrorString(e_) + " at " +         \
                                                 __FILE__ + ":" + std::to_string(__LINE__)); \
        }                                                                                  \
    } while (0)

#define AMG_CHECK_LAUNCH() AMG_CUDA(cudaGetLastError())

inline void require(bool ok, const std::string &msg) {
    if (!ok) throw Error(AMG_ERR_INVALID, msg);
}
// literal messages bind here: nothing is constructed unless the check fails
// (the host-side validation loops call this once per matrix entry)
inline void require(bool ok, const char *msg) {
    if (!ok) throw Error(AMG_ERR_INVALID, msg);
}

// ---------------------------------------------------------------------------
// device buffers (RAII); every persistent allocation of the library goes
// through DevBuf so amg_device_bytes can account for it.
// ---------------------------------------------------------------------------
// A device buffer owned by a hierarchy (or a server).  Memory comes from the
// device's stream-ordered pool (kept warm: freed blocks stay in the pool for
// the next setup instead of going back to the driver); the allocation is
// complete when alloc() returns, so any stream may use it.  release() waits
// for the whole device unless the owner has already done so and opened an
// IdleRelease scope.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    explicit DevBuf(size_t b) { alloc(b); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : ptr(o.ptr), bytes(o.bytes) { o.ptr = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr; bytes = o.bytes;
            o.ptr = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t b);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// Bulk teardown: the owner synchronizes the device, then calls enter(); every
// DevBuf released on this thread until the guard is destroyed goes back to
// the pool without another device-wide wait.  Declare the guard as the
// owner's first member so it outlives the members it covers.
struct IdleRelease {
    bool active = false;
    void enter();
    ~IdleRelease();
};

// While an entry point runs on stream s, buffers it allocates are ordered on
// s (no wait for the allocation); whoever later uses them on another stream
// does so after the entry point has synchronized s.  Without a scope,
// allocation waits for the pool's own stream.
struct AllocOn {
    cudaStream_t prev;
    bool prev_scoped;
    explicit AllocOn(cudaStream_t s);
    ~AllocOn();
};

// A temporary device buffer with stream-ordered lifetime: allocated with
// cudaMallocAsync and returned with cudaFreeAsync on the stream that uses it,
// so freeing never waits for the device (the pool keeps the memory).
struct TmpBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    TmpBuf() = default;
    TmpBuf(size_t b, cudaStream_t s) { alloc(b, s); }
    TmpBuf(const TmpBuf &) = delete;
    TmpBuf &operator=(const TmpBuf &) = delete;
    ~TmpBuf() { release(); }
    void alloc(size_t b, cudaStream_t s);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// A CSR matrix resident on the device (library-owned).
struct DevCSR {
    int32_t nrows = 0, ncols = 0;
    int64_t nnz = 0;
    DevBuf rowptr, col, val;  // int32[nrows+1], int32[nnz(+pad)], double[nnz(+pad)]
    const int32_t *rp() const { return rowptr.as<int32_t>(); }
    const int32_t *ci() const { return col.as<int32_t>(); }
    const double *v() const { return val.as<double>(); }
    int32_t *rp() { return rowptr.as<int32_t>(); }
    int32_t *ci() { return col.as<int32_t>(); }
    double *v() { return val.as<double>(); }
    size_t bytes() const { return rowptr.bytes + col.bytes + val.bytes; }
    // allocate with `pad` spare entries so vector loads past the last row stay in bounds
    void allocate(int32_t r, int32_t c, int64_t z);
};

constexpr int64_t kPad = 16;  // spare entries at the end of every CSR array

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
inline int div_up(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

// exclusive scan of n int32 counts into out[0..n] (out[n] = total); returns total
int64_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
int64_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
int64_t exclusive_scan_i64_from_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
// the same without reading back: out[n] and *total (device) are written on the stream
void exclusive_scan_i64_async(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s);
// int32 scan whose total the caller already knows (no read-back)
void exclusive_scan_i32_known(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);

// Copies `bytes` (at most kReadBackMax) of device memory to dst once the
// stream's work before it has finished.  A one-block kernel writes them into
// mapped pinned host memory of the calling thread and the stream is
// synchronised: on this part that round trip costs what the synchronisation
// alone costs, where a copy into pageable (pinned) memory added 5 (3) us.
constexpr size_t kReadBackMax = 256;
void read_back(void *dst, const void *dsrc, size_t bytes, cudaStream_t s);

template <typename T> T read_scalar(const T *dptr, cudaStream_t s) {
    T v;
    read_back(&v, dptr, sizeof(T), s);
    return v;
}

}  // namespace amg
