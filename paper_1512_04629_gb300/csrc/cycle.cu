// cycle.cu -- V-cycle and PCG kernels.
//
// Every kernel here is a streaming pass over a sparse matrix or a few
// vectors, so HBM bandwidth bounds it.  Two SpMV layouts serve all of them:
//  * vector-CSR: a group of T lanes (T = 2..32) owns a row; each lane loads
//    16-byte vectors of values and column indices (2 FP64 / 4 FP32 / 8 BF16
//    entries) read through the non-coherent path, masks the entries outside
//    its row, gathers x, and the group reduces with xor shuffles;
//  * SELL-C (C = 32, 16, 8): C-row slices stored column-major, read by one
//    warp with T = 32 / C lanes per row -- lane l takes row l % C and every
//    T-th entry from l / C -- so each warp load is one contiguous
//    128/256-byte segment whatever C; a shorter C splits long rows over more
//    lanes (shorter dependent chains per thread) and pads less.
// Reductions for PCG are deterministic: fixed grid, per-block partials, and
// the last block to arrive sums them in block order.
#include <cuda_bf16.h>

#include <cstdlib>
#include <type_traits>
#include <utility>

#include "common.cuh"
#include "cycle_ops.cuh"

namespace amg {
namespace cyc {

namespace {

// Programmatic dependent launch: the solve-path kernels go out with the
// stream-serialisation attribute, so the next kernel's blocks are scheduled
// while the current one runs (its launch latency is hidden), and every such
// kernel begins with pdl_begin(): it lets its own dependent launch, then
// waits until the kernel before it has completed and its writes are visible.
// Without the attribute (or with AMG_PDL=0) both instructions do nothing.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;\n\tgriddepcontrol.wait;" ::: "memory");
}

static bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("AMG_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
static void pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
    if (!pdl_enabled()) {
        kern<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

constexpr int kThreads = 256;


template <typename VT, typename XT> __device__ __forceinline__ XT cvt(VT v) { return (XT)v; }
template <> __device__ __forceinline__ float cvt<__nv_bfloat16, float>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// 16-byte vector loads of V consecutive entries
template <typename VT> struct Vec;
template <> struct Vec<double> {
    static constexpr int V = 2;
    __device__ __forceinline__ static void load(const double *v, const int32_t *c, int64_t q, double (&vv)[2], int32_t (&cc)[2]) {
        double2 a = __ldg(reinterpret_cast<const double2 *>(v + q));
        int2 b = __ldg(reinterpret_cast<const int2 *>(c + q));
        vv[0] = a.x; vv[1] = a.y; cc[0] = b.x; cc[1] = b.y;
    }
};
template <> struct Vec<float> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void load(const float *v, const int32_t *c, int64_t q, float (&vv)[4], int32_t (&cc)[4]) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(v + q));
        int4 b = __ldg(reinterpret_cast<const int4 *>(c + q));
        vv[0] = a.x; vv[1] = a.y; vv[2] = a.z; vv[3] = a.w;
        cc[0] = b.x; cc[1] = b.y; cc[2] = b.z; cc[3] = b.w;
    }
};
template <> struct Vec<__nv_bfloat16> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16 *v, const int32_t *c, int64_t q,
                                                __nv_bfloat16 (&vv)[8], int32_t (&cc)[8]) {
        uint4 a = __ldg(reinterpret_cast<const uint4 *>(v + q));
        int4 b0 = __ldg(reinterpret_cast<const int4 *>(c + q));
        int4 b1 = __ldg(reinterpret_cast<const int4 *>(c + q + 4));
        const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&a);
#pragma unroll
        for (int u = 0; u < 8; ++u) vv[u] = h[u];
        cc[0] = b0.x; cc[1] = b0.y; cc[2] = b0.z; cc[3] = b0.w;
        cc[4] = b1.x; cc[5] = b1.y; cc[6] = b1.z; cc[7] = b1.w;
    }
};

// sum over one CSR row by a group of T lanes (all lanes get the sum)
template <typename VT, typename XT, int T, class G>
__device__ __forceinline__ XT csr_row_sum(int32_t p0, int32_t p1, int t, const int32_t *__restrict__ ci,
                                          const VT *__restrict__ v, G gather) {
    constexpr int V = Vec<VT>::V;
    XT acc = XT(0);
    for (int32_t q = (p0 & ~(V - 1)) + t * V; q < p1; q += T * V) {
        VT vv[V];
        int32_t cc[V];
        Vec<VT>::load(v, ci, q, vv, cc);
#pragma unroll
        for (int u = 0; u < V; ++u) {
            int32_t e = q + u;
            if (e >= p0 && e < p1) acc += cvt<VT, XT>(vv[u]) * gather(cc[u]);
        }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, T);
    return acc;
}

// SELL column indices: int32 columns, or int16 offsets from the row (when
// every |column - row| of the operator fits; 2 bytes less per stored entry)
struct SellIdx {
    const int32_t *col;
    const int16_t *delta;
};
// a read-only load; CS: with the evict-first (streaming) policy, for
// operators much larger than L2 (the finest level's, always, and any whose
// stored entries pass kStreamBytes): read once per pass, they would only
// push the gathered vectors and the smaller levels out of L1 and L2
template <bool CS, typename T> __device__ __forceinline__ T ld_ro(const T *p) {
    if constexpr (CS && (std::is_same<T, double>::value || std::is_same<T, float>::value ||
                         std::is_same<T, int32_t>::value || std::is_same<T, int16_t>::value))
        return __ldcs(p);
    else
        return __ldg(p);
}
template <bool D16, bool CS = false>
__device__ __forceinline__ int32_t sell_col(const SellIdx &ix, int32_t p, int32_t row) {
    if constexpr (D16) return row + (int32_t)ld_ro<CS>(ix.delta + p);
    else return ld_ro<CS>(ix.col + p);
}

constexpr int kShortMax = 8;  // widest slice of the load-first path

// a slice of width W (W <= 8): every value and column load first, then every
// gather, then the products in k order -- short rows (interpolation P,
// coarse operators) otherwise pay a load -> gather round trip per entry
template <int W, typename VT, typename XT, bool D16, class G, bool CS = false>
__device__ __forceinline__ XT sell_short_sum(int32_t off, int32_t row, const SellIdx &ix,
                                             const VT *__restrict__ sv, G gather) {
    VT v[W];
    int32_t c[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        v[k] = ld_ro<CS>(sv + off + k * 32);
        c[k] = sell_col<D16, CS>(ix, off + k * 32, row);
    }
    XT g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = gather(c[k]);
    XT acc = XT(0);
#pragma unroll
    for (int k = 0; k < W; ++k) acc += cvt<VT, XT>(v[k]) * g[k];
    return acc;
}

// the same for the last W (< 4) entries of a lane in the SELL-C kernels,
// added into acc in k order after every load and gather is in flight
template <int W, typename VT, typename XT, bool D16, bool CS, class G>
__device__ __forceinline__ void sell_tail_acc(XT &acc, int32_t off, int32_t row, const SellIdx &ix,
                                              const VT *__restrict__ sv, G gather) {
    VT v[W];
    int32_t c[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        v[k] = ld_ro<CS>(sv + off + k * 32);
        c[k] = sell_col<D16, CS>(ix, off + k * 32, row);
    }
    XT g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = gather(c[k]);
#pragma unroll
    for (int k = 0; k < W; ++k) acc += cvt<VT, XT>(v[k]) * g[k];
}

// sum over the row stored at SELL position pos (slice pos / 32, lane pos % 32),
// entries in k order whatever the path; SHORT: slices of width <= 8 take the
// load-everything-first path (the transfer operators P and R, whose rows are
// short; the relaxation kernels measured slower with it)
template <typename VT, typename XT, bool D16, bool SHORT = false, bool CS = false, class G>
__device__ __forceinline__ XT sell_row_sum(int32_t pos, int32_t row, const int32_t *__restrict__ soff,
                                           const int32_t *__restrict__ sw, const SellIdx &ix,
                                           const VT *__restrict__ sv, G gather) {
    int32_t s = pos >> 5, lane = pos & 31;
    int32_t off = __ldg(soff + s) + lane, w = __ldg(sw + s);
    if constexpr (SHORT) {
        switch (w) {  // uniform over the warp (one slice)
            case 1: return sell_short_sum<1, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 2: return sell_short_sum<2, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 3: return sell_short_sum<3, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 4: return sell_short_sum<4, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 5: return sell_short_sum<5, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 6: return sell_short_sum<6, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 7: return sell_short_sum<7, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            case 8: return sell_short_sum<8, VT, XT, D16, G, CS>(off, row, ix, sv, gather);
            default: break;
        }
    }
    XT acc = XT(0);
#pragma unroll 4
    for (int32_t k = 0; k < w; ++k) {
        int32_t p = off + k * 32;
        acc += cvt<VT, XT>(ld_ro<CS>(sv + p)) * gather(sell_col<D16, CS>(ix, p, row));
    }
    return acc;
}

enum Op { kPre = 0, kPost = 1, kSpmv = 2, kSpmvAdd = 3, kSpmvScale = 4, kResX = 5 };

template <typename VT, typename XT, int T, int OP>
__global__ void __launch_bounds__(kThreads)
csr_op_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const VT *__restrict__ v,
              const XT *__restrict__ b, const XT *__restrict__ dinv, const XT *__restrict__ x,
              XT *__restrict__ o1, XT *__restrict__ o2) {
    pdl_begin();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t i = (int32_t)(g / T);
    int t = (int)(g % T);
    int32_t p0 = 0, p1 = 0;
    if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
    XT s;
    if (OP == kPre) s = csr_row_sum<VT, XT, T>(p0, p1, t, ci, v, [&](int32_t j) { return __ldg(b + j) * __ldg(dinv + j); });
    else s = csr_row_sum<VT, XT, T>(p0, p1, t, ci, v, [&](int32_t j) { return __ldg(x + j); });
    if (i >= n || t != 0) return;
    if (OP == kPre) {
        XT bi = b[i];
        o1[i] = bi * dinv[i];
        o2[i] = bi - s;
    } else if (OP == kPost) {
        o1[i] = x[i] + dinv[i] * (b[i] - s);
    } else if (OP == kSpmv) {
        o1[i] = s;
    } else if (OP == kSpmvScale) {
        o1[i] = s;
        o2[i] = s * dinv[i];
    } else if (OP == kResX) {
        o2[i] = b[i] - s;
    } else {
        o1[i] += s;
    }
}

// One lane per row of a SELL-32 operator; SHORT: every slice fits the
// load-first path; CS: the operator's entries load with the evict-first
// policy (CycMat::stream)
template <typename VT, typename XT, int OP, bool D16, bool SHORT, bool CS>
__global__ void __launch_bounds__(kThreads)
sell_op_kernel(int32_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ soff, const int32_t *__restrict__ sw,
               SellIdx ix, const VT *__restrict__ sv, const XT *__restrict__ b,
               const XT *__restrict__ dinv, const XT *__restrict__ x, XT *__restrict__ o1, XT *__restrict__ o2) {
    pdl_begin();
    int32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    const int32_t i = perm ? __ldg(perm + pos) : pos;
    // transfers (P, R: short rows, latency-bound): the row's own operand is
    // loaded before the row sum so its latency overlaps the gathers
    constexpr bool kTransfer = OP == kSpmvAdd || OP == kSpmvScale;
    XT own = XT(0);
    if (OP == kSpmvAdd) own = o1[i];
    if (OP == kSpmvScale) own = dinv[i];
    XT s;
    if (OP == kPre) s = sell_row_sum<VT, XT, D16, SHORT || kTransfer, CS>(pos, i, soff, sw, ix, sv, [&](int32_t j) { return __ldg(b + j) * __ldg(dinv + j); });
    else s = sell_row_sum<VT, XT, D16, SHORT || kTransfer, CS>(pos, i, soff, sw, ix, sv, [&](int32_t j) { return __ldg(x + j); });
    if (OP == kPre) {
        XT bi = b[i];
        o1[i] = bi * dinv[i];
        o2[i] = bi - s;
    } else if (OP == kPost) {
        o1[i] = x[i] + dinv[i] * (b[i] - s);
    } else if (OP == kSpmv) {
        o1[i] = s;
    } else if (OP == kSpmvScale) {
        o1[i] = s;
        o2[i] = s * own;
    } else if (OP == kResX) {
        o2[i] = b[i] - s;
    } else {
        o1[i] = own + s;
    }
}

// ---------------------------------------------------------------------------
// Row-partitioned execution (amg_partition): before each product every block
// gathers its ghost values from the global vector -- the exchange that a
// distributed run performs by messages -- then the same CSR kernels run with
// a gather that reads owned columns from the block's slice of the vector and
// ghosts from its part of the ghost buffer.  The loops, grids and sums are the
// unpartitioned kernels', so the results are the same bits.
// ---------------------------------------------------------------------------
__global__ void part_exchange_kernel(int64_t nghost, const int32_t *__restrict__ gcol, const double *__restrict__ src,
                                     const double *__restrict__ scale, double *__restrict__ gbuf) {
    pdl_begin();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nghost) return;
    const int32_t j = __ldg(gcol + k);
    gbuf[k] = scale ? __ldg(src + j) * __ldg(scale + j) : __ldg(src + j);
}

// block of row i (rows past the end, which gather nothing, get block 0)
__device__ __forceinline__ int part_of(const PartView &pv, int32_t i) {
    int p = 0;
    while (p + 1 < pv.parts && __ldg(pv.row0 + p + 1) <= i) ++p;
    return p;
}

// where row i's gathers read: owned columns from src + col0[p] (times
// scale + col0[p] when given), ghosts from gbuf + goff[p]
struct PartRow {
    const double *xl, *dl, *g;
    int32_t nloc;
};
__device__ __forceinline__ PartRow part_row(const PartView &pv, int32_t i, int32_t n, const double *src,
                                            const double *scale) {
    const int p = i < n ? part_of(pv, i) : 0;
    const int32_t c0 = __ldg(pv.col0 + p);
    return PartRow{src + c0, scale ? scale + c0 : nullptr, pv.gbuf + __ldg(pv.goff + p), __ldg(pv.col0 + p + 1) - c0};
}

template <int T, int OP>
__global__ void __launch_bounds__(kThreads)
part_op_kernel(int32_t n, const int32_t *__restrict__ rp, PartView pv, const double *__restrict__ v,
               const double *__restrict__ b, const double *__restrict__ dinv, const double *__restrict__ x,
               double *__restrict__ o1, double *__restrict__ o2) {
    pdl_begin();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t i = (int32_t)(g / T);
    int t = (int)(g % T);
    int32_t p0 = 0, p1 = 0;
    if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
    double s;
    if (OP == kPre) {
        const PartRow pr = part_row(pv, i, n, b, dinv);
        s = csr_row_sum<double, double, T>(p0, p1, t, pv.cext, v, [&](int32_t c) {
            return c < pr.nloc ? __ldg(pr.xl + c) * __ldg(pr.dl + c) : __ldg(pr.g + (c - pr.nloc));
        });
    } else {
        const PartRow pr = part_row(pv, i, n, x, nullptr);
        s = csr_row_sum<double, double, T>(p0, p1, t, pv.cext, v, [&](int32_t c) {
            return c < pr.nloc ? __ldg(pr.xl + c) : __ldg(pr.g + (c - pr.nloc));
        });
    }
    if (i >= n || t != 0) return;
    if (OP == kPre) {
        double bi = b[i];
        o1[i] = bi * dinv[i];
        o2[i] = bi - s;
    } else if (OP == kPost) {
        o1[i] = x[i] + dinv[i] * (b[i] - s);
    } else if (OP == kSpmv) {
        o1[i] = s;
    } else if (OP == kSpmvScale) {
        o1[i] = s;
        o2[i] = s * dinv[i];
    } else if (OP == kResX) {
        o2[i] = b[i] - s;
    } else {
        o1[i] += s;
    }
}

// the exchange for an operator whose products gather src (times scale)
void part_exchange(const PartView &pv, const double *src, const double *scale, cudaStream_t s) {
    if (pv.nghost == 0) return;
    { pdl_launch(part_exchange_kernel, (int)div_up(pv.nghost, (int64_t)kThreads), kThreads, 0, s, pv.nghost, pv.gcol, src, scale, pv.gbuf); ::amg::count_launch(); }
}

template <int OP>
void part_op(const CycMat<double> &A, const double *b, const double *dinv, const double *x, double *o1, double *o2,
             cudaStream_t s) {
    const int32_t n = A.nrows;
    if (OP == kPre) part_exchange(A.part, b, dinv, s);
    else part_exchange(A.part, x, nullptr, s);
    // one lane per row: the order of the unpartitioned one-lane kernels
    { pdl_launch(part_op_kernel<1, OP>, (int)div_up((int64_t)n, (int64_t)kThreads), kThreads, 0, s, n, A.rp, A.part, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

// SELL-C with C < 32: one warp per slice of C rows, T = 32 / C lanes per
// row.  Lane l holds row l % C and the entries k = l / C, l / C + T, ... (the
// slice width is a multiple of T); its part of the row is loaded U entries
// at a time -- all values and columns, then all gathers, then the products
// -- and the T parts are added by xor shuffles.  The row's sum therefore
// runs in another order than a sequential one (not bit-equal to CSR).
// CS: the operator's entries load with the evict-first policy.
template <typename VT, typename XT, int OP, bool D16, int C, bool CS>
__global__ void __launch_bounds__(kThreads)
sell_lanes_op_kernel(int32_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ soff,
                     const int32_t *__restrict__ sw, SellIdx ix, const VT *__restrict__ sv, const XT *__restrict__ b,
                     const XT *__restrict__ dinv, const XT *__restrict__ x, XT *__restrict__ o1, XT *__restrict__ o2) {
    pdl_begin();
    constexpr int T = 32 / C, U = 4;
    const int32_t slice = (int32_t)(((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31, r = lane % C, t = lane / C;
    if (slice * C >= n) return;  // whole warp: slices are warp-uniform
    const int32_t pos = slice * C + r;
    const bool valid = pos < n;
    const int32_t i = valid ? (perm ? __ldg(perm + pos) : pos) : 0;
    const int32_t off = __ldg(soff + slice) + lane, w = __ldg(sw + slice);
    auto gather = [&](int32_t j) {
        if (OP == kPre) return __ldg(b + j) * __ldg(dinv + j);
        return __ldg(x + j);
    };
    XT acc = XT(0);
    if (valid) {
        const int32_t nk = w / T;  // entries of this lane
        int32_t k = 0;
        if ((OP == kSpmvAdd || OP == kSpmvScale) && nk <= kShortMax) {
            // transfers: a lane's part of a row is short, so all of it loads
            // first (nk is the same for the whole warp), rather than one
            // load -> gather round trip per entry in the tail loop
            switch (nk) {
                case 1: acc = sell_short_sum<1, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 2: acc = sell_short_sum<2, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 3: acc = sell_short_sum<3, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 4: acc = sell_short_sum<4, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 5: acc = sell_short_sum<5, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 6: acc = sell_short_sum<6, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 7: acc = sell_short_sum<7, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                case 8: acc = sell_short_sum<8, VT, XT, D16, decltype(gather), CS>(off, i, ix, sv, gather); break;
                default: break;
            }
            k = nk;
        }
        for (; k + U <= nk; k += U) {
            VT v[U];
            int32_t c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t p = off + (k + u) * 32;
                v[u] = ld_ro<CS>(sv + p);
                c[u] = sell_col<D16, CS>(ix, p, i);
            }
            XT g[U];
#pragma unroll
            for (int u = 0; u < U; ++u) g[u] = gather(c[u]);
#pragma unroll
            for (int u = 0; u < U; ++u) acc += cvt<VT, XT>(v[u]) * g[u];
        }
        // the last nk - k < U entries, loaded together (a warp-uniform count)
        switch (nk - k) {
            case 1: sell_tail_acc<1, VT, XT, D16, CS>(acc, off + k * 32, i, ix, sv, gather); break;
            case 2: sell_tail_acc<2, VT, XT, D16, CS>(acc, off + k * 32, i, ix, sv, gather); break;
            case 3: sell_tail_acc<3, VT, XT, D16, CS>(acc, off + k * 32, i, ix, sv, gather); break;
            default: break;
        }
    }
#pragma unroll
    for (int o = 16; o >= C; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!valid || t != 0) return;
    const XT sum = acc;
    if (OP == kPre) {
        XT bi = b[i];
        o1[i] = bi * dinv[i];
        o2[i] = bi - sum;
    } else if (OP == kPost) {
        o1[i] = x[i] + dinv[i] * (b[i] - sum);
    } else if (OP == kSpmv) {
        o1[i] = sum;
    } else if (OP == kSpmvScale) {
        o1[i] = sum;
        o2[i] = sum * dinv[i];
    } else if (OP == kResX) {
        o2[i] = b[i] - sum;
    } else {
        o1[i] += sum;
    }
}

template <typename VT, typename XT, int OP, int C>
void launch_sell_lanes(const CycMat<VT> &A, const XT *b, const XT *dinv, const XT *x, XT *o1, XT *o2,
                       cudaStream_t s) {
    const int32_t n = A.nrows;
    const SellIdx ix{A.sci, A.sd};
    const int64_t warps = div_up((int64_t)n, (int64_t)C);
    const int g = (int)div_up(warps * 32, (int64_t)kThreads);
    auto launch = [&](auto cs) {
        constexpr bool CS = decltype(cs)::value;
        if (A.sd)
            { pdl_launch(sell_lanes_op_kernel<VT, XT, OP, true, C, CS>, g, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, b, dinv, x, o1, o2); ::amg::count_launch(); }
        else
            { pdl_launch(sell_lanes_op_kernel<VT, XT, OP, false, C, CS>, g, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, b, dinv, x, o1, o2); ::amg::count_launch(); }
    };
    if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
        if (A.stream) launch(std::true_type());
        else launch(std::false_type());
    } else {
        launch(std::false_type());
    }
}

template <typename VT, typename XT, int OP>
void dispatch_op(const CycMat<VT> &A, const XT *b, const XT *dinv, const XT *x, XT *o1, XT *o2, cudaStream_t s) {
    int32_t n = A.nrows;
    if (n == 0) return;
    if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
        if (A.part.parts) {
            part_op<OP>(A, b, dinv, x, o1, o2, s);
            return;
        }
    }
    if ((A.variant == AMG_SPMV_SELL16 || A.variant == AMG_SPMV_SELL8) && A.sv && A.sell_c == sell_height(A.variant)) {
        if (A.sell_c == 16) launch_sell_lanes<VT, XT, OP, 16>(A, b, dinv, x, o1, o2, s);
        else launch_sell_lanes<VT, XT, OP, 8>(A, b, dinv, x, o1, o2, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    if (A.variant == AMG_SPMV_SELL32 && A.sv && A.sell_c == 32) {
        const SellIdx ix{A.sci, A.sd};
        // the load-first path for operators whose rows all fit it (measured:
        // faster at level 0, slower on the longer, irregular coarse rows)
        const bool sh = A.max_row > 0 && A.max_row <= kShortMax;
        const int g = div_up(n, kThreads);
        auto launch = [&](auto cs) {
            constexpr bool CS = decltype(cs)::value;
            if (A.sd && sh)
                { pdl_launch(sell_op_kernel<VT, XT, OP, true, true, CS>, g, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, b, dinv, x, o1, o2); ::amg::count_launch(); }
            else if (A.sd)
                { pdl_launch(sell_op_kernel<VT, XT, OP, true, false, CS>, g, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, b, dinv, x, o1, o2); ::amg::count_launch(); }
            else if (sh)
                { pdl_launch(sell_op_kernel<VT, XT, OP, false, true, CS>, g, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, b, dinv, x, o1, o2); ::amg::count_launch(); }
            else
                { pdl_launch(sell_op_kernel<VT, XT, OP, false, false, CS>, g, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, b, dinv, x, o1, o2); ::amg::count_launch(); }
        };
        // the streaming loads only in FP64 (the reduced-precision copies are half the size or less)
        if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
            if (A.stream) launch(std::true_type());
            else launch(std::false_type());
        } else {
            launch(std::false_type());
        }
    } else {
        int T = threads_per_row(A.variant);
        int blocks = div_up((int64_t)n * T, kThreads);
        switch (T) {
            case 1: { pdl_launch(csr_op_kernel<VT, XT, 1, OP>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); } break;
            case 2: { pdl_launch(csr_op_kernel<VT, XT, 2, OP>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); } break;
            case 4: { pdl_launch(csr_op_kernel<VT, XT, 4, OP>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); } break;
            case 8: { pdl_launch(csr_op_kernel<VT, XT, 8, OP>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); } break;
            case 16: { pdl_launch(csr_op_kernel<VT, XT, 16, OP>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); } break;
            default: { pdl_launch(csr_op_kernel<VT, XT, 32, OP>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, b, dinv, x, o1, o2); ::amg::count_launch(); } break;
        }
    }
    AMG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// deterministic block reduction with last-block finish
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
    __shared__ double sh[NV][kThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
    __syncthreads();
}

// Block partials without a block-wide barrier at the end: each warp reduces
// its values with shuffles and parks them in shared memory; the last warp of
// the block to arrive (a shared arrival counter, zeroed when the kernel
// starts) adds the warp values in warp order and stores the block partial.
// Warps that finish early leave at once instead of waiting for the block's
// slowest gathers.  A one-block finisher kernel launched next sums the block
// partials in block order: no atomics on floating-point values, no fences on
// the producers' critical path, a deterministic result.
__device__ __forceinline__ unsigned *arrival_counter() {
    __shared__ unsigned c;
    return &c;
}

// every kernel that calls block_partials calls this first (all threads)
__device__ __forceinline__ void block_partials_begin() {
    if (threadIdx.x == 0) *arrival_counter() = 0u;
    __syncthreads();
}

template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], Reduce red) {
    __shared__ double sh[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double x[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        x[k] = v[k];
        for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_xor_sync(0xffffffffu, x[k], o);
    }
    if (lane != 0) return;
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = x[k];
    __threadfence_block();
    const unsigned nw = blockDim.x >> 5;
    if (atomicAdd(arrival_counter(), 1u) != nw - 1) return;
    __threadfence_block();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = 0.0;
        for (unsigned i = 0; i < nw; ++i) t += ((volatile double *)sh[k])[i];
        red.partials[k * kMaxReduceBlocks + blockIdx.x] = t;
    }
}

enum Fin { kFinAp = 0, kFinXr = 1, kFinRz = 2, kFinTt = 3 };

constexpr int kFinThreads = 1024;

// finish of r.z / z.q: beta and rho (start: beta = 0)
__device__ __forceinline__ void finish_rz(PcgScalars *sc, double rz, double zq) {
    if (!sc->start) {
        sc->zq = zq;
        sc->beta = sc->flexible ? (-sc->alpha * zq) / sc->rho : rz / sc->rho;
    } else {
        sc->beta = 0.0;
    }
    sc->rho = rz;
    sc->start = 0;
}

template <int NV, int FIN>
__global__ void __launch_bounds__(kFinThreads)
finish_kernel(int nblocks, Reduce red, PcgScalars *sc, cudaGraphConditionalHandle handle, int use_handle) {
    pdl_begin();
    __shared__ double sh[NV][kFinThreads / 32];
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = 0.0;
#pragma unroll 8
    for (int b = threadIdx.x; b < nblocks; b += kFinThreads) {
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] += red.partials[k * kMaxReduceBlocks + b];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = t[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (w != 0) return;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = sh[k][lane];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        t[k] = x;
    }
    if (lane != 0) return;
    if (FIN == kFinAp) {
        sc->pq = t[0];
        bool ok = t[0] > 0.0 && sc->rho > 0.0;
        if (!ok) sc->breakdown = 1;
        sc->alpha = ok ? sc->rho / t[0] : 0.0;
    } else if (FIN == kFinXr) {
        sc->rr = t[0];
        int its = sc->its + 1;
        sc->its = its;
        if (sc->divf > 0.0 && !sc->breakdown) {
            // the window test, in the oracle's form: norms, not squares
            const double rn = sqrt(t[0]);
            const bool end = its % sc->kwin == 0;
            if (!isfinite(rn) || (end && rn > sc->divf * sc->rn_ws)) sc->diverged = 1;
            else if (end) sc->rn_ws = rn;
        }
        if (use_handle) {
            bool go = t[0] > sc->thresh2 && its < sc->max_its && !sc->breakdown && !sc->diverged && isfinite(t[0]);
            cudaGraphSetConditional(handle, go ? 1u : 0u);
        }
    } else if (FIN == kFinRz) {
        finish_rz(sc, t[0], NV > 1 ? t[NV - 1] : 0.0);
    } else {
        sc->tt = t[0];
    }
}

template <int NV, int FIN>
void launch_finish(int nblocks, Reduce red, PcgScalars *sc, cudaStream_t s,
                   cudaGraphConditionalHandle handle = cudaGraphConditionalHandle{}, bool use_handle = false) {
    { pdl_launch(finish_kernel<NV, FIN>, 1, kFinThreads, 0, s, nblocks, red, sc, handle, use_handle ? 1 : 0); ::amg::count_launch(); }
}

// Grid of a reducing kernel: at most one resident wave, so every thread
// loops over several rows and the shuffle tree of the block reduction (FP64
// adds, the scarce pipe on this part) runs once per thread, not once per row.
int reduce_blocks(int64_t threads_needed) {
    int64_t b = (threads_needed + kThreads - 1) / kThreads;
    int64_t cap = ::amg::resident_blocks(kThreads);
    if (b > cap) b = cap;
    if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
    if (b < 1) b = 1;
    return (int)b;
}
static_assert(kThreads == 256, "two-level reduction assumes groups of 256 blocks and 256 threads");

// ---------------------------------------------------------------------------
// PCG kernels (FP64)
// ---------------------------------------------------------------------------
__global__ void p_update_kernel(int32_t n, const double *__restrict__ z, double *__restrict__ p,
                                const PcgScalars *sc) {
    pdl_begin();
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = z[i] + sc->beta * p[i];
}

// q = A p (SELL-32, one thread per row) and p . q; each warp walks slices
// with a stride of the grid's warp count.  RESID: q = b - A p and q . q (the
// true residual of p = x)
template <bool D16, bool SHORT, bool RESID>
__global__ void __launch_bounds__(kThreads)
ap_sell_kernel(int32_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ soff, const int32_t *__restrict__ sw,
               SellIdx ix, const double *__restrict__ sv, const double *__restrict__ p, const double *__restrict__ b,
               double *__restrict__ q, PcgScalars *sc, Reduce red) {
    pdl_begin();
    block_partials_begin();
    double part[1] = {0.0};
    const int lane = threadIdx.x & 31;
    const int32_t nsl = (n + 31) >> 5, nwarps = (int32_t)((gridDim.x * kThreads) >> 5);
    for (int32_t sl = (int32_t)((blockIdx.x * kThreads + threadIdx.x) >> 5); sl < nsl; sl += nwarps) {
        const int32_t pos = sl * 32 + lane;
        if (pos >= n) continue;
        const int32_t i = perm ? __ldg(perm + pos) : pos;
        double s = sell_row_sum<double, double, D16, SHORT, true>(pos, i, soff, sw, ix, sv, [&](int32_t j) { return __ldg(p + j); });
        if (RESID) {
            const double e = b[i] - s;
            q[i] = e;
            part[0] += e * e;
        } else {
            q[i] = s;
            part[0] += p[i] * s;
        }
    }
    block_partials<1>(part, red);
}

// q = A p (vector-CSR, T lanes per row) and p . q
template <int T, bool PART = false>
__global__ void __launch_bounds__(kThreads)
ap_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
          const double *__restrict__ p, double *__restrict__ q, PcgScalars *sc, Reduce red, PartView pv = PartView()) {
    pdl_begin();
    block_partials_begin();
    double part[1] = {0.0};
    int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < (int64_t)((n + (kThreads / T) - 1) / (kThreads / T)) * (kThreads / T) * T; g += stride) {
        int32_t i = (int32_t)(g / T);
        int t = (int)(g % T);
        int32_t p0 = 0, p1 = 0;
        if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
        double s;
        if constexpr (PART) {  // ci: block-local columns
            const PartRow pr = part_row(pv, i, n, p, nullptr);
            s = csr_row_sum<double, double, T>(p0, p1, t, ci, v, [&](int32_t c) {
                return c < pr.nloc ? __ldg(pr.xl + c) : __ldg(pr.g + (c - pr.nloc));
            });
        } else {
            s = csr_row_sum<double, double, T>(p0, p1, t, ci, v, [&](int32_t j) { return __ldg(p + j); });
        }
        if (i < n && t == 0) {
            q[i] = s;
            part[0] += p[i] * s;
        }
    }
    block_partials<1>(part, red);
}

__global__ void __launch_bounds__(kThreads)
xr_update_kernel(int32_t n, const double *__restrict__ p, const double *__restrict__ q, double *__restrict__ x,
                 double *__restrict__ r, const PcgScalars *sc, Reduce red, const double *__restrict__ dinv0,
                 double *__restrict__ x0, double *__restrict__ xs) {
    pdl_begin();
    block_partials_begin();
    const double alpha = sc->alpha;
    const bool step = alpha != 0.0;  // 0: breakdown -- x and r stay as they are
    // this step starts a divergence-test window: keep x as it was
    const bool ckpt = xs != nullptr && sc->divf > 0.0 && sc->its % sc->kwin == 0;
    double part[1] = {0.0};
    for (int32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        double ri = r[i];
        if (ckpt) xs[i] = x[i];
        if (step) {
            x[i] += alpha * p[i];
            ri -= alpha * q[i];
            r[i] = ri;
        }
        if (x0) x0[i] = ri * dinv0[i];  // the next cycle's level-0 pre-smooth from zero
        part[0] += ri * ri;
    }
    block_partials<1>(part, red);
}

__global__ void __launch_bounds__(kThreads)
rz_kernel(int32_t n, const double *__restrict__ r, const double *__restrict__ z, const double *__restrict__ q,
          PcgScalars *sc, Reduce red) {
    pdl_begin();
    block_partials_begin();
    int first = sc->start;
    double part[2] = {0.0, 0.0};
    for (int32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        double zi = z[i];
        part[0] += r[i] * zi;
        if (!first) part[1] += zi * q[i];
    }
    block_partials<2>(part, red);
}

template <int T, bool PART = false>
__global__ void __launch_bounds__(kThreads)
resid_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
             const double *__restrict__ b, const double *__restrict__ x, double *__restrict__ t_out,
             PcgScalars *sc, Reduce red, PartView pv = PartView()) {
    pdl_begin();
    block_partials_begin();
    double part[1] = {0.0};
    int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < (int64_t)((n + (kThreads / T) - 1) / (kThreads / T)) * (kThreads / T) * T; g += stride) {
        int32_t i = (int32_t)(g / T);
        int t = (int)(g % T);
        int32_t p0 = 0, p1 = 0;
        if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
        double s;
        if constexpr (PART) {
            const PartRow pr = part_row(pv, i, n, x, nullptr);
            s = csr_row_sum<double, double, T>(p0, p1, t, ci, v, [&](int32_t c) {
                return c < pr.nloc ? __ldg(pr.xl + c) : __ldg(pr.g + (c - pr.nloc));
            });
        } else {
            s = csr_row_sum<double, double, T>(p0, p1, t, ci, v, [&](int32_t j) { return __ldg(x + j); });
        }
        if (i < n && t == 0) {
            double e = b[i] - s;
            t_out[i] = e;
            part[0] += e * e;
        }
    }
    block_partials<1>(part, red);
}

// level-0 post-smoothing z = x + d (b - A x) with r.z (r = b) and, for
// flexible CG only (ZQ), z.q -- plain CG's beta needs no z.q, so the FP64
// cycle reads no q and issues one FMA less per row
template <int T, bool ZQ, bool PART = false>
__global__ void __launch_bounds__(kThreads)
post_rz_csr_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
                   const double *__restrict__ x, const double *__restrict__ b, const double *__restrict__ dinv,
                   double *__restrict__ z, const double *__restrict__ q, PcgScalars *sc, Reduce red,
                   PartView pv = PartView()) {
    pdl_begin();
    block_partials_begin();
    double part[ZQ ? 2 : 1];
#pragma unroll
    for (int k = 0; k < (ZQ ? 2 : 1); ++k) part[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t gend = (int64_t)((n + (kThreads / T) - 1) / (kThreads / T)) * (kThreads / T) * T;
    for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < gend; g += stride) {
        const int32_t i = (int32_t)(g / T);
        const int t = (int)(g % T);
        int32_t p0 = 0, p1 = 0;
        if (i < n) { p0 = __ldg(rp + i); p1 = __ldg(rp + i + 1); }
        double s;
        if constexpr (PART) {
            const PartRow pr = part_row(pv, i, n, x, nullptr);
            s = csr_row_sum<double, double, T>(p0, p1, t, ci, v, [&](int32_t c) {
                return c < pr.nloc ? __ldg(pr.xl + c) : __ldg(pr.g + (c - pr.nloc));
            });
        } else {
            s = csr_row_sum<double, double, T>(p0, p1, t, ci, v, [&](int32_t j) { return __ldg(x + j); });
        }
        if (i < n && t == 0) {
            double bi = b[i];
            double zi = x[i] + dinv[i] * (bi - s);
            z[i] = zi;
            part[0] += bi * zi;
            if (ZQ) part[ZQ ? 1 : 0] += zi * q[i];
        }
    }
    block_partials<ZQ ? 2 : 1>(part, red);
}

template <bool D16, bool ZQ>
__global__ void __launch_bounds__(kThreads)
post_rz_sell_kernel(int32_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ soff,
                    const int32_t *__restrict__ sw, SellIdx ix, const double *__restrict__ sv,
                    const double *__restrict__ x, const double *__restrict__ b, const double *__restrict__ dinv,
                    double *__restrict__ z, const double *__restrict__ q, PcgScalars *sc, Reduce red) {
    pdl_begin();
    block_partials_begin();
    double part[ZQ ? 2 : 1];
#pragma unroll
    for (int k = 0; k < (ZQ ? 2 : 1); ++k) part[k] = 0.0;
    const int lane = threadIdx.x & 31;
    const int32_t nsl = (n + 31) >> 5, nwarps = (int32_t)((gridDim.x * kThreads) >> 5);
    for (int32_t sl = (int32_t)((blockIdx.x * kThreads + threadIdx.x) >> 5); sl < nsl; sl += nwarps) {
        const int32_t pos = sl * 32 + lane;
        if (pos >= n) continue;
        const int32_t i = perm ? __ldg(perm + pos) : pos;
        double s = sell_row_sum<double, double, D16, false, true>(pos, i, soff, sw, ix, sv, [&](int32_t j) { return __ldg(x + j); });
        double bi = b[i];
        double zi = x[i] + dinv[i] * (bi - s);
        z[i] = zi;
        part[0] += bi * zi;
        if (ZQ) part[ZQ ? 1 : 0] += zi * q[i];
    }
    block_partials<ZQ ? 2 : 1>(part, red);
}

__global__ void __launch_bounds__(kThreads)
to_f64_rz_kernel(int32_t n, const float *__restrict__ z32, double *__restrict__ z, const double *__restrict__ r,
                 const double *__restrict__ q, PcgScalars *sc, Reduce red) {
    pdl_begin();
    block_partials_begin();
    double part[2] = {0.0, 0.0};
    for (int32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        double zi = (double)z32[i];
        z[i] = zi;
        part[0] += r[i] * zi;
        part[1] += zi * q[i];
    }
    block_partials<2>(part, red);
}

template <typename XT>
__global__ void scale_kernel(int64_t n, const XT *__restrict__ a, const XT *__restrict__ d, XT *__restrict__ out) {
    pdl_begin();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * d[i];
}

__global__ void to_f32_scaled_kernel(int64_t n, const double *__restrict__ src, const float *__restrict__ d,
                                     float *__restrict__ dst, float *__restrict__ xdst) {
    pdl_begin();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = (float)src[i];
    dst[i] = v;
    xdst[i] = v * d[i];
}

// ---------------------------------------------------------------------------
// coarse solve: x = inv b, one warp per row
// ---------------------------------------------------------------------------
template <typename XT>
__global__ void coarse_kernel(int32_t n, const double *__restrict__ inv, const XT *__restrict__ b, XT *__restrict__ x) {
    pdl_begin();
    int lane = threadIdx.x & 31;
    int32_t row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (row >= n) return;
    double s = 0.0;
    for (int32_t j = lane; j < n; j += 32) s += inv[(size_t)row * n + j] * (double)b[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = (XT)s;
}

// ---------------------------------------------------------------------------
// conversions and SELL construction
// ---------------------------------------------------------------------------
template <typename VT>
__global__ void convert_kernel(const double *src, VT *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (VT)src[i];
}
template <>
__global__ void convert_kernel<__nv_bfloat16>(const double *src, __nv_bfloat16 *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __double2bfloat16(src[i]);
}

template <typename XT>
__global__ void to_f64_kernel(const XT *src, double *dst, int64_t n) {
    pdl_begin();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// rows sorted by length (descending, then index) inside windows of
// kSellSigma rows: one block sorts one window with a bitonic network
__global__ void __launch_bounds__(512) sell_sort_kernel(int32_t n, const int32_t *rp, int32_t *perm) {
    __shared__ unsigned long long key[kSellSigma];
    int32_t w0 = blockIdx.x * kSellSigma;
    for (int t = threadIdx.x; t < kSellSigma; t += blockDim.x) {
        int32_t i = w0 + t;
        key[t] = i < n ? ((unsigned long long)(0x7fffffff - (rp[i + 1] - rp[i])) << 32) | (unsigned)i : ~0ull;
    }
    __syncthreads();
    for (int size = 2; size <= kSellSigma; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kSellSigma; t += blockDim.x) {
                int partner = t ^ stride;
                if (partner > t) {
                    bool up = (t & size) == 0;
                    unsigned long long a = key[t], c = key[partner];
                    if ((a > c) == up) { key[t] = c; key[partner] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < kSellSigma; t += blockDim.x) {
        int32_t i = w0 + t;
        if (i < n) perm[i] = (int32_t)(key[t] & 0xffffffffu);
    }
}

// width of each slice of C rows: its longest row, rounded up to a multiple
// of the 32 / C lanes that share a row
__global__ void slice_width_kernel(int32_t n, const int32_t *rp, const int32_t *perm, int32_t *sw, int C) {
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t nsl = (n + C - 1) / C;
    if (s >= nsl) return;
    int32_t w = 0;
    for (int32_t pos = s * C; pos < min(n, s * C + C); ++pos) {
        int32_t i = perm ? perm[pos] : pos;
        w = max(w, rp[i + 1] - rp[i]);
    }
    const int32_t T = 32 / C;
    sw[s] = (w + T - 1) / T * T;
}

__global__ void slice_size_kernel(int32_t nsl, const int32_t *sw, int32_t *sz, int C) {
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsl) sz[s] = sw[s] * C;
}

template <typename VT>
__global__ void sell_fill_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const VT *v, const int32_t *perm,
                                 const int32_t *soff, const int32_t *sw, int32_t *sci, VT *sv, int16_t *sd, int C) {
    int32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t nsl = (n + C - 1) / C;
    if (pos >= nsl * C) return;
    int32_t s = pos / C, lane = pos % C;
    int32_t off = soff[s] + lane, w = sw[s];
    int32_t i = pos < n ? (perm ? perm[pos] : pos) : -1;
    int32_t p0 = i >= 0 ? rp[i] : 0, len = i >= 0 ? rp[i + 1] - p0 : 0;
    // padding: value 0 at a column the row itself holds (its last one), or
    // column 0 for an empty row -- always inside x, also for rectangular
    // operators (P is n x n_c); with int16 offsets an empty row pads with
    // its own index (offset 0; those operators are square)
    const int32_t pad_col = len > 0 ? ci[p0 + len - 1] : (sd ? (i >= 0 ? i : 0) : 0);
    for (int32_t k = 0; k < w; ++k) {
        int32_t p = off + k * C;
        const int32_t c = k < len ? ci[p0 + k] : pad_col;
        if (sd) sd[p] = (int16_t)(i >= 0 ? c - i : 0);
        else sci[p] = c;
        sv[p] = k < len ? v[p0 + k] : VT(0);
    }
}

// out[0] = max |column - row|, out[1] = max stored entries of a row
__global__ void max_col_offset_kernel(int32_t n, const int32_t *rp, const int32_t *ci, int *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int m = 0, len = 0;
    if (i < n) {
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) m = max(m, abs(ci[p] - i));
        len = rp[i + 1] - rp[i];
    }
    m = __reduce_max_sync(0xffffffffu, (unsigned)m);
    len = __reduce_max_sync(0xffffffffu, (unsigned)len);
    // one atomic per block: atomics of every warp on one address serialise
    __shared__ int sm[kThreads / 32], sl[kThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sm[w] = m; sl[w] = len; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { m = max(m, sm[k]); len = max(len, sl[k]); }
        if (m) atomicMax(out, m);
        if (len) atomicMax(out + 1, len);
    }
}

}  // namespace

int threads_per_row(int variant) {
    switch (variant) {
        case AMG_SPMV_CSR1: return 1;
        case AMG_SPMV_CSR2: return 2;
        case AMG_SPMV_CSR4: return 4;
        case AMG_SPMV_CSR8: return 8;
        case AMG_SPMV_CSR16: return 16;
        case AMG_SPMV_CSR32: return 32;
        default: return 4;
    }
}

template <typename VT, typename XT>
void pre_smooth_residual(const CycMat<VT> &A, const XT *b, const XT *dinv, XT *x, XT *r, cudaStream_t s) {
    dispatch_op<VT, XT, kPre>(A, b, dinv, nullptr, x, r, s);
}
template <typename VT, typename XT>
void post_smooth(const CycMat<VT> &A, const XT *x, const XT *b, const XT *dinv, XT *xo, cudaStream_t s) {
    dispatch_op<VT, XT, kPost>(A, b, dinv, x, xo, nullptr, s);
}
template <typename VT, typename XT>
void spmv(const CycMat<VT> &A, const XT *x, XT *y, bool accumulate, cudaStream_t s) {
    if (accumulate) dispatch_op<VT, XT, kSpmvAdd>(A, nullptr, nullptr, x, y, nullptr, s);
    else dispatch_op<VT, XT, kSpmv>(A, nullptr, nullptr, x, y, nullptr, s);
}
template <typename VT, typename XT>
void spmv_scaled(const CycMat<VT> &A, const XT *x, const XT *d, XT *y, XT *xs, cudaStream_t s) {
    dispatch_op<VT, XT, kSpmvScale>(A, nullptr, d, x, y, xs, s);
}
template <typename VT, typename XT>
void residual_from_x(const CycMat<VT> &A, const XT *b, const XT *x, XT *r, cudaStream_t s) {
    dispatch_op<VT, XT, kResX>(A, b, nullptr, x, nullptr, r, s);
}

template <typename XT>
void coarse_solve(int32_t n, const double *inv, const XT *b, XT *x, cudaStream_t s) {
    if (n == 0) return;
    { pdl_launch(coarse_kernel<XT>, div_up(n, 8), 256, 0, s, n, inv, b, x); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void pcg_p_update(int32_t n, const double *z, double *p, const PcgScalars *sc, cudaStream_t s) {
    { pdl_launch(p_update_kernel, div_up(n, kThreads), kThreads, 0, s, n, z, p, sc); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

template <int T>
static void launch_ap(const CycMat<double> &A, const double *p, double *q, PcgScalars *sc, Reduce red, cudaStream_t s) {
    int blocks = reduce_blocks((int64_t)A.nrows * T);
    { pdl_launch(ap_kernel<T>, blocks, kThreads, 0, s, A.nrows, A.rp, A.ci, A.v, p, q, sc, red, PartView()); ::amg::count_launch(); }
    launch_finish<1, kFinAp>(blocks, red, sc, s);
}

// the SELL forms of A p and of the true residual; returns the block count
template <bool RESID>
static int launch_ap_sell(const CycMat<double> &A, const double *p, const double *b, double *q, PcgScalars *sc,
                          Reduce red, cudaStream_t s) {
    const int blocks = reduce_blocks(A.nrows);
    const SellIdx ix{A.sci, A.sd};
    const bool sh = A.max_row > 0 && A.max_row <= kShortMax;
    if (A.sd && sh)
        { pdl_launch(ap_sell_kernel<true, true, RESID>, blocks, kThreads, 0, s, A.nrows, A.perm, A.soff, A.sw, ix, A.sv, p, b, q, sc, red); ::amg::count_launch(); }
    else if (A.sd)
        { pdl_launch(ap_sell_kernel<true, false, RESID>, blocks, kThreads, 0, s, A.nrows, A.perm, A.soff, A.sw, ix, A.sv, p, b, q, sc, red); ::amg::count_launch(); }
    else if (sh)
        { pdl_launch(ap_sell_kernel<false, true, RESID>, blocks, kThreads, 0, s, A.nrows, A.perm, A.soff, A.sw, ix, A.sv, p, b, q, sc, red); ::amg::count_launch(); }
    else
        { pdl_launch(ap_sell_kernel<false, false, RESID>, blocks, kThreads, 0, s, A.nrows, A.perm, A.soff, A.sw, ix, A.sv, p, b, q, sc, red); ::amg::count_launch(); }
    return blocks;
}

void pcg_ap(const CycMat<double> &A, const double *p, double *q, PcgScalars *sc, Reduce red, cudaStream_t s) {
    if (A.part.parts) {  // row-partitioned: exchange, then the one-lane kernel's loop
        part_exchange(A.part, p, nullptr, s);
        const int blocks = reduce_blocks(A.nrows);
        { pdl_launch(ap_kernel<1, true>, blocks, kThreads, 0, s, A.nrows, A.rp, A.part.cext, A.v, p, q, sc, red, A.part); ::amg::count_launch(); }
        launch_finish<1, kFinAp>(blocks, red, sc, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    if (A.variant == AMG_SPMV_SELL32 && A.sv && A.sell_c == 32) {
        const int blocks = launch_ap_sell<false>(A, p, nullptr, q, sc, red, s);
        launch_finish<1, kFinAp>(blocks, red, sc, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    switch (threads_per_row(A.variant == AMG_SPMV_SELL32 ? AMG_SPMV_CSR4 : A.variant)) {
        case 1: launch_ap<1>(A, p, q, sc, red, s); break;
        case 2: launch_ap<2>(A, p, q, sc, red, s); break;
        case 4: launch_ap<4>(A, p, q, sc, red, s); break;
        case 8: launch_ap<8>(A, p, q, sc, red, s); break;
        case 16: launch_ap<16>(A, p, q, sc, red, s); break;
        default: launch_ap<32>(A, p, q, sc, red, s); break;
    }
    AMG_CHECK_LAUNCH();
}

void pcg_xr_update(int32_t n, const double *p, const double *q, double *x, double *r, PcgScalars *sc,
                   Reduce red, cudaGraphConditionalHandle handle, bool use_handle, const double *dinv0,
                   double *x0, double *xs, cudaStream_t s) {
    int blocks = reduce_blocks(n);
    { pdl_launch(xr_update_kernel, blocks, kThreads, 0, s, n, p, q, x, r, sc, red, dinv0, x0, xs); ::amg::count_launch(); }
    launch_finish<1, kFinXr>(blocks, red, sc, s, handle, use_handle);
    AMG_CHECK_LAUNCH();
}

template <bool ZQ>
static void post_smooth_rz_launch(const CycMat<double> &A, const double *x, const double *b, const double *dinv,
                                  double *z, const double *q, PcgScalars *sc, Reduce red, cudaStream_t s) {
    const int32_t n = A.nrows;
    constexpr int NV = ZQ ? 2 : 1;
    if (A.part.parts) {
        part_exchange(A.part, x, nullptr, s);
        const int blocks = reduce_blocks(n);
        { pdl_launch(post_rz_csr_kernel<1, ZQ, true>, blocks, kThreads, 0, s, n, A.rp, A.part.cext, A.v, x, b, dinv, z, q, sc, red, A.part); ::amg::count_launch(); }
        launch_finish<NV, kFinRz>(blocks, red, sc, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    if (A.variant == AMG_SPMV_SELL32 && A.sv && A.sell_c == 32) {
        int blocks = reduce_blocks(n);
        const SellIdx ix{A.sci, A.sd};
        if (A.sd)
            { pdl_launch(post_rz_sell_kernel<true, ZQ>, blocks, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, x, b, dinv, z, q, sc, red); ::amg::count_launch(); }
        else
            { pdl_launch(post_rz_sell_kernel<false, ZQ>, blocks, kThreads, 0, s, n, A.perm, A.soff, A.sw, ix, A.sv, x, b, dinv, z, q, sc, red); ::amg::count_launch(); }
        launch_finish<NV, kFinRz>(blocks, red, sc, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    int T = threads_per_row(A.variant);
    int blocks = reduce_blocks((int64_t)n * T);
    switch (T) {
        case 1: { pdl_launch(post_rz_csr_kernel<1, ZQ>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, x, b, dinv, z, q, sc, red, PartView()); ::amg::count_launch(); } break;
        case 2: { pdl_launch(post_rz_csr_kernel<2, ZQ>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, x, b, dinv, z, q, sc, red, PartView()); ::amg::count_launch(); } break;
        case 4: { pdl_launch(post_rz_csr_kernel<4, ZQ>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, x, b, dinv, z, q, sc, red, PartView()); ::amg::count_launch(); } break;
        case 8: { pdl_launch(post_rz_csr_kernel<8, ZQ>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, x, b, dinv, z, q, sc, red, PartView()); ::amg::count_launch(); } break;
        case 16: { pdl_launch(post_rz_csr_kernel<16, ZQ>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, x, b, dinv, z, q, sc, red, PartView()); ::amg::count_launch(); } break;
        default: { pdl_launch(post_rz_csr_kernel<32, ZQ>, blocks, kThreads, 0, s, n, A.rp, A.ci, A.v, x, b, dinv, z, q, sc, red, PartView()); ::amg::count_launch(); } break;
    }
    launch_finish<NV, kFinRz>(blocks, red, sc, s);
    AMG_CHECK_LAUNCH();
}

bool post_smooth_rz(const CycMat<double> &A, const double *x, const double *b, const double *dinv, double *z,
                    const double *q, PcgScalars *sc, Reduce red, cudaStream_t s) {
    if (A.nrows == 0) return false;
    if (q) post_smooth_rz_launch<true>(A, x, b, dinv, z, q, sc, red, s);
    else post_smooth_rz_launch<false>(A, x, b, dinv, z, q, sc, red, s);
    return true;
}

void to_f64_rz(int32_t n, const float *z32, double *z, const double *r, const double *q, PcgScalars *sc, Reduce red,
               cudaStream_t s) {
    int blocks = reduce_blocks(n);
    { pdl_launch(to_f64_rz_kernel, blocks, kThreads, 0, s, n, z32, z, r, q, sc, red); ::amg::count_launch(); }
    launch_finish<2, kFinRz>(blocks, red, sc, s);
    AMG_CHECK_LAUNCH();
}

template <typename XT> void scale(int64_t n, const XT *a, const XT *d, XT *out, cudaStream_t s) {
    if (n <= 0) return;
    { pdl_launch(scale_kernel<XT>, div_up(n, kThreads), kThreads, 0, s, n, a, d, out); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}
template void scale<double>(int64_t, const double *, const double *, double *, cudaStream_t);
template void scale<float>(int64_t, const float *, const float *, float *, cudaStream_t);

void to_f32_scaled(int64_t n, const double *src, const float *d, float *dst, float *xdst, cudaStream_t s) {
    if (n <= 0) return;
    { pdl_launch(to_f32_scaled_kernel, div_up(n, kThreads), kThreads, 0, s, n, src, d, dst, xdst); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void pcg_rz(int32_t n, const double *r, const double *z, const double *q, PcgScalars *sc, Reduce red,
            cudaStream_t s) {
    int blocks = reduce_blocks(n);
    { pdl_launch(rz_kernel, blocks, kThreads, 0, s, n, r, z, q, sc, red); ::amg::count_launch(); }
    launch_finish<2, kFinRz>(blocks, red, sc, s);
    AMG_CHECK_LAUNCH();
}

void true_residual(const CycMat<double> &A, const double *b, const double *x, double *t, PcgScalars *sc,
                   Reduce red, cudaStream_t s) {
    if (A.part.parts) {  // row-partitioned: the four-lane kernel's loop, as below
        part_exchange(A.part, x, nullptr, s);
        const int blocks = reduce_blocks((int64_t)A.nrows * 4);
        { pdl_launch(resid_kernel<4, true>, blocks, kThreads, 0, s, A.nrows, A.rp, A.part.cext, A.v, b, x, t, sc, red, A.part); ::amg::count_launch(); }
        launch_finish<1, kFinTt>(blocks, red, sc, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    if (A.variant == AMG_SPMV_SELL32 && A.sv && A.sell_c == 32) {  // the operator's tuned SELL copy, as A p uses
        const int blocks = launch_ap_sell<true>(A, x, b, t, sc, red, s);
        launch_finish<1, kFinTt>(blocks, red, sc, s);
        AMG_CHECK_LAUNCH();
        return;
    }
    int blocks = reduce_blocks((int64_t)A.nrows * 4);
    { pdl_launch(resid_kernel<4>, blocks, kThreads, 0, s, A.nrows, A.rp, A.ci, A.v, b, x, t, sc, red, PartView()); ::amg::count_launch(); }
    launch_finish<1, kFinTt>(blocks, red, sc, s);
    AMG_CHECK_LAUNCH();
}

template <typename VT> void convert_values(const double *src, VT *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    { convert_kernel<VT><<<div_up(n, kThreads), kThreads, 0, s>>>(src, dst, n); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}
template <typename XT> void convert_vec_from_f64(const double *src, XT *dst, int64_t n, cudaStream_t s) {
    convert_values<XT>(src, dst, n, s);
}
template <typename XT> void convert_vec_to_f64(const XT *src, double *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    { pdl_launch(to_f64_kernel<XT>, div_up(n, kThreads), kThreads, 0, s, src, dst, n); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

int64_t sell_layout(int32_t n, const int32_t *rp, int32_t *perm, int32_t *soff, int32_t *sw, cudaStream_t s, int C) {
    if (C != 32 && C != 16 && C != 8) throw Error(AMG_ERR_INVALID, "SELL slice height must be 32, 16 or 8");
    int32_t nsl = (n + C - 1) / C;
    if (nsl == 0) return 0;
    TmpBuf sz(sizeof(int32_t) * (nsl + 1), s);
    if (perm) { sell_sort_kernel<<<div_up(n, kSellSigma), 512, 0, s>>>(n, rp, perm); ::amg::count_launch(); }
    { slice_width_kernel<<<div_up(nsl, kThreads), kThreads, 0, s>>>(n, rp, perm, sw, C); ::amg::count_launch(); }
    { slice_size_kernel<<<div_up(nsl, kThreads), kThreads, 0, s>>>(nsl, sw, sz.as<int32_t>(), C); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    return exclusive_scan_i32(sz.as<int32_t>(), soff, nsl, s);
}

template <typename VT>
void sell_fill(int32_t n, const int32_t *rp, const int32_t *ci, const VT *v, const int32_t *perm, const int32_t *soff,
               const int32_t *sw, int32_t *sci, VT *sv, cudaStream_t s, int16_t *sd, int C) {
    int32_t nsl = (n + C - 1) / C;
    if (nsl == 0) return;
    { sell_fill_kernel<VT><<<div_up((int64_t)nsl * C, kThreads), kThreads, 0, s>>>(n, rp, ci, v, perm, soff, sw, sci, sv, sd, C); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

int32_t max_col_offset(int32_t n, const int32_t *rp, const int32_t *ci, cudaStream_t s, int32_t *max_row) {
    if (max_row) *max_row = 0;
    if (n == 0) return 0;
    TmpBuf out(sizeof(int) * 2, s);
    AMG_CUDA(cudaMemsetAsync(out.ptr, 0, sizeof(int) * 2, s));
    { max_col_offset_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, rp, ci, out.as<int>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    int h[2];
    read_back(h, out.ptr, sizeof(h), s);
    if (max_row) *max_row = h[1];
    return h[0];
}

// explicit instantiations
#define AMG_INST(VT, XT)                                                                                  \
    template void pre_smooth_residual<VT, XT>(const CycMat<VT> &, const XT *, const XT *, XT *, XT *, cudaStream_t); \
    template void post_smooth<VT, XT>(const CycMat<VT> &, const XT *, const XT *, const XT *, XT *, cudaStream_t); \
    template void spmv<VT, XT>(const CycMat<VT> &, const XT *, XT *, bool, cudaStream_t); \
    template void spmv_scaled<VT, XT>(const CycMat<VT> &, const XT *, const XT *, XT *, XT *, cudaStream_t); \
    template void residual_from_x<VT, XT>(const CycMat<VT> &, const XT *, const XT *, XT *, cudaStream_t);
AMG_INST(double, double)
AMG_INST(float, float)
AMG_INST(__nv_bfloat16, float)
#undef AMG_INST
template void coarse_solve<double>(int32_t, const double *, const double *, double *, cudaStream_t);
template void coarse_solve<float>(int32_t, const double *, const float *, float *, cudaStream_t);
template void convert_values<float>(const double *, float *, int64_t, cudaStream_t);
template void convert_values<__nv_bfloat16>(const double *, __nv_bfloat16 *, int64_t, cudaStream_t);
template void convert_vec_from_f64<float>(const double *, float *, int64_t, cudaStream_t);
template void convert_vec_to_f64<float>(const float *, double *, int64_t, cudaStream_t);
template void sell_fill<double>(int32_t, const int32_t *, const int32_t *, const double *, const int32_t *,
                                const int32_t *, const int32_t *, int32_t *, double *, cudaStream_t, int16_t *, int);
template void sell_fill<float>(int32_t, const int32_t *, const int32_t *, const float *, const int32_t *,
                               const int32_t *, const int32_t *, int32_t *, float *, cudaStream_t, int16_t *, int);
template void sell_fill<__nv_bfloat16>(int32_t, const int32_t *, const int32_t *, const __nv_bfloat16 *,
                                       const int32_t *, const int32_t *, const int32_t *, int32_t *, __nv_bfloat16 *,
                                       cudaStream_t, int16_t *, int);

}  // namespace cyc
}  // namespace amg
