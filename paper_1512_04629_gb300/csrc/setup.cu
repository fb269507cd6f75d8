// setup.cu -- setup-phase kernels: strength, PMIS, direct interpolation,
// transpose, Galerkin SpGEMM, minimal pattern, sparsify with diagonal lumping,
// ell1 diagonals and the coarsest-level dense inverse.
//
// Compiled with -fmad=false: each FP64 result is the IEEE evaluation of the
// formula as written, with sums taken sequentially in increasing column order
// (one thread per row, or one ordered accumulator per output entry), so the
// setup is deterministic and repeatable run to run.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "common.cuh"
#include "setup_ops.cuh"

namespace amg {
namespace setup {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int32_t lower_bound_i32(const int32_t *a, int32_t lo, int32_t hi,
                                                   int32_t key) {
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains(const int32_t *a, int32_t lo, int32_t hi, int32_t key) {
    int32_t p = lower_bound_i32(a, lo, hi, key);
    return p < hi && a[p] == key;
}

// ---------------------------------------------------------------------------
// validation and structural maps
// ---------------------------------------------------------------------------
enum : int { kBadCol = 1, kUnsorted = 2, kNoDiag = 4, kBadDiag = 8, kNonFinite = 16, kAsym = 32 };

__global__ void validate_kernel(int32_t n, int32_t ncols, const int32_t *rp, const int32_t *ci,
                                const double *v, int32_t *diagpos, int *err) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = 0;
    int32_t dp = -1, prev = -1;
    int32_t p0 = rp[i], p1 = rp[i + 1];
    if (p1 < p0) e |= kUnsorted;
    for (int32_t p = p0; p < p1; ++p) {
        int32_t j = ci[p];
        if (j < 0 || j >= ncols) { e |= kBadCol; continue; }
        if (j <= prev) e |= kUnsorted;
        prev = j;
        if (!isfinite(v[p])) e |= kNonFinite;
        if (j == i) dp = p;
    }
    if (dp < 0) e |= kNoDiag;
    else if (!(v[dp] > 0.0)) e |= kBadDiag;
    diagpos[i] = dp;
    if (e) atomicOr(err, e);
}

__global__ void tpos_kernel(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *tpos,
                            int *err) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t j = ci[p];
        int32_t q = lower_bound_i32(ci, rp[j], rp[j + 1], i);
        if (q < rp[j + 1] && ci[q] == i) tpos[p] = q;
        else { tpos[p] = p; atomicOr(err, (int)kAsym); }
    }
}

// ---------------------------------------------------------------------------
// strength: j in S_i iff j != i and -a_ij >= theta * max_{k != i}(-a_ik) > 0
// ---------------------------------------------------------------------------
__global__ void strength_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                                double theta, uint8_t *strong) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p0 = rp[i], p1 = rp[i + 1];
    double m = 0.0;
    bool any = false;
    for (int32_t p = p0; p < p1; ++p) {
        if (ci[p] == i) continue;
        double t = -v[p];
        if (!any || t > m) { m = t; any = true; }
    }
    double t = theta * m;
    for (int32_t p = p0; p < p1; ++p)
        strong[p] = (uint8_t)(any && m > 0.0 && ci[p] != i && -v[p] >= t);
}

// ---------------------------------------------------------------------------
// PMIS
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t key) {
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

enum : int8_t { kU = 0, kC = 1, kF = -1 };

__global__ void pmis_init_kernel(int32_t n, const int32_t *rp, const int32_t *tpos,
                                 const uint8_t *strong, uint64_t seed, int32_t level, double *w,
                                 int8_t *state, int *undecided) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int add = 0;
    if (i < n) {
        int32_t cnt = 0;  // |S^T_i|: rows j whose strong set holds i
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) cnt += strong[tpos[p]];
        uint64_t key = seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)i;
        double u = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
        w[i] = (double)cnt + u;
        state[i] = cnt == 0 ? kF : kU;
        add = cnt != 0;
    }
    add = __syncthreads_count(add);
    if (threadIdx.x == 0 && add) atomicAdd(undecided, add);
}

__global__ void pmis_select_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                   const int32_t *tpos, const uint8_t *strong, const double *w,
                                   const int8_t *state, uint8_t *newc) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t win = 0;
    if (state[i] == kU) {
        win = 1;
        double wi = w[i];
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (!(strong[p] || strong[tpos[p]])) continue;  // S_i u S^T_i
            int32_t j = ci[p];
            if (state[j] != kU) continue;
            double wj = w[j];
            if (wj > wi || (wj == wi && j > i)) { win = 0; break; }
        }
    }
    newc[i] = win;
}

__global__ void pmis_apply_c_kernel(int32_t n, const uint8_t *newc, int8_t *state) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && newc[i]) state[i] = kC;
}

__global__ void pmis_apply_f_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                    const uint8_t *strong, int8_t *state, int *undecided) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int still = 0;
    if (i < n && state[i] == kU) {
        bool f = false;
        for (int32_t p = rp[i]; p < rp[i + 1] && !f; ++p)
            if (strong[p] && state[ci[p]] == kC) f = true;
        if (f) state[i] = kF; else still = 1;
    }
    still = __syncthreads_count(still);
    if (threadIdx.x == 0 && still) atomicAdd(undecided, still);
}

// ---------------------------------------------------------------------------
// coarse numbering
// ---------------------------------------------------------------------------
__global__ void is_c_kernel(int32_t n, const int8_t *cf, int32_t *flag) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cf[i] == kC;
}

__global__ void cmap_kernel(int32_t n, const int8_t *cf, int32_t *cmap, int32_t *cpts) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == kC) cpts[cmap[i]] = i;
    else cmap[i] = -1;
}

// ---------------------------------------------------------------------------
// direct interpolation (count, then fill with the sums in column order)
// ---------------------------------------------------------------------------
__global__ void interp_count_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                    const uint8_t *strong, const int8_t *cf, int32_t *cnt) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == kC) { cnt[i] = 1; return; }
    int32_t c = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
        if (strong[p] && cf[ci[p]] == kC) ++c;
    cnt[i] = c;
}

__global__ void interp_fill_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                   const double *v, const uint8_t *strong, const int8_t *cf,
                                   const int32_t *cmap, const int32_t *prp, int32_t *pci,
                                   double *pv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t pos = prp[i];
    if (cf[i] == kC) { pci[pos] = cmap[i]; pv[pos] = 1.0; return; }
    if (prp[i + 1] == pos) return;  // no strong C neighbour: empty row
    double diag = 0.0, sum_neg = 0.0, sum_pos = 0.0, sum_neg_c = 0.0, sum_pos_c = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t j = ci[p];
        double a = v[p];
        if (j == i) { diag = a; continue; }
        if (a < 0.0) sum_neg += a;
        if (a > 0.0) sum_pos += a;
        if (strong[p] && cf[j] == kC) {
            if (a < 0.0) sum_neg_c += a;
            if (a > 0.0) sum_pos_c += a;
        }
    }
    double alpha = (sum_neg_c != 0.0) ? sum_neg / sum_neg_c : 0.0;
    double beta = 0.0;
    if (sum_pos_c != 0.0) beta = sum_pos / sum_pos_c;
    else diag = diag + sum_pos;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t j = ci[p];
        if (j == i || !strong[p] || cf[j] != kC) continue;
        double a = v[p];
        pci[pos] = cmap[j];
        pv[pos] = (a < 0.0) ? (-alpha * a) / diag : (-beta * a) / diag;
        ++pos;
    }
}

// ---------------------------------------------------------------------------
// transpose (counting; rows sorted afterwards by insertion sort)
// ---------------------------------------------------------------------------
__global__ void col_count_kernel(int64_t nnz, const int32_t *ci, int32_t *cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) atomicAdd(&cnt[ci[p]], 1);
}

__global__ void transpose_fill_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                      const double *v, int32_t *fill, int32_t *tci, double *tv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t q = atomicAdd(&fill[ci[p]], 1);
        tci[q] = i;
        tv[q] = v[p];
    }
}

__global__ void sort_rows_kernel(int32_t n, const int32_t *rp, int32_t *ci, double *v) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = rp[i] + 1; p < rp[i + 1]; ++p) {
        int32_t c = ci[p];
        double x = v[p];
        int32_t q = p - 1;
        while (q >= rp[i] && ci[q] > c) { ci[q + 1] = ci[q]; v[q + 1] = v[q]; --q; }
        ci[q + 1] = c;
        v[q + 1] = x;
    }
}

// ---------------------------------------------------------------------------
// SpGEMM C = A B.  Each row: hash the product columns (symbolic count), then
// hash again, sort the distinct columns (bitonic), and accumulate the values:
// entry (i,j) starts at 0.0 and adds a_ik b_kj for k in increasing order of
// A's row -- one ordered accumulator per entry, hence deterministic.
// A row is processed by one "group": a warp (shared tables), a block (shared
// tables) or a block with tables in global memory, chosen by the row's upper
// bound ub = sum_k nnz(B_k) on the number of distinct columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash32(int32_t k) { return (uint32_t)k * 2654435761u; }

template <int NT> __device__ __forceinline__ void gsync() {
    if (NT == 32) __syncwarp(); else __syncthreads();
}

struct RowTables {
    int32_t *keys;  // hs slots, -1 = empty
    int32_t *rank;  // hs slots: position of the key in the sorted list
    int32_t *list;  // umax: distinct columns
    double *acc;    // umax: accumulators
    int32_t hs;     // table capacity (power of two)
    int32_t umax;   // power of two >= distinct count
};

// slots used for one row: the smallest power of two >= 2 ub (at least 64),
// capped by the table capacity -- load factor <= 1/2 since u <= ub
__device__ __forceinline__ int32_t row_slots(int64_t ub, int32_t cap) {
    int32_t h = 64;
    while (h < cap && (int64_t)h < 2 * ub) h <<= 1;
    return h;
}

// Inserts every product column of row i; returns the number of distinct columns.
template <int NT>
__device__ int32_t row_insert(int32_t i, int32_t lane, const int32_t *arp, const int32_t *aci,
                              const int32_t *brp, const int32_t *bci, RowTables &t,
                              int32_t *counter, int64_t ub) {
    t.hs = row_slots(ub, t.umax * 2);
    for (int32_t s = lane; s < t.hs; s += NT) t.keys[s] = -1;
    if (lane == 0) *counter = 0;
    gsync<NT>();
    uint32_t mask = (uint32_t)t.hs - 1;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t k = aci[p];
        for (int32_t q = brp[k] + lane; q < brp[k + 1]; q += NT) {
            int32_t j = bci[q];
            uint32_t s = hash32(j) & mask;
            while (true) {
                int32_t old = atomicCAS(&t.keys[s], -1, j);
                if (old == -1) { atomicAdd(counter, 1); break; }
                if (old == j) break;
                s = (s + 1) & mask;
            }
        }
    }
    gsync<NT>();
    int32_t u = *counter;
    gsync<NT>();
    return u;
}

__device__ __forceinline__ int32_t row_lookup(const RowTables &t, int32_t j) {
    uint32_t mask = (uint32_t)t.hs - 1;
    uint32_t s = hash32(j) & mask;
    while (t.keys[s] != j) s = (s + 1) & mask;
    return t.rank[s];
}

template <int NT>
__device__ int32_t row_numeric(int32_t i, int32_t lane, const int32_t *arp, const int32_t *aci,
                               const double *av, const int32_t *brp, const int32_t *bci,
                               const double *bv, RowTables &t, int32_t *counter,
                               const int64_t *obase, int32_t *cci, double *cv, int64_t ub) {
    int32_t u = row_insert<NT>(i, lane, arp, aci, brp, bci, t, counter, ub);
    // compact the distinct keys, pad to a power of two, bitonic sort
    if (lane == 0) *counter = 0;
    gsync<NT>();
    for (int32_t s = lane; s < t.hs; s += NT) {
        int32_t k = t.keys[s];
        if (k >= 0) t.list[atomicAdd(counter, 1)] = k;
    }
    int32_t m = 1;
    while (m < u) m <<= 1;
    for (int32_t r = u + lane; r < m; r += NT) t.list[r] = INT_MAX;
    gsync<NT>();
    for (int32_t size = 2; size <= m; size <<= 1) {
        for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (int32_t r = lane; r < m; r += NT) {
                int32_t partner = r ^ stride;
                if (partner > r) {
                    bool up = (r & size) == 0;
                    int32_t a = t.list[r], b = t.list[partner];
                    if ((a > b) == up) { t.list[r] = b; t.list[partner] = a; }
                }
            }
            gsync<NT>();
        }
    }
    // rank of each key, output columns, zero accumulators
    uint32_t mask = (uint32_t)t.hs - 1;
    const int64_t base = obase[i];
    for (int32_t r = lane; r < u; r += NT) {
        int32_t j = t.list[r];
        uint32_t s = hash32(j) & mask;
        while (t.keys[s] != j) s = (s + 1) & mask;
        t.rank[s] = r;
        t.acc[r] = 0.0;
        cci[base + r] = j;
    }
    gsync<NT>();
    // ordered accumulation: k in A's row order; within one k the columns of
    // B_k are distinct, so lanes never collide
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t k = aci[p];
        double a = av[p];
        for (int32_t q = brp[k] + lane; q < brp[k + 1]; q += NT) {
            int32_t r = row_lookup(t, bci[q]);
            t.acc[r] += a * bv[q];
        }
        gsync<NT>();
    }
    for (int32_t r = lane; r < u; r += NT) cv[base + r] = t.acc[r];
    gsync<NT>();
    return u;
}

__global__ void spgemm_ub_kernel(int32_t n, const int32_t *arp, const int32_t *aci,
                                 const int32_t *brp, int64_t *ub) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = 0;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t k = aci[p];
        s += brp[k + 1] - brp[k];
    }
    ub[i] = s;
}

constexpr int kBlockHS = 8192, kBlockUmax = 4096, kBlockThreads = 256;
constexpr int kTinyUmax = 64, kTinyWarps = 8;     // bin 0: <= 64 products per row
constexpr int kSmallUmax = 512, kSmallWarps = 4;  // bin 1: <= 512 products per row

__global__ void bin_rows_kernel(int32_t n, const int64_t *ub, int32_t *bins, int32_t *bin_count) {
    __shared__ int32_t local[4], base[4];
    if (threadIdx.x < 4) local[threadIdx.x] = 0;
    __syncthreads();
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int b = -1;
    int32_t my = 0;
    if (i < n) {
        int64_t u = ub[i];
        b = u <= kTinyUmax ? 0 : (u <= kSmallUmax ? 1 : (u <= kBlockUmax ? 2 : 3));
        my = atomicAdd(&local[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < 4) base[threadIdx.x] = local[threadIdx.x] ? atomicAdd(&bin_count[threadIdx.x], local[threadIdx.x]) : 0;
    __syncthreads();
    if (b >= 0) bins[(int64_t)b * n + base[b] + my] = i;
}

// Per-warp shared layout for rows of at most U products: product values,
// hash keys and ranks (2U slots), distinct columns, per-column counts /
// cursors, product columns (later ranks), and the stable permutation.
template <int U> struct WarpTab {
    static constexpr size_t kBytes = (size_t)U * 8 + (size_t)4 * U * 4 + (size_t)(U + 4) * 4 + (size_t)U * 4 * 3;
    double *pv;
    int32_t *keys, *rank, *list, *cnt, *pj, *perm;
    __device__ WarpTab(unsigned char *base) {
        pv = reinterpret_cast<double *>(base);
        keys = reinterpret_cast<int32_t *>(base + (size_t)U * 8);
        rank = keys + 2 * U;
        cnt = rank + 2 * U;
        list = cnt + U + 4;
        pj = list + U;
        perm = pj + U;
    }
};

constexpr unsigned kFull = 0xffffffffu;

// One row of C = A B by one warp, all lanes working on the flattened product
// space.  Symbolic: returns the number of distinct columns.  Numeric: writes
// the sorted columns and, for every column, the sum of its products in the
// order of A's row (a stable scatter keeps product order), i.e. exactly the
// dense-accumulator order.
template <int U, bool NUMERIC>
__device__ int32_t warp_row(int32_t i, int lane, const int32_t *__restrict__ arp, const int32_t *__restrict__ aci,
                            const double *__restrict__ av, const int32_t *__restrict__ brp,
                            const int32_t *__restrict__ bci, const double *__restrict__ bv, WarpTab<U> &t,
                            int64_t ub, const int64_t *__restrict__ obase, int32_t *__restrict__ cci,
                            double *__restrict__ cv) {
    const int32_t hs = row_slots(ub, 2 * U);
    const uint32_t mask = (uint32_t)hs - 1;
    for (int32_t s = lane; s < hs; s += 32) t.keys[s] = -1;
    __syncwarp();
    const int32_t p0 = arp[i], nA = arp[i + 1] - p0;
    int32_t np = 0, uniq = 0;
    for (int32_t c0 = 0; c0 < nA; c0 += 32) {
        int32_t idx = c0 + lane, b0 = 0, len = 0;
        double a = 0.0;
        if (idx < nA) {
            int32_t k = aci[p0 + idx];
            if (NUMERIC) a = av[p0 + idx];
            b0 = brp[k];
            len = brp[k + 1] - b0;
        }
        int32_t incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t excl = incl - len;
        const int32_t total = __shfl_sync(kFull, incl, 31);
        for (int32_t eb = 0; eb < total; eb += 32) {
            const int32_t e = eb + lane;
            int lo = 0;
            for (int st = 16; st > 0; st >>= 1) {
                int cand = lo + st;
                int32_t ex = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && ex <= e) lo = cand;
            }
            const int32_t kb0 = __shfl_sync(kFull, b0, lo);
            const int32_t kex = __shfl_sync(kFull, excl, lo);
            const double ka = __shfl_sync(kFull, a, lo);
            if (e < total) {
                const int32_t q = kb0 + (e - kex);
                const int32_t j = bci[q];
                const int32_t E = np + e;
                if (NUMERIC) {
                    t.pj[E] = j;
                    t.pv[E] = ka * bv[q];
                }
                uint32_t sl = hash32(j) & mask;
                while (true) {
                    int32_t old = atomicCAS(&t.keys[sl], -1, j);
                    if (old == -1) { ++uniq; break; }
                    if (old == j) break;
                    sl = (sl + 1) & mask;
                }
            }
        }
        np += total;
    }
    for (int o = 16; o > 0; o >>= 1) uniq += __shfl_xor_sync(kFull, uniq, o);
    __syncwarp();
    if (!NUMERIC) return uniq;
    const int32_t u = uniq;
    // distinct columns -> list (ballot compaction), pad, bitonic sort
    int32_t base = 0;
    for (int32_t s0 = 0; s0 < hs; s0 += 32) {
        int32_t key = s0 + lane < hs ? t.keys[s0 + lane] : -1;
        unsigned m = __ballot_sync(kFull, key >= 0);
        if (key >= 0) t.list[base + __popc(m & ((1u << lane) - 1u))] = key;
        base += __popc(m);
    }
    int32_t m2 = 1;
    while (m2 < u) m2 <<= 1;
    for (int32_t r = u + lane; r < m2; r += 32) t.list[r] = INT_MAX;
    __syncwarp();
    for (int32_t size = 2; size <= m2; size <<= 1) {
        for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (int32_t r = lane; r < m2; r += 32) {
                int32_t partner = r ^ stride;
                if (partner > r) {
                    bool up = (r & size) == 0;
                    int32_t x = t.list[r], y = t.list[partner];
                    if ((x > y) == up) { t.list[r] = y; t.list[partner] = x; }
                }
            }
            __syncwarp();
        }
    }
    const int64_t cbase = obase[i];
    for (int32_t r = lane; r < u; r += 32) {
        int32_t j = t.list[r];
        uint32_t sl = hash32(j) & mask;
        while (t.keys[sl] != j) sl = (sl + 1) & mask;
        t.rank[sl] = r;
        t.cnt[r] = 0;
        cci[cbase + r] = j;
    }
    __syncwarp();
    // products per column
    for (int32_t e = lane; e < np; e += 32) {
        int32_t j = t.pj[e];
        uint32_t sl = hash32(j) & mask;
        while (t.keys[sl] != j) sl = (sl + 1) & mask;
        int32_t r = t.rank[sl];
        t.pj[e] = r;
        atomicAdd(&t.cnt[r], 1);
    }
    __syncwarp();
    // counts -> start offsets
    int32_t carry = 0;
    for (int32_t r0 = 0; r0 < u; r0 += 32) {
        int32_t r = r0 + lane;
        int32_t c = r < u ? t.cnt[r] : 0;
        int32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (r < u) t.cnt[r] = carry + incl - c;
        carry += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();
    // stable scatter: product e goes to the next free slot of its column, in e order
    for (int32_t eb = 0; eb < np; eb += 32) {
        const int32_t e = eb + lane;
        const bool valid = e < np;
        const int32_t r = valid ? t.pj[e] : -1 - lane;
        const unsigned peers = __match_any_sync(kFull, r);
        const int32_t within = __popc(peers & ((1u << lane) - 1u));
        const int32_t pos = valid ? t.cnt[r] + within : 0;
        __syncwarp();
        if (valid) {
            t.perm[pos] = e;
            if (lane == __ffs(peers) - 1) t.cnt[r] += __popc(peers);
        }
        __syncwarp();
    }
    // cnt[r] now holds the end of column r's segment (= start of r + 1)
    for (int32_t r = lane; r < u; r += 32) {
        int32_t s0 = r == 0 ? 0 : t.cnt[r - 1], s1 = t.cnt[r];
        double acc = 0.0;
        for (int32_t p = s0; p < s1; ++p) acc += t.pv[t.perm[p]];
        cv[cbase + r] = acc;
    }
    __syncwarp();
    return u;
}

template <int U, int WARPS, bool NUMERIC>
__global__ void __launch_bounds__(WARPS * 32)
spgemm_warp_kernel(const int32_t *rows, int32_t nrows, const int32_t *arp, const int32_t *aci,
                   const double *av, const int32_t *brp, const int32_t *bci, const double *bv,
                   int32_t *cnt, const int64_t *obase, int32_t *cci, double *cv, const int64_t *ub) {
    extern __shared__ __align__(16) unsigned char smem[];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTab<U> t(smem + (size_t)w * WarpTab<U>::kBytes);
    for (int32_t r = blockIdx.x * WARPS + w; r < nrows; r += gridDim.x * WARPS) {
        int32_t i = rows[r];
        int32_t u = warp_row<U, NUMERIC>(i, lane, arp, aci, av, brp, bci, bv, t, ub[i], obase, cci, cv);
        if (lane == 0) cnt[i] = u;
    }
}

template <bool NUMERIC>
__global__ void __launch_bounds__(kBlockThreads)
spgemm_block_kernel(const int32_t *rows, int32_t nrows, const int32_t *arp, const int32_t *aci,
                    const double *av, const int32_t *brp, const int32_t *bci, const double *bv,
                    int32_t *cnt, const int64_t *obase, int32_t *cci, double *cv, const int64_t *ub,
                    unsigned char *gscratch, int32_t ghs, int32_t gumax) {
    extern __shared__ __align__(16) unsigned char smem[];
    RowTables t;
    unsigned char *base;
    if (gscratch) {
        base = gscratch + (size_t)blockIdx.x * ((size_t)ghs * 8 + (size_t)gumax * 12);
        t.hs = ghs;
        t.umax = gumax;
    } else {
        base = smem;
        t.hs = kBlockHS;
        t.umax = kBlockUmax;
    }
    t.acc = reinterpret_cast<double *>(base);
    t.keys = reinterpret_cast<int32_t *>(base + (size_t)t.umax * 8);
    t.rank = t.keys + t.hs;
    t.list = t.rank + t.hs;
    __shared__ int32_t counter;
    for (int32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        int32_t i = rows[r];
        if (NUMERIC) {
            int32_t u = row_numeric<kBlockThreads>(i, threadIdx.x, arp, aci, av, brp, bci, bv, t, &counter,
                                                   obase, cci, cv, ub[i]);
            if (threadIdx.x == 0) cnt[i] = u;
        } else {
            int32_t u = row_insert<kBlockThreads>(i, threadIdx.x, arp, aci, brp, bci, t, &counter, ub[i]);
            if (threadIdx.x == 0) cnt[i] = u;
        }
    }
}

// ---------------------------------------------------------------------------
// minimal pattern: (i,j) in M iff j in AP[cpts[i]] or i in AP[cpts[j]]
// ---------------------------------------------------------------------------
__global__ void minimal_pattern_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                       const int32_t *aprp, const int32_t *apci,
                                       const int32_t *cpts, uint8_t *inM) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t fi = cpts[i];
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t j = ci[p];
        int32_t fj = cpts[j];
        bool m = contains(apci, aprp[fi], aprp[fi + 1], j) || contains(apci, aprp[fj], aprp[fj + 1], i);
        inM[p] = (uint8_t)m;
    }
}

// ---------------------------------------------------------------------------
// sparsify (Algorithm 3 first loop + Algorithm 3b)
// ---------------------------------------------------------------------------
__global__ void sparsify_flag_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                     const double *v, const uint8_t *inM, double gamma,
                                     double *rowmax, uint8_t *flag) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] != i && fabs(v[p]) > m) m = fabs(v[p]);
    rowmax[i] = m;
    double t = gamma * m;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
        flag[p] = (uint8_t)(ci[p] != i && (inM[p] || fabs(v[p]) >= t));
}

__global__ void sparsify_sym_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                    const double *v, const int32_t *tpos, const uint8_t *flag,
                                    const double *rowmax, uint8_t *keep, uint8_t *guard) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool any_off = false;
    double rs = 0.0, ra = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        bool k = ci[p] == i || flag[p] || flag[tpos[p]];
        keep[p] = (uint8_t)k;
        if (k && ci[p] != i) any_off = true;
        rs += v[p];
        ra += fabs(v[p]);
    }
    guard[i] = (uint8_t)(!any_off && rowmax[i] > 0.0 && fabs(rs) <= 1e-12 * ra);
}

__global__ void sparsify_guard_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                      const double *v, const int32_t *tpos, const uint8_t *guard,
                                      const double *rowmax, uint8_t *keep, int32_t *cnt) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t j = ci[p];
        if (!keep[p] && j != i) {
            if ((guard[i] && fabs(v[p]) == rowmax[i]) || (guard[j] && fabs(v[tpos[p]]) == rowmax[j]))
                keep[p] = 1;
        }
        c += keep[p];
    }
    cnt[i] = c;
}

__global__ void sparsify_compact_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                        const double *v, const int32_t *diagpos,
                                        const uint8_t *keep, const int32_t *hrp, int32_t *hci,
                                        double *hv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = v[diagpos[i]];
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
        if (!keep[p]) d += v[p];
    int32_t pos = hrp[i];
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        if (!keep[p]) continue;
        hci[pos] = ci[p];
        hv[pos] = (ci[p] == i) ? d : v[p];
        ++pos;
    }
}

__global__ void fill_u8_kernel(int64_t n, uint8_t *a, uint8_t val) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) a[p] = val;
}

__global__ void l1_kernel(int32_t n, const int32_t *rp, const double *v, double *d, double *dinv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) s += fabs(v[p]);
    d[i] = s;
    dinv[i] = 1.0 / s;
}

// ---------------------------------------------------------------------------
// coarsest level: dense Cholesky (one block), triangular inverse, A^{-1}
// ---------------------------------------------------------------------------
__global__ void densify_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                               double *a) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t j = 0; j < n; ++j) a[(size_t)i * n + j] = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) a[(size_t)i * n + ci[p]] = v[p];
}

__global__ void cholesky_kernel(int32_t n, double *a, int *err) {
    // right-looking, lower triangle of the row-major matrix
    __shared__ double piv;
    for (int32_t j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double d = a[(size_t)j * n + j];
            if (!(d > 0.0)) { *err = 1; d = 1.0; }
            piv = sqrt(d);
            a[(size_t)j * n + j] = piv;
        }
        __syncthreads();
        for (int32_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) a[(size_t)i * n + j] /= piv;
        __syncthreads();
        int32_t m = n - j - 1;
        for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
            int32_t r = j + 1 + (int32_t)(t / m), c = j + 1 + (int32_t)(t % m);
            if (c <= r) a[(size_t)r * n + c] -= a[(size_t)r * n + j] * a[(size_t)c * n + j];
        }
        __syncthreads();
    }
}

// column c of L^{-1} by forward substitution (one thread per column)
__global__ void tri_inverse_kernel(int32_t n, const double *L, double *Linv) {
    int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int32_t i = 0; i < n; ++i) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int32_t k = c; k < i; ++k) s -= L[(size_t)i * n + k] * Linv[(size_t)k * n + c];
        Linv[(size_t)i * n + c] = (i < c) ? 0.0 : s / L[(size_t)i * n + i];
    }
}

// inv = Linv^T Linv
__global__ void gram_kernel(int32_t n, const double *Linv, double *inv) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    int32_t i = (int32_t)(t / n), j = (int32_t)(t % n);
    double s = 0.0;
    for (int32_t k = max(i, j); k < n; ++k) s += Linv[(size_t)k * n + i] * Linv[(size_t)k * n + j];
    inv[t] = s;
}

// copy each row's entries from its product-bound slot to the final CSR
__global__ void spgemm_compact_kernel(int32_t n, const int64_t *obase, const int32_t *crp, const int32_t *tci,
                                      const double *tv, int32_t *cci, double *cv) {
    int32_t i = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    int64_t src = obase[i];
    int32_t dst = crp[i], len = crp[i + 1] - crp[i];
    for (int32_t e = lane; e < len; e += 32) {
        cci[dst + e] = tci[src + e];
        cv[dst + e] = tv[src + e];
    }
}

}  // namespace

// ===========================================================================
// host entry points
// ===========================================================================
void validate(const DevCSR &A, int32_t *diagpos, cudaStream_t s) {
    TmpBuf err(sizeof(int), s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    if (A.nrows > 0)
        { validate_kernel<<<div_up(A.nrows, kThreads), kThreads, 0, s>>>(
            A.nrows, A.ncols, A.rp(), A.ci(), A.v(), diagpos, err.as<int>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    int e = read_scalar(err.as<int>(), s);
    if (e) {
        std::string m = "invalid matrix:";
        if (e & kBadCol) m += " column index out of range;";
        if (e & kUnsorted) m += " columns not strictly increasing;";
        if (e & kNoDiag) m += " missing diagonal;";
        if (e & kBadDiag) m += " non-positive diagonal;";
        if (e & kNonFinite) m += " non-finite value;";
        throw Error(AMG_ERR_INVALID, m);
    }
}

void transpose_positions(const DevCSR &A, int32_t *tpos, cudaStream_t s) {
    TmpBuf err(sizeof(int), s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    if (A.nrows > 0)
        { tpos_kernel<<<div_up(A.nrows, kThreads), kThreads, 0, s>>>(A.nrows, A.rp(), A.ci(), tpos,
                                                                   err.as<int>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    if (read_scalar(err.as<int>(), s))
        throw Error(AMG_ERR_INVALID, "invalid matrix: sparsity pattern is not symmetric");
}

void strength(const DevCSR &A, double theta, uint8_t *strong, cudaStream_t s) {
    if (A.nrows == 0) return;
    { strength_kernel<<<div_up(A.nrows, kThreads), kThreads, 0, s>>>(A.nrows, A.rp(), A.ci(), A.v(),
                                                                   theta, strong); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

int64_t pmis(const DevCSR &A, const uint8_t *strong, const int32_t *tpos, uint64_t seed,
             int32_t level, int8_t *cf, cudaStream_t s) {
    int32_t n = A.nrows;
    if (n == 0) return 0;
    TmpBuf w(sizeof(double) * n, s), newc(n, s), cnt(sizeof(int), s);
    int g = div_up(n, kThreads);
    AMG_CUDA(cudaMemsetAsync(cnt.ptr, 0, sizeof(int), s));
    { pmis_init_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), tpos, strong, seed, level, w.as<double>(),
                                            cf, cnt.as<int>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    int undecided = read_scalar(cnt.as<int>(), s);
    int rounds = 0;
    while (undecided > 0) {
        if (++rounds > 10000) throw Error(AMG_ERR_CUDA, "PMIS did not terminate");
        { pmis_select_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), tpos, strong, w.as<double>(),
                                                  cf, newc.as<uint8_t>()); ::amg::count_launch(); }
        { pmis_apply_c_kernel<<<g, kThreads, 0, s>>>(n, newc.as<uint8_t>(), cf); ::amg::count_launch(); }
        AMG_CUDA(cudaMemsetAsync(cnt.ptr, 0, sizeof(int), s));
        { pmis_apply_f_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), strong, cf, cnt.as<int>()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        int next = read_scalar(cnt.as<int>(), s);
        if (next >= undecided) throw Error(AMG_ERR_CUDA, "PMIS made no progress");
        undecided = next;
    }
    TmpBuf flag(sizeof(int32_t) * n, s), scan(sizeof(int32_t) * (n + 1), s);
    { is_c_kernel<<<g, kThreads, 0, s>>>(n, cf, flag.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    return exclusive_scan_i32(flag.as<int32_t>(), scan.as<int32_t>(), n, s);
}

void coarse_map(const int8_t *cf, int32_t n, int32_t *cmap, int32_t *cpts, cudaStream_t s) {
    if (n == 0) return;
    TmpBuf flag(sizeof(int32_t) * n, s);
    int g = div_up(n, kThreads);
    { is_c_kernel<<<g, kThreads, 0, s>>>(n, cf, flag.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    // cmap has n+1 slots: exclusive scan of the C flags
    exclusive_scan_i32(flag.as<int32_t>(), cmap, n, s);
    { cmap_kernel<<<g, kThreads, 0, s>>>(n, cf, cmap, cpts); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void direct_interp(const DevCSR &A, const uint8_t *strong, const int8_t *cf, const int32_t *cmap,
                   int32_t nc, DevCSR &P, cudaStream_t s) {
    int32_t n = A.nrows;
    TmpBuf cnt(sizeof(int32_t) * (n + 1), s);
    P.rowptr.alloc(sizeof(int32_t) * (n + 1));
    int g = div_up(n, kThreads);
    if (n > 0) { interp_count_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), strong, cf, cnt.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    int64_t nnz = exclusive_scan_i32(cnt.as<int32_t>(), P.rp(), n, s);
    P.nrows = n;
    P.ncols = nc;
    P.nnz = nnz;
    P.col.alloc(sizeof(int32_t) * (nnz + kPad));
    P.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(P.col.ptr, 0, P.col.bytes, s));
    AMG_CUDA(cudaMemsetAsync(P.val.ptr, 0, P.val.bytes, s));
    if (n > 0)
        { interp_fill_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), strong, cf, cmap, P.rp(),
                                                  P.ci(), P.v()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void transpose(const DevCSR &M, DevCSR &T, cudaStream_t s) {
    int32_t m = M.ncols;
    TmpBuf cnt(sizeof(int32_t) * (m + 1), s), fill(sizeof(int32_t) * (m + 1), s);
    AMG_CUDA(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    if (M.nnz > 0) { col_count_kernel<<<div_up(M.nnz, kThreads), kThreads, 0, s>>>(M.nnz, M.ci(), cnt.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    T.rowptr.alloc(sizeof(int32_t) * (m + 1));
    int64_t nnz = exclusive_scan_i32(cnt.as<int32_t>(), T.rp(), m, s);
    T.nrows = m;
    T.ncols = M.nrows;
    T.nnz = nnz;
    T.col.alloc(sizeof(int32_t) * (nnz + kPad));
    T.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(T.col.ptr, 0, T.col.bytes, s));
    AMG_CUDA(cudaMemsetAsync(T.val.ptr, 0, T.val.bytes, s));
    AMG_CUDA(cudaMemcpyAsync(fill.ptr, T.rp(), sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToDevice, s));
    if (M.nrows > 0)
        { transpose_fill_kernel<<<div_up(M.nrows, kThreads), kThreads, 0, s>>>(
            M.nrows, M.rp(), M.ci(), M.v(), fill.as<int32_t>(), T.ci(), T.v()); ::amg::count_launch(); }
    if (m > 0) { sort_rows_kernel<<<div_up(m, kThreads), kThreads, 0, s>>>(m, T.rp(), T.ci(), T.v()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

static int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

void spgemm(const DevCSR &A, const DevCSR &B, DevCSR &Cm, cudaStream_t s) {
    require(A.ncols == B.nrows, "spgemm: inner dimensions differ");
    int32_t n = A.nrows;
    Cm.nrows = n;
    Cm.ncols = B.ncols;
    Cm.rowptr.alloc(sizeof(int32_t) * (n + 1));
    if (n == 0) {
        Cm.nnz = 0;
        AMG_CUDA(cudaMemsetAsync(Cm.rowptr.ptr, 0, sizeof(int32_t), s));
        Cm.col.alloc(sizeof(int32_t) * kPad);
        Cm.val.alloc(sizeof(double) * kPad);
        return;
    }
    TmpBuf ub(sizeof(int64_t) * n, s), bins(sizeof(int32_t) * 4 * (size_t)n, s), bcount(sizeof(int32_t) * 4, s),
        cnt(sizeof(int32_t) * (n + 1), s);
    int g = div_up(n, kThreads);
    { spgemm_ub_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), B.rp(), ub.as<int64_t>()); ::amg::count_launch(); }
    AMG_CUDA(cudaMemsetAsync(bcount.ptr, 0, bcount.bytes, s));
    { bin_rows_kernel<<<g, kThreads, 0, s>>>(n, ub.as<int64_t>(), bins.as<int32_t>(), bcount.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    int32_t nb[4];
    AMG_CUDA(cudaMemcpyAsync(nb, bcount.ptr, sizeof(nb), cudaMemcpyDeviceToHost, s));
    // largest upper bound in the global-table bin
    int64_t max_ub = 0;
    if (true) {
        std::vector<int64_t> h_ub(n);
        AMG_CUDA(cudaMemcpyAsync(h_ub.data(), ub.ptr, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        for (int32_t i = 0; i < n; ++i) max_ub = std::max(max_ub, h_ub[i]);
    }
    const int32_t *rows0 = bins.as<int32_t>();
    const int32_t *rows1 = rows0 + n;
    const int32_t *rows2 = rows0 + 2 * (size_t)n;
    const int32_t *rows3 = rows0 + 3 * (size_t)n;
    size_t tiny_smem = (size_t)kTinyWarps * WarpTab<kTinyUmax>::kBytes;
    size_t small_smem = (size_t)kSmallWarps * WarpTab<kSmallUmax>::kBytes;
    size_t block_smem = (size_t)kBlockHS * 8 + (size_t)kBlockUmax * 12;
    static bool attrs = false;
    if (!attrs) {
        AMG_CUDA(cudaFuncSetAttribute(spgemm_warp_kernel<kTinyUmax, kTinyWarps, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiny_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_warp_kernel<kTinyUmax, kTinyWarps, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiny_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_warp_kernel<kSmallUmax, kSmallWarps, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_warp_kernel<kSmallUmax, kSmallWarps, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem));
        attrs = true;
    }
    int64_t gumax = next_pow2(std::max<int64_t>(max_ub, 1));
    int64_t ghs = 2 * gumax;
    int gblocks = 0;
    TmpBuf gscr;
    if (nb[3] > 0) {
        size_t per = (size_t)ghs * 8 + (size_t)gumax * 12;
        int64_t cap = std::max<int64_t>(1, (int64_t)(((size_t)2 << 30) / per));  // <= 2 GiB scratch
        gblocks = (int)std::min<int64_t>({(int64_t)nb[3], 304, cap});
        gscr.alloc(per * gblocks, s);
    }
    const int64_t *ubp = ub.as<int64_t>();
    // launch(numeric, obase, out_cols, out_vals): one pass over the bins
    auto launch = [&](bool numeric, const int64_t *ob, int32_t *cc, double *cvv) {
        int32_t *cp = cnt.as<int32_t>();
        if (nb[0] > 0) {
            int blocks = std::min(div_up(nb[0], kTinyWarps), 152 * 32);
            if (numeric)
                { spgemm_warp_kernel<kTinyUmax, kTinyWarps, true><<<blocks, kTinyWarps * 32, tiny_smem, s>>>(
                    rows0, nb[0], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv, ubp); ::amg::count_launch(); }
            else
                { spgemm_warp_kernel<kTinyUmax, kTinyWarps, false><<<blocks, kTinyWarps * 32, tiny_smem, s>>>(
                    rows0, nb[0], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv, ubp); ::amg::count_launch(); }
        }
        if (nb[1] > 0) {
            int blocks = std::min(div_up(nb[1], kSmallWarps), 152 * 16);
            if (numeric)
                { spgemm_warp_kernel<kSmallUmax, kSmallWarps, true><<<blocks, kSmallWarps * 32, small_smem, s>>>(
                    rows1, nb[1], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv, ubp); ::amg::count_launch(); }
            else
                { spgemm_warp_kernel<kSmallUmax, kSmallWarps, false><<<blocks, kSmallWarps * 32, small_smem, s>>>(
                    rows1, nb[1], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv, ubp); ::amg::count_launch(); }
        }
        if (nb[2] > 0) {
            int blocks = std::min(nb[2], 152 * 4);
            if (numeric)
                { spgemm_block_kernel<true><<<blocks, kBlockThreads, block_smem, s>>>(
                    rows2, nb[2], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv,
                    ubp, nullptr, 0, 0); ::amg::count_launch(); }
            else
                { spgemm_block_kernel<false><<<blocks, kBlockThreads, block_smem, s>>>(
                    rows2, nb[2], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv,
                    ubp, nullptr, 0, 0); ::amg::count_launch(); }
        }
        if (nb[3] > 0) {
            if (numeric)
                { spgemm_block_kernel<true><<<gblocks, kBlockThreads, 0, s>>>(
                    rows3, nb[3], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv,
                    ubp, gscr.as<unsigned char>(), (int32_t)ghs, (int32_t)gumax); ::amg::count_launch(); }
            else
                { spgemm_block_kernel<false><<<gblocks, kBlockThreads, 0, s>>>(
                    rows3, nb[3], A.rp(), A.ci(), A.v(), B.rp(), B.ci(), B.v(), cp, ob, cc, cvv,
                    ubp, gscr.as<unsigned char>(), (int32_t)ghs, (int32_t)gumax); ::amg::count_launch(); }
        }
        AMG_CHECK_LAUNCH();
    };
    // one numeric pass into slots sized by each row's product bound, then a
    // compaction -- unless the bound does not fit: then count first (symbolic)
    TmpBuf obase(sizeof(int64_t) * (n + 1), s);
    int64_t total_ub = exclusive_scan_i64(ub.as<int64_t>(), obase.as<int64_t>(), n, s);
    size_t fr = 0, tot = 0;
    AMG_CUDA(cudaMemGetInfo(&fr, &tot));
    // AMG_SPGEMM_TWO_PASS=1 forces the counting path (it is otherwise taken
    // only when the product bound would not fit in free memory)
    const char *force = std::getenv("AMG_SPGEMM_TWO_PASS");
    bool one_pass = (double)total_ub * 12.0 < 0.4 * (double)fr && !(force && force[0] == '1');
    int64_t nnz;
    if (one_pass) {
        TmpBuf tci(sizeof(int32_t) * (total_ub + kPad), s), tv(sizeof(double) * (total_ub + kPad), s);
        launch(true, obase.as<int64_t>(), tci.as<int32_t>(), tv.as<double>());
        nnz = exclusive_scan_i32(cnt.as<int32_t>(), Cm.rp(), n, s);
        require(nnz < ((int64_t)1 << 31), "spgemm: product has 2^31 or more entries");
        Cm.nnz = nnz;
        Cm.col.alloc(sizeof(int32_t) * (nnz + kPad));
        Cm.val.alloc(sizeof(double) * (nnz + kPad));
        AMG_CUDA(cudaMemsetAsync(Cm.col.ptr, 0, Cm.col.bytes, s));
        AMG_CUDA(cudaMemsetAsync(Cm.val.ptr, 0, Cm.val.bytes, s));
        { spgemm_compact_kernel<<<div_up((int64_t)n * 32, 256), 256, 0, s>>>(n, obase.as<int64_t>(), Cm.rp(), tci.as<int32_t>(), tv.as<double>(), Cm.ci(), Cm.v()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        return;  // the temporaries' stream-ordered frees follow the compaction
    }
    launch(false, nullptr, nullptr, nullptr);
    nnz = exclusive_scan_i32(cnt.as<int32_t>(), Cm.rp(), n, s);
    require(nnz < ((int64_t)1 << 31), "spgemm: product has 2^31 or more entries");
    Cm.nnz = nnz;
    Cm.col.alloc(sizeof(int32_t) * (nnz + kPad));
    Cm.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(Cm.col.ptr, 0, Cm.col.bytes, s));
    AMG_CUDA(cudaMemsetAsync(Cm.val.ptr, 0, Cm.val.bytes, s));
    exclusive_scan_i64_from_i32(cnt.as<int32_t>(), obase.as<int64_t>(), n, s);
    launch(true, obase.as<int64_t>(), Cm.ci(), Cm.v());
}

void minimal_pattern(const DevCSR &Ac, const DevCSR &AP, const int32_t *cpts, uint8_t *inM,
                     cudaStream_t s) {
    if (Ac.nrows == 0) return;
    { minimal_pattern_kernel<<<div_up(Ac.nrows, kThreads), kThreads, 0, s>>>(
        Ac.nrows, Ac.rp(), Ac.ci(), AP.rp(), AP.ci(), cpts, inM); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

int64_t sparsify(const DevCSR &A, const uint8_t *inM, const int32_t *tpos, const int32_t *diagpos,
                 double gamma, uint8_t *keep, DevCSR &H, cudaStream_t s) {
    int32_t n = A.nrows;
    TmpBuf rowmax(sizeof(double) * (n + 1), s), flag(A.nnz + 1, s), guard(n + 1, s), cnt(sizeof(int32_t) * (n + 1), s);
    int g = div_up(n, kThreads);
    if (n > 0) {
        { sparsify_flag_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), inM, gamma,
                                                    rowmax.as<double>(), flag.as<uint8_t>()); ::amg::count_launch(); }
        { sparsify_sym_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), tpos, flag.as<uint8_t>(),
                                                   rowmax.as<double>(), keep, guard.as<uint8_t>()); ::amg::count_launch(); }
        { sparsify_guard_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), tpos, guard.as<uint8_t>(),
                                                     rowmax.as<double>(), keep, cnt.as<int32_t>()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
    }
    H.rowptr.alloc(sizeof(int32_t) * (n + 1));
    int64_t nnz = exclusive_scan_i32(cnt.as<int32_t>(), H.rp(), n, s);
    H.nrows = n;
    H.ncols = A.ncols;
    H.nnz = nnz;
    H.col.alloc(sizeof(int32_t) * (nnz + kPad));
    H.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(H.col.ptr, 0, H.col.bytes, s));
    AMG_CUDA(cudaMemsetAsync(H.val.ptr, 0, H.val.bytes, s));
    if (n > 0) {
        { sparsify_compact_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), diagpos, keep, H.rp(),
                                                       H.ci(), H.v()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
    }
    return nnz;
}

void copy_all(const DevCSR &A, uint8_t *keep, DevCSR &H, cudaStream_t s) {
    H.nrows = A.nrows;
    H.ncols = A.ncols;
    H.nnz = A.nnz;
    H.rowptr.alloc(A.rowptr.bytes);
    H.col.alloc(A.col.bytes);
    H.val.alloc(A.val.bytes);
    AMG_CUDA(cudaMemcpyAsync(H.rowptr.ptr, A.rowptr.ptr, A.rowptr.bytes, cudaMemcpyDeviceToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(H.col.ptr, A.col.ptr, A.col.bytes, cudaMemcpyDeviceToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(H.val.ptr, A.val.ptr, A.val.bytes, cudaMemcpyDeviceToDevice, s));
    if (A.nnz > 0) { fill_u8_kernel<<<div_up(A.nnz, kThreads), kThreads, 0, s>>>(A.nnz, keep, 1); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void l1_diag(const DevCSR &A, double *d, double *dinv, cudaStream_t s) {
    if (A.nrows == 0) return;
    { l1_kernel<<<div_up(A.nrows, kThreads), kThreads, 0, s>>>(A.nrows, A.rp(), A.v(), d, dinv); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void cholesky_inverse(const DevCSR &A, double *inv, cudaStream_t s) {
    int32_t n = A.nrows;
    if (n == 0) return;
    require(n <= 8192, "coarsest level too large for the dense direct solve (n > 8192)");
    TmpBuf a(sizeof(double) * (size_t)n * n, s), linv(sizeof(double) * (size_t)n * n, s), err(sizeof(int), s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    { densify_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), a.as<double>()); ::amg::count_launch(); }
    { cholesky_kernel<<<1, 1024, 0, s>>>(n, a.as<double>(), err.as<int>()); ::amg::count_launch(); }
    { tri_inverse_kernel<<<div_up(n, 128), 128, 0, s>>>(n, a.as<double>(), linv.as<double>()); ::amg::count_launch(); }
    { gram_kernel<<<div_up((int64_t)n * n, kThreads), kThreads, 0, s>>>(n, linv.as<double>(), inv); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    if (read_scalar(err.as<int>(), s))
        throw Error(AMG_BREAKDOWN, "coarsest operator is not positive definite (Cholesky pivot <= 0)");
}

}  // namespace setup
}  // namespace amg
