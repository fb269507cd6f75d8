// setup.cu -- setup-phase kernels: strength, PMIS, direct interpolation,
// transpose, Galerkin SpGEMM, minimal pattern, sparsify with diagonal lumping,
// ell1 diagonals and the coarsest-level dense inverse.
//
// Compiled with -fmad=false: each FP64 result is the IEEE evaluation of the
// formula as written, with sums taken sequentially in increasing column order
// (one thread per row, or one ordered accumulator per output entry), so the
// setup is deterministic and repeatable run to run.
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <climits>
#include <cstdlib>
#include <cstring>

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
enum : int { kBadCol = 1, kUnsorted = 2, kNoDiag = 4, kBadDiag = 8, kNonFinite = 16, kAsym = 32, kBadRowptr = 64 };

// FP64 instructions are the scarce pipe on this part (a few per SM and
// clock), comparisons included; the tests below decide the same IEEE
// comparisons of non-NaN doubles on the integer pipes, through an order key
// of the bit pattern: key(x) < key(y) iff x < y, and key(+0) = key(-0).
__device__ __forceinline__ int64_t f64_key(double x) {
    const int64_t b = __double_as_longlong(x);
    return b >= 0 ? b : -(b & 0x7fffffffffffffffll);
}
// key(-x), the sign flipped on the integer pipes
__device__ __forceinline__ int64_t f64_key_neg(double x) {
    return f64_key(__longlong_as_double(__double_as_longlong(x) ^ (int64_t)0x8000000000000000ull));
}
// |x| as a key (the bit pattern without its sign)
__device__ __forceinline__ int64_t f64_abs_key(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffll; }
// Row kernels map a group of T lanes (T = 2..32, a power of two near the
// mean row length) to each row; the lanes take the row's entries with stride
// T, so the gathers of a row are in flight together instead of one after
// another.  Group reductions below are exact (integer max / or / sum).
template <int T> __device__ __forceinline__ bool group_any(bool x) {
    const unsigned b = __ballot_sync(0xffffffffu, x);
    if constexpr (T == 32) {
        return b != 0u;
    } else {
        const int base = (threadIdx.x & 31) & ~(T - 1);
        return ((b >> base) & ((1u << T) - 1u)) != 0u;
    }
}
template <int T> __device__ __forceinline__ int64_t group_max_i64(int64_t x) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) x = max(x, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)x, o, T));
    return x;
}
template <int T> __device__ __forceinline__ int32_t group_sum_i32(int32_t x) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, T);
    return x;
}
// the double whose order key is k (inverse of f64_key, +0.0 for key 0)
__device__ __forceinline__ double f64_from_key(int64_t k) {
    return __longlong_as_double(k >= 0 ? k : ((-k) | (int64_t)0x8000000000000000ull));
}

// 0.0 + x without an FP64 add: x itself, except that -0.0 becomes +0.0
__device__ __forceinline__ double f64_zero_plus(double x) {
    const int64_t b = __double_as_longlong(x);
    return __longlong_as_double(b == (int64_t)0x8000000000000000ull ? 0ll : b);
}

// Every row range is checked against [0, nnz] before its entries are read,
// so the kernel stays in bounds on any row-pointer array.
__device__ __forceinline__ bool row_in_bounds(int32_t p0, int32_t p1, int64_t nnz) {
    return p0 >= 0 && p0 <= p1 && (int64_t)p1 <= nnz;
}

// With TPOS (square matrices) the same pass also records, for every entry
// (i, j), the position of (j, i) in row j -- found by binary search in the
// sorted row, followed only once j and row j's bounds are known to be valid;
// a missing mirror entry is reported as an asymmetric pattern.
template <int T, bool TPOS>
__global__ void validate_kernel(int32_t n, int32_t ncols, int64_t nnz, const int32_t *rp, const int32_t *ci,
                                const double *v, int32_t *diagpos, int32_t *tpos, int *err) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: the group reductions need every lane
    int e = 0;
    int32_t p0 = 0, p1 = 0;
    bool inb = false;
    if (live) {
        p0 = rp[i];
        p1 = rp[i + 1];
        if ((i == 0 && p0 != 0) || (i == n - 1 && (int64_t)p1 != nnz)) e |= kBadRowptr;
        inb = row_in_bounds(p0, p1, nnz);
        if (!inb) e |= kBadRowptr;
    }
    int32_t dp = -1;
    if (inb) {
        for (int32_t p = p0 + t; p < p1; p += T) {
            const int32_t j = ci[p];
            if (j < 0 || j >= ncols) {
                e |= kBadCol;
                if (TPOS) tpos[p] = p;  // reported, not followed
                continue;
            }
            if (p > p0 && ci[p - 1] >= j) e |= kUnsorted;  // strictly increasing columns
            if (!isfinite(v[p])) e |= kNonFinite;
            if (j == i) dp = p;
            if (TPOS) {
                const int32_t q0 = rp[j], q1 = rp[j + 1];
                if (!row_in_bounds(q0, q1, nnz)) {
                    tpos[p] = p;
                    e |= kBadRowptr;
                    continue;
                }
                const int32_t q = lower_bound_i32(ci, q0, q1, i);
                if (q < q1 && ci[q] == i) {
                    tpos[p] = q;
                } else {
                    tpos[p] = p;
                    e |= kAsym;
                }
            }
        }
    }
    dp = (int32_t)group_max_i64<T>((int64_t)dp);  // the diagonal position, if stored (one lane holds it)
    if (live && t == 0 && inb) {
        if (dp < 0) e |= kNoDiag;
        else if (!(f64_key(v[dp]) > 0)) e |= kBadDiag;
        diagpos[i] = dp;
    } else if (live && t == 0) {
        diagpos[i] = -1;
    }
    if (e) atomicOr(err, e);
}

// ---------------------------------------------------------------------------
// strength: j in S_i iff j != i and -a_ij >= theta * max_{k != i}(-a_ik) > 0
// ---------------------------------------------------------------------------
template <int T>
__global__ void strength_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                                double theta, uint8_t *strong) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: the group reduction needs every lane
    int32_t p0 = 0, p1 = 0;
    if (live) { p0 = rp[i]; p1 = rp[i + 1]; }
    constexpr int64_t kNone = INT64_MIN;  // below every key
    int64_t mk = kNone;                   // max over j != i of -a_ij (as a key)
    for (int32_t p = p0 + t; p < p1; p += T)
        if (ci[p] != i) mk = max(mk, f64_key_neg(v[p]));
    mk = group_max_i64<T>(mk);
    if (!live || mk <= 0) {  // no off-diagonal, or max(-a_ij) <= 0: no strong entry
        for (int32_t p = p0 + t; p < p1; p += T) strong[p] = 0;
        return;
    }
    const int64_t tk = f64_key(theta * f64_from_key(mk));
    for (int32_t p = p0 + t; p < p1; p += T)
        strong[p] = (uint8_t)(ci[p] != i && f64_key_neg(v[p]) >= tk);
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

// Appends row i to a list when `keep` holds, with one global atomic per
// block (warps reserve their places in shared memory first): a global
// counter that every warp of a large grid increments serialises on one
// address (measured: PMIS's first pass at 128^3, 262K warp atomics, 187 us).
// Every thread of the block must call it (it holds two block barriers).  The
// list's order varies from run to run, its contents do not.
__device__ __forceinline__ void block_append(bool keep, int32_t i, int32_t *list, int *count) {
    __shared__ int s_count, s_base;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31;
    int wbase = 0;
    if (lane == 0 && m) wbase = atomicAdd(&s_count, __popc(m));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_count ? atomicAdd(count, s_count) : 0;
    __syncthreads();
    if (keep) list[s_base + wbase + __popc(m & ((1u << lane) - 1u))] = i;
}

template <int T>
__global__ void pmis_init_kernel(int32_t n, const int32_t *rp, const int32_t *tpos,
                                 const uint8_t *strong, uint64_t seed, int32_t level, double *w,
                                 int8_t *state, int *undecided, uint8_t *sym, int32_t *list) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: the group reduction and the append need every lane
    int32_t cnt = 0;  // |S^T_i|: rows j whose strong set holds i
    if (live) {
        const int32_t p0 = rp[i], p1 = rp[i + 1];
        for (int32_t pb = p0 + t; pb < p1; pb += T * 4) {  // four entries' loads in flight per lane
            int32_t tp[4];
            uint8_t own[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t p = pb + u * T;
                tp[u] = p < p1 ? tpos[p] : 0;
                own[u] = p < p1 ? strong[p] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t p = pb + u * T;
                if (p >= p1) continue;
                const uint8_t st = strong[tp[u]];
                cnt += st;
                sym[p] = (uint8_t)(st | own[u]);  // j in S_i u S^T_i, read by every round
            }
        }
    }
    cnt = group_sum_i32<T>(cnt);
    bool und = false;
    if (live && t == 0) {
        uint64_t key = seed ^ ((uint64_t)(uint32_t)level << 40) ^ (uint64_t)i;
        double u = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
        w[i] = (double)cnt + u;
        state[i] = cnt == 0 ? kF : kU;
        und = cnt != 0;
    }
    block_append(und, i, list, undecided);
}

// Every round works on the list of rows still undecided when it starts (the
// previous round's output, with its length on the device).  Rounds are
// launched in batches without reading back in between, on a grid of at most
// one wave of resident blocks that strides over the list; a kernel reads the
// list's actual length first and does nothing once it is zero.  Every block
// takes the same number of strides, so the block barriers of the append are
// reached by all of its threads.
constexpr int kPmisChunk = 4;

// DENSE (the first round, when nearly every row is undecided): the rows
// 0 .. n-1 themselves, the undecided ones taking part -- coalesced, and one
// dependent load shorter than going through the list.
template <int T, bool DENSE>
__global__ void pmis_select_kernel(const int32_t *list, const int *len, int32_t n, const int32_t *rp,
                                   const int32_t *ci, const uint8_t *sym, const double *w, const int8_t *state,
                                   uint8_t *newc) {
    const int m = DENSE ? n : *len;  // the same for the whole grid
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g - threadIdx.x < (int64_t)m * T;
         g += stride) {
        const int64_t k = g / T;
        const int t = (int)(g % T);
        const int32_t i = k < m ? (DENSE ? (int32_t)k : list[k]) : 0;
        // the row's bounds, weight and state are independent loads, issued together
        const int32_t p0 = k < m ? rp[i] : 0, p1 = k < m ? rp[i + 1] : 0;
        const int64_t wi = k < m ? __double_as_longlong(w[i]) : 0;  // weights >= 0 order like their bits
        const bool live = k < m && (!DENSE || state[i] == kU);  // no early exit: the group reduction needs every lane
        bool lose = false;
        if (live) {
            // kPmisChunk entries a lane per step: their flags and columns, then
            // their neighbours' states and weights, are each in flight together
            for (int32_t pb = p0 + t; pb < p1; pb += T * kPmisChunk) {
                int32_t jj[kPmisChunk];
                bool sy[kPmisChunk];
#pragma unroll
                for (int u = 0; u < kPmisChunk; ++u) {
                    const int32_t p = pb + u * T;
                    sy[u] = p < p1 && sym[p];  // S_i u S^T_i
                    jj[u] = p < p1 ? ci[p] : i;
                }
#pragma unroll
                for (int u = 0; u < kPmisChunk; ++u) {
                    if (!sy[u]) continue;
                    const int32_t j = jj[u];
                    const int8_t sj = state[j];
                    const int64_t wj = __double_as_longlong(w[j]);
                    if (sj == kU && (wj > wi || (wj == wi && j > i))) lose = true;
                }
            }
        }
        lose = group_any<T>(lose);
        if (live && t == 0) newc[i] = (uint8_t)!lose;
    }
}

// The round's two steps in one pass: a selected row becomes C; any other row
// of the list becomes F when one of its strong neighbours j (j in S_i) is C --
// from an earlier round (state C) or selected in this one (state still U
// when read, newc[j] set: j is on this round's list, so newc[j] is this
// round's).  A row's own state is written only by its own group, and a
// neighbour read before or after its write gives the same answer, so the
// result does not depend on the order of the groups.  Undecided rows go to
// the next round's list.
template <int T, bool DENSE>
__global__ void pmis_apply_kernel(const int32_t *list, const int *len, int32_t n, const int32_t *rp,
                                  const int32_t *ci, const uint8_t *strong, const uint8_t *newc, int8_t *state,
                                  int32_t *next, int *next_len, int *ccount) {
    const int m = DENSE ? n : *len;  // the same for the whole grid
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g - threadIdx.x < (int64_t)m * T;
         g += stride) {
        const int64_t k = g / T;
        const int t = (int)(g % T);
        const int32_t i = k < m ? (DENSE ? (int32_t)k : list[k]) : 0;
        const int32_t p0 = k < m ? rp[i] : 0, p1 = k < m ? rp[i + 1] : 0;
        const bool live = k < m && (!DENSE || state[i] == kU);  // a row's state is written by its own group only
        const bool c = live && newc[i];
        const bool und = live && !c;
        bool f = false;
        if (und)
            for (int32_t pb = p0 + t; pb < p1; pb += T * kPmisChunk) {
                int32_t jj[kPmisChunk];
                bool st[kPmisChunk];
#pragma unroll
                for (int u = 0; u < kPmisChunk; ++u) {
                    const int32_t p = pb + u * T;
                    st[u] = p < p1 && strong[p];
                    jj[u] = p < p1 ? ci[p] : i;
                }
#pragma unroll
                for (int u = 0; u < kPmisChunk; ++u) {
                    if (!st[u]) continue;
                    const int32_t j = jj[u];
                    const int8_t sj = *(volatile const int8_t *)&state[j];
                    const bool cj = newc[j] != 0;
                    if (sj == kC || (sj == kU && cj)) f = true;
                }
            }
        f = group_any<T>(f);
        if (live && t == 0) {
            if (c) state[i] = kC;
            else if (f) state[i] = kF;
        }
        const int cb = __syncthreads_count(live && t == 0 && c);  // the block's new C points
        if (threadIdx.x == 0 && cb) atomicAdd(ccount, cb);
        block_append(und && t == 0 && !f, i, next, next_len);
    }
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
template <int T>
__global__ void interp_count_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                    const uint8_t *strong, const int8_t *cf, int32_t *cnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool fpt = i < n && cf[i] != kC;
    int32_t c = 0;
    if (fpt)
        for (int32_t p = rp[i] + t; p < rp[i + 1]; p += T)
            if (strong[p] && cf[ci[p]] == kC) ++c;
    c = group_sum_i32<T>(c);
    if (i < n && t == 0) cnt[i] = fpt ? c : 1;
}

// Direct interpolation in two passes.  The row pass forms the row sums in
// column order and the two ratios (alpha, beta) and the lumped diagonal,
// and lays out P's pattern with a_ij in place of the weight; the entry pass
// turns every a_ij into (-alpha a_ij) / d or (-beta a_ij) / d, one entry per
// thread -- the divisions are the FP64-heavy part, and there every lane of a
// warp holds a live entry.
__global__ void interp_rows_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                   const double *v, const uint8_t *strong, const int8_t *cf,
                                   const int32_t *cmap, const int32_t *prp, int32_t *pci,
                                   double *pv, int32_t *prow, double *coef) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t pos = prp[i];
    if (cf[i] == kC) { pci[pos] = cmap[i]; pv[pos] = 1.0; prow[pos] = -1; return; }
    if (prp[i + 1] == pos) return;  // no strong C neighbour: empty row
    double diag = 0.0, sum_neg = 0.0, sum_pos = 0.0, sum_neg_c = 0.0, sum_pos_c = 0.0;
    // one pass: the row sums in column order, and P's pattern with a_ij in
    // place of the weight (the weights need the finished sums).  An entry
    // changes at most two sums -- its sign's total and, for a strong C
    // neighbour, its sign's C sum -- so two FP64 additions are issued per
    // entry (a warp instruction costs the FP64 pipe the same however few of
    // its lanes take it): the sums of the entry's sign are selected, added
    // to, and written back.  Adding +0.0 (a zero entry, or no strong C
    // neighbour) leaves a sum unchanged: every sum starts at +0.0 and
    // accumulates values of one sign, so it is never -0.0.
    // entries in chunks of 8: the chunk's loads, then its C/F gathers, are
    // issued together before the sums walk it in column order
    const int32_t pe = rp[i + 1];
    for (int32_t p0 = rp[i]; p0 < pe; p0 += 8) {
        int32_t jj[8];
        double aa[8];
        bool sc8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int32_t p = p0 + u;
            const bool in = p < pe;
            jj[u] = in ? ci[p] : i;
            aa[u] = in ? v[p] : 0.0;
            sc8[u] = in && strong[p];  // the diagonal is never strong
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (sc8[u]) sc8[u] = cf[jj[u]] == kC;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (p0 + u >= pe) break;
            const int32_t j = jj[u];
            const double a = aa[u];
            if (j == i) { diag = a; continue; }
            const int64_t ak = f64_key(a);
            const bool sc = sc8[u];
            const bool is_neg = ak < 0, is_pos = ak > 0;
            const double tot = (is_neg ? sum_neg : sum_pos) + a;
            const double csum = (is_neg ? sum_neg_c : sum_pos_c) + (sc ? a : 0.0);
            if (is_neg) { sum_neg = tot; sum_neg_c = csum; }
            if (is_pos) { sum_pos = tot; sum_pos_c = csum; }
            if (sc) {
                pci[pos] = cmap[j];
                pv[pos] = a;
                prow[pos] = i;
                ++pos;
            }
        }
    }
    double alpha = f64_key(sum_neg_c) != 0 ? sum_neg / sum_neg_c : 0.0;
    double beta = 0.0;
    if (f64_key(sum_pos_c) != 0) beta = sum_pos / sum_pos_c;
    else diag = diag + sum_pos;
    coef[3 * (int64_t)i] = alpha;
    coef[3 * (int64_t)i + 1] = beta;
    coef[3 * (int64_t)i + 2] = diag;
}

__global__ void interp_weights_kernel(int64_t nnz, const int32_t *prow, const double *coef, double *pv) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int32_t i = prow[e];
    if (i < 0) return;  // C row: weight 1
    const double a = pv[e];
    const double c = coef[3 * (int64_t)i + (f64_key(a) < 0 ? 0 : 1)];
    pv[e] = (-c * a) / coef[3 * (int64_t)i + 2];
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

// Sorts every row of the transpose by column, in place.  A group of W lanes
// holds a row of up to 4W entries in registers; each entry's rank is the
// number of smaller columns in the row (columns are distinct), found by
// broadcasting the row's entries one by one; entries are written back to
// their ranks.  Longer rows are sorted by one lane (insertion sort).
template <int W>
__global__ void sort_rows_kernel(int32_t n, const int32_t *rp, int32_t *ci, double *v) {
    constexpr int E = 4;
    const int sl = threadIdx.x & (W - 1);
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / W);
    const bool live = i < n;
    int32_t p0 = 0, len = 0;
    if (live) { p0 = rp[i]; len = rp[i + 1] - p0; }
    const bool small = len <= E * W;
    int32_t key[E];
    double val[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int32_t e = r * W + sl;
        key[r] = INT_MAX;
        val[r] = 0.0;
        if (small && e < len) { key[r] = ci[p0 + e]; val[r] = v[p0 + e]; }
    }
    const int32_t m = small ? len : 0;
    const int32_t mmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)m);
    int32_t rank[E] = {};
    for (int32_t src = 0; src < mmax; ++src) {  // every entry of the row is broadcast once
        const int rsrc = src / W;
        int32_t kv = key[0];
#pragma unroll
        for (int r = 1; r < E; ++r)
            if (rsrc == r) kv = key[r];
        const int32_t other = __shfl_sync(0xffffffffu, kv, src & (W - 1), W);
        if (src < m) {
#pragma unroll
            for (int r = 0; r < E; ++r) rank[r] += other < key[r];
        }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int32_t e = r * W + sl;
        if (small && e < len) { ci[p0 + rank[r]] = key[r]; v[p0 + rank[r]] = val[r]; }
    }
    if (!small && live && sl == 0) {
        for (int32_t p = p0 + 1; p < p0 + len; ++p) {
            int32_t c = ci[p];
            double x = v[p];
            int32_t q = p - 1;
            while (q >= p0 && ci[q] > c) { ci[q + 1] = ci[q]; v[q + 1] = v[q]; --q; }
            ci[q + 1] = c;
            v[q + 1] = x;
        }
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

template <int R>
__device__ __forceinline__ void warp_bitonic_sort(int32_t (&k)[R], int lane);

// t.list[0 .. u) (u <= 32 R) sorted in place by the first warp of the block
template <int R, int NT>
__device__ __forceinline__ void block_list_sort_warp(int32_t *list, int32_t u, int32_t lane) {
    if (lane < 32) {
        int32_t k[R];
#pragma unroll
        for (int r = 0; r < R; ++r) k[r] = lane + 32 * r < u ? list[lane + 32 * r] : INT_MAX;
        warp_bitonic_sort<R>(k, lane);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (lane + 32 * r < u) list[lane + 32 * r] = k[r];
    }
}

// Inserts every product column of row i; returns the number of distinct columns.
template <int NT>
__device__ int32_t row_insert(int32_t i, int32_t lane, const int32_t *arp, const int32_t *aci,
                              const int32_t *bbeg, const int32_t *bend, const int32_t *bci, RowTables &t,
                              int32_t *counter, int64_t ub) {
    t.hs = row_slots(ub, t.umax * 2);
    for (int32_t s = lane; s < t.hs; s += NT) t.keys[s] = -1;
    if (lane == 0) *counter = 0;
    gsync<NT>();
    uint32_t mask = (uint32_t)t.hs - 1;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t k = aci[p];
        for (int32_t q = bbeg[k] + lane; q < bend[k]; q += NT) {
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
                               const double *av, const int32_t *bbeg, const int32_t *bend, const int32_t *bci,
                               const double *bv, RowTables &t, int32_t *counter,
                               const int64_t *obase, int32_t *cci, double *cv, int64_t ub) {
    int32_t u = row_insert<NT>(i, lane, arp, aci, bbeg, bend, bci, t, counter, ub);
    // compact the distinct keys, pad to a power of two, bitonic sort
    if (lane == 0) *counter = 0;
    gsync<NT>();
    for (int32_t s = lane; s < t.hs; s += NT) {
        int32_t k = t.keys[s];
        if (k >= 0) t.list[atomicAdd(counter, 1)] = k;
    }
    int32_t m = 1;
    while (m < u) m <<= 1;
    if (m <= 128) {  // one warp sorts in registers: two barriers instead of one per pass
        gsync<NT>();
        if (m <= 32) block_list_sort_warp<1, NT>(t.list, u, lane);
        else if (m <= 64) block_list_sort_warp<2, NT>(t.list, u, lane);
        else block_list_sort_warp<4, NT>(t.list, u, lane);
        gsync<NT>();
    } else {
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
        for (int32_t q = bbeg[k] + lane; q < bend[k]; q += NT) {
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
                                 const int32_t *bbeg, const int32_t *bend, int64_t *ub) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = 0;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t k = aci[p];
        s += bend[k] - bbeg[k];
    }
    ub[i] = s;
}

constexpr int kBlockHS = 8192, kBlockUmax = 4096, kBlockThreads = 256;
// Row bins by product bound: three register-sort widths (one row per 8, 16
// or 32 lanes), two warp hash-accumulator sizes, a block table, a global table.
constexpr int kNumBins = 7;
constexpr int kSortW0 = 8, kSortW1 = 16, kSortW2 = 32;
constexpr int kAccU0 = 128, kAccU1 = 512;
constexpr int kAccWarps0 = 8, kAccWarps1 = 4;
// bin of a row with product bound u (upper limits 8, 16, 32, 128, 512, 4096)
__device__ __forceinline__ int bin_of(int64_t u) {
    return (u > kSortW0) + (u > kSortW1) + (u > kSortW2) + (u > kAccU0) + (u > kAccU1) + (u > kBlockUmax);
}

// Row counts of the SpGEMM bins, the largest product bound of the last bin
// and the total product bound: read back together in one copy.
struct SpgemmCounts {
    int32_t nb[kNumBins];
    int32_t pad;
    unsigned long long max_ub_global;
    int64_t total_ub;
};

__global__ void bin_rows_kernel(int32_t n, const int64_t *ub, int32_t *bins, SpgemmCounts *cnt) {
    __shared__ int32_t local[kNumBins], base[kNumBins];
    __shared__ unsigned long long lmax;
    if (threadIdx.x < kNumBins) local[threadIdx.x] = 0;
    if (threadIdx.x == 0) lmax = 0ull;
    __syncthreads();
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int b = -1;
    int32_t my = 0;
    if (i < n) {
        int64_t u = ub[i];
        b = bin_of(u);
        my = atomicAdd(&local[b], 1);
        if (b == kNumBins - 1) atomicMax(&lmax, (unsigned long long)u);
    }
    __syncthreads();
    if (threadIdx.x < kNumBins)
        base[threadIdx.x] = local[threadIdx.x] ? atomicAdd(&cnt->nb[threadIdx.x], local[threadIdx.x]) : 0;
    if (threadIdx.x == 0 && lmax) atomicMax(&cnt->max_ub_global, lmax);
    __syncthreads();
    if (b >= 0) bins[(int64_t)b * n + base[b] + my] = i;
}

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Rows with at most W products (W = 8, 16, 32): one row per group of W lanes.
// Every lane holds one product (column j, value a_ik b_kj, index e in the
// order of A's row and then B's row); a bitonic network across the group
// sorts the keys (j, e), so equal columns become adjacent and keep product
// order; the first lane of every run sums its run from 0.0 in that order --
// the dense-accumulator order of the definition, so the result is exact to
// the bit with it.  With KEY32 (every column below 2^27 - 1) the key is one
// 32-bit word, j above the lane index, and only keys move through the
// network: each lane then fetches its product's value from the lane that
// formed it, and a run's head, knowing its run length from the ballot of
// heads, adds the following values without comparing keys again.
// ---------------------------------------------------------------------------
template <int W, bool NUMERIC, bool KEY32>
__global__ void __launch_bounds__(256, 8)  // 32 registers: a full SM of warps to hide the load chains
spgemm_sort_kernel(const int32_t *__restrict__ rows, int32_t nrows, const int32_t *__restrict__ arp,
                   const int32_t *__restrict__ aci, const double *__restrict__ av, const int32_t *__restrict__ bbeg, const int32_t *__restrict__ bend,
                   const int32_t *__restrict__ bci, const double *__restrict__ bv, int32_t *__restrict__ cnt,
                   const int64_t *__restrict__ obase, int32_t *__restrict__ cci, double *__restrict__ cv) {
    constexpr int G = 32 / W;  // rows per warp
    const int lane = threadIdx.x & 31, sl = lane % W, sub = lane / W;
    const unsigned gmask = W == 32 ? kFull : (((1u << W) - 1u) << (sub * W));
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the next iteration's row and its A-row bounds are loaded one iteration
    // ahead, so two of the four dependent loads per row overlap with work
    const int64_t step = nwarps * G;
    int64_t rb = warp * G;
    int32_t i_nx = rb + sub < nrows ? rows[rb + sub] : 0;
    int32_t p0_nx = rb + sub < nrows ? arp[i_nx] : 0, p1_nx = rb + sub < nrows ? arp[i_nx + 1] : 0;
    for (; rb < nrows; rb += step) {
        const int64_t r = rb + sub;
        const bool live = r < nrows;
        const int32_t i = i_nx;
        const int32_t p0 = p0_nx, nA = p1_nx - p0_nx;
        const int64_t rn = rb + step + sub;
        i_nx = rn < nrows ? rows[rn] : 0;
        // expansion: lane sl owns product e = sl (there are at most W)
        bool valid = false;
        int32_t j = 0;
        double val = 0.0;
        int32_t done = 0;  // products of earlier chunks of A's row
        for (int32_t c0 = 0; c0 < nA; c0 += W) {  // uniform within the group
            const int32_t idx = c0 + sl;
            int32_t b0 = 0, len = 0;
            double a = 0.0;
            if (idx < nA) {
                const int32_t k = aci[p0 + idx];
                if (NUMERIC) a = av[p0 + idx];
                b0 = bbeg[k];
                len = bend[k] - b0;
            }
            int32_t incl = len;
#pragma unroll
            for (int o = 1; o < W; o <<= 1) {
                int32_t y = __shfl_up_sync(gmask, incl, o, W);
                if (sl >= o) incl += y;
            }
            const int32_t excl = incl - len;
            const int32_t total = __shfl_sync(gmask, incl, W - 1, W);
            // owner of product e = sl within this chunk: last lane with excl <= e - done
            const int32_t e = sl - done;
            int lo = 0;
#pragma unroll
            for (int st = W / 2; st > 0; st >>= 1) {
                const int cand = lo + st;
                const int32_t ex = __shfl_sync(gmask, excl, cand & (W - 1), W);
                if (cand < W && ex <= e) lo = cand;
            }
            const int32_t kb0 = __shfl_sync(gmask, b0, lo, W);
            const int32_t kex = __shfl_sync(gmask, excl, lo, W);
            const double ka = __shfl_sync(gmask, a, lo, W);
            if (e >= 0 && e < total) {
                const int32_t q = kb0 + (e - kex);
                j = bci[q];
                if (NUMERIC) val = ka * bv[q];
                valid = true;
            }
            done += total;
        }
        p0_nx = rn < nrows ? arp[i_nx] : 0;
        p1_nx = rn < nrows ? arp[i_nx + 1] : 0;
        if constexpr (KEY32) {
            constexpr int LB = W == 8 ? 3 : (W == 16 ? 4 : 5);
            uint32_t key = valid ? (((uint32_t)j << LB) | (uint32_t)sl) : 0xffffffffu;  // empty lanes last
#pragma unroll
            for (int size = 2; size <= W; size <<= 1) {
#pragma unroll
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    const uint32_t ok = __shfl_xor_sync(gmask, key, stride, W);
                    const bool up = (sl & size) == 0;
                    const bool lower = (sl & stride) == 0;
                    key = lower == up ? min(key, ok) : max(key, ok);
                }
            }
            valid = key != 0xffffffffu;
            j = (int32_t)(key >> LB);
            if (NUMERIC) val = __shfl_sync(gmask, val, (int)(key & (uint32_t)(W - 1)), W);
            const int32_t jprev = __shfl_up_sync(gmask, j, 1, W);
            const bool head = valid && (sl == 0 || jprev != j);
            const unsigned hb = (__ballot_sync(gmask, head) & gmask) >> (sub * W);
            const int32_t u = __popc(hb);
            if (NUMERIC) {
                // valid keys form a prefix of the group; a run ends at the next head
                const int nvalid = __popc((__ballot_sync(gmask, valid) & gmask) >> (sub * W));
                int len = 0;
                if (head) {
                    const unsigned later = sl + 1 < 32 ? hb & ~((2u << sl) - 1u) : 0u;
                    len = (later ? __ffs(later) - 1 : nvalid) - sl;
                }
                const int lmax = (int)__reduce_max_sync(kFull, (unsigned)len);  // whole warp: uniform bound
                double acc = f64_zero_plus(val);  // run sums in product order, from 0.0
                for (int d = 1; d < lmax; ++d) {
                    const double vd = __shfl_down_sync(gmask, val, d, W);
                    if (d < len) acc += vd;
                }
                if (head) {
                    const int32_t pos = __popc(hb & ((1u << sl) - 1u));
                    const int64_t cb = obase[i];
                    cci[cb + pos] = j;
                    cv[cb + pos] = acc;
                }
            }
            if (live && sl == 0) cnt[i] = u;
            continue;
        }
        // bitonic sort of (j, e) across the group; empty lanes sort last
        uint64_t key = valid ? (((uint64_t)(uint32_t)j << 8) | (uint64_t)sl) : ~0ull;
#pragma unroll
        for (int size = 2; size <= W; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const uint64_t ok = __shfl_xor_sync(gmask, key, stride, W);
                double ov = 0.0;
                if (NUMERIC) ov = __shfl_xor_sync(gmask, val, stride, W);
                const bool up = (sl & size) == 0;
                const bool lower = (sl & stride) == 0;
                const bool take = lower == up ? ok < key : ok > key;
                if (take) {
                    key = ok;
                    if (NUMERIC) val = ov;
                }
            }
        }
        valid = key != ~0ull;
        j = (int32_t)(key >> 8);
        const int32_t jprev = __shfl_up_sync(gmask, j, 1, W);
        const bool head = valid && (sl == 0 || jprev != j);
        const unsigned hb = (__ballot_sync(gmask, head) & gmask) >> (sub * W);
        const int32_t u = __popc(hb);
        if (NUMERIC) {
            // run sums in product order, from 0.0
            double acc = f64_zero_plus(val);
            bool more = head;
            for (int d = 1; d < W; ++d) {
                if (!__any_sync(gmask, more)) break;
                const double vd = __shfl_down_sync(gmask, val, d, W);
                const uint64_t kd = __shfl_down_sync(gmask, key, d, W);
                if (more) {
                    if (sl + d < W && kd != ~0ull && (int32_t)(kd >> 8) == j) acc += vd;
                    else more = false;
                }
            }
            if (head) {
                const int32_t pos = __popc(hb & ((1u << sl) - 1u));
                const int64_t cb = obase[i];
                cci[cb + pos] = j;
                cv[cb + pos] = acc;
            }
        }
        if (live && sl == 0) cnt[i] = u;
    }
}

// ---------------------------------------------------------------------------
// Rows with at most U products (U = 128, 512): one warp per row with a
// shared hash table of the row's distinct columns and their accumulators.
// Products are generated 32 at a time in product order; within such a round
// the lanes that hold the same column (different k) are found with a match,
// and the first of them adds the round's values to the accumulator one by
// one in lane order -- so every accumulator receives its products in the
// order of A's row, starting from 0.0, as the definition does.  The distinct
// columns are then sorted and written with their sums.
// ---------------------------------------------------------------------------
template <int U> struct AccTab {
    static constexpr int kSlots = 2 * U;
    static constexpr size_t kBytes = (size_t)kSlots * 8 + (size_t)kSlots * 4 + (size_t)U * 4;
    double *val;
    int32_t *keys, *list;
    __device__ AccTab(unsigned char *base) {
        val = reinterpret_cast<double *>(base);
        keys = reinterpret_cast<int32_t *>(base + (size_t)kSlots * 8);
        list = keys + kSlots;
    }
};

// Bitonic sort of 32 R keys held in registers (position p = lane + 32 r),
// ascending: partners in other lanes by shuffles, partners in the same lane
// (strides >= 32) by register swaps -- no shared memory, no warp barriers.
template <int R>
__device__ __forceinline__ void warp_bitonic_sort(int32_t (&k)[R], int lane) {
    constexpr int N = 32 * R;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int rs = stride >> 5;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int pr = r ^ rs;
                    if (pr > r) {
                        const bool asc = ((lane + 32 * r) & size) == 0;
                        const int32_t a = k[r], b = k[pr];
                        const bool sw = (a > b) == asc;
                        k[r] = sw ? b : a;
                        k[pr] = sw ? a : b;
                    }
                }
            } else {
                const bool lower = (lane & stride) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const bool asc = ((lane + 32 * r) & size) == 0;
                    const int32_t y = __shfl_xor_sync(kFull, k[r], stride);
                    k[r] = (lower == asc) ? min(k[r], y) : max(k[r], y);
                }
            }
        }
    }
}

// the row's u <= 32 R distinct columns (t.list[0 .. u)) sorted in registers,
// then written with their accumulated values
template <int R, int U>
__device__ __forceinline__ void warp_emit_sorted(AccTab<U> &t, int32_t u, uint32_t mask, int lane, int64_t cbase,
                                                 int32_t *__restrict__ cci, double *__restrict__ cv) {
    int32_t k[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int p = lane + 32 * r;
        k[r] = p < u ? t.list[p] : INT_MAX;
    }
    warp_bitonic_sort<R>(k, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int p = lane + 32 * r;
        if (p < u) {
            const int32_t j = k[r];
            uint32_t sl = hash32(j) & mask;
            while (t.keys[sl] != j) sl = (sl + 1) & mask;
            cci[cbase + p] = j;
            cv[cbase + p] = t.val[sl];
        }
    }
}

// CAP: a row with more products than the table's distinct capacity U, in
// the table sized for U; the distinct columns are counted after every round
// of at most 32 insertions, and a row that passes U (the table, of 2 U
// slots, then holds at most U + 32 keys, so probing always ends) is given up
// with -1 for the larger-table kernels.  Rows that fit are formed exactly as
// by the unbounded path.
template <int U, bool NUMERIC, bool CAP = false>
__device__ int32_t warp_row_acc(int32_t i, int lane, const int32_t *__restrict__ arp, const int32_t *__restrict__ aci,
                                const double *__restrict__ av, const int32_t *__restrict__ bbeg, const int32_t *__restrict__ bend,
                                const int32_t *__restrict__ bci, const double *__restrict__ bv, AccTab<U> &t,
                                int64_t ub, const int64_t *__restrict__ obase, int32_t *__restrict__ cci,
                                double *__restrict__ cv) {
    const int32_t hs = CAP ? AccTab<U>::kSlots : row_slots(ub, AccTab<U>::kSlots);
    const uint32_t mask = (uint32_t)hs - 1;
    for (int32_t s = lane; s < hs; s += 32) t.keys[s] = -1;
    __syncwarp();
    const int32_t p0 = arp[i], nA = arp[i + 1] - p0;
    int32_t tot = 0;  // CAP: distinct columns so far (the same in every lane)
    // Long rows of B (12 or more products per entry of A's row on average):
    // one round per k, the lanes covering B_k -- columns within a round are
    // distinct, so no matching is needed and rounds follow k's order.  Only
    // for the smaller table: with the large one a warp's shared memory limits
    // residency to a quarter, and the extra rounds' latency then dominates
    // (measured slower).
    const bool per_k = U <= 128 && ub >= 12 * (int64_t)nA;
    int32_t uniq = 0;
    for (int32_t c0 = 0; c0 < nA; c0 += 32) {
        const int32_t idx = c0 + lane;
        int32_t b0 = 0, len = 0;
        double a = 0.0;
        if (idx < nA) {
            const int32_t k = aci[p0 + idx];
            if (NUMERIC) a = av[p0 + idx];
            b0 = bbeg[k];
            len = bend[k] - b0;
        }
        if (per_k) {
            const int kend = min(32, nA - c0);
            for (int kk = 0; kk < kend; ++kk) {
                const int32_t kb0 = __shfl_sync(kFull, b0, kk), klen = __shfl_sync(kFull, len, kk);
                const double ka = __shfl_sync(kFull, a, kk);
                for (int32_t e0 = 0; e0 < klen; e0 += 32) {
                    const int32_t e = e0 + lane;
                    bool fresh = false;
                    if (e < klen) {
                        const int32_t j = bci[kb0 + e];
                        uint32_t sl = hash32(j) & mask;
                        while (true) {
                            const int32_t old = atomicCAS(&t.keys[sl], -1, j);
                            if (old == -1) { fresh = true; break; }
                            if (old == j) break;
                            sl = (sl + 1) & mask;
                        }
                        uniq += fresh;
                        if (NUMERIC) {
                            const double prod = ka * bv[kb0 + e];
                            t.val[sl] = fresh ? f64_zero_plus(prod) : t.val[sl] + prod;
                        }
                    }
                    __syncwarp();
                    if (CAP) {
                        tot += __popc(__ballot_sync(kFull, fresh));
                        if (tot > U) return -1;
                    }
                }
            }
            continue;
        }
        int32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t excl = incl - len;
        const int32_t total = __shfl_sync(kFull, incl, 31);
        for (int32_t eb = 0; eb < total; eb += 32) {
            const int32_t e = eb + lane;
            int lo = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int cand = lo + st;
                const int32_t ex = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && ex <= e) lo = cand;
            }
            const int32_t kb0 = __shfl_sync(kFull, b0, lo);
            const int32_t kex = __shfl_sync(kFull, excl, lo);
            const double ka = __shfl_sync(kFull, a, lo);
            const bool valid = e < total;
            int32_t j = -1 - lane;  // distinct placeholder for empty lanes
            double prod = 0.0;
            if (valid) {
                const int32_t q = kb0 + (e - kex);
                j = bci[q];
                if (NUMERIC) prod = ka * bv[q];
            }
            const unsigned peers = __match_any_sync(kFull, j);
            const bool leader = valid && lane == __ffs(peers) - 1;
            int32_t slot = 0;
            bool fresh = false;
            if (leader) {
                uint32_t sl = hash32(j) & mask;
                while (true) {
                    const int32_t old = atomicCAS(&t.keys[sl], -1, j);
                    if (old == -1) { fresh = true; break; }
                    if (old == j) break;
                    sl = (sl + 1) & mask;
                }
                slot = (int32_t)sl;
                uniq += fresh;
            }
            if (NUMERIC) {
                // the leader adds its peers' values in lane order (itself
                // first); a fresh accumulator starts from 0.0
                double acc = (leader && !fresh) ? t.val[slot] : 0.0;
                bool first = leader && fresh;
                unsigned rest = leader ? peers : 0u;
                const int npeer = __reduce_max_sync(kFull, (unsigned)__popc(rest));
                for (int q = 0; q < npeer; ++q) {
                    const int src = rest ? __ffs(rest) - 1 : lane;
                    const double v = __shfl_sync(kFull, prod, src);
                    if (rest) {
                        acc = first ? f64_zero_plus(v) : acc + v;
                        first = false;
                        rest &= rest - 1u;
                    }
                }
                if (leader) t.val[slot] = acc;
            }
            __syncwarp();
            if (CAP) {
                tot += __popc(__ballot_sync(kFull, fresh));
                if (tot > U) return -1;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) uniq += __shfl_xor_sync(kFull, uniq, o);
    if (!NUMERIC) return uniq;
    const int32_t u = uniq;
    // distinct columns -> list (ballot compaction), pad to a power of two, bitonic sort
    int32_t base = 0;
    for (int32_t s0 = 0; s0 < hs; s0 += 32) {
        const int32_t key = s0 + lane < hs ? t.keys[s0 + lane] : -1;
        const unsigned m = __ballot_sync(kFull, key >= 0);
        if (key >= 0) t.list[base + __popc(m & ((1u << lane) - 1u))] = key;
        base += __popc(m);
    }
    __syncwarp();
    const int64_t cbase = obase[i];
    // up to 128 distinct columns: sorted in registers (the shared-memory
    // network below was most of this kernel's instructions)
    if (u <= 32) { warp_emit_sorted<1, U>(t, u, mask, lane, cbase, cci, cv); __syncwarp(); return u; }
    if (u <= 64) { warp_emit_sorted<2, U>(t, u, mask, lane, cbase, cci, cv); __syncwarp(); return u; }
    if (u <= 128) { warp_emit_sorted<4, U>(t, u, mask, lane, cbase, cci, cv); __syncwarp(); return u; }
    int32_t m2 = 1;
    while (m2 < u) m2 <<= 1;
    for (int32_t r = u + lane; r < m2; r += 32) t.list[r] = INT_MAX;
    __syncwarp();
    for (int32_t size = 2; size <= m2; size <<= 1) {
        for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (int32_t r = lane; r < m2; r += 32) {
                const int32_t partner = r ^ stride;
                if (partner > r) {
                    const bool up = (r & size) == 0;
                    const int32_t x = t.list[r], y = t.list[partner];
                    if ((x > y) == up) { t.list[r] = y; t.list[partner] = x; }
                }
            }
            __syncwarp();
        }
    }
    for (int32_t r = lane; r < u; r += 32) {
        const int32_t j = t.list[r];
        uint32_t sl = hash32(j) & mask;
        while (t.keys[sl] != j) sl = (sl + 1) & mask;
        cci[cbase + r] = j;
        cv[cbase + r] = t.val[sl];
    }
    __syncwarp();
    return u;
}

// Blocks of the small table kept resident per SM: shared memory admits 7,
// and 6 leave 40 registers a thread (at 8 the kernel spills).
#ifndef AMG_ACC_MIN_BLOCKS
#define AMG_ACC_MIN_BLOCKS 6
#endif
// CAP: rows of more than U products whose distinct columns fit the table;
// a row that does not fit is appended to `ovf` (count in *novf) for the
// larger-table kernels.  nrows_dev, when given, holds the row count (a list
// whose length is known on the device only).
template <int U, int WARPS, bool NUMERIC, bool CAP = false>
__global__ void __launch_bounds__(WARPS * 32, U <= 128 ? AMG_ACC_MIN_BLOCKS : 1)
spgemm_acc_kernel(const int32_t *rows, int32_t nrows, const int32_t *arp, const int32_t *aci,
                  const double *av, const int32_t *bbeg, const int32_t *bend, const int32_t *bci, const double *bv,
                  int32_t *cnt, const int64_t *obase, int32_t *cci, double *cv, const int64_t *ub,
                  int32_t *ovf = nullptr, int32_t *novf = nullptr, const int32_t *nrows_dev = nullptr) {
    if (nrows_dev) nrows = *nrows_dev;
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    AccTab<U> t(smem + (size_t)w * AccTab<U>::kBytes);
    const int32_t step = gridDim.x * WARPS;
    int32_t r = blockIdx.x * WARPS + w;
    int32_t i_nx = r < nrows ? rows[r] : 0;  // loaded one row ahead
    int64_t ub_nx = r < nrows ? ub[i_nx] : 0;
    for (; r < nrows; r += step) {
        const int32_t i = i_nx;
        const int64_t ubi = ub_nx;
        if (r + step < nrows) {
            i_nx = rows[r + step];
            ub_nx = ub[i_nx];
        }
        const int32_t u = warp_row_acc<U, NUMERIC, CAP>(i, lane, arp, aci, av, bbeg, bend, bci, bv, t, ubi, obase, cci, cv);
        if (lane == 0) {
            if (CAP && u < 0) ovf[atomicAdd(novf, 1)] = i;
            else cnt[i] = u;
        }
    }
}

template <bool NUMERIC>
__global__ void __launch_bounds__(kBlockThreads)
spgemm_block_kernel(const int32_t *rows, int32_t nrows, const int32_t *arp, const int32_t *aci,
                    const double *av, const int32_t *bbeg, const int32_t *bend, const int32_t *bci, const double *bv,
                    int32_t *cnt, const int64_t *obase, int32_t *cci, double *cv, const int64_t *ub,
                    unsigned char *gscratch, int32_t ghs, int32_t gumax, const int32_t *nrows_dev = nullptr) {
    if (nrows_dev) nrows = *nrows_dev;  // the same for the whole grid
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
            int32_t u = row_numeric<kBlockThreads>(i, threadIdx.x, arp, aci, av, bbeg, bend, bci, bv, t, &counter,
                                                   obase, cci, cv, ub[i]);
            if (threadIdx.x == 0) cnt[i] = u;
        } else {
            int32_t u = row_insert<kBlockThreads>(i, threadIdx.x, arp, aci, bbeg, bend, bci, t, &counter, ub[i]);
            if (threadIdx.x == 0) cnt[i] = u;
        }
    }
}

// ---------------------------------------------------------------------------
// minimal pattern: (i,j) in M iff j in AP[cpts[i]] or i in AP[cpts[j]]
// ---------------------------------------------------------------------------
// The same through the symmetric pattern of Ac: a first pass flags (i, j)
// when j is in AP[cpts[i]] -- one search per entry, in the row shared by the
// lanes of the group -- and the second ORs in the mirrored entry's flag, which
// is the test "i in AP[cpts[j]]".
template <int T>
__global__ void minimal_pattern_rows_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const int32_t *apbeg,
                                            const int32_t *apend, const int32_t *apci, const int32_t *cpts,
                                            uint8_t *first) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    if (i >= n) return;
    const int32_t fi = cpts[i];
    const int32_t b = apbeg[fi], e = apend[fi];
    for (int32_t p = rp[i] + t; p < rp[i + 1]; p += T) first[p] = (uint8_t)contains(apci, b, e, ci[p]);
}

__global__ void mirror_or_kernel(int64_t nnz, const uint8_t *first, const int32_t *tpos, uint8_t *inM) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) inM[p] = first[p] | first[tpos[p]];
}

template <int T>
__global__ void minimal_pattern_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                       const int32_t *apbeg, const int32_t *apend, const int32_t *apci,
                                       const int32_t *cpts, uint8_t *inM) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    if (i >= n) return;
    const int32_t fi = cpts[i];
    for (int32_t p = rp[i] + t; p < rp[i + 1]; p += T) {
        const int32_t j = ci[p];
        const int32_t fj = cpts[j];
        const bool m = contains(apci, apbeg[fi], apend[fi], j) || contains(apci, apbeg[fj], apend[fj], i);
        inM[p] = (uint8_t)m;
    }
}

// ---------------------------------------------------------------------------
// sparsify (Algorithm 3 first loop + Algorithm 3b)
// ---------------------------------------------------------------------------
template <int T>
__global__ void sparsify_flag_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                     const double *v, const uint8_t *inM, double gamma,
                                     double *rowmax, uint8_t *flag) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: the group reduction needs every lane
    int32_t p0 = 0, p1 = 0;
    if (live) { p0 = rp[i]; p1 = rp[i + 1]; }
    int64_t mk = 0;  // key of max |a_ij| over j != i (0: +0.0)
    for (int32_t p = p0 + t; p < p1; p += T)
        if (ci[p] != i) mk = max(mk, f64_abs_key(v[p]));
    mk = group_max_i64<T>(mk);
    if (!live) return;
    const double m = __longlong_as_double(mk);
    if (t == 0) rowmax[i] = m;
    const int64_t tk = f64_abs_key(gamma * m);  // gamma * m >= 0
    for (int32_t p = p0 + t; p < p1; p += T)
        flag[p] = (uint8_t)(ci[p] != i && (inM[p] || f64_abs_key(v[p]) >= tk));
}

template <int T>
__global__ void sparsify_sym_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                    const double *v, const int32_t *tpos, const uint8_t *flag,
                                    const double *rowmax, uint8_t *keep, uint8_t *guard) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: the group reduction needs every lane
    int32_t p0 = 0, p1 = 0;
    if (live) { p0 = rp[i]; p1 = rp[i + 1]; }
    bool any_off = false;
    for (int32_t p = p0 + t; p < p1; p += T) {
        const bool k = ci[p] == i || flag[p] || flag[tpos[p]];
        keep[p] = (uint8_t)k;
        if (k && ci[p] != i) any_off = true;
    }
    any_off = group_any<T>(any_off);
    if (!live || t != 0) return;
    // Algorithm 3b guard, for rows left with no off-diagonal entry: the row
    // sums (in column order) are only needed there
    bool gd = false;
    if (!any_off && f64_key(rowmax[i]) > 0) {
        double rs = 0.0, ra = 0.0;
        for (int32_t p = p0; p < p1; ++p) {
            rs += v[p];
            ra += fabs(v[p]);
        }
        gd = f64_abs_key(rs) <= f64_key(1e-12 * ra);
    }
    guard[i] = (uint8_t)gd;
}

template <int T>
__global__ void sparsify_guard_kernel(int32_t n, const int32_t *rp, const int32_t *ci,
                                      const double *v, const int32_t *tpos, const uint8_t *guard,
                                      const double *rowmax, uint8_t *keep, int32_t *cnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: the group reduction needs every lane
    int32_t p0 = 0, p1 = 0;
    if (live) { p0 = rp[i]; p1 = rp[i + 1]; }
    const bool gi = live && guard[i];
    int32_t c = 0;
    for (int32_t p = p0 + t; p < p1; p += T) {
        const int32_t j = ci[p];
        if (!keep[p] && j != i) {
            if ((gi && f64_abs_key(v[p]) == f64_key(rowmax[i])) ||
                (guard[j] && f64_abs_key(v[tpos[p]]) == f64_key(rowmax[j])))
                keep[p] = 1;
        }
        c += keep[p];
    }
    c = group_sum_i32<T>(c);
    if (live && t == 0) cnt[i] = c;
}

// The same with a group of T lanes per row: chunks of T consecutive entries
// are read together (coalesced), a kept entry's output slot is the row's
// running count plus its place among the chunk's kept entries (ballot), and
// lane 0 adds the chunk's dropped entries to the lumped diagonal in lane
// order -- column order, as the one-thread kernel, so the same bits.
template <int T>
__global__ void __launch_bounds__(kThreads)
sparsify_compact_lanes_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                              const int32_t *diagpos, const uint8_t *keep, const int32_t *hrp, int32_t *hci,
                              double *hv) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    const bool live = i < n;  // no early exit: ballots and shuffles need every lane
    const int lane = threadIdx.x & 31;
    const int first = lane & ~(T - 1);  // the group's first lane in the warp
    const unsigned gbits = T == 32 ? 0xffffffffu : ((1u << T) - 1u);
    int32_t p0 = 0, p1 = 0, out = 0;
    double d = 0.0;
    if (live) {
        p0 = rp[i];
        p1 = rp[i + 1];
        out = hrp[i];
        if (t == 0) d = v[diagpos[i]];
    }
    const int32_t nch = (p1 - p0 + T - 1) / T;
    const int32_t nch_max = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)nch);
    int32_t dpos = -1;
    for (int32_t c = 0; c < nch_max; ++c) {
        const int32_t p = p0 + c * T + t;
        const bool in = live && p < p1;
        bool k = false;
        double a = 0.0;
        int32_t j = 0;
        if (in) {
            a = v[p];
            k = keep[p] != 0;
            j = ci[p];
        }
        const unsigned kb = (__ballot_sync(0xffffffffu, in && k) >> first) & gbits;
        const unsigned db = (__ballot_sync(0xffffffffu, in && !k) >> first) & gbits;
        if (in && k) {
            const int32_t q = out + __popc(kb & ((1u << t) - 1u));
            hci[q] = j;
            hv[q] = a;
            if (j == i) dpos = q;
        }
        out += __popc(kb);
        const int nd = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(db));
        unsigned rest = db;  // the same in every lane of the group
        for (int r = 0; r < nd; ++r) {
            const int src = rest ? first + __ffs(rest) - 1 : lane;
            const double x = __shfl_sync(0xffffffffu, a, src);
            if (rest) {
                if (t == 0) d += x;
                rest &= rest - 1u;
            }
        }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) dpos = max(dpos, __shfl_xor_sync(0xffffffffu, dpos, o, T));
    if (live && t == 0 && dpos >= 0) hv[dpos] = d;  // the diagonal's value last
}

// ---------------------------------------------------------------------------
// Algorithm 3's own loop: full lumping to strong neighbours.  Every dropped
// entry (i,j) becomes a list of "lump edges" (k, t): for each k in
// W = {k : S_jk != 0, (i,k) kept}, t = (|a_jk| / sum_W |a_jm|) a_ij, or one
// fallback edge (~i, a_ij) when W is empty (the value goes to a_ii).  Edges
// are numbered in entry order, each entry's in increasing k -- the order in
// which the sequential loop applies the updates.  Each edge's first update
// lands on the kept position (i,k) (the fallback's on (i,i)); the edges are
// grouped by that position (a counting sort, then each small group ordered
// by edge number), and a kept entry gathers in the loop's order, without
// atomics on values:
//   (r,c), r != c: the group of (r,c) (updates (i,k) from row r) and the
//     group of the mirror (c,r) (updates (k,i) from row c), the lower row's
//     first;
//   (r,r): over the kept columns i of row r in increasing order -- for i = r
//     the group of (r,r): a fallback adds its value, an edge with k = r adds
//     t, adds t, subtracts t (updates (i,k), (k,i), (k,k)); for i != r the
//     group of the mirror (i,r), whose edges have k = r: subtract t (update
//     (k,k)).
// The kept pattern is symmetric (N is), so the mirror position of every kept
// entry exists and row r finds every row that can reach (r,r) among its own
// kept columns.
// ---------------------------------------------------------------------------
// W in increasing k: row j's strong entries merged with row i's sorted
// columns; f(q, pk) for q = position of (j,k), pk = position of (i,k)
template <class F>
__device__ __forceinline__ void walk_w(const int32_t *ci, const uint8_t *keep, const uint8_t *S, int32_t pi0,
                                       int32_t pi1, int32_t pj0, int32_t pj1, F &&f) {
    int32_t a = pi0;
    for (int32_t q = pj0; q < pj1; ++q) {
        if (!S[q]) continue;
        const int32_t k = ci[q];
        while (a < pi1 && ci[a] < k) ++a;
        if (a == pi1) return;
        if (ci[a] == k && keep[a]) f(q, a);
    }
}

// per dropped entry: |W| (edges; 1 for the fallback) and sum_W |a_jm| in
// increasing m
template <int T>
__global__ void lump_count_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                                  const uint8_t *keep, const uint8_t *S, double *den, int32_t *ecnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    if (i >= n) return;
    const int32_t p0 = rp[i], p1 = rp[i + 1];
    for (int32_t p = p0 + t; p < p1; p += T) {
        if (keep[p]) {
            ecnt[p] = 0;
            continue;
        }
        const int32_t j = ci[p];
        double d = 0.0;
        int32_t w = 0;
        walk_w(ci, keep, S, p0, p1, rp[j], rp[j + 1], [&](int32_t q, int32_t) {
            d += fabs(v[q]);
            ++w;
        });
        den[p] = d;
        ecnt[p] = (d > 0.0) ? w : 1;
    }
}

// the edges: ek = k (or ~i for the fallback), et = t, etg = the position of
// the first update's target
template <int T>
__global__ void lump_emit_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                                 const uint8_t *keep, const uint8_t *S, const int32_t *diagpos, const double *den,
                                 const int64_t *eoff, int32_t *ek, double *et, int32_t *etg) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t i = (int32_t)(g / T);
    const int t = (int)(g % T);
    if (i >= n) return;
    const int32_t p0 = rp[i], p1 = rp[i + 1];
    for (int32_t p = p0 + t; p < p1; p += T) {
        if (keep[p]) continue;
        int64_t e = eoff[p];
        const double a = v[p], d = den[p];
        if (!(d > 0.0)) {
            ek[e] = ~i;
            et[e] = a;
            etg[e] = diagpos[i];
            continue;
        }
        const int32_t j = ci[p];
        walk_w(ci, keep, S, p0, p1, rp[j], rp[j + 1], [&](int32_t q, int32_t pk) {
            ek[e] = ci[q];
            et[e] = (fabs(v[q]) / d) * a;
            etg[e] = pk;
            ++e;
        });
    }
}

__global__ void lump_hist_kernel(int64_t E, const int32_t *etg, int32_t *tcnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E) atomicAdd(&tcnt[etg[e]], 1);
}

// unordered placement into the groups (the next kernel orders each group)
__global__ void lump_place_kernel(int64_t E, const int32_t *etg, const int64_t *toff, int32_t *tfill,
                                  int32_t *tlist) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int32_t q = etg[e];
    tlist[toff[q] + atomicAdd(&tfill[q], 1)] = (int32_t)e;
}

// each group in increasing edge number (insertion sort: groups hold a few edges)
__global__ void lump_group_sort_kernel(int64_t nnz, const int64_t *toff, int32_t *tlist) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    const int64_t a = toff[q], b = toff[q + 1];
    for (int64_t s = a + 1; s < b; ++s) {
        const int32_t x = tlist[s];
        int64_t u = s - 1;
        while (u >= a && tlist[u] > x) {
            tlist[u + 1] = tlist[u];
            --u;
        }
        tlist[u + 1] = x;
    }
}

template <int T>
__global__ void lump_gather_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                                   const uint8_t *keep, const int32_t *tpos, const int64_t *toff,
                                   const int32_t *tlist, const int32_t *ek, const double *et, double *hval) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t r = (int32_t)(g / T);
    const int t = (int)(g % T);
    if (r >= n) return;
    const int32_t p0 = rp[r], p1 = rp[r + 1];
    for (int32_t p = p0 + t; p < p1; p += T) {
        if (!keep[p]) continue;
        const int32_t c = ci[p];
        double x = v[p];
        if (c != r) {
            const int32_t first = r < c ? p : tpos[p], second = r < c ? tpos[p] : p;
            for (int64_t s = toff[first]; s < toff[first + 1]; ++s) x += et[tlist[s]];
            for (int64_t s = toff[second]; s < toff[second + 1]; ++s) x += et[tlist[s]];
        } else {
            for (int32_t q = p0; q < p1; ++q) {
                if (!keep[q]) continue;
                if (ci[q] == r) {
                    for (int64_t s = toff[q]; s < toff[q + 1]; ++s) {
                        const int32_t e = tlist[s];
                        const double tt = et[e];
                        if (ek[e] < 0) {
                            x += tt;
                        } else {
                            x += tt;
                            x += tt;
                            x -= tt;
                        }
                    }
                } else {
                    const int32_t m = tpos[q];
                    for (int64_t s = toff[m]; s < toff[m + 1]; ++s) x -= et[tlist[s]];
                }
            }
        }
        hval[p] = x;
    }
}

// compaction of the kept entries with their gathered values
__global__ void compact_values_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const uint8_t *keep,
                                      const double *hval, const int32_t *hrp, int32_t *hci, double *hv) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t pos = hrp[i];
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        if (!keep[p]) continue;
        hci[pos] = ci[p];
        hv[pos] = hval[p];
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

// Small coarsest levels (n <= kSmemCoarse): the Cholesky factor by one block
// in shared memory, then A^{-1} one column per block by two substitutions --
// the global-memory kernels above walk long chains of dependent loads, and
// the triangular inverse and its Gram product would keep a single SM's FP64
// pipe busy for as long again.  The coarsest solve's explicit inverse is
// checked against the oracle's triangular solves within tolerance, so the
// updates use fused multiply-adds and reciprocal square roots.
constexpr int kSmemCoarse = 160;  // n^2 doubles = 200 KB of shared memory

// Right-looking A = L L^T without a column-scaling pass: step j subtracts
// (a_rj / a_jj) a_cj from the trailing entries -- the unscaled column j, so
// its entries need no barrier of their own -- and the columns are scaled by
// 1 / sqrt(a_jj) once at the end.  L (lower, row-major) and 1 / L_jj go out.
__global__ void __launch_bounds__(1024)
coarse_chol_smem_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, double *lout,
                        double *rdiag, int *err) {
    extern __shared__ __align__(16) double a[];
    __shared__ double rpv[kSmemCoarse];
    __shared__ double rinv;
    const int32_t tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int32_t t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = 0.0;
    __syncthreads();
    for (int32_t i = ty; i < n; i += 32)  // one warp per row
        for (int32_t p = rp[i] + tx; p < rp[i + 1]; p += 32) a[i * n + ci[p]] = v[p];
    for (int32_t j = 0; j < n; ++j) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = a[j * n + j];
            if (!(d > 0.0)) { *err = 1; d = 1.0; }
            const double r = rsqrt(d);
            rpv[j] = r;
            rinv = r * r;
        }
        __syncthreads();
        const double ri = rinv;
        for (int32_t r = j + 1 + ty; r < n; r += 32) {
            const double t = a[r * n + j] * ri;
            for (int32_t c = j + 1 + tx; c <= r; c += 32) a[r * n + c] = fma(-t, a[c * n + j], a[r * n + c]);
        }
    }
    __syncthreads();
    for (int32_t t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int32_t r = t / n, c = t % n;
        lout[t] = c < r ? a[t] * rpv[c] : (c == r ? a[t] * rpv[c] : 0.0);  // L_rc = a_rc / sqrt(a_cc)
    }
    for (int32_t j = threadIdx.x; j < n; j += blockDim.x) rdiag[j] = rpv[j];  // 1 / L_jj
}

// Column c of A^{-1}: L y = e_c, then L^T x = y, one block per column with L
// in shared memory; each step finalises one entry (times 1 / L_ii) and
// updates the rest, one barrier a step.  Written as row c (A^{-1} is
// symmetric).
__global__ void __launch_bounds__(128)
coarse_inv_col_kernel(int32_t n, const double *L, const double *rdiag, double *inv) {
    extern __shared__ __align__(16) double sl[];
    double *w = sl + (size_t)n * n, *x = w + n;
    const int32_t c = blockIdx.x;
    for (int32_t t = threadIdx.x; t < n * n; t += blockDim.x) sl[t] = L[t];
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
        w[i] = i == c ? 1.0 : 0.0;
        x[i] = 0.0;
    }
    __syncthreads();
    for (int32_t i = c; i < n; ++i) {  // forward: rows above c stay 0
        const double yi = w[i] * rdiag[i];
        if (threadIdx.x == 0) x[i] = yi;
        for (int32_t r = i + 1 + threadIdx.x; r < n; r += blockDim.x) w[r] = fma(-sl[r * n + i], yi, w[r]);
        __syncthreads();
    }
    for (int32_t i = n - 1; i >= 0; --i) {  // backward into w; L^T's column i is L's row i
        const double xi = x[i] * rdiag[i];
        if (threadIdx.x == 0) w[i] = xi;
        for (int32_t r = threadIdx.x; r < i; r += blockDim.x) x[r] = fma(-sl[i * n + r], xi, x[r]);
        __syncthreads();
    }
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) inv[(size_t)c * n + i] = w[i];
}

__global__ void gram_kernel(int32_t n, const double *Linv, double *inv) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    int32_t i = (int32_t)(t / n), j = (int32_t)(t % n);
    double s = 0.0;
    for (int32_t k = max(i, j); k < n; ++k) s += Linv[(size_t)k * n + i] * Linv[(size_t)k * n + j];
    inv[t] = s;
}

// Gauss-Jordan inverse with partial pivoting (one block): the coarsest-level
// direct solve when the relaxed operator is not positive definite (full
// lumping can make it indefinite).  Pivot: the first row of largest |a_ik|,
// i >= k.  err = 1 if a pivot is 0 (singular operator).
__global__ void __launch_bounds__(1024)
gauss_jordan_kernel(int32_t n, double *a, double *inv, double *fac, int *err) {
    __shared__ double wv[32];
    __shared__ int wi[32];
    __shared__ int piv;
    __shared__ double pv;
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) inv[t] = (t / n == t % n) ? 1.0 : 0.0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int32_t k = 0; k < n; ++k) {
        __syncthreads();
        double bv = -1.0;
        int bi = n;
        for (int32_t i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double x = fabs(a[(size_t)i * n + k]);
            if (x > bv) { bv = x; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { wv[w] = bv; wi[w] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int bix = n;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
                if (wv[q] > b || (wv[q] == b && wi[q] < bix)) { b = wv[q]; bix = wi[q]; }
            piv = bix < n ? bix : k;
            pv = a[(size_t)piv * n + k];
            if (!(fabs(pv) > 0.0)) *err = 1;
        }
        __syncthreads();
        if (!(fabs(pv) > 0.0)) return;  // uniform: every thread reads the same pivot
        const int32_t r = piv;
        if (r != k)
            for (int32_t c = threadIdx.x; c < n; c += blockDim.x) {
                double t = a[(size_t)k * n + c]; a[(size_t)k * n + c] = a[(size_t)r * n + c]; a[(size_t)r * n + c] = t;
                t = inv[(size_t)k * n + c]; inv[(size_t)k * n + c] = inv[(size_t)r * n + c]; inv[(size_t)r * n + c] = t;
            }
        __syncthreads();
        for (int32_t c = threadIdx.x; c < n; c += blockDim.x) {
            a[(size_t)k * n + c] /= pv;
            inv[(size_t)k * n + c] /= pv;
        }
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) fac[i] = (i == k) ? 0.0 : a[(size_t)i * n + k];
        __syncthreads();
        for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
            const int32_t i = (int32_t)(t / n), c = (int32_t)(t % n);
            const double f = fac[i];
            if (f == 0.0) continue;
            if (c >= k) a[t] -= f * a[(size_t)k * n + c];
            inv[t] -= f * inv[(size_t)k * n + c];
        }
    }
}

// copy each row's entries from its product-bound slot to the final CSR
// compaction of the product-bound slots: eight lanes per row
constexpr int kCompactLanes = 8;
// row i of a product left in its slots: [obase_i, obase_i + count_i)
__global__ void slot_bounds_kernel(int32_t n, const int64_t *obase, const int32_t *cnt, int32_t *beg, int32_t *end) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = (int32_t)obase[i];
    beg[i] = b;
    end[i] = b + cnt[i];
}

__global__ void spgemm_compact_kernel(int32_t n, const int64_t *obase, const int32_t *crp, const int32_t *tci,
                                      const double *tv, int32_t *cci, double *cv) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t i = (int32_t)(g / kCompactLanes);
    int lane = (int)(g % kCompactLanes);
    if (i >= n) return;
    int64_t src = obase[i];
    int32_t dst = crp[i], len = crp[i + 1] - crp[i];
    for (int32_t e = lane; e < len; e += kCompactLanes) {
        cci[dst + e] = tci[src + e];
        cv[dst + e] = tv[src + e];
    }
}

}  // namespace

// lanes per row for the row kernels: the power of two (2..cap) at or above
// half the mean row length (about two entries per lane)
static int row_lanes(const DevCSR &A, int cap = 32) {
    const double half = A.nrows > 0 ? 0.5 * (double)A.nnz / (double)A.nrows : 0.0;
    int T = 2;
    while (T < cap && (double)T < half) T <<= 1;
    return T;
}
template <class F> static void with_row_lanes(int T, F &&f) {
    switch (T) {
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 16: f(std::integral_constant<int, 16>{}); break;
        default: f(std::integral_constant<int, 32>{}); break;
    }
}

// ===========================================================================
// host entry points
// ===========================================================================
// Validation and transpose positions in one pass over the stream with one
// read-back.  The transpose-position kernel checks every column index itself
// before following it, so it is safe on a matrix that fails validation.
void level_maps(const DevCSR &A, int32_t *diagpos, int32_t *tpos, cudaStream_t s, bool check) {
    TmpBuf err(sizeof(int), s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    if (A.nrows > 0) {
        with_row_lanes(row_lanes(A), [&](auto tc) {
            constexpr int L = decltype(tc)::value;
            const int gl = div_up((int64_t)A.nrows * L, kThreads);
            if (A.nrows == A.ncols)
                validate_kernel<L, true><<<gl, kThreads, 0, s>>>(A.nrows, A.ncols, A.nnz, A.rp(), A.ci(), A.v(),
                                                                 diagpos, tpos, err.as<int>());
            else
                validate_kernel<L, false><<<gl, kThreads, 0, s>>>(A.nrows, A.ncols, A.nnz, A.rp(), A.ci(), A.v(),
                                                                  diagpos, nullptr, err.as<int>());
            ::amg::count_launch();
        });
    }
    AMG_CHECK_LAUNCH();
    if (!check) return;  // an operator this library formed: sorted, symmetric pattern by construction
    int e = read_scalar(err.as<int>(), s);
    if (e) {
        std::string m = "invalid matrix:";
        if (e & kBadCol) m += " column index out of range;";
        if (e & kUnsorted) m += " columns not strictly increasing;";
        if (e & kNoDiag) m += " missing diagonal;";
        if (e & kBadDiag) m += " non-positive diagonal;";
        if (e & kNonFinite) m += " non-finite value;";
        if (e & kAsym) m += " sparsity pattern is not symmetric;";
        if (e & kBadRowptr) m += " row pointers out of order or out of [0, nnz];";
        throw Error(AMG_ERR_INVALID, m);
    }
    require(A.nrows == A.ncols, "invalid matrix: not square");
}

// rectangular operators given by the caller (interpolation): row pointers,
// column range, strictly increasing columns, finite values
__global__ void validate_rect_kernel(int32_t n, int32_t ncols, int64_t nnz, const int32_t *rp, const int32_t *ci,
                                     const double *v, int *err) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = 0;
    const int32_t p0 = rp[i], p1 = rp[i + 1];
    if ((i == 0 && p0 != 0) || (i == n - 1 && (int64_t)p1 != nnz)) e |= kBadRowptr;
    if (!row_in_bounds(p0, p1, nnz)) { atomicOr(err, e | kBadRowptr); return; }
    int32_t prev = -1;
    for (int32_t p = p0; p < p1; ++p) {
        const int32_t j = ci[p];
        if (j < 0 || j >= ncols) { e |= kBadCol; continue; }
        if (j <= prev) e |= kUnsorted;
        prev = j;
        if (!isfinite(v[p])) e |= kNonFinite;
    }
    if (e) atomicOr(err, e);
}

void validate_rect(const DevCSR &M, const char *what, cudaStream_t s) {
    TmpBuf err(sizeof(int), s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    if (M.nrows > 0)
        { validate_rect_kernel<<<div_up(M.nrows, kThreads), kThreads, 0, s>>>(
            M.nrows, M.ncols, M.nnz, M.rp(), M.ci(), M.v(), err.as<int>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    int e = read_scalar(err.as<int>(), s);
    if (e) {
        std::string m = std::string("invalid ") + what + ":";
        if (e & kBadCol) m += " column index out of range;";
        if (e & kUnsorted) m += " columns not strictly increasing;";
        if (e & kNonFinite) m += " non-finite value;";
        if (e & kBadRowptr) m += " row pointers out of order or out of [0, nnz];";
        throw Error(AMG_ERR_INVALID, m);
    }
}

void strength(const DevCSR &A, double theta, uint8_t *strong, cudaStream_t s) {
    if (A.nrows == 0) return;
    with_row_lanes(row_lanes(A), [&](auto tc) {
        constexpr int L = decltype(tc)::value;
        strength_kernel<L><<<div_up((int64_t)A.nrows * L, kThreads), kThreads, 0, s>>>(A.nrows, A.rp(), A.ci(),
                                                                                   A.v(), theta, strong);
        ::amg::count_launch();
    });
    AMG_CHECK_LAUNCH();
}

int64_t pmis(const DevCSR &A, const uint8_t *strong, const int32_t *tpos, uint64_t seed,
             int32_t level, int8_t *cf, int32_t *cmap, cudaStream_t s) {
    int32_t n = A.nrows;
    if (n == 0) {
        AMG_CUDA(cudaMemsetAsync(cmap, 0, sizeof(int32_t), s));
        return 0;
    }
    // eight rounds per read-back: the levels of the test problems finish
    // within one batch, and a round whose list is empty costs one short launch
    constexpr int kBatch = 8, kMaxRounds = 10000;
    // cnt[0]: C points so far; dc = cnt + 1: dc[0] undecided after the
    // initial split, dc[r] after round r (the first batch reads the C count
    // with the round counts); the undecided rows alternate between two lists
    TmpBuf w(sizeof(double) * n, s), newc(n, s), cnt(sizeof(int) * (kMaxRounds + 2), s), sym(A.nnz + 1, s),
        lists(sizeof(int32_t) * 2 * (size_t)n, s);
    int *ccount = cnt.as<int>();
    int *dc = ccount + 1;
    int32_t *list[2] = {lists.as<int32_t>(), lists.as<int32_t>() + n};
    int g = div_up(n, kThreads);
    const int T = row_lanes(A, 8);
    const int64_t nres = ::amg::resident_blocks(kThreads);
    AMG_CUDA(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    with_row_lanes(T, [&](auto tc) {
        constexpr int L = decltype(tc)::value;
        pmis_init_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(
            n, A.rp(), tpos, strong, seed, level, w.as<double>(), cf, dc, sym.as<uint8_t>(), list[0]);
        ::amg::count_launch();
    });
    AMG_CHECK_LAUNCH();
    int done = 0;   // rounds launched
    int last = n;   // bound on the list length at the start of the batch
    bool first = true;
    int64_t nc = -1;  // C points, when the first batch finished the split
    while (true) {
        if (done + kBatch > kMaxRounds) throw Error(AMG_ERR_CUDA, "PMIS did not terminate");
        const int64_t bound = std::max(last, 1);
        for (int b = 0; b < kBatch; ++b) {
            const int r = done + b + 1;
            const int32_t *cur = list[(r - 1) & 1];
            int32_t *nxt = list[r & 1];
            with_row_lanes(T, [&](auto tc) {
                constexpr int L = decltype(tc)::value;
                if (r == 1) {  // every row, undecided or not (the list holds nearly all of them)
                    const int gl = (int)std::min<int64_t>(div_up((int64_t)n * L, kThreads), nres);
                    pmis_select_kernel<L, true><<<gl, kThreads, 0, s>>>(
                        cur, dc + r - 1, n, A.rp(), A.ci(), sym.as<uint8_t>(), w.as<double>(), cf, newc.as<uint8_t>());
                    ::amg::count_launch();
                    pmis_apply_kernel<L, true><<<gl, kThreads, 0, s>>>(cur, dc + r - 1, n, A.rp(), A.ci(), strong,
                                                                       newc.as<uint8_t>(), cf, nxt, dc + r, ccount);
                    ::amg::count_launch();
                    return;
                }
                const int gl = (int)std::min<int64_t>(div_up(bound * L, kThreads), nres);
                pmis_select_kernel<L, false><<<gl, kThreads, 0, s>>>(
                    cur, dc + r - 1, n, A.rp(), A.ci(), sym.as<uint8_t>(), w.as<double>(), cf, newc.as<uint8_t>());
                ::amg::count_launch();
                pmis_apply_kernel<L, false><<<gl, kThreads, 0, s>>>(cur, dc + r - 1, n, A.rp(), A.ci(), strong,
                                                                    newc.as<uint8_t>(), cf, nxt, dc + r, ccount);
                ::amg::count_launch();
            });
        }
        AMG_CHECK_LAUNCH();
        int hc[kBatch + 1];
        if (first) {  // the C count comes with the first batch (usually the only one)
            int hb[kBatch + 2];
            read_back(hb, ccount, sizeof(hb), s);
            nc = hb[0];
            std::memcpy(hc, hb + 1, sizeof(hc));
        } else {
            read_back(hc, dc + done, sizeof(hc), s);
            nc = -1;
        }
        if (!first && hc[0] != last) throw Error(AMG_ERR_CUDA, "PMIS counters inconsistent");
        // every round that started with undecided points must have decided some
        for (int b = 0; b < kBatch; ++b)
            if (hc[b] > 0 && hc[b + 1] >= hc[b]) throw Error(AMG_ERR_CUDA, "PMIS made no progress");
        first = false;
        done += kBatch;
        last = hc[kBatch];
        if (hc[kBatch] == 0) break;
    }
    TmpBuf flag(sizeof(int32_t) * n, s);
    { is_c_kernel<<<g, kThreads, 0, s>>>(n, cf, flag.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    if (nc < 0) return exclusive_scan_i32(flag.as<int32_t>(), cmap, n, s);  // more than one batch
    exclusive_scan_i32_known(flag.as<int32_t>(), cmap, n, s);  // its total is the C count read back
    return nc;
}

void coarse_points(const int8_t *cf, int32_t n, int32_t *cmap, int32_t *cpts, cudaStream_t s) {
    if (n == 0) return;
    { cmap_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, cf, cmap, cpts); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
}

void coarse_map(const int8_t *cf, int32_t n, int32_t *cmap, int32_t *cpts, int64_t nc, cudaStream_t s) {
    if (n == 0) return;
    TmpBuf flag(sizeof(int32_t) * n, s);
    int g = div_up(n, kThreads);
    { is_c_kernel<<<g, kThreads, 0, s>>>(n, cf, flag.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    // cmap has n+1 slots: exclusive scan of the C flags
    const int64_t c = exclusive_scan_i32(flag.as<int32_t>(), cmap, n, s);
    if (c != nc) throw Error(AMG_ERR_INVALID, "C/F markers: the number of C points differs from the coarse size");
    coarse_points(cf, n, cmap, cpts, s);
}

void direct_interp(const DevCSR &A, const uint8_t *strong, const int8_t *cf, const int32_t *cmap,
                   int32_t nc, DevCSR &P, cudaStream_t s) {
    int32_t n = A.nrows;
    TmpBuf cnt(sizeof(int32_t) * (n + 1), s);
    P.rowptr.alloc(sizeof(int32_t) * (n + 1));
    int g = div_up(n, kThreads);
    if (n > 0)
        with_row_lanes(row_lanes(A), [&](auto tc) {
            constexpr int L = decltype(tc)::value;
            interp_count_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(n, A.rp(), A.ci(), strong, cf,
                                                                                       cnt.as<int32_t>());
            ::amg::count_launch();
        });
    AMG_CHECK_LAUNCH();
    int64_t nnz = exclusive_scan_i32(cnt.as<int32_t>(), P.rp(), n, s);
    P.nrows = n;
    P.ncols = nc;
    P.nnz = nnz;
    P.col.alloc(sizeof(int32_t) * (nnz + kPad));
    P.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(P.ci() + nnz, 0, sizeof(int32_t) * kPad, s));  // the fill writes rows [0, nnz)
    AMG_CUDA(cudaMemsetAsync(P.v() + nnz, 0, sizeof(double) * kPad, s));
    if (n > 0) {
        TmpBuf prow(sizeof(int32_t) * (nnz + 1), s), coef(sizeof(double) * 3 * (size_t)n, s);
        { interp_rows_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), strong, cf, cmap, P.rp(), P.ci(),
                                                  P.v(), prow.as<int32_t>(), coef.as<double>()); ::amg::count_launch(); }
        if (nnz > 0)
            { interp_weights_kernel<<<div_up(nnz, kThreads), kThreads, 0, s>>>(nnz, prow.as<int32_t>(),
                                                                             coef.as<double>(), P.v()); ::amg::count_launch(); }
    }
    AMG_CHECK_LAUNCH();
}

void transpose(const DevCSR &M, DevCSR &T, cudaStream_t s) {
    int32_t m = M.ncols;
    TmpBuf cnt(sizeof(int32_t) * (m + 1), s), fill(sizeof(int32_t) * (m + 1), s);
    AMG_CUDA(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    if (M.nnz > 0) { col_count_kernel<<<div_up(M.nnz, kThreads), kThreads, 0, s>>>(M.nnz, M.ci(), cnt.as<int32_t>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    T.rowptr.alloc(sizeof(int32_t) * (m + 1));
    const int64_t nnz = M.nnz;  // every entry moves: no read-back of the scan total
    exclusive_scan_i32_known(cnt.as<int32_t>(), T.rp(), m, s);
    T.nrows = m;
    T.ncols = M.nrows;
    T.nnz = nnz;
    T.col.alloc(sizeof(int32_t) * (nnz + kPad));
    T.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(T.ci() + nnz, 0, sizeof(int32_t) * kPad, s));  // the fill writes [0, nnz)
    AMG_CUDA(cudaMemsetAsync(T.v() + nnz, 0, sizeof(double) * kPad, s));
    AMG_CUDA(cudaMemcpyAsync(fill.ptr, T.rp(), sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToDevice, s));
    if (M.nrows > 0)
        { transpose_fill_kernel<<<div_up(M.nrows, kThreads), kThreads, 0, s>>>(
            M.nrows, M.rp(), M.ci(), M.v(), fill.as<int32_t>(), T.ci(), T.v()); ::amg::count_launch(); }
    if (m > 0) {
        const double mean = (double)nnz / (double)m;
        int W = 2;
        while (W < 32 && (double)W < mean) W <<= 1;
        with_row_lanes(W, [&](auto tc) {
            constexpr int L = decltype(tc)::value;
            sort_rows_kernel<L><<<div_up((int64_t)m * L, kThreads), kThreads, 0, s>>>(m, T.rp(), T.ci(), T.v());
            ::amg::count_launch();
        });
    }
    AMG_CHECK_LAUNCH();
}

static int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// The shared driver: C = A B into Cm (CSR), or -- with slots given and the
// one-pass form available -- left in its product slots.
static void spgemm_impl(const DevCSR &A, const SpRows &B, DevCSR &Cm, SlotProduct *slots, cudaStream_t s) {
    require(A.ncols == B.nrows, "spgemm: inner dimensions differ");
    if (slots) slots->rows = SpRows{};
    int32_t n = A.nrows;
    Cm.nrows = n;
    Cm.ncols = B.ncols;
    if (n == 0) {
        Cm.rowptr.alloc(sizeof(int32_t) * (n + 1));
        Cm.nnz = 0;
        AMG_CUDA(cudaMemsetAsync(Cm.rowptr.ptr, 0, sizeof(int32_t), s));
        Cm.col.alloc(sizeof(int32_t) * kPad);
        Cm.val.alloc(sizeof(double) * kPad);
        return;
    }
    TmpBuf ub(sizeof(int64_t) * n, s), bins(sizeof(int32_t) * kNumBins * (size_t)n, s),
        dcounts(sizeof(SpgemmCounts), s), cnt(sizeof(int32_t) * (n + 1), s), obase(sizeof(int64_t) * (n + 1), s);
    int g = div_up(n, kThreads);
    SpgemmCounts *dc = dcounts.as<SpgemmCounts>();
    { spgemm_ub_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), B.beg, B.end, ub.as<int64_t>()); ::amg::count_launch(); }
    AMG_CUDA(cudaMemsetAsync(dcounts.ptr, 0, sizeof(SpgemmCounts), s));
    { bin_rows_kernel<<<g, kThreads, 0, s>>>(n, ub.as<int64_t>(), bins.as<int32_t>(), dc); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    // product-bound offsets of the one-pass numeric kernel (total into the same record)
    exclusive_scan_i64_async(ub.as<int64_t>(), obase.as<int64_t>(), n, &dc->total_ub, s);
    SpgemmCounts hc;
    static_assert(sizeof(SpgemmCounts) <= kReadBackMax, "SpgemmCounts read back in one piece");
    read_back(&hc, dc, sizeof(hc), s);
    const int32_t *nb = hc.nb;
    const int64_t max_ub = (int64_t)hc.max_ub_global;
    const int64_t total_ub = hc.total_ub;
    auto rows_of = [&](int b) { return bins.as<int32_t>() + (size_t)b * n; };
    constexpr size_t acc0_smem = (size_t)kAccWarps0 * AccTab<kAccU0>::kBytes;
    constexpr size_t acc1_smem = (size_t)kAccWarps1 * AccTab<kAccU1>::kBytes;
    constexpr size_t block_smem = (size_t)kBlockHS * 8 + (size_t)kBlockUmax * 12;
    static std::atomic<bool> attrs[64];
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    if (dev >= 64 || !attrs[dev].load()) {
        AMG_CUDA(cudaFuncSetAttribute(spgemm_acc_kernel<kAccU0, kAccWarps0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc0_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_acc_kernel<kAccU0, kAccWarps0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc0_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_acc_kernel<kAccU0, kAccWarps0, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc0_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_acc_kernel<kAccU0, kAccWarps0, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc0_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_acc_kernel<kAccU1, kAccWarps1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc1_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_acc_kernel<kAccU1, kAccWarps1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc1_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem));
        AMG_CUDA(cudaFuncSetAttribute(spgemm_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem));
        if (dev < 64) attrs[dev].store(true);
    }
    const int nres = ::amg::resident_blocks(256);  // blocks of 256 threads that fit at once
    int64_t gumax = next_pow2(std::max<int64_t>(max_ub, 1));
    int64_t ghs = 2 * gumax;
    int gblocks = 0;
    TmpBuf gscr;
    if (nb[kNumBins - 1] > 0) {
        size_t per = (size_t)ghs * 8 + (size_t)gumax * 12;
        int64_t cap = std::max<int64_t>(1, (int64_t)(((size_t)2 << 30) / per));  // <= 2 GiB scratch
        gblocks = (int)std::min<int64_t>({(int64_t)nb[kNumBins - 1], 304, cap});
        gscr.alloc(per * gblocks, s);
    }
    const int64_t *ubp = ub.as<int64_t>();
    const bool key32 = B.ncols < (1 << 27) - 1;  // a column and a lane index in one 32-bit sort key
    // launch(numeric, obase, out_cols, out_vals): one pass over the bins
    auto launch = [&](bool numeric, const int64_t *ob, int32_t *cc, double *cvv) {
        int32_t *cp = cnt.as<int32_t>();
        auto sort_bin = [&](auto kern_num, auto kern_sym, int b, int W) {
            if (nb[b] == 0) return;
            const int64_t warps = ((int64_t)nb[b] * W + 31) / 32;
            const int blocks = (int)std::min<int64_t>((warps + 7) / 8, nres);
            if (numeric)
                { kern_num<<<blocks, 256, 0, s>>>(rows_of(b), nb[b], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv); ::amg::count_launch(); }
            else
                { kern_sym<<<blocks, 256, 0, s>>>(rows_of(b), nb[b], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv); ::amg::count_launch(); }
        };
        if (key32) {
            sort_bin(spgemm_sort_kernel<kSortW0, true, true>, spgemm_sort_kernel<kSortW0, false, true>, 0, kSortW0);
            sort_bin(spgemm_sort_kernel<kSortW1, true, true>, spgemm_sort_kernel<kSortW1, false, true>, 1, kSortW1);
            sort_bin(spgemm_sort_kernel<kSortW2, true, true>, spgemm_sort_kernel<kSortW2, false, true>, 2, kSortW2);
        } else {
            sort_bin(spgemm_sort_kernel<kSortW0, true, false>, spgemm_sort_kernel<kSortW0, false, false>, 0, kSortW0);
            sort_bin(spgemm_sort_kernel<kSortW1, true, false>, spgemm_sort_kernel<kSortW1, false, false>, 1, kSortW1);
            sort_bin(spgemm_sort_kernel<kSortW2, true, false>, spgemm_sort_kernel<kSortW2, false, false>, 2, kSortW2);
        }
        if (nb[3] > 0) {
            const int blocks = std::min(div_up(nb[3], kAccWarps0), 152 * 16);
            if (numeric)
                { spgemm_acc_kernel<kAccU0, kAccWarps0, true><<<blocks, kAccWarps0 * 32, acc0_smem, s>>>(
                    rows_of(3), nb[3], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv, ubp); ::amg::count_launch(); }
            else
                { spgemm_acc_kernel<kAccU0, kAccWarps0, false><<<blocks, kAccWarps0 * 32, acc0_smem, s>>>(
                    rows_of(3), nb[3], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv, ubp); ::amg::count_launch(); }
        }
        // rows of more than 128 products: first in the small table (a warp per
        // row, a full SM of warps -- the distinct columns of such rows are
        // usually far fewer than their products); the rows whose distinct
        // columns pass 128 go on to their bin's larger table
        if (nb[4] > 0 || nb[5] > 0 || nb[6] > 0) {
            TmpBuf ovf(sizeof(int32_t) * ((size_t)nb[4] + nb[5] + nb[6] + 1), s), novf(3 * sizeof(int32_t), s);
            int32_t *ovf4 = ovf.as<int32_t>(), *ovf5 = ovf4 + nb[4], *ovf6 = ovf5 + nb[5], *nov = novf.as<int32_t>();
            AMG_CUDA(cudaMemsetAsync(nov, 0, 3 * sizeof(int32_t), s));
            for (int bin : {4, 5, 6}) {
                if (nb[bin] == 0) continue;
                int32_t *list = bin == 4 ? ovf4 : (bin == 5 ? ovf5 : ovf6);
                const int blocks = std::min(div_up(nb[bin], kAccWarps0), 152 * 16);
                if (numeric)
                    { spgemm_acc_kernel<kAccU0, kAccWarps0, true, true><<<blocks, kAccWarps0 * 32, acc0_smem, s>>>(
                        rows_of(bin), nb[bin], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv, ubp,
                        list, nov + (bin - 4)); ::amg::count_launch(); }
                else
                    { spgemm_acc_kernel<kAccU0, kAccWarps0, false, true><<<blocks, kAccWarps0 * 32, acc0_smem, s>>>(
                        rows_of(bin), nb[bin], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv, ubp,
                        list, nov + (bin - 4)); ::amg::count_launch(); }
            }
            if (nb[4] > 0) {
                const int blocks = std::min(div_up(nb[4], kAccWarps1), 152 * 16);
                if (numeric)
                    { spgemm_acc_kernel<kAccU1, kAccWarps1, true><<<blocks, kAccWarps1 * 32, acc1_smem, s>>>(
                        ovf4, nb[4], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv, ubp,
                        nullptr, nullptr, nov); ::amg::count_launch(); }
                else
                    { spgemm_acc_kernel<kAccU1, kAccWarps1, false><<<blocks, kAccWarps1 * 32, acc1_smem, s>>>(
                        ovf4, nb[4], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv, ubp,
                        nullptr, nullptr, nov); ::amg::count_launch(); }
            }
            if (nb[5] > 0) {
                const int blocks = std::min(nb[5], 152 * 4);
                if (numeric)
                    { spgemm_block_kernel<true><<<blocks, kBlockThreads, block_smem, s>>>(
                        ovf5, nb[5], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv,
                        ubp, nullptr, 0, 0, nov + 1); ::amg::count_launch(); }
                else
                    { spgemm_block_kernel<false><<<blocks, kBlockThreads, block_smem, s>>>(
                        ovf5, nb[5], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv,
                        ubp, nullptr, 0, 0, nov + 1); ::amg::count_launch(); }
            }
            if (nb[6] > 0) {
                if (numeric)
                    { spgemm_block_kernel<true><<<gblocks, kBlockThreads, 0, s>>>(
                        ovf6, nb[6], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv,
                        ubp, gscr.as<unsigned char>(), (int32_t)ghs, (int32_t)gumax, nov + 2); ::amg::count_launch(); }
                else
                    { spgemm_block_kernel<false><<<gblocks, kBlockThreads, 0, s>>>(
                        ovf6, nb[6], A.rp(), A.ci(), A.v(), B.beg, B.end, B.ci, B.v, cp, ob, cc, cvv,
                        ubp, gscr.as<unsigned char>(), (int32_t)ghs, (int32_t)gumax, nov + 2); ::amg::count_launch(); }
            }
        }
        AMG_CHECK_LAUNCH();
    };
    // one numeric pass into slots sized by each row's product bound, then a
    // compaction -- unless the bound does not fit: then count first (symbolic)
    size_t fr = 0, tot = 0;
    if ((double)total_ub * 12.0 > (double)((size_t)1 << 30)) AMG_CUDA(cudaMemGetInfo(&fr, &tot));  // only when it may matter
    else fr = (size_t)1 << 40;
    // AMG_SPGEMM_TWO_PASS=1 forces the counting path (it is otherwise taken
    // only when the product bound would not fit in free memory)
    const char *force = std::getenv("AMG_SPGEMM_TWO_PASS");
    bool one_pass = (double)total_ub * 12.0 < 0.4 * (double)fr && !(force && force[0] == '1');
    int64_t nnz;
    if (one_pass && slots && total_ub < ((int64_t)1 << 31) - kPad) {
        // the rows stay where the numeric pass wrote them: no count scan, no compaction
        SlotProduct &P = *slots;
        P.ci.alloc(sizeof(int32_t) * (total_ub + kPad), s);
        P.v.alloc(sizeof(double) * (total_ub + kPad), s);
        P.beg.alloc(sizeof(int32_t) * (n + 1), s);
        P.end.alloc(sizeof(int32_t) * (n + 1), s);
        launch(true, obase.as<int64_t>(), P.ci.as<int32_t>(), P.v.as<double>());
        { slot_bounds_kernel<<<g, kThreads, 0, s>>>(n, obase.as<int64_t>(), cnt.as<int32_t>(), P.beg.as<int32_t>(),
                                                   P.end.as<int32_t>()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        P.rows = SpRows{P.beg.as<int32_t>(), P.end.as<int32_t>(), P.ci.as<int32_t>(), P.v.as<double>(), n, B.ncols};
        return;
    }
    if (one_pass) {
        TmpBuf tci(sizeof(int32_t) * (total_ub + kPad), s), tv(sizeof(double) * (total_ub + kPad), s);
        launch(true, obase.as<int64_t>(), tci.as<int32_t>(), tv.as<double>());
        Cm.rowptr.alloc(sizeof(int32_t) * (n + 1));
        nnz = exclusive_scan_i32(cnt.as<int32_t>(), Cm.rp(), n, s);
        require(nnz < ((int64_t)1 << 31), "spgemm: product has 2^31 or more entries");
        Cm.nnz = nnz;
        Cm.col.alloc(sizeof(int32_t) * (nnz + kPad));
        Cm.val.alloc(sizeof(double) * (nnz + kPad));
        AMG_CUDA(cudaMemsetAsync(Cm.ci() + nnz, 0, sizeof(int32_t) * kPad, s));
        AMG_CUDA(cudaMemsetAsync(Cm.v() + nnz, 0, sizeof(double) * kPad, s));
        { spgemm_compact_kernel<<<div_up((int64_t)n * kCompactLanes, 256), 256, 0, s>>>(n, obase.as<int64_t>(), Cm.rp(), tci.as<int32_t>(), tv.as<double>(), Cm.ci(), Cm.v()); ::amg::count_launch(); }
        AMG_CHECK_LAUNCH();
        return;  // the temporaries' stream-ordered frees follow the compaction
    }
    launch(false, nullptr, nullptr, nullptr);
    Cm.rowptr.alloc(sizeof(int32_t) * (n + 1));
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

void spgemm(const DevCSR &A, const SpRows &B, DevCSR &C, cudaStream_t s) { spgemm_impl(A, B, C, nullptr, s); }

void spgemm_slots(const DevCSR &A, const DevCSR &B, SlotProduct &C, cudaStream_t s) {
    spgemm_impl(A, rows_of(B), C.csr, &C, s);
    if (!C.rows.beg) C.rows = rows_of(C.csr);  // formed as CSR (empty, or too large for its slots)
}

void minimal_pattern(const DevCSR &Ac, const SpRows &AP, const int32_t *cpts, uint8_t *inM, cudaStream_t s,
                     const int32_t *tpos) {
    if (Ac.nrows == 0) return;
    if (tpos) {
        TmpBuf first(Ac.nnz + 1, s);
        with_row_lanes(row_lanes(Ac), [&](auto tc) {
            constexpr int L = decltype(tc)::value;
            minimal_pattern_rows_kernel<L><<<div_up((int64_t)Ac.nrows * L, kThreads), kThreads, 0, s>>>(
                Ac.nrows, Ac.rp(), Ac.ci(), AP.beg, AP.end, AP.ci, cpts, first.as<uint8_t>());
            ::amg::count_launch();
        });
        if (Ac.nnz > 0) {
            mirror_or_kernel<<<div_up(Ac.nnz, kThreads), kThreads, 0, s>>>(Ac.nnz, first.as<uint8_t>(), tpos, inM);
            ::amg::count_launch();
        }
        AMG_CHECK_LAUNCH();
        return;
    }
    with_row_lanes(row_lanes(Ac), [&](auto tc) {
        constexpr int L = decltype(tc)::value;
        minimal_pattern_kernel<L><<<div_up((int64_t)Ac.nrows * L, kThreads), kThreads, 0, s>>>(
            Ac.nrows, Ac.rp(), Ac.ci(), AP.beg, AP.end, AP.ci, cpts, inM);
        ::amg::count_launch();
    });
    AMG_CHECK_LAUNCH();
}

int64_t sparsify(const DevCSR &A, const uint8_t *inM, const int32_t *tpos, const int32_t *diagpos,
                 double gamma, uint8_t *keep, DevCSR &H, cudaStream_t s, const uint8_t *S) {
    int32_t n = A.nrows;
    const bool full = S != nullptr;
    TmpBuf rowmax(sizeof(double) * (n + 1), s), flag(A.nnz + 1, s), guard(n + 1, s), cnt(sizeof(int32_t) * (n + 1), s);
    int g = div_up(n, kThreads);
    TmpBuf hval;
    if (n > 0) {
        with_row_lanes(row_lanes(A), [&](auto tc) {
            constexpr int L = decltype(tc)::value;
            sparsify_flag_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(
                n, A.rp(), A.ci(), A.v(), inM, gamma, rowmax.as<double>(), flag.as<uint8_t>());
            ::amg::count_launch();
        });
        with_row_lanes(row_lanes(A), [&](auto tc) {
            constexpr int L = decltype(tc)::value;
            const int gl = div_up((int64_t)n * L, kThreads);
            sparsify_sym_kernel<L><<<gl, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), tpos, flag.as<uint8_t>(),
                                                           rowmax.as<double>(), keep, guard.as<uint8_t>());
            ::amg::count_launch();
            // Algorithm 3 has no ismax guard: with every guard clear the
            // guard kernel only counts the kept entries of each row
            if (full) AMG_CUDA(cudaMemsetAsync(guard.ptr, 0, n, s));
            sparsify_guard_kernel<L><<<gl, kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), tpos, guard.as<uint8_t>(),
                                                             rowmax.as<double>(), keep, cnt.as<int32_t>());
            ::amg::count_launch();
        });
        AMG_CHECK_LAUNCH();
        if (full) {
            TmpBuf den(sizeof(double) * (A.nnz + 1), s), ecnt(sizeof(int32_t) * (A.nnz + 1), s),
                eoff(sizeof(int64_t) * (A.nnz + 1), s);
            const int lanes = row_lanes(A);
            with_row_lanes(lanes, [&](auto tc) {
                constexpr int L = decltype(tc)::value;
                lump_count_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(
                    n, A.rp(), A.ci(), A.v(), keep, S, den.as<double>(), ecnt.as<int32_t>());
                ::amg::count_launch();
            });
            AMG_CHECK_LAUNCH();
            const int64_t E = exclusive_scan_i64_from_i32(ecnt.as<int32_t>(), eoff.as<int64_t>(), A.nnz, s);
            require(E < ((int64_t)1 << 31), "full lumping: 2^31 or more lump edges");
            TmpBuf ek(sizeof(int32_t) * (E + 1), s), et(sizeof(double) * (E + 1), s), etg(sizeof(int32_t) * (E + 1), s),
                tlist(sizeof(int32_t) * (E + 1), s), tcnt(sizeof(int32_t) * (A.nnz + 1), s),
                toff(sizeof(int64_t) * (A.nnz + 1), s);
            hval.alloc(sizeof(double) * (A.nnz + 1), s);
            with_row_lanes(lanes, [&](auto tc) {
                constexpr int L = decltype(tc)::value;
                lump_emit_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(
                    n, A.rp(), A.ci(), A.v(), keep, S, diagpos, den.as<double>(), eoff.as<int64_t>(),
                    ek.as<int32_t>(), et.as<double>(), etg.as<int32_t>());
                ::amg::count_launch();
            });
            AMG_CUDA(cudaMemsetAsync(tcnt.ptr, 0, sizeof(int32_t) * A.nnz, s));
            if (E > 0) {
                lump_hist_kernel<<<div_up(E, kThreads), kThreads, 0, s>>>(E, etg.as<int32_t>(), tcnt.as<int32_t>());
                ::amg::count_launch();
            }
            exclusive_scan_i64_from_i32(tcnt.as<int32_t>(), toff.as<int64_t>(), A.nnz, s);
            AMG_CUDA(cudaMemsetAsync(tcnt.ptr, 0, sizeof(int32_t) * A.nnz, s));
            if (E > 0) {
                lump_place_kernel<<<div_up(E, kThreads), kThreads, 0, s>>>(E, etg.as<int32_t>(), toff.as<int64_t>(),
                                                                          tcnt.as<int32_t>(), tlist.as<int32_t>());
                ::amg::count_launch();
                lump_group_sort_kernel<<<div_up(A.nnz, kThreads), kThreads, 0, s>>>(A.nnz, toff.as<int64_t>(),
                                                                                   tlist.as<int32_t>());
                ::amg::count_launch();
            }
            with_row_lanes(lanes, [&](auto tc) {
                constexpr int L = decltype(tc)::value;
                lump_gather_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(
                    n, A.rp(), A.ci(), A.v(), keep, tpos, toff.as<int64_t>(), tlist.as<int32_t>(), ek.as<int32_t>(),
                    et.as<double>(), hval.as<double>());
                ::amg::count_launch();
            });
            AMG_CHECK_LAUNCH();
        }
    }
    H.rowptr.alloc(sizeof(int32_t) * (n + 1));
    int64_t nnz = exclusive_scan_i32(cnt.as<int32_t>(), H.rp(), n, s);
    H.nrows = n;
    H.ncols = A.ncols;
    H.nnz = nnz;
    H.col.alloc(sizeof(int32_t) * (nnz + kPad));
    H.val.alloc(sizeof(double) * (nnz + kPad));
    AMG_CUDA(cudaMemsetAsync(H.ci() + nnz, 0, sizeof(int32_t) * kPad, s));  // the compaction writes [0, nnz)
    AMG_CUDA(cudaMemsetAsync(H.v() + nnz, 0, sizeof(double) * kPad, s));
    if (n > 0) {
        if (full) {
            compact_values_kernel<<<g, kThreads, 0, s>>>(n, A.rp(), A.ci(), keep, hval.as<double>(), H.rp(), H.ci(),
                                                        H.v());
        } else {
            // at most 8 lanes a row: the lumped diagonal's additions are
            // issued by one lane per row, so a warp of one row would spend a
            // whole FP64 warp instruction on each dropped entry
            with_row_lanes(std::min(row_lanes(A), 8), [&](auto tc) {
                constexpr int L = decltype(tc)::value;
                sparsify_compact_lanes_kernel<L><<<div_up((int64_t)n * L, kThreads), kThreads, 0, s>>>(
                    n, A.rp(), A.ci(), A.v(), diagpos, keep, H.rp(), H.ci(), H.v());
            });
        }
        ::amg::count_launch();
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
    TmpBuf linv(sizeof(double) * (size_t)n * n, s), err(sizeof(int), s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    if (n <= kSmemCoarse) {
        TmpBuf rdiag(sizeof(double) * (size_t)n, s);
        const size_t smem_f = sizeof(double) * (size_t)n * n, smem_i = sizeof(double) * ((size_t)n * n + 2 * (size_t)n);
        AMG_CUDA(cudaFuncSetAttribute(coarse_chol_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * kSmemCoarse * kSmemCoarse)));
        AMG_CUDA(cudaFuncSetAttribute(coarse_inv_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * (kSmemCoarse * kSmemCoarse + 2 * kSmemCoarse))));
        { coarse_chol_smem_kernel<<<1, 1024, smem_f, s>>>(n, A.rp(), A.ci(), A.v(), linv.as<double>(),
                                                          rdiag.as<double>(), err.as<int>()); ::amg::count_launch(); }
        { coarse_inv_col_kernel<<<n, 128, smem_i, s>>>(n, linv.as<double>(), rdiag.as<double>(), inv); ::amg::count_launch(); }
    } else {
        TmpBuf a(sizeof(double) * (size_t)n * n, s);
        { densify_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), a.as<double>()); ::amg::count_launch(); }
        { cholesky_kernel<<<1, 1024, 0, s>>>(n, a.as<double>(), err.as<int>()); ::amg::count_launch(); }
        { tri_inverse_kernel<<<div_up(n, 128), 128, 0, s>>>(n, a.as<double>(), linv.as<double>()); ::amg::count_launch(); }
        { gram_kernel<<<div_up((int64_t)n * n, kThreads), kThreads, 0, s>>>(n, linv.as<double>(), inv); ::amg::count_launch(); }
    }
    AMG_CHECK_LAUNCH();
    if (!read_scalar(err.as<int>(), s)) return;
    // not positive definite: Gauss-Jordan with partial pivoting instead
    TmpBuf a(sizeof(double) * (size_t)n * n, s), fac(sizeof(double) * (size_t)n, s);
    AMG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    { densify_kernel<<<div_up(n, kThreads), kThreads, 0, s>>>(n, A.rp(), A.ci(), A.v(), a.as<double>()); ::amg::count_launch(); }
    { gauss_jordan_kernel<<<1, 1024, 0, s>>>(n, a.as<double>(), inv, fac.as<double>(), err.as<int>()); ::amg::count_launch(); }
    AMG_CHECK_LAUNCH();
    if (read_scalar(err.as<int>(), s))
        throw Error(AMG_BREAKDOWN, "coarsest operator is singular (zero pivot in Gauss-Jordan elimination)");
}

}  // namespace setup
}  // namespace amg
