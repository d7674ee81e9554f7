// Device setup of the CPR preconditioner B (the setup behind Alg. 1, Sec. 3.1):
// pressure decoupling, the AMG hierarchy (classical strength, PMIS C/F split,
// direct interpolation, R = P^T, Galerkin R A P) with the Eq. 5.1 coloring of
// every smoothed level (Jones-Plassmann with hashed keys), the dense coarsest
// solve, and the multicolor block ILU(0) second stage.
//
// Every floating-point operation whose result decides a discrete outcome
// (strength, interpolation weights, coarse matrices) is written with explicit
// round-to-nearest intrinsics in a fixed order (the ascending-column order of
// the plain definitions), so colors, C/F splits and sparsity patterns are
// reproducible bit for bit.  Discrete rounds (JP, PMIS) are round-synchronous:
// every decision of a round reads the state at the start of the round.
#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <atomic>
#include <type_traits>

#include "cpr_internal.cuh"

namespace cpr {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool key_greater(int a1, uint32_t h1, int i1, int a2, uint32_t h2,
                                            int i2) {
    if (a1 != a2) return a1 > a2;
    if (h1 != h2) return h1 > h2;
    return i1 > i2;
}

// Lower bound of j in col[lo, hi); the caller checks col[result] == j.
__device__ __forceinline__ int find_col(const int *col, int lo, int hi, int j) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// ------------------------------------------------------------- validation

__global__ void k_validate_bsr(const int *rowptr, const int *col, int nb, int nnzb, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int a = rowptr[i], b = rowptr[i + 1];
    if ((i == 0 && a != 0) || (i == nb - 1 && b != nnzb) || b < a || a < 0 || b > nnzb) {
        set_err(err, CPR_ERR_INVALID);
        return;
    }
    int prev = -1;
    bool diag = false;
    for (int p = a; p < b; p++) {
        int c = col[p];
        if (c < 0 || c >= nb || c <= prev) {
            set_err(err, CPR_ERR_INVALID);
            return;
        }
        prev = c;
        diag |= c == i;
    }
    if (!diag) set_err(err, CPR_ERR_INVALID);
}

__global__ void k_diagpos(int n, const int *rowptr, const int *col, int *diag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = rowptr[i + 1];
    int p = find_col(col, rowptr[i], e, i);
    diag[i] = (p < e && col[p] == i) ? p : -1;
}

// ------------------------------------------------------------- decoupling

// w_i = D_i^-T e_1 = (C00, C10, C20) / det(D_i) by the adjugate, or e_1 (mode 0).
__global__ void k_decouple(int nb, const int *diag, const double *val, int mode, double *w,
                           int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    if (mode == 0) {
        w[3 * i] = 1.0;
        w[3 * i + 1] = 0.0;
        w[3 * i + 2] = 0.0;
        return;
    }
    const double *d = val + 9 * (size_t)diag[i];
    double c00 = __dsub_rn(__dmul_rn(d[4], d[8]), __dmul_rn(d[5], d[7]));
    double c10 = __dsub_rn(__dmul_rn(d[2], d[7]), __dmul_rn(d[1], d[8]));
    double c20 = __dsub_rn(__dmul_rn(d[1], d[5]), __dmul_rn(d[2], d[4]));
    double det = __dadd_rn(__dadd_rn(__dmul_rn(d[0], c00), __dmul_rn(d[3], c10)), __dmul_rn(d[6], c20));
    if (det == 0.0 || !isfinite(det)) {
        set_err(err, CPR_ERR_SINGULAR);
        det = 1.0;
    }
    w[3 * i] = __ddiv_rn(c00, det);
    w[3 * i + 1] = __ddiv_rn(c10, det);
    w[3 * i + 2] = __ddiv_rn(c20, det);
}

// A_P[i][j] = w_i . A_ij e_1 on the block pattern.
__global__ void k_pressure_matrix(int nb, const int *rowptr, const double *val, const double *w,
                                  double *apval) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double w0 = w[3 * i], w1 = w[3 * i + 1], w2 = w[3 * i + 2];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        const double *a = val + 9 * (size_t)p;
        apval[p] = __dadd_rn(__dadd_rn(__dmul_rn(w0, a[0]), __dmul_rn(w1, a[3])), __dmul_rn(w2, a[6]));
    }
}

// Column 0 of every block of A (the copy B keeps for the second residual of Alg. 1), with rows
// taken in position order and columns renumbered to positions.  Count pass
// (crow == nullptr: row lengths) or fill pass.
__global__ void k_col0_perm(int nb, const int *order, const int *iperm, const int *rowptr, const int *col,
                            const double *val, const int *crow, int *ccol, double *cval, int *cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    int i = order[t];
    if (!crow) {
        cnt[t] = rowptr[i + 1] - rowptr[i];
        return;
    }
    int q = crow[t];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++, q++) {
        const double *a = val + 9 * (size_t)p;
        ccol[q] = iperm[col[p]];
        cval[3 * (size_t)q] = a[0];
        cval[3 * (size_t)q + 1] = a[3];
        cval[3 * (size_t)q + 2] = a[6];
    }
}

// The fill pass of k_col0_perm with G lanes per row (a lane per block, so a
// warp reads whole rows of blocks instead of one block from each of 32 rows).
template <int G>
__global__ void k_col0_fill(int nb, const int *order, const int *iperm, const int *rowptr, const int *col,
                            const double *val, const int *crow, int *ccol, double *cval) {
    long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    if (t >= nb) return;
    int i = order[t];
    int a = rowptr[i], q0 = crow[t] - a;
    for (int p = a + lane; p < rowptr[i + 1]; p += G) {
        const double *b = val + 9 * (size_t)p;
        size_t q = (size_t)(q0 + p);
        ccol[q] = iperm[col[p]];
        cval[3 * q] = b[0];
        cval[3 * q + 1] = b[3];
        cval[3 * q + 2] = b[6];
    }
}

__global__ void k_compose(int n, const int *first, const int *second, int *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = second[first ? first[t] : t];
}

// -------------------------------------------------------- strength (Eq. 5.1)

// The strength tests compare FP64 values on the integer pipe (B300's FP64
// pipe is 1/64 of its FP32 rate): ord_key maps a double's bits to a signed
// integer with key(x) < key(y) iff x < y and equal keys for equal values
// (-0 taken as +0).  A NaN has no place in that order; the callers skip it,
// so a NaN entry is never strong and never the row's maximum.
constexpr long long kSignBit = (long long)0x8000000000000000ULL;
constexpr long long kMagBits = 0x7fffffffffffffffLL;
__device__ __forceinline__ long long ord_key(long long u) {
    if (u == kSignBit) u = 0;
    return u >= 0 ? u : u ^ kMagBits;
}
__device__ __forceinline__ bool nan_bits(long long u) { return (u & kMagBits) > 0x7ff0000000000000LL; }

// Eq. 5.1: j in S_i iff j != i and |a_ij| > theta * sum_k |a_ik| (the sum in
// row order over the whole row).  srowptr == nullptr: count pass (out =
// counts), which also leaves each row's threshold in thr; otherwise fill
// pass (out = columns), which reads it back instead of summing again.
// Row i of Eq. 5.1's strength set.  Without srowptr: the row's threshold
// theta * sum_k |a_ik| (summed in entry order) goes to thr[i] and the count
// of its strong entries is returned; with srowptr: the threshold is read from
// thr[i] and the strong columns are written from out[srowptr[i]] on.
__device__ __forceinline__ int strength51_row(int i, const int *rowptr, const int *col, const double *val,
                                              double theta, const int *srowptr, int *out, double *thr) {
    int a = rowptr[i], b = rowptr[i + 1];
    const long long *vb = reinterpret_cast<const long long *>(val);
    long long tb;
    if (srowptr) {
        tb = __double_as_longlong(thr[i]);
    } else {
        double rowsum = 0.0;
        for (int p = a; p < b; p++) rowsum = __dadd_rn(rowsum, __longlong_as_double(vb[p] & kMagBits));
        double t = __dmul_rn(theta, rowsum);
        thr[i] = t;
        tb = __double_as_longlong(t);
    }
    int q = srowptr ? srowptr[i] : 0, c = 0;
    if (!nan_bits(tb)) {
        long long tk = ord_key(tb);
        for (int p = a; p < b; p++) {
            int j = col[p];
            long long u = vb[p] & kMagBits;   // |a_ij|: its bits are its key
            if (j != i && !nan_bits(u) && u > tk) {
                if (srowptr) out[q + c] = j;
                c++;
            }
        }
    }
    return c;
}

__global__ void k_strength51(int n, const int *rowptr, const int *col, const double *val,
                             double theta, const int *srowptr, int *out, double *thr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = strength51_row(i, rowptr, col, val, theta, srowptr, out, thr);
    if (!srowptr) out[i] = c;
}

// Classical strength: with s = sign(a_ii), j in S_i iff
// -s a_ij >= theta max_{k!=i}(-s a_ik) > 0.  -s a_ij is a_ij with its sign
// bit flipped when a_ii >= 0, so the maximum and the tests are integer work;
// the threshold is the one FP64 product of the row.
__global__ void k_strength_rs(int n, const int *rowptr, const int *col, const double *val,
                              double theta, const int *srowptr, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rowptr[i], b = rowptr[i + 1];
    const long long *vb = reinterpret_cast<const long long *>(val);
    double aii = 0.0;
    for (int p = a; p < b; p++)
        if (col[p] == i) aii = val[p];
    long long flip = aii < 0.0 ? 0 : kSignBit;
    long long mk = LLONG_MIN;
    for (int p = a; p < b; p++) {
        long long u = vb[p] ^ flip;
        if (col[p] != i && !nan_bits(u)) mk = max(mk, ord_key(u));
    }
    int q = srowptr ? srowptr[i] : 0, c = 0;
    if (mk > 0) {   // the largest -s a_ik is positive: its key is its bits
        long long tk = ord_key(__double_as_longlong(__dmul_rn(theta, __longlong_as_double(mk))));
        for (int p = a; p < b; p++) {
            int j = col[p];
            long long u = vb[p] ^ flip;
            if (j != i && !nan_bits(u) && ord_key(u) >= tk) {
                if (srowptr) out[q + c] = j;
                c++;
            }
        }
    }
    if (!srowptr) out[i] = c;
}

// Warp-per-row form of the classical strength kernel for levels with long
// rows (coarse levels average 16-40 entries per row): a row's entries are
// loaded by all lanes at once instead of one after another by one thread.
// Same tests on the same keys (the maximum an integer warp reduction) and
// the same output order (ballot compaction in entry order).
__global__ void k_strength_rs_warp(int n, const int *rowptr, const int *col, const double *val,
                                   double theta, const int *srowptr, int *out) {
    int lane = threadIdx.x & 31;
    int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;
    int a = rowptr[i], b = rowptr[i + 1];
    const long long *vb = reinterpret_cast<const long long *>(val);
    unsigned lt = (1u << lane) - 1u;
    double aii = 0.0;
    bool found = false;
    for (int p = a + lane; p < b; p += 32)
        if (col[p] == i) {
            aii = val[p];
            found = true;
        }
    unsigned fm = __ballot_sync(0xffffffffu, found);
    aii = fm ? __shfl_sync(0xffffffffu, aii, __ffs(fm) - 1) : 0.0;
    long long flip = aii < 0.0 ? 0 : kSignBit;
    long long mk = LLONG_MIN;
    for (int p = a + lane; p < b; p += 32) {
        long long u = vb[p] ^ flip;
        if (col[p] != i && !nan_bits(u)) mk = max(mk, ord_key(u));
    }
    for (int sh = 16; sh > 0; sh >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, sh));
    int q = srowptr ? srowptr[i] : 0, c = 0;
    if (mk > 0) {
        long long tk = ord_key(__double_as_longlong(__dmul_rn(theta, __longlong_as_double(mk))));
        for (int p0 = a; p0 < b; p0 += 32) {
            int p = p0 + lane, j = 0;
            bool keep = false;
            if (p < b) {
                j = col[p];
                long long u = vb[p] ^ flip;
                keep = j != i && !nan_bits(u) && ord_key(u) >= tk;
            }
            unsigned bm = __ballot_sync(0xffffffffu, keep);
            if (keep && srowptr) out[q + c + __popc(bm & lt)] = j;
            c += __popc(bm);
        }
    }
    if (!srowptr && lane == 0) out[i] = c;
}

// Off-diagonal block pattern (the BILU graph at theta = 0).
__global__ void k_offdiag_pattern(int n, const int *rowptr, const int *col, const int *srowptr,
                                  int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = srowptr ? srowptr[i] : 0, c = 0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
        if (col[p] != i) {
            if (srowptr) out[q + c] = col[p];
            c++;
        }
    if (!srowptr) out[i] = c;
}

// --------------------------------------------------------------- transpose

__global__ void k_count_cols(long nnz, const int *col, int *cnt) {
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < nnz; p += (long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[p]], 1);
}

__global__ void k_scatter_t(int n, const int *rowptr, const int *col, const double *val,
                            int *cursor, int *tcol, double *tval) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int q = atomicAdd(&cursor[col[p]], 1);
        tcol[q] = i;
        if (val) tval[q] = val[p];
    }
}

// Sort each row by column: rows of up to 32 entries in registers (one thread
// per row); longer rows are listed (in any order) for k_sort_long_rows.
constexpr int kRegSort = 32;
__global__ void k_sort_rows(int n, const int *rowptr, int *col, double *val, int *longrows, int *nlong) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rowptr[i], b = rowptr[i + 1];
    int L = b - a;
    if (L > kRegSort) longrows[atomicAdd(nlong, 1)] = i;
    if (L <= 1 || L > kRegSort) return;
    {
        int c[kRegSort];
        double v[kRegSort];
#pragma unroll
        for (int k = 0; k < kRegSort; k++)
            if (k < L) {
                c[k] = col[a + k];
                v[k] = val ? val[a + k] : 0.0;
            }
        // odd-even transposition sort over the first L entries
        for (int pass = 0; pass < L; pass++) {
#pragma unroll
            for (int k = 0; k + 1 < kRegSort; k++) {
                if ((k & 1) != (pass & 1) || k + 1 >= L) continue;
                if (c[k] > c[k + 1]) {
                    int tc = c[k];
                    c[k] = c[k + 1];
                    c[k + 1] = tc;
                    double tv = v[k];
                    v[k] = v[k + 1];
                    v[k + 1] = tv;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kRegSort; k++)
            if (k < L) {
                col[a + k] = c[k];
                if (val) val[a + k] = v[k];
            }
        return;
    }
}

// The listed rows (longer than kRegSort): one warp per row, bitonic sort of
// (column, value) pairs in shared memory (rows up to kLongSort entries),
// grid-stride over the list.  Rows beyond kLongSort (none in practice) take a
// serial insertion sort.
constexpr int kLongSort = 1024;
constexpr int kSortWarps = 4;
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_long_rows(const int *longrows, const int *nlong,
                                                                     const int *rowptr, int *col, double *val) {
    __shared__ int sk[kSortWarps][kLongSort];
    __shared__ double sv[kSortWarps][kLongSort];
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    int *K = sk[wl];
    double *Vv = sv[wl];
    int nl = *nlong;
    for (int w = blockIdx.x * kSortWarps + wl; w < nl; w += gridDim.x * kSortWarps) {
        int i = longrows[w];
        int a = rowptr[i], b = rowptr[i + 1];
        int L = b - a;
        if (L > kLongSort) {
            if (lane == 0)
                for (int p = a + 1; p < b; p++) {
                    int c = col[p];
                    double v = val ? val[p] : 0.0;
                    int q = p - 1;
                    while (q >= a && col[q] > c) {
                        col[q + 1] = col[q];
                        if (val) val[q + 1] = val[q];
                        q--;
                    }
                    col[q + 1] = c;
                    if (val) val[q + 1] = v;
                }
            __syncwarp();
            continue;
        }
        int P = 64;
        while (P < L) P <<= 1;
        for (int t = lane; t < P; t += 32) {
            K[t] = t < L ? col[a + t] : INT_MAX;
            Vv[t] = (t < L && val) ? val[a + t] : 0.0;
        }
        __syncwarp();
        for (int size = 2; size <= P; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < P / 2; t += 32) {
                    int x = (t / stride) * 2 * stride + (t % stride);
                    int y = x + stride;
                    bool up = (x & size) == 0;
                    int u = K[x], v = K[y];
                    if ((u > v) == up) {
                        K[x] = v;
                        K[y] = u;
                        double tv = Vv[x];
                        Vv[x] = Vv[y];
                        Vv[y] = tv;
                    }
                }
                __syncwarp();
            }
        for (int t = lane; t < L; t += 32) {
            col[a + t] = K[t];
            if (val) val[a + t] = Vv[t];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ Jones-Plassmann

constexpr unsigned long long kUncolored = ~0ull;
constexpr int kSmallLevel = 4096;    // levels up to this size run their rounds in one CTA
constexpr int kJpBatch = 16;         // JP rounds launched per host check of the remaining count
constexpr int kPmisBatch = 6;        // PMIS rounds launched per host check of the undecided count

// The symmetric graph G = S u S^T that JP colors, held as two disjoint
// adjacency lists: S (no diagonal, rows sorted) and T, the entries of S^T
// that S lacks (rows in any order; empty when S is symmetric).  The degree in
// the key is |S_i u S^T_i| = |S_i| + |T_i|.
struct JpGraph {
    const int *sr, *sc, *tr, *tc, *deg;
};

// One JP round r for vertex i.  A vertex uncolored at the start of the round
// (never colored, or colored in this very round by someone else) whose key
// (degree, hash, index) beats every neighbour uncolored at the start of the
// round takes the smallest color not held by a neighbour colored in an
// earlier round.  state packs (round << 32 | color) into one 64-bit word,
// written in one store.  A state written in this round reads as uncolored
// whether or not the store is seen yet, so the loads need no volatile and
// may hit L1.
//
// G lanes share the vertex: lane l takes entries l, l + G, ... of the
// concatenation of S_i and T_i, P at a time, loading all their columns,
// then all their states and degrees, before comparing.  A vertex thus waits
// on about deg / (G P) dependent load pairs instead of one pair per
// neighbour.  The lanes' verdicts are AND-ed and their masks of the colors
// below 64 held by earlier-colored neighbours OR-ed; a vertex whose
// neighbours hold all of them searches on from 64 on lane 0.  The outcome
// is the one of a neighbour-by-neighbour walk.  Every lane of the warp calls
// this (act false for an empty slot); the result is valid on the group's
// lane 0, which also writes the state.
constexpr int kJpPre = 4;      // entries per lane and batch in the multi-CTA rounds
constexpr long kResidentThreads = 148L * 2048;   // threads resident at once on B300
constexpr int kJpPreSmall = 8; // in the one-CTA kernels, whose few lanes each walk many entries

template <int G>
__device__ __forceinline__ bool group_all(bool v) {
    unsigned x = v ? 1u : 0u;
    for (int o = G >> 1; o > 0; o >>= 1) x &= __shfl_xor_sync(0xffffffffu, x, o, G);
    return x != 0;
}

template <int G>
__device__ __forceinline__ bool group_any(bool v) {
    unsigned x = v ? 1u : 0u;
    for (int o = G >> 1; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o, G);
    return x != 0;
}

template <int G>
__device__ __forceinline__ unsigned long long group_or64(unsigned long long v) {
    for (int o = G >> 1; o > 0; o >>= 1) {
        unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)v, o, G);
        unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), o, G);
        v |= ((unsigned long long)hi << 32) | lo;
    }
    return v;
}

// The smallest color >= 64 not held by a neighbour of i colored before round r.
__device__ int jp_color_from64(int i, const JpGraph &g, const unsigned long long *vs, unsigned r) {
    for (int base = 64;; base += 64) {
        unsigned long long mask = 0;
        for (int pass = 0; pass < 2; pass++) {
            const int *R = pass ? g.tr : g.sr, *C = pass ? g.tc : g.sc;
            for (int p = R[i]; p < R[i + 1]; p++) {
                unsigned long long sj = vs[C[p]];
                if (sj == kUncolored || (unsigned)(sj >> 32) >= r) continue;
                int cj = (int)(unsigned)sj;
                if (cj >= base && cj < base + 64) mask |= 1ull << (cj - base);
            }
        }
        if (mask != ~0ull) return base + __ffsll((long long)~mask) - 1;
    }
}

template <int G, int P>
__device__ int jp_vertex(int i, bool act, int lane, const JpGraph &g, uint32_t hbase, unsigned long long *state,
                         unsigned r) {
    const unsigned long long *vs = state;
    bool cand = act && vs[i] == kUncolored;   // the same on every lane of the group
    int di = 0, a0 = 0, na = 0, b0 = 0, nt = 0;
    uint32_t hi = 0;
    if (cand) {
        di = g.deg[i];
        hi = fmix32((uint32_t)i ^ hbase);
        a0 = g.sr[i];
        na = g.sr[i + 1] - a0;
        b0 = g.tr[i];
        nt = na + (g.tr[i + 1] - b0);
    }
    bool win = cand;
    unsigned long long used = 0;   // colors below 64 of neighbours colored in earlier rounds
    for (int q0 = 0; q0 < nt; q0 += G * P) {
        int jj[P];
#pragma unroll
        for (int u = 0; u < P; u++) {
            int q = q0 + lane + u * G;
            jj[u] = q < nt ? (q < na ? g.sc[a0 + q] : g.tc[b0 + q - na]) : -1;
        }
        unsigned long long sj[P];
        int dj[P];
#pragma unroll
        for (int u = 0; u < P; u++) {
            sj[u] = jj[u] >= 0 ? vs[jj[u]] : 0ull;
            dj[u] = jj[u] >= 0 ? g.deg[jj[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < P; u++) {
            int j = jj[u];
            if (j < 0 || j == i) continue;
            bool unc = sj[u] == kUncolored || (unsigned)(sj[u] >> 32) == r;
            if (unc) {
                if (!key_greater(di, hi, i, dj[u], fmix32((uint32_t)j ^ hbase), j)) win = false;
            } else {
                int cj = (int)(unsigned)sj[u];
                if (cj < 64) used |= 1ull << cj;
            }
        }
    }
    win = group_all<G>(win);
    used = group_or64<G>(used);
    int c = -1;
    if (win && lane == 0) {
        c = used != ~0ull ? __ffsll((long long)~used) - 1 : jp_color_from64(i, g, vs, r);
        state[i] = ((unsigned long long)r << 32) | (unsigned)c;
    }
    return c;
}

// Whether row j of S (sorted) holds column i.
__device__ __forceinline__ bool row_has(const int *sr, const int *sc, int j, int i) {
    int lo = sr[j], hi = sr[j + 1], end = hi;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sc[mid] < i) lo = mid + 1;
        else hi = mid;
    }
    return lo < end && sc[lo] == i;
}

// T, the one-way part of S^T: entry (i, j) of S puts i into row j of T
// unless j's own row of S already holds i.  Without tcol, counts per T row;
// with it, scatters (rows in any order).  One thread per row of S, so the
// entry count of S need not be known on the host.
__global__ void k_oneway_t(int n, const int *sr, const int *sc, int *cnt_or_cursor, int *tcol) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = sr[i]; p < sr[i + 1]; p++) {
        int j = sc[p];
        if (row_has(sr, sc, j, i)) continue;
        int q = atomicAdd(&cnt_or_cursor[j], 1);
        if (tcol) tcol[q] = i;
    }
}

__global__ void k_sym_degree(int n, const int *sr, const int *tr, int *deg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) deg[i] = (sr[i + 1] - sr[i]) + (tr[i + 1] - tr[i]);
}

// One JP round over a worklist: the vertices still uncolored when the round
// starts (round 0: all n, list_in == nullptr), G lanes per vertex.  A
// vertex's decision depends only on the states left by earlier rounds, so the
// order of the list does not matter; the losers are appended to list_out
// (warp-aggregated).  Counts cycle through three slots: this round reads
// cnt[r % 3], appends to cnt[(r+1) % 3] (zeroed by the previous round) and
// zeroes cnt[(r+2) % 3] for the next one.  Rounds are launched in batches
// between host checks; once the list is empty the rest of the batch returns
// at once.
template <int G>
__global__ void k_jp_round(int n, const int *list_in, int *list_out, int *cnt, JpGraph g, uint32_t hbase,
                           unsigned long long *state, unsigned r, int *maxcolor) {
    int m = list_in ? *(volatile const int *)&cnt[r % 3] : n;
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(r + 2) % 3] = 0;
    int *out_cnt = &cnt[(r + 1) % 3];
    int lane32 = threadIdx.x & 31, lane = threadIdx.x % G;
    int per = blockDim.x / G;
    int cmax = -1;
    // v0 is uniform over the block, so whole warps run each pass together
    for (long v0 = (long)blockIdx.x * per; v0 < m; v0 += (long)gridDim.x * per) {
        long t = v0 + threadIdx.x / G;
        bool act = t < m;
        int i = act ? (list_in ? list_in[t] : (int)t) : 0;
        int c = jp_vertex<G, kJpPre>(i, act, lane, g, hbase, state, r);
        bool lead = act && lane == 0;
        if (lead && c >= 0) cmax = max(cmax, c);
        bool lost = lead && c < 0;
        unsigned b = __ballot_sync(0xffffffffu, lost);
        if (b) {
            int leader = __ffs(b) - 1, base = 0;
            if (lane32 == leader) base = atomicAdd(out_cnt, __popc(b));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (lost) list_out[base + __popc(b & ((1u << lane32) - 1u))] = i;
        }
    }
    if (cmax >= 0) atomicMax(maxcolor, cmax);
}

// All JP rounds of a small graph in one CTA, rounds separated by barriers
// (the same rounds as k_jp_round, without host round trips).
template <int G>
__global__ void __launch_bounds__(1024) k_jp_small(int n, JpGraph g, uint32_t hbase, unsigned long long *state,
                                                   int *maxcolor) {
    __shared__ int rem;
    __shared__ int mx;
    if (threadIdx.x == 0) {
        rem = n;
        mx = 0;
    }
    __syncthreads();
    int lane = threadIdx.x % G, per = blockDim.x / G;
    for (unsigned r = 0; r < (unsigned)n + 8; r++) {
        int left = rem;
        __syncthreads();
        if (left == 0) break;
        for (int v0 = 0; v0 < n; v0 += per) {   // uniform over the block
            int i = v0 + (int)threadIdx.x / G;
            int c = jp_vertex<G, kJpPreSmall>(i, i < n, lane, g, hbase, state, r);
            if (i < n && lane == 0 && c >= 0) {
                atomicSub(&rem, 1);
                atomicMax(&mx, c);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *maxcolor = mx;
}

__global__ void k_state_to_color(int n, const unsigned long long *state, int *color) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) color[i] = (int)(unsigned)state[i];
}

// Whether row j of S holds column i, for the one-CTA coloring: a row of up
// to 64 entries is scanned with independent loads (one round trip to L2)
// instead of a binary search's chain of dependent ones; longer rows search.
__device__ __forceinline__ bool row_has_short(const int *sr, const int *sc, int j, int i) {
    int lo = sr[j], hi = sr[j + 1];
    if (hi - lo > 64) return row_has(sr, sc, j, i);
    bool f = false;
#pragma unroll 8
    for (int p = lo; p < hi; p++) f |= sc[p] == i;
    return f;
}

// Exclusive scan of a[0 .. n) in place, a[n] = the total, by one CTA of
// kSmallLevel / 4 threads, each taking four consecutive entries (n <= kSmallLevel).
__device__ void cta_scan_small(int *a, int n) {
    __shared__ int wsum[32];
    int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int base = 4 * t, v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = base + k < n ? a[base + k] : 0;
        sum += v[k];
    }
    int x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int e = x - sum + (wid > 0 ? wsum[wid - 1] : 0);
    int total = wsum[(blockDim.x >> 5) - 1];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (base + k < n) a[base + k] = e;
        e += v[k];
    }
    if (t == 0) a[n] = total;
    __syncthreads();
}

// The smoother's coloring of a level of n <= kSmallLevel rows in one CTA and
// one launch: Eq. 5.1's strength set S (k_strength51's row logic: counts, a
// scan, the columns), T, the entries of S^T that S lacks (counts, a scan,
// a scatter), the degrees |S_i| + |T_i|, the JP rounds of k_jp_small, and the
// rows grouped by color, index-ascending within a color.  The same S, keys
// and rounds as the multi-launch path, so the same colors and order.  info[0]
// receives the color count, info[1 .. ncolors + 1] the color offsets.
template <int G>
__global__ void __launch_bounds__(kSmallLevel / 4) k_color_small(int n, const int *rowptr, const int *col,
                                                                const double *val, double theta, uint32_t hbase,
                                                                double *thr, int *srow, int *scol, int *trow,
                                                                int *tcol, int *deg, unsigned long long *state,
                                                                int *color, int *rows, int *info) {
    __shared__ int rem, mx, run;
    __shared__ int cnt[kSmallLevel / 4 + 1];
    int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < n; i += nt) srow[i] = strength51_row(i, rowptr, col, val, theta, nullptr, nullptr, thr);
    __syncthreads();
    cta_scan_small(srow, n);
    for (int i = t; i < n; i += nt) strength51_row(i, rowptr, col, val, theta, srow, scol, thr);
    for (int i = t; i < n; i += nt) trow[i] = 0;
    __syncthreads();
    for (int i = t; i < n; i += nt)
        for (int p = srow[i]; p < srow[i + 1]; p++) {
            int j = scol[p];
            if (!row_has_short(srow, scol, j, i)) atomicAdd(&trow[j], 1);
        }
    __syncthreads();
    cta_scan_small(trow, n);
    for (int i = t; i < n; i += nt) deg[i] = trow[i];   // scatter cursors
    __syncthreads();
    for (int i = t; i < n; i += nt)
        for (int p = srow[i]; p < srow[i + 1]; p++) {
            int j = scol[p];
            if (!row_has_short(srow, scol, j, i)) tcol[atomicAdd(&deg[j], 1)] = i;
        }
    __syncthreads();
    for (int i = t; i < n; i += nt) {
        deg[i] = (srow[i + 1] - srow[i]) + (trow[i + 1] - trow[i]);
        state[i] = kUncolored;
    }
    if (t == 0) {
        rem = n;
        mx = 0;
    }
    __syncthreads();
    JpGraph g{srow, scol, trow, tcol, deg};
    int lane = t % G, per = nt / G;
    for (unsigned r = 0; r < (unsigned)n + 8; r++) {
        int left = rem;
        __syncthreads();
        if (left == 0) break;
        for (int v0 = 0; v0 < n; v0 += per) {   // uniform over the block
            int i = v0 + t / G;
            int c = jp_vertex<G, kJpPreSmall>(i, i < n, lane, g, hbase, state, r);
            if (i < n && lane == 0 && c >= 0) {
                atomicSub(&rem, 1);
                atomicMax(&mx, c);
            }
        }
        __syncthreads();
    }
    int nc = n ? mx + 1 : 0;
    for (int i = t; i < n; i += nt) color[i] = (int)(unsigned)state[i];
    if (t == 0) run = 0;
    __syncthreads();
    // color c's rows in index order: each thread's four consecutive rows, a
    // scan of the per-thread counts, then the scatter after the running offset
    for (int c = 0; c < nc; c++) {
        int base = 4 * t, f = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (base + k < n && color[base + k] == c) f |= 1 << k;
        cnt[t] = __popc(f);
        __syncthreads();
        cta_scan_small(cnt, nt);
        int off = run + cnt[t];
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (f & (1 << k)) rows[off++] = base + k;
        if (t == 0) info[1 + c] = run;
        __syncthreads();
        if (t == 0) run += cnt[nt];
        __syncthreads();
    }
    if (t == 0) {
        info[0] = nc;
        info[1 + nc] = run;
    }
}

// One round of the level sets of natural-order block ILU(0) over a worklist
// (round 0: all n rows, list_in == nullptr).  A row whose neighbours of lower
// index in G (the symmetrised block graph) all have levels takes 1 + the
// largest of them, or 0 with none; the others are appended to list_out.  A
// level, once written, is final, so a row may read one written earlier in
// this same round: rounds decide only when a row is reached, never its value.
// Count slots cycle as in k_jp_round.
__global__ void k_level_round(int n, const int *list_in, int *list_out, int *cnt, JpGraph g, int *level,
                              unsigned r, int *maxlevel) {
    int m = list_in ? *(volatile const int *)&cnt[r % 3] : n;
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(r + 2) % 3] = 0;
    int *out_cnt = &cnt[(r + 1) % 3];
    int lane = threadIdx.x & 31;
    int lmax = -1;
    for (int t0 = blockIdx.x * blockDim.x; t0 < m; t0 += gridDim.x * blockDim.x) {
        int t = t0 + threadIdx.x, i = 0;
        bool wait = false;
        if (t < m) {
            i = list_in ? list_in[t] : t;
            int lv = 0;
            for (int pass = 0; pass < 2 && !wait; pass++) {
                const int *R = pass ? g.tr : g.sr, *C = pass ? g.tc : g.sc;
                for (int p = R[i]; p < R[i + 1]; p++) {
                    int j = C[p];
                    if (j >= i) continue;
                    int lj = *(volatile const int *)&level[j];
                    if (lj < 0) {
                        wait = true;
                        break;
                    }
                    lv = max(lv, lj + 1);
                }
            }
            if (!wait) {
                level[i] = lv;
                lmax = max(lmax, lv);
            }
        }
        unsigned b = __ballot_sync(0xffffffffu, wait);
        if (b) {
            int leader = __ffs(b) - 1, base = 0;
            if (lane == leader) base = atomicAdd(out_cnt, __popc(b));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (wait) list_out[base + __popc(b & ((1u << lane) - 1u))] = i;
        }
    }
    if (lmax >= 0) atomicMax(maxlevel, lmax);
}

// ---------------------------- Alg. 4-5: VerticesSplitting / VerticesGrouping
//
// The paper's own coloring of the strong-connection matrix S (Eq. 5.1, rows
// as computed, not symmetrised), with the readings of its loosely defined
// parts: "any take" picks, among the candidates of largest |S_i|, the lowest
// index; the candidates are the second-circle set W^ (restricted to V) when
// it is not empty, else all of V; S^_i = (union of S_k, k in S_i) minus
// (S_i and i); W-bar takes only the members of S_i still in V.  The greedy
// takes one vertex at a time, so it runs on one warp: vertices are ranked once
// by (|S_i| descending, index), and a pick is the first vertex in rank order
// that is a candidate, found by ballots over a rank-indexed bitmap of W^ or
// by a pointer into the ranks that only moves forward within a call (a
// vertex that leaves the candidates never returns in that call).

constexpr int kGroupSortThreads = 1024;
constexpr unsigned kGroupIndexBits = 14;   // kMaxGroupingRows = 2^14

// order[r] = the vertex of rank r, rank[i] = the rank of vertex i: a bitonic
// sort of packed keys ((2^14 - 1 - |S_i|) << 14 | i) in shared memory.
__global__ void __launch_bounds__(kGroupSortThreads) k_group_order(int n, const int *sr, int *order, int *rank) {
    extern __shared__ unsigned keys[];
    int m = 1;
    while (m < n) m <<= 1;
    const unsigned top = (1u << kGroupIndexBits) - 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        unsigned key = ~0u;
        if (i < n) {
            unsigned d = (unsigned)min(sr[i + 1] - sr[i], (int)top);
            key = ((top - d) << kGroupIndexBits) | (unsigned)i;
        }
        keys[i] = key;
    }
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned a = keys[i], b = keys[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        int v = (int)(keys[r] & top);
        order[r] = v;
        rank[v] = r;
    }
}

__device__ __forceinline__ int warp_sum_i(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Alg. 5: calls of Alg. 4 with colors 0, 1, ... until every vertex has one;
// one warp.  Shared memory: inV, inBar, inW per vertex, then the bitmaps hat
// (W^, by rank) and si (S_i of the current pick, by vertex).
__global__ void __launch_bounds__(32) k_vertices_grouping(int n, const int *sr, const int *sc, const int *order,
                                                          const int *rank, int *color, int *ncolors, int *err) {
    extern __shared__ unsigned char gsm[];
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x;
    int nw = (n + 31) >> 5;
    unsigned char *inV = gsm, *inBar = gsm + n, *inW = gsm + 2 * n;
    unsigned *hat = reinterpret_cast<unsigned *>(gsm + ((3 * n + 15) & ~15));
    unsigned *si = hat + nw;
    for (int i = lane; i < n; i += 32) {
        inV[i] = 1;
        color[i] = -1;
    }
    __syncwarp();
    int total = n, c = 0;
    long steps = 0, cap = (long)n * n + 64;
    while (total > 0) {
        // one call of Alg. 4 (VerticesSplitting) on V, giving color c to W
        int left = 0;
        for (int i = lane; i < n; i += 32) {
            inW[i] = 0;
            inBar[i] = 0;
            left += inV[i];
        }
        for (int w = lane; w < nw; w += 32) {
            hat[w] = 0u;
            si[w] = 0u;
        }
        left = warp_sum_i(left);
        __syncwarp();
        int nhat = 0, hmin = 0, pa = 0, nW = 0;
        while (left > 0) {
            if (++steps > cap) {
                if (lane == 0) set_err(err, CPR_ERR_CUDA);
                return;
            }
            // the pick: the first candidate in rank order
            int i = -1;
            if (nhat > 0) {
                for (int w0 = hmin; w0 < nw && i < 0; w0 += 32) {
                    int w = w0 + lane;
                    unsigned bits = w < nw ? hat[w] : 0u;
                    unsigned ball = __ballot_sync(full, bits != 0u);
                    if (ball) {
                        int f = __ffs(ball) - 1;
                        unsigned wb = __shfl_sync(full, bits, f);
                        int r = (w0 + f) * 32 + __ffs(wb) - 1;
                        i = order[r];
                        hmin = w0 + f;
                    }
                }
            } else {
                while (pa < n) {
                    int r = pa + lane;
                    int v = r < n ? order[r] : -1;
                    bool av = v >= 0 && inV[v] && !inBar[v] && !inW[v];
                    unsigned ball = __ballot_sync(full, av);
                    if (ball) {
                        int f = __ffs(ball) - 1;
                        i = __shfl_sync(full, v, f);
                        pa += f;
                        break;
                    }
                    pa += 32;
                }
            }
            if (i < 0) {   // left > 0 guarantees a candidate; never taken
                if (lane == 0) set_err(err, CPR_ERR_CUDA);
                return;
            }
            int e0 = sr[i], e1 = sr[i + 1];
            bool any_w = false;
            for (int p = e0 + lane; p < e1; p += 32) any_w |= inW[sc[p]] != 0;
            any_w = __any_sync(full, any_w);
            int ri = rank[i];
            unsigned bi = 1u << (ri & 31);
            bool in_hat = (hat[ri >> 5] & bi) != 0u;
            __syncwarp();
            if (in_hat) {
                if (lane == 0) hat[ri >> 5] &= ~bi;
                nhat--;
            }
            left--;
            __syncwarp();
            if (any_w) {   // a strong neighbour is in W already: i waits for a later call
                if (lane == 0) inBar[i] = 1;
                __syncwarp();
                continue;
            }
            if (lane == 0) {
                inW[i] = 1;
                color[i] = c;
            }
            nW++;
            // S_i: marked in si; its members still in V leave for W-bar
            int nbar = 0, nout = 0;
            for (int p = e0 + lane; p < e1; p += 32) {
                int j = sc[p];
                atomicOr(&si[j >> 5], 1u << (j & 31));
                if (inV[j] && !inBar[j] && !inW[j]) {
                    inBar[j] = 1;
                    nbar++;
                    int rj = rank[j];
                    unsigned bj = 1u << (rj & 31);
                    if (atomicAnd(&hat[rj >> 5], ~bj) & bj) nout++;
                }
            }
            left -= warp_sum_i(nbar);
            nhat -= warp_sum_i(nout);
            __syncwarp();
            // the second circle of i joins W^
            for (int q = e0; q < e1; q++) {
                int k = sc[q];
                int f0 = sr[k], f1 = sr[k + 1];
                int nin = 0, wmin = nw;
                for (int p = f0 + lane; p < f1; p += 32) {
                    int j = sc[p];
                    if (j == i || !inV[j] || inBar[j] || inW[j]) continue;
                    if (si[j >> 5] & (1u << (j & 31))) continue;
                    int rj = rank[j];
                    unsigned bj = 1u << (rj & 31);
                    if (!(atomicOr(&hat[rj >> 5], bj) & bj)) {
                        nin++;
                        wmin = min(wmin, rj >> 5);
                    }
                }
                nhat += warp_sum_i(nin);
                wmin = __reduce_min_sync(full, (unsigned)wmin);
                hmin = min(hmin, wmin);
                __syncwarp();
            }
            for (int p = e0 + lane; p < e1; p += 32) {
                int j = sc[p];
                atomicAnd(&si[j >> 5], ~(1u << (j & 31)));
            }
            __syncwarp();
        }
        // the next call's V is this call's W-bar
        for (int i = lane; i < n; i += 32) inV[i] = inBar[i];
        __syncwarp();
        total -= nW;
        c++;
    }
    if (lane == 0) *ncolors = c;
}

// ---------------------------------------------------------------------- PMIS

__global__ void k_pmis_init(int n, const int *sr, const int *tr, int *cf, int *undecided) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool isolated = sr[i + 1] == sr[i] && tr[i + 1] == tr[i];
    cf[i] = isolated ? 0 : -1;
    if (!isolated) atomicAdd(undecided, 1);
}

// An undecided point whose key (lambda = |S^T_i|, hash, index) beats every
// undecided point of S_i u S^T_i is selected (cf is not written in this pass).
// G lanes share the point and load its entries P at a time, as in
// jp_vertex; every lane of the warp calls this, and the verdict is the
// group's.
template <int G, int P>
__device__ bool pmis_select(int i, bool act, int lane, const int *sr, const int *sc, const int *tr, const int *tc,
                            uint32_t hbase, const int *cf) {
    bool cand = act && cf[i] == -1;
    int li = 0, a0 = 0, na = 0, b0 = 0, nt = 0;
    uint32_t hi = 0;
    if (cand) {
        a0 = sr[i];
        na = sr[i + 1] - a0;
        b0 = tr[i];
        li = tr[i + 1] - b0;
        nt = na + li;
        hi = fmix32((uint32_t)i ^ hbase);
    }
    bool win = cand;
    for (int q0 = 0; q0 < nt; q0 += G * P) {
        int jj[P];
#pragma unroll
        for (int u = 0; u < P; u++) {
            int q = q0 + lane + u * G;
            jj[u] = q < nt ? (q < na ? sc[a0 + q] : tc[b0 + q - na]) : -1;
        }
        int cj[P], t0[P], t1[P];
#pragma unroll
        for (int u = 0; u < P; u++) {
            bool in = jj[u] >= 0;
            cj[u] = in ? cf[jj[u]] : 0;
            t0[u] = in ? tr[jj[u]] : 0;
            t1[u] = in ? tr[jj[u] + 1] : 0;
        }
#pragma unroll
        for (int u = 0; u < P; u++) {
            int j = jj[u];
            if (j < 0 || cj[u] != -1) continue;
            if (!key_greater(li, hi, i, t1[u] - t0[u], fmix32((uint32_t)j ^ hbase), j)) win = false;
        }
    }
    return group_all<G>(win);
}

// Selected points become C; undecided points with a C point in S_i become F.
// Returns, on the group's lane 0, whether point i was decided in this call.
// A point made C in this pass is also selected, so cf needs no volatile
// read.  Every lane of the warp calls this.
template <int G, int P>
__device__ bool pmis_commit(int i, bool act, int lane, const int *sr, const int *sc, int *cf, const int *sel) {
    bool si = act && sel[i] != 0;
    bool und = act && !si && cf[i] == -1;
    int a0 = 0, na = 0;
    if (und) {
        a0 = sr[i];
        na = sr[i + 1] - a0;
    }
    bool found = false;
    for (int q0 = 0; q0 < na; q0 += G * P) {
        int jj[P];
#pragma unroll
        for (int u = 0; u < P; u++) {
            int q = q0 + lane + u * G;
            jj[u] = q < na ? sc[a0 + q] : -1;
        }
        int sj[P], cj[P];
#pragma unroll
        for (int u = 0; u < P; u++) {
            bool in = jj[u] >= 0;
            sj[u] = in ? sel[jj[u]] : 0;
            cj[u] = in ? cf[jj[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < P; u++)
            if (jj[u] >= 0 && (sj[u] || cj[u] == 1)) found = true;
    }
    found = group_any<G>(found);
    if (lane != 0) return false;
    if (si) {
        cf[i] = 1;
        return true;
    }
    if (und && found) {
        cf[i] = 0;
        return true;
    }
    return false;
}

// The undecided count as lane 0 of the warp reads it, given to every lane, so
// that a warp returns early as a whole.
__device__ __forceinline__ int warp_read(const int *p) {
    int v = (threadIdx.x & 31) == 0 ? *(volatile const int *)p : 0;
    return __shfl_sync(0xffffffffu, v, 0);
}

// Rounds are launched in batches between host checks.  Once every point is
// decided the count is 0 and both kernels return at once.  The count reaches 0
// only with the last decision, and a point with a decision pending still
// counts itself, so no commit that is due is skipped.  G lanes per point.
template <int G>
__global__ void k_pmis_select(int n, const int *sr, const int *sc, const int *tr, const int *tc,
                              uint32_t hbase, const int *cf, int *sel, const int *undecided) {
    if (warp_read(undecided) == 0) return;
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    bool act = t < n;
    int i = act ? (int)t : 0;
    bool w = pmis_select<G, kJpPre>(i, act, lane, sr, sc, tr, tc, hbase, cf);
    if (act && lane == 0) sel[i] = w ? 1 : 0;
}

template <int G>
__global__ void k_pmis_commit(int n, const int *sr, const int *sc, int *cf, const int *sel, int *undecided) {
    if (warp_read(undecided) == 0) return;
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    bool act = t < n;
    int i = act ? (int)t : 0;
    bool d = pmis_commit<G, kJpPre>(i, act, lane, sr, sc, cf, sel);
    unsigned b = __ballot_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0 && b) atomicSub(undecided, __popc(b));
}

// All PMIS rounds of a small level in one CTA (the same rounds as above).
template <int G>
__global__ void __launch_bounds__(1024) k_pmis_small(int n, const int *sr, const int *sc, const int *tr,
                                                     const int *tc, uint32_t hbase, int *cf, int *sel,
                                                     const int *undecided0) {
    __shared__ int und;
    if (threadIdx.x == 0) und = *undecided0;
    __syncthreads();
    int lane = threadIdx.x % G, per = blockDim.x / G;
    for (int round = 0; round < n + 8; round++) {
        int left = und;
        __syncthreads();
        if (left == 0) break;
        for (int v0 = 0; v0 < n; v0 += per) {   // uniform over the block
            int i = v0 + (int)threadIdx.x / G;
            bool w = pmis_select<G, kJpPreSmall>(i, i < n, lane, sr, sc, tr, tc, hbase, cf);
            if (i < n && lane == 0) sel[i] = w ? 1 : 0;
        }
        __syncthreads();
        for (int v0 = 0; v0 < n; v0 += per) {
            int i = v0 + (int)threadIdx.x / G;
            if (pmis_commit<G, kJpPreSmall>(i, i < n, lane, sr, sc, cf, sel)) atomicSub(&und, 1);
        }
        __syncthreads();
    }
}

__global__ void k_is_c(int n, const int *cf, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cf[i] == 1;
}

// ------------------------------------------------- pairwise aggregation (UA-AMG)
//
// One matching pass of the pairwise aggregation Sec. 6 names for its first
// stage, taken on the symmetric part of A: c_ij = (a_ij + a_ji) / 2, and j is
// a strong neighbour of i when c_ij < 0 and -c_ij >= beta max_{k != i}(-c_ik).
// Nodes pair up in handshake rounds: every unmatched node points to its
// unmatched candidate (a strong neighbour in either direction) of smallest
// edge key (c_ij, smaller hash, larger hash, index); mutual pointers pair, and
// a node with no unmatched candidate is left alone.  A node left alone that
// has a candidate then joins the pair of its best candidate (rounds alone
// leave many singletons on heterogeneous media, and coarsening stalls); the
// others stay single.  Aggregates are numbered by the smaller node of their
// pair (or the single node).  Every FP64 operation is the plain
// definition's, in its order, so the result equals a sequential evaluation.

// The symmetric couplings of row i, merged from row i of A and of A^T (both
// sorted); f(j, c) is called for every j != i in ascending order.
template <class F>
__device__ __forceinline__ void pair_couplings(int i, int n, const int *ar, const int *ac, const double *av,
                                               const int *tr, const int *tc, const double *tv, F f) {
    int p = ar[i], pe = ar[i + 1], q = tr[i], qe = tr[i + 1];
    while (p < pe || q < qe) {
        int a = p < pe ? ac[p] : n, b = q < qe ? tc[q] : n;
        int j = a < b ? a : b;
        double c = 0.0;
        if (a == j) c = __dadd_rn(c, av[p++]);
        if (b == j) c = __dadd_rn(c, tv[q++]);
        if (j == i) continue;
        f(j, __dmul_rn(0.5, c));
    }
}

// Strong neighbours of each row: counts (scol == nullptr) or columns and
// couplings at srow[i].
__global__ void k_pair_strong(int n, const int *ar, const int *ac, const double *av, const int *tr,
                              const int *tc, const double *tv, double beta, const int *srow, int *cnt,
                              int *scol, double *sval) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double maxneg = 0.0;
    pair_couplings(i, n, ar, ac, av, tr, tc, tv, [&](int, double c) {
        if (-c > maxneg) maxneg = -c;
    });
    double lim = __dmul_rn(beta, maxneg);
    int o = scol ? srow[i] : 0;
    pair_couplings(i, n, ar, ac, av, tr, tc, tv, [&](int j, double c) {
        if (c < 0.0 && maxneg > 0.0 && -c >= lim) {
            if (scol) {
                scol[o] = j;
                sval[o] = c;
            }
            o++;
        }
    });
    if (!scol) cnt[i] = o;
}

constexpr int kUnmatched = -2, kAlone = -1;

// The unmatched candidate of smallest edge key among S_i and (S^T)_i.
__device__ int hs_best(int i, const int *sr, const int *sc, const double *sv, const int *tr, const int *tc,
                       const double *tv, const int *mate, uint32_t hb) {
    int bj = -1;
    double bc = 0.0;
    uint32_t blo = 0, bhi = 0;
    uint32_t hi_ = fmix32((uint32_t)i ^ hb);
    volatile const int *vm = mate;
    for (int pass = 0; pass < 2; pass++) {
        const int *R = pass ? tr : sr, *Cc = pass ? tc : sc;
        const double *V = pass ? tv : sv;
        for (int t = R[i]; t < R[i + 1]; t++) {
            int j = Cc[t];
            if (j == i || vm[j] != kUnmatched) continue;
            uint32_t hj = fmix32((uint32_t)j ^ hb);
            uint32_t lo = hi_ < hj ? hi_ : hj, hi = hi_ < hj ? hj : hi_;
            double c = V[t];
            bool better = bj < 0 || c < bc ||
                          (c == bc && (lo < blo || (lo == blo && (hi < bhi || (hi == bhi && j < bj)))));
            if (better) {
                bj = j;
                bc = c;
                blo = lo;
                bhi = hi;
            }
        }
    }
    return bj;
}

// A round: pointers from the round-start state, then the commits.  The count
// of unmatched nodes reaches 0 with the last commit; then both kernels return
// at once (rounds run in batches between host checks).
__global__ void k_hs_point(int n, const int *sr, const int *sc, const double *sv, const int *tr, const int *tc,
                           const double *tv, const int *mate, int *ptr, uint32_t hb, const int *left) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || *(volatile const int *)left == 0) return;
    ptr[i] = mate[i] == kUnmatched ? hs_best(i, sr, sc, sv, tr, tc, tv, mate, hb) : -1;
}

__device__ __forceinline__ int hs_commit(int i, int *mate, const int *ptr) {
    if (mate[i] != kUnmatched) return 0;
    int p = ptr[i];
    if (p < 0) {
        mate[i] = kAlone;
        return 1;
    }
    if (ptr[p] == i) {
        mate[i] = p;
        return 1;
    }
    return 0;
}

__global__ void k_hs_commit(int n, int *mate, const int *ptr, int *left) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || *(volatile int *)left == 0) return;
    if (hs_commit(i, mate, ptr)) atomicSub(left, 1);
}

// All rounds of a small level in one CTA (the same rounds).
__global__ void __launch_bounds__(1024) k_hs_small(int n, const int *sr, const int *sc, const double *sv,
                                                   const int *tr, const int *tc, const double *tv, int *mate,
                                                   int *ptr, uint32_t hb) {
    __shared__ int left;
    if (threadIdx.x == 0) left = n;
    __syncthreads();
    for (int round = 0; round < n + 8; round++) {
        int l = left;
        __syncthreads();
        if (l == 0) break;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            ptr[i] = mate[i] == kUnmatched ? hs_best(i, sr, sc, sv, tr, tc, tv, mate, hb) : -1;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (hs_commit(i, mate, ptr)) atomicSub(&left, 1);
        __syncthreads();
    }
}

// After the rounds, a node left alone that has a candidate joins the pair of
// its candidate of smallest edge key (all its candidates are paired: an
// unmatched one would have kept both nodes pointing); host[i] = that
// candidate, or -1.
__global__ void k_hs_host(int n, const int *sr, const int *sc, const double *sv, const int *tr, const int *tc,
                          const double *tv, const int *mate, uint32_t hb, int *host) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bj = -1;
    if (mate[i] == kAlone) {
        double bc = 0.0;
        uint32_t blo = 0, bhi = 0;
        uint32_t hi_ = fmix32((uint32_t)i ^ hb);
        for (int pass = 0; pass < 2; pass++) {
            const int *R = pass ? tr : sr, *Cc = pass ? tc : sc;
            const double *V = pass ? tv : sv;
            for (int t = R[i]; t < R[i + 1]; t++) {
                int j = Cc[t];
                if (j == i) continue;
                uint32_t hj = fmix32((uint32_t)j ^ hb);
                uint32_t lo = hi_ < hj ? hi_ : hj, hi = hi_ < hj ? hj : hi_;
                double c = V[t];
                bool better = bj < 0 || c < bc ||
                              (c == bc && (lo < blo || (lo == blo && (hi < bhi || (hi == bhi && j < bj)))));
                if (better) {
                    bj = j;
                    bc = c;
                    blo = lo;
                    bhi = hi;
                }
            }
        }
    }
    host[i] = bj;
}

// Aggregates are numbered by their leader: the smaller node of a pair, or a
// node left alone with no host.
__global__ void k_hs_leader(int n, const int *mate, const int *host, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = mate[i] >= 0 ? mate[i] > i : host[i] < 0;
}

__global__ void k_hs_number(int n, const int *mate, const int *host, const int *idx, int *agg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = host[i] >= 0 ? host[i] : i;   // a joining node takes its host pair's number
    int m = mate[k];
    agg[i] = idx[m >= 0 && m < k ? m : k];
}

__global__ void k_fill_int(int n, int *a, int v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// Unsmoothed aggregation's P: row i is the unit row of aggregate agg[i].
__global__ void k_unit_p(int n, const int *agg, int *rowptr, int *col, double *val) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    rowptr[i] = i;
    if (i == n) return;
    col[i] = agg[i];
    val[i] = 1.0;
}

// agg[i] <- second[first[i]]: the two passes composed.
__global__ void k_compose_agg(int n, const int *first, const int *second, int *agg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = second[first[i]];
}

// ------------------------------------------------------ direct interpolation

__global__ void k_interp_count(int n, const int *sr, const int *sc, const int *cf, int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == 1) {
        cnt[i] = 1;
        return;
    }
    int c = 0;
    for (int p = sr[i]; p < sr[i + 1]; p++) c += cf[sc[p]] == 1;
    cnt[i] = c;
}

// Row i of Stueben's direct interpolation with separate negative/positive
// scaling and lumping of the positive part into the diagonal when C_i has no
// positive entry, for an F point.  col/val: row i of A (len entries, sorted);
// sc: row i of the strength set (slen entries, sorted), of which the entries
// with cf == 1 are C_i (cf == nullptr: sc holds C_i alone); pc/pv: row i of
// P.  Every sum runs in row order.
__device__ void interp_row(int i, const int *col, const double *val, int len, const int *sc, int slen,
                           const int *cf, const int *cidx, int *pc, double *pv) {
    double aii = 0.0;
    for (int p = 0; p < len; p++)
        if (col[p] == i) aii = val[p];
    double s = aii < 0.0 ? -1.0 : 1.0;
    double sum_n_neg = 0.0, sum_n_pos = 0.0;
    for (int p = 0; p < len; p++) {
        if (col[p] == i) continue;
        double v = __dmul_rn(s, val[p]);
        if (v < 0.0) sum_n_neg = __dadd_rn(sum_n_neg, v);
        else sum_n_pos = __dadd_rn(sum_n_pos, v);
    }
    double sum_c_neg = 0.0, sum_c_pos = 0.0;
    int pa = 0;
    for (int t = 0; t < slen; t++) {
        int j = sc[t];
        if (cf && cf[j] != 1) continue;
        while (col[pa] != j) pa++;
        double v = __dmul_rn(s, val[pa]);
        if (v < 0.0) sum_c_neg = __dadd_rn(sum_c_neg, v);
        else sum_c_pos = __dadd_rn(sum_c_pos, v);
    }
    double d = __dmul_rn(s, aii);
    double alpha = 0.0, beta = 0.0;
    if (sum_c_neg != 0.0) alpha = __ddiv_rn(sum_n_neg, sum_c_neg);
    if (sum_c_pos != 0.0) beta = __ddiv_rn(sum_n_pos, sum_c_pos);
    else d = __dadd_rn(d, sum_n_pos);
    pa = 0;
    int q = 0;
    for (int t = 0; t < slen; t++) {
        int j = sc[t];
        if (cf && cf[j] != 1) continue;
        while (col[pa] != j) pa++;
        double v = __dmul_rn(s, val[pa]);
        double f = v < 0.0 ? -alpha : -beta;
        pc[q] = cidx[j];
        pv[q] = __ddiv_rn(__dmul_rn(f, v), d);
        q++;
    }
}

// Direct interpolation, one thread per row: a C point's row is the unit row
// of its coarse index.
__global__ void k_interp_fill(int n, const int *ar, const int *ac, const double *av,
                              const int *sr, const int *sc, const int *cf, const int *cidx,
                              const int *pr, int *pc, double *pv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = pr[i];
    if (cf[i] == 1) {
        pc[q] = cidx[i];
        pv[q] = 1.0;
        return;
    }
    int a = ar[i];
    interp_row(i, ac + a, av + a, ar[i + 1] - a, sc + sr[i], sr[i + 1] - sr[i], cf, cidx, pc + q, pv + q);
}

// Direct interpolation for long rows on small levels, one warp per row (there
// a thread per row leaves most of the GPU idle and walks its row alone).
// The warp stages row i of A with coalesced loads, finds a_ii, scales the row
// by its sign s and looks up C_i's entries, all across the lanes; one lane
// folds the four sums in row order; then each lane writes its share of P's
// row, one quotient per entry.  The arithmetic, and the order of every sum,
// is interp_row's.  A row larger than the staging area (row of A, or its
// strength row) runs interp_row on global memory.
constexpr int kInterpWarps = 4;
constexpr int kInterpCapA = 512;
constexpr int kInterpCapS = 256;
constexpr int kInterpWarpRows = 16384;   // levels up to this size take the warp kernel
__global__ void __launch_bounds__(kInterpWarps * 32) k_interp_fill_warp(int n, const int *ar, const int *ac,
                                                                        const double *av, const int *sr,
                                                                        const int *sc, const int *cf,
                                                                        const int *cidx, const int *pr, int *pc,
                                                                        double *pv) {
    __shared__ int scol[kInterpWarps][kInterpCapA];
    __shared__ double sval[kInterpWarps][kInterpCapA];   // a_ij, then s a_ij
    __shared__ int sC[kInterpWarps][kInterpCapS];        // C_i in strength-row order
    __shared__ double sv[kInterpWarps][kInterpCapS];     // s a_ij for j in C_i
    __shared__ double scal[kInterpWarps][3];             // d, alpha, beta
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    unsigned lt = (1u << lane) - 1u;
    int *col = scol[wl], *C = sC[wl];
    double *val = sval[wl], *cv = sv[wl];
    for (int i = blockIdx.x * kInterpWarps + wl; i < n; i += gridDim.x * kInterpWarps) {
        int q = pr[i];
        if (cf[i] == 1) {
            if (lane == 0) {
                pc[q] = cidx[i];
                pv[q] = 1.0;
            }
            continue;
        }
        int a = ar[i], len = ar[i + 1] - a, s0 = sr[i], slen = sr[i + 1] - s0;
        if (len > kInterpCapA || slen > kInterpCapS) {
            if (lane == 0) interp_row(i, ac + a, av + a, len, sc + s0, slen, cf, cidx, pc + q, pv + q);
            __syncwarp();
            continue;
        }
        double aii = 0.0;
        bool diag = false;
        for (int t = lane; t < len; t += 32) {
            int c = ac[a + t];
            double v = av[a + t];
            col[t] = c;
            val[t] = v;
            if (c == i) {
                aii = v;
                diag = true;
            }
        }
        unsigned has = __ballot_sync(0xffffffffu, diag);   // a row holds its diagonal once
        aii = has ? __shfl_sync(0xffffffffu, aii, 31 - __clz(has)) : 0.0;
        double s = aii < 0.0 ? -1.0 : 1.0;
        for (int t = lane; t < len; t += 32) val[t] = __dmul_rn(s, val[t]);
        int m = 0;
        for (int t0 = 0; t0 < slen; t0 += 32) {
            int t = t0 + lane;
            int j = t < slen ? sc[s0 + t] : 0;
            bool c = t < slen && cf[j] == 1;
            unsigned bal = __ballot_sync(0xffffffffu, c);
            if (c) C[m + __popc(bal & lt)] = j;
            m += __popc(bal);
        }
        __syncwarp();
        for (int t = lane; t < m; t += 32) {   // C_i lies in row i's pattern
            int pos = min(find_col(col, 0, len, C[t]), len - 1);
            cv[t] = val[pos];
        }
        __syncwarp();
        if (lane == 0) {
            double sum_n_neg = 0.0, sum_n_pos = 0.0, sum_c_neg = 0.0, sum_c_pos = 0.0;
            for (int p = 0; p < len; p++) {
                if (col[p] == i) continue;
                double v = val[p];
                if (v < 0.0) sum_n_neg = __dadd_rn(sum_n_neg, v);
                else sum_n_pos = __dadd_rn(sum_n_pos, v);
            }
            for (int t = 0; t < m; t++) {
                double v = cv[t];
                if (v < 0.0) sum_c_neg = __dadd_rn(sum_c_neg, v);
                else sum_c_pos = __dadd_rn(sum_c_pos, v);
            }
            double d = __dmul_rn(s, aii);
            double alpha = 0.0, beta = 0.0;
            if (sum_c_neg != 0.0) alpha = __ddiv_rn(sum_n_neg, sum_c_neg);
            if (sum_c_pos != 0.0) beta = __ddiv_rn(sum_n_pos, sum_c_pos);
            else d = __dadd_rn(d, sum_n_pos);
            scal[wl][0] = d;
            scal[wl][1] = alpha;
            scal[wl][2] = beta;
        }
        __syncwarp();
        double d = scal[wl][0], alpha = scal[wl][1], beta = scal[wl][2];
        for (int t = lane; t < m; t += 32) {
            double v = cv[t];
            double f = v < 0.0 ? -alpha : -beta;
            pc[q + t] = cidx[C[t]];
            pv[q + t] = __ddiv_rn(__dmul_rn(f, v), d);
        }
        __syncwarp();
    }
}

// Direct interpolation into P's pattern: warp per row on small levels whose
// rows average more than 16 entries, else thread per row.
void interp_fill(const DCsr &A, const int *sr, const int *sc, const int *cf, const int *cidx, DCsr &P,
                 cudaStream_t s) {
    int n = A.n;
    if (!n) return;
    if (n <= kInterpWarpRows && A.nnz > 16L * n)
        k_interp_fill_warp<<<grid_for(n, kInterpWarps), kInterpWarps * 32, 0, s>>>(
            n, A.rowptr.p, A.col.p, A.val.p, sr, sc, cf, cidx, P.rowptr.p, P.col.p, P.val.p);
    else
        k_interp_fill<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, sr, sc, cf, cidx,
                                                            P.rowptr.p, P.col.p, P.val.p);
    CK_LAUNCH();
}

// ------------------------------------------------- SpGEMM with per-warp hashing
//
// One warp per row of C = A B.  Symbolic: the row's candidate columns (B_k for
// k in A_i) go into a shared-memory hash set.  Numeric: the warp extracts and
// sorts the row's columns, then adds a_ik b_kJ into a shared accumulator with k
// in ascending order (one k at a time, lanes over B_k's distinct columns), so
// every C entry is summed in the same order as Gustavson's row-by-row product.
// Rows with more distinct columns than the table holds take an exact slow path.

// Six tiers, chosen per row from its length in A and its candidate product
// count (sum over k in A_i of |B_k|).  The first three take one thread per
// row.  Rows with at most 8 (or 9 to 16) entries in A and few candidates
// (every row of A P at levels 0 and 1, most rows of R (A P) at level 0) are
// merged from their B rows (each sorted) held as list heads in registers:
// the smallest head column is the next C column, and its products are added
// in list order, i.e. ascending k.  Other rows with at most kTinyCand
// candidates insertion-sort their products by column in the thread's own
// arrays (stable, so each column's products stay in ascending k) and sum each
// column's run in that order.  Rows up to kSmallCand candidates run with small
// per-warp tables at full occupancy, rows up to kMidCand (most of R (A P) at
// the coarser levels) with medium tables, still at full occupancy, the rest
// with large tables.  A merge costs the thread one step per C column and list
// head, so long merges go to the tables, whose warps split a row's products.
//   CAP: hash slots per warp (power of two); HMAX: distinct columns handled
//   in shared memory, a power of two (larger rows take the exact slow path);
//   WARPS per block.
constexpr int kMerge8Cand = 64;    // merge tier 0: at most 8 entries in A and this many candidates
constexpr int kMerge16Cand = 48;   // merge tier 1: 9 to 16 entries in A and this many candidates
constexpr int kTinyCand = 24;
constexpr int kSmallCand = 32;
constexpr int kMidCand = 160;      // rows above kSmallCand and up to this: 256-slot tables
enum { kTierMerge8, kTierMerge16, kTierTiny, kTierSmall, kTierMid, kTierBig };

__device__ __forceinline__ int spgemm_tier(int len, int cand) {
    if (len <= 8 && cand <= kMerge8Cand) return kTierMerge8;
    if (len <= 16 && cand <= kMerge16Cand) return kTierMerge16;
    if (cand <= kTinyCand) return kTierTiny;
    if (cand <= kSmallCand) return kTierSmall;
    return cand <= kMidCand ? kTierMid : kTierBig;
}
constexpr int kEmpty = -1;

// Per-warp scratch for enumerating the products of one chunk of 32 A entries:
// product t of the chunk belongs to entry e with off[e] <= t < off[e + 1] and
// reads B entry st[e] + t - off[e].
struct ProdChunk {
    int off[33];
    int st[32];
    double av[32];
};

// Loads one chunk of row entries [a0, min(a0 + 32, b)) and scans their B row
// lengths; returns the chunk's product count.
__device__ __forceinline__ int load_chunk(int a0, int b, const int *ac, const double *av, const int *br,
                                          ProdChunk &pc, int lane) {
    int p = a0 + lane, len = 0, st = 0;
    double v = 0.0;
    if (p < b) {
        int k = ac[p];
        st = br[k];
        len = br[k + 1] - st;
        if (av) v = av[p];
    }
    int inc = len;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    pc.off[lane] = inc - len;
    pc.st[lane] = st;
    pc.av[lane] = v;
    int tot = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 31) pc.off[32] = tot;
    __syncwarp();
    return tot;
}

// The chunk entry that product t belongs to (the last e with off[e] <= t).
__device__ __forceinline__ int chunk_owner(const ProdChunk &pc, int t) {
    int lo = 0, hi = 31;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pc.off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Insert every candidate column of row i into a table of *cap slots (sized
// from the row's candidate count, 32..CAP); returns the distinct count, or
// HMAX+1 when the row is too large for the shared path.  All products
// of a chunk of 32 A entries are enumerated at once (one per lane), so the
// row costs one chain of dependent loads per chunk, not one per A entry.
// With SKIP, a row with more than HMAX candidates is left alone (returns -1).
template <int CAP, int HMAX, bool SKIP>
__device__ int hash_row(int i, const int *ar, const int *ac, const int *br, const int *bc, int *tab,
                        int *cnt, int lane, int *cap_out, ProdChunk &pc) {
    int a = ar[i], b = ar[i + 1];
    int cand = 0;
    for (int p = a + lane; p < b; p += 32) {
        int k = ac[p];
        cand += br[k + 1] - br[k];
    }
    for (int sh = 16; sh > 0; sh >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, sh);
    if (SKIP && cand > HMAX) return -1;
    int cap = 32;
    while (cap < CAP && cap < 2 * cand) cap <<= 1;
    *cap_out = cap;
    for (int t = lane; t < cap; t += 32) tab[t] = kEmpty;
    if (lane == 0) *cnt = 0;
    __syncwarp();
    bool overflow = false;
    int limit = min(HMAX, cap / 2 + cap / 4);
    for (int a0 = a; a0 < b; a0 += 32) {
        int tot = load_chunk(a0, b, ac, nullptr, br, pc, lane);
        for (int t = lane; t < tot && !overflow; t += 32) {
            int e = chunk_owner(pc, t);
            int J = bc[pc.st[e] + t - pc.off[e]];
            unsigned slot = ((unsigned)J * 2654435761u) & (cap - 1);
            for (int probe = 0; probe < cap; probe++) {
                int prev = atomicCAS(&tab[slot], kEmpty, J);
                if (prev == kEmpty) {
                    if (atomicAdd(cnt, 1) >= limit) overflow = true;
                    break;
                }
                if (prev == J) break;
                slot = (slot + 1) & (cap - 1);
            }
        }
        __syncwarp();
    }
    __syncwarp();
    int c = *cnt;
    return c > limit ? HMAX + 1 : c;
}

// Exact slow path for a large row: the next distinct column above `last`,
// found by one pass over all candidates (warp minimum).
__device__ int next_col(int i, long last, const int *ar, const int *ac, const int *br, const int *bc,
                        int lane) {
    int m = INT_MAX;
    for (int p = ar[i] + lane; p < ar[i + 1]; p += 32) {
        int k = ac[p];
        for (int q = br[k]; q < br[k + 1]; q++) {
            int J = bc[q];
            if (J > last && J < m) m = J;
        }
    }
    for (int sh = 16; sh > 0; sh >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, sh));
    return m;
}

// The rows of the three table tiers: `small`, `mid` and `big`, each list in
// any order.  cnt: their lengths.
__global__ void k_spgemm_cand(int n, const int *ar, const int *ac, const int *br, int *small, int *mid, int *big,
                              int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int p = ar[i]; p < ar[i + 1]; p++) {
        int k = ac[p];
        c += br[k + 1] - br[k];
    }
    int tier = spgemm_tier(ar[i + 1] - ar[i], c);
    if (tier == kTierBig) big[atomicAdd(&cnt[2], 1)] = i;
    else if (tier == kTierMid) mid[atomicAdd(&cnt[1], 1)] = i;
    else if (tier == kTierSmall) small[atomicAdd(&cnt[0], 1)] = i;
}

// A merge tier (ML list heads: tier kTierMerge8 or kTierMerge16), one thread
// per row of that tier (other rows are skipped).  Without cr, counts the
// row's distinct columns into ucnt; with cr, writes the row's columns
// (ascending) and values.
template <int ML, int TIER>
__global__ void k_spgemm_merge(int n, const int *ar, const int *ac, const double *av, const int *br,
                               const int *bc, const double *bv, const int *cr, int *cc, double *cv, int *ucnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = ar[i], b = ar[i + 1];
    if (b - a > ML) return;
    int q[ML], e[ML], hd[ML];
    double x[ML];
    int cand = 0;
#pragma unroll
    for (int t = 0; t < ML; t++) {
        bool in = a + t < b;
        int k = in ? ac[a + t] : 0;
        q[t] = in ? br[k] : 0;
        e[t] = in ? br[k + 1] : 0;
        x[t] = in && cr ? av[a + t] : 0.0;
        cand += e[t] - q[t];
    }
    if (spgemm_tier(b - a, cand) != TIER) return;
#pragma unroll
    for (int t = 0; t < ML; t++) hd[t] = q[t] < e[t] ? bc[q[t]] : INT_MAX;
    int o = cr ? cr[i] : 0, c = 0;
    for (;;) {
        int J = INT_MAX;
#pragma unroll
        for (int t = 0; t < ML; t++) J = min(J, hd[t]);
        if (J == INT_MAX) break;
        double sum = 0.0;
#pragma unroll
        for (int t = 0; t < ML; t++)
            if (hd[t] == J) {   // a B row holds each column once
                if (cr) sum = __dadd_rn(sum, __dmul_rn(x[t], bv[q[t]]));
                q[t]++;
                hd[t] = q[t] < e[t] ? bc[q[t]] : INT_MAX;
            }
        if (cr) {
            cc[o] = J;
            cv[o] = sum;
            o++;
        }
        c++;
    }
    if (!cr) ucnt[i] = c;
}

// The tiny tier: one thread per row of tier kTierTiny (other rows are
// skipped).  Without cr, counts the row's distinct columns into ucnt; with
// cr, writes the row's columns (ascending) and values.
__global__ void k_spgemm_tiny(int n, const int *ar, const int *ac, const double *av, const int *br,
                              const int *bc, const double *bv, const int *cr, int *cc, double *cv, int *ucnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = ar[i], b = ar[i + 1];
    int cand = 0;
    for (int p = a; p < b; p++) {
        int k = ac[p];
        cand += br[k + 1] - br[k];
    }
    if (spgemm_tier(b - a, cand) != kTierTiny) return;
    int J[kTinyCand];
    double V[kTinyCand];
    int m = 0;
    for (int p = a; p < b; p++) {
        int k = ac[p];
        double x = cr ? av[p] : 0.0;
        for (int q = br[k]; q < br[k + 1]; q++) {
            int j = bc[q];
            double v = cr ? __dmul_rn(x, bv[q]) : 0.0;
            int pos = m++;
            while (pos > 0 && J[pos - 1] > j) {   // stable: equal columns keep their k order
                J[pos] = J[pos - 1];
                V[pos] = V[pos - 1];
                pos--;
            }
            J[pos] = j;
            V[pos] = v;
        }
    }
    if (!cr) {
        int c = 0;
        for (int t = 0; t < m; t++) c += t == 0 || J[t] != J[t - 1];
        ucnt[i] = c;
        return;
    }
    int o = cr[i];
    for (int t = 0; t < m;) {
        int j = J[t];
        double sum = 0.0;
        for (; t < m && J[t] == j; t++) sum = __dadd_rn(sum, V[t]);
        cc[o] = j;
        cv[o] = sum;
        o++;
    }
}

// One warp per row, grid-stride: rows 0..n-1, or the *nrows rows listed in
// `rows` (a count on the device, so the launch needs no read-back).  With
// SKIP, rows with more than HMAX candidates are left to the large-table launch.
template <int CAP, int HMAX, int WARPS, bool SKIP>
__global__ void __launch_bounds__(WARPS * 32) k_spgemm_rowcount(int n, const int *rows, const int *nrows,
                                                                const int *ar, const int *ac, const int *br,
                                                                const int *bc, int *ucnt) {
    __shared__ int tab[WARPS][CAP];
    __shared__ int cnt[WARPS];
    __shared__ ProdChunk pcs[WARPS];
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    int nn = rows ? *nrows : n;
    for (int w = blockIdx.x * WARPS + wl; w < nn; w += gridDim.x * WARPS) {
        int i = rows ? rows[w] : w;
        int cap;
        int c = hash_row<CAP, HMAX, SKIP>(i, ar, ac, br, bc, tab[wl], &cnt[wl], lane, &cap, pcs[wl]);
        if (c < 0) continue;
        if (c > HMAX) {
            c = 0;
            for (long last = -1;;) {
                int J = next_col(i, last, ar, ac, br, bc, lane);
                if (J == INT_MAX) break;
                c++;
                last = J;
            }
        }
        if (lane == 0) ucnt[i] = c;
        __syncwarp();
    }
}

// Numeric row i of C = A B with this warp's shared tables (see below).
template <int CAP, int HMAX, bool SKIP>
__device__ void spgemm_fill_row(int i, const int *ar, const int *ac, const double *av, const int *br,
                                const int *bc, const double *bv, const int *cr, int *cc, double *cv, int *tab,
                                int *keys, double *acc, int *cnt, ProdChunk &pc, int lane) {
    unsigned lt = (1u << lane) - 1u;
    int cap;
    int c = hash_row<CAP, HMAX, SKIP>(i, ar, ac, br, bc, tab, cnt, lane, &cap, pc);
    if (c < 0) return;
    int base = cr[i];
    int a = ar[i], b = ar[i + 1];
    if (c > HMAX) {
        // slow path: columns by repeated minimum, values pulled per column
        int e = 0;
        for (long last = -1;;) {
            int J = next_col(i, last, ar, ac, br, bc, lane);
            if (J == INT_MAX) break;
            if (lane == 0) cc[base + e] = J;
            e++;
            last = J;
        }
        __syncwarp();
        for (int q = base + lane; q < base + e; q += 32) {
            int J = cc[q];
            double s = 0.0;
            for (int p = a; p < b; p++) {
                int k = ac[p];
                int lo = br[k], hi = br[k + 1];
                int f = find_col(bc, lo, hi, J);
                if (f < hi && bc[f] == J) s = __dadd_rn(s, __dmul_rn(av[p], bv[f]));
            }
            cv[q] = s;
        }
        return;
    }
    // compact the hash table into keys[0..c), then sort (bitonic)
    int *K = keys;
    int w = 0;
    for (int t0 = 0; t0 < cap; t0 += 32) {
        int v = tab[t0 + lane];
        bool keep = v != kEmpty;
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) K[w + __popc(m & lt)] = v;
        w += __popc(m);
    }
    int P = 1;
    while (P < c) P <<= 1;
    for (int t = c + lane; t < P; t += 32) K[t] = INT_MAX;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < P / 2; t += 32) {
                int x = (t / stride) * 2 * stride + (t % stride);
                int y = x + stride;
                bool up = (x & size) == 0;
                int u = K[x], v = K[y];
                if ((u > v) == up) {
                    K[x] = v;
                    K[y] = u;
                }
            }
            __syncwarp();
        }
    double *S = acc;
    for (int t = lane; t < c; t += 32) {
        S[t] = 0.0;
        cc[base + t] = K[t];
    }
    __syncwarp();
    // Products in (A entry, B entry) order, one per lane; each lane finds its
    // column's slot, then the lanes add in ascending A entry (ascending k)
    // order.  The columns of one B row are distinct, so lanes of one A entry
    // never collide, and every C entry is summed in Gustavson's order.
    for (int a0 = a; a0 < b; a0 += 32) {
        int tot = load_chunk(a0, b, ac, av, br, pc, lane);
        for (int t0 = 0; t0 < tot; t0 += 32) {
            int t = t0 + lane;
            int e = 32, slot = 0;
            double prod = 0.0;
            if (t < tot) {
                e = chunk_owner(pc, t);
                int q = pc.st[e] + t - pc.off[e];
                int J = bc[q];
                int lo = 0, hi = c;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (K[mid] < J) lo = mid + 1;
                    else hi = mid;
                }
                slot = lo;
                prod = __dmul_rn(pc.av[e], bv[q]);
            }
            int e_first = __shfl_sync(0xffffffffu, e, 0);
            int e_last = __shfl_sync(0xffffffffu, e, min(31, tot - 1 - t0));
            for (int ee = e_first; ee <= e_last; ee++) {
                if (e == ee) S[slot] = __dadd_rn(S[slot], prod);
                __syncwarp();
            }
        }
        __syncwarp();
    }
    for (int t = lane; t < c; t += 32) cv[base + t] = S[t];
}

template <int CAP, int HMAX, int WARPS, bool SKIP>
__global__ void __launch_bounds__(WARPS * 32) k_spgemm_rowfill(int n, const int *rows, const int *nrows,
                                                               const int *ar, const int *ac, const double *av,
                                                               const int *br, const int *bc, const double *bv,
                                                               const int *cr, int *cc, double *cv) {
    static_assert((HMAX & (HMAX - 1)) == 0, "HMAX bounds the bitonic sort: a power of two");
    __shared__ int tab[WARPS][CAP];
    __shared__ int keys[WARPS][HMAX];
    __shared__ double acc[WARPS][HMAX];
    __shared__ int cnt[WARPS];
    __shared__ ProdChunk pcs[WARPS];
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    int nn = rows ? *nrows : n;
    for (int w = blockIdx.x * WARPS + wl; w < nn; w += gridDim.x * WARPS) {
        spgemm_fill_row<CAP, HMAX, SKIP>(rows ? rows[w] : w, ar, ac, av, br, bc, bv, cr, cc, cv, tab[wl], keys[wl],
                                         acc[wl], &cnt[wl], pcs[wl], lane);
        __syncwarp();
    }
}

// C = A B for products with few columns (B.ncol <= kDenseCols): one warp per
// row of C with a dense accumulator of B.ncol values and a bitmap of the
// columns present, both in shared memory.  The row's products are taken in
// (A entry, B entry) order, one per lane, and the lanes add them in
// ascending A entry (ascending k) order, as the table tiers do, so every C
// entry is summed in Gustavson's order; the columns leave in ascending order
// from the bitmap.  Count pass (FILL false: ucnt = distinct columns) or fill
// pass.  The accumulator is zero between rows: a row's extraction clears
// what it used.  Dynamic shared memory: kDenseWarps * (ncol doubles when
// FILL, then ceil(ncol / 32) words).
constexpr int kDenseCols = 4096;
constexpr int kDenseWarps = 4;
template <bool FILL>
__global__ void __launch_bounds__(kDenseWarps * 32) k_spgemm_dense(int n, int ncol, const int *ar, const int *ac,
                                                                   const double *av, const int *br, const int *bc,
                                                                   const double *bv, const int *cr, int *cc,
                                                                   double *cv, int *ucnt) {
    extern __shared__ double dsm[];
    __shared__ ProdChunk pcs[kDenseWarps];
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    int nw = (ncol + 31) / 32;
    size_t per_warp = (FILL ? (size_t)ncol * sizeof(double) : 0) + (size_t)nw * sizeof(unsigned);
    per_warp = (per_warp + 15) & ~(size_t)15;
    char *base = reinterpret_cast<char *>(dsm) + wl * per_warp;
    double *acc = reinterpret_cast<double *>(base);
    unsigned *bits = reinterpret_cast<unsigned *>(base + (FILL ? (size_t)ncol * sizeof(double) : 0));
    if (FILL)
        for (int t = lane; t < ncol; t += 32) acc[t] = 0.0;
    for (int t = lane; t < nw; t += 32) bits[t] = 0u;
    __syncwarp();
    ProdChunk &pc = pcs[wl];
    for (int i = blockIdx.x * kDenseWarps + wl; i < n; i += gridDim.x * kDenseWarps) {
        int a = ar[i], b = ar[i + 1];
        for (int a0 = a; a0 < b; a0 += 32) {
            int tot = load_chunk(a0, b, ac, FILL ? av : nullptr, br, pc, lane);
            for (int t0 = 0; t0 < tot; t0 += 32) {
                int t = t0 + lane;
                int e = 32, J = 0;
                double prod = 0.0;
                if (t < tot) {
                    e = chunk_owner(pc, t);
                    int q = pc.st[e] + t - pc.off[e];
                    J = bc[q];
                    atomicOr(&bits[J >> 5], 1u << (J & 31));
                    if (FILL) prod = __dmul_rn(pc.av[e], bv[q]);
                }
                if (FILL) {
                    int e_first = __shfl_sync(0xffffffffu, e, 0);
                    int e_last = __shfl_sync(0xffffffffu, e, min(31, tot - 1 - t0));
                    for (int ee = e_first; ee <= e_last; ee++) {   // a B row holds each column once
                        if (e == ee) acc[J] = __dadd_rn(acc[J], prod);
                        __syncwarp();
                    }
                }
            }
            __syncwarp();
        }
        // the row's columns in ascending order: words across the lanes, a warp scan of their counts
        int o = FILL ? cr[i] : 0, total = 0;
        for (int w0 = 0; w0 < nw; w0 += 32) {
            int w = w0 + lane;
            unsigned word = w < nw ? bits[w] : 0u;
            int c = __popc(word), inc = c;
            for (int sh = 1; sh < 32; sh <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, inc, sh);
                if (lane >= sh) inc += y;
            }
            if (FILL) {
                int q = o + total + inc - c;
                while (word) {
                    int J = (w << 5) + __ffs(word) - 1;
                    word &= word - 1;
                    cc[q] = J;
                    cv[q] = acc[J];
                    acc[J] = 0.0;
                    q++;
                }
            }
            if (w < nw) bits[w] = 0u;
            total += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (!FILL && lane == 0) ucnt[i] = total;
        __syncwarp();
    }
}

// The product lists of C = A B on C's pattern (an earlier product of the
// same patterns; rows of B and C sorted).  G lanes per row of C walk the
// row's A entries k in ascending order, the lanes over B_k's columns; a B
// row holds each column once, so the lanes of one step never meet, and
// every entry's list comes out in ascending k, the order in which the tiered
// product above sums it.  Count pass (cur: zeroed, receives the list
// lengths) or fill pass (cur: each list's next free slot).  G divides 32 and
// the block, so a group's lanes share a warp and leave together.
template <int G, bool FILL>
__global__ void k_plan_pairs(int n, const int *ar, const int *ac, const int *br, const int *bc, const int *cr,
                             const int *cc, int *cur, int *pa, int *pb, int *err) {
    long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long i = tid / G;
    int lane = (int)(tid % G);
    if (i >= n) return;
    int wl = threadIdx.x & 31;
    unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (wl & ~(G - 1));
    int c0 = cr[i], c1 = cr[i + 1];
    for (int p = ar[i]; p < ar[i + 1]; p++) {
        int k = ac[p];
        for (int q = br[k] + lane; q < br[k + 1]; q += G) {
            int J = bc[q];
            int pos = find_col(cc, c0, c1, J);
            if (pos < c1 && cc[pos] == J) {
                int t = cur[pos]++;
                if (FILL) {
                    pa[t] = p;
                    pb[t] = q;
                }
            } else {
                set_err(err, CPR_ERR_INVALID);   // not the pattern this C was built for
            }
        }
        __syncwarp(gmask);
    }
}

// C's values from its product lists: each entry's products rounded and
// summed from zero in list order, exactly as the tiered product sums them.
__global__ void k_plan_values(int nnz, const int *ptr, const int *pa, const int *pb, const double *av,
                              const double *bv, double *cv) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nnz; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = ptr[c]; t < ptr[c + 1]; t++) s = __dadd_rn(s, __dmul_rn(av[pa[t]], bv[pb[t]]));
        cv[c] = s;
    }
}

// -------------------------------------------------------- level helpers

// A zero or non-finite diagonal records CPR_ERR_SINGULAR; dinv (when set)
// receives 1/a_ii, with 1 standing in for a bad pivot.
__global__ void k_check_diag(int n, const int *diag, const double *val, double *dinv, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = diag[i];
    double d = p >= 0 ? val[p] : 0.0;
    if (d == 0.0 || !isfinite(d)) {
        set_err(err, CPR_ERR_SINGULAR);
        d = 1.0;
    }
    if (dinv) dinv[i] = 1.0 / d;
}

// The values of R = P^T from P's (R's pattern kept: rows sorted by column,
// so P entry (i, j) sits at i's place in row j).
__global__ void k_transpose_values(int n, const int *pr, const int *pc, const double *pv, const int *rr,
                                   const int *rc, double *rv, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = pr[i]; p < pr[i + 1]; p++) {
        int j = pc[p];
        int e = rr[j + 1];
        int q = find_col(rc, rr[j], e, i);
        if (q < e && rc[q] == i) rv[q] = pv[p];
        else set_err(err, CPR_ERR_INVALID);
    }
}

// Per-color row counts: a block-local histogram in shared memory (colors
// below 1024), then one global atomic per block and color.
__global__ void k_color_hist(int n, int ncolors, const int *color, int *hist) {
    __shared__ int sh[1024];
    bool local = ncolors <= 1024;
    if (local)
        for (int c = threadIdx.x; c < ncolors; c += blockDim.x) sh[c] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (local) atomicAdd(&sh[color[i]], 1);
        else atomicAdd(&hist[color[i]], 1);
    }
    __syncthreads();
    if (local)
        for (int c = threadIdx.x; c < ncolors; c += blockDim.x)
            if (sh[c]) atomicAdd(&hist[c], sh[c]);
}

__global__ void k_flag_color(int n, const int *color, int c, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = color[i] == c;
}

__global__ void k_scatter_color(int n, const int *color, int c, const int *pos, int base,
                                int *rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && color[i] == c) rows[base + pos[i]] = i;
}

// Counting sort of rows by color (index order kept within a color), for up to
// kSortColors colors: tiles of kColorTile rows.  cnt is color-major,
// cnt[c * ntiles + tile], so one exclusive scan of it gives every (color,
// tile) its first output position directly.
constexpr int kColorTile = 1024;
constexpr int kSortColors = 64;

__global__ void __launch_bounds__(kColorTile) k_color_tile_counts(int n, int ncolors, int ntiles,
                                                                   const int *color, int *cnt) {
    __shared__ int sh[kSortColors];
    for (int c = threadIdx.x; c < ncolors; c += blockDim.x) sh[c] = 0;
    __syncthreads();
    int i = blockIdx.x * kColorTile + threadIdx.x;
    if (i < n) atomicAdd(&sh[color[i]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < ncolors; c += blockDim.x) cnt[(size_t)c * ntiles + blockIdx.x] = sh[c];
}

// rows[pos(color_i, tile) + rank of i among the tile's rows of that color] = i
__global__ void __launch_bounds__(kColorTile) k_color_tile_scatter(int n, int ncolors, int ntiles,
                                                                    const int *color, const int *pos, int *rows) {
    __shared__ int wc[kColorTile / 32][kSortColors];   // per-warp color counts
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kColorTile / 32) * kSortColors; k += blockDim.x) (&wc[0][0])[k] = 0;
    __syncthreads();
    int i = blockIdx.x * kColorTile + threadIdx.x;
    int c = i < n ? color[i] : -1;
    unsigned same = __match_any_sync(0xffffffffu, c);
    int in_warp = __popc(same & ((1u << lane) - 1u));
    if (c >= 0 && in_warp == 0) wc[w][c] = __popc(same);
    __syncthreads();
    if (c < 0) return;
    int before = 0;
    for (int v = 0; v < w; v++) before += wc[v][c];
    rows[pos[(size_t)c * ntiles + blockIdx.x] + before + in_warp] = i;
}

// The same counting sort for more than kSortColors colors (the level sets of
// the natural-order BILU(0)): tiles of kColorTileMany rows, the per-tile and
// per-warp counts in dynamic shared memory (ncolors and
// (kColorTileMany / 32) * ncolors ints).
constexpr int kColorTileMany = 256;
constexpr int kSortColorsMany = 1024;

__global__ void __launch_bounds__(kColorTileMany) k_color_tile_counts_many(int n, int ncolors, int ntiles,
                                                                           const int *color, int *cnt) {
    extern __shared__ int sh_many[];
    for (int c = threadIdx.x; c < ncolors; c += blockDim.x) sh_many[c] = 0;
    __syncthreads();
    int i = blockIdx.x * kColorTileMany + threadIdx.x;
    if (i < n && (unsigned)color[i] < (unsigned)ncolors) atomicAdd(&sh_many[color[i]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < ncolors; c += blockDim.x) cnt[(size_t)c * ntiles + blockIdx.x] = sh_many[c];
}

__global__ void __launch_bounds__(kColorTileMany) k_color_tile_scatter_many(int n, int ncolors, int ntiles,
                                                                            const int *color, const int *pos,
                                                                            int *rows) {
    extern __shared__ int wc_many[];   // [warp][color]
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kColorTileMany / 32) * ncolors; k += blockDim.x) wc_many[k] = 0;
    __syncthreads();
    int i = blockIdx.x * kColorTileMany + threadIdx.x;
    int c = i < n && (unsigned)color[i] < (unsigned)ncolors ? color[i] : -1;
    unsigned same = __match_any_sync(0xffffffffu, c);
    int in_warp = __popc(same & ((1u << lane) - 1u));
    if (c >= 0 && in_warp == 0) wc_many[w * ncolors + c] = __popc(same);
    __syncthreads();
    if (c < 0) return;
    int before = 0;
    for (int v = 0; v < w; v++) before += wc_many[v * ncolors + c];
    rows[pos[(size_t)c * ntiles + blockIdx.x] + before + in_warp] = i;
}

__global__ void k_iperm(int n, const int *order, int *iperm) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) iperm[order[t]] = t;
}

// Row lengths of the renumbered copy: row t is natural row order[t] (order ==
// nullptr: identity), without its diagonal entry when skip_diag.
__global__ void k_perm_count(int n, const int *order, const int *rowptr, const int *col,
                             bool skip_diag, int *cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int i = order ? order[t] : t;
    int c = rowptr[i + 1] - rowptr[i];
    if (skip_diag)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) c -= col[p] == i;
    cnt[t] = c;
}

// Fill the renumbered copy, G lanes per row; columns mapped through icol
// (nullptr: unchanged); entries keep the natural (ascending-column) order of
// their row.  With skip_diag the diagonal is dropped: the diagonals before a
// lane's entry are counted from a ballot of the lane's group.  nval32, when
// set, receives the values rounded to FP32 as well.
template <int G>
__global__ void k_perm_fill(int n, const int *order, const int *rowptr, const int *col,
                            const double *val, bool skip_diag, const int *icol, const int *nrow,
                            int *ncol, double *nval, float *nval32) {
    long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    if (t >= n) return;   // whole groups: G divides the block
    int wl = threadIdx.x & 31;
    unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (wl & ~(G - 1));
    unsigned below = gmask & ((1u << wl) - 1u);
    int i = order ? order[t] : (int)t;
    int a = rowptr[i], b = rowptr[i + 1];
    int q = nrow[t] - a;   // source entry p lands at q + p, less the diagonals before it
    int skipped = 0;
    for (int p0 = a; p0 < b; p0 += G) {
        int p = p0 + lane;
        bool in = p < b;
        int j = in ? col[p] : 0;
        bool d = skip_diag && in && j == i;
        unsigned m = __ballot_sync(gmask, d);
        if (in && !d) {
            int o = q + p - skipped - __popc(m & below);
            ncol[o] = icol ? icol[j] : j;
            double v = val[p];
            nval[o] = v;
            if (nval32) nval32[o] = (float)v;
        }
        skipped += __popc(m);
    }
}

// The diagonal and its reciprocal in color order (dpos: each natural row's
// diagonal position, -1 for none, which reads as 0).
__global__ void k_perm_diag(int n, const int *order, const int *dpos, const double *val, double *diag,
                            double *dinv, float *diag32, float *dinv32) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int p = dpos[order[t]];
    double d = p >= 0 ? val[p] : 0.0;
    double r = 1.0 / d;
    diag[t] = d;
    dinv[t] = r;
    if (diag32) {   // the FP32 shadows, rounded from the FP64 values
        diag32[t] = (float)d;
        dinv32[t] = (float)r;
    }
}

__global__ void k_csr_to_dense(int n, const int *rowptr, const int *col, const double *val,
                               double *a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) a[(size_t)i * n + col[p]] = val[p];
}

// |x| as an integer key that orders as the magnitudes do (IEEE doubles of one
// sign order as their bit patterns), so the pivot search needs no FP64
// instruction; a NaN is the smallest key, so it never wins, as it never
// compares larger.
__device__ __forceinline__ long long abs_key(double x) {
    long long k = __double_as_longlong(x) & 0x7fffffffffffffffLL;
    return k > 0x7ff0000000000000LL ? -1 : k;
}

// The larger of two (key, position) candidates, the lower position on ties.
__device__ __forceinline__ void pivot_max(long long &best, int &bi, long long ov, int oi) {
    if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
    }
}

// Dense LU with partial pivoting of the coarsest matrix (largest |a|, lowest
// position on ties), one CTA of 32 warps.  Rows are never moved: perm[k] is
// the storage row at position k, kept in shared memory.  Step k finds the
// pivot (integer keys: the warps holding candidates, then warp 0), scales
// column k below it into the multipliers, then updates the trailing rows, a
// warp per row and the lanes over its columns.  The factors leave in
// position order in `lu` (row-major, row k = position k) when the matrix is
// staged in shared memory; otherwise `lu` holds the copy factored in storage
// order.  Dynamic shared memory: n*n doubles when use_smem, then n ints.
constexpr int kLuThreads = 1024;
__global__ void __launch_bounds__(kLuThreads) k_dense_lu(int n, const double *a_g, double *lu, int *perm_g,
                                                         int use_smem, int *err) {
    extern __shared__ double sm[];
    __shared__ long long wv[kLuThreads / 32];
    __shared__ int wi[kLuThreads / 32];
    __shared__ int prow;
    __shared__ double pinv;
    double *a = use_smem ? sm : lu;
    int *perm = reinterpret_cast<int *>(sm + (use_smem ? (size_t)n * n : 0));
    int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    if (use_smem)
        for (long e = tid; e < (long)n * n; e += nt) a[e] = a_g[e];
    for (int i = tid; i < n; i += nt) perm[i] = i;
    __syncthreads();
    for (int k = 0; k < n; k++) {
        int cw = min(nw, (n - k + 31) / 32);   // warps holding candidates
        if (wid < cw) {
            long long best = -1;
            int bi = INT_MAX;
            for (int i = k + tid; i < n; i += nt) pivot_max(best, bi, abs_key(a[(size_t)perm[i] * n + k]), i);
            for (int sh = 16; sh > 0; sh >>= 1)
                pivot_max(best, bi, __shfl_xor_sync(0xffffffffu, best, sh), __shfl_xor_sync(0xffffffffu, bi, sh));
            if (lane == 0) {
                wv[wid] = best;
                wi[wid] = bi;
            }
        }
        __syncthreads();
        if (wid == 0) {
            long long best = lane < cw ? wv[lane] : -1;
            int bi = lane < cw ? wi[lane] : INT_MAX;
            for (int sh = 16; sh > 0; sh >>= 1)
                pivot_max(best, bi, __shfl_xor_sync(0xffffffffu, best, sh), __shfl_xor_sync(0xffffffffu, bi, sh));
            if (lane == 0) {
                if (best <= 0) {   // zero or NaN column
                    set_err(err, CPR_ERR_SINGULAR);
                    bi = k;
                }
                int t = perm[k];
                perm[k] = perm[bi];
                perm[bi] = t;
                prow = perm[k];
                double pv = a[(size_t)prow * n + k];
                pinv = pv == 0.0 ? 1.0 : 1.0 / pv;
            }
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < n; i += nt) {
            double *ri = a + (size_t)perm[i] * n;
            ri[k] = ri[k] * pinv;
        }
        __syncthreads();
        const double *pr = a + (size_t)prow * n;
        for (int i = k + 1 + wid; i < n; i += nw) {
            double *ri = a + (size_t)perm[i] * n;
            double l = ri[k];
            for (int j = k + 1 + lane; j < n; j += 32) ri[j] -= l * pr[j];
        }
        __syncthreads();
    }
    // factors in position order (in place is safe only through the staging copy)
    if (use_smem) {
        for (long e = tid; e < (long)n * n; e += nt) {
            int k = (int)(e / n), q = (int)(e % n);
            lu[e] = a[(size_t)perm[k] * n + q];
        }
    }
    for (int i = tid; i < n; i += nt) perm_g[i] = perm[i];
}

// out[k*n + q] = in[perm[k]*n + q] (rows gathered into position order).
__global__ void k_gather_rows(int n, const double *in, const int *perm, double *out) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    int k = (int)(e / n), q = (int)(e % n);
    out[e] = in[(size_t)perm[k] * n + q];
}

// Column j of A^-1 from the LU factors, one CTA per column: the factors are
// staged in shared memory when `staged` (n*n doubles), then one warp runs the
// substitutions column by column -- y = L^-1 P e_j (unit L; y_k = 1 where
// perm[k] = j), x = U^-1 y -- each step taking the finished entry and
// updating the ones after (before) it across the lanes.  The reciprocals of
// U's diagonal are formed first, off that chain.  Written row-major
// (inv[i*n + j]).  Dynamic shared memory: 2n doubles, then the factors.
constexpr int kInvThreads = 128;
__global__ void __launch_bounds__(kInvThreads) k_dense_inv_cols(int n, const double *lu, const int *perm,
                                                                double *inv, int staged) {
    extern __shared__ double sm[];
    double *x = sm, *rd = sm + n;
    const double *f = lu;
    int tid = threadIdx.x, nt = blockDim.x, j = blockIdx.x;
    if (staged) {
        double *fs = sm + 2 * (size_t)n;
        for (long e = tid; e < (long)n * n; e += nt) fs[e] = lu[e];
        f = fs;
    }
    for (int i = tid; i < n; i += nt) {
        x[i] = perm[i] == j ? 1.0 : 0.0;
        rd[i] = 1.0 / lu[(size_t)i * n + i];
    }
    __syncthreads();
    if (tid >= 32) return;
    int lane = tid;
    for (int k = 0; k < n; k++) {
        double xk = x[k];
        for (int i = k + 1 + lane; i < n; i += 32) x[i] -= f[(size_t)i * n + k] * xk;
        __syncwarp();
    }
    for (int k = n - 1; k >= 0; k--) {
        double xk = x[k] * rd[k];
        for (int i = lane; i < k; i += 32) x[i] -= f[(size_t)i * n + k] * xk;
        __syncwarp();
        if (lane == 0) x[k] = xk;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) inv[(size_t)i * n + j] = x[i];
}

// ------------------------------------------------------------------ BILU(0)

__device__ __forceinline__ void mat3_mul_rn(const double *a, const double *b, double *c) {
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double t = 0.0;
            for (int k = 0; k < 3; k++) t = __dadd_rn(t, __dmul_rn(a[3 * r + k], b[3 * k + s]));
            c[3 * r + s] = t;
        }
}

__device__ __forceinline__ bool mat3_inv_rn(const double *a, double *inv) {
    double c00 = __dsub_rn(__dmul_rn(a[4], a[8]), __dmul_rn(a[5], a[7]));
    double c01 = __dsub_rn(__dmul_rn(a[5], a[6]), __dmul_rn(a[3], a[8]));
    double c02 = __dsub_rn(__dmul_rn(a[3], a[7]), __dmul_rn(a[4], a[6]));
    double det = __dadd_rn(__dadd_rn(__dmul_rn(a[0], c00), __dmul_rn(a[1], c01)), __dmul_rn(a[2], c02));
    if (det == 0.0 || !isfinite(det)) return false;
    inv[0] = __ddiv_rn(c00, det);
    inv[1] = __ddiv_rn(__dsub_rn(__dmul_rn(a[2], a[7]), __dmul_rn(a[1], a[8])), det);
    inv[2] = __ddiv_rn(__dsub_rn(__dmul_rn(a[1], a[5]), __dmul_rn(a[2], a[4])), det);
    inv[3] = __ddiv_rn(c01, det);
    inv[4] = __ddiv_rn(__dsub_rn(__dmul_rn(a[0], a[8]), __dmul_rn(a[2], a[6])), det);
    inv[5] = __ddiv_rn(__dsub_rn(__dmul_rn(a[2], a[3]), __dmul_rn(a[0], a[5])), det);
    inv[6] = __ddiv_rn(c02, det);
    inv[7] = __ddiv_rn(__dsub_rn(__dmul_rn(a[1], a[6]), __dmul_rn(a[0], a[7])), det);
    inv[8] = __ddiv_rn(__dsub_rn(__dmul_rn(a[0], a[4]), __dmul_rn(a[1], a[3])), det);
    return true;
}

template <class T>
__device__ __forceinline__ void mat3_mul_t(const T *a, const T *b, T *c);
template <>
__device__ __forceinline__ void mat3_mul_t<double>(const double *a, const double *b, double *c) {
    mat3_mul_rn(a, b, c);
}
template <>
__device__ __forceinline__ void mat3_mul_t<float>(const float *a, const float *b, float *c) {
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) c[3 * r + s] = fmaf(a[3 * r + 2], b[6 + s], fmaf(a[3 * r + 1], b[3 + s], a[3 * r] * b[s]));
}
__device__ __forceinline__ double sub_t(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_t(float a, float b) { return a - b; }
__device__ __forceinline__ bool mat3_inv_t(const double *a, double *inv) { return mat3_inv_rn(a, inv); }
__device__ __forceinline__ bool mat3_inv_t(const float *a, float *inv) {
    float c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    float det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == 0.0f || !isfinite(det)) return false;
    float r = 1.0f / det;
    inv[0] = c00 * r;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) * r;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) * r;
    inv[3] = c01 * r;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) * r;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) * r;
    inv[6] = c02 * r;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) * r;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) * r;
    return true;
}

// Factor the block rows of one color; rows of lower colors are final.  For
// row i, the entries k before i in (color, index) order are eliminated in that
// order: L_ik = A_ik U_kk^-1, then A_ij -= L_ik U_kj for j after k in row k
// that lies in row i's pattern.  Same-color rows are never adjacent (the
// block coloring is at theta = 0), so "after k" means "higher color than k".
// With natural set, the colors are the natural-order level sets and the k
// before i are taken in index order alone: the operations, and their order,
// of sequential block ILU(0) in index order.  FP64: every operation rounded as the plain definition orders it; FP32 (the
// FP32-preconditioner mode, whose B only ever uses FP32 factors): FMA allowed.
//
// G lanes per row: the lanes search the row for the next k together (a
// group minimum), one lane forms L_ik, and the lanes share the updates of
// row k's entries, each of which lands on its own block of row i.  Every
// block operation is the one-thread form's, in the same order.  G divides
// 32 and the block, so a group's lanes share a warp and leave together.
template <class T, int G>
__global__ void k_bilu_factor_color(const int *rows, int cnt, const int *rowptr, const int *col,
                                    const int *color, const int *diag, T *lu, int *err, int natural) {
    long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    if (t >= cnt) return;
    int wl = threadIdx.x & 31;
    unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (wl & ~(G - 1));
    int i = rows[t];
    int a = rowptr[i], b = rowptr[i + 1];
    int ci = color[i];
    int last_c = -1, last_k = -1;
    for (;;) {
        int best = -1, bc = INT_MAX, bk = INT_MAX;
        for (int p = a + lane; p < b; p += G) {
            int k = col[p];
            int ck = color[k];
            if (ck >= ci) continue;
            if (natural) ck = 0;   // lower neighbours eliminated by index alone
            bool after_last = ck > last_c || (ck == last_c && k > last_k);
            bool before_best = ck < bc || (ck == bc && k < bk);
            if (after_last && before_best) {
                best = p;
                bc = ck;
                bk = k;
            }
        }
        for (int o = G / 2; o > 0; o >>= 1) {
            int obest = __shfl_xor_sync(gmask, best, o), obc = __shfl_xor_sync(gmask, bc, o),
                obk = __shfl_xor_sync(gmask, bk, o);
            if (obc < bc || (obc == bc && obk < bk)) {
                best = obest;
                bc = obc;
                bk = obk;
            }
        }
        if (best < 0) break;
        int k = bk;
        T *Lb = lu + 9 * (size_t)best;
        if (lane == 0) {
            T L[9];
            mat3_mul_t<T>(Lb, lu + 9 * (size_t)diag[k], L);
            for (int e = 0; e < 9; e++) Lb[e] = L[e];
        }
        __syncwarp(gmask);
        T L[9];
        for (int e = 0; e < 9; e++) L[e] = Lb[e];
        int ck = color[k];
        for (int q = rowptr[k] + lane; q < rowptr[k + 1]; q += G) {
            int j = col[q];
            if (j == k || color[j] <= ck) continue;
            int r = find_col(col, a, b, j);
            if (r >= b || col[r] != j) continue;
            T P[9];
            mat3_mul_t<T>(L, lu + 9 * (size_t)q, P);
            for (int e = 0; e < 9; e++) lu[9 * (size_t)r + e] = sub_t(lu[9 * (size_t)r + e], P[e]);
        }
        __syncwarp(gmask);
        last_c = bc;
        last_k = bk;
    }
    if (lane != 0) return;
    T inv[9];
    T *D = lu + 9 * (size_t)diag[i];
    if (!mat3_inv_t(D, inv)) {
        set_err(err, CPR_ERR_SINGULAR);
        return;
    }
    for (int e = 0; e < 9; e++) D[e] = inv[e];
}

// Row lengths of L (lower colors) and U (higher colors) per position t.
__global__ void k_bilu_split_count(int nb, const int *order, const int *rowptr, const int *col,
                                   const int *color, int *lcnt, int *ucnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    int i = order[t];
    int l = 0, u = 0, ci = color[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int j = col[p];
        if (j == i) continue;
        if (color[j] < ci) l++;
        else u++;
    }
    lcnt[t] = l;
    ucnt[t] = u;
}

// G lanes per natural block row i: each entry of the factor array goes to L
// (lower color), U (higher color) or D^-1 (the diagonal) at the row's
// position, its index within L or U counted by group ballots, its column
// renumbered to its position.  G divides 32 and the block.
template <class T, int G>
__global__ void k_bilu_split_fill(int nb, const int *rowptr, const int *col, const int *color, const int *iperm,
                                  const T *lu, const int *lr, int *lc, T *lv, const int *ur, int *uc, T *uv,
                                  T *dinv) {
    long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long i = tid / G;
    int lane = (int)(tid % G);
    if (i >= nb) return;
    int wl = threadIdx.x & 31;
    unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (wl & ~(G - 1));
    unsigned below = gmask & ((1u << wl) - 1u);
    int ci = color[i], t = iperm[(int)i];
    int nl = lr[t], nu = ur[t];   // next free slots of the row's L and U parts
    for (int p0 = rowptr[i]; p0 < rowptr[i + 1]; p0 += G) {
        int p = p0 + lane;
        bool in = p < rowptr[i + 1];
        int j = in ? col[p] : 0;
        bool d = in && j == i;
        bool lower = in && !d && color[j] < ci;
        bool upper = in && !d && !lower;
        unsigned ml = __ballot_sync(gmask, lower), mu = __ballot_sync(gmask, upper);
        T *dst = nullptr;
        if (d) {
            dst = dinv + 9 * (size_t)t;
        } else if (lower) {
            int k = nl + __popc(ml & below);
            lc[k] = iperm[j];
            dst = lv + 9 * (size_t)k;
        } else if (upper) {
            int k = nu + __popc(mu & below);
            uc[k] = iperm[j];
            dst = uv + 9 * (size_t)k;
        }
        if (dst) {
            const T *src = lu + 9 * (size_t)p;
            for (int e = 0; e < 9; e++) dst[e] = src[e];
        }
        nl += __popc(ml);
        nu += __popc(mu);
    }
}

__global__ void k_d2f(long n, const double *a, float *b) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ------------------------------------------------------------ host helpers

struct Graph {
    int n = 0, nnz = 0;
    DVec<int> rowptr, col;
};

void check_err(cpr_handle *h, const char *what) {
    int e = read_int(h->err.p, h->stream);
    if (e != 0) {
        CK(cudaMemsetAsync(h->err.p, 0, sizeof(int), h->stream));
        fail(e, what);
    }
}

// A pattern CSR from a count pass and a fill pass over rows.
template <class CountFill>
Graph build_pattern(int n, cudaStream_t s, CountFill cf) {
    Graph g;
    g.n = n;
    DVec<int> cnt;
    cnt.alloc(n, s);
    cf(nullptr, cnt.p);
    g.rowptr.alloc(n + 1, s);
    exclusive_scan(cnt.p, g.rowptr.p, n, s);
    g.nnz = read_int(g.rowptr.p + n, s);
    g.col.alloc(std::max(g.nnz, 1), s);
    cf(g.rowptr.p, g.col.p);
    return g;
}

// The same with at most ub entries allocated and no read-back of the count
// (nnz = -1: known on the device only).
template <class CountFill>
Graph build_pattern_ub(int n, long ub, cudaStream_t s, CountFill cf) {
    Graph g;
    g.n = n;
    g.nnz = -1;
    DVec<int> cnt;
    cnt.alloc(std::max(n, 1), s);
    cf(nullptr, cnt.p);
    g.rowptr.alloc(n + 1, s);
    exclusive_scan(cnt.p, g.rowptr.p, n, s);
    g.col.alloc(std::max<long>(ub, 1), s);
    cf(g.rowptr.p, g.col.p);
    return g;
}

// Transpose (pattern, or with values when val != nullptr); rows of the
// result sorted, or (sorted false) in the order the scatter left them.
void transpose(int n, int ncol, int nnz, const int *rowptr, const int *col, const double *val,
               DVec<int> &trow, DVec<int> &tcol, DVec<double> *tval, cudaStream_t s, bool sorted = true) {
    DVec<int> cnt, cursor;
    cnt.alloc(std::max(ncol, 1), s);
    cnt.zero();
    if (nnz) {
        k_count_cols<<<grid_for(nnz, kBlock, 148 * 32), kBlock, 0, s>>>(nnz, col, cnt.p);
        CK_LAUNCH();
    }
    trow.alloc(ncol + 1, s);
    exclusive_scan(cnt.p, trow.p, ncol, s);
    cursor.alloc(std::max(ncol, 1), s);
    if (ncol) CK(cudaMemcpyAsync(cursor.p, trow.p, sizeof(int) * ncol, cudaMemcpyDeviceToDevice, s));
    tcol.alloc(std::max(nnz, 1), s);
    if (tval) tval->alloc(std::max(nnz, 1), s);
    k_scatter_t<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, rowptr, col, val, cursor.p, tcol.p,
                                                      tval ? tval->p : nullptr);
    CK_LAUNCH();
    if (ncol && sorted) {
        DVec<int> longrows, nlong;
        longrows.alloc(ncol, s);
        nlong.alloc(1, s);
        CK(cudaMemsetAsync(nlong.p, 0, sizeof(int), s));
        k_sort_rows<<<grid_for(ncol, kBlock), kBlock, 0, s>>>(ncol, trow.p, tcol.p, tval ? tval->p : nullptr,
                                                              longrows.p, nlong.p);
        CK_LAUNCH();
        k_sort_long_rows<<<grid_for(ncol, kSortWarps, 148 * 4), kSortWarps * 32, 0, s>>>(
            longrows.p, nlong.p, trow.p, tcol.p, tval ? tval->p : nullptr);
        CK_LAUNCH();
    }
}

// G = S u S^T for JP: S itself, its one-way transpose part T (rows unsorted)
// and the union degrees.  S may carry only a bound of its entry count (ub):
// nothing here reads the count back.
struct SymGraph {
    int n = 0;
    long ub = 0;   // bound of S's entry count (an average degree estimate for the lanes per vertex)
    Graph S;
    DVec<int> trow, tcol, deg;
    JpGraph dev() const { return JpGraph{S.rowptr.p, S.col.p, trow.p, tcol.p, deg.p}; }
};

SymGraph sym_graph(Graph &&S, long ub, cudaStream_t s) {
    SymGraph g;
    int n = g.n = S.n;
    g.ub = ub;
    g.S = std::move(S);
    DVec<int> cnt, cursor;
    cnt.alloc(std::max(n, 1), s);
    cnt.zero();
    k_oneway_t<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, g.S.rowptr.p, g.S.col.p, cnt.p, nullptr);
    CK_LAUNCH();
    g.trow.alloc(n + 1, s);
    exclusive_scan(cnt.p, g.trow.p, n, s);
    cursor.alloc(std::max(n, 1), s);
    if (n) CK(cudaMemcpyAsync(cursor.p, g.trow.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    g.tcol.alloc(std::max<long>(ub, 1), s);
    k_oneway_t<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, g.S.rowptr.p, g.S.col.p, cursor.p, g.tcol.p);
    CK_LAUNCH();
    g.deg.alloc(std::max(n, 1), s);
    k_sym_degree<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, g.S.rowptr.p, g.trow.p, g.deg.p);
    CK_LAUNCH();
    return g;
}

// Jones-Plassmann coloring of graph G; returns the number of colors.
int jp_color(cpr_handle *h, const SymGraph &G, int salt, int level, DVec<int> &color, cudaStream_t s) {
    int n = G.n;
    DVec<unsigned long long> state;
    state.alloc(n, s);
    CK(cudaMemsetAsync(state.p, 0xff, sizeof(unsigned long long) * n, s));
    DVec<int> counters;  // list counts (three slots), max color
    counters.alloc(4, s);
    CK(cudaMemsetAsync(counters.p, 0, 4 * sizeof(int), s));
    uint32_t hb = hash_base(h->opt.seed, salt, level);
    // lanes per vertex: about kJpPre of a typical row's entries per lane, as
    // long as every vertex of the round still has its lanes resident at once
    int lanes = 1;
    while (lanes < 16 && (long)lanes * kJpPre * n < G.ub && 2L * lanes * n <= kResidentThreads) lanes <<= 1;
    if (n <= kSmallLevel) {
        // one CTA: lanes only while every vertex still fits one pass of its 1024 threads
        lanes = 1;
        while (lanes < 8 && (long)2 * lanes * n <= 1024) lanes <<= 1;
        auto small = [&](auto kern) {
            kern<<<1, 1024, 0, s>>>(n, G.dev(), hb, state.p, counters.p + 3);
            CK_LAUNCH();
        };
        switch (lanes) {
        case 1: small(k_jp_small<1>); break;
        case 2: small(k_jp_small<2>); break;
        case 4: small(k_jp_small<4>); break;
        case 8: small(k_jp_small<8>); break;
        default: small(k_jp_small<16>); break;
        }
        color.alloc(n, s);
        k_state_to_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, state.p, color.p);
        CK_LAUNCH();
        return read_int(counters.p + 3, s) + 1;
    }
    DVec<int> lists;   // two worklists, used alternately
    lists.alloc(2 * (size_t)n, s);
    int grid = grid_for((long)n * lanes, kBlock, 148 * 8);
    unsigned r = 0;
    auto round = [&](auto kern, const int *in, int *out) {
        kern<<<grid, kBlock, 0, s>>>(n, in, out, counters.p, G.dev(), hb, state.p, r, counters.p + 3);
        CK_LAUNCH();
    };
    for (;;) {
        for (int k = 0; k < kJpBatch; k++, r++) {
            const int *in = r == 0 ? nullptr : lists.p + (size_t)(r % 2) * n;
            int *out = lists.p + (size_t)((r + 1) % 2) * n;
            switch (lanes) {
            case 1: round(k_jp_round<1>, in, out); break;
            case 2: round(k_jp_round<2>, in, out); break;
            case 4: round(k_jp_round<4>, in, out); break;
            case 8: round(k_jp_round<8>, in, out); break;
            default: round(k_jp_round<16>, in, out); break;
            }
        }
        if (read_int(counters.p + r % 3, s) == 0) break;
        if (r > (unsigned)n + 8) fail(CPR_ERR_CUDA, "coloring did not terminate");
    }
    if (getenv("CPR_SETUP_TIMING")) fprintf(stderr, "[cpr setup] jp n=%d rounds<=%u\n", n, r);
    color.alloc(n, s);
    k_state_to_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, state.p, color.p);
    CK_LAUNCH();
    return read_int(counters.p + 3, s) + 1;
}

// Alg. 4-5 on S (the raw Eq. 5.1 strength pattern, n <= kMaxGroupingRows);
// returns the number of groups (colors).
int vertices_grouping(cpr_handle *h, const Graph &S, DVec<int> &color, cudaStream_t s) {
    int n = S.n;
    int m = 1;
    while (m < n) m <<= 1;
    size_t sort_smem = sizeof(unsigned) * (size_t)m;
    int nw = (n + 31) / 32;
    size_t group_smem = (size_t)((3 * n + 15) & ~15) + 2 * sizeof(unsigned) * (size_t)nw;
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        CK(cudaFuncSetAttribute(k_group_order, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(unsigned) * kMaxGroupingRows)));
        CK(cudaFuncSetAttribute(k_vertices_grouping, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                3 * kMaxGroupingRows + 16 + 2 * (kMaxGroupingRows / 32) * (int)sizeof(unsigned)));
        attr_set.fetch_or(bit);
    }
    DVec<int> order, rank, out;   // out: [0] number of groups, [1] error flag
    order.alloc(std::max(n, 1), s);
    rank.alloc(std::max(n, 1), s);
    out.alloc(2, s);
    out.zero();
    color.alloc(std::max(n, 1), s);
    k_group_order<<<1, kGroupSortThreads, sort_smem, s>>>(n, S.rowptr.p, order.p, rank.p);
    CK_LAUNCH();
    k_vertices_grouping<<<1, 32, group_smem, s>>>(n, S.rowptr.p, S.col.p, order.p, rank.p, color.p, out.p,
                                                  out.p + 1);
    CK_LAUNCH();
    int res[2] = {0, 0};
    CK(cudaMemcpyAsync(res, out.p, sizeof(res), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (res[1]) fail(CPR_ERR_CUDA, "Alg. 4-5 grouping did not complete");
    return res[0];
}

// Level sets of natural-order block ILU(0) over G (k_level_round), with
// batches of rounds between host checks; returns the number of levels.
int level_sets(const SymGraph &G, DVec<int> &level, cudaStream_t s) {
    constexpr int kLevelBatch = 16;
    int n = G.n;
    level.alloc(n, s);
    CK(cudaMemsetAsync(level.p, 0xff, sizeof(int) * n, s));
    DVec<int> counters, lists;
    counters.alloc(4, s);
    CK(cudaMemsetAsync(counters.p, 0, 4 * sizeof(int), s));
    lists.alloc(2 * (size_t)n, s);
    int grid = grid_for(n, kBlock, 148 * 8);
    unsigned r = 0;
    for (;;) {
        for (int k = 0; k < kLevelBatch; k++, r++) {
            const int *in = r == 0 ? nullptr : lists.p + (size_t)(r % 2) * n;
            int *out = lists.p + (size_t)((r + 1) % 2) * n;
            k_level_round<<<grid, kBlock, 0, s>>>(n, in, out, counters.p, G.dev(), level.p, r, counters.p + 3);
            CK_LAUNCH();
        }
        if (read_int(counters.p + r % 3, s) == 0) break;
        // every round settles at least the lowest unsettled row
        if (r > (unsigned)n + kLevelBatch) fail(CPR_ERR_CUDA, "level sets did not terminate");
    }
    if (getenv("CPR_SETUP_TIMING")) fprintf(stderr, "[cpr setup] levels n=%d rounds<=%u\n", n, r);
    return read_int(counters.p + 3, s) + 1;
}

// The smoother's coloring of a level of at most kSmallLevel rows in one
// launch (k_color_small) and one read-back: the colors, the color offsets and
// the rows grouped by color, as the strength / graph / JP / ordering launches
// of the larger levels give them.
int color_small(cpr_handle *h, const DCsr &A, int level, DVec<int> &color, std::vector<int> &off, DVec<int> &rows,
                cudaStream_t s) {
    int n = A.n;
    size_t ub = std::max<size_t>((size_t)A.nnz, 1);   // S holds at most A's entries
    DVec<double> thr;
    DVec<int> srow, scol, trow, tcol, deg, info;
    DVec<unsigned long long> state;
    thr.alloc(n, s);
    srow.alloc(n + 1, s);
    scol.alloc(ub, s);
    trow.alloc(n + 1, s);
    tcol.alloc(ub, s);
    deg.alloc(n, s);
    state.alloc(n, s);
    info.alloc(n + 2, s);
    color.alloc(n, s);
    rows.alloc(n, s);
    uint32_t hb = hash_base(h->opt.seed, 0, level);
    // lanes per vertex as in the one-CTA JP rounds
    int lanes = 1;
    while (lanes < 8 && 2L * lanes * n <= kSmallLevel / 4) lanes <<= 1;
    auto go = [&](auto kern) {
        kern<<<1, kSmallLevel / 4, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, h->opt.theta_color, hb, thr.p, srow.p,
                                           scol.p, trow.p, tcol.p, deg.p, state.p, color.p, rows.p, info.p);
        CK_LAUNCH();
    };
    switch (lanes) {
    case 1: go(k_color_small<1>); break;
    case 2: go(k_color_small<2>); break;
    case 4: go(k_color_small<4>); break;
    default: go(k_color_small<8>); break;
    }
    int head[64];
    int m = std::min(n + 2, 64);
    CK(cudaMemcpyAsync(head, info.p, sizeof(int) * m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int nc = head[0];
    off.assign(nc + 1, 0);
    if (nc + 2 <= m) {
        for (int c = 0; c <= nc; c++) off[c] = head[1 + c];
    } else {   // more colors than the first read-back held
        CK(cudaMemcpyAsync(off.data(), info.p + 1, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return nc;
}

// Rows grouped by color, index-ascending within a color.
void rows_by_color(int n, const int *color, int ncolors, std::vector<int> &off, DVec<int> &rows,
                   cudaStream_t s) {
    DVec<int> hist, flag, pos;
    hist.alloc(ncolors, s);
    hist.zero();
    k_color_hist<<<grid_for(n, kBlock, 148 * 4), kBlock, 0, s>>>(n, ncolors, color, hist.p);
    CK_LAUNCH();
    std::vector<int> hh(ncolors);
    CK(cudaMemcpyAsync(hh.data(), hist.p, sizeof(int) * ncolors, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    off.assign(ncolors + 1, 0);
    for (int c = 0; c < ncolors; c++) off[c + 1] = off[c] + hh[c];
    rows.alloc(n, s);
    if (ncolors <= kSortColors) {
        int ntiles = (n + kColorTile - 1) / kColorTile;
        DVec<int> cnt;
        cnt.alloc((size_t)ncolors * ntiles, s);
        pos.alloc((size_t)ncolors * ntiles + 1, s);
        k_color_tile_counts<<<ntiles, kColorTile, 0, s>>>(n, ncolors, ntiles, color, cnt.p);
        CK_LAUNCH();
        exclusive_scan(cnt.p, pos.p, ncolors * ntiles, s);
        k_color_tile_scatter<<<ntiles, kColorTile, 0, s>>>(n, ncolors, ntiles, color, pos.p, rows.p);
        CK_LAUNCH();
        return;
    }
    if (ncolors <= kSortColorsMany) {
        int ntiles = (n + kColorTileMany - 1) / kColorTileMany;
        DVec<int> cnt;
        cnt.alloc((size_t)ncolors * ntiles, s);
        pos.alloc((size_t)ncolors * ntiles + 1, s);
        k_color_tile_counts_many<<<ntiles, kColorTileMany, sizeof(int) * ncolors, s>>>(n, ncolors, ntiles, color,
                                                                                      cnt.p);
        CK_LAUNCH();
        exclusive_scan(cnt.p, pos.p, ncolors * ntiles, s);
        k_color_tile_scatter_many<<<ntiles, kColorTileMany, sizeof(int) * (kColorTileMany / 32) * ncolors, s>>>(
            n, ncolors, ntiles, color, pos.p, rows.p);
        CK_LAUNCH();
        return;
    }
    flag.alloc(n, s);
    pos.alloc(n + 1, s);
    for (int c = 0; c < ncolors; c++) {
        k_flag_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, color, c, flag.p);
        CK_LAUNCH();
        exclusive_scan(flag.p, pos.p, n, s);
        k_scatter_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, color, c, pos.p, off[c], rows.p);
        CK_LAUNCH();
    }
}

// C = A B (structural pattern, sorted; values in Gustavson order; the rows of
// B sorted).  Each row belongs to exactly one tier (spgemm_tier) and is
// written by exactly one launch: the three per-thread tiers over all rows,
// the table tiers over their lists.
size_t dense_smem(int ncol, bool fill) {
    size_t per_warp = (fill ? (size_t)ncol * sizeof(double) : 0) + (size_t)((ncol + 31) / 32) * sizeof(unsigned);
    return kDenseWarps * ((per_warp + 15) & ~(size_t)15);
}

// C = A B with the dense-accumulator kernel (B.ncol <= kDenseCols): a count
// pass, a scan, one read-back of the size, a fill pass.
void spgemm_dense(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
    int n = A.n, ncol = B.ncol;
    static std::once_flag attr;   // the same ceiling for every handle and thread
    std::call_once(attr, [] {
        CK(cudaFuncSetAttribute(k_spgemm_dense<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dense_smem(kDenseCols, true)));
    });
    DVec<int> ucnt;
    ucnt.alloc(std::max(n, 1), s);
    unsigned blocks = (unsigned)grid_for(std::max(n, 1), kDenseWarps, 148 * 8);
    k_spgemm_dense<false><<<blocks, kDenseWarps * 32, dense_smem(ncol, false), s>>>(
        n, ncol, A.rowptr.p, A.col.p, nullptr, B.rowptr.p, B.col.p, nullptr, nullptr, nullptr, nullptr, ucnt.p);
    CK_LAUNCH();
    C.n = n;
    C.ncol = ncol;
    C.rowptr.alloc(n + 1, s);
    exclusive_scan(ucnt.p, C.rowptr.p, n, s);
    C.nnz = read_int(C.rowptr.p + n, s);
    if (C.nnz < 0) fail(CPR_ERR_OOM, "Galerkin product too large");
    C.col.alloc(std::max(C.nnz, 1), s);
    C.val.alloc(std::max(C.nnz, 1), s);
    k_spgemm_dense<true><<<blocks, kDenseWarps * 32, dense_smem(ncol, true), s>>>(
        n, ncol, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p, C.rowptr.p, C.col.p, C.val.p, nullptr);
    CK_LAUNCH();
}

void spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
    constexpr int kSW = 16, kMW = 8, kBW = 4;   // warps per block: small, medium and large tables
    int n = A.n;
    if (B.ncol <= kDenseCols) {   // few columns: a dense accumulator per row
        spgemm_dense(A, B, C, s);
        return;
    }
    DVec<int> ucnt, small, mid, big, cnts;
    ucnt.alloc(std::max(n, 1), s);
    small.alloc(std::max(n, 1), s);
    mid.alloc(std::max(n, 1), s);
    big.alloc(std::max(n, 1), s);
    cnts.alloc(3, s);
    cnts.zero();
    k_spgemm_cand<<<grid_for(std::max(n, 1), kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, B.rowptr.p, small.p,
                                                                      mid.p, big.p, cnts.p);
    CK_LAUNCH();
    // the listed rows run on fixed grids that read their counts on the device
    unsigned tblocks = (unsigned)grid_for(std::max(n, 1), kBlock);
    unsigned sblocks = (unsigned)grid_for(n, kSW, 148 * 8);
    unsigned mblocks = (unsigned)grid_for(n, kMW, 148 * 8);
    unsigned bblocks = (unsigned)grid_for(n, kBW, 148 * 8);
    k_spgemm_merge<8, kTierMerge8><<<tblocks, kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, nullptr, B.rowptr.p, B.col.p,
                                                     nullptr, nullptr, nullptr, nullptr, ucnt.p);
    CK_LAUNCH();
    k_spgemm_merge<16, kTierMerge16><<<tblocks, kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, nullptr, B.rowptr.p,
                                                            B.col.p, nullptr, nullptr, nullptr, nullptr, ucnt.p);
    CK_LAUNCH();
    k_spgemm_tiny<<<tblocks, kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, nullptr, B.rowptr.p, B.col.p, nullptr, nullptr,
                                             nullptr, nullptr, ucnt.p);
    CK_LAUNCH();
    k_spgemm_rowcount<64, kSmallCand, kSW, false><<<sblocks, kSW * 32, 0, s>>>(n, small.p, cnts.p, A.rowptr.p,
                                                                               A.col.p, B.rowptr.p, B.col.p, ucnt.p);
    CK_LAUNCH();
    k_spgemm_rowcount<256, 128, kMW, false><<<mblocks, kMW * 32, 0, s>>>(n, mid.p, cnts.p + 1, A.rowptr.p, A.col.p,
                                                                          B.rowptr.p, B.col.p, ucnt.p);
    CK_LAUNCH();
    k_spgemm_rowcount<1024, 512, kBW, false><<<bblocks, kBW * 32, 0, s>>>(n, big.p, cnts.p + 2, A.rowptr.p, A.col.p,
                                                                           B.rowptr.p, B.col.p, ucnt.p);
    CK_LAUNCH();
    C.n = n;
    C.ncol = B.ncol;
    C.rowptr.alloc(n + 1, s);
    exclusive_scan(ucnt.p, C.rowptr.p, n, s);
    C.nnz = read_int(C.rowptr.p + n, s);
    if (C.nnz < 0) fail(CPR_ERR_OOM, "Galerkin product too large");
    // the tier counts are read back: printed at CPR_SETUP_TIMING=2 only
    if (const char *t = getenv("CPR_SETUP_TIMING"); t && atoi(t) >= 2)
        fprintf(stderr, "[cpr setup] spgemm n=%d annz=%d bnnz=%d cnnz=%d small=%d mid=%d big=%d\n", n, A.nnz,
                B.nnz, C.nnz, read_int(cnts.p, s), read_int(cnts.p + 1, s), read_int(cnts.p + 2, s));
    C.col.alloc(std::max(C.nnz, 1), s);
    C.val.alloc(std::max(C.nnz, 1), s);
    k_spgemm_merge<8, kTierMerge8><<<tblocks, kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p,
                                                     B.val.p, C.rowptr.p, C.col.p, C.val.p, nullptr);
    CK_LAUNCH();
    k_spgemm_merge<16, kTierMerge16><<<tblocks, kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p,
                                                            B.col.p, B.val.p, C.rowptr.p, C.col.p, C.val.p,
                                                            nullptr);
    CK_LAUNCH();
    k_spgemm_tiny<<<tblocks, kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p,
                                             C.rowptr.p, C.col.p, C.val.p, nullptr);
    CK_LAUNCH();
    k_spgemm_rowfill<64, kSmallCand, kSW, false><<<sblocks, kSW * 32, 0, s>>>(
        n, small.p, cnts.p, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p, C.rowptr.p, C.col.p,
        C.val.p);
    CK_LAUNCH();
    k_spgemm_rowfill<256, 128, kMW, false><<<mblocks, kMW * 32, 0, s>>>(
        n, mid.p, cnts.p + 1, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p, C.rowptr.p, C.col.p,
        C.val.p);
    CK_LAUNCH();
    k_spgemm_rowfill<1024, 512, kBW, false><<<bblocks, kBW * 32, 0, s>>>(
        n, big.p, cnts.p + 2, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p, C.rowptr.p, C.col.p,
        C.val.p);
    CK_LAUNCH();
}

constexpr int kHsBatch = 6;   // handshake rounds launched per host check of the unmatched count

// P (n x na) of unsmoothed aggregation from the aggregate of every node.
void unit_p(int n, int na, const int *agg, DCsr &P, cudaStream_t s) {
    P.n = n;
    P.ncol = na;
    P.nnz = n;
    P.rowptr.alloc(n + 1, s);
    P.col.alloc(std::max(n, 1), s);
    P.val.alloc(std::max(n, 1), s);
    k_unit_p<<<grid_for(n + 1, kBlock), kBlock, 0, s>>>(n, agg, P.rowptr.p, P.col.p, P.val.p);
    CK_LAUNCH();
}

// One pairwise matching pass on A; agg gets each node's aggregate, the
// return value is the number of aggregates.
int pairwise_pass(const DCsr &A, double beta, uint32_t hb, DVec<int> &agg, cudaStream_t s) {
    int n = A.n;
    DVec<int> tr, tc;
    DVec<double> tv;
    transpose(n, n, A.nnz, A.rowptr.p, A.col.p, A.val.p, tr, tc, &tv, s);
    // the strong set S with its couplings, and S^T
    DVec<int> cnt, sr, sc;
    DVec<double> sv;
    cnt.alloc(std::max(n, 1), s);
    k_pair_strong<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, tr.p, tc.p, tv.p, beta,
                                                        nullptr, cnt.p, nullptr, nullptr);
    CK_LAUNCH();
    sr.alloc(n + 1, s);
    exclusive_scan(cnt.p, sr.p, n, s);
    int snnz = read_int(sr.p + n, s);
    sc.alloc(std::max(snnz, 1), s);
    sv.alloc(std::max(snnz, 1), s);
    k_pair_strong<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, tr.p, tc.p, tv.p, beta,
                                                        sr.p, nullptr, sc.p, sv.p);
    CK_LAUNCH();
    DVec<int> str, stc;
    DVec<double> stv;
    transpose(n, n, snnz, sr.p, sc.p, sv.p, str, stc, &stv, s);
    // handshake rounds
    DVec<int> mate, ptr, left;
    mate.alloc(std::max(n, 1), s);
    ptr.alloc(std::max(n, 1), s);
    k_fill_int<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, mate.p, kUnmatched);
    CK_LAUNCH();
    if (n <= kSmallLevel) {
        k_hs_small<<<1, 1024, 0, s>>>(n, sr.p, sc.p, sv.p, str.p, stc.p, stv.p, mate.p, ptr.p, hb);
        CK_LAUNCH();
    } else {
        left.alloc(1, s);
        CK(cudaMemcpyAsync(left.p, &n, sizeof(int), cudaMemcpyHostToDevice, s));
        int rounds = 0;
        do {
            for (int k = 0; k < kHsBatch; k++, rounds++) {
                k_hs_point<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, sr.p, sc.p, sv.p, str.p, stc.p, stv.p, mate.p,
                                                                 ptr.p, hb, left.p);
                CK_LAUNCH();
                k_hs_commit<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, mate.p, ptr.p, left.p);
                CK_LAUNCH();
            }
            if (rounds > n + 8) fail(CPR_ERR_CUDA, "pairwise matching did not terminate");
        } while (read_int(left.p, s) > 0);
    }
    DVec<int> host, flag, idx;
    host.alloc(std::max(n, 1), s);
    k_hs_host<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, sr.p, sc.p, sv.p, str.p, stc.p, stv.p, mate.p, hb, host.p);
    CK_LAUNCH();
    flag.alloc(std::max(n, 1), s);
    idx.alloc(n + 1, s);
    k_hs_leader<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, mate.p, host.p, flag.p);
    CK_LAUNCH();
    exclusive_scan(flag.p, idx.p, n, s);
    int na = read_int(idx.p + n, s);
    agg.alloc(std::max(n, 1), s);
    k_hs_number<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, mate.p, host.p, idx.p, agg.p);
    CK_LAUNCH();
    return na;
}

// Double pairwise aggregation: a pass on A, then a pass on the pair operator
// P1^T A P1 (hash hb ^ 0x9e3779b9), so aggregates hold at most four nodes.
int aggregate_double(const DCsr &A, double beta, uint32_t hb, DVec<int> &agg, cudaStream_t s) {
    int n = A.n;
    DVec<int> a1, a2;
    int n1 = pairwise_pass(A, beta, hb, a1, s);
    DCsr P1, R1, AP, A1;
    unit_p(n, n1, a1.p, P1, s);
    R1.n = n1;
    R1.ncol = n;
    R1.nnz = n;
    transpose(n, n1, n, P1.rowptr.p, P1.col.p, P1.val.p, R1.rowptr, R1.col, &R1.val, s);
    spgemm(A, P1, AP, s);
    spgemm(R1, AP, A1, s);
    int n2 = pairwise_pass(A1, beta, hb ^ 0x9e3779b9u, a2, s);
    agg.alloc(std::max(n, 1), s);
    k_compose_agg<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, a1.p, a2.p, agg.p);
    CK_LAUNCH();
    return n2;
}

void to_f32(const DVec<double> &a, DVec<float> &b, cudaStream_t s) {
    b.alloc(std::max<size_t>(a.n, 1), s);
    if (a.n) {
        k_d2f<<<grid_for((long)a.n, kBlock, 148 * 16), kBlock, 0, s>>>((long)a.n, a.p, b.p);
        CK_LAUNCH();
    }
}

int lanes_for(double avg, long rows, long target);

// The entries of dst (its row pointers already in place) from src's: the
// fill pass of perm_csr, also run alone to refresh dst's values.
void perm_fill(const DCsr &src, const int *order, const int *icol, bool skip_diag, DCsr &dst, cudaStream_t s,
               float *val32) {
    int n = src.n;
    if (!n) return;
    // lanes per row: a few entries per lane, at least 2^17 threads
    int g = std::min(8, lanes_for((double)src.nnz / std::max(n, 1), n, 1L << 17));
    auto fill = [&](auto kern, int G) {
        kern<<<grid_for((long)n * G, kBlock), kBlock, 0, s>>>(n, order, src.rowptr.p, src.col.p, src.val.p,
                                                             skip_diag, icol, dst.rowptr.p, dst.col.p, dst.val.p,
                                                             val32);
    };
    switch (g) {
    case 1: fill(k_perm_fill<1>, 1); break;
    case 2: fill(k_perm_fill<2>, 2); break;
    case 4: fill(k_perm_fill<4>, 4); break;
    default: fill(k_perm_fill<8>, 8); break;
    }
    CK_LAUNCH();
}

// dst = src with rows taken in `order` and columns mapped through icol.
void perm_csr(const DCsr &src, const int *order, const int *icol, int ncol, bool skip_diag, DCsr &dst,
              cudaStream_t s, DVec<float> *val32 = nullptr) {
    int n = src.n;
    DVec<int> cnt;
    cnt.alloc(std::max(n, 1), s);
    k_perm_count<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, order, src.rowptr.p, src.col.p, skip_diag, cnt.p);
    CK_LAUNCH();
    dst.n = n;
    dst.ncol = ncol;
    dst.rowptr.alloc(n + 1, s);
    exclusive_scan(cnt.p, dst.rowptr.p, n, s);
    // no read-back: the copy keeps every entry (less one diagonal per row when
    // skip_diag, each level row holding exactly one), so the source's count
    // bounds the allocation and the host count is exact for level matrices
    dst.nnz = skip_diag ? std::max(src.nnz - n, 0) : src.nnz;
    dst.col.alloc(std::max(src.nnz, 1), s);
    dst.val.alloc(std::max(src.nnz, 1), s);
    if (val32) val32->alloc(std::max(src.nnz, 1), s);   // the FP32 shadow, filled alongside
    perm_fill(src, order, icol, skip_diag, dst, s, val32 ? val32->p : nullptr);
}

// Lanes per row for a mean row length: about four entries per lane (1..32
// lanes), so short rows keep many rows, and several independent loads per
// lane, in flight.
// Lanes per row for a launch over `rows` rows averaging `avg` entries: at
// least a quarter of the row length, and enough lanes that the launch has
// `target` threads (up to 32 lanes).  A lane's work is a chain of dependent
// loads (row extent, entries, gathered x), so small launches wait on that
// chain and gain from spreading each row over more lanes.  The rule and its
// thread targets come from sweeping 1..32 lanes per kernel family and level
// on B300 (128x128x32 and 60x220x85 hierarchies): it matches the fastest
// width, or comes within a few percent of it, on every level.
int lanes_for(double avg, long rows, long target) {
    int g = 1;
    while (g < 32 && (4 * g < avg || rows * g < target)) g <<= 1;
    return g;
}

void copy_ints(DVec<int> &dst, const int *src, size_t n, cudaStream_t s) {
    dst.alloc(std::max<size_t>(n, 1), s);
    if (n) CK(cudaMemcpyAsync(dst.p, src, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
}

// ---------------------------------------------- value passes of the setup
//
// Each fills buffers that are already in place from the current values, so
// the full setup and the numeric refresh (resetup = 1) run the same kernels.

// The product lists of C = A B (C from an earlier spgemm of A and B's
// patterns): count pass, scan, fill pass; lanes per row from B's mean row
// length.
void plan_product(const DCsr &A, const DCsr &B, const DCsr &C, ProdPlan &pl, int *err, cudaStream_t s) {
    int n = A.n, nnz = C.nnz;
    DVec<int> cur;
    cur.alloc(std::max(nnz, 1), s);
    cur.zero();
    int g = lanes_for((double)B.nnz / std::max(B.n, 1), n, 1L << 17);
    auto run = [&](auto kern, int G) {
        kern<<<grid_for((long)n * G, kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, B.rowptr.p, B.col.p,
                                                             C.rowptr.p, C.col.p, cur.p, pl.pa.p, pl.pb.p, err);
        CK_LAUNCH();
    };
    auto pass = [&](auto fill) {
        constexpr bool F = decltype(fill)::value;
        if (!n) return;
        switch (g) {
        case 1: run(k_plan_pairs<1, F>, 1); break;
        case 2: run(k_plan_pairs<2, F>, 2); break;
        case 4: run(k_plan_pairs<4, F>, 4); break;
        case 8: run(k_plan_pairs<8, F>, 8); break;
        case 16: run(k_plan_pairs<16, F>, 16); break;
        default: run(k_plan_pairs<32, F>, 32); break;
        }
    };
    pass(std::false_type{});
    pl.ptr.alloc((size_t)nnz + 1, s);
    exclusive_scan(cur.p, pl.ptr.p, nnz, s);
    int np = read_int(pl.ptr.p + nnz, s);
    if (np < 0) fail(CPR_ERR_OOM, "product lists of a Galerkin product too large");
    pl.pa.alloc(std::max(np, 1), s);
    pl.pb.alloc(std::max(np, 1), s);
    if (nnz) CK(cudaMemcpyAsync(cur.p, pl.ptr.p, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s));
    pass(std::true_type{});
}

// C's values from its product lists.
void plan_values(const ProdPlan &pl, const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
    if (!C.nnz) return;
    k_plan_values<<<grid_for(C.nnz, kBlock), kBlock, 0, s>>>(C.nnz, pl.ptr.p, pl.pa.p, pl.pb.p, A.val.p, B.val.p,
                                                             C.val.p);
    CK_LAUNCH();
}

// Lanes per block row in k_bilu_factor_color: FP32 rows take a group of
// lanes; FP64 rows one thread each (B300's FP64 pipe pays for every issued
// instruction whatever its active lanes, so idle lanes of a group cost FP64
// throughput).
constexpr int kBiluFactorLanesF32 = 8;

// The BILU(0) factors of the current A on the kept ordering and L/U patterns:
// A's blocks copied (FP64) or rounded (FP32 mode) into the factor array,
// factored color by color, then split into L, U and the inverted diagonal
// blocks in position order.
void bilu_values(cpr_handle *h, const int *bdiag, cudaStream_t s) {
    Bilu &B = h->bilu;
    int nb = h->nb, nnzb = h->nnzb;
    auto factor_and_split = [&](auto *lu, auto *Lv, auto *Uv, auto *Dv) {
        using T = std::remove_pointer_t<decltype(lu)>;
        for (int c = 0; c < B.ncolors; c++) {
            int cnt = B.color_off[c + 1] - B.color_off[c];
            if (!cnt) continue;
            constexpr int G = sizeof(T) == 4 ? kBiluFactorLanesF32 : 1;
            k_bilu_factor_color<T, G><<<grid_for((long)cnt * G, 128), 128, 0, s>>>(
                B.rows_by_color.p + B.color_off[c], cnt, h->rowptr.p, h->col.p, B.color.p, bdiag, lu, h->err.p,
                h->opt.bilu_order);
            CK_LAUNCH();
        }
        // a singular pivot block is reported by the caller's error check
        k_bilu_split_fill<T, 8><<<grid_for(8L * nb, kBlock), kBlock, 0, s>>>(
            nb, h->rowptr.p, h->col.p, B.color.p, B.iperm.p, lu, B.Lrowptr.p, B.Lcol.p, Lv, B.Urowptr.p, B.Ucol.p,
            Uv, Dv);
        CK_LAUNCH();
    };
    if (h->opt.precond_fp32) {
        k_d2f<<<grid_for(9L * nnzb, kBlock, 148 * 16), kBlock, 0, s>>>(9L * nnzb, h->val.p, B.lu32.p);
        CK_LAUNCH();
        factor_and_split(B.lu32.p, B.Lval32.p, B.Uval32.p, B.Dinv32.p);
    } else {
        CK(cudaMemcpyAsync(B.lu.p, h->val.p, sizeof(double) * 9 * (size_t)nnzb, cudaMemcpyDeviceToDevice, s));
        factor_and_split(B.lu.p, B.Lval.p, B.Uval.p, B.Dinv.p);
    }
}

// Column 0 of A's blocks in positions (the copy B keeps for the second
// residual of Alg. 1), and its FP32 shadow when that exists.
void col0_values(cpr_handle *h, cudaStream_t s) {
    const Bilu &B = h->bilu;
    int nb = h->nb;
    k_col0_fill<8><<<grid_for(8L * nb, kBlock), kBlock, 0, s>>>(nb, B.rows_by_color.p, B.iperm.p, h->rowptr.p,
                                                               h->col.p, h->val.p, h->c0rowptr.p, h->c0col.p,
                                                               h->pcol0.p);
    CK_LAUNCH();
    size_t n = std::min(h->pcol0.n, h->pcol0_32.n);
    if (h->pcol0_32.p && n) {
        k_d2f<<<grid_for((long)n, kBlock, 148 * 16), kBlock, 0, s>>>((long)n, h->pcol0.p, h->pcol0_32.p);
        CK_LAUNCH();
    }
}

// The dense LU factorisation of the coarsest matrix: larger than this it is
// factored in global memory.
constexpr int kLuSmemMax = 200 * 1024;

bool lu_in_smem(int n) { return (size_t)n * n * sizeof(double) <= kLuSmemMax; }

// The shared-memory ceiling of k_dense_lu (the staged matrix and the row
// order), set before its first launch and outside any capture: always the
// same value, so handles set up on other host threads never see a smaller
// limit than the one they launch with.
void lu_smem_attr() {
    CK(cudaFuncSetAttribute(k_dense_lu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            kLuSmemMax + (int)sizeof(int) * kMaxCoarse));
    // staged factors (n*n*8 <= kLuSmemMax, so n <= 160) and 2n doubles; unstaged, 2n doubles
    CK(cudaFuncSetAttribute(k_dense_inv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            std::max(kLuSmemMax + 16 * 160, 16 * kMaxCoarse)));
}

// h->cinv = the inverse of the coarsest matrix by dense LU with partial
// pivoting, on stream q; a, lu (n*n) and piv (n) are scratch.
void coarse_values(cpr_handle *h, double *a, double *lu, int *piv, cudaStream_t q) {
    const Level &C = h->lev.back();
    int n = C.A.n;
    size_t bytes = sizeof(double) * (size_t)n * n;
    CK(cudaMemsetAsync(a, 0, bytes, q));
    k_csr_to_dense<<<grid_for(n, kBlock), kBlock, 0, q>>>(n, C.A.rowptr.p, C.A.col.p, C.A.val.p, a);
    CK_LAUNCH();
    int use_smem = lu_in_smem(n) ? 1 : 0;
    // global path: factor a copy in storage order, then gather rows into position order
    if (!use_smem) CK(cudaMemcpyAsync(lu, a, bytes, cudaMemcpyDeviceToDevice, q));
    k_dense_lu<<<1, kLuThreads, (use_smem ? bytes : 0) + sizeof(int) * n, q>>>(n, a, lu, piv, use_smem, h->err.p);
    CK_LAUNCH();   // a zero pivot is reported by the caller's error check
    if (!use_smem) {
        k_gather_rows<<<grid_for((long)n * n, kBlock), kBlock, 0, q>>>(n, lu, piv, a);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(lu, a, bytes, cudaMemcpyDeviceToDevice, q));
    }
    size_t inv_smem = sizeof(double) * (2 * (size_t)n + (use_smem ? (size_t)n * n : 0));
    k_dense_inv_cols<<<n, kInvThreads, inv_smem, q>>>(n, lu, piv, h->cinv.p, use_smem);
    CK_LAUNCH();
}

}  // namespace

// ================================================================== public

void validate_bsr(const int *rowptr, const int *col, int nb, int nnzb, int *derr, cudaStream_t s) {
    k_validate_bsr<<<grid_for(nb, kBlock), kBlock, 0, s>>>(rowptr, col, nb, nnzb, derr);
    CK_LAUNCH();
}

void free_preconditioner(cpr_handle *h) {
    if (h->nr_exec) cudaGraphExecDestroy(h->nr_exec);
    if (h->nr_graph) cudaGraphDestroy(h->nr_graph);
    h->nr_exec = nullptr;
    h->nr_graph = nullptr;
    h->nr_kernels = 0;
    h->nr_ready = false;
    h->bdiag.release();
    h->c_a.release();
    h->c_lu.release();
    h->c_piv.release();
    h->tail_top = -1;
    h->lev.clear();
    h->pcol0.release();
    h->pcol0_32.release();
    h->c0rowptr.release();
    h->c0col.release();
    h->ep_map.release();
    h->w.release();
    h->w32.release();
    h->cinv.release();
    h->bilu = Bilu{};
    h->cn = 0;
    h->have_B = false;
}

// A kept B takes the current A for its second residual (reuse_refresh): the
// column-0 copy, and its FP32 shadow, are refilled in place.  Pattern and
// positions are A's and B's, both unchanged, so the step graphs captured for
// B stay valid.
void refresh_second_residual(cpr_handle *h) { col0_values(h, h->stream); }

// Phase marks of a setup, printed to stderr when CPR_SETUP_TIMING is set
// (diagnostics only).  A mark records a timing event on its clock's stream
// and the host time; each prints as name=host/device, both in ms since the
// setup began: when the host issued the mark and when the stream reached it.
// Marks do not synchronise, so both chains run as they do untimed.
struct PhaseClock {
    bool on = getenv("CPR_SETUP_TIMING") != nullptr;
    cudaStream_t s = nullptr;
    const char *tag = "";
    const PhaseClock *origin = nullptr;   // the clock whose start is time zero (this one when null)
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    cudaEvent_t e0 = nullptr;
    struct Mark {
        const char *name;
        double host;
        cudaEvent_t ev;
    };
    std::vector<Mark> marks;
    void start(cudaStream_t stream) {
        s = stream;
        if (on && !e0 && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, s);
    }
    void mark(const char *name) {
        if (!on) return;
        const PhaseClock &o = origin ? *origin : *this;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, s);
        marks.push_back(
            {name, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - o.t0).count(), e});
    }
    ~PhaseClock() {
        if (!on) return;
        const PhaseClock &o = origin ? *origin : *this;
        std::string line;
        for (auto &m : marks) {
            float d = -1.0f;
            if (cudaEventSynchronize(m.ev) == cudaSuccess && o.e0) cudaEventElapsedTime(&d, o.e0, m.ev);
            char buf[96];
            snprintf(buf, sizeof(buf), " %s=%.2f/%.2f", m.name, m.host, d);
            line += buf;
            cudaEventDestroy(m.ev);
        }
        if (e0) cudaEventDestroy(e0);
        fprintf(stderr, "[cpr setup ms host/dev]%s%s\n", tag, line.c_str());
    }
};

// Setup work that needs only its own inputs -- the BILU(0) second stage
// (needs A) and each level's smoother coloring (needs A_l) -- runs on a
// worker host thread with its own stream while this thread builds the AMG
// chain.  Both chains are long sequences of small kernels with host
// read-backs, so running them side by side keeps the GPU and the host busy.
// A task starts behind an event of the main stream; join() makes the main
// stream wait for everything the worker issued and rethrows its error.
class SideWorker {
  public:
    SideWorker(cpr_handle *h, const PhaseClock *origin) : h_(h) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if (!h->side) {
            // the side chain (BILU(0) values, the level colorings) has slack
            // behind the main AMG chain, so it takes no priority over it: at
            // the highest priority 20 warm setups of 128x128x32 took 7.84 and
            // 8.39 ms (median; up to 13.6), at this one 7.72 and 7.70 (up to 8.4)
            int lo = 0, hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, lo));
        }
        clk_.s = h->side;
        clk_.tag = " side:";
        clk_.origin = origin;
        th_ = std::thread([this, dev] { run(dev); });
    }
    ~SideWorker() {
        if (th_.joinable()) {   // unwinding: let the side work finish before the caller's buffers go
            stop();
            th_.join();
            cudaStreamSynchronize(h_->side);
        }
    }
    cudaStream_t stream() const { return h_->side; }
    void mark(const char *name) {   // phase times of the worker's own tasks
        if (std::this_thread::get_id() == th_.get_id()) clk_.mark(name);
    }
    // Queue f(stream) for the worker.  Callers post right after a host
    // read-back of the main stream, so everything f reads from it is already
    // complete and no cross-stream event is needed.
    using Task = std::function<void(cudaStream_t)>;
    void post(Task f) {
        std::lock_guard<std::mutex> lk(mu_);
        q_.push_back(std::move(f));
        cv_.notify_one();
    }
    // Run tasks the worker has not started yet on the calling thread and
    // stream s, newest first, while the worker goes on from the oldest.
    void help(cudaStream_t s) {
        for (;;) {
            Task f;
            {
                std::lock_guard<std::mutex> lk(mu_);
                if (q_.empty() || err_) return;
                f = std::move(q_.back());
                q_.pop_back();
            }
            f(s);
        }
    }
    // Task `key` has finished; the task recorded an event for its stream work.
    void finished(int key) {
        std::lock_guard<std::mutex> lk(mu_);
        if ((size_t)key >= finished_.size()) finished_.resize(key + 1, 0);
        finished_[key] = 1;
        cvd_.notify_all();
    }
    // Wait until task `key` has finished, running queued tasks (newest first)
    // on this thread and stream s meanwhile.
    void wait(int key, cudaStream_t s) {
        for (;;) {
            Task f;
            {
                std::unique_lock<std::mutex> lk(mu_);
                for (;;) {
                    if (err_) std::rethrow_exception(err_);
                    if ((size_t)key < finished_.size() && finished_[key]) return;
                    if (!q_.empty()) break;
                    if (!busy_) fail(CPR_ERR_CUDA, "setup waited on a side task that was never posted");
                    cvd_.wait(lk);
                }
                f = std::move(q_.back());
                q_.pop_back();
            }
            f(s);
        }
    }
    // Wait for the worker and for everything it issued on the side stream.
    void join() {
        stop();
        th_.join();
        if (err_) std::rethrow_exception(err_);
        CK(cudaStreamSynchronize(h_->side));
    }

  private:
    void stop() {
        std::lock_guard<std::mutex> lk(mu_);
        done_ = true;
        cv_.notify_one();
    }
    void run(int dev) {
        cudaSetDevice(dev);
        use_side_pool(true);
        for (;;) {
            Task f;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return done_ || !q_.empty(); });
                if (q_.empty()) return;
                f = std::move(q_.front());
                q_.pop_front();
                if (err_) continue;   // after a failure, drain without running
                busy_ = true;
            }
            try {
                f(h_->side);
            } catch (...) {
                std::lock_guard<std::mutex> lk(mu_);
                err_ = std::current_exception();
            }
            std::lock_guard<std::mutex> lk(mu_);
            busy_ = false;
            cvd_.notify_all();
        }
    }
    cpr_handle *h_;
    PhaseClock clk_;
    std::thread th_;
    std::mutex mu_;
    std::condition_variable cv_, cvd_;
    std::deque<Task> q_;
    std::vector<char> finished_;
    bool done_ = false, busy_ = false;
    std::exception_ptr err_;
};


// Build B from the handle's current A (Sec. 3.1; the setup steps of Alg. 6 per level).
void build_preconditioner(cpr_handle *h) {
    // BILU(0)'s coloring (JP at theta = 0 on the off-diagonal block pattern,
    // hashed by the seed), its order and its L/U pattern, and the column-0
    // copy's pattern are functions of A's block pattern alone: while that is
    // unchanged they are kept from the last setup, bit for bit what a rebuild
    // would give, and only their values are recomputed.
    bool keep = h->bilu.pattern == h->pattern_id && h->bilu.ncolors > 0 && h->c0rowptr.p && h->c0col.p;
    Bilu kept_bilu;
    DVec<int> kept_c0rowptr, kept_c0col;
    if (keep) {
        kept_bilu = std::move(h->bilu);
        kept_c0rowptr = std::move(h->c0rowptr);
        kept_c0col = std::move(h->c0col);
    }
    free_preconditioner(h);
    if (keep) {
        h->bilu = std::move(kept_bilu);
        h->c0rowptr = std::move(kept_c0rowptr);
        h->c0col = std::move(kept_c0col);
    }
    Nvtx nv("setup");
    cudaStream_t s = h->stream;
    PhaseClock clk;
    clk.start(s);
    const cpr_opts &o = h->opt;
    int nb = h->nb, nnzb = h->nnzb;
    bool f32 = o.precond_fp32 != 0;
    // levels are referenced by the side worker while this thread appends: no reallocation
    h->lev.reserve((size_t)std::max(1, o.max_levels) + 1);
    // one event per level coloring: the layout of a level waits on its own and
    // the next level's coloring, not on the whole side worker
    while (h->ev_color.size() < (size_t)std::max(1, o.max_levels) + 1) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->ev_color.push_back(e);
    }

    // ---- decoupling and the pressure matrix A_P (level 0) ----
    DVec<int> &bdiag = h->bdiag;   // kept: the numeric refresh reads it
    bdiag.alloc(nb, s);
    k_diagpos<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->col.p, bdiag.p);
    CK_LAUNCH();
    h->w.alloc(3 * (size_t)nb, s);
    k_decouple<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, bdiag.p, h->val.p, o.decouple, h->w.p, h->err.p);
    CK_LAUNCH();
    check_err(h, "singular diagonal block in the decoupling");
    h->lev.emplace_back();
    {
        Level &L0 = h->lev[0];
        L0.A.n = L0.A.ncol = nb;
        L0.A.nnz = nnzb;
        copy_ints(L0.A.rowptr, h->rowptr.p, nb + 1, s);
        copy_ints(L0.A.col, h->col.p, nnzb, s);
        L0.A.val.alloc(nnzb, s);
        k_pressure_matrix<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->val.p, h->w.p,
                                                                 L0.A.val.p);
        CK_LAUNCH();
    }

    clk.mark("decouple");
    // ---- second stage: multicolor BILU(0), on the side worker ----
    SideWorker side(h, &clk);
    side.post([h, nb, nnzb, f32, keep, &bdiag, &side](cudaStream_t s) {
        Nvtx r("BILU(0) setup");
        Bilu &B = h->bilu;
        int nl = 0, nu = 0;
        if (keep) {   // the kept structure
            nl = B.nl;
            nu = B.nu;
            side.mark("bilu_kept");
        } else {
            // every row holds exactly one diagonal block: nnzb - nb entries
            SymGraph G = sym_graph(build_pattern_ub(nb, (long)nnzb - nb, s, [&](const int *srow, int *out) {
                                       k_offdiag_pattern<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p,
                                                                                                h->col.p, srow, out);
                                       CK_LAUNCH();
                                   }),
                                   (long)nnzb - nb, s);
            side.mark("bilu_graph");
            // multicolor (JP at theta = 0), or the natural order's level sets
            B.ncolors = h->opt.bilu_order ? level_sets(G, B.color, s) : jp_color(h, G, 2, 0, B.color, s);
            side.mark("bilu_jp");
            rows_by_color(nb, B.color.p, B.ncolors, B.color_off, B.rows_by_color, s);
            B.iperm.alloc(nb, s);
            k_iperm<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, B.rows_by_color.p, B.iperm.p);
            CK_LAUNCH();
            DVec<int> lcnt, ucnt;
            lcnt.alloc(nb, s);
            ucnt.alloc(nb, s);
            k_bilu_split_count<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, B.rows_by_color.p, h->rowptr.p, h->col.p,
                                                                      B.color.p, lcnt.p, ucnt.p);
            CK_LAUNCH();
            B.Lrowptr.alloc(nb + 1, s);
            B.Urowptr.alloc(nb + 1, s);
            exclusive_scan(lcnt.p, B.Lrowptr.p, nb, s);
            exclusive_scan(ucnt.p, B.Urowptr.p, nb, s);
            nl = read_int(B.Lrowptr.p + nb, s);
            nu = read_int(B.Urowptr.p + nb, s);
            B.nl = nl;
            B.nu = nu;
            B.Lcol.alloc(std::max(nl, 1), s);
            B.Ucol.alloc(std::max(nu, 1), s);
            side.mark("bilu_order");
        }
        // value buffers: a kept structure keeps them too (every entry is rewritten)
        auto sized = [s](auto &v, size_t count) {
            if (v.n != count || !v.p) v.alloc(count, s);
        };
        if (f32) {
            sized(B.lu32, 9 * (size_t)nnzb);
            sized(B.Lval32, 9 * (size_t)std::max(nl, 1));
            sized(B.Uval32, 9 * (size_t)std::max(nu, 1));
            sized(B.Dinv32, 9 * (size_t)nb);
        } else {
            sized(B.lu, 9 * (size_t)nnzb);
            sized(B.Lval, 9 * (size_t)std::max(nl, 1));
            sized(B.Uval, 9 * (size_t)std::max(nu, 1));
            sized(B.Dinv, 9 * (size_t)nb);
        }
        bilu_values(h, bdiag.p, s);
        side.mark("bilu_factor");
        // the frozen column-0 copy of A in positions
        if (!keep) {
            DVec<int> ccnt;
            ccnt.alloc(nb, s);
            k_col0_perm<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, B.rows_by_color.p, B.iperm.p, h->rowptr.p,
                                                               h->col.p, h->val.p, nullptr, nullptr, nullptr, ccnt.p);
            CK_LAUNCH();
            h->c0rowptr.alloc(nb + 1, s);
            exclusive_scan(ccnt.p, h->c0rowptr.p, nb, s);
            h->c0col.alloc(nnzb, s);
        }
        h->pcol0.alloc(3 * (size_t)nnzb, s);
        col0_values(h, s);   // its FP32 shadow is made after the side work has joined
        side.mark("col0");
    });
    // ---- the AMG hierarchy ----
    for (int l = 0;; l++) {
        int n = h->lev[l].A.n;
        Nvtx r("AMG level");
        {
            Level &L = h->lev[l];
            L.dpos.alloc(n, s);
            k_diagpos<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p, L.dpos.p);
            CK_LAUNCH();
            k_check_diag<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.dpos.p, L.A.val.p, nullptr, h->err.p);
            CK_LAUNCH();   // a zero diagonal is reported by the check at the end of the setup
        }
        if (n <= o.coarse_max || l + 1 >= o.max_levels) break;
        Level &L = h->lev[l];
        clk.mark("diag");
        Graph S;
        DVec<int> flag, cidx;
        int nc = 0;
        bool ua = o.amg == 1;
        if (ua) {   // UA-AMG (Sec. 6): cf holds every node's aggregate
            nc = aggregate_double(L.A, o.theta_amg, hash_base(o.seed, 3, l), L.cf, s);
            clk.mark("aggregate");
            if (nc == 0 || (double)nc > 0.95 * (double)n) {
                L.cf.release();
                break;
            }
        } else {
            // classical strength and PMIS
            bool long_rows = L.A.nnz > 16L * n;   // warp per row pays once rows average over 16 entries
            S = build_pattern(n, s, [&](const int *srow, int *out) {
                if (long_rows)
                    k_strength_rs_warp<<<grid_for((long)n * 32, kBlock), kBlock, 0, s>>>(
                        n, L.A.rowptr.p, L.A.col.p, L.A.val.p, o.theta_amg, srow, out);
                else
                    k_strength_rs<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p, L.A.val.p,
                                                                        o.theta_amg, srow, out);
                CK_LAUNCH();
            });
            clk.mark("strength");
            DVec<int> trow, tcol;
            // PMIS reads S^T's rows as sets (|S^T_i| and all-neighbour tests): left unsorted
            transpose(n, n, S.nnz, S.rowptr.p, S.col.p, nullptr, trow, tcol, nullptr, s, false);
            clk.mark("st");
            L.cf.alloc(n, s);
            DVec<int> sel, und;
            sel.alloc(n, s);
            und.alloc(1, s);
            und.zero();
            k_pmis_init<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, trow.p, L.cf.p, und.p);
            CK_LAUNCH();
            uint32_t hb = hash_base(o.seed, 1, l);
            int rounds = 0;
            // lanes per point: about kJpPre of a typical |S_i| + |S^T_i| entries per
            // lane, as long as every point still has its lanes resident at once
            int lanes = 1;
            while (lanes < 16 && (long)lanes * kJpPre * n < 2L * S.nnz && 2L * lanes * n <= kResidentThreads)
                lanes <<= 1;
            if (n <= kSmallLevel) {
                // one CTA: lanes only while every point still fits one pass of its 1024 threads
                lanes = 1;
                while (lanes < 8 && (long)2 * lanes * n <= 1024) lanes <<= 1;
                auto small = [&](auto kern) {
                    kern<<<1, 1024, 0, s>>>(n, S.rowptr.p, S.col.p, trow.p, tcol.p, hb, L.cf.p, sel.p, und.p);
                    CK_LAUNCH();
                };
                switch (lanes) {
                case 1: small(k_pmis_small<1>); break;
                case 2: small(k_pmis_small<2>); break;
                case 4: small(k_pmis_small<4>); break;
                case 8: small(k_pmis_small<8>); break;
                default: small(k_pmis_small<16>); break;
                }
            }
            if (n > kSmallLevel) {
                unsigned grid = grid_for((long)n * lanes, kBlock);
                auto round = [&](auto ksel, auto kcom) {
                    ksel<<<grid, kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, trow.p, tcol.p, hb, L.cf.p, sel.p, und.p);
                    CK_LAUNCH();
                    kcom<<<grid, kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, L.cf.p, sel.p, und.p);
                    CK_LAUNCH();
                };
                do {
                    for (int k = 0; k < kPmisBatch; k++, rounds++) {
                        switch (lanes) {
                        case 1: round(k_pmis_select<1>, k_pmis_commit<1>); break;
                        case 2: round(k_pmis_select<2>, k_pmis_commit<2>); break;
                        case 4: round(k_pmis_select<4>, k_pmis_commit<4>); break;
                        case 8: round(k_pmis_select<8>, k_pmis_commit<8>); break;
                        default: round(k_pmis_select<16>, k_pmis_commit<16>); break;
                        }
                    }
                    if (rounds > n + 8) fail(CPR_ERR_CUDA, "C/F splitting did not terminate");
                } while (read_int(und.p, s) > 0);
                if (getenv("CPR_SETUP_TIMING")) fprintf(stderr, "[cpr setup] pmis n=%d rounds<=%d\n", n, rounds);
            }
            clk.mark("pmis");
            flag.alloc(n, s);
            cidx.alloc(n + 1, s);
            k_is_c<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.cf.p, flag.p);
            CK_LAUNCH();
            exclusive_scan(flag.p, cidx.p, n, s);
            nc = read_int(cidx.p + n, s);
            clk.mark("nc");
            if (nc == 0 || (double)nc > 0.95 * (double)n) {
                L.cf.release();
                break;
            }
        }
        L.nc = nc;
        // the smoother's coloring of this level (Eq. 5.1 strength, symmetrised,
        // JP), on the side worker: it needs only A_l, and
        // level l is smoothed now that it is not the coarsest
        side.post([h, l, n, &side](cudaStream_t s) {
            Nvtx r("level coloring");
            side.mark("idle");
            Level &L = h->lev[l];
            if (n <= kSmallLevel && !(h->opt.coloring == 1 && n <= h->opt.coloring_rows)) {
                // a small level (JP): the whole coloring in one launch
                L.ncolors = color_small(h, L.A, l, L.color, L.color_off, L.rows_by_color, s);
                CK(cudaEventRecord(h->ev_color[l], s));
                side.mark("c_small");
                side.finished(l);
                return;
            }
            // the strength pattern is a subset of A_l's: at most nnz(A_l) entries
            long ub = L.A.nnz;
            DVec<double> thr;   // each row's threshold, from the count pass to the fill pass
            thr.alloc(std::max(n, 1), s);
            Graph S51 = build_pattern_ub(n, ub, s, [&](const int *srow, int *out) {
                k_strength51<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p, L.A.val.p,
                                                                   h->opt.theta_color, srow, out, thr.p);
                CK_LAUNCH();
            });
            side.mark("c_str");
            SymGraph G = sym_graph(std::move(S51), ub, s);
            side.mark("c_graph");
            // the paper's Alg. 4-5 on small levels (coloring = 1), else JP
            if (h->opt.coloring == 1 && n <= h->opt.coloring_rows) L.ncolors = vertices_grouping(h, G.S, L.color, s);
            else L.ncolors = jp_color(h, G, 0, l, L.color, s);
            side.mark("c_jp");
            rows_by_color(n, L.color.p, L.ncolors, L.color_off, L.rows_by_color, s);
            CK(cudaEventRecord(h->ev_color[l], s));
            side.mark("c_order");
            side.finished(l);
        });
        if (ua) {   // unsmoothed aggregation: unit rows, R = P^T
            unit_p(n, nc, L.cf.p, L.P, s);
            L.R.n = nc;
            L.R.ncol = n;
            L.R.nnz = n;
            transpose(n, nc, n, L.P.rowptr.p, L.P.col.p, L.P.val.p, L.R.rowptr, L.R.col, &L.R.val, s);
        } else {   // direct interpolation P and R = P^T
            DVec<int> cnt;
            cnt.alloc(n, s);
            k_interp_count<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, L.cf.p, cnt.p);
            CK_LAUNCH();
            L.P.n = n;
            L.P.ncol = nc;
            L.P.rowptr.alloc(n + 1, s);
            exclusive_scan(cnt.p, L.P.rowptr.p, n, s);
            L.P.nnz = read_int(L.P.rowptr.p + n, s);
            clk.mark("p_nnz");
            L.P.col.alloc(std::max(L.P.nnz, 1), s);
            L.P.val.alloc(std::max(L.P.nnz, 1), s);
            interp_fill(L.A, S.rowptr.p, S.col.p, L.cf.p, cidx.p, L.P, s);
            clk.mark("p_fill");
            L.R.n = nc;
            L.R.ncol = n;
            L.R.nnz = L.P.nnz;
            transpose(n, nc, L.P.nnz, L.P.rowptr.p, L.P.col.p, L.P.val.p, L.R.rowptr, L.R.col, &L.R.val, s);
        }
        // the strength set and coarse indices stay with the level (the numeric refresh reads them)
        L.Srow = std::move(S.rowptr);
        L.Scol = std::move(S.col);
        L.Snnz = S.nnz;
        L.cidx = std::move(cidx);
        clk.mark("interp");
        // Galerkin coarse matrix A_{l+1} = R (A P); the numeric refresh keeps A P
        DCsr AP, Ac;
        spgemm(L.A, L.P, AP, s);
        clk.mark("ap");
        spgemm(L.R, AP, Ac, s);
        if (o.resetup) L.AP = std::move(AP);
        else AP = DCsr{};
        clk.mark("rap");
        h->lev.emplace_back();
        h->lev[l + 1].A = std::move(Ac);
    }

    // ---- coarsest level: dense inverse, on a stream of its own ----
    // The factorisation is FP64 work on one SM (about 0.8 ms at n = 200) that
    // only the solve reads, so it runs beside the layout below.  The guard
    // makes the main stream wait for it before the final error check, and on
    // every unwinding path, so no buffer is released or reused while that
    // stream still writes it.
    struct CoarseJoin {
        cudaStream_t s = nullptr, q = nullptr;
        cudaEvent_t e = nullptr;
        void finish() {
            if (!q) return;
            cudaEventRecord(e, q);
            cudaStreamWaitEvent(s, e, 0);
            q = nullptr;
        }
        ~CoarseJoin() { finish(); }
    } coarse_join;
    {
        Nvtx r("coarse LU");
        for (auto &e : h->ev_coarse)
            if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        if (!h->lu_stream) CK(cudaStreamCreateWithFlags(&h->lu_stream, cudaStreamNonBlocking));
        Level &C = h->lev.back();
        int n = C.A.n;
        if (n > kMaxCoarse) fail(CPR_ERR_INVALID, "coarsest level larger than the dense-solve limit");
        h->cn = n;
        h->cinv.alloc((size_t)n * n, s);    // a handle buffer: allocated and released on the main stream
        cudaStream_t q = h->lu_stream;
        // scratch of the handle (the numeric refresh reuses it), allocated on the main stream
        h->c_a.alloc((size_t)n * n, s);
        h->c_lu.alloc((size_t)n * n, s);
        h->c_piv.alloc(std::max(n, 1), s);
        lu_smem_attr();
        CK(cudaEventRecord(h->ev_coarse[0], s));
        CK(cudaStreamWaitEvent(q, h->ev_coarse[0], 0));
        coarse_join.s = s;
        coarse_join.e = h->ev_coarse[1];
        coarse_join.q = q;
        coarse_values(h, h->c_a.p, h->c_lu.p, h->c_piv.p, q);
    }
    clk.mark("coarse");

    // ---- solve copies in color order, FP32 shadows, work vectors ----
    // Level l's copies need the colorings of levels l and l+1 (the coarsest
    // level is not colored), so each level is laid out as soon as those two
    // side tasks have finished, while the worker goes on with the rest.
    int L = (int)h->lev.size();
    auto layout = [&](int l) {
        Nvtx r("level layout");
        Level &Lv = h->lev[l];
        Level &Nx = h->lev[l + 1];
        int n = Lv.A.n;
        const int *next_iperm = (l + 1 == L - 1) ? nullptr : Nx.iperm.p;
        const int *next_order = (l + 1 == L - 1) ? nullptr : Nx.rows_by_color.p;
        // the FP32 shadows are written by the same kernels
        perm_csr(Lv.A, Lv.rows_by_color.p, Lv.iperm.p, n, true, Lv.Ao, s, f32 ? &Lv.Aoval32 : nullptr);
        perm_csr(Lv.P, Lv.rows_by_color.p, next_iperm, Lv.P.ncol, false, Lv.Pp, s, f32 ? &Lv.Ppval32 : nullptr);
        perm_csr(Lv.R, next_order, Lv.iperm.p, n, false, Lv.Rp, s, f32 ? &Lv.Rpval32 : nullptr);
        Lv.diag.alloc(n, s);
        Lv.dinv.alloc(n, s);
        if (f32) {
            Lv.diag32.alloc(n, s);
            Lv.dinv32.alloc(n, s);
        }
        k_perm_diag<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, Lv.rows_by_color.p, Lv.dpos.p, Lv.A.val.p,
                                                          Lv.diag.p, Lv.dinv.p,
                                                          f32 ? Lv.diag32.p : nullptr, f32 ? Lv.dinv32.p : nullptr);
        CK_LAUNCH();
        // smoothing launches cover one color (n / ncolors rows on average);
        // the residual kernel shares their width
        Lv.gA = lanes_for((double)Lv.Ao.nnz / n, n / std::max(1, Lv.ncolors), 1L << 16);
        Lv.gP = lanes_for((double)Lv.Pp.nnz / n, n, 1L << 16);
        Lv.gR = lanes_for((double)Lv.Rp.nnz / std::max(1, Lv.Rp.n), Lv.Rp.n, 1L << 18);
        Lv.bs = 256;
        if (!f32) {   // FP64: an FP64 instruction costs its issue slot whatever its active lanes
            if (n >= 4096 && Lv.gA >= 8) Lv.gA /= 2;
            Lv.gP = std::min(Lv.gP, 4);
        }
        // a schedule the autotuner chose for a level of these sizes takes precedence
        auto it = h->sched.find({Lv.A.n, (long)Lv.A.nnz});
        if (it != h->sched.end()) {
            Lv.gA = it->second.lanes_a;
            Lv.gP = it->second.lanes_p;
            Lv.gR = it->second.lanes_r;
            Lv.bs = it->second.block;
        }
    };
    for (int l = 0; l < L - 1; l++) {
        side.wait(l, s);
        CK(cudaStreamWaitEvent(s, h->ev_color[l], 0));
        Level &Lv = h->lev[l];
        Lv.iperm.alloc(Lv.A.n, s);
        k_iperm<<<grid_for(Lv.A.n, kBlock), kBlock, 0, s>>>(Lv.A.n, Lv.rows_by_color.p, Lv.iperm.p);
        CK_LAUNCH();
        if (l > 0) layout(l - 1);
    }
    if (L > 1) layout(L - 2);
    clk.mark("perm");
    side.help(s);
    clk.mark("side_help");
    side.join();
    clk.mark("side_join");
    {
        // final V-cycle commit: level-0 solve row -> BILU position
        const int *order0 = L > 1 ? h->lev[0].rows_by_color.p : nullptr;
        h->ep_map.alloc(nb, s);
        k_compose<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, order0, h->bilu.iperm.p, h->ep_map.p);
        CK_LAUNCH();
    }
    if (f32) {
        to_f32(h->pcol0, h->pcol0_32, s);
        to_f32(h->w, h->w32, s);
    }
    for (int l = 0; l < L; l++) {
        Level &Lv = h->lev[l];
        int n = Lv.A.n;
        Lv.x.alloc(n, s);
        Lv.b.alloc(n, s);
        Lv.r.alloc(n, s);
        Lv.s0.alloc(n, s);
        Lv.s1.alloc(n, s);
        if (f32) {
            Lv.x32.alloc(n, s);
            Lv.b32.alloc(n, s);
            Lv.r32.alloc(n, s);
            Lv.s0_32.alloc(n, s);
            Lv.s1_32.alloc(n, s);
        }
        // amg = 1: the GCR work of the coarse corrections on levels 1 .. L-2
        if (o.amg == 1 && l >= 1 && l < L - 1) {
            size_t m = (size_t)std::max(1, o.amli_iters);
            if (f32) {
                Lv.gv32.alloc(m * n, s);
                Lv.gw32.alloc(m * n, s);
            } else {
                Lv.gv.alloc(m * n, s);
                Lv.gw.alloc(m * n, s);
            }
            Lv.gscal.alloc(2 * m + 2, s);
            Lv.gscal.zero();
            // partials of the widest launch: the level's matrix-vector kernel, up to 32 lanes a
            // row in CTAs of at least 128 threads
            Lv.gpart.alloc(2 * ((32 * (size_t)n + 127) / 128 + 1184), s);
            Lv.gcnt.alloc(2, s);
            Lv.gcnt.zero();
        }
    }
    coarse_join.finish();
    if (!o.resetup) {   // the coarse scratch serves only the numeric refresh from here on
        h->c_a.release();
        h->c_lu.release();
        h->c_piv.release();
    }
    choose_tail(h);
    // Kernels that meet a zero or non-finite pivot (an AMG level's diagonal,
    // the coarsest matrix, a BILU(0) block) record CPR_ERR_SINGULAR and go on
    // with a unit stand-in, so the setup runs to completion without host
    // round trips and fails here.
    check_err(h, "zero or non-finite pivot: an AMG level's diagonal, the coarsest matrix or a BILU(0) block");
    clk.mark("layout");
    h->have_B = true;
    h->bilu.pattern = h->pattern_id;
    h->nr_ready = o.resetup != 0;
    h->epoch++;
}

namespace {

// The launches of the numeric refresh on h->stream, with two branches that
// join back before the end: the second stage (BILU(0) and the column-0 copy,
// which need only A) on h->side, the coarse inverse on h->lu_stream.  Every
// launch is a value pass of the full setup on the kept structure, so B comes
// out bit for bit as a full setup on the same pattern builds it.
void record_refresh(cpr_handle *h) {
    cudaStream_t s = h->stream, side = h->side, q = h->lu_stream;
    const cpr_opts &o = h->opt;
    int nb = h->nb, L = (int)h->lev.size();
    bool f32 = o.precond_fp32 != 0;
    int *err = h->err.p;
    CK(cudaEventRecord(h->ev_nr[0], s));
    CK(cudaStreamWaitEvent(side, h->ev_nr[0], 0));
    bilu_values(h, h->bdiag.p, side);
    col0_values(h, side);
    CK(cudaEventRecord(h->ev_nr[1], side));
    // decoupling and A_P, then each level's P, R and Galerkin product
    k_decouple<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->bdiag.p, h->val.p, o.decouple, h->w.p, err);
    CK_LAUNCH();
    if (f32) {
        k_d2f<<<grid_for(3L * nb, kBlock, 148 * 16), kBlock, 0, s>>>(3L * nb, h->w.p, h->w32.p);
        CK_LAUNCH();
    }
    k_pressure_matrix<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->val.p, h->w.p, h->lev[0].A.val.p);
    CK_LAUNCH();
    for (int l = 0; l < L; l++) {
        Level &Lv = h->lev[l];
        int n = Lv.A.n;
        k_check_diag<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, Lv.dpos.p, Lv.A.val.p, nullptr, err);
        CK_LAUNCH();
        if (l == L - 1) break;
        if (o.amg == 0) {   // direct interpolation on the kept strength set and split; R = P^T
            interp_fill(Lv.A, Lv.Srow.p, Lv.Scol.p, Lv.cf.p, Lv.cidx.p, Lv.P, s);
            k_transpose_values<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, Lv.P.rowptr.p, Lv.P.col.p, Lv.P.val.p,
                                                                     Lv.R.rowptr.p, Lv.R.col.p, Lv.R.val.p, err);
            CK_LAUNCH();
        }   // unsmoothed aggregation: P and R are unit, unchanged
        plan_values(Lv.pap, Lv.A, Lv.P, Lv.AP, s);
        plan_values(Lv.prap, Lv.R, Lv.AP, h->lev[l + 1].A, s);
    }
    CK(cudaEventRecord(h->ev_nr[2], s));
    CK(cudaStreamWaitEvent(q, h->ev_nr[2], 0));
    coarse_values(h, h->c_a.p, h->c_lu.p, h->c_piv.p, q);
    CK(cudaEventRecord(h->ev_nr[3], q));
    // the solve's copies in color order and their FP32 shadows
    for (int l = 0; l + 1 < L; l++) {
        Level &Lv = h->lev[l];
        Level &Nx = h->lev[l + 1];
        int n = Lv.A.n;
        perm_fill(Lv.A, Lv.rows_by_color.p, Lv.iperm.p, true, Lv.Ao, s, f32 ? Lv.Aoval32.p : nullptr);
        if (o.amg == 0) {
            bool last = l + 1 == L - 1;   // the coarsest level keeps its natural order
            perm_fill(Lv.P, Lv.rows_by_color.p, last ? nullptr : Nx.iperm.p, false, Lv.Pp, s,
                      f32 ? Lv.Ppval32.p : nullptr);
            perm_fill(Lv.R, last ? nullptr : Nx.rows_by_color.p, Lv.iperm.p, false, Lv.Rp, s,
                      f32 ? Lv.Rpval32.p : nullptr);
        }
        k_perm_diag<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, Lv.rows_by_color.p, Lv.dpos.p, Lv.A.val.p,
                                                          Lv.diag.p, Lv.dinv.p,
                                                          f32 ? Lv.diag32.p : nullptr, f32 ? Lv.dinv32.p : nullptr);
        CK_LAUNCH();
    }
    CK(cudaStreamWaitEvent(s, h->ev_nr[1], 0));
    CK(cudaStreamWaitEvent(s, h->ev_nr[3], 0));
}

}  // namespace

// Alg. 3's rebuild of B with resetup = 1 and an unchanged pattern: every
// value of B recomputed from the current A into the buffers of the last full
// setup, whose discrete structure (levels, strength sets, C/F splits or
// aggregates, colorings, BILU(0) ordering, every pattern) is kept.  The
// launches are captured once into a CUDA graph and replayed on every later
// refresh; no buffer moves, so the Arnoldi step graphs stay valid.
void numeric_refresh(cpr_handle *h) {
    Nvtx nv("numeric refresh");
    cudaStream_t s = h->stream;
    if (!h->nr_ready || !h->side || !h->lu_stream) fail(CPR_ERR_INVALID, "numeric refresh without a kept setup");
    if (!h->nr_exec) {
        // the Galerkin products' lists, once per kept structure
        for (int l = 0; l + 1 < (int)h->lev.size(); l++) {
            Level &Lv = h->lev[l];
            plan_product(Lv.A, Lv.P, Lv.AP, Lv.pap, h->err.p, s);
            plan_product(Lv.R, Lv.AP, h->lev[l + 1].A, Lv.prap, h->err.p, s);
        }
        check_err(h, "numeric resetup: the kept Galerkin patterns do not fit");
        for (auto &e : h->ev_nr)
            if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        lu_smem_attr();
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        set_capturing(true);
        try {
            record_refresh(h);
        } catch (...) {
            set_capturing(false);
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        set_capturing(false);
        CK(cudaStreamEndCapture(s, &g));
        h->nr_graph = g;
        h->nr_kernels = graph_kernel_nodes(g);
        CK(cudaGraphInstantiate(&h->nr_exec, g, 0));
    }
    CK(cudaGraphLaunch(h->nr_exec, s));
    count_launches(h->nr_kernels);
    int e = read_int(h->err.p, s);
    if (e != 0) {
        CK(cudaMemsetAsync(h->err.p, 0, sizeof(int), s));
        free_preconditioner(h);   // B matches no A now: the next update sets up afresh
        fail(e, e == CPR_ERR_SINGULAR
                    ? "zero or non-finite pivot in the numeric resetup: a decoupling block, an AMG level's "
                      "diagonal, the coarsest matrix or a BILU(0) block"
                    : "numeric resetup: A's pattern is not the one B was set up for");
    }
}

}  // namespace cpr
