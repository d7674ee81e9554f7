// Solve phase: one application of the CPR preconditioner B (Alg. 1 from x = 0,
// Eq. 3.1) and the flexible GMRES(m) outer loop of Alg. 2.
//
// Kernels are templated on the preconditioner's value type T (double, or
// float in FP32-preconditioner mode: FP32 storage and accumulation inside B).
// The outer operator, the Arnoldi process (CGS), the Givens rotations and the
// true residual always run in FP64.  Every step is a sparse, bandwidth-bound
// sweep: no tensor cores.  Kernels that belong to one Arnoldi step read the
// step index j and a "done" flag from device memory, so a step never needs a
// host round trip and whole steps can be replayed as a graph.
#include <algorithm>
#include <cmath>

#include "cpr_internal.cuh"
#include <atomic>

#include "sweeps.cuh"
#include "tail.cuh"

namespace cpr {

namespace {

constexpr int kBlock = 256;
constexpr int kRedBlocks = 1184;  // 8 CTAs of 256 threads per SM on 148 SMs
constexpr int kDotGroup = 8;      // vectors per register group in the batched dot kernel
constexpr int kCgsBlocks = 296;   // CGS update: 2 CTAs of 256 threads per SM on 148 SMs (102 registers)
constexpr int kCgsDotBlocks = 444; // CGS dots: 3 CTAs per SM (80 registers), more loads in flight
constexpr int kCgsGroup = 16;     // basis vectors per pass of the CGS dot kernel

// Layout of the device scalar block (doubles) for restart length m.
struct ScalLayout {
    int m;
    __host__ __device__ int H(int i, int j) const { return i * m + j; }   // (m+1) x m
    __host__ __device__ int cs() const { return (m + 1) * m; }
    __host__ __device__ int sn() const { return cs() + m; }
    __host__ __device__ int g() const { return sn() + m; }                 // m+1
    __host__ __device__ int y() const { return g() + m + 1; }              // m
    __host__ __device__ int hcol() const { return y() + m; }               // m+1
    __host__ __device__ int norm0() const { return hcol() + m + 1; }
    __host__ __device__ int rnorm() const { return norm0() + 1; }
    __host__ __device__ int inv_hn() const { return norm0() + 2; }
    __host__ __device__ int rtol() const { return norm0() + 3; }
    __host__ __device__ int est() const { return norm0() + 4; }
    __host__ __device__ int size() const { return norm0() + 5; }
};
// Device ints: [0] step j, [1] done, [2] steps in this cycle, [3] breakdown.
enum { I_J = 0, I_DONE = 1, I_K = 2, I_BREAK = 3, I_ZERO = 4, I_CNT_DOT = 5, I_CNT_UPD = 6, I_SEQ = 7, I_COUNT = 8 };


constexpr int kPre = 4;   // row entries per lane loaded before the dependency wait

// The first kPre entries of a lane's share of row i (entries e0+lane, +G, ...).
template <class T, int G>
struct RowPre {
    int e0 = 0, e1 = 0;
    int c[kPre];
    T v[kPre];
    __device__ __forceinline__ void load(const int *__restrict__ rowptr, const int *__restrict__ col,
                                         const T *__restrict__ val, int i, int lane, bool active) {
        if (active) {
            e0 = rowptr[i];
            e1 = rowptr[i + 1];
        }
#pragma unroll
        for (int u = 0; u < kPre; u++) {
            int p = e0 + lane + u * G;
            bool in = p < e1;
            c[u] = in ? col[p] : 0;
            v[u] = in ? val[p] : (T)0;
        }
    }
    // sum over the lane's entries in ascending order of v_p * xv(col_p)
    template <class XV>
    __device__ __forceinline__ T dot(const int *__restrict__ col, const T *__restrict__ val, int lane,
                                     XV xv) const {
        T s = 0;
#pragma unroll
        for (int u = 0; u < kPre; u++)
            if (e0 + lane + u * G < e1) s += v[u] * xv(c[u]);
#pragma unroll 4
        for (int p = e0 + lane + kPre * G; p < e1; p += G) s += val[p] * xv(col[p]);
        return s;
    }
};

// --------------------------------------------------------------- BSR SpMV

// y = A x, or y = b - A x.  G lanes per block row; each lane takes whole 3x3
// blocks (blocks lane, lane+G, ...) and accumulates its three row sums with
// one FMA per stored value -- B300's FP64 rate, not its bandwidth, bounds
// this kernel, so no value costs more than one FP64 instruction.  G = 1 (one
// thread per block row, no cross-lane FP64 additions at all) measured fastest
// on B300 at 128x128x32: 119 us against 135 (G = 2), 137 (G = 4), 152 (G = 8).
template <int G>
__global__ void k_bsr3_spmv(int nb, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ x_base,
                            long xld, const int *jptr, const double *__restrict__ b,
                            double *__restrict__ y, const int *done) {
    if (done && *done) return;
    const double *x = x_base + (size_t)step_of(jptr) * xld;
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int row = (int)(tid / G), lane = (int)(tid % G);
    bool active = row < nb;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (active) {
        int e = rowptr[row + 1];
        for (int p = rowptr[row] + lane; p < e; p += G) {
            const double *v = val + 9 * (size_t)p;
            const double *xj = x + 3 * (size_t)col[p];
            double x0 = xj[0], x1 = xj[1], x2 = xj[2];
            a0 = fma(v[0], x0, a0);
            a0 = fma(v[1], x1, a0);
            a0 = fma(v[2], x2, a0);
            a1 = fma(v[3], x0, a1);
            a1 = fma(v[4], x1, a1);
            a1 = fma(v[5], x2, a1);
            a2 = fma(v[6], x0, a2);
            a2 = fma(v[7], x1, a2);
            a2 = fma(v[8], x2, a2);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o, G);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o, G);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o, G);
    }
    if (active && lane == 0) {
        size_t q = 3 * (size_t)row;
        if (b) {
            y[q] = b[q] - a0;
            y[q + 1] = b[q + 1] - a1;
            y[q + 2] = b[q + 2] - a2;
        } else {
            y[q] = a0;
            y[q + 1] = a1;
            y[q + 2] = a2;
        }
    }
}

// --------------------------------------------------- restriction / prolongation

// r_P = Pi_P^T v with decoupling weights: r_P[t] = w_i . v_i for block row
// i = order[t] (order: level 0's color order, nullptr = identity); v = v_base + j*ld.
template <class T>
__global__ void k_restrict(int nb, const int *order, const double *v_base, long ld, const int *jptr,
                           const T *w, T *rp, const int *done) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = t < nb;
    int i = 0;
    T w0 = 0, w1 = 0, w2 = 0;
    if (active) {
        i = order ? order[t] : t;
        w0 = w[3 * i];
        w1 = w[3 * i + 1];
        w2 = w[3 * i + 2];
    }
    pdl_wait();
    pdl_trigger();
    if (!active || (done && *done)) return;
    const double *v = v_base + (size_t)step_of(jptr) * ld + 3 * (size_t)i;
    rp[t] = (w0 * (T)v[0] + w1 * (T)v[1]) + w2 * (T)v[2];
}

// k_restrict fused with level 0's first pre-smoothing color (from x = 0): the
// rows of color 0, [c0, c1), get r_P / a_ii in the staging vector sc, every
// other row of x is zeroed.
template <class T>
__global__ void k_restrict_first(int nb, const int *order, const double *v_base, long ld, const int *jptr,
                                 const T *w, T *rp, const T *__restrict__ dinv, T *x, T *sc, int c0, int c1,
                                 const int *done) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = t < nb;
    int i = 0;
    T w0 = 0, w1 = 0, w2 = 0;
    bool mine = active && t >= c0 && t < c1;
    T di = mine ? dinv[t] : (T)0;
    if (active) {
        i = order ? order[t] : t;
        w0 = w[3 * i];
        w1 = w[3 * i + 1];
        w2 = w[3 * i + 2];
    }
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    if (!active) return;
    const double *v = v_base + (size_t)step_of(jptr) * ld + 3 * (size_t)i;
    T r = (w0 * (T)v[0] + w1 * (T)v[1]) + w2 * (T)v[2];
    if (dn) return;
    rp[t] = r;
    if (mine) sc[t] = r * di;
    else x[t] = (T)0;
}

// Second residual of Alg. 1: r = v - A z with z = Pi_P e_P, so only column 0 of
// every block (the frozen copy c0, 3 values per block) takes part.  Rows and
// columns are BILU positions (position t is natural block row border[t]); r
// leaves in positions.  G lanes per block row, whole blocks per lane.
template <class T, int G>
__global__ void k_prolong_resid(int nb, const int *__restrict__ rowptr, const int *__restrict__ col,
                                const T *__restrict__ c0, const T *__restrict__ ep, const int *__restrict__ border,
                                const double *v_base, long ld, const int *jptr, T *__restrict__ r,
                                const int *done) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int row = (int)(tid / G), lane = (int)(tid % G);
    bool active = row < nb;
    int e0 = 0, e1 = 0, brow = 0;
    int cj[kPre];
    T cv[kPre][3];
    if (active) {
        e0 = rowptr[row];
        e1 = rowptr[row + 1];
        brow = border[row];
    }
#pragma unroll
    for (int u = 0; u < kPre; u++) {
        int p = e0 + lane + u * G;
        bool in = p < e1;
        cj[u] = in ? col[p] : 0;
        cv[u][0] = in ? c0[3 * (size_t)p] : (T)0;
        cv[u][1] = in ? c0[3 * (size_t)p + 1] : (T)0;
        cv[u][2] = in ? c0[3 * (size_t)p + 2] : (T)0;
    }
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    // v's three entries of this row are loaded with the gathers, not after them
    bool lead = active && lane == 0;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (lead) {
        const double *v = v_base + (size_t)step_of(jptr) * ld + 3 * (size_t)brow;
        v0 = v[0];
        v1 = v[1];
        v2 = v[2];
    }
    T a0 = 0, a1 = 0, a2 = 0;
    if (active) {
#pragma unroll
        for (int u = 0; u < kPre; u++)
            if (e0 + lane + u * G < e1) {
                T ej = ep[cj[u]];
                a0 = fma(cv[u][0], ej, a0);
                a1 = fma(cv[u][1], ej, a1);
                a2 = fma(cv[u][2], ej, a2);
            }
        for (int p = e0 + lane + kPre * G; p < e1; p += G) {
            T ej = ep[col[p]];
            const T *c = c0 + 3 * (size_t)p;
            a0 = fma(c[0], ej, a0);
            a1 = fma(c[1], ej, a1);
            a2 = fma(c[2], ej, a2);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o, G);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o, G);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o, G);
    }
    if (dn) return;
    if (lead) {
        r[3 * (size_t)row] = (T)v0 - a0;
        r[3 * (size_t)row + 1] = (T)v1 - a1;
        r[3 * (size_t)row + 2] = (T)v2 - a2;
    }
}

// The same product on the sliced-ELL copy: one warp per slice of 32 block
// rows, lane = row.  A row's blocks are taken in the same order with the same
// FMA sequence as k_bsr3_spmv<1>, so the result is bit-identical; the value
// loads of a warp are 256 contiguous bytes per block entry.
__global__ void __launch_bounds__(256) k_sell_spmv(int nslices, int nb, const int *__restrict__ off,
                                                   const int *__restrict__ col, const double *__restrict__ val,
                                                   const double *__restrict__ x_base, long xld, const int *jptr,
                                                   const double *__restrict__ b, double *__restrict__ y,
                                                   const int *done) {
    pdl_wait();
    if (done && *done) return;
    int slice = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (slice >= nslices) return;
    const double *x = x_base + (size_t)step_of(jptr) * xld;
    int row = slice * 32 + lane;
    int k0 = off[slice], k1 = off[slice + 1];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = k0; k < k1; k++) {
        int c = col[(size_t)k * 32 + lane];
        if (c < 0) continue;
        const double *v = val + (size_t)k * 288 + lane;
        const double *xj = x + 3 * (size_t)c;
        double x0 = xj[0], x1 = xj[1], x2 = xj[2];
        a0 = fma(v[0], x0, a0);
        a0 = fma(v[32], x1, a0);
        a0 = fma(v[64], x2, a0);
        a1 = fma(v[96], x0, a1);
        a1 = fma(v[128], x1, a1);
        a1 = fma(v[160], x2, a1);
        a2 = fma(v[192], x0, a2);
        a2 = fma(v[224], x1, a2);
        a2 = fma(v[256], x2, a2);
    }
    pdl_trigger();
    if (row < nb) {
        size_t q = 3 * (size_t)row;
        if (b) {
            y[q] = b[q] - a0;
            y[q + 1] = b[q + 1] - a1;
            y[q + 2] = b[q + 2] - a2;
        } else {
            y[q] = a0;
            y[q + 1] = a1;
            y[q + 2] = a2;
        }
    }
}

// Sliced-ELL build: slot count per slice (its longest row), then each block's
// column in its slot, then the values.
__global__ void k_sell_width(int nb, int nslices, const int *rowptr, int *width) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int w = 0;
    for (int i = s * 32; i < min(nb, s * 32 + 32); i++) w = max(w, rowptr[i + 1] - rowptr[i]);
    width[s] = w;
}

__global__ void k_sell_pattern(int nb, const int *rowptr, const int *col, const int *off, int *scol) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int s = i >> 5, lane = i & 31;
    int slot = off[s];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++, slot++) scol[(size_t)slot * 32 + lane] = col[p];
}

// The values, one CTA per slice, in output order: element t of the slice's
// slots is (slot k, entry e, lane l) with t = 288 k + 32 e + l, so a warp
// writes 32 consecutive doubles, while its reads stay inside the slice's own
// contiguous run of blocks (rows 32 s .. 32 s + 31), which L1 holds.  Padding
// slots are not written: the SpMV skips them by their column (-1).
__global__ void __launch_bounds__(256) k_sell_values(int nb, const int *rowptr, const int *off,
                                                     const double *val, double *sval) {
    int s = blockIdx.x, r0 = s * 32;
    int w = off[s + 1] - off[s];
    double *out = sval + (size_t)off[s] * 288;
    for (int t = threadIdx.x; t < w * 288; t += blockDim.x) {
        int k = t / 288, rem = t - k * 288, e = rem >> 5, r = r0 + (rem & 31);
        if (r >= nb) continue;
        int p = rowptr[r] + k;
        if (p < rowptr[r + 1]) out[t] = val[9 * (size_t)p + e];
    }
}

// ------------------------------------------------------ multi-color GS (Alg. 6)
//
// Levels are renumbered so that each color is a contiguous row range.  A
// color's rows relax Jacobi-style: their new values go to a staging buffer
// (s0/s1, alternating), every x_j is read as of the start of the color, and the
// next kernel commits the staged range into x while reading that range from
// the staging buffer ("pending" range [p0, p1)).  G lanes share a row.


template <class T>
__device__ __forceinline__ T xval(const T *x, const T *sp, int p0, int p1, int j) {
    return (j >= p0 && j < p1) ? sp[j] : x[j];
}

// First color of a sweep that starts from x = 0: the staged rows get b/a_ii,
// every other row of x is zeroed.
template <class T>
__global__ void k_smooth_first(int n, int c0, int c1, const T *b, const T *dinv, T *x, T *sc,
                               const int *done) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool mine = t >= c0 && t < c1;
    T di = mine ? dinv[t] : (T)0;
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    T bt = mine && t < n ? b[t] : (T)0;
    if (t >= n || dn) return;
    if (mine) sc[t] = bt * di;
    else x[t] = (T)0;
}

// Relax rows [c0, c1) into sc; commit the pending range [p0, p1) of sp into x.
template <class T, int G>
__global__ void k_smooth_color(int c0, int c1, int p0, int p1, const int *__restrict__ rowptr,
                               const int *__restrict__ col, const T *__restrict__ val,
                               const T *b, const T *__restrict__ dinv, T *x,
                               const T *sp, T *sc, const int *done) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nthr = (long)gridDim.x * blockDim.x;
    long g = tid / G;
    int lane = (int)(tid % G);
    bool active = g < c1 - c0;
    int i = c0 + (int)g;
    RowPre<T, G> rp;
    rp.load(rowptr, col, val, i, lane, active);
    T di = active ? dinv[i] : (T)0;
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    // every read of the pending range goes to sp, so its commit into x can
    // wait until the row's gathers are issued: a commit store ahead of them
    // would hold them back by a round trip (the compiler cannot reorder loads
    // of x past a store to x)
    long np = p1 - p0;
    T cv = tid < np ? sp[p0 + tid] : (T)0;
    T bi = active && lane == 0 ? b[i] : (T)0;
    T s = 0;
    if (active) s = rp.dot(col, val, lane, [&](int j) { return xval(x, sp, p0, p1, j); });
    s = group_sum(s, G);
    if (dn) return;
    if (active && lane == 0) sc[i] = (bi - s) * di;
    if (tid < np) x[p0 + tid] = cv;
    for (long t = tid + nthr; t < np; t += nthr) x[p0 + t] = sp[p0 + t];
}

// r = b - A x with x's pending range read from sp (and committed into x).
template <class T, int G>
__global__ void k_resid_commit(int n, int p0, int p1, const int *__restrict__ rowptr,
                               const int *__restrict__ col, const T *__restrict__ val,
                               const T *__restrict__ diag, const T *b, T *x, const T *sp,
                               T *r, const int *done) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nthr = (long)gridDim.x * blockDim.x;
    long g = tid / G;
    int lane = (int)(tid % G);
    bool active = g < n;
    int i = (int)g;
    RowPre<T, G> rp;
    rp.load(rowptr, col, val, i, lane, active);
    T dg = active ? diag[i] : (T)0;
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    // the row's own b_i and x_i are loaded with its gathers, not after them
    bool lead = active && lane == 0;
    T bi = lead ? b[i] : (T)0;
    T xi = lead ? xval(x, sp, p0, p1, i) : (T)0;
    T s = 0;
    if (active) s = rp.dot(col, val, lane, [&](int j) { return xval(x, sp, p0, p1, j); });
    s = group_sum(s, G);
    if (dn) return;
    if (lead) r[i] = bi - s - dg * xi;
    // commit after every read of this kernel's own rows is done is not
    // guaranteed across CTAs, so readers above take the pending range from sp
    for (long t = tid; t < p1 - p0; t += nthr) x[p0 + t] = sp[p0 + t];
}

// y = M x (R: restriction) or y += M x (P: prolongation), with x's pending
// range [p0, p1) read from sp.
template <class T, int G>
__global__ void k_transfer(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                           const T *__restrict__ val, const T *x, const T *sp, int p0, int p1, T *y,
                           bool add, const int *done) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long g = tid / G;
    int lane = (int)(tid % G);
    bool active = g < n;
    int i = (int)g;
    RowPre<T, G> rp;
    rp.load(rowptr, col, val, i, lane, active);
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    bool lead = active && lane == 0;
    T yi = lead && add ? y[i] : (T)0;   // loaded with the gathers
    T s = 0;
    if (active) s = rp.dot(col, val, lane, [&](int j) { return xval(x, sp, p0, p1, j); });
    s = group_sum(s, G);
    if (dn) return;
    if (lead) y[i] = add ? yi + s : s;
}

// Restriction fused with the first pre-smoothing color of the coarser level
// (k_transfer with add = false, then k_smooth_first's work for row i): b_C =
// R r, and from x_C = 0 the rows of color 0, [c0, c1), get b_C / a_ii in the
// staging vector sc while every other row of x_C is zeroed.
template <class T, int G>
__global__ void k_transfer_first(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                 const T *__restrict__ val, const T *x, T *y, const T *__restrict__ dinv,
                                 T *xc, T *sc, int c0, int c1, const int *done) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long g = tid / G;
    int lane = (int)(tid % G);
    bool active = g < n;
    int i = (int)g;
    RowPre<T, G> rp;
    rp.load(rowptr, col, val, i, lane, active);
    bool mine = active && i >= c0 && i < c1;
    T di = mine ? dinv[i] : (T)0;
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    T s = 0;
    if (active) s = rp.dot(col, val, lane, [&](int j) { return x[j]; });
    s = group_sum(s, G);
    if (dn) return;
    if (active && lane == 0) {
        y[i] = s;
        if (mine) sc[i] = s * di;
        else xc[i] = (T)0;
    }
}

// Level 0's result renumbered: out[map[t]] = x[t] (pending range from sp).
template <class T>
__global__ void k_commit_natural(int n, const int *order, const T *x, const T *sp, int p0, int p1,
                                 T *out, const int *done) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int o = t < n ? order[t] : 0;
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    T v = t < n ? xval(x, sp, p0, p1, t) : (T)0;
    if (t >= n || dn) return;
    out[o] = v;
}

// Coarsest level: x = A_L^-1 b, one warp per row of the row-major inverse.
template <class T>
__global__ void k_coarse_solve(int n, const double *__restrict__ inv, const T *b, T *x,
                               const int *done) {
    constexpr int kPreC = 8;   // row entries per lane loaded before the wait (n <= 256)
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = (int)(tid >> 5), lane = (int)(tid & 31);
    double a[kPreC];
#pragma unroll
    for (int u = 0; u < kPreC; u++) {
        int j = lane + 32 * u;
        a[u] = (i < n && j < n) ? inv[(size_t)i * n + j] : 0.0;
    }
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    double s = 0.0;
    if (i < n) {
#pragma unroll
        for (int u = 0; u < kPreC; u++)
            if (lane + 32 * u < n) s += a[u] * (double)b[lane + 32 * u];
        for (int j = lane + 32 * kPreC; j < n; j += 32) s += inv[(size_t)i * n + j] * (double)b[j];
    }
    s = group_sum(s, 32);
    if (dn) return;
    if (i < n && lane == 0) x[i] = (T)s;
}


// ------------------------------------------------------------- BILU(0) sweeps
// (k_bilu_fwd / k_bilu_bwd live in sweeps.cuh)




// ------------------------------------------------------------- small kernels

template <class T>
__global__ void k_cast(long n, const double *a, T *b) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        b[i] = (T)a[i];
}

// y[t] = (T) x[order[t]] (order == nullptr: identity).
template <class T>
__global__ void k_gather_cast(int n, const int *order, const double *x, T *y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) y[t] = (T)x[order ? order[t] : t];
}

// x[i] = (double) y[map[i]] (natural i from positions).
template <class T>
__global__ void k_gather_widen(int n, const int *map, const T *y, double *x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (double)y[map[i]];
}

// y[t] = (T) r[order[t]] for the 3 values of block row t.
template <class T>
__global__ void k_gather3(int nb, const int *order, const double *r, T *y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const double *src = r + 3 * (size_t)order[t];
    y[3 * (size_t)t] = (T)src[0];
    y[3 * (size_t)t + 1] = (T)src[1];
    y[3 * (size_t)t + 2] = (T)src[2];
}

template <class T>
__global__ void k_widen(long n, const T *a, double *b) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

template <class T>
__global__ void k_zero(long n, T *a, const int *done) {
    if (done && *done) return;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        a[i] = 0;
}

__global__ void k_has_nonfinite_b(long n, const double *a, int *flag) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) atomicExch(flag, 1);
}

// ------------------------------------------------------------ Krylov kernels

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of v into out (thread 0), deterministic order.
__device__ double block_sum(double v) {
    __shared__ double ws[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += ws[w];
    return s;
}

// Partial sums of a.b per block: part[blockIdx.x].
__global__ void k_dot_partial(long n, const double *a, const double *b, double *part) {
    double s = 0.0;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
        s += a[q] * b[q];
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Last-block-done: returns true in the one block that arrives last, after
// every block's partials are visible (the partial writes are fenced first).
__device__ bool arrive_last(int *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1) == (int)gridDim.x - 1;
    __syncthreads();
    return last;
}

// ------------------------------------------- nonlinear AMLI-cycle (amg = 1)
//
// The coarse correction of Sec. 6's AMLI-cycle on level k: amli_iters steps
// of flexible GCR on A_k e = r from e = 0, each preconditioned by the cycle of
// level k.  Step t: v_t = cycle(res), w_t = A_k v_t, w_t and v_t made
// orthogonal to the earlier w_u one u at a time (beta_u = (w_t, w_u) /
// (w_u, w_u)), alpha_t = (w_t, res) / (w_t, w_t), e += alpha_t v_t,
// res -= alpha_t w_t; a step with (w_t, w_t) = 0 ends the correction.  The
// vectors are the preconditioner's type T; dot products accumulate in FP64 as
// per-block partials that the last block sums in a fixed order, so the
// scalars are deterministic.  Device scalars of a level (gscal): [0, m) the
// (w_u, w_u), [m, 2m) the beta_u, 2m alpha, 2m+1 the stop flag.

struct AmliScal {
    int m;
    __device__ int ww(int u) const { return u; }
    __device__ int beta(int u) const { return m + u; }
    __device__ int alpha() const { return 2 * m; }
    __device__ int stop() const { return 2 * m + 1; }
};

// Block sums of (a, b) into part[2 blk], part[2 blk + 1]; the block that
// arrives last gets the totals (fixed order), else returns false.
__device__ bool amli_reduce(double a, double b, double *part, int *counter, double &sa, double &sb) {
    a = block_sum(a);
    __syncthreads();
    b = block_sum(b);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (!arrive_last(counter) || threadIdx.x >= 32) return false;
    double ta = 0.0, tb = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) {
        ta += __ldcg(part + 2 * k);
        tb += __ldcg(part + 2 * k + 1);
    }
    ta = warp_sum(ta);
    tb = warp_sum(tb);
    if (threadIdx.x == 0) *counter = 0;
    sa = ta;
    sb = tb;
    return threadIdx.x == 0;
}

// w_t = A v_t with v's pending range [p0, p1) read from sp and committed into
// v.  t = 0: the partials of (w, w) and (w, res) give ww_0 and alpha (or the
// stop flag); t > 0: the partials of (w, w_0) give beta_0.
template <class T, int G>
__global__ void k_amli_mv(int n, int p0, int p1, const int *__restrict__ rowptr, const int *__restrict__ col,
                          const T *__restrict__ val, const T *__restrict__ diag, T *v, const T *sp, T *w,
                          const T *y, int t, double *sc, int m, double *part, int *counter, const int *done) {
    AmliScal L{m};
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nthr = (long)gridDim.x * blockDim.x;
    long g = tid / G;
    int lane = (int)(tid % G);
    bool active = g < n;
    int i = (int)g;
    RowPre<T, G> rp;
    rp.load(rowptr, col, val, i, lane, active);
    T dg = active ? diag[i] : (T)0;
    pdl_wait();
    pdl_trigger();
    if (done && *done) return;
    T s = 0;
    if (active) s = rp.dot(col, val, lane, [&](int j) { return xval(v, sp, p0, p1, j); });
    s = group_sum(s, G);
    double da = 0.0, db = 0.0;
    if (active && lane == 0) {
        T wi = s + dg * xval(v, sp, p0, p1, i);
        w[i] = wi;
        da = t == 0 ? (double)wi * (double)wi : 0.0;
        db = (double)wi * (double)y[i];
    }
    for (long q = tid; q < p1 - p0; q += nthr) v[p0 + q] = sp[p0 + q];
    double ta, tb;
    if (!amli_reduce(da, db, part, counter, ta, tb)) return;
    if (t == 0) {
        sc[L.ww(0)] = ta;
        sc[L.stop()] = ta == 0.0 ? 1.0 : 0.0;
        sc[L.alpha()] = ta == 0.0 ? 0.0 : tb / ta;
    } else {
        double den = sc[L.ww(0)];
        sc[L.beta(0)] = den == 0.0 ? 0.0 : tb / den;
    }
}

// w -= beta_u w_u, v -= beta_u v_u; then the partials of (w, w_{u+1}) give
// beta_{u+1} (u + 1 < t), or those of (w, w) and (w, res) give ww_t and alpha
// (u + 1 == t).
template <class T>
__global__ void k_amli_orth(int n, T *w, T *v, const T *wu, const T *vu, const T *y, int u, int t, double *sc, int m,
                            double *part, int *counter, const int *done) {
    pdl_wait();   // everything below reads what earlier kernels wrote
    pdl_trigger();
    if (done && *done) return;
    AmliScal L{m};
    T beta = (T)sc[L.beta(u)];
    bool last = u + 1 == t;
    double da = 0.0, db = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        T wi = w[i] - beta * wu[i];
        w[i] = wi;
        v[i] = v[i] - beta * vu[i];
        if (last) da += (double)wi * (double)wi;
        db += (double)wi * (double)y[i];
    }
    double ta, tb;
    if (!amli_reduce(da, db, part, counter, ta, tb)) return;
    if (last) {
        sc[L.ww(t)] = ta;
        bool stop = sc[L.stop()] != 0.0 || ta == 0.0;
        sc[L.stop()] = stop ? 1.0 : 0.0;
        sc[L.alpha()] = ta == 0.0 ? 0.0 : tb / ta;
    } else {
        double den = sc[L.ww(u + 1)];
        sc[L.beta(u + 1)] = den == 0.0 ? 0.0 : tb / den;
    }
}

// e += alpha v, res -= alpha w (t = 0: e = 0 + alpha v); nothing once a step
// has stopped the correction (t = 0: e = 0).
template <class T>
__global__ void k_amli_update(int n, T *e, T *res, const T *v, const T *w, int t, const double *sc, int m,
                              const int *done) {
    pdl_wait();   // everything below reads what earlier kernels wrote
    pdl_trigger();
    if (done && *done) return;
    AmliScal L{m};
    bool stop = sc[L.stop()] != 0.0;
    T alpha = (T)sc[L.alpha()];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (stop) {
            if (t == 0) e[i] = (T)0;
            continue;
        }
        T ei = t == 0 ? (T)0 : e[i];
        e[i] = ei + alpha * v[i];
        res[i] = res[i] - alpha * w[i];
    }
}

// Transpose-reduction of 16 per-lane partials over a warp: four halving steps
// in which each lane keeps one half of its vectors and adds its partner's copy
// of that half, then one plain step.  Afterwards lanes L and L^1 both hold the
// warp's sum for vector (L >> 1) & 15.  16 additions per lane instead of the
// 80 of sixteen butterfly sums; FP64 additions are scarce on B300.
__device__ __forceinline__ double warp_transpose_sum16(double (&a)[16], int lane) {
    const unsigned full = 0xffffffffu;
    bool up = lane & 16;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        double keep = up ? a[k + 8] : a[k], send = up ? a[k] : a[k + 8];
        a[k] = keep + __shfl_xor_sync(full, send, 16);
    }
    up = lane & 8;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double keep = up ? a[k + 4] : a[k], send = up ? a[k] : a[k + 4];
        a[k] = keep + __shfl_xor_sync(full, send, 8);
    }
    up = lane & 4;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        double keep = up ? a[k + 2] : a[k], send = up ? a[k] : a[k + 2];
        a[k] = keep + __shfl_xor_sync(full, send, 4);
    }
    up = lane & 2;
    {
        double keep = up ? a[1] : a[0], send = up ? a[0] : a[1];
        a[0] = keep + __shfl_xor_sync(full, send, 2);
    }
    return a[0] + __shfl_xor_sync(full, a[0], 1);
}

// CGS dots of Alg. 2, h_ij = (w, v_i) for i = 0..j, sixteen basis vectors per
// pass over w: per-block partials (warp transpose-sums, then warps summed in
// order), then the last block sums each column over the blocks in a fixed
// order (deterministic).
// acc[k] += sum_q V_{g0+k}[q] w[q] for k < NV over this thread's q.
template <int NV>
__device__ __forceinline__ void cgs_dots_pass(long N, const double *__restrict__ Vg, const double *__restrict__ w,
                                              double (&acc)[kCgsGroup]) {
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x) {
        double v[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = Vg[(size_t)k * N + q];
        double wq = w[q];
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] = fma(v[k], wq, acc[k]);
    }
}

#define CPR_NV_DISPATCH(nv, CALL)                                                                   \
    switch (nv) {                                                                                   \
    case 1: { constexpr int NV = 1; CALL; break; }   case 2: { constexpr int NV = 2; CALL; break; }   \
    case 3: { constexpr int NV = 3; CALL; break; }   case 4: { constexpr int NV = 4; CALL; break; }   \
    case 5: { constexpr int NV = 5; CALL; break; }   case 6: { constexpr int NV = 6; CALL; break; }   \
    case 7: { constexpr int NV = 7; CALL; break; }   case 8: { constexpr int NV = 8; CALL; break; }   \
    case 9: { constexpr int NV = 9; CALL; break; }   case 10: { constexpr int NV = 10; CALL; break; } \
    case 11: { constexpr int NV = 11; CALL; break; } case 12: { constexpr int NV = 12; CALL; break; } \
    case 13: { constexpr int NV = 13; CALL; break; } case 14: { constexpr int NV = 14; CALL; break; } \
    case 15: { constexpr int NV = 15; CALL; break; } default: { constexpr int NV = 16; CALL; break; } \
    }

__global__ void __launch_bounds__(kBlock) k_cgs_dots(long N, const double *__restrict__ V,
                                                     const double *__restrict__ w, const int *jptr,
                                                     double *part, int ldp, double *hcol, int *counter,
                                                     const int *done) {
    pdl_wait();
    if (*done) return;
    __shared__ double red[kBlock / 32][kCgsGroup];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nvec = *jptr + 1;
    for (int g0 = 0; g0 < nvec; g0 += kCgsGroup) {
        double acc[kCgsGroup];
#pragma unroll
        for (int k = 0; k < kCgsGroup; k++) acc[k] = 0.0;
        const double *Vg = V + (size_t)g0 * N;
        CPR_NV_DISPATCH(min(nvec - g0, kCgsGroup), (cgs_dots_pass<NV>(N, Vg, w, acc)));
        double v = warp_transpose_sum16(acc, lane);
        if (!(lane & 1)) red[wid][(lane >> 1) & 15] = v;
        __syncthreads();
        if (threadIdx.x < kCgsGroup && g0 + (int)threadIdx.x < nvec) {
            double t = 0.0;
            for (int k = 0; k < kBlock / 32; k++) t += red[k][threadIdx.x];
            part[(size_t)blockIdx.x * ldp + g0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
    pdl_trigger();
    if (!arrive_last(counter)) return;
    for (int i = wid; i < nvec; i += kBlock / 32) {
        double t = 0.0;
#pragma unroll 4
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + (size_t)b * ldp + i);
        t = warp_sum(t);
        if (lane == 0) hcol[i] = t;
    }
    if (threadIdx.x == 0) *counter = 0;
}

// wq -= sum_{k < NV} h[k] V_k[q], h in registers.
template <int NV>
__device__ __forceinline__ double cgs_update_chunk(long N, const double *__restrict__ Vg, const double (&h)[NV],
                                                   long q, double wq) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = Vg[(size_t)k * N + q];
#pragma unroll
    for (int k = 0; k < NV; k++) wq = fma(-h[k], v[k], wq);
    return wq;
}

// w -= V h over this thread's q for NA + NB basis vectors (NB from V_16 on);
// returns the thread's part of ||w||^2.
template <int NA, int NB>
__device__ __forceinline__ double cgs_update_loop(long N, const double *__restrict__ V, const double *h,
                                                  double *__restrict__ w) {
    double ha[NA], hb[NB > 0 ? NB : 1];
#pragma unroll
    for (int k = 0; k < NA; k++) ha[k] = h[k];
#pragma unroll
    for (int k = 0; k < NB; k++) hb[k] = h[kCgsGroup + k];
    double s = 0.0;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x) {
        double wq = w[q];
        wq = cgs_update_chunk<NA>(N, V, ha, q, wq);
        if constexpr (NB > 0)
            wq = cgs_update_chunk<NB>(N, V + (size_t)kCgsGroup * N, reinterpret_cast<const double(&)[NB]>(hb), q, wq);
        w[q] = wq;
        s = fma(wq, wq, s);
    }
    return s;
}

// w -= sum_{i<=j} h_i V_i with per-block partials of ||w||^2; the last block
// sums them (fixed order) and performs the Givens step of column j (Saad's
// form) in shared memory: apply the previous rotations, form the new one,
// update g, estimate |g_{j+1}| / ||r_0|| and take the stop decision of Alg. 2.
__global__ void __launch_bounds__(kBlock) k_cgs_update_givens(long N, const double *__restrict__ V,
                                                              double *__restrict__ w, double *part,
                                                              int *counter, double *sc, int m, int *di) {
    pdl_wait();
    if (di[I_DONE]) return;
    ScalLayout SL{m};
    __shared__ double sh[kMaxRestart + 2], rc[kMaxRestart], rs[kMaxRestart];
    int j = di[I_J];
    int nvec = j + 1;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) sh[i] = sc[SL.hcol() + i];
    __syncthreads();
    double s = 0.0;
    if (nvec <= kCgsGroup) {
        CPR_NV_DISPATCH(nvec, (s = cgs_update_loop<NV, 0>(N, V, sh, w)));
    } else if (nvec <= 2 * kCgsGroup) {
        CPR_NV_DISPATCH(nvec - kCgsGroup, (s = cgs_update_loop<kCgsGroup, NV>(N, V, sh, w)));
    } else {
        for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x) {
            double wq = w[q];
            for (int i = 0; i < nvec; i++) wq = fma(-sh[i], V[(size_t)i * N + q], wq);
            w[q] = wq;
            s = fma(wq, wq, s);
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    pdl_trigger();
    if (!arrive_last(counter)) return;
    if (threadIdx.x >= 32) return;
    int lane = threadIdx.x;
    double hn2 = 0.0;
#pragma unroll 4
    for (int b = lane; b < (int)gridDim.x; b += 32) hn2 += __ldcg(part + b);
    hn2 = warp_sum(hn2);
    for (int i = lane; i < j; i += 32) {
        rc[i] = sc[SL.cs() + i];
        rs[i] = sc[SL.sn() + i];
    }
    __syncwarp();
    double hn = sqrt(hn2);
    if (lane == 0) {
        *counter = 0;
        sh[j + 1] = hn;
        for (int i = 0; i < j; i++) {
            double a = sh[i], c = sh[i + 1];
            sh[i] = rc[i] * a + rs[i] * c;
            sh[i + 1] = -rs[i] * a + rc[i] * c;
        }
        double a = sh[j], c = sh[j + 1];
        double den = sqrt(a * a + c * c);
        double cj = den == 0.0 ? 1.0 : a / den, sj = den == 0.0 ? 0.0 : c / den;
        sc[SL.cs() + j] = cj;
        sc[SL.sn() + j] = sj;
        sh[j] = den;
        sh[j + 1] = 0.0;
        double gj = sc[SL.g() + j];
        double gn = -sj * gj;
        sc[SL.g() + j + 1] = gn;
        sc[SL.g() + j] = cj * gj;
        double est = fabs(gn) / sc[SL.norm0()];
        sc[SL.est()] = est;
        sc[SL.inv_hn()] = hn > 0.0 ? 1.0 / hn : 0.0;
        di[I_K] = j + 1;
        di[I_J] = j + 1;
        bool brk = !isfinite(hn) || !isfinite(est);
        if (brk) di[I_BREAK] = 1;
        if (brk || hn == 0.0 || est < sc[SL.rtol()] || j + 1 >= m) di[I_DONE] = 1;
    }
    __syncwarp();
    for (int i = lane; i <= j + 1; i += 32) sc[SL.H(i, j)] = sh[i];
}

// V_{j+1} = w / h_{j+1,j} (after k_givens advanced the step index to j+1).
// The step's flags (di[0 .. 3]: step index, stop, steps done, breakdown) also
// go to the host: into slot (seq & 1) of two page-locked slots, seq counting
// the steps launched in this cycle, stopped ones included.  Written here, at
// the end of every step graph, they spare a copy between the step graphs.
__global__ void k_next_basis(long N, const double *w, double *V, const double *sc, int m,
                             int *di, int *flags_host) {
    pdl_wait();
    if (flags_host && blockIdx.x == 0 && threadIdx.x == 0) {
        int q = di[I_SEQ];
        int *f = flags_host + 4 * (q & 1);
        for (int k = 0; k < 4; k++) f[k] = di[k];
        __threadfence_system();
        di[I_SEQ] = q + 1;
    }
    if (di[I_DONE]) return;
    ScalLayout L{m};
    double s = sc[L.inv_hn()];
    double *v = V + (size_t)di[I_J] * N;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x)
        v[q] = w[q] * s;
}

// Start of a cycle: beta = sqrt(sum part), V_0 = r / beta, g = beta e_1, j = 0.
// On the first cycle (first != 0) also ||r_0|| = beta.
__global__ void k_cycle_start_scal(const double *part, int nblk, double *sc, int m, int *di,
                                   int first, double rtol) {
    ScalLayout L{m};
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += part[b];
    s = warp_sum(s);
    if (threadIdx.x != 0) return;
    double beta = sqrt(s);
    if (first) {
        sc[L.norm0()] = beta;
        sc[L.rtol()] = rtol;
    }
    sc[L.rnorm()] = beta;
    for (int i = 0; i <= m; i++) sc[L.g() + i] = 0.0;
    sc[L.g()] = beta;
    sc[L.inv_hn()] = beta > 0.0 ? 1.0 / beta : 0.0;
    di[I_J] = 0;
    di[I_K] = 0;
    di[I_BREAK] = isfinite(beta) ? 0 : 1;
    di[I_DONE] = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
    di[I_ZERO] = 0;
    di[I_SEQ] = 0;
}

__global__ void k_scale_into(long N, const double *r, double *v, const double *sc, int m) {
    ScalLayout L{m};
    double s = sc[L.inv_hn()];
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x)
        v[q] = r[q] * s;
}

// y = H_k^-1 g_k (upper triangular back substitution), k = steps of the cycle.
__global__ void k_solve_y(double *sc, int m, const int *di) {
    ScalLayout L{m};
    int k = di[I_K];
    for (int i = k - 1; i >= 0; i--) {
        double s = sc[L.g() + i];
        for (int q = i + 1; q < k; q++) s -= sc[L.H(i, q)] * sc[L.y() + q];
        sc[L.y() + i] = s / sc[L.H(i, i)];
    }
}

// x += sum_{i<k} y_i Z_i.
__global__ void k_update_x(long N, const double *__restrict__ Z, double *x, const double *sc, int m,
                           const int *di) {
    __shared__ double sy[kMaxRestart];
    ScalLayout L{m};
    int k = di[I_K];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sy[i] = sc[L.y() + i];
    __syncthreads();
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x) {
        double s = x[q];
        for (int i = 0; i < k; i++) s += sy[i] * Z[(size_t)i * N + q];
        x[q] = s;
    }
}

// ------------------------------------------------------------ host helpers

template <class T>
struct Vals;
template <>
struct Vals<double> {
    static const double *Ao(const Level &L) { return L.Ao.val.p; }
    static const double *P(const Level &L) { return L.Pp.val.p; }
    static const double *R(const Level &L) { return L.Rp.val.p; }
    static const double *diag(const Level &L) { return L.diag.p; }
    static const double *dinv(const Level &L) { return L.dinv.p; }
    static double *x(Level &L) { return L.x.p; }
    static double *b(Level &L) { return L.b.p; }
    static double *r(Level &L) { return L.r.p; }
    static double *s(Level &L, int k) { return k ? L.s1.p : L.s0.p; }
    static const double *w(const cpr_handle *h) { return h->w.p; }
    static const double *c0(const cpr_handle *h) { return h->pcol0.p; }
    static const double *Lv(const cpr_handle *h) { return h->bilu.Lval.p; }
    static const double *Uv(const cpr_handle *h) { return h->bilu.Uval.p; }
    static const double *Dv(const cpr_handle *h) { return h->bilu.Dinv.p; }
    static double *tmp(cpr_handle *h) { return h->t64a.p; }
    static double *ep(cpr_handle *h) { return h->ep64.p; }
    static double *gv(Level &L) { return L.gv.p; }
    static double *gw(Level &L) { return L.gw.p; }
};
template <>
struct Vals<float> {
    static const float *Ao(const Level &L) { return L.Aoval32.p; }
    static const float *P(const Level &L) { return L.Ppval32.p; }
    static const float *R(const Level &L) { return L.Rpval32.p; }
    static const float *diag(const Level &L) { return L.diag32.p; }
    static const float *dinv(const Level &L) { return L.dinv32.p; }
    static float *x(Level &L) { return L.x32.p; }
    static float *b(Level &L) { return L.b32.p; }
    static float *r(Level &L) { return L.r32.p; }
    static float *s(Level &L, int k) { return k ? L.s1_32.p : L.s0_32.p; }
    static const float *w(const cpr_handle *h) { return h->w32.p; }
    static const float *c0(const cpr_handle *h) { return h->pcol0_32.p; }
    static const float *Lv(const cpr_handle *h) { return h->bilu.Lval32.p; }
    static const float *Uv(const cpr_handle *h) { return h->bilu.Uval32.p; }
    static const float *Dv(const cpr_handle *h) { return h->bilu.Dinv32.p; }
    static float *tmp(cpr_handle *h) { return h->t32a.p; }
    static float *ep(cpr_handle *h) { return h->ep32.p; }
    static float *gv(Level &L) { return L.gv32.p; }
    static float *gw(Level &L) { return L.gw32.p; }
};

// The staged ("pending") range of a level: rows [p0, p1) whose newest values
// are in staging buffer k rather than in x.
struct Pending {
    int p0 = 0, p1 = 0, k = 0;
};

template <int G, class F>
void with_lanes(int g, F f);

#define CPR_LANES_DISPATCH(g, CALL) \
    switch (g) {                    \
    case 1: { constexpr int G = 1; CALL; break; }   \
    case 2: { constexpr int G = 2; CALL; break; }   \
    case 4: { constexpr int G = 4; CALL; break; }   \
    case 8: { constexpr int G = 8; CALL; break; }   \
    case 16: { constexpr int G = 16; CALL; break; } \
    default: { constexpr int G = 32; CALL; break; } \
    }

inline unsigned blocks_for(long threads, int block = kBlock) {
    return (unsigned)std::max<long>(1, (threads + block - 1) / block);
}

// Launch one kernel of the B-application chain: with programmatic dependent
// launch when `pdl` (the kernel's prologue may then overlap its predecessor),
// else in plain stream order.
template <class... KArgs, class... Args>
void launch_pdl(bool pdl, void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
                Args &&...args) {
    if (pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
    } else {
        kern<<<grid, block, 0, s>>>(std::forward<Args>(args)...);
    }
    CK_LAUNCH();
}

template <class... KArgs, class... Args>
void launch_b(const cpr_handle *h, void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
              Args &&...args) {
    launch_pdl(h->opt.pdl != 0, kern, grid, block, s, std::forward<Args>(args)...);
}

// One smoothing sweep over the colors of level L (ascending or descending).
// From zero: the first color writes b/a_ii into staging and zeroes x.
template <class T>
void mcgs_sweep(cpr_handle *h, Level &L, bool descending, bool from_zero, Pending &pd,
                const int *done, bool first_done, const T *b, T *x) {
    cudaStream_t s = h->stream;
    int n = L.A.n;
    for (int t = 0; t < L.ncolors; t++) {
        int c = descending ? L.ncolors - 1 - t : t;
        int c0 = L.color_off[c], c1 = L.color_off[c + 1];
        int k = 1 - pd.k;
        if (from_zero && t == 0 && first_done) {
            // the producer of b already did this color's from-zero work
        } else if (from_zero && t == 0) {
            launch_b(h, k_smooth_first<T>, blocks_for(n, L.bs), L.bs, s, n, c0, c1, b, Vals<T>::dinv(L), x,
                     Vals<T>::s(L, k), done);
        } else {
            long thr = std::max<long>((long)(c1 - c0) * L.gA, pd.p1 - pd.p0);
            bool fine = &L == &h->lev[0];
            if (fine) prof_begin(h, CPR_PROF_SMOOTH0);
            CPR_LANES_DISPATCH(L.gA, (launch_b(h, k_smooth_color<T, G>, blocks_for(thr, L.bs), L.bs, s, c0, c1, pd.p0,
                                               pd.p1, L.Ao.rowptr.p, L.Ao.col.p, Vals<T>::Ao(L), b,
                                               Vals<T>::dinv(L), x, Vals<T>::s(L, pd.k), Vals<T>::s(L, k), done)));
            if (fine) prof_end(h);
        }
        pd = Pending{c0, c1, k};
    }
}

// The cluster tail from level h->tail_top down: one launch of one cluster.
template <class T>
void launch_tail(cpr_handle *h, const int *done) {
    TailArgs<T> a{};
    int L = (int)h->lev.size(), t = h->tail_top;
    a.nlev = L - 1 - t;
    int off = 0;
    for (int q = 0; q < a.nlev; q++) {
        Level &Lv = h->lev[t + q];
        TailLevel<T> &d = a.lev[q];
        d.n = Lv.A.n;
        d.ncolors = Lv.ncolors;
        d.gA = Lv.gA;
        d.gP = Lv.gP;
        d.gR = Lv.gR;
        for (int c = 0; c <= Lv.ncolors; c++) d.color_off[c] = Lv.color_off[c];
        d.arow = Lv.Ao.rowptr.p;
        d.acol = Lv.Ao.col.p;
        d.aval = Vals<T>::Ao(Lv);
        d.diag = Vals<T>::diag(Lv);
        d.dinv = Vals<T>::dinv(Lv);
        d.prow = Lv.Pp.rowptr.p;
        d.pcol = Lv.Pp.col.p;
        d.pval = Vals<T>::P(Lv);
        d.rrow = Lv.Rp.rowptr.p;
        d.rcol = Lv.Rp.col.p;
        d.rval = Vals<T>::R(Lv);
        d.ox = off;
        d.os = off + d.n;
        d.orr = off + 2 * d.n;
        d.ob = off + 3 * d.n;
        off += 4 * d.n;
    }
    a.nc = h->lev.back().A.n;
    a.obc = off;
    a.oxc = off + a.nc;
    off += 2 * a.nc;
    a.cinv = h->cinv.p;
    a.b_top = Vals<T>::b(h->lev[t]);
    a.x_top = Vals<T>::x(h->lev[t]);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kTailCTAs);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = (size_t)off * sizeof(T);
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kTailCTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_tail_vcycle<T>, a, done));
    CK_LAUNCH();
}

// Shared-memory ceiling of both tail kernels, set once per device.
void tail_attr() {
    static std::atomic<unsigned long long> set{0};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    unsigned long long bit = 1ull << (dev & 63);
    if (set.load(std::memory_order_acquire) & bit) return;
    CK(cudaFuncSetAttribute(k_tail_vcycle<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemMax));
    CK(cudaFuncSetAttribute(k_tail_vcycle<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemMax));
    // the replicas are small: leave the rest of the SM's memory to L1, which
    // holds this CTA's rows of the tail matrices (prefetched at kernel start)
    CK(cudaFuncSetAttribute(k_tail_vcycle<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                            cudaSharedmemCarveoutMaxL1));
    CK(cudaFuncSetAttribute(k_tail_vcycle<double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                            cudaSharedmemCarveoutMaxL1));
    set.fetch_or(bit, std::memory_order_release);
}

// V(pre, post) cycle on level l from x_l = 0 (pre-smoothing colors ascending,
// post-smoothing descending).  On return the level's result is x with the
// range `out` still staged.  first_done: the kernel that wrote b_l also did
// the first pre-smoothing color (x_l zeroed, color 0 staged in s1).
template <class T>
void vcycle(cpr_handle *h, int l, Pending &out, const int *done, bool first_done = false) {
    cudaStream_t s = h->stream;
    Level &L = h->lev[l];
    int n = L.A.n;
    if (l == h->tail_top) {   // this level and everything below in one cluster
        launch_tail<T>(h, done);
        out = Pending{};
        return;
    }
    if (l == (int)h->lev.size() - 1) {
        launch_b(h, k_coarse_solve<T>, blocks_for((long)n * 32), kBlock, s, n, h->cinv.p, Vals<T>::b(L),
                 Vals<T>::x(L), done);
        out = Pending{};
        return;
    }
    Pending pd;
    if (h->opt.pre == 0) {
        k_zero<T><<<grid_for(n, kBlock, 148 * 8), kBlock, 0, s>>>(n, Vals<T>::x(L), done);
        CK_LAUNCH();
    }
    for (int k = 0; k < h->opt.pre; k++)
        mcgs_sweep<T>(h, L, false, k == 0, pd, done, first_done && k == 0, Vals<T>::b(L), Vals<T>::x(L));
    long thr = std::max<long>((long)n * L.gA, pd.p1 - pd.p0);
    CPR_LANES_DISPATCH(L.gA, (launch_b(h, k_resid_commit<T, G>, blocks_for(thr, L.bs), L.bs, s, n, pd.p0, pd.p1,
                                       L.Ao.rowptr.p, L.Ao.col.p, Vals<T>::Ao(L), Vals<T>::diag(L), Vals<T>::b(L),
                                       Vals<T>::x(L), Vals<T>::s(L, pd.k), Vals<T>::r(L), done)));
    pd = Pending{};
    Level &C = h->lev[l + 1];
    // C is smoothed from zero by the next kernel unless the cluster tail takes it
    bool fuse = l + 1 < (int)h->lev.size() - 1 && h->opt.pre > 0 && l + 1 != h->tail_top;
    if (fuse) {
        CPR_LANES_DISPATCH(L.gR, (launch_b(h, k_transfer_first<T, G>, blocks_for((long)L.Rp.n * L.gR, L.bs), L.bs, s,
                                           L.Rp.n, L.Rp.rowptr.p, L.Rp.col.p, Vals<T>::R(L), Vals<T>::r(L),
                                           Vals<T>::b(C), Vals<T>::dinv(C), Vals<T>::x(C), Vals<T>::s(C, 1),
                                           C.color_off[0], C.color_off[1], done)));
    } else {
        CPR_LANES_DISPATCH(L.gR, (launch_b(h, k_transfer<T, G>, blocks_for((long)L.Rp.n * L.gR, L.bs), L.bs, s,
                                           L.Rp.n, L.Rp.rowptr.p, L.Rp.col.p, Vals<T>::R(L), Vals<T>::r(L),
                                           Vals<T>::r(L), 0, 0, Vals<T>::b(C), false, done)));
    }
    Pending cp;
    vcycle<T>(h, l + 1, cp, done, fuse);
    CPR_LANES_DISPATCH(L.gP, (launch_b(h, k_transfer<T, G>, blocks_for((long)n * L.gP, L.bs), L.bs, s, n,
                                       L.Pp.rowptr.p, L.Pp.col.p, Vals<T>::P(L), Vals<T>::x(C),
                                       Vals<T>::s(C, cp.k), cp.p0, cp.p1, Vals<T>::x(L), true, done)));
    for (int k = 0; k < h->opt.post; k++) mcgs_sweep<T>(h, L, true, false, pd, done, false, Vals<T>::b(L), Vals<T>::x(L));
    out = pd;
}

// e_P = B_P r_P on level 0: r_P arrives in level 0's b (level 0's color
// order); the result leaves in BILU positions in ep.
template <class T>
void vcycle_top(cpr_handle *h, T *ep, const int *done, bool first_done = false) {
    Level &L0 = h->lev[0];
    Pending pd;
    vcycle<T>(h, 0, pd, done, first_done);
    int n = L0.A.n;
    launch_b(h, k_commit_natural<T>, blocks_for(n), kBlock, h->stream, n, h->ep_map.p, Vals<T>::x(L0),
             Vals<T>::s(L0, pd.k), pd.p0, pd.p1, ep, done);
}

// ------------------------------------------------ the AMLI-cycle (amg = 1)

template <class T>
void amli_coarse(cpr_handle *h, int k, const int *done);

// The nonlinear AMLI-cycle for A_l x = b from x = 0 (Sec. 6's first stage):
// the V-cycle's smoothing and transfers, with the coarse problem solved
// exactly on the coarsest level and by amli_coarse elsewhere.  b and x are
// any vectors of level l (internal numbering); on return x's range `out` is
// still staged.  first_done as for vcycle (level 0 only).
template <class T>
void kcycle(cpr_handle *h, int l, const T *b, T *x, Pending &out, const int *done, bool first_done = false) {
    cudaStream_t s = h->stream;
    Level &L = h->lev[l];
    int n = L.A.n;
    int last = (int)h->lev.size() - 1;
    if (l == last) {
        launch_b(h, k_coarse_solve<T>, blocks_for((long)n * 32), kBlock, s, n, h->cinv.p, b, x, done);
        out = Pending{};
        return;
    }
    Pending pd;
    if (h->opt.pre == 0) {
        k_zero<T><<<grid_for(n, kBlock, 148 * 8), kBlock, 0, s>>>(n, x, done);
        CK_LAUNCH();
    }
    for (int k = 0; k < h->opt.pre; k++) mcgs_sweep<T>(h, L, false, k == 0, pd, done, first_done && k == 0, b, x);
    long thr = std::max<long>((long)n * L.gA, pd.p1 - pd.p0);
    CPR_LANES_DISPATCH(L.gA, (launch_b(h, k_resid_commit<T, G>, blocks_for(thr, L.bs), L.bs, s, n, pd.p0, pd.p1,
                                       L.Ao.rowptr.p, L.Ao.col.p, Vals<T>::Ao(L), Vals<T>::diag(L), b, x,
                                       Vals<T>::s(L, pd.k), Vals<T>::r(L), done)));
    pd = Pending{};
    Level &C = h->lev[l + 1];
    CPR_LANES_DISPATCH(L.gR, (launch_b(h, k_transfer<T, G>, blocks_for((long)L.Rp.n * L.gR, L.bs), L.bs, s, L.Rp.n,
                                       L.Rp.rowptr.p, L.Rp.col.p, Vals<T>::R(L), Vals<T>::r(L), Vals<T>::r(L), 0, 0,
                                       Vals<T>::b(C), false, done)));
    if (l + 1 == last)
        launch_b(h, k_coarse_solve<T>, blocks_for((long)C.A.n * 32), kBlock, s, C.A.n, h->cinv.p, Vals<T>::b(C),
                 Vals<T>::x(C), done);
    else
        amli_coarse<T>(h, l + 1, done);   // e = x(C), fully written
    CPR_LANES_DISPATCH(L.gP, (launch_b(h, k_transfer<T, G>, blocks_for((long)n * L.gP, L.bs), L.bs, s, n,
                                       L.Pp.rowptr.p, L.Pp.col.p, Vals<T>::P(L), Vals<T>::x(C), Vals<T>::s(C, 0), 0,
                                       0, x, true, done)));
    for (int k = 0; k < h->opt.post; k++) mcgs_sweep<T>(h, L, true, false, pd, done, false, b, x);
    out = pd;
}

// The coarse correction on level k (1 <= k < L-1): GCR on A_k e = r with r in
// b(k) (used in place as the residual) and e in x(k); see k_amli_mv.
template <class T>
void amli_coarse(cpr_handle *h, int k, const int *done) {
    cudaStream_t s = h->stream;
    Level &L = h->lev[k];
    int n = L.A.n, m = std::max(1, h->opt.amli_iters);
    T *res = Vals<T>::b(L), *e = Vals<T>::x(L);
    unsigned eb = (unsigned)grid_for(n, kBlock, 148 * 4);
    for (int t = 0; t < m; t++) {
        T *v = Vals<T>::gv(L) + (size_t)t * n, *w = Vals<T>::gw(L) + (size_t)t * n;
        Pending pv;
        kcycle<T>(h, k, res, v, pv, done);
        long thr = std::max<long>((long)n * L.gA, pv.p1 - pv.p0);
        const T *y = t == 0 ? res : Vals<T>::gw(L);
        CPR_LANES_DISPATCH(L.gA, (launch_b(h, k_amli_mv<T, G>, blocks_for(thr, L.bs), L.bs, s, n, pv.p0, pv.p1,
                                           L.Ao.rowptr.p, L.Ao.col.p, Vals<T>::Ao(L), Vals<T>::diag(L), v,
                                           Vals<T>::s(L, pv.k), w, y, t, L.gscal.p, m, L.gpart.p, L.gcnt.p, done)));
        for (int u = 0; u < t; u++) {
            const T *yu = u + 1 == t ? res : Vals<T>::gw(L) + (size_t)(u + 1) * n;
            launch_b(h, k_amli_orth<T>, eb, kBlock, s, n, w, v, Vals<T>::gw(L) + (size_t)u * n,
                     Vals<T>::gv(L) + (size_t)u * n, yu, u, t, L.gscal.p, m, L.gpart.p, L.gcnt.p + 1, done);
        }
        launch_b(h, k_amli_update<T>, eb, kBlock, s, n, e, res, (const T *)v, (const T *)w, t,
                 (const double *)L.gscal.p, m, done);
    }
}

// e_P = B_P r_P with the AMLI-cycle (the counterpart of vcycle_top).
template <class T>
void kcycle_top(cpr_handle *h, T *ep, const int *done, bool first_done = false) {
    Level &L0 = h->lev[0];
    Pending pd;
    kcycle<T>(h, 0, Vals<T>::b(L0), Vals<T>::x(L0), pd, done, first_done);
    int n = L0.A.n;
    launch_b(h, k_commit_natural<T>, blocks_for(n), kBlock, h->stream, n, h->ep_map.p, Vals<T>::x(L0),
             Vals<T>::s(L0, pd.k), pd.p0, pd.p1, ep, done);
}

// B_P: the V-cycle, or the AMLI-cycle when amg = 1.
template <class T>
void pressure_top(cpr_handle *h, T *ep, const int *done, bool first_done = false) {
    if (h->opt.amg == 1) kcycle_top<T>(h, ep, done, first_done);
    else vcycle_top<T>(h, ep, done, first_done);
}

// BILU(0) solve in place on y (forward by ascending colors, backward by
// descending colors); the backward sweep writes out (+ Pi_P e_P when ep).
template <class T>
void bilu_solve(cpr_handle *h, T *y, const T *ep, double *out_base, long ld, const int *jptr,
                const int *done) {
    cudaStream_t s = h->stream;
    Bilu &B = h->bilu;
    // the lowest color has no lower neighbours (L holds lower colors only), so
    // its forward substitution leaves y unchanged and is skipped
    constexpr int G = sizeof(T) == 4 ? kBiluLanesF32 : 1;
    // FP64 sweeps (one thread per block row, 56-72 registers) measured slower
    // with dependent launch on B300 (241 -> 268 us per application at
    // 128x128x32), FP32 sweeps faster (90.6 -> 86.1 us)
    bool pdl = h->opt.pdl && sizeof(T) == 4;
    // the highest non-empty color has no upper neighbours (L and U split by
    // color, and same-colored rows are never adjacent), so its forward and
    // backward steps run as one launch
    int last = B.ncolors - 1;
    while (last > 0 && B.color_off[last + 1] == B.color_off[last]) last--;
    for (int c = 1; c < last; c++) {
        int cnt = B.color_off[c + 1] - B.color_off[c];
        if (!cnt) continue;
        launch_pdl(pdl, k_bilu_fwd<T, G>, grid_for((long)cnt * G, kBlock), kBlock, s, B.color_off[c], cnt,
                   B.Lrowptr.p, B.Lcol.p, Vals<T>::Lv(h), y, done);
    }
    if (last >= 0) {
        int cnt = B.color_off[last + 1] - B.color_off[last];
        if (cnt)
            launch_pdl(pdl, k_bilu_last<T, G>, grid_for((long)cnt * G, kBlock), kBlock, s, B.color_off[last], cnt,
                       B.Lrowptr.p, B.Lcol.p, Vals<T>::Lv(h), Vals<T>::Dv(h), y, ep, B.rows_by_color.p, out_base,
                       ld, jptr, done);
    }
    for (int c = last - 1; c >= 0; c--) {
        int cnt = B.color_off[c + 1] - B.color_off[c];
        if (!cnt) continue;
        launch_pdl(pdl, k_bilu_bwd<T, G>, grid_for((long)cnt * G, kBlock), kBlock, s, B.color_off[c], cnt,
                   B.Urowptr.p, B.Ucol.p, Vals<T>::Uv(h), Vals<T>::Dv(h), y, ep, B.rows_by_color.p, out_base, ld,
                   jptr, done);
    }
}

#ifndef CPR_SPMV_LANES
#define CPR_SPMV_LANES 1
#endif
constexpr int kSpmvLanes = CPR_SPMV_LANES;  // outer BSR SpMV (lanes per block row)
// second residual: lanes per block row (FP32 2, FP64 1: one FP64 instruction
// costs its issue slot whatever its active lanes; FP64 solve at 128x128x32
// 32.54 -> 32.23 ms with 1 lane, FP32 22.31 -> 22.39 ms)
template <class T>
constexpr int kResidLanes = sizeof(T) == 4 ? 2 : 1;

template <class T>
void apply_B_t(cpr_handle *h, const double *v_base, long v_ld, const int *jptr, double *z_base,
               long z_ld, const int *done) {
    cudaStream_t s = h->stream;
    int nb = h->nb;
    Level &L0 = h->lev[0];
    const int *order0 = h->lev.size() > 1 ? L0.rows_by_color.p : nullptr;
    Nvtx nv("B application");
    // r_P = Pi_P^T v
    // level 0 is smoothed from zero unless it is the coarsest level
    bool fuse = h->lev.size() > 1 && h->opt.pre > 0;
    if (fuse)
        launch_b(h, k_restrict_first<T>, grid_for(nb, kBlock), kBlock, s, nb, order0, v_base, v_ld, jptr,
                 Vals<T>::w(h), Vals<T>::b(L0), Vals<T>::dinv(L0), Vals<T>::x(L0), Vals<T>::s(L0, 1),
                 L0.color_off[0], L0.color_off[1], done);
    else
        launch_b(h, k_restrict<T>, grid_for(nb, kBlock), kBlock, s, nb, order0, v_base, v_ld, jptr, Vals<T>::w(h),
                 Vals<T>::b(L0), done);
    // e_P = B_P r_P (BILU positions)
    prof_begin(h, CPR_PROF_VCYCLE);
    {
        Nvtx r("pressure cycle");
        pressure_top<T>(h, Vals<T>::ep(h), done, fuse);
    }
    prof_end(h);
    // r = v - A Pi_P e_P
    long threads = (long)nb * kResidLanes<T>;
    prof_begin(h, CPR_PROF_RESID2);
    launch_b(h, k_prolong_resid<T, kResidLanes<T>>, (unsigned)((threads + kBlock - 1) / kBlock), kBlock, s, nb,
             h->c0rowptr.p, h->c0col.p, Vals<T>::c0(h), Vals<T>::ep(h), h->bilu.rows_by_color.p, v_base, v_ld,
             jptr, Vals<T>::tmp(h), done);
    prof_end(h);
    // z = Pi_P e_P + (LU)^-1 r
    prof_begin(h, CPR_PROF_BILU);
    {
        Nvtx r("BILU(0) sweeps");
        bilu_solve<T>(h, Vals<T>::tmp(h), Vals<T>::ep(h), z_base, z_ld, jptr, done);
    }
    prof_end(h);
}

void spmv_launch(int nb, const int *rowptr, const int *col, const double *val, const double *x,
                 long xld, const int *jptr, const double *b, double *y, cudaStream_t s,
                 const int *done) {
    long threads = (long)nb * kSpmvLanes;
    k_bsr3_spmv<kSpmvLanes><<<(unsigned)((threads + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        nb, rowptr, col, val, x, xld, jptr, b, y, done);
    CK_LAUNCH();
}

// y = A x (or b - A x) with the handle's outer operator: the sliced-ELL copy
// when it is current, else the BSR arrays.
void spmv_h(cpr_handle *h, const double *x, long xld, const int *jptr, const double *b, double *y,
            cudaStream_t s, const int *done) {
    if (!h->sell_ok) {
        spmv_launch(h->nb, h->rowptr.p, h->col.p, h->val.p, x, xld, jptr, b, y, s, done);
        return;
    }
    unsigned blocks = (unsigned)((h->sell_slices + 7) / 8);
    launch_pdl(h->opt.pdl != 0, k_sell_spmv, blocks, 256, s, h->sell_slices, h->nb, h->sell_off.p, h->sell_col.p,
               h->sell_val.p, x, xld, jptr, b, y, done);
}

// ||a||^2 partials into h->red, then a one-thread kernel consumes them.
void norm_partials(cpr_handle *h, const double *a, long n) {
    k_dot_partial<<<kRedBlocks, kBlock, 0, h->stream>>>(n, a, a, h->red.p);
    CK_LAUNCH();
}

}  // namespace

// ================================================================== public

// Rebuild the sliced-ELL copy of the outer operator after a new A: its
// pattern when the pattern changed (or was never built), always its values.
void refresh_outer(cpr_handle *h, bool pattern_changed) {
    cudaStream_t s = h->stream;
    int nb = h->nb;
    if (pattern_changed || !h->sell_ok) {
        h->sell_ok = false;
        int nsl = (nb + 31) / 32;
        DVec<int> width;
        width.alloc(nsl, s);
        k_sell_width<<<grid_for(nsl, kBlock), kBlock, 0, s>>>(nb, nsl, h->rowptr.p, width.p);
        CK_LAUNCH();
        h->sell_off.alloc(nsl + 1, s);
        exclusive_scan(width.p, h->sell_off.p, nsl, s);
        int slots = read_int(h->sell_off.p + nsl, s);
        h->sell_col.alloc(32 * (size_t)std::max(slots, 1), s);
        CK(cudaMemsetAsync(h->sell_col.p, 0xff, sizeof(int) * 32 * (size_t)std::max(slots, 1), s));
        k_sell_pattern<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->col.p, h->sell_off.p,
                                                              h->sell_col.p);
        CK_LAUNCH();
        h->sell_val.alloc(288 * (size_t)std::max(slots, 1), s);
        h->sell_slices = nsl;
    }
    k_sell_values<<<h->sell_slices, 256, 0, s>>>(nb, h->rowptr.p, h->sell_off.p, h->val.p, h->sell_val.p);
    CK_LAUNCH();
    h->sell_ok = true;
}

void bsr3_spmv(int nb, const int *rowptr, const int *col, const double *val, const double *x,
               const double *b, double *y, cudaStream_t s) {
    spmv_launch(nb, rowptr, col, val, x, 0, nullptr, b, y, s, nullptr);
}

void ensure_workspace(cpr_handle *h) {
    cudaStream_t s = h->stream;
    int m = h->opt.restart;
    long N = 3L * h->nb;
    bool size_ok = h->V.n == (size_t)(m + 1) * N && h->m_alloc == m;
    if (!size_ok) {
        h->V.alloc((size_t)(m + 1) * N, s);
        h->Z.alloc((size_t)m * N, s);
        h->wv.alloc(N, s);
        h->r.alloc(N, s);
        h->dev_b.alloc(N, s);
        h->dev_x.alloc(N, s);
        h->t64a.alloc(N, s);
        h->m_alloc = m;
        ScalLayout L{m};
        h->dscal.alloc(L.size(), s);
        h->dscal.zero();
        h->red.alloc((size_t)kRedBlocks * (kMaxRestart + 3), s);
        h->dint.alloc(I_COUNT, s);
        h->dint.zero();
        h->epoch++;
    }
    if (h->opt.precond_fp32 && h->t32a.n != (size_t)N) h->t32a.alloc(N, s);
    if (h->opt.precond_fp32 && h->ep32.n != (size_t)h->nb) h->ep32.alloc(h->nb, s);
    if (!h->opt.precond_fp32 && h->ep64.n != (size_t)h->nb) h->ep64.alloc(h->nb, s);
    if (!h->pinned) {
        CK(cudaMallocHost((void **)&h->pinned, 64 * sizeof(double)));
        // the step kernels write their flags into these page-locked slots directly
        void *d = nullptr;
        CK(cudaHostGetDevicePointer(&d, h->pinned, 0));
        h->pinned_dev_flags = reinterpret_cast<int *>(reinterpret_cast<double *>(d) + 8);
    }
    for (auto &e : h->step_done)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

void apply_B(cpr_handle *h, const double *v_base, long v_ld, const int *jptr, double *z_base,
             long z_ld) {
    if (h->opt.precond_fp32) apply_B_t<float>(h, v_base, v_ld, jptr, z_base, z_ld, nullptr);
    else apply_B_t<double>(h, v_base, v_ld, jptr, z_base, z_ld, nullptr);
}

void vcycle_apply(cpr_handle *h, const double *b, double *x) {
    cudaStream_t s = h->stream;
    Level &L0 = h->lev[0];
    int n = L0.A.n;
    const int *order0 = h->lev.size() > 1 ? L0.rows_by_color.p : nullptr;
    if (h->opt.precond_fp32) {
        k_gather_cast<float><<<grid_for(n, kBlock), kBlock, 0, s>>>(n, order0, b, L0.b32.p);
        CK_LAUNCH();
        pressure_top<float>(h, h->ep32.p, nullptr);
        k_gather_widen<float><<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->bilu.iperm.p, h->ep32.p, x);
        CK_LAUNCH();
    } else {
        k_gather_cast<double><<<grid_for(n, kBlock), kBlock, 0, s>>>(n, order0, b, L0.b.p);
        CK_LAUNCH();
        pressure_top<double>(h, h->ep64.p, nullptr);
        k_gather_widen<double><<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->bilu.iperm.p, h->ep64.p, x);
        CK_LAUNCH();
    }
}

namespace {

// Capture `reps` repetitions of body() into one graph on the handle's stream
// and return the device microseconds per repetition (best of three launches).
template <class F>
double graph_us(cpr_handle *h, int reps, F body) {
    cudaStream_t s = h->stream;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaStreamSynchronize(s));
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
        for (int r = 0; r < reps; r++) body();
    } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    CK(cudaStreamEndCapture(s, &g));
    float best = 1e30f;
    try {
        CK(cudaGraphInstantiate(&ge, g, 0));
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaGraphLaunch(ge, s));
        for (int t = 0; t < 3; t++) {
            CK(cudaEventRecord(e0, s));
            CK(cudaGraphLaunch(ge, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ge) cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    return 1000.0 * best / reps;
}

// The launches of one part of level l's V-cycle work, as vcycle() issues
// them: 0 pre-smoothing sweep, 1 residual, 2 restriction, 3 prolongation,
// 4 post-smoothing sweep.
template <class T>
void level_part(cpr_handle *h, int l, int part) {
    cudaStream_t s = h->stream;
    Level &L = h->lev[l];
    int n = L.A.n;
    Pending pd;
    if (part == 0) {
        mcgs_sweep<T>(h, L, false, true, pd, nullptr, false, Vals<T>::b(L), Vals<T>::x(L));
    } else if (part == 1) {
        pd = Pending{L.color_off[L.ncolors - 1], L.color_off[L.ncolors], 0};
        long thr = std::max<long>((long)n * L.gA, pd.p1 - pd.p0);
        CPR_LANES_DISPATCH(L.gA, (launch_b(h, k_resid_commit<T, G>, blocks_for(thr, L.bs), L.bs, s, n, pd.p0, pd.p1,
                                           L.Ao.rowptr.p, L.Ao.col.p, Vals<T>::Ao(L), Vals<T>::diag(L),
                                           Vals<T>::b(L), Vals<T>::x(L), Vals<T>::s(L, 0), Vals<T>::r(L),
                                           (const int *)nullptr)));
    } else if (part == 2) {
        Level &C = h->lev[l + 1];
        CPR_LANES_DISPATCH(L.gR, (launch_b(h, k_transfer<T, G>, blocks_for((long)L.Rp.n * L.gR, L.bs), L.bs, s,
                                           L.Rp.n, L.Rp.rowptr.p, L.Rp.col.p, Vals<T>::R(L), Vals<T>::r(L),
                                           Vals<T>::r(L), 0, 0, Vals<T>::b(C), false, (const int *)nullptr)));
    } else if (part == 3) {
        Level &C = h->lev[l + 1];
        CPR_LANES_DISPATCH(L.gP, (launch_b(h, k_transfer<T, G>, blocks_for((long)n * L.gP, L.bs), L.bs, s, n,
                                           L.Pp.rowptr.p, L.Pp.col.p, Vals<T>::P(L), Vals<T>::x(C),
                                           Vals<T>::s(C, 0), 0, 0, Vals<T>::x(L), true, (const int *)nullptr)));
    } else {
        mcgs_sweep<T>(h, L, true, false, pd, nullptr, false, Vals<T>::b(L), Vals<T>::x(L));
    }
}

template <class T>
int profile_levels_t(cpr_handle *h, int reps, double *us, int n_us) {
    int L = (int)h->lev.size();
    int need = 3 + 5 * (L - 1);
    if (n_us < need) fail(CPR_ERR_INVALID, "output array shorter than 3 + 5 * (levels - 1)");
    DVec<double> out;
    out.alloc(3 * (size_t)h->nb, h->stream);
    us[0] = graph_us(h, reps, [&] { pressure_top<T>(h, Vals<T>::ep(h), nullptr); });
    us[1] = graph_us(h, reps, [&] { bilu_solve<T>(h, Vals<T>::tmp(h), nullptr, out.p, 0, nullptr, nullptr); });
    Level &C = h->lev.back();
    us[2] = graph_us(h, reps, [&] {
        launch_b(h, k_coarse_solve<T>, blocks_for((long)C.A.n * 32), kBlock, h->stream, C.A.n, h->cinv.p,
                 Vals<T>::b(C), Vals<T>::x(C), (const int *)nullptr);
    });
    for (int l = 0; l < L - 1; l++)
        for (int part = 0; part < 5; part++)
            us[3 + 5 * l + part] = graph_us(h, reps, [&] { level_part<T>(h, l, part); });
    return need;
}

}  // namespace

// The cluster tail covers the last one or two smoothed levels (never level
// 0) when they and the coarse level are small enough for one cluster's shared
// memory, the cycle is V(1,1), and the cluster can be scheduled.
void choose_tail(cpr_handle *h) {
    h->tail_top = -1;
    const cpr_opts &o = h->opt;
    int L = (int)h->lev.size();
    if (!o.tail || o.pre != 1 || o.post != 1 || L < 3 || o.amg == 1) return;
    int nc = h->lev[L - 1].A.n;
    if (nc > kTailMaxCoarse) return;
    size_t elt = o.precond_fp32 ? sizeof(float) : sizeof(double);
    size_t elems = 2 * (size_t)nc;
    int top = -1;
    for (int l = L - 2; l >= 1 && L - 1 - l <= kTailMaxLevels; l--) {
        const Level &Lv = h->lev[l];
        if (Lv.A.n > kTailMaxRows || Lv.ncolors < 1 || Lv.ncolors > kTailMaxColors) break;
        size_t e = elems + 4 * (size_t)Lv.A.n;
        if (e * elt > (size_t)kTailSmemMax) break;
        elems = e;
        top = l;
    }
    if (top < 0) return;
    tail_attr();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kTailCTAs);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = elems * elt;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kTailCTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = o.precond_fp32 ? cudaOccupancyMaxActiveClusters(&nclusters, k_tail_vcycle<float>, &cfg)
                                   : cudaOccupancyMaxActiveClusters(&nclusters, k_tail_vcycle<double>, &cfg);
    if (e != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return;
    }
    h->tail_top = top;
}

bool schedule_ok(const cpr_schedule &s) {
    auto lanes = [](int g) { return g >= 1 && g <= 32 && (g & (g - 1)) == 0; };
    return lanes(s.lanes_a) && lanes(s.lanes_p) && lanes(s.lanes_r) &&
           (s.block == 128 || s.block == 256 || s.block == 512);
}

namespace {

// The tuner of cpr_autotune, per level: the lanes of each kernel family (the
// smoothing sweeps with the residual, the restriction, the prolongation)
// timed over the candidates with the others fixed, then the CTA size over
// all five parts.  A candidate replaces the current choice only when it is at
// least 2 % faster, so timing noise does not flip a choice back and forth.
template <class T>
void autotune_t(cpr_handle *h, int reps, double *before_us, double *after_us) {
    static const int lanes[] = {1, 2, 4, 8, 16, 32};
    static const int blocks[] = {128, 256, 512};
    auto vc = [&] { return graph_us(h, reps, [&] { pressure_top<T>(h, Vals<T>::ep(h), nullptr); }); };
    double before = vc();
    int L = (int)h->lev.size();
    for (int l = 0; l < L - 1; l++) {
        Level &Lv = h->lev[l];
        auto parts = [&](std::initializer_list<int> ps) {
            double t = 0.0;
            for (int part : ps) t += graph_us(h, reps, [&] { level_part<T>(h, l, part); });
            return t;
        };
        auto pick = [&](int *field, std::initializer_list<int> ps, const int *cand, int ncand) {
            double best = parts(ps);
            int choice = *field;
            for (int k = 0; k < ncand; k++) {
                if (cand[k] == choice) continue;
                int keep = *field;
                *field = cand[k];
                double t = parts(ps);
                if (t < 0.98 * best) {
                    best = t;
                    choice = cand[k];
                } else {
                    *field = keep;
                }
                *field = choice;
            }
        };
        pick(&Lv.gA, {0, 1, 4}, lanes, 6);
        pick(&Lv.gR, {2}, lanes, 6);
        pick(&Lv.gP, {3}, lanes, 6);
        pick(&Lv.bs, {0, 1, 2, 3, 4}, blocks, 3);
        h->sched[{Lv.A.n, (long)Lv.A.nnz}] = cpr_schedule{Lv.gA, Lv.gP, Lv.gR, Lv.bs};
    }
    h->epoch++;   // the step graphs are recaptured with the new schedule
    double after = vc();
    if (before_us) *before_us = before;
    if (after_us) *after_us = after;
}

}  // namespace

void autotune(cpr_handle *h, int reps, double *before_us, double *after_us) {
    bool prof = h->prof;
    h->prof = false;   // no event nodes inside the timed graphs
    try {
        if (h->opt.precond_fp32) autotune_t<float>(h, reps, before_us, after_us);
        else autotune_t<double>(h, reps, before_us, after_us);
    } catch (...) {
        h->prof = prof;
        throw;
    }
    h->prof = prof;
}

int profile_vcycle_levels(cpr_handle *h, int reps, double *us, int n_us) {
    bool prof = h->prof;
    h->prof = false;   // no event nodes inside these graphs
    int r;
    try {
        r = h->opt.precond_fp32 ? profile_levels_t<float>(h, reps, us, n_us)
                                : profile_levels_t<double>(h, reps, us, n_us);
    } catch (...) {
        h->prof = prof;
        throw;
    }
    h->prof = prof;
    return r;
}

void bilu_apply(cpr_handle *h, const double *r, double *z) {
    cudaStream_t s = h->stream;
    int nb = h->nb;
    if (h->opt.precond_fp32) {
        k_gather3<float><<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->bilu.rows_by_color.p, r, h->t32a.p);
        CK_LAUNCH();
        bilu_solve<float>(h, h->t32a.p, nullptr, z, 0, nullptr, nullptr);
    } else {
        k_gather3<double><<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->bilu.rows_by_color.p, r, h->t64a.p);
        CK_LAUNCH();
        bilu_solve<double>(h, h->t64a.p, nullptr, z, 0, nullptr, nullptr);
    }
}

// The launches of one Arnoldi step j (j read from device memory).
void record_step(cpr_handle *h) {
    cudaStream_t s = h->stream;
    int m = h->opt.restart;
    long N = 3L * h->nb;
    ScalLayout SL{m};
    int *di = h->dint.p;
    double *sc = h->dscal.p;
    const int *done = di + I_DONE;
    int ldp = kMaxRestart + 2;
    // z_j = B v_j ; w = A z_j
    if (h->opt.precond_fp32) apply_B_t<float>(h, h->V.p, N, di + I_J, h->Z.p, N, done);
    else apply_B_t<double>(h, h->V.p, N, di + I_J, h->Z.p, N, done);
    prof_begin(h, CPR_PROF_SPMV);
    spmv_h(h, h->Z.p, N, di + I_J, nullptr, h->wv.p, s, done);
    prof_end(h);
    // CGS: h_ij = (w, v_i), w -= sum h_ij v_i, h_{j+1,j} = ||w||, Givens
    prof_begin(h, CPR_PROF_CGS);
    bool pdl = h->opt.pdl != 0;
    launch_pdl(pdl, k_cgs_dots, kCgsDotBlocks, kBlock, s, N, (const double *)h->V.p, (const double *)h->wv.p,
               (const int *)(di + I_J), h->red.p, ldp, sc + SL.hcol(), di + I_CNT_DOT, done);
    launch_pdl(pdl, k_cgs_update_givens, kCgsBlocks, kBlock, s, N, (const double *)h->V.p, h->wv.p,
               h->red.p + (size_t)kCgsDotBlocks * ldp, di + I_CNT_UPD, sc, m, di);
    prof_end(h);
    launch_pdl(pdl, k_next_basis, grid_for(N, kBlock, 148 * 8), kBlock, s, N, (const double *)h->wv.p, h->V.p,
               (const double *)sc, m, di, h->pinned_dev_flags);
}

// (Re)capture the step graphs when B, the workspace or profiling changed.
// With profiling on, the two graphs differ in their event nodes and steps
// alternate between them; without it one graph serves both slots (launches of
// one executable graph run in stream order).  An executable graph kept from an
// earlier capture without profiling is updated in place when the new graph has
// its topology -- a new setup of the same level and color counts -- which
// costs less than instantiating it afresh.
void ensure_step_graphs(cpr_handle *h) {
    unsigned pm = h->prof ? h->prof_mask : 0u;
    if (h->sg_epoch == h->epoch && h->sg_prof == pm && h->sg[0].exec && h->sg[1].exec) return;
    Nvtx nv("capture Arnoldi step graphs");
    auto capture = [&](int k) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = k;
        set_capturing(true);
        try {
            record_step(h);
        } catch (...) {
            h->capturing = -1;
            set_capturing(false);
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        h->capturing = -1;
        set_capturing(false);
        CK(cudaStreamEndCapture(h->stream, &g));
        return g;
    };
    if (pm == 0) {
        bool reuse = h->sg_prof == 0 && h->sg[0].exec && h->sg[1].exec == h->sg[0].exec;
        cudaGraph_t g = capture(0);
        if (reuse) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(h->sg[0].exec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                reuse = false;
            }
        }
        if (!reuse) {
            destroy_step_graphs(h);
            cudaGraphExec_t e = nullptr;
            cudaError_t err = cudaGraphInstantiate(&e, g, 0);
            if (err != cudaSuccess) {
                cudaGraphDestroy(g);
                CK(err);
            }
            h->sg[0].exec = h->sg[1].exec = e;
        } else if (h->sg[0].graph) {
            cudaGraphDestroy(h->sg[0].graph);
        }
        h->sg[0].graph = g;
        h->sg[0].kernels = h->sg[1].kernels = graph_kernel_nodes(g);
    } else {
        destroy_step_graphs(h);
        for (int k = 0; k < 2; k++) {
            cudaGraph_t g = capture(k);
            h->sg[k].graph = g;
            h->sg[k].kernels = graph_kernel_nodes(g);
            CK(cudaGraphInstantiate(&h->sg[k].exec, g, 0));
        }
    }
    h->sg_epoch = h->epoch;
    h->sg_prof = pm;
}

// Flexible GMRES(m), right-preconditioned with B (Alg. 2): CGS Arnoldi, Givens
// rotations on the device, stop on |g_{j+1}| < rtol ||r_0|| or h_{j+1,j} = 0,
// true residual after every cycle.  The host reads each step's flags from the
// page-locked slot its last kernel wrote, and one norm per cycle.  It runs as a state machine (FgmresState): each call of
// fgmres_advance issues what can be issued and, unless `block`, returns
// instead of waiting on the device, so one host thread can drive many solves.
// Blocking or not, the same work is launched in the same order.
//
// Steps: step j's graph is launched before the host reads step j-1's flags
// (at most two steps in flight); a step launched after convergence finds
// `done` set and does nothing.

namespace {

bool event_ready(cudaEvent_t e, bool block) {
    if (block) {
        CK(cudaEventSynchronize(e));
        return true;
    }
    cudaError_t q = cudaEventQuery(e);
    if (q == cudaErrorNotReady) {
        cudaGetLastError();
        return false;
    }
    CK(q);
    return true;
}

// r = b - A x, beta = ||r|| and its host copy; first: the cycle-0 scalars.
void issue_cycle_start(cpr_handle *h, bool first) {
    FgmresState &F = h->fs;
    cudaStream_t s = h->stream;
    int m = h->opt.restart;
    long N = 3L * h->nb;
    ScalLayout SL{m};
    spmv_h(h, F.x, 0, nullptr, F.b, h->r.p, s, nullptr);
    norm_partials(h, h->r.p, N);
    k_cycle_start_scal<<<1, 32, 0, s>>>(h->red.p, kRedBlocks, h->dscal.p, m, h->dint.p, first, F.rtol);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(h->pinned, h->dscal.p + SL.rnorm(), sizeof(double), cudaMemcpyDeviceToHost, s));
    if (first)
        CK(cudaMemcpyAsync(reinterpret_cast<int *>(h->pinned + 16), h->bflag.p, sizeof(int),
                           cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h->ev_norm, s));
}

}  // namespace

void fgmres_begin(cpr_handle *h, const double *b, double *x, double rtol) {
    FgmresState &F = h->fs;
    F = FgmresState{};
    F.b = b;
    F.x = x;
    F.rtol = rtol;
    F.rc = CPR_NOT_CONVERGED;
    F.phase = FgmresState::START;
    cudaStream_t s = h->stream;
    if (!h->ev_norm) CK(cudaEventCreateWithFlags(&h->ev_norm, cudaEventDisableTiming));
    if (!h->bflag.p) h->bflag.alloc(1, s);
    CK(cudaMemsetAsync(h->bflag.p, 0, sizeof(int), s));
    k_has_nonfinite_b<<<grid_for(3L * h->nb, 256, 1184), 256, 0, s>>>(3L * h->nb, b, h->bflag.p);
    CK_LAUNCH();
}

int fgmres_advance(cpr_handle *h, bool block) {
    FgmresState &F = h->fs;
    cudaStream_t s = h->stream;
    int m = h->opt.restart;
    long N = 3L * h->nb;
    int *di = h->dint.p;
    double *sc = h->dscal.p;
    int *pin = reinterpret_cast<int *>(h->pinned + 8);   // two slots of 4 ints
    auto check = [&](int step) {
        const int *f = pin + 4 * (step & 1);
        if (f[I_K] == step + 1) {
            F.steps = step + 1;
            if (h->prof) prof_collect_graph(h, step & 1);
        }
        if (f[I_BREAK]) {
            F.rc = CPR_ERR_BREAKDOWN;
            F.stop = true;
        } else if (f[I_DONE]) {
            F.stop = true;
        }
    };
    for (;;) {
        switch (F.phase) {
        case FgmresState::START:
            if (F.cycle >= h->opt.max_restarts) {
                if (F.rc == CPR_NOT_CONVERGED && F.cycles == h->opt.max_restarts) {
                    issue_cycle_start(h, false);   // the true residual after the last cycle
                    F.phase = FgmresState::WAIT_FINAL;
                } else {
                    F.phase = FgmresState::DONE;
                }
                continue;
            }
            issue_cycle_start(h, F.cycle == 0);
            // capture (after a new setup) while the device computes the residual
            ensure_step_graphs(h);
            F.phase = FgmresState::WAIT_START;
            continue;
        case FgmresState::WAIT_START: {
            if (!event_ready(h->ev_norm, block)) return 1;
            if (F.cycle == 0 && reinterpret_cast<int *>(h->pinned + 16)[0]) {
                set_last_error("non-finite right-hand side");
                F.rc = CPR_ERR_BREAKDOWN;
                F.phase = FgmresState::DONE;
                continue;
            }
            F.rnorm = h->pinned[0];
            if (F.cycle == 0) F.norm0 = F.rnorm;
            bool fin = true;
            if (!std::isfinite(F.rnorm)) F.rc = CPR_ERR_BREAKDOWN;
            else if (F.cycle == 0 && F.norm0 == 0.0) F.rc = CPR_OK;
            else if (F.cycle > 0 && F.rnorm / F.norm0 < F.rtol) F.rc = CPR_OK;
            else fin = false;
            if (fin) {
                F.phase = FgmresState::DONE;
                continue;
            }
            k_scale_into<<<grid_for(N, kBlock, 148 * 8), kBlock, 0, s>>>(N, h->r.p, h->V.p, sc, m);
            CK_LAUNCH();
            F.cycles++;
            ensure_step_graphs(h);
            F.launched = F.checked = F.steps = 0;
            F.stop = false;
            F.phase = FgmresState::STEPS;
            continue;
        }
        case FgmresState::STEPS: {
            // launch step j once steps 0 .. j-2 are checked
            if (!F.stop && F.launched < m && F.checked >= F.launched - 1) {
                int j = F.launched;
                CK(cudaGraphLaunch(h->sg[j & 1].exec, s));
                count_launches(h->sg[j & 1].kernels);
                // the graph's last kernel has written step j's flags into pin slot j & 1
                CK(cudaEventRecord(h->step_done[j & 1], s));
                F.launched = j + 1;
                continue;
            }
            // check step j-1 once step j is launched
            if (!F.stop && F.checked < F.launched - 1) {
                if (!event_ready(h->step_done[F.checked & 1], block)) return 1;
                check(F.checked);
                F.checked++;
                continue;
            }
            // the cycle's last step (everything launched has completed)
            if (!event_ready(h->step_done[(F.launched - 1) & 1], block)) return 1;
            if (!F.stop) {
                check(F.launched - 1);
            } else if (F.launched - 1 >= F.steps && F.rc != CPR_ERR_BREAKDOWN) {
                const int *f = pin + 4 * ((F.launched - 1) & 1);
                if (f[I_K] == F.launched) {
                    F.steps = F.launched;
                    if (h->prof) prof_collect_graph(h, (F.launched - 1) & 1);
                }
            }
            F.iters += F.steps;
            if (F.rc == CPR_ERR_BREAKDOWN) {
                F.phase = FgmresState::DONE;
                continue;
            }
            // y = H^-1 g, x += Z y
            k_solve_y<<<1, 1, 0, s>>>(sc, m, di);
            CK_LAUNCH();
            k_update_x<<<grid_for(N, kBlock, 148 * 8), kBlock, 0, s>>>(N, h->Z.p, F.x, sc, m, di);
            CK_LAUNCH();
            F.cycle++;
            F.phase = FgmresState::START;
            continue;
        }
        case FgmresState::WAIT_FINAL:
            if (!event_ready(h->ev_norm, block)) return 1;
            F.rnorm = h->pinned[0];
            if (F.rnorm / F.norm0 < F.rtol) F.rc = CPR_OK;
            F.phase = FgmresState::DONE;
            continue;
        case FgmresState::DONE:
            h->last_iters = F.iters;
            return F.rc;
        default:
            fail(CPR_ERR_INVALID, "no solve in progress");
        }
    }
}

void fgmres_stats(const cpr_handle *h, cpr_stats *st) {
    const FgmresState &F = h->fs;
    st->iters = F.iters;
    st->restarts = F.cycles;
    st->converged = F.rc == CPR_OK;
    st->rel_res = F.norm0 > 0.0 ? F.rnorm / F.norm0 : 0.0;
}

int fgmres(cpr_handle *h, const double *b, double *x, double rtol, cpr_stats *st) {
    fgmres_begin(h, b, x, rtol);
    int rc;
    while ((rc = fgmres_advance(h, true)) == 1) {
    }
    if (st) fgmres_stats(h, st);
    h->fs.phase = FgmresState::IDLE;
    return rc;
}


// ===================================================================== batch
//
// FGMRES(m) for many systems at once (Alg. 2 per system, in lockstep): the
// systems' vectors are segments of one concatenated vector and B is the
// block-diagonal CPR preconditioner of the concatenated operator.  Dots and
// norms are reduced per system over fixed chunks in a fixed order; every
// system keeps its own Hessenberg matrix, rotations, residual estimate and
// stop decision.  A stopped system's rows keep flowing through the shared
// kernels, but nothing of it is updated any more.

namespace {

constexpr int kChunk = 4096;   // vector elements per chunk
enum { S_DONE = 0, S_K = 1, S_BREAK = 2, S_CONV = 3, S_ITERS = 4, S_NINT = 5 };

__global__ void k_bdots(const double *__restrict__ V, const double *__restrict__ w, long N,
                        const int *jptr, const int *cbeg, const int *cend, double *part, int ldp,
                        const int *done) {
    if (*done) return;
    int c = blockIdx.x;
    int nvec = *jptr + 1;
    int beg = cbeg[c], end = cend[c];
    for (int g0 = 0; g0 < nvec; g0 += kDotGroup) {
        double acc[kDotGroup];
#pragma unroll
        for (int k = 0; k < kDotGroup; k++) acc[k] = 0.0;
        for (int q = beg + threadIdx.x; q < end; q += blockDim.x) {
            double wq = w[q];
#pragma unroll
            for (int k = 0; k < kDotGroup; k++)
                if (g0 + k < nvec) acc[k] += V[(size_t)(g0 + k) * N + q] * wq;
        }
#pragma unroll
        for (int k = 0; k < kDotGroup; k++) {
            double sm = block_sum(acc[k]);
            if (threadIdx.x == 0 && g0 + k < nvec) part[(size_t)c * ldp + g0 + k] = sm;
        }
    }
}

// hcol of system s = sum over its chunks (fixed order), one block per system.
__global__ void k_bdots_reduce(const int *sco, const double *part, int ldp, const int *jptr, double *scal,
                               int ssz, int m, const int *sint, const int *done) {
    if (*done) return;
    int sys = blockIdx.x;
    if (sint[S_NINT * sys + S_DONE]) return;
    ScalLayout SL{m};
    int nvec = *jptr + 1;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int c0 = sco[sys], c1 = sco[sys + 1];
    for (int i = wid; i < nvec; i += nw) {
        double sm = 0.0;
        for (int c = c0 + lane; c < c1; c += 32) sm += part[(size_t)c * ldp + i];
        sm = warp_sum(sm);
        if (lane == 0) scal[(size_t)sys * ssz + SL.hcol() + i] = sm;
    }
}

// w -= sum_i h_i V_i on each chunk with its system's h; chunk partials of ||w||^2.
__global__ void k_bupdate(const double *__restrict__ V, double *__restrict__ w, long N, const int *jptr,
                          const int *csys, const int *cbeg, const int *cend, const double *scal, int ssz, int m,
                          const int *sint, double *part2, const int *done) {
    if (*done) return;
    __shared__ double sh[kMaxRestart + 1];
    int c = blockIdx.x, sys = csys[c];
    if (sint[S_NINT * sys + S_DONE]) {
        if (threadIdx.x == 0) part2[c] = 0.0;
        return;
    }
    ScalLayout SL{m};
    int nvec = *jptr + 1;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) sh[i] = scal[(size_t)sys * ssz + SL.hcol() + i];
    __syncthreads();
    double sm = 0.0;
    for (int q = cbeg[c] + threadIdx.x; q < cend[c]; q += blockDim.x) {
        double wq = w[q];
        for (int i = 0; i < nvec; i++) wq -= sh[i] * V[(size_t)i * N + q];
        w[q] = wq;
        sm += wq * wq;
    }
    sm = block_sum(sm);
    if (threadIdx.x == 0) part2[c] = sm;
}

// One Givens step per running system (thread per system), then the shared
// step counter advances; `done` is raised when every system has stopped.
__global__ void k_bgivens(int nsys, const int *sco, const double *part2, double *scal, int ssz, int m,
                          int *sint, int *di) {
    if (di[I_DONE]) return;
    ScalLayout SL{m};
    int j = di[I_J];
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    for (int sys = threadIdx.x; sys < nsys; sys += blockDim.x) {
        int *si = sint + S_NINT * sys;
        if (si[S_DONE]) continue;
        double *sc = scal + (size_t)sys * ssz;
        double hn2 = 0.0;
        for (int c = sco[sys]; c < sco[sys + 1]; c++) hn2 += part2[c];
        double hn = sqrt(hn2);
        for (int i = 0; i <= j; i++) sc[SL.H(i, j)] = sc[SL.hcol() + i];
        sc[SL.H(j + 1, j)] = hn;
        for (int i = 0; i < j; i++) {
            double a = sc[SL.H(i, j)], cc = sc[SL.H(i + 1, j)];
            sc[SL.H(i, j)] = sc[SL.cs() + i] * a + sc[SL.sn() + i] * cc;
            sc[SL.H(i + 1, j)] = -sc[SL.sn() + i] * a + sc[SL.cs() + i] * cc;
        }
        double a = sc[SL.H(j, j)], cc = sc[SL.H(j + 1, j)];
        double den = sqrt(a * a + cc * cc);
        double cj = den == 0.0 ? 1.0 : a / den, sj = den == 0.0 ? 0.0 : cc / den;
        sc[SL.cs() + j] = cj;
        sc[SL.sn() + j] = sj;
        sc[SL.H(j, j)] = den;
        sc[SL.H(j + 1, j)] = 0.0;
        double gj = sc[SL.g() + j];
        sc[SL.g() + j + 1] = -sj * gj;
        sc[SL.g() + j] = cj * gj;
        double est = fabs(sc[SL.g() + j + 1]) / sc[SL.norm0()];
        sc[SL.est()] = est;
        sc[SL.inv_hn()] = hn > 0.0 ? 1.0 / hn : 0.0;
        si[S_K] = j + 1;
        bool brk = !isfinite(hn) || !isfinite(est);
        if (brk) si[S_BREAK] = 1;
        if (brk || hn == 0.0 || est < sc[SL.rtol()] || j + 1 >= m) si[S_DONE] = 1;
        else atomicAdd(&running, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        di[I_J] = j + 1;
        di[I_K] = j + 1;
        if (running == 0) di[I_DONE] = 1;
    }
}

// V_{j+1} = w / h_{j+1,j} per chunk, for systems still running.
__global__ void k_bnext(const double *w, double *V, long N, const int *csys, const int *cbeg, const int *cend,
                        const double *scal, int ssz, int m, const int *sint, const int *di) {
    if (di[I_DONE]) return;
    int c = blockIdx.x, sys = csys[c];
    if (sint[S_NINT * sys + S_DONE]) return;
    ScalLayout SL{m};
    double f = scal[(size_t)sys * ssz + SL.inv_hn()];
    double *v = V + (size_t)di[I_J] * N;
    for (int q = cbeg[c] + threadIdx.x; q < cend[c]; q += blockDim.x) v[q] = w[q] * f;
}

__global__ void k_bnorm_part(const double *r, const int *cbeg, const int *cend, double *part2) {
    int c = blockIdx.x;
    double sm = 0.0;
    for (int q = cbeg[c] + threadIdx.x; q < cend[c]; q += blockDim.x) sm += r[q] * r[q];
    sm = block_sum(sm);
    if (threadIdx.x == 0) part2[c] = sm;
}

// Start of a cycle for every system: beta = ||r_s||; a system whose true
// residual already meets rtol (or whose r_0 is zero or non-finite) stops.
__global__ void k_bcycle_start(int nsys, const int *sco, const double *part2, double *scal, int ssz, int m,
                               int *sint, int *di, int first, double rtol, int *nrunning) {
    ScalLayout SL{m};
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    for (int sys = threadIdx.x; sys < nsys; sys += blockDim.x) {
        double *sc = scal + (size_t)sys * ssz;
        int *si = sint + S_NINT * sys;
        double ss = 0.0;
        for (int c = sco[sys]; c < sco[sys + 1]; c++) ss += part2[c];
        double beta = sqrt(ss);
        if (first) {
            sc[SL.norm0()] = beta;
            sc[SL.rtol()] = rtol;
            si[S_CONV] = 0;
            si[S_ITERS] = 0;
            si[S_BREAK] = 0;
        }
        sc[SL.rnorm()] = beta;
        double n0 = sc[SL.norm0()];
        bool conv = si[S_CONV] || n0 == 0.0 || (!first && beta / n0 < rtol);
        if (!isfinite(beta)) si[S_BREAK] = 1;
        si[S_CONV] = conv;
        for (int i = 0; i <= m; i++) sc[SL.g() + i] = 0.0;
        sc[SL.g()] = beta;
        sc[SL.inv_hn()] = beta > 0.0 ? 1.0 / beta : 0.0;
        si[S_K] = 0;
        si[S_DONE] = conv || si[S_BREAK];
        if (!si[S_DONE]) atomicAdd(&running, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        di[I_J] = 0;
        di[I_K] = 0;
        di[I_BREAK] = 0;
        di[I_DONE] = running == 0;
        *nrunning = running;
    }
}

__global__ void k_bscale(const double *r, double *V, const int *csys, const int *cbeg, const int *cend,
                         const double *scal, int ssz, int m) {
    int c = blockIdx.x, sys = csys[c];
    ScalLayout SL{m};
    double f = scal[(size_t)sys * ssz + SL.inv_hn()];
    for (int q = cbeg[c] + threadIdx.x; q < cend[c]; q += blockDim.x) V[q] = r[q] * f;
}

// y_s = H_s^-1 g_s for every system (thread per system); steps are counted.
__global__ void k_bsolve_y(int nsys, double *scal, int ssz, int m, int *sint) {
    ScalLayout SL{m};
    for (int sys = blockIdx.x * blockDim.x + threadIdx.x; sys < nsys; sys += gridDim.x * blockDim.x) {
        double *sc = scal + (size_t)sys * ssz;
        int k = sint[S_NINT * sys + S_K];
        sint[S_NINT * sys + S_ITERS] += k;
        for (int i = k - 1; i >= 0; i--) {
            double v = sc[SL.g() + i];
            for (int q = i + 1; q < k; q++) v -= sc[SL.H(i, q)] * sc[SL.y() + q];
            sc[SL.y() + i] = v / sc[SL.H(i, i)];
        }
    }
}

__global__ void k_bupdate_x(const double *__restrict__ Z, double *x, long N, const int *csys, const int *cbeg,
                            const int *cend, const double *scal, int ssz, int m, const int *sint) {
    __shared__ double sy[kMaxRestart];
    int c = blockIdx.x, sys = csys[c];
    int k = sint[S_NINT * sys + S_K];
    if (k == 0) return;
    ScalLayout SL{m};
    for (int i = threadIdx.x; i < k; i += blockDim.x) sy[i] = scal[(size_t)sys * ssz + SL.y() + i];
    __syncthreads();
    for (int q = cbeg[c] + threadIdx.x; q < cend[c]; q += blockDim.x) {
        double v = x[q];
        for (int i = 0; i < k; i++) v += sy[i] * Z[(size_t)i * N + q];
        x[q] = v;
    }
}

void record_step_batch(cpr_handle *h) {
    cudaStream_t s = h->stream;
    BatchInfo &B = *h->batch;
    int m = h->opt.restart;
    long N = 3L * h->nb;
    ScalLayout SL{m};
    int ssz = SL.size();
    int *di = h->dint.p;
    const int *done = di + I_DONE;
    int ldp = kMaxRestart + 2;
    if (h->opt.precond_fp32) apply_B_t<float>(h, h->V.p, N, di + I_J, h->Z.p, N, done);
    else apply_B_t<double>(h, h->V.p, N, di + I_J, h->Z.p, N, done);
    spmv_h(h, h->Z.p, N, di + I_J, nullptr, h->wv.p, s, done);
    k_bdots<<<B.nchunk, kBlock, 0, s>>>(h->V.p, h->wv.p, N, di + I_J, B.chunk_beg.p, B.chunk_end.p, B.part.p, ldp,
                                        done);
    CK_LAUNCH();
    k_bdots_reduce<<<B.nsys, kBlock, 0, s>>>(B.sys_chunk_off.p, B.part.p, ldp, di + I_J, B.scal.p, ssz, m,
                                             B.sint.p, done);
    CK_LAUNCH();
    k_bupdate<<<B.nchunk, kBlock, 0, s>>>(h->V.p, h->wv.p, N, di + I_J, B.chunk_sys.p, B.chunk_beg.p,
                                          B.chunk_end.p, B.scal.p, ssz, m, B.sint.p, B.part2.p, done);
    CK_LAUNCH();
    k_bgivens<<<1, 1024, 0, s>>>(B.nsys, B.sys_chunk_off.p, B.part2.p, B.scal.p, ssz, m, B.sint.p, di);
    CK_LAUNCH();
    k_bnext<<<B.nchunk, kBlock, 0, s>>>(h->wv.p, h->V.p, N, B.chunk_sys.p, B.chunk_beg.p, B.chunk_end.p, B.scal.p,
                                        ssz, m, B.sint.p, di);
    CK_LAUNCH();
}

}  // namespace

// Chunk tables and per-system buffers for the handle's batch description.
void batch_prepare(cpr_handle *h) {
    BatchInfo &B = *h->batch;
    cudaStream_t s = h->stream;
    std::vector<int> csys, cbeg, cend, sco(B.nsys + 1, 0);
    for (int sys = 0; sys < B.nsys; sys++) {
        int beg = 3 * B.boff[sys], end = 3 * B.boff[sys + 1];
        sco[sys] = (int)csys.size();
        for (int q = beg; q < end; q += kChunk) {
            csys.push_back(sys);
            cbeg.push_back(q);
            cend.push_back(std::min(end, q + kChunk));
        }
    }
    sco[B.nsys] = (int)csys.size();
    B.nchunk = (int)csys.size();
    auto up = [&](DVec<int> &d, const std::vector<int> &v) {
        d.alloc(std::max<size_t>(v.size(), 1), s);
        CK(cudaMemcpyAsync(d.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
    };
    up(B.chunk_sys, csys);
    up(B.chunk_beg, cbeg);
    up(B.chunk_end, cend);
    up(B.sys_chunk_off, sco);
    int m = h->opt.restart;
    ScalLayout SL{m};
    B.scal.alloc((size_t)B.nsys * SL.size(), s);
    B.scal.zero();
    B.sint.alloc((size_t)B.nsys * S_NINT, s);
    B.sint.zero();
    B.part.alloc((size_t)B.nchunk * (kMaxRestart + 2), s);
    B.part2.alloc(B.nchunk, s);
    B.b.alloc(3L * h->nb, s);
    B.x.alloc(3L * h->nb, s);
    CK(cudaStreamSynchronize(s));
}

// Lockstep FGMRES for every system of the batch; B.b and B.x hold the
// concatenated right-hand sides and initial guesses; st[s] gets system s's stats.
int fgmres_batch(cpr_handle *h, double rtol, cpr_stats *st) {
    cudaStream_t s = h->stream;
    BatchInfo &B = *h->batch;
    int m = h->opt.restart;
    long N = 3L * h->nb;
    ScalLayout SL{m};
    int ssz = SL.size();
    int *di = h->dint.p;
    double *x = B.x.p;
    int *pin = reinterpret_cast<int *>(h->pinned + 8);
    int rc = CPR_NOT_CONVERGED;
    if (h->sgb_epoch != h->epoch || !h->sgb[0].exec || !h->sgb[1].exec) {
        for (auto &g : h->sgb) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            g = cpr_handle::StepGraph{};
        }
        bool prof = h->prof;
        h->prof = false;
        for (int k = 0; k < 2; k++) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            set_capturing(true);
            try {
                record_step_batch(h);
            } catch (...) {
                set_capturing(false);
                cudaStreamEndCapture(s, &g);
                if (g) cudaGraphDestroy(g);
                h->prof = prof;
                throw;
            }
            set_capturing(false);
            CK(cudaStreamEndCapture(s, &g));
            h->sgb[k].graph = g;
            h->sgb[k].kernels = graph_kernel_nodes(g);
            CK(cudaGraphInstantiate(&h->sgb[k].exec, g, 0));
        }
        h->prof = prof;
        h->sgb_epoch = h->epoch;
    }
    int cycles = 0;
    for (int cycle = 0; cycle <= h->opt.max_restarts; cycle++) {
        spmv_h(h, x, 0, nullptr, B.b.p, h->r.p, s, nullptr);
        k_bnorm_part<<<B.nchunk, kBlock, 0, s>>>(h->r.p, B.chunk_beg.p, B.chunk_end.p, B.part2.p);
        CK_LAUNCH();
        k_bcycle_start<<<1, 1024, 0, s>>>(B.nsys, B.sys_chunk_off.p, B.part2.p, B.scal.p, ssz, m, B.sint.p, di,
                                          cycle == 0, rtol, di + I_ZERO);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(pin + 8, di + I_ZERO, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (pin[8] == 0 || cycle == h->opt.max_restarts) break;
        k_bscale<<<B.nchunk, kBlock, 0, s>>>(h->r.p, h->V.p, B.chunk_sys.p, B.chunk_beg.p, B.chunk_end.p, B.scal.p,
                                             ssz, m);
        CK_LAUNCH();
        cycles++;
        bool stop = false;
        for (int j = 0; j < m && !stop; j++) {
            CK(cudaGraphLaunch(h->sgb[j & 1].exec, s));
            count_launches(h->sgb[j & 1].kernels);
            CK(cudaMemcpyAsync(pin + 4 * (j & 1), di, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaEventRecord(h->step_done[j & 1], s));
            if (j >= 1) {
                CK(cudaEventSynchronize(h->step_done[(j - 1) & 1]));
                stop = pin[4 * ((j - 1) & 1) + I_DONE] != 0;
            }
        }
        CK(cudaStreamSynchronize(s));
        k_bsolve_y<<<grid_for(B.nsys, 128), 128, 0, s>>>(B.nsys, B.scal.p, ssz, m, B.sint.p);
        CK_LAUNCH();
        k_bupdate_x<<<B.nchunk, kBlock, 0, s>>>(h->Z.p, x, N, B.chunk_sys.p, B.chunk_beg.p, B.chunk_end.p, B.scal.p,
                                                ssz, m, B.sint.p);
        CK_LAUNCH();
    }
    std::vector<int> si((size_t)B.nsys * S_NINT);
    std::vector<double> sc((size_t)B.nsys * ssz);
    CK(cudaMemcpyAsync(si.data(), B.sint.p, sizeof(int) * si.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(sc.data(), B.scal.p, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool all = true, brk = false;
    long total = 0;
    for (int sys = 0; sys < B.nsys; sys++) {
        const int *q = &si[(size_t)sys * S_NINT];
        const double *c = &sc[(size_t)sys * ssz];
        all = all && q[S_CONV];
        brk = brk || q[S_BREAK];
        total = std::max<long>(total, q[S_ITERS]);
        if (st) {
            st[sys].iters = q[S_ITERS];
            st[sys].restarts = cycles;
            st[sys].converged = q[S_CONV];
            st[sys].rel_res = c[SL.norm0()] > 0.0 ? c[SL.rnorm()] / c[SL.norm0()] : 0.0;
        }
    }
    h->last_iters = total;
    rc = brk ? CPR_ERR_BREAKDOWN : (all ? CPR_OK : CPR_NOT_CONVERGED);
    return rc;
}

}  // namespace cpr
