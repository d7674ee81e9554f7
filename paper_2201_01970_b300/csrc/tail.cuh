// The tail of the V-cycle in one kernel: the last (at most two) smoothed
// levels and the coarse solve (Sec. 3.1's B_P, Alg. 5 per level) run on one
// thread-block cluster, phases separated by cluster barriers instead of
// kernel boundaries.  A bare cluster barrier costs about 0.3 us on B300
// against about 2 us for a kernel boundary between dependent launches, but
// each phase here still waits on its dependent loads and on the release of
// its remote stores: at 128x128x32 (levels 4 and 5, 22 phases) the kernel
// takes about 80 us where the kernel-per-phase chain takes 54 us, with 8 or
// 16 CTAs and with the rows prefetched into L1.  It is therefore off by
// default (cpr_opts.tail).
//
// Layout: each CTA keeps a full replica of the tail's vectors in shared
// memory (per level x, the staging vector s, r and b; the coarse b and x).
// CTA k owns the k-th chunk of every color's row range (and of the coarse
// rows); a value it computes is stored into every CTA's replica through
// distributed shared memory, and the next phase starts after a cluster
// barrier.  Matrices are read from global memory (L2).
//
// Every product is the one of the standalone kernels (k_smooth_first,
// k_smooth_color, k_resid_commit, k_transfer, k_transfer_first,
// k_coarse_solve): the same G lanes per row, each lane summing its entries
// in ascending order, the same shuffle tree, the same expressions, and the
// same Jacobi-within-a-color staging (a color's new values go to s and are
// committed into x by the next phase).  The results are therefore bit for
// bit those of the kernel-per-phase V-cycle.
#pragma once

#include <cooperative_groups.h>

#include "sweeps.cuh"

namespace cpr {
namespace {

namespace cg = cooperative_groups;

constexpr int kTailCTAs = 8;          // cluster size (portable)
constexpr int kTailThreads = 1024;
constexpr int kTailMaxLevels = 2;
constexpr int kTailMaxColors = 16;
constexpr int kTailMaxRows = 4096;    // rows of a tail level
constexpr int kTailMaxCoarse = 1024;  // rows of the coarse level
constexpr int kTailSmemMax = 160 * 1024;

template <class T>
struct TailLevel {
    int n, ncolors, gA, gP, gR;
    int color_off[kTailMaxColors + 1];
    const int *arow, *acol;    // A_l without its diagonal, color order
    const T *aval, *diag, *dinv;
    const int *prow, *pcol;    // P_l: this level's rows, next level's columns
    const T *pval;
    const int *rrow, *rcol;    // R_l: next level's rows, this level's columns
    const T *rval;
    int ox, os, orr, ob;       // replica offsets in shared memory (elements of T)
};

template <class T>
struct TailArgs {
    int nlev, nc, obc, oxc;
    TailLevel<T> lev[kTailMaxLevels];
    const double *cinv;        // coarse inverse, row-major FP64
    const T *b_top;            // b of the top tail level (written by the restriction above)
    T *x_top;                  // its result (read by the prolongation above)
};

// The chunk of rows [a, b) owned by CTA k.
__device__ __forceinline__ void tail_chunk(int a, int b, int k, int &r0, int &r1) {
    long len = b - a;
    r0 = a + (int)(len * k / kTailCTAs);
    r1 = a + (int)(len * (k + 1) / kTailCTAs);
}

// v into every CTA's replica of vec at index i.
template <class T>
__device__ __forceinline__ void tail_put(const cg::cluster_group &cl, T *vec, int i, T v) {
#pragma unroll
    for (int q = 0; q < kTailCTAs; q++) cl.map_shared_rank(vec, q)[i] = v;
}

// This lane's share of row `row`'s product with xs: entries lane, lane+G, ...
template <class T>
__device__ __forceinline__ T tail_dot(const int *rp, const int *col, const T *val, int row, int lane, int G,
                                      const T *xs) {
    T s = 0;
    int e1 = rp[row + 1];
    for (int p = rp[row] + lane; p < e1; p += G) s += val[p] * xs[col[p]];
    return s;
}

// Copy the staged range [p0, p1) of s into x (this CTA's replica).
template <class T>
__device__ __forceinline__ void tail_commit(T *x, const T *s, int &p0, int &p1) {
    for (int i = p0 + (int)threadIdx.x; i < p1; i += kTailThreads) x[i] = s[i];
    p0 = p1 = 0;
    __syncthreads();
}

// Relax the owned rows of color c into s (after committing the previous
// color): s_i = (b_i - sum_j a_ij x_j) / a_ii.
template <class T>
__device__ void tail_smooth(const cg::cluster_group &cl, int k, T *sm, const TailLevel<T> &L, int c, int &p0,
                            int &p1) {
    T *x = sm + L.ox, *s = sm + L.os;
    const T *b = sm + L.ob;
    tail_commit(x, s, p0, p1);
    int r0, r1;
    tail_chunk(L.color_off[c], L.color_off[c + 1], k, r0, r1);
    int G = L.gA, per = kTailThreads / G, g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int base = r0; base < r1; base += per) {   // uniform over the block
        int row = base + g;
        bool act = row < r1;
        T sum = act ? tail_dot(L.arow, L.acol, L.aval, row, lane, G, x) : (T)0;
        sum = group_sum(sum, G);
        if (act && lane == 0) tail_put(cl, s, row, (b[row] - sum) * L.dinv[row]);
    }
    cl.sync();
    p0 = L.color_off[c];
    p1 = L.color_off[c + 1];
}

// r = b - A x on the owned rows, into every replica.
template <class T>
__device__ void tail_resid(const cg::cluster_group &cl, int k, T *sm, const TailLevel<T> &L, int &p0, int &p1) {
    T *x = sm + L.ox, *r = sm + L.orr;
    const T *b = sm + L.ob;
    tail_commit(x, sm + L.os, p0, p1);
    int G = L.gA, per = kTailThreads / G, g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int c = 0; c < L.ncolors; c++) {
        int r0, r1;
        tail_chunk(L.color_off[c], L.color_off[c + 1], k, r0, r1);
        for (int base = r0; base < r1; base += per) {
            int row = base + g;
            bool act = row < r1;
            T sum = act ? tail_dot(L.arow, L.acol, L.aval, row, lane, G, x) : (T)0;
            sum = group_sum(sum, G);
            if (act && lane == 0) tail_put(cl, r, row, b[row] - sum - L.diag[row] * x[row]);
        }
    }
    cl.sync();
}

// b_N = R_L r_L on N's owned rows (b is needed by its owner only); from
// x_N = 0, N's color-0 rows are staged as b/a_ii.  N's pending range becomes
// color 0.
template <class T>
__device__ void tail_restrict_level(const cg::cluster_group &cl, int k, T *sm, const TailLevel<T> &L,
                                    const TailLevel<T> &N, int &q0, int &q1) {
    const T *r = sm + L.orr;
    T *bN = sm + N.ob, *sN = sm + N.os;
    int G = L.gR, per = kTailThreads / G, g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int c = 0; c < N.ncolors; c++) {
        int r0, r1;
        tail_chunk(N.color_off[c], N.color_off[c + 1], k, r0, r1);
        for (int base = r0; base < r1; base += per) {
            int row = base + g;
            bool act = row < r1;
            T sum = act ? tail_dot(L.rrow, L.rcol, L.rval, row, lane, G, r) : (T)0;
            sum = group_sum(sum, G);
            if (act && lane == 0) {
                bN[row] = sum;
                if (c == 0) tail_put(cl, sN, row, sum * N.dinv[row]);
            }
        }
    }
    cl.sync();
    q0 = N.color_off[0];
    q1 = N.color_off[1];
}

// b_c = R_L r_L on the owned coarse rows, into every replica.
template <class T>
__device__ void tail_restrict_coarse(const cg::cluster_group &cl, int k, T *sm, const TailLevel<T> &L,
                                     const TailArgs<T> &a) {
    const T *r = sm + L.orr;
    T *bc = sm + a.obc;
    int r0, r1;
    tail_chunk(0, a.nc, k, r0, r1);
    int G = L.gR, per = kTailThreads / G, g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int base = r0; base < r1; base += per) {
        int row = base + g;
        bool act = row < r1;
        T sum = act ? tail_dot(L.rrow, L.rcol, L.rval, row, lane, G, r) : (T)0;
        sum = group_sum(sum, G);
        if (act && lane == 0) tail_put(cl, bc, row, sum);
    }
    cl.sync();
}

// x_c = A_c^-1 b_c on the owned coarse rows (FP64 dot, one warp per row).
template <class T>
__device__ void tail_coarse(const cg::cluster_group &cl, int k, T *sm, const TailArgs<T> &a) {
    const T *bc = sm + a.obc;
    T *xc = sm + a.oxc;
    int r0, r1;
    tail_chunk(0, a.nc, k, r0, r1);
    int n = a.nc, per = kTailThreads / 32, g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int base = r0; base < r1; base += per) {
        int row = base + g;
        bool act = row < r1;
        double s = 0.0;
        if (act)
            for (int j = lane; j < n; j += 32) s += a.cinv[(size_t)row * n + j] * (double)bc[j];
        s = group_sum(s, 32);
        if (act && lane == 0) tail_put(cl, xc, row, (T)s);
    }
    cl.sync();
}

// x_L += P_L xn on L's owned rows (every color), into every replica.
template <class T>
__device__ void tail_prolong(const cg::cluster_group &cl, int k, T *sm, const TailLevel<T> &L, const T *xn) {
    T *x = sm + L.ox;
    int G = L.gP, per = kTailThreads / G, g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int c = 0; c < L.ncolors; c++) {
        int r0, r1;
        tail_chunk(L.color_off[c], L.color_off[c + 1], k, r0, r1);
        for (int base = r0; base < r1; base += per) {
            int row = base + g;
            bool act = row < r1;
            T sum = act ? tail_dot(L.prow, L.pcol, L.pval, row, lane, G, xn) : (T)0;
            sum = group_sum(sum, G);
            if (act && lane == 0) tail_put(cl, x, row, x[row] + sum);
        }
    }
    cl.sync();
}

// Bring [p, p + bytes) into this SM's L1, spread over the block's threads.
__device__ __forceinline__ void tail_pf(const void *p, long bytes) {
    const char *c = (const char *)p;
    for (long o = (long)threadIdx.x * 128; o < bytes; o += (long)kTailThreads * 128)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(c + o));
}

// Prefetch everything this CTA reads of level L: its rows of A, P, diag and
// 1/a_ii, and the rows of R that restrict into the next level's owned rows
// (next level: noff/nnc colors, or the coarse rows [0, nc) when nnc == 0).
template <class T>
__device__ void tail_prefetch(int k, const TailLevel<T> &L, const int *noff, int nnc, int nc) {
    for (int c = 0; c < L.ncolors; c++) {
        int r0, r1;
        tail_chunk(L.color_off[c], L.color_off[c + 1], k, r0, r1);
        if (r1 <= r0) continue;
        int a0 = L.arow[r0], a1 = L.arow[r1], q0 = L.prow[r0], q1 = L.prow[r1];
        tail_pf(L.arow + r0, 4L * (r1 - r0 + 1));
        tail_pf(L.acol + a0, 4L * (a1 - a0));
        tail_pf(L.aval + a0, (long)sizeof(T) * (a1 - a0));
        tail_pf(L.diag + r0, (long)sizeof(T) * (r1 - r0));
        tail_pf(L.dinv + r0, (long)sizeof(T) * (r1 - r0));
        tail_pf(L.prow + r0, 4L * (r1 - r0 + 1));
        tail_pf(L.pcol + q0, 4L * (q1 - q0));
        tail_pf(L.pval + q0, (long)sizeof(T) * (q1 - q0));
    }
    int nchunks = nnc ? nnc : 1;
    for (int c = 0; c < nchunks; c++) {
        int r0, r1;
        if (nnc) tail_chunk(noff[c], noff[c + 1], k, r0, r1);
        else tail_chunk(0, nc, k, r0, r1);
        if (r1 <= r0) continue;
        int a0 = L.rrow[r0], a1 = L.rrow[r1];
        tail_pf(L.rrow + r0, 4L * (r1 - r0 + 1));
        tail_pf(L.rcol + a0, 4L * (a1 - a0));
        tail_pf(L.rval + a0, (long)sizeof(T) * (a1 - a0));
    }
}

// One V(1,1) cycle from x = 0 on the tail levels, their coarse solve
// included; b of the top level comes from global memory, its x goes back.
template <class T>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail_vcycle(const __grid_constant__ TailArgs<T> a,
                                                                   const int *done) {
    extern __shared__ __align__(16) unsigned char tail_raw[];
    T *sm = reinterpret_cast<T *>(tail_raw);
    cg::cluster_group cl = cg::this_cluster();
    if (done && *done) return;   // the same flag for every CTA of the cluster
    int k = (int)cl.block_rank();
    const TailLevel<T> &T0 = a.lev[0];
    for (int i = threadIdx.x; i < T0.n; i += kTailThreads) {
        sm[T0.ox + i] = (T)0;
        sm[T0.ob + i] = a.b_top[i];
    }
    if (a.nlev > 1)
        for (int i = threadIdx.x; i < a.lev[1].n; i += kTailThreads) sm[a.lev[1].ox + i] = (T)0;
    // every later phase reads this CTA's rows from L1
    if (a.nlev > 1) {
        tail_prefetch(k, T0, a.lev[1].color_off, a.lev[1].ncolors, 0);
        tail_prefetch(k, a.lev[1], nullptr, 0, a.nc);
    } else {
        tail_prefetch(k, T0, nullptr, 0, a.nc);
    }
    cl.sync();   // every CTA runs before any store into its shared memory
    int p0 = 0, p1 = 0, q0 = 0, q1 = 0;   // staged ranges of the two levels
    // top level: color 0 from zero (b/a_ii), then the other colors ascending
    {
        int r0, r1;
        tail_chunk(T0.color_off[0], T0.color_off[1], k, r0, r1);
        for (int i = r0 + threadIdx.x; i < r1; i += kTailThreads)
            tail_put(cl, sm + T0.os, i, sm[T0.ob + i] * T0.dinv[i]);
        cl.sync();
        p0 = T0.color_off[0];
        p1 = T0.color_off[1];
    }
    for (int c = 1; c < T0.ncolors; c++) tail_smooth(cl, k, sm, T0, c, p0, p1);
    tail_resid(cl, k, sm, T0, p0, p1);
    if (a.nlev > 1) {
        const TailLevel<T> &T1 = a.lev[1];
        tail_restrict_level(cl, k, sm, T0, T1, q0, q1);
        for (int c = 1; c < T1.ncolors; c++) tail_smooth(cl, k, sm, T1, c, q0, q1);
        tail_resid(cl, k, sm, T1, q0, q1);
        tail_restrict_coarse(cl, k, sm, T1, a);
        tail_coarse(cl, k, sm, a);
        tail_prolong(cl, k, sm, T1, sm + a.oxc);
        for (int c = T1.ncolors - 1; c >= 0; c--) tail_smooth(cl, k, sm, T1, c, q0, q1);
        tail_commit(sm + T1.ox, sm + T1.os, q0, q1);
        tail_prolong(cl, k, sm, T0, sm + T1.ox);
    } else {
        tail_restrict_coarse(cl, k, sm, T0, a);
        tail_coarse(cl, k, sm, a);
        tail_prolong(cl, k, sm, T0, sm + a.oxc);
    }
    for (int c = T0.ncolors - 1; c >= 0; c--) tail_smooth(cl, k, sm, T0, c, p0, p1);
    tail_commit(sm + T0.ox, sm + T0.os, p0, p1);
    // no remote store reaches this CTA after the last barrier
    int r0, r1;
    tail_chunk(0, T0.n, k, r0, r1);
    for (int i = r0 + threadIdx.x; i < r1; i += kTailThreads) a.x_top[i] = sm[T0.ox + i];
}

}  // namespace
}  // namespace cpr
