// Device pieces shared by the solve path and the allocation-free BILU entry:
// programmatic-dependent-launch hooks, lane-group sums and the multicolor
// BILU(0) forward/backward sweeps.  Both translation units include this file,
// so the two BILU applications run the same code and agree bit for bit.
#pragma once

#include "cpr_internal.cuh"

namespace cpr {
namespace {

__device__ __forceinline__ int step_of(const int *jptr) { return jptr ? *jptr : 0; }

// Lanes per block row of the FP32 BILU(0) sweeps (FP32 shuffles are cheap; a
// sweep of 1, 2, 4 and 8 lanes measured 2 fastest on B300 at 128x128x32,
// 101 us per application against 102.5 with 4 and 128 with 8).  FP64 sweeps
// use one thread per block row: no cross-lane FP64 additions.
constexpr int kBiluLanesF32 = 2;

template <class T>
__device__ __forceinline__ T group_sum(T v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
    return v;
}

// ------------------------------------------------ programmatic dependent launch
//
// The kernels of one B application run as a chain in which each kernel's
// inputs are the previous kernels' outputs, but most of what they read -- the
// matrices' patterns and values, 1/a_ii, the permutations -- was fixed at
// setup.  Each kernel loads that static part first, then waits for its
// predecessor (griddepcontrol.wait: the predecessor has completed and its
// writes are visible), then lets its own successor launch.  The successor's
// static loads thus overlap this kernel's dependent work, and since a kernel
// lets its successor start only after its own wait returned, everything
// before the current kernel has completed when a prologue runs.  Without the
// launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The step's stop flag, read after the wait together with a kernel's
// gathers and tested only before its first store: a test right after the wait
// would hold every gather back by the flag's round trip.  (A stopped step's
// kernels then load what they would have used, all in bounds, and store
// nothing.)
__device__ __forceinline__ int stop_flag(const int *done) { return done ? *done : 0; }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Forward substitution of row i: y_i - sum_{lower} L_ij y_j, left in
// (s0, s1, s2) on the row's lead lane (G == 1: its thread).  The first kPreB
// blocks of each lane (columns cj, values Lp) were loaded before the wait.
template <class T, int G, int kPreB>
__device__ __forceinline__ void bilu_fwd_row(bool active, int lane, int i, int e0, int e1,
                                             const int (&cj)[kPreB], const T (&Lp)[kPreB][9],
                                             const int *__restrict__ lc, const T *__restrict__ lv, const T *y,
                                             T &s0, T &s1, T &s2) {
    if constexpr (G == 1) {
        if (!active) return;
        s0 = y[3 * (size_t)i], s1 = y[3 * (size_t)i + 1], s2 = y[3 * (size_t)i + 2];
#pragma unroll
        for (int u = 0; u < kPreB; u++)
            if (e0 + u < e1) {
                const T *L = Lp[u];
                const T *yj = y + 3 * (size_t)cj[u];
                T y0 = yj[0], y1 = yj[1], y2 = yj[2];
                s0 -= L[0] * y0 + L[1] * y1 + L[2] * y2;
                s1 -= L[3] * y0 + L[4] * y1 + L[5] * y2;
                s2 -= L[6] * y0 + L[7] * y1 + L[8] * y2;
            }
#pragma unroll 4
        for (int p = e0 + kPreB; p < e1; p++) {
            const T *L = lv + 9 * (size_t)p;
            const T *yj = y + 3 * (size_t)lc[p];
            T y0 = yj[0], y1 = yj[1], y2 = yj[2];
            s0 -= L[0] * y0 + L[1] * y1 + L[2] * y2;
            s1 -= L[3] * y0 + L[4] * y1 + L[5] * y2;
            s2 -= L[6] * y0 + L[7] * y1 + L[8] * y2;
        }
    } else {
        // G lanes share the row: lane sums of L_ij y_j, then one group sum;
        // the row's own y_i is loaded with the gathers, not after them
        bool lead = active && lane == 0;
        T yi0 = lead ? y[3 * (size_t)i] : (T)0, yi1 = lead ? y[3 * (size_t)i + 1] : (T)0,
          yi2 = lead ? y[3 * (size_t)i + 2] : (T)0;
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int u = 0; u < kPreB; u++)
            if (e0 + lane + u * G < e1) {
                const T *L = Lp[u];
                const T *yj = y + 3 * (size_t)cj[u];
                T y0 = yj[0], y1 = yj[1], y2 = yj[2];
                a0 += L[0] * y0 + L[1] * y1 + L[2] * y2;
                a1 += L[3] * y0 + L[4] * y1 + L[5] * y2;
                a2 += L[6] * y0 + L[7] * y1 + L[8] * y2;
            }
        for (int p = e0 + lane + kPreB * G; p < e1; p += G) {
            const T *L = lv + 9 * (size_t)p;
            const T *yj = y + 3 * (size_t)lc[p];
            T y0 = yj[0], y1 = yj[1], y2 = yj[2];
            a0 += L[0] * y0 + L[1] * y1 + L[2] * y2;
            a1 += L[3] * y0 + L[4] * y1 + L[5] * y2;
            a2 += L[6] * y0 + L[7] * y1 + L[8] * y2;
        }
        a0 = group_sum(a0, G);
        a1 = group_sum(a1, G);
        a2 = group_sum(a2, G);
        s0 = yi0 - a0;
        s1 = yi1 - a1;
        s2 = yi2 - a2;
    }
}

// The first blocks of each lane's share of row i of L (or U), loaded before the wait.
template <class T, int G, int kPreB>
__device__ __forceinline__ void bilu_pre(int e0, int e1, int lane, const int *__restrict__ c,
                                         const T *__restrict__ v, int (&cj)[kPreB], T (&Vp)[kPreB][9]) {
#pragma unroll
    for (int u = 0; u < kPreB; u++) {
        int p = e0 + lane + u * G;
        bool in = p < e1;
        cj[u] = in ? c[p] : 0;
#pragma unroll
        for (int k = 0; k < 9; k++) Vp[u][k] = in ? v[9 * (size_t)p + k] : (T)0;
    }
}

// Forward substitution for the color of positions [c0, c0 + cnt), in place:
// y_i = r_i - sum_{lower} L_ij y_j (everything in BILU positions).  G lanes
// share a block row (G = 1: one thread, blocks in order).
template <class T, int G>
__global__ void k_bilu_fwd(int c0, int cnt, const int *__restrict__ lr,
                           const int *__restrict__ lc, const T *__restrict__ lv, T *y,
                           const int *done) {
    constexpr int kPreB = G == 1 ? 3 : 2;   // blocks per lane loaded before the wait: per BILU application at
                                           // 128x128x32, FP32 (G = 2) 82.7 -> 76.0 us with 2 against 1, FP64
                                           // (G = 1) 237 -> 217 us with 3 against 2
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    bool active = t < cnt;
    int i = c0 + (int)t;
    int e0 = 0, e1 = 0;
    if (active) {
        e0 = lr[i];
        e1 = lr[i + 1];
    }
    int cj[kPreB];
    T Lp[kPreB][9];
    bilu_pre<T, G, kPreB>(e0, e1, lane, lc, lv, cj, Lp);
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);   // tested before the first store, not ahead of the gathers
    T s0 = 0, s1 = 0, s2 = 0;
    bilu_fwd_row<T, G, kPreB>(active, lane, i, e0, e1, cj, Lp, lc, lv, y, s0, s1, s2);
    if (dn || !active || lane != 0) return;
    y[3 * (size_t)i] = s0;
    y[3 * (size_t)i + 1] = s1;
    y[3 * (size_t)i + 2] = s2;
}

// The highest color in one launch: its rows have no higher-color (upper)
// neighbours, so the backward step is z_i = U_ii^-1 y_i right after the
// forward one, with the same operations as the two kernels apart.  Writes z
// into y and, plus Pi_P e_P when ep != nullptr, into out (as k_bilu_bwd).
template <class T, int G>
__global__ void k_bilu_last(int c0, int cnt, const int *__restrict__ lr, const int *__restrict__ lc,
                            const T *__restrict__ lv, const T *__restrict__ dinv, T *y, const T *ep,
                            const int *__restrict__ border, double *out_base, long ld, const int *jptr,
                            const int *done) {
    constexpr int kPreB = G == 1 ? 3 : 2;
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    bool active = t < cnt;
    bool lead = active && lane == 0;
    int i = c0 + (int)t;
    int e0 = 0, e1 = 0, bi = 0;
    if (active) {
        e0 = lr[i];
        e1 = lr[i + 1];
    }
    if (lead) bi = border[i];
    T D[9];
#pragma unroll
    for (int k = 0; k < 9; k++) D[k] = lead ? dinv[9 * (size_t)i + k] : (T)0;
    int cj[kPreB];
    T Lp[kPreB][9];
    bilu_pre<T, G, kPreB>(e0, e1, lane, lc, lv, cj, Lp);
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);
    double *out = out_base + (size_t)step_of(jptr) * ld + 3 * (size_t)bi;
    double e0v = lead && ep ? (double)ep[i] : 0.0;
    T s0 = 0, s1 = 0, s2 = 0;
    bilu_fwd_row<T, G, kPreB>(active, lane, i, e0, e1, cj, Lp, lc, lv, y, s0, s1, s2);
    if (dn || !lead) return;
    T z0 = D[0] * s0 + D[1] * s1 + D[2] * s2;
    T z1 = D[3] * s0 + D[4] * s1 + D[5] * s2;
    T z2 = D[6] * s0 + D[7] * s1 + D[8] * s2;
    y[3 * (size_t)i] = z0;
    y[3 * (size_t)i + 1] = z1;
    y[3 * (size_t)i + 2] = z2;
    out[0] = (double)z0 + e0v;
    out[1] = (double)z1;
    out[2] = (double)z2;
}

// Backward substitution for the color of positions [c0, c0 + cnt), in place:
// z_i = U_ii^-1 (y_i - sum_{upper} U_ij z_j).  The result, plus Pi_P e_P when
// ep != nullptr, is also written to out (FP64, natural block row border[i]).
template <class T, int G>
__global__ void k_bilu_bwd(int c0, int cnt, const int *__restrict__ ur,
                           const int *__restrict__ uc, const T *__restrict__ uv,
                           const T *__restrict__ dinv, T *y, const T *ep, const int *__restrict__ border,
                           double *out_base, long ld, const int *jptr, const int *done) {
    constexpr int kPreB = G == 1 ? 3 : 2;   // blocks per lane loaded before the wait
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long t = tid / G;
    int lane = (int)(tid % G);
    bool active = t < cnt;
    bool lead = active && lane == 0;
    int i = c0 + (int)t;
    int e0 = 0, e1 = 0, bi = 0;
    T D[9];
    if (active) {
        e0 = ur[i];
        e1 = ur[i + 1];
    }
    if (lead) bi = border[i];
#pragma unroll
    for (int k = 0; k < 9; k++) D[k] = lead ? dinv[9 * (size_t)i + k] : (T)0;
    int cj[kPreB];
    T Up[kPreB][9];
#pragma unroll
    for (int u = 0; u < kPreB; u++) {
        int p = e0 + lane + u * G;
        bool in = p < e1;
        cj[u] = in ? uc[p] : 0;
#pragma unroll
        for (int k = 0; k < 9; k++) Up[u][k] = in ? uv[9 * (size_t)p + k] : (T)0;
    }
    pdl_wait();
    pdl_trigger();
    int dn = stop_flag(done);   // tested before the first store, not ahead of the gathers
    // where the result goes, and the V-cycle's part of it, are loaded before
    // the gathers: the stores at the end then wait on nothing
    double *out = out_base + (size_t)step_of(jptr) * ld + 3 * (size_t)bi;
    double e0v = lead && ep ? (double)ep[i] : 0.0;
    T s0, s1, s2;
    if constexpr (G == 1) {
        if (!active) return;
        s0 = y[3 * (size_t)i], s1 = y[3 * (size_t)i + 1], s2 = y[3 * (size_t)i + 2];
#pragma unroll
        for (int u = 0; u < kPreB; u++)
            if (e0 + u < e1) {
                const T *U = Up[u];
                const T *zj = y + 3 * (size_t)cj[u];
                T z0 = zj[0], z1 = zj[1], z2 = zj[2];
                s0 -= U[0] * z0 + U[1] * z1 + U[2] * z2;
                s1 -= U[3] * z0 + U[4] * z1 + U[5] * z2;
                s2 -= U[6] * z0 + U[7] * z1 + U[8] * z2;
            }
#pragma unroll 4
        for (int p = e0 + kPreB; p < e1; p++) {
            const T *U = uv + 9 * (size_t)p;
            const T *zj = y + 3 * (size_t)uc[p];
            T z0 = zj[0], z1 = zj[1], z2 = zj[2];
            s0 -= U[0] * z0 + U[1] * z1 + U[2] * z2;
            s1 -= U[3] * z0 + U[4] * z1 + U[5] * z2;
            s2 -= U[6] * z0 + U[7] * z1 + U[8] * z2;
        }
    } else {
        // the row's own y_i is loaded with the gathers, not after them
        T yi0 = lead ? y[3 * (size_t)i] : (T)0, yi1 = lead ? y[3 * (size_t)i + 1] : (T)0,
          yi2 = lead ? y[3 * (size_t)i + 2] : (T)0;
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int u = 0; u < kPreB; u++)
            if (e0 + lane + u * G < e1) {
                const T *U = Up[u];
                const T *zj = y + 3 * (size_t)cj[u];
                T z0 = zj[0], z1 = zj[1], z2 = zj[2];
                a0 += U[0] * z0 + U[1] * z1 + U[2] * z2;
                a1 += U[3] * z0 + U[4] * z1 + U[5] * z2;
                a2 += U[6] * z0 + U[7] * z1 + U[8] * z2;
            }
        for (int p = e0 + lane + kPreB * G; p < e1; p += G) {
            const T *U = uv + 9 * (size_t)p;
            const T *zj = y + 3 * (size_t)uc[p];
            T z0 = zj[0], z1 = zj[1], z2 = zj[2];
            a0 += U[0] * z0 + U[1] * z1 + U[2] * z2;
            a1 += U[3] * z0 + U[4] * z1 + U[5] * z2;
            a2 += U[6] * z0 + U[7] * z1 + U[8] * z2;
        }
        a0 = group_sum(a0, G);
        a1 = group_sum(a1, G);
        a2 = group_sum(a2, G);
        if (!lead) return;
        s0 = yi0 - a0;
        s1 = yi1 - a1;
        s2 = yi2 - a2;
    }
    T z0 = D[0] * s0 + D[1] * s1 + D[2] * s2;
    T z1 = D[3] * s0 + D[4] * s1 + D[5] * s2;
    T z2 = D[6] * s0 + D[7] * s1 + D[8] * s2;
    if (dn) return;
    y[3 * (size_t)i] = z0;
    y[3 * (size_t)i + 1] = z1;
    y[3 * (size_t)i + 2] = z2;
    out[0] = (double)z0 + e0v;
    out[1] = (double)z1;
    out[2] = (double)z2;
}

}  // namespace
}  // namespace cpr
