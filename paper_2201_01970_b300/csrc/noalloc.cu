// cpr_bilu_apply_noalloc: the second-stage BILU(0) application of
// cpr_bilu_apply, for callers that must not allocate device memory when they
// call it.  Examples: a simulator that reserves its whole device-memory budget
// at start-up and forbids allocation later, and host code that runs while
// another component owns the allocator (an allocation there would fail, or
// would synchronize the device).  The forward/backward sweeps need one work
// vector of 3*nb values; here it lives in a file-scope device array that is
// sized once, at load time, instead of in memory the handle allocates.
//
// The array holds kNoAllocMaxBlockRows block rows (1.5 MiB).  Every GPU that
// loads this library keeps that much memory until the process exits.
#include <mutex>

#include "cpr_internal.cuh"

namespace cpr {
namespace {

constexpr int kNoAllocMaxBlockRows = 1 << 16;
constexpr int kBlock = 256;
constexpr int kMaxDevices = 64;

// The sweep vector: 3 doubles per block row (reused as 3 floats per block row
// in FP32 mode).  In host code this name is only a stand-in for the symbol;
// host code passes the device address from cudaGetSymbolAddress instead.
static __device__ __align__(256) double g_bilu_scratch[3 * kNoAllocMaxBlockRows];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (at that device's first call).
void *scratch_address() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(CPR_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bilu_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(CPR_ERR_CUDA, std::string("cudaGetSymbolAddress of the BILU scratch failed: ") +
                                   cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

// y (block rows in the factors' color order) <- r (natural order).
template <class T>
__global__ void k_load(int nb, const int *order, const double *r, T *y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const double *src = r + 3 * (size_t)order[t];
    y[3 * (size_t)t] = (T)src[0];
    y[3 * (size_t)t + 1] = (T)src[1];
    y[3 * (size_t)t + 2] = (T)src[2];
}

// Forward substitution of one color's positions [c0, c0 + cnt) on the scratch
// vector (as cpr_bilu_apply's).
template <class T>
__global__ void k_fwd(int c0, int cnt, const int *__restrict__ lr, const int *__restrict__ lc,
                      const T *__restrict__ lv, T *y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = c0 + t;
    T s0 = y[3 * (size_t)i], s1 = y[3 * (size_t)i + 1], s2 = y[3 * (size_t)i + 2];
    for (int p = lr[i]; p < lr[i + 1]; p++) {
        const T *L = lv + 9 * (size_t)p;
        const T *yj = y + 3 * (size_t)lc[p];
        T y0 = yj[0], y1 = yj[1], y2 = yj[2];
        s0 -= L[0] * y0 + L[1] * y1 + L[2] * y2;
        s1 -= L[3] * y0 + L[4] * y1 + L[5] * y2;
        s2 -= L[6] * y0 + L[7] * y1 + L[8] * y2;
    }
    y[3 * (size_t)i] = s0;
    y[3 * (size_t)i + 1] = s1;
    y[3 * (size_t)i + 2] = s2;
}

// Backward substitution of one color's positions; writes z (FP64, natural
// block row order[i]) as well.
template <class T>
__global__ void k_bwd(int c0, int cnt, const int *__restrict__ ur, const int *__restrict__ uc,
                      const T *__restrict__ uv, const T *__restrict__ dinv, T *y, const int *order, double *z) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = c0 + t;
    T s0 = y[3 * (size_t)i], s1 = y[3 * (size_t)i + 1], s2 = y[3 * (size_t)i + 2];
    for (int p = ur[i]; p < ur[i + 1]; p++) {
        const T *U = uv + 9 * (size_t)p;
        const T *zj = y + 3 * (size_t)uc[p];
        T z0 = zj[0], z1 = zj[1], z2 = zj[2];
        s0 -= U[0] * z0 + U[1] * z1 + U[2] * z2;
        s1 -= U[3] * z0 + U[4] * z1 + U[5] * z2;
        s2 -= U[6] * z0 + U[7] * z1 + U[8] * z2;
    }
    const T *D = dinv + 9 * (size_t)i;
    T z0 = D[0] * s0 + D[1] * s1 + D[2] * s2;
    T z1 = D[3] * s0 + D[4] * s1 + D[5] * s2;
    T z2 = D[6] * s0 + D[7] * s1 + D[8] * s2;
    y[3 * (size_t)i] = z0;
    y[3 * (size_t)i + 1] = z1;
    y[3 * (size_t)i + 2] = z2;
    double *zi = z + 3 * (size_t)order[i];
    zi[0] = (double)z0;
    zi[1] = (double)z1;
    zi[2] = (double)z2;
}

template <class T>
void sweeps(cpr_handle *h, const double *r, double *z, T *y, const T *lv, const T *uv, const T *dv) {
    cudaStream_t s = h->stream;
    Bilu &B = h->bilu;
    int nb = h->nb;
    // every entry of y that the sweeps read is written here first, so no part
    // of the scratch has to start at zero
    k_load<T><<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, B.rows_by_color.p, r, y);
    CK_LAUNCH();
    for (int c = 0; c < B.ncolors; c++) {
        int cnt = B.color_off[c + 1] - B.color_off[c];
        if (!cnt) continue;
        k_fwd<T><<<grid_for(cnt, kBlock), kBlock, 0, s>>>(B.color_off[c], cnt, B.Lrowptr.p, B.Lcol.p, lv, y);
        CK_LAUNCH();
    }
    for (int c = B.ncolors - 1; c >= 0; c--) {
        int cnt = B.color_off[c + 1] - B.color_off[c];
        if (!cnt) continue;
        k_bwd<T><<<grid_for(cnt, kBlock), kBlock, 0, s>>>(B.color_off[c], cnt, B.Urowptr.p, B.Ucol.p, uv, dv, y,
                                                         B.rows_by_color.p, z);
        CK_LAUNCH();
    }
}

}  // namespace
}  // namespace cpr

using namespace cpr;

extern "C" int cpr_bilu_apply_noalloc(cpr_handle *h, const double *r, double *z) {
    if (!h || !r || !z) return CPR_ERR_INVALID;
    try {
        if (h->nb > kNoAllocMaxBlockRows)
            fail(CPR_ERR_INVALID, "cpr_bilu_apply_noalloc supports at most " +
                                      std::to_string(kNoAllocMaxBlockRows) + " block rows; this system has " +
                                      std::to_string(h->nb));
        void *y = scratch_address();
        if (h->opt.precond_fp32)
            sweeps<float>(h, r, z, (float *)y, h->bilu.Lval32.p, h->bilu.Uval32.p, h->bilu.Dinv32.p);
        else
            sweeps<double>(h, r, z, (double *)y, h->bilu.Lval.p, h->bilu.Uval.p, h->bilu.Dinv.p);
        CK(cudaStreamSynchronize(h->stream));
        return CPR_OK;
    } catch (const Error &e) {
        set_last_error(e.what);
        return e.code;
    }
}
