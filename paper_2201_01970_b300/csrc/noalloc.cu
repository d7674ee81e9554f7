// cpr_bilu_apply_noalloc: the second-stage BILU(0) application of
// cpr_bilu_apply, for callers that must not allocate device memory when they
// call it.  Examples: a simulator that reserves its whole device-memory budget
// at start-up and forbids allocation later, and host code that runs while
// another component owns the allocator (an allocation there would fail, or
// would synchronize the device).  The forward/backward sweeps need one work
// vector of 3*nb values; here it lives in a file-scope device array of a fixed
// maximum size instead of in memory the handle allocates.
//
// The array holds kNoAllocMaxBlockRows block rows (1.5 MiB).  The library's
// device code for this file is a module of its own, which CUDA maps onto a
// device (and so allocates the array there) the first time its address is
// looked up.  cpr_setup does that lookup on the handle's device, where an
// allocation is allowed, and loads the entry's kernels there, so a later call
// finds both in place; every device that has had a handle set up keeps the
// 1.5 MiB until the process exits.
#include <mutex>

#include "cpr_internal.cuh"
#include "sweeps.cuh"

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

// Device address of the scratch array on device `dev` (which must be
// current), looked up once per device.
void *scratch_address(int dev) {
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

template <class T>
void sweeps(cpr_handle *h, const double *r, double *z, T *y, const T *lv, const T *uv, const T *dv) {
    cudaStream_t s = h->stream;
    Bilu &B = h->bilu;
    int nb = h->nb;
    // the same sweep kernels, lane split and color order as cpr_bilu_apply, so
    // the two entries agree bit for bit
    constexpr int G = sizeof(T) == 4 ? kBiluLanesF32 : 1;
    // every entry of y that the sweeps read is written here first, so no part
    // of the scratch has to start at zero
    k_load<T><<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, B.rows_by_color.p, r, y);
    CK_LAUNCH();
    for (int c = 1; c < B.ncolors; c++) {   // the lowest color has no lower neighbours
        int cnt = B.color_off[c + 1] - B.color_off[c];
        if (!cnt) continue;
        k_bilu_fwd<T, G><<<grid_for((long)cnt * G, kBlock), kBlock, 0, s>>>(B.color_off[c], cnt, B.Lrowptr.p,
                                                                           B.Lcol.p, lv, y, nullptr);
        CK_LAUNCH();
    }
    for (int c = B.ncolors - 1; c >= 0; c--) {
        int cnt = B.color_off[c + 1] - B.color_off[c];
        if (!cnt) continue;
        k_bilu_bwd<T, G><<<grid_for((long)cnt * G, kBlock), kBlock, 0, s>>>(
            B.color_off[c], cnt, B.Urowptr.p, B.Ucol.p, uv, dv, y, nullptr, B.rows_by_color.p, z, 0, nullptr,
            nullptr);
        CK_LAUNCH();
    }
}

}  // namespace

// Called by cpr_setup with the handle's device current: maps the array and,
// with CUDA's lazy loading, loads the code of every kernel the entry launches,
// so that neither happens inside a later call.
void noalloc_prepare() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    scratch_address(dev);
    static std::mutex mu;
    static bool loaded[kMaxDevices] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (loaded[dev]) return;
    cudaFuncAttributes a;
    CK(cudaFuncGetAttributes(&a, k_load<float>));
    CK(cudaFuncGetAttributes(&a, k_load<double>));
    CK(cudaFuncGetAttributes(&a, k_bilu_fwd<float, kBiluLanesF32>));
    CK(cudaFuncGetAttributes(&a, k_bilu_fwd<double, 1>));
    CK(cudaFuncGetAttributes(&a, k_bilu_bwd<float, kBiluLanesF32>));
    CK(cudaFuncGetAttributes(&a, k_bilu_bwd<double, 1>));
    loaded[dev] = true;
}

}  // namespace cpr

using namespace cpr;

extern "C" int cpr_bilu_apply_noalloc(cpr_handle *h, const double *r, double *z) {
    if (!h || !r || !z) return CPR_ERR_INVALID;
    return guarded([&] {
        // the handle's device, whichever device the caller has current
        DeviceGuard dg(h->device);
        if (h->nb > kNoAllocMaxBlockRows)
            fail(CPR_ERR_INVALID, "cpr_bilu_apply_noalloc supports at most " +
                                      std::to_string(kNoAllocMaxBlockRows) + " block rows; this system has " +
                                      std::to_string(h->nb));
        void *y = scratch_address(h->device);
        if (h->opt.precond_fp32)
            sweeps<float>(h, r, z, (float *)y, h->bilu.Lval32.p, h->bilu.Uval32.p, h->bilu.Dinv32.p);
        else
            sweeps<double>(h, r, z, (double *)y, h->bilu.Lval.p, h->bilu.Uval.p, h->bilu.Dinv.p);
        CK(cudaStreamSynchronize(h->stream));
        return CPR_OK;
    });
}
