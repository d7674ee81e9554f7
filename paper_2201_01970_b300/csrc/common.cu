// Shared host utilities: errors, scans, small device reads.
#include <atomic>
#include <cstdio>
#include <mutex>
#include <vector>

#include "cpr_internal.cuh"

namespace cpr {

void fail(int code, const std::string &what) { throw Error{code, what}; }

DeviceGuard::DeviceGuard(int dev) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != dev) {
        CK(cudaSetDevice(dev));
        prev = cur;
    }
}
DeviceGuard::~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
}

// Library-wide device bytes and their cap (0 = no cap).
static std::atomic<unsigned long long> g_bytes{0}, g_cap{0};

void reserve_bytes(size_t bytes) {
    unsigned long long cap = g_cap.load(std::memory_order_relaxed);
    unsigned long long now = g_bytes.fetch_add(bytes, std::memory_order_relaxed) + bytes;
    if (cap && now > cap) {
        g_bytes.fetch_sub(bytes, std::memory_order_relaxed);
        fail(CPR_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes would pass the library's "
                          "memory limit of " + std::to_string(cap) + " bytes");
    }
}
void unreserve_bytes(size_t bytes) { g_bytes.fetch_sub(bytes, std::memory_order_relaxed); }

static unsigned long long g_launches = 0;
static thread_local bool t_capturing = false;
void count_launch() {
    if (!t_capturing) __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
}
void count_launches(unsigned long long n) { __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED); }
void set_capturing(bool on) { t_capturing = on; }

unsigned long long graph_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    CK(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) CK(cudaGraphGetNodes(g, nodes.data(), &n));
    unsigned long long k = 0;
    for (size_t i = 0; i < n; i++) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void check_cuda(cudaError_t e, const char *expr, const char *file, int line) {
    if (e == cudaSuccess) return;
    int code = e == cudaErrorMemoryAllocation ? CPR_ERR_OOM : CPR_ERR_CUDA;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed at %s:%d: %s", expr, file, line, cudaGetErrorString(e));
    fail(code, buf);
}

// Two pools per device: 0 for the handle's own stream, 1 for the setup's side
// worker thread (selected per host thread), so buffers allocated and freed on
// the side stream never interleave with the main stream's in one pool.
static thread_local int t_pool = 0;
void use_side_pool(bool on) { t_pool = on ? 1 : 0; }

cudaMemPool_t library_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64][2] = {};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(CPR_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev][t_pool]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CK(cudaMemPoolCreate(&pools[dev][t_pool], &props));
        uint64_t keep = UINT64_MAX;
        CK(cudaMemPoolSetAttribute(pools[dev][t_pool], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    return pools[dev][t_pool];
}

int grid_for(long n, int block, int cap) {
    long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------- scan
// Exclusive scan of n ints into n+1 outputs (out[n] = total): per-tile sums,
// a recursive scan of the tile sums, then a per-tile scan plus the offset.

namespace {
constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ int block_exclusive_scan(int v, int *total) {
    __shared__ int warp_sums[kScanBlock / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kScanBlock / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanBlock / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (wid > 0 ? warp_sums[wid - 1] : 0);
    *total = warp_sums[kScanBlock / 32 - 1];
    __syncthreads();
    return excl;
}

__global__ void k_tile_sums(const int *in, int n, int *sums) {
    long base = (long)blockIdx.x * kScanTile;
    int s = 0;
    for (int k = 0; k < kScanItems; k++) {
        long i = base + (long)k * kScanBlock + threadIdx.x;
        if (i < n) s += in[i];
    }
    int total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_tile_scan(const int *in, int n, const int *tile_off, int *out) {
    long base = (long)blockIdx.x * kScanTile;
    int v[kScanItems];
    int s = 0;
    for (int k = 0; k < kScanItems; k++) {
        long i = base + (long)threadIdx.x * kScanItems + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int total;
    int excl = block_exclusive_scan(s, &total) + (tile_off ? tile_off[blockIdx.x] : 0);
    for (int k = 0; k < kScanItems; k++) {
        long i = base + (long)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = excl;
        excl += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanBlock - 1) out[n] = excl;
}
// Whole scan in one CTA for up to kScanSingleMax elements (one launch
// instead of three): a coalesced copy of the input into shared memory
// (skewed by one word per 32 against bank conflicts), one contiguous chunk
// per thread summed there, one block scan of the chunk sums, the chunk's
// prefixes written back in place, and a coalesced copy out.
constexpr int kScanSingleMax = 8 * kScanTile;
constexpr int kScanSingleSmem = (kScanSingleMax + kScanSingleMax / 32) * (int)sizeof(int);
__device__ __forceinline__ int skew32(int i) { return i + (i >> 5); }
__global__ void __launch_bounds__(kScanBlock) k_scan_single(const int *in, int n, int *out) {
    extern __shared__ int sm[];
    for (int i = threadIdx.x; i < n; i += kScanBlock) sm[skew32(i)] = in[i];
    __syncthreads();
    int chunk = (n + kScanBlock - 1) / kScanBlock;
    int b = threadIdx.x * chunk, e = min(b + chunk, n);
    int s = 0;
#pragma unroll 8
    for (int i = b; i < e; i++) s += sm[skew32(i)];
    int total;
    int excl = block_exclusive_scan(s, &total);
    for (int i = b; i < e; i++) {
        int v = sm[skew32(i)];
        sm[skew32(i)] = excl;
        excl += v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kScanBlock) out[i] = sm[skew32(i)];
    if (threadIdx.x == 0) out[n] = total;
}

// The shared-memory ceiling of k_scan_single, set once per device.
void scan_single_attr() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    CK(cudaFuncSetAttribute(k_scan_single, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSingleSmem));
    done.fetch_or(bit, std::memory_order_release);
}
}  // namespace

void exclusive_scan(const int *in, int *out, int n, cudaStream_t s) {
    if (n <= 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(int), s));
        return;
    }
    int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_tile_scan<<<1, kScanBlock, 0, s>>>(in, n, nullptr, out);
        CK_LAUNCH();
        return;
    }
    if (n <= kScanSingleMax) {
        scan_single_attr();
        k_scan_single<<<1, kScanBlock, kScanSingleSmem, s>>>(in, n, out);
        CK_LAUNCH();
        return;
    }
    DVec<int> sums, offs;
    sums.alloc(tiles, s);
    offs.alloc(tiles + 1, s);
    k_tile_sums<<<tiles, kScanBlock, 0, s>>>(in, n, sums.p);
    CK_LAUNCH();
    exclusive_scan(sums.p, offs.p, tiles, s);
    k_tile_scan<<<tiles, kScanBlock, 0, s>>>(in, n, offs.p, out);
    CK_LAUNCH();
}

int read_int(const int *dptr, cudaStream_t s) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, dptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return v;
}

// Hash weight of vertex i is fmix32(i ^ base), base = fmix32(seed32 + 1000003*salt + level);
// salt 0 = smoother coloring, 1 = PMIS, 2 = BILU coloring (MurmurHash3's finalizer).
uint32_t hash_base(uint64_t seed, int salt, int level) {
    uint32_t s32 = (uint32_t)(seed ^ (seed >> 32));
    return fmix32(s32 + 1000003u * (uint32_t)salt + (uint32_t)level);
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace cpr

extern "C" {

void cpr_set_memory_limit(uint64_t bytes) { cpr::g_cap.store(bytes, std::memory_order_relaxed); }

uint64_t cpr_memory_in_use(void) { return cpr::g_bytes.load(std::memory_order_relaxed); }

}  // extern "C"
