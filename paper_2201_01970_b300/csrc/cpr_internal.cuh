// Internal declarations of the B300 CPR-FGMRES library: device buffers, the
// handle, the hierarchy, and the host-side entry points of each part.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "cpr.h"

namespace cpr {

// ------------------------------------------------------------------ errors

struct Error {
    int code;
    std::string what;
};

[[noreturn]] void fail(int code, const std::string &what);

// The text of the calling thread's last failure (cpr_last_error_detail).
void set_last_error(const std::string &what);

// Runs f() and maps every exception to a return code, so that nothing escapes
// a C-ABI function: library errors keep their code, a failed host allocation
// is CPR_ERR_OOM, anything else CPR_ERR_CUDA.
template <class F>
int guarded(F f) {
    try {
        return f();
    } catch (const Error &e) {
        set_last_error(e.what);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return CPR_ERR_OOM;
    } catch (...) {
        set_last_error("unknown failure");
        return CPR_ERR_CUDA;
    }
}

// Makes `dev` the current device for one entry point's work and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// Device bytes held by the library in this process, against the cap set with
// cpr_set_memory_limit: reserve_bytes fails with CPR_ERR_OOM beyond the cap.
void reserve_bytes(size_t bytes);
void unreserve_bytes(size_t bytes);
void check_cuda(cudaError_t e, const char *expr, const char *file, int line);
#define CK(x) ::cpr::check_cuda((x), #x, __FILE__, __LINE__)
void count_launch();                      // one kernel launched (not counted while capturing)
void count_launches(unsigned long long n); // n kernels launched through a graph
void set_capturing(bool on);              // this thread is capturing a graph
unsigned long long graph_kernel_nodes(cudaGraph_t g);
#define CK_LAUNCH()                                                                   \
    do {                                                                              \
        ::cpr::count_launch();                                                        \
        ::cpr::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__);   \
    } while (0)

// An NVTX range for the life of the object (visible in Nsight timelines; no
// cost without a profiler attached).  Ranges name the entry points, the setup's
// phases and, outside graph capture, the kernel families of a B application.
struct Nvtx {
    explicit Nvtx(const char *name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
    Nvtx(const Nvtx &) = delete;
    Nvtx &operator=(const Nvtx &) = delete;
};

// ------------------------------------------------------------ device buffers

// The library's stream-ordered memory pool on the current device.  Its release
// threshold is unlimited: memory freed by one setup is reused by the next
// instead of going back to the driver at every synchronisation.
cudaMemPool_t library_pool();
void use_side_pool(bool on);   // this host thread allocates from the side pool

// Stream-ordered device allocation from the library pool; move-only.
template <class T>
struct DVec {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DVec() = default;
    DVec(const DVec &) = delete;
    DVec &operator=(const DVec &) = delete;
    DVec(DVec &&o) noexcept { *this = std::move(o); }
    DVec &operator=(DVec &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            s = o.s;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DVec() { release(); }
    void alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        if (count) {
            reserve_bytes(count * sizeof(T));
            cudaError_t e = cudaMallocFromPoolAsync((void **)&p, count * sizeof(T), library_pool(), stream);
            if (e != cudaSuccess) {
                unreserve_bytes(count * sizeof(T));
                p = nullptr;
                if (e == cudaErrorMemoryAllocation) {
                    cudaGetLastError();
                    fail(CPR_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes");
                }
                CK(e);
            }
        }
        n = count;
    }
    void zero() {
        if (n) CK(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    void release() {
        if (p) {
            cudaFreeAsync(p, s);
            unreserve_bytes(n * sizeof(T));
        }
        p = nullptr;
        n = 0;
    }
};

// Scalar CSR matrix on the device.
struct DCsr {
    int n = 0, ncol = 0, nnz = 0;
    DVec<int> rowptr, col;
    DVec<double> val;
};

// The product lists of a sparse product C = A B on C's pattern: entry c of C
// is the sum, in list order (ascending k), of av[pa[t]] * bv[pb[t]] for t in
// [ptr[c], ptr[c+1]).
struct ProdPlan {
    DVec<int> ptr, pa, pb;
};

// One AMG level.  A, P, R hold the setup result in natural numbering
// (bit-identical to the plain definition's; used for inspection).  The solve
// uses copies renumbered into color order, so each color is a contiguous row
// range [color_off[c], color_off[c+1]): Ao (A without its diagonal), diag and
// dinv, Pp (rows in this level's order, columns in the next level's), Rp.
struct Level {
    DCsr A, P, R;
    DVec<int> color, cf;
    int ncolors = 0, nc = 0;
    DVec<int> Srow, Scol;         // classical strength set the interpolation used (kept for resetup = 1)
    int Snnz = 0;
    std::vector<int> color_off;
    DVec<int> rows_by_color;      // order: internal row t is natural row rows_by_color[t]
    DVec<int> iperm;              // natural row i is internal row iperm[i]
    DCsr Ao, Pp, Rp;
    DVec<double> diag, dinv;      // internal numbering
    DVec<float> Aoval32, Ppval32, Rpval32, diag32, dinv32;
    int gA = 8, gP = 4, gR = 8;   // lanes per row of the solve kernels
    int bs = 256;                 // threads per CTA of the level's V-cycle kernels
    // work vectors (internal numbering); s0, s1: staging of the color being relaxed
    DVec<double> x, b, r, s0, s1;
    DVec<float> x32, b32, r32, s0_32, s1_32;
    // resetup = 1: what the in-place numeric refresh needs besides the above
    DVec<int> dpos;               // position of each row's diagonal in A
    DVec<int> cidx;               // coarse index of each C point (classical AMG)
    DCsr AP;                      // the Galerkin product's left factor A P
    ProdPlan pap, prap;           // the product lists of A P and R (A P)
    // amg = 1, levels 1 .. L-2: the GCR vectors of this level's coarse
    // correction (amli_iters x n each), its scalars and reduction partials
    DVec<double> gv, gw, gscal, gpart;
    DVec<float> gv32, gw32;
    DVec<int> gcnt;
};

// Multicolor BILU(0).  The factor array lu (lu32 in FP32 mode) is in A's
// pattern and natural numbering (inspection).  The sweeps use block rows
// renumbered into color order (position t holds natural row rows_by_color[t],
// each color a contiguous range [color_off[c], color_off[c+1])): L (lower
// colors), U (higher colors) and D^-1 with rows and columns in positions.
struct Bilu {
    int pattern = -1;              // the handle's pattern_id the structure below was built for
    DVec<int> color;
    int ncolors = 0;
    std::vector<int> color_off;
    DVec<int> rows_by_color;       // position -> natural block row
    DVec<int> iperm;               // natural block row -> position
    DVec<double> lu;
    DVec<float> lu32;
    DVec<int> Lrowptr, Lcol, Urowptr, Ucol;
    int nl = 0, nu = 0;            // entries of L and U
    DVec<double> Lval, Uval, Dinv;
    DVec<float> Lval32, Uval32, Dinv32;
};

// Many independent systems concatenated into one block-diagonal operator: the
// preconditioner runs on the concatenation, the Krylov process per system.
struct BatchInfo {
    int nsys = 0;
    std::vector<int> boff;        // block-row offset of each system (nsys + 1)
    int nchunk = 0;               // vector chunks, each inside one system
    DVec<int> chunk_sys, chunk_beg, chunk_end;
    DVec<int> sys_chunk_off;      // chunks of system s: [sys_chunk_off[s], sys_chunk_off[s+1])
    DVec<double> scal;            // per-system scalar blocks (Hessenberg, rotations, g, y, norms)
    DVec<int> sint;               // per-system ints: done, steps this cycle, breakdown, converged, total steps
    DVec<double> part, part2;     // chunk partial sums
    DVec<double> b, x;            // concatenated right-hand sides and iterates
};

}  // namespace cpr

namespace cpr {
// A solve in progress: FGMRES (Alg. 2) as a state machine that the blocking
// cpr_solve drives to the end and cpr_solve_poll advances without waiting.
struct FgmresState {
    enum { IDLE = 0, START = 1, WAIT_START = 2, STEPS = 3, WAIT_FINAL = 4, DONE = 5 };
    int phase = IDLE;
    const double *b = nullptr;   // device right-hand side
    double *x = nullptr;         // device iterate
    double *x_out = nullptr;     // the caller's host x, written at the end (null: x is the caller's)
    double rtol = 0.0, norm0 = 0.0, rnorm = 0.0, t0 = 0.0;
    int cycle = 0, cycles = 0, iters = 0, rc = 0;
    int launched = 0, checked = 0, steps = 0;
    bool stop = false;
};
}  // namespace cpr

// The opaque handle of the C ABI.
struct cpr_handle {
    cpr_opts opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;      // setup's side worker stream (created on first use)
    cudaStream_t lu_stream = nullptr; // setup's coarse factorisation stream (created on first use)
    cudaEvent_t ev_coarse[2] = {nullptr, nullptr};  // main -> LU stream -> main around the coarse factorisation
    std::vector<cudaEvent_t> ev_color;              // per level: its coloring's stream work is complete
    // Sliced-ELL copy of the outer operator for the SpMV: slices of 32 block
    // rows; slot k of a slice holds each of its rows' k-th block (column -1
    // past a row's end), the nine values of a slot lane-contiguous per block
    // entry, so a warp's loads are contiguous.  Refreshed with every new A.
    cpr::DVec<int> sell_off, sell_col;
    cpr::DVec<double> sell_val;
    int sell_slices = 0;
    bool sell_ok = false;
    bool own_stream = false;
    int device = 0;                 // the CUDA device the handle was set up on
    int nb = 0, nnzb = 0;
    cpr::DVec<int> rowptr, col;     // outer operator A^(k) (copy)
    cpr::DVec<double> val;
    // bumped whenever A's block pattern changes (cpr_setup, cpr_update with a new pattern)
    int pattern_id = 0;
    // --- the preconditioner B (frozen between setups) ---
    bool have_B = false;
    // column 0 of every block of the A that B was built from (Alg. 1, second residual),
    // rows and columns in BILU positions
    cpr::DVec<int> c0rowptr, c0col;
    cpr::DVec<double> pcol0;
    cpr::DVec<float> pcol0_32;
    cpr::DVec<int> ep_map;          // level-0 solve row -> BILU position (final V-cycle commit)
    cpr::DVec<double> w;            // decoupling weights, 3 per block row
    cpr::DVec<float> w32;
    std::vector<cpr::Level> lev;
    int cn = 0;                     // coarsest size
    cpr::DVec<double> cinv;         // dense inverse of the coarsest A, row-major
    cpr::Bilu bilu;
    // --- Krylov workspace ---
    int m_alloc = 0;
    cpr::DVec<double> V, Z, wv, r;  // V: (m+1) x N, Z: m x N
    cpr::DVec<double> dscal;        // device scalars (H, g, cs, sn, norms)
    cpr::DVec<double> red;          // reduction partials
    cpr::DVec<int> dint;            // device ints (step index, flags)
    cpr::DVec<float> t32a, t32b;    // FP32 vectors of length 3*nb inside B
    cpr::DVec<double> t64a;         // FP64 vector of length 3*nb inside B
    cpr::DVec<double> ep64;         // e_P = B_P r_P in BILU positions
    cpr::DVec<float> ep32;
    cpr::DVec<double> dev_b, dev_x; // device copies of host b / x
    double *pinned = nullptr;       // pinned host scalars
    int *pinned_dev_flags = nullptr; // device address of the two step-flag slots in pinned (at pinned + 8)
    cpr::DVec<int> err;             // device error flag
    // resetup = 1: the in-place numeric refresh of B (numeric_refresh) and its graph
    bool nr_ready = false;          // the last full setup kept what the refresh needs
    cpr::DVec<int> bdiag;           // each block row's diagonal position
    cpr::DVec<double> c_a, c_lu;    // coarse factorisation scratch
    cpr::DVec<int> c_piv;
    cudaGraph_t nr_graph = nullptr;
    cudaGraphExec_t nr_exec = nullptr;
    unsigned long long nr_kernels = 0;
    cudaEvent_t ev_nr[4] = {nullptr, nullptr, nullptr, nullptr};   // fork/join of its side branches
    // --- adaptive state (Alg. 3) ---
    long last_iters = -1;
    int setup_count = 0, setup_called = 0, updates = 0;
    double setup_ms = 0.0;
    // --- event brackets of kernel families (cpr_profile) ---
    bool prof = false;
    unsigned prof_mask = 0;           // families bracketed while prof is on (bit f = family f)
    static constexpr int kProfSlots = 512;
    cudaEvent_t ev_a[kProfSlots] = {}, ev_b[kProfSlots] = {};
    int ev_fam[kProfSlots] = {};
    int ev_n = 0;
    std::vector<int> prof_open;      // open (possibly nested) brackets: slot or graph-event index, -1 = dropped
    long prof_cnt[CPR_PROF_NFAMILIES] = {};
    double prof_ms[CPR_PROF_NFAMILIES] = {};
    // --- graphs of one Arnoldi step (two instances, used on alternate steps) ---
    int epoch = 0;                   // bumped whenever B or the workspace changes
    struct StepGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> ev_a, ev_b;   // event-record nodes (profiling)
        std::vector<int> fam;
        unsigned long long kernels = 0;        // kernel nodes: launches per graph launch
    } sg[2];
    int sg_epoch = -1;
    unsigned sg_prof = 0;            // prof_mask the step graphs were captured with (0: none)
    int capturing = -1;              // index of the step graph being captured, -1 = none
    StepGraph sgb[2];                // the batched step graphs
    int sgb_epoch = -1;
    cpr::BatchInfo *batch = nullptr;
    cudaEvent_t step_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_norm = nullptr;   // a cycle's start (residual norm, flags) is on the host
    cpr::FgmresState fs;
    cpr::DVec<int> bflag;            // b holds a NaN or Inf (checked with the first norm)
    int tail_top = -1;               // first level run by the cluster tail kernel, -1 = none
    // V-cycle schedules chosen by cpr_autotune, keyed by a level's (rows, nonzeros);
    // a setup that builds a level of a known signature takes its schedule
    std::map<std::pair<int, long>, cpr_schedule> sched;
};

namespace cpr {

constexpr int kMaxRestart = 64;
constexpr int kMaxCoarse = 4096;
constexpr int kMaxAmli = 8;             // GCR steps of an AMLI coarse correction
constexpr int kMaxGroupingRows = 16384; // largest level Alg. 4-5 colors on the device

int grid_for(long n, int block, int cap = 1 << 30);

// MurmurHash3's 32-bit finalizer (Appleby's published mixing function): the
// bijective hash of the coloring, C/F splitting and matching keys.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
void exclusive_scan(const int *in, int *out, int n, cudaStream_t s);   // out has n+1 entries
int read_int(const int *dptr, cudaStream_t s);
uint32_t hash_base(uint64_t seed, int salt, int level);
bool is_device_ptr(const void *p);

// event brackets (api.cu)
void prof_begin(cpr_handle *h, int family);
void prof_end(cpr_handle *h);
void prof_flush(cpr_handle *h);
void prof_collect_graph(cpr_handle *h, int which);
void destroy_step_graphs(cpr_handle *h);

// setup.cu
// The full setup of B from the handle's current A; with resetup = 1 it also
// keeps what numeric_refresh needs.
void build_preconditioner(cpr_handle *h);
void free_preconditioner(cpr_handle *h);
// resetup = 1 with an unchanged pattern: every value of B recomputed from the
// current A in place (the structure of the last full setup kept), replayed as
// one CUDA graph; the step graphs stay valid
void numeric_refresh(cpr_handle *h);
void refresh_second_residual(cpr_handle *h);   // reuse_refresh: the kept B's copy of A := the current A

// noalloc.cu: resolve (and so load) the allocation-free entry's scratch array
// on the current device
void noalloc_prepare();
void validate_bsr(const int *rowptr, const int *col, int nb, int nnzb, int *derr, cudaStream_t s);

// solve.cu
void ensure_workspace(cpr_handle *h);
void apply_B(cpr_handle *h, const double *v_base, long v_ld, const int *jptr, double *z_base,
             long z_ld);
void vcycle_apply(cpr_handle *h, const double *b, double *x);
void bilu_apply(cpr_handle *h, const double *r, double *z);
void refresh_outer(cpr_handle *h, bool pattern_changed);
void choose_tail(cpr_handle *h);   // decide which levels the cluster tail kernel runs
int profile_vcycle_levels(cpr_handle *h, int reps, double *us, int n_us);
void autotune(cpr_handle *h, int reps, double *before_us, double *after_us);
bool schedule_ok(const cpr_schedule &s);
int fgmres(cpr_handle *h, const double *b, double *x, double rtol, cpr_stats *st);
void fgmres_begin(cpr_handle *h, const double *b, double *x, double rtol);
int fgmres_advance(cpr_handle *h, bool block);   // 1 while running, else the solve's return code
void fgmres_stats(const cpr_handle *h, cpr_stats *st);
void batch_prepare(cpr_handle *h);
int fgmres_batch(cpr_handle *h, double rtol, cpr_stats *st);
void bsr3_spmv(int nb, const int *rowptr, const int *col, const double *val, const double *x,
               const double *b, double *y, cudaStream_t s);

}  // namespace cpr
