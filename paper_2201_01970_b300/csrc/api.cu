// The C ABI (include/cpr.h): handle lifetime, the adaptive setup rule of
// Alg. 3, host/device argument marshalling, and the inspection copies.
#include <chrono>
#include <cmath>
#include <cstdio>

#include "cpr_internal.cuh"

using namespace cpr;

namespace {

thread_local std::string g_last_error;

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// The Python binding mirrors cpr_opts field by field; its test checks the same size.
static_assert(sizeof(cpr_opts) == 112, "cpr_opts changed: update the binding's Opts and this check");

void check_opts(const cpr_opts &o) {
    bool ok = o.restart >= 1 && o.restart <= kMaxRestart && o.max_restarts >= 1 && o.pre >= 0 &&
              o.post >= 0 && o.coarse_max >= 1 && o.coarse_max <= kMaxCoarse && o.max_levels >= 1 &&
              o.theta_color >= 0.0 && o.theta_color <= 1.0 && o.theta_amg >= 0.0 && o.theta_amg <= 1.0 &&
              o.mu >= 0 && (o.decouple == 0 || o.decouple == 1) && (o.precond_fp32 == 0 || o.precond_fp32 == 1) &&
              (o.pdl == 0 || o.pdl == 1) && (o.tail == 0 || o.tail == 1) &&
              (o.bilu_order == 0 || o.bilu_order == 1) && (o.reuse_refresh == 0 || o.reuse_refresh == 1) &&
              (o.resetup == 0 || o.resetup == 1) && (o.amg == 0 || o.amg == 1) && o.amli_iters >= 1 &&
              o.amli_iters <= kMaxAmli && (o.coloring == 0 || o.coloring == 1) && o.coloring_rows >= 0 &&
              o.coloring_rows <= kMaxGroupingRows;
    if (!ok) fail(CPR_ERR_INVALID, "options out of range");
}

void copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (!bytes) return;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

// Upload A's pattern into (rowptr, col) and validate it.
void load_pattern(cpr_handle *h, const cpr_bsr3 *A, DVec<int> &rowptr, DVec<int> &col) {
    if (!A || A->nb < 1 || A->nnzb < A->nb || !A->rowptr || !A->col || !A->val)
        fail(CPR_ERR_INVALID, "bad matrix descriptor");
    cudaStream_t s = h->stream;
    rowptr.alloc(A->nb + 1, s);
    col.alloc(A->nnzb, s);
    // the copies' sizes come from the descriptor alone; the contents, host or
    // device, are checked on the device (a host-side walk of a 3.6M-entry
    // pattern cost several ms per call)
    copy_in(rowptr.p, A->rowptr, sizeof(int) * (A->nb + 1), s);
    copy_in(col.p, A->col, sizeof(int) * (size_t)A->nnzb, s);
    validate_bsr(rowptr.p, col.p, A->nb, A->nnzb, h->err.p, s);
    int e = read_int(h->err.p, s);
    if (e) {
        CK(cudaMemsetAsync(h->err.p, 0, sizeof(int), s));
        fail(CPR_ERR_INVALID, "malformed BSR pattern");
    }
}

__global__ void k_compare(long n, const int *a, const int *b, int *diff) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (a[i] != b[i]) atomicExch(diff, 1);
}

// The rebuild of B that Alg. 3 asks for: the numeric refresh when `numeric`
// (resetup = 1, same pattern, a B set up with resetup = 1 in place), else
// the full setup.
void build_timed(cpr_handle *h, bool numeric = false) {
    double t0 = now_ms();
    if (numeric && h->nr_ready) numeric_refresh(h);
    else build_preconditioner(h);
    h->setup_ms = now_ms() - t0;
    h->setup_count++;
    h->setup_called = 1;
    h->last_iters = -1;
    ensure_workspace(h);
}

}  // namespace

namespace cpr {
unsigned long long launch_count();

void set_last_error(const std::string &what) { g_last_error = what; }

void prof_begin(cpr_handle *h, int family) {
    if (!h->prof) return;
    if (!(h->prof_mask & (1u << family))) {   // family not selected: an empty bracket for prof_end to close
        h->prof_open.push_back(-1);
        return;
    }
    if (h->capturing >= 0) {
        auto &g = h->sg[h->capturing];
        cudaEvent_t a;
        CK(cudaEventCreate(&a));
        CK(cudaEventRecordWithFlags(a, h->stream, cudaEventRecordExternal));
        h->prof_open.push_back((int)g.ev_a.size());
        g.ev_a.push_back(a);
        g.ev_b.push_back(nullptr);
        g.fam.push_back(family);
        return;
    }
    if (h->ev_n == cpr_handle::kProfSlots) {
        if (!h->prof_open.empty()) {      // no slot free inside an open bracket: drop this one
            h->prof_open.push_back(-1);
            return;
        }
        prof_flush(h);
    }
    int k = h->ev_n++;
    if (!h->ev_a[k]) {
        CK(cudaEventCreate(&h->ev_a[k]));
        CK(cudaEventCreate(&h->ev_b[k]));
    }
    h->ev_fam[k] = family;
    h->prof_open.push_back(k);
    CK(cudaEventRecord(h->ev_a[k], h->stream));
}

// Closes the innermost open bracket.
void prof_end(cpr_handle *h) {
    if (!h->prof || h->prof_open.empty()) return;
    int k = h->prof_open.back();
    h->prof_open.pop_back();
    if (k < 0) return;
    if (h->capturing >= 0) {
        auto &g = h->sg[h->capturing];
        cudaEvent_t b;
        CK(cudaEventCreate(&b));
        CK(cudaEventRecordWithFlags(b, h->stream, cudaEventRecordExternal));
        g.ev_b[k] = b;
        return;
    }
    CK(cudaEventRecord(h->ev_b[k], h->stream));
}

// Accumulate the event-node brackets of step graph `which` (its last launch has completed).
void prof_collect_graph(cpr_handle *h, int which) {
    auto &g = h->sg[which];
    for (size_t k = 0; k < g.ev_a.size() && k < g.ev_b.size(); k++) {
        if (!g.ev_b[k]) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g.ev_a[k], g.ev_b[k]));
        h->prof_cnt[g.fam[k]]++;
        h->prof_ms[g.fam[k]] += ms;
    }
}

void destroy_step_graphs(cpr_handle *h) {
    if (h->sg[1].exec == h->sg[0].exec) h->sg[1].exec = nullptr;   // one graph served both slots
    for (auto &g : h->sg) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        for (auto e : g.ev_a) cudaEventDestroy(e);
        for (auto e : g.ev_b)
            if (e) cudaEventDestroy(e);
        g = cpr_handle::StepGraph{};
    }
    h->sg_epoch = -1;
}

// Accumulates the closed eager brackets (called with no bracket open).
void prof_flush(cpr_handle *h) {
    if (!h->ev_n) return;
    for (int k = 0; k < h->ev_n; k++) {
        float ms = 0.f;
        CK(cudaEventSynchronize(h->ev_b[k]));
        CK(cudaEventElapsedTime(&ms, h->ev_a[k], h->ev_b[k]));
        h->prof_cnt[h->ev_fam[k]]++;
        h->prof_ms[h->ev_fam[k]] += ms;
    }
    h->ev_n = 0;
}
}  // namespace cpr

extern "C" {

uint64_t cpr_launch_count(void) { return (uint64_t)cpr::launch_count(); }

int cpr_profile(cpr_handle *h, int enable) {
    if (!h) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        prof_flush(h);
        h->prof_open.clear();
        h->prof_mask = (unsigned)enable & ((1u << CPR_PROF_NFAMILIES) - 1u);
        h->prof = h->prof_mask != 0;
        for (int f = 0; f < CPR_PROF_NFAMILIES; f++) {
            h->prof_cnt[f] = 0;
            h->prof_ms[f] = 0.0;
        }
        return CPR_OK;
    });
}

int cpr_profile_read(const cpr_handle *h, int family, long *count, double *ms) {
    if (!h || family < 0 || family >= CPR_PROF_NFAMILIES) return CPR_ERR_INVALID;
    if (count) *count = h->prof_cnt[family];
    if (ms) *ms = h->prof_ms[family];
    return CPR_OK;
}

void cpr_default_opts(cpr_opts *o) {
    o->theta_color = 0.05;
    o->theta_amg = 0.25;
    o->mu = 30;
    o->restart = 30;
    o->max_restarts = 100;
    o->precond_fp32 = 0;
    o->decouple = 1;
    o->pre = 1;
    o->post = 1;
    o->coarse_max = 256;
    o->max_levels = 20;
    o->seed = 0;
    o->stream = nullptr;
    o->pdl = 1;
    o->tail = 0;
    o->bilu_order = 0;
    o->reuse_refresh = 0;
    o->resetup = 0;
    o->amg = 0;
    o->amli_iters = 2;
    o->coloring = 0;
    o->coloring_rows = 4096;
}

const char *cpr_strerror(int code) {
    switch (code) {
    case CPR_OK: return "ok";
    case CPR_NOT_CONVERGED: return "not converged within max_restarts cycles";
    case CPR_ERR_INVALID: return "invalid argument or malformed matrix";
    case CPR_ERR_CUDA: return "CUDA call failed";
    case CPR_ERR_OOM: return "out of device memory";
    case CPR_ERR_SINGULAR: return "singular pivot (block diagonal, smoother diagonal or coarse LU)";
    case CPR_ERR_BREAKDOWN: return "NaN/Inf in the iteration or right-hand side";
    case CPR_ERR_TIMEOUT: return "bounded device wait gave up";
    default: return "unknown code";
    }
}

// Detail of the last failure on this thread (diagnostics; not part of the stable ABI).
const char *cpr_last_error_detail(void) { return g_last_error.c_str(); }

int cpr_setup(cpr_handle **out, const cpr_bsr3 *A, const cpr_opts *opts) {
    if (!out) return CPR_ERR_INVALID;
    *out = nullptr;
    cpr_handle *h = new (std::nothrow) cpr_handle();
    if (!h) return CPR_ERR_OOM;
    int rc = guarded([&] {
        if (opts) h->opt = *opts;
        else cpr_default_opts(&h->opt);
        check_opts(h->opt);
        Nvtx nv("cpr_setup");
        CK(cudaGetDevice(&h->device));
        // the allocation-free entry's scratch array is mapped here, where
        // allocating is allowed, rather than at its first call
        noalloc_prepare();
        if (h->opt.stream) {
            h->stream = (cudaStream_t)h->opt.stream;
        } else {
            // a blocking stream: ordered with the legacy default stream that callers
            // (torch included) use unless they pass their own stream
            CK(cudaStreamCreate(&h->stream));
            h->own_stream = true;
        }
        h->err.alloc(1, h->stream);
        h->err.zero();
        load_pattern(h, A, h->rowptr, h->col);
        h->nb = A->nb;
        h->nnzb = A->nnzb;
        h->val.alloc(9 * (size_t)A->nnzb, h->stream);
        copy_in(h->val.p, A->val, sizeof(double) * 9 * (size_t)A->nnzb, h->stream);
        refresh_outer(h, true);
        h->updates = 1;
        build_timed(h);
        return CPR_OK;
    });
    if (rc != CPR_OK) {
        cpr_destroy(h);
        return rc;
    }
    *out = h;
    return CPR_OK;
}

int cpr_update(cpr_handle *h, const cpr_bsr3 *A) {
    if (!h || h->fs.phase != FgmresState::IDLE) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        Nvtx nv("cpr_update");
        cudaStream_t s = h->stream;
        DVec<int> rp, cl;
        load_pattern(h, A, rp, cl);
        bool same = A->nb == h->nb && A->nnzb == h->nnzb;
        if (same) {
            DVec<int> diff;
            diff.alloc(1, s);
            diff.zero();
            k_compare<<<grid_for(h->nb + 1, 256, 1184), 256, 0, s>>>(h->nb + 1, rp.p, h->rowptr.p, diff.p);
            k_compare<<<grid_for(h->nnzb, 256, 1184), 256, 0, s>>>(h->nnzb, cl.p, h->col.p, diff.p);
            CK_LAUNCH();
            same = read_int(diff.p, s) == 0;
        }
        if (!same) {
            h->pattern_id++;   // structure kept from the old pattern is stale
            h->rowptr = std::move(rp);
            h->col = std::move(cl);
            h->nb = A->nb;
            h->nnzb = A->nnzb;
            h->val.alloc(9 * (size_t)A->nnzb, s);
        }
        copy_in(h->val.p, A->val, sizeof(double) * 9 * (size_t)A->nnzb, s);
        refresh_outer(h, !same);
        h->updates++;
        // Alg. 3: reuse B^(k-1) iff k > 1 and It^(k-1) <= mu (and Remark 4.2: same size/pattern)
        bool reuse = same && h->have_B && h->last_iters >= 0 && h->last_iters <= h->opt.mu;
        if (reuse) {
            if (h->opt.reuse_refresh) refresh_second_residual(h);
            h->setup_called = 0;
            h->setup_ms = 0.0;
            return CPR_OK;
        }
        // resetup = 1: same pattern, so only the values are rebuilt
        build_timed(h, h->opt.resetup && same && h->have_B);
        return CPR_OK;
    });
}

int cpr_update_values(cpr_handle *h, const double *val) {
    if (!h || !val || h->batch || h->fs.phase != FgmresState::IDLE) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        Nvtx nv("cpr_update_values");
        copy_in(h->val.p, val, sizeof(double) * 9 * (size_t)h->nnzb, h->stream);
        refresh_outer(h, false);
        h->updates++;
        // Alg. 3 with an unchanged pattern (Remark 4.2 holds by the caller's guarantee)
        bool reuse = h->have_B && h->last_iters >= 0 && h->last_iters <= h->opt.mu;
        if (reuse) {
            if (h->opt.reuse_refresh) refresh_second_residual(h);
            h->setup_called = 0;
            h->setup_ms = 0.0;
            return CPR_OK;
        }
        build_timed(h, h->opt.resetup && h->have_B);
        return CPR_OK;
    });
}

namespace {

// b and x of a solve on the device: host buffers are copied into the
// handle's vectors (x is copied back by finish_solve).
void solve_prelude(cpr_handle *h, const double *b, double *x, double rtol) {
    double t0 = now_ms();
    cudaStream_t s = h->stream;
    size_t bytes = sizeof(double) * 3 * (size_t)h->nb;
    const double *db = b;
    double *dx = x;
    if (!is_device_ptr(b)) {
        CK(cudaMemcpyAsync(h->dev_b.p, b, bytes, cudaMemcpyHostToDevice, s));
        db = h->dev_b.p;
    }
    bool xdev = is_device_ptr(x);
    if (!xdev) {
        CK(cudaMemcpyAsync(h->dev_x.p, x, bytes, cudaMemcpyHostToDevice, s));
        dx = h->dev_x.p;
    }
    fgmres_begin(h, db, dx, rtol);
    h->fs.x_out = xdev ? nullptr : x;
    h->fs.t0 = t0;
}

int finish_solve(cpr_handle *h, int rc, cpr_stats *st) {
    cudaStream_t s = h->stream;
    prof_flush(h);
    if (h->fs.x_out)
        CK(cudaMemcpyAsync(h->fs.x_out, h->fs.x, sizeof(double) * 3 * (size_t)h->nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cpr_stats local{};
    fgmres_stats(h, &local);
    local.setup_called = h->setup_called;
    local.setup_count = h->setup_count;
    local.levels = (int)h->lev.size();
    local.tail_levels = h->tail_top >= 0 ? (int)h->lev.size() - 1 - h->tail_top : 0;
    local.setup_ms = h->setup_called ? h->setup_ms : 0.0;
    local.solve_ms = now_ms() - h->fs.t0;
    h->fs.phase = FgmresState::IDLE;
    if (st) *st = local;
    return rc;
}

bool solving(const cpr_handle *h) { return h->fs.phase != FgmresState::IDLE; }

}  // namespace

int cpr_solve(cpr_handle *h, const double *b, double *x, double rtol, cpr_stats *st) {
    if (!h || !b || !x || !(rtol > 0.0) || h->batch || solving(h)) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        Nvtx nv("cpr_solve");
        solve_prelude(h, b, x, rtol);
        int rc;
        while ((rc = fgmres_advance(h, true)) == 1) {
        }
        return finish_solve(h, rc, st);
    });
}

int cpr_solve_start(cpr_handle *h, const double *b, double *x, double rtol) {
    if (!h || !b || !x || !(rtol > 0.0) || h->batch || solving(h)) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        Nvtx nv("cpr_solve_start");
        solve_prelude(h, b, x, rtol);
        int rc = fgmres_advance(h, false);
        if (rc != 1) {   // finished at once (zero right-hand side, a non-finite b seen immediately)
            h->fs.phase = FgmresState::DONE;
            h->fs.rc = rc;
        }
        return CPR_OK;
    });
}

int cpr_solve_poll(cpr_handle *h, cpr_stats *st) {
    if (!h || !solving(h)) return CPR_ERR_INVALID;
    int rc = guarded([&] {
        DeviceGuard dg(h->device);
        int r = fgmres_advance(h, false);
        if (r == 1) return CPR_RUNNING;
        return finish_solve(h, r, st);
    });
    if (rc < 0 && rc != CPR_RUNNING) h->fs.phase = FgmresState::IDLE;
    return rc;
}

void cpr_destroy(cpr_handle *h) {
    if (!h) return;
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != h->device) cudaSetDevice(h->device);
    else prev = -1;
    if (h->stream) cudaStreamSynchronize(h->stream);
    try {
        free_preconditioner(h);
    } catch (...) {
    }
    cudaStream_t s = h->stream;
    bool own = h->own_stream;
    destroy_step_graphs(h);
    for (auto &g : h->sgb) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    delete h->batch;
    h->batch = nullptr;
    for (auto e : h->step_done)
        if (e) cudaEventDestroy(e);
    for (auto e : h->ev_coarse)
        if (e) cudaEventDestroy(e);
    for (auto e : h->ev_nr)
        if (e) cudaEventDestroy(e);
    for (auto e : h->ev_color) cudaEventDestroy(e);
    if (h->pinned) cudaFreeHost(h->pinned);
    for (int k = 0; k < cpr_handle::kProfSlots; k++) {
        if (h->ev_a[k]) cudaEventDestroy(h->ev_a[k]);
        if (h->ev_b[k]) cudaEventDestroy(h->ev_b[k]);
    }
    h->pinned = nullptr;
    h->pinned_dev_flags = nullptr;
    cudaStream_t side = h->side, lu = h->lu_stream;
    delete h;  // DVec destructors free on the stream each buffer was allocated on
    if (s) cudaStreamSynchronize(s);
    if (own && s) cudaStreamDestroy(s);
    for (cudaStream_t q : {side, lu})
        if (q) {
            cudaStreamSynchronize(q);
            cudaStreamDestroy(q);
        }
    if (prev >= 0) cudaSetDevice(prev);
}

int cpr_apply(cpr_handle *h, const double *v, double *z) {
    if (!h || !v || !z) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        apply_B(h, v, 0, nullptr, z, 0);
        CK(cudaStreamSynchronize(h->stream));
        return CPR_OK;
    });
}

int cpr_vcycle(cpr_handle *h, const double *b, double *x) {
    if (!h || !b || !x) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        vcycle_apply(h, b, x);
        CK(cudaStreamSynchronize(h->stream));
        return CPR_OK;
    });
}

int cpr_profile_vcycle_levels(cpr_handle *h, int reps, double *us, int n_us) {
    if (!h || !us || reps < 1 || h->lev.empty()) return CPR_ERR_INVALID;
    int written = 0;
    int rc = guarded([&] {
        DeviceGuard dg(h->device);
        written = profile_vcycle_levels(h, reps, us, n_us);
        return CPR_OK;
    });
    return rc == CPR_OK ? written : rc;
}

int cpr_get_schedule(const cpr_handle *h, int level, cpr_schedule *s) {
    if (!h || !s || level < 0 || level >= (int)h->lev.size() - 1) return CPR_ERR_INVALID;
    const Level &L = h->lev[level];
    *s = cpr_schedule{L.gA, L.gP, L.gR, L.bs};
    return CPR_OK;
}

int cpr_set_schedule(cpr_handle *h, int level, const cpr_schedule *s) {
    if (!h || !s || level < 0 || level >= (int)h->lev.size() - 1 || !schedule_ok(*s)) return CPR_ERR_INVALID;
    Level &L = h->lev[level];
    L.gA = s->lanes_a;
    L.gP = s->lanes_p;
    L.gR = s->lanes_r;
    L.bs = s->block;
    h->epoch++;   // the step graphs are recaptured
    return CPR_OK;
}

int cpr_autotune(cpr_handle *h, int reps, double *before_us, double *after_us) {
    if (!h || reps < 1 || h->lev.size() < 2) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        Nvtx nv("cpr_autotune");
        autotune(h, reps, before_us, after_us);
        return CPR_OK;
    });
}

int cpr_bilu_apply(cpr_handle *h, const double *r, double *z) {
    if (!h || !r || !z) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        bilu_apply(h, r, z);
        CK(cudaStreamSynchronize(h->stream));
        return CPR_OK;
    });
}

int cpr_bsr3_spmv(const cpr_bsr3 *A, const double *x, const double *b, double *y, void *stream) {
    if (!A || A->nb < 1 || !A->rowptr || !A->col || !A->val || !x || !y) return CPR_ERR_INVALID;
    return guarded([&] {
        bsr3_spmv(A->nb, A->rowptr, A->col, A->val, x, b, y, (cudaStream_t)stream);
        return CPR_OK;
    });
}

int cpr_num_levels(const cpr_handle *h) { return h ? (int)h->lev.size() : 0; }

int cpr_get_level_info(const cpr_handle *h, int level, cpr_level_info *info) {
    if (!h || !info || level < 0 || level >= (int)h->lev.size()) return CPR_ERR_INVALID;
    const Level &L = h->lev[level];
    info->n = L.A.n;
    info->nnz = L.A.nnz;
    info->ncolors = L.ncolors;
    info->nc = L.nc;
    info->nnz_p = L.P.nnz;
    return CPR_OK;
}

int cpr_copy_level(const cpr_handle *h, int level, int32_t *rowptr, int32_t *col, double *val,
                   int32_t *color, int32_t *cf, int32_t *prow, int32_t *pcol, double *pval) {
    if (!h || level < 0 || level >= (int)h->lev.size()) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        const Level &L = h->lev[level];
        cudaStream_t s = h->stream;
        auto d2h = [&](void *dst, const void *src, size_t bytes) {
            if (dst && src && bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        };
        d2h(rowptr, L.A.rowptr.p, sizeof(int) * (L.A.n + 1));
        d2h(col, L.A.col.p, sizeof(int) * (size_t)L.A.nnz);
        d2h(val, L.A.val.p, sizeof(double) * (size_t)L.A.nnz);
        if (L.ncolors) d2h(color, L.color.p, sizeof(int) * L.A.n);
        if (L.nc) {
            d2h(cf, L.cf.p, sizeof(int) * L.A.n);
            d2h(prow, L.P.rowptr.p, sizeof(int) * (L.A.n + 1));
            d2h(pcol, L.P.col.p, sizeof(int) * (size_t)L.P.nnz);
            d2h(pval, L.P.val.p, sizeof(double) * (size_t)L.P.nnz);
        }
        CK(cudaStreamSynchronize(s));
        return CPR_OK;
    });
}

int cpr_copy_weights(const cpr_handle *h, double *w) {
    if (!h || !w) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        CK(cudaMemcpyAsync(w, h->w.p, sizeof(double) * 3 * (size_t)h->nb, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return CPR_OK;
    });
}

int cpr_copy_bilu(const cpr_handle *h, int32_t *bcolor, double *lu, int *nbcolors) {
    if (!h) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        cudaStream_t s = h->stream;
        if (bcolor) CK(cudaMemcpyAsync(bcolor, h->bilu.color.p, sizeof(int) * h->nb, cudaMemcpyDeviceToHost, s));
        std::vector<float> tmp;
        if (lu && h->opt.precond_fp32) {
            tmp.resize(9 * (size_t)h->nnzb);
            CK(cudaMemcpyAsync(tmp.data(), h->bilu.lu32.p, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, s));
        } else if (lu) {
            CK(cudaMemcpyAsync(lu, h->bilu.lu.p, sizeof(double) * 9 * (size_t)h->nnzb, cudaMemcpyDeviceToHost, s));
        }
        if (nbcolors) *nbcolors = h->bilu.ncolors;
        CK(cudaStreamSynchronize(s));
        for (size_t k = 0; k < tmp.size(); k++) lu[k] = tmp[k];
        return CPR_OK;
    });
}

}  // extern "C"
