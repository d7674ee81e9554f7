/*
 * cpr.h -- C ABI of the B300 (sm_103a) CPR-preconditioned FGMRES solver for
 * fully implicit black-oil Jacobians in 3x3 block sparse row form.
 *
 * Method: arXiv 2201.01970, "Parallel Multi-Stage Preconditioners with
 * Adaptive Setup for the Black Oil Model".
 *   - the CPR preconditioner B: Eq. 3.1 and Alg. 1 (Sec. 3.1);
 *   - the outer solver: right-preconditioned GMRES, Alg. 2 (Sec. 4), run here
 *     in its flexible form (FGMRES) with restart length m;
 *   - the adaptive setup rule: Alg. 3 and Remark 4.2 (Sec. 4);
 *   - the AMG smoother: multi-color Gauss-Seidel over the colors of the
 *     strong-connection matrix, Eq. 5.1 and Alg. 6 (Sec. 5.2).
 *   - the second stage's BILU(0): multicolor by default, or the natural-order,
 *     level-scheduled BILU of Sec. 6 (cpr_opts.bilu_order).
 *
 * Conventions for every call below
 *   - Block rows: nb >= 1.  A 3x3 block is 9 doubles, row-major.  rowptr has
 *     nb+1 entries starting at 0; col indices of a row are strictly increasing
 *     and each row holds its diagonal block.  Violations return CPR_ERR_INVALID.
 *   - Vectors have 3*nb doubles, ordered (P, S_1, S_2) per block row (Eq. 2.8);
 *     well rows (Eq. 2.7) are ordinary block rows.
 *   - Pointers passed to cpr_setup, cpr_update and cpr_solve may be host or
 *     device (CUDA) pointers; the library detects which.  Host buffers are
 *     copied in and out inside the call (pinned host memory copies fastest).
 *   - All GPU work is ordered on opts.stream (NULL: a stream the handle
 *     creates).  cpr_solve returns after the result is in x.
 *   - Ownership: the caller owns A, b and x.  The library copies A's values
 *     into its own storage, so A may be freed or overwritten after the call
 *     returns.  The handle owns everything else until cpr_destroy.
 *   - Errors: 0 = success, 1 = CPR_NOT_CONVERGED (x holds the last iterate),
 *     negative = failure (see CPR_ERR_*).  After a failure the handle may only
 *     be destroyed, except for CPR_ERR_INVALID from cpr_update/cpr_solve,
 *     which leaves it unchanged.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Devices: a handle belongs to the CUDA device that was current when it
 *     was set up.  Every call on it runs on that device, whichever device the
 *     caller has current, and leaves the caller's current device as it was.
 */
#ifndef CPR_B300_H
#define CPR_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPR_OK 0
#define CPR_NOT_CONVERGED 1
#define CPR_RUNNING 2          /* cpr_solve_poll: the solve is still in progress */
#define CPR_ERR_INVALID (-1)   /* malformed matrix, sizes or options */
#define CPR_ERR_CUDA (-2)      /* a CUDA call failed */
#define CPR_ERR_OOM (-3)       /* device memory exhausted */
#define CPR_ERR_SINGULAR (-4)  /* zero pivot: block diagonal, smoother diagonal or coarse LU */
#define CPR_ERR_BREAKDOWN (-5) /* NaN/Inf in the iteration or the right-hand side */
#define CPR_ERR_TIMEOUT (-6)   /* reserved for a bounded device-side wait that gives up; no kernel
                                  of this library waits on another, so no call returns it today */

typedef struct cpr_handle cpr_handle;

/* A 3x3 BSR matrix (Eq. 2.7/2.8): val has 9*nnzb doubles. */
typedef struct {
    int32_t nb, nnzb;
    const int32_t *rowptr;
    const int32_t *col;
    const double *val;
} cpr_bsr3;

typedef struct {
    double theta_color; /* Eq. 5.1 strength threshold for the smoother's coloring; default 0.05 */
    double theta_amg;   /* classical strength threshold for C/F splitting; default 0.25 */
    int mu;             /* Alg. 3 threshold: reuse B while It^(k-1) <= mu; 0 = setup every time; default 30 */
    int restart;        /* FGMRES restart length m, 1..64; default 30 */
    int max_restarts;   /* maximum restart cycles (MaxIt of Alg. 2); default 100 */
    int precond_fp32;   /* 1: B computes in FP32 (storage and accumulation); outer FGMRES stays FP64 */
    int decouple;       /* 1: ABF weights w_i = D_i^-T e_1 for Pi_P^T; 0: plain injection; default 1 */
    int pre, post;      /* V-cycle smoothing sweeps; default 1, 1 */
    int coarse_max;     /* coarsest level size solved densely; default 256, at most 4096 */
    int max_levels;     /* default 20 */
    uint64_t seed;      /* hash seed of coloring and C/F splitting; default 0 */
    void *stream;       /* cudaStream_t; NULL = the handle creates its own */
    int pdl;            /* 1 (default): the kernels of a B application use programmatic
                           dependent launch, each loading its setup-time operands while its
                           predecessor runs (FP64 BILU(0) sweeps excepted: slower so on
                           B300); 0: plain stream order.  Results are identical either way. */
    int tail;           /* 1: the last one or two smoothed AMG levels (never level 0) and the
                           coarse solve run as one kernel on one thread-block cluster when
                           they are small enough (at most 4096 rows per level, 16 colors, a
                           coarse level of at most 1024 rows) and the cycle is V(1,1);
                           0 (default, measured faster on B300): one kernel per phase.
                           Results are identical either way. */
    int bilu_order;     /* second stage's BILU(0) order.  0 (default): multicolor, blocks in
                           (JP color, index) order, one launch per color.  1: natural block
                           order, as the paper's level-scheduled BILU (Sec. 6): the same
                           factors as sequential block ILU(0) in index order, run one level
                           set at a time (level = 1 + the largest level among a row's
                           neighbours of lower index), so a sweep has as many launches as
                           there are levels (nx + ny + nz - 2 on a 7-point grid). */
    int reuse_refresh;  /* what a B kept by Alg. 3 applies.  0 (default): B as built, with the
                           copy of A^(k-1) it was built from in its second residual (Alg. 1).
                           1: the second residual takes the current A^(k); the decoupling,
                           the AMG hierarchy and the BILU(0) factors stay those of A^(k-1). */
    int resetup;        /* what Alg. 3's rebuild of B does when the pattern is unchanged.
                           0 (default): the full setup.  1: numeric only -- the last setup's
                           number of levels, classical strength sets, C/F splits, smoother
                           colorings and BILU(0) ordering are kept, and every value (weights,
                           A_P, interpolation, Galerkin products, coarse LU, BILU(0) factors)
                           is recomputed from A^(k).  The recomputation writes into the
                           buffers of the last full setup and is replayed as one CUDA graph
                           (captured on the first such rebuild, which also builds the
                           Galerkin products' lists); the handle then holds each level's
                           A P and those lists besides B.  Not in the paper. */
    int amg;            /* first stage's AMG.  0 (default): classical -- strength, PMIS C/F split,
                           direct interpolation, R A P -- with a V(pre,post) cycle.  1: the paper's
                           own first stage (Sec. 6): unsmoothed aggregation by double pairwise
                           matching on the symmetric part of A_l (strong when c_ij < 0 and
                           -c_ij >= theta_amg max_k -c_ik), matched in handshake rounds (each node
                           points to its strongest unmatched candidate, mutual pointers pair; a node
                           left alone joins its strongest candidate's pair), unit-entry P, and the
                           nonlinear AMLI-cycle: the V-cycle's smoothing and transfers
                           with each coarse problem above the coarsest solved by amli_iters steps
                           of flexible GCR preconditioned by the cycle one level down. */
    int amli_iters;     /* amg = 1: GCR steps of each coarse correction, 1..8; default 2 */
    int coloring;       /* smoother coloring.  0 (default): Jones-Plassmann on S u S^T.  1: the
                           paper's VerticesSplitting/Grouping (Alg. 4-5) on every smoothed level
                           of at most coloring_rows rows (JP above): a sequential greedy, run by
                           one thread block on the device. */
    int coloring_rows;  /* coloring = 1: the largest level that takes Alg. 4-5; default 4096,
                           at most 16384 */
} cpr_opts;

typedef struct {
    int iters;          /* inner (Arnoldi) steps of this solve = It of Alg. 3 */
    int restarts;       /* restart cycles used */
    int setup_called;   /* 1 if the last cpr_setup/cpr_update built B */
    int setup_count;    /* total builds of B by this handle */
    int levels;         /* AMG levels, coarsest included */
    int converged;
    double rel_res;     /* ||b - A x|| / ||b - A x_0||, true FP64 residual */
    double setup_ms;    /* wall time of the last build of B (0 if reused) */
    double solve_ms;    /* wall time of this cpr_solve */
    int tail_levels;    /* smoothed levels run by the cluster tail kernel (0: none) */
} cpr_stats;

/* Fill *o with the defaults listed above. */
void cpr_default_opts(cpr_opts *o);

/*
 * Build the handle and the preconditioner B^(1) from A^(1) (Alg. 2's first setup, with
 * k = 1; Alg. 1's setup: decoupling, AMG hierarchy with Eq. 5.1 colorings,
 * BILU(0)), all on the device.  opts may be NULL for defaults.
 * Returns CPR_ERR_INVALID (also for an empty system, nb < 1), _OOM, _SINGULAR
 * or _CUDA on failure (*h = NULL).
 */
int cpr_setup(cpr_handle **h, const cpr_bsr3 *A, const cpr_opts *opts);

/*
 * Hand the next Newton Jacobian A^(k) to the handle (Alg. 3): the outer
 * operator becomes A^(k); B is kept iff the previous solve took
 * It^(k-1) <= mu steps and the size and pattern are unchanged (Remark 4.2),
 * otherwise B is rebuilt from A^(k).  A kept B keeps the copy of A it was
 * built from for its own second residual (the second residual of Alg. 1).
 */
int cpr_update(cpr_handle *h, const cpr_bsr3 *A);

/*
 * cpr_update for a Jacobian with exactly the current A's block pattern:
 * only its 9*nnzb values are passed (host or device pointer).  The pattern is
 * neither uploaded, validated nor compared, so the call makes no host round
 * trip before Alg. 3's decision; the caller guarantees the pattern (a Newton
 * sequence of one simulation keeps it).  Not for batch handles.
 */
int cpr_update_values(cpr_handle *h, const double *val);

/*
 * Solve A^(k) x = b by FGMRES(m) right-preconditioned with B (Alg. 2): x is
 * the initial guess on entry and the solution on return.  Stops when the true
 * residual satisfies ||b - A x|| < rtol ||b - A x_0|| or after max_restarts
 * cycles (CPR_NOT_CONVERGED).  b with NaN/Inf: CPR_ERR_BREAKDOWN.  st may be
 * NULL.
 */
int cpr_solve(cpr_handle *h, const double *b, double *x, double rtol, cpr_stats *st);

/*
 * cpr_solve in two halves, for a host thread that drives many handles (a
 * serving loop): cpr_solve_start issues the solve's first work and returns
 * without waiting; each cpr_solve_poll issues what the finished device work
 * allows (the next Arnoldi steps, the next restart cycle) and returns
 * CPR_RUNNING, or, once the solve has finished, its cpr_solve return code with
 * x (host x copied back) and st filled.  The same kernels run in the same
 * order as in cpr_solve, so results are bit-identical.  While a solve is in
 * progress the handle accepts only cpr_solve_poll and cpr_destroy (other
 * calls return CPR_ERR_INVALID).  b and x must stay valid until it finishes.
 */
int cpr_solve_start(cpr_handle *h, const double *b, double *x, double rtol);
int cpr_solve_poll(cpr_handle *h, cpr_stats *st);

/* Release every resource of the handle (NULL is accepted). */
void cpr_destroy(cpr_handle *h);

/* A static string describing a return code. */
const char *cpr_strerror(int code);

/* A text description of the most recent failure on the calling thread (valid
 * until the next failing call on that thread). */
const char *cpr_last_error_detail(void);

/* ------------------------------------------------------------------------
 * Batched solves: many independent systems of uneven size in one handle.
 * The systems' matrices are concatenated into one block-diagonal matrix, so
 * the preconditioner's setup and every preconditioner kernel run once over all
 * systems (B is the block-diagonal CPR preconditioner); FGMRES (Alg. 2) runs
 * per system in lockstep, each with its own Hessenberg matrix, rotations and
 * stop decision, and each Arnoldi step of the whole batch is one graph launch.
 * cpr_solve rejects a batch handle.  The component and inspection calls below
 * accept one and work on the concatenated system (vectors of 3 * total block
 * rows, systems in order); cpr_destroy frees it.
 * ---------------------------------------------------------------------- */

/* Build a batch handle from nsys systems A[0..nsys-1] (host or device pointers,
 * each following the conventions above). */
int cpr_batch_setup(cpr_handle **h, int nsys, const cpr_bsr3 *A, const cpr_opts *opts);

/* New matrices with unchanged sizes (Alg. 3 decides reuse, with It^(k-1) the
 * largest step count of the previous batch solve: the system with the largest
 * stats[].iters decides for the whole batch). */
int cpr_batch_update(cpr_handle *h, const cpr_bsr3 *A);

/* Solve every system: b[k], x[k] (host or device; x[k] is the initial guess and
 * receives the solution); st, when not NULL, holds nsys entries. */
int cpr_batch_solve(cpr_handle *h, const double *const *b, double *const *x, double rtol, cpr_stats *st);

/* Number of systems of a batch handle (0 for a single-system handle). */
int cpr_batch_size(const cpr_handle *h);

/* ------------------------------------------------------------------------
 * Component entry points: one application of a part of B.  All vectors are
 * DEVICE pointers with the handle's sizes; work is ordered on the handle's
 * stream and the call returns after it completes.  In FP32 mode the inputs
 * are rounded to FP32 on entry and results widened on exit.
 * ---------------------------------------------------------------------- */

/* z = B v: one CPR application from x = 0 (Alg. 1, Eq. 3.1); v, z: 3*nb. */
int cpr_apply(cpr_handle *h, const double *v, double *z);

/* x = B_P b: one AMG V(pre,post) cycle on the pressure matrix A_P (Sec. 3.1,
 * smoother Alg. 6) from x = 0; b, x: nb. */
int cpr_vcycle(cpr_handle *h, const double *b, double *x);

/* z = R r with R = (L U)^-1, the multicolor BILU(0) second stage (Eq. 3.1);
 * r, z: 3*nb. */
int cpr_bilu_apply(cpr_handle *h, const double *r, double *z);

/* z = R r exactly as cpr_bilu_apply, for callers that must not allocate
 * device memory at call time -- e.g. a simulator that reserves its whole
 * device-memory budget at start-up, or code that runs while another component
 * owns the allocator.  The paper has no counterpart: this is an interface
 * variant only.  The sweeps' work vector (3*nb values) lives in a fixed
 * device array of 65,536 block rows (1.5 MiB) that every GPU loading this
 * library holds until the process exits; a handle with more block rows gets
 * CPR_ERR_INVALID (for a batch handle the limit applies to the total of its
 * systems).  The call allocates nothing and frees nothing.  The array is
 * mapped onto a device, and its device address looked up, when the first
 * handle is set up there (cpr_setup, where allocating is allowed): the call
 * itself only reads that cached address.  All calls share
 * the one array and leave their last contents in it; nothing in it needs to
 * start at zero (each call writes every entry it reads first).  Calls whose
 * GPU work overlaps -- two streams, two handles, two threads -- race on the
 * array: serialise them.  r, z: DEVICE pointers, 3*nb; ordered on the handle's
 * stream; returns after completion. */
int cpr_bilu_apply_noalloc(cpr_handle *h, const double *r, double *z);

/* y = A x (or r = b - A x when b != NULL) for a 3x3 BSR matrix (Eq. 2.8),
 * all DEVICE pointers, stateless, ordered on `stream` (cudaStream_t; NULL =
 * legacy default stream), asynchronous. */
int cpr_bsr3_spmv(const cpr_bsr3 *A, const double *x, const double *b, double *y, void *stream);

/* ------------------------------------------------------------------------
 * Inspection: copies of the current B's setup results into HOST buffers, in
 * the natural (input) numbering, for checking and diagnostics.
 * ---------------------------------------------------------------------- */

typedef struct {
    int n, nnz;    /* size and nonzeros of A_l */
    int ncolors;   /* colors of the Eq. 5.1 coloring (0 on the coarsest level) */
    int nc;        /* C points = size of level l+1 (0 on the coarsest level) */
    int nnz_p;     /* nonzeros of the interpolation P_l (0 on the coarsest level) */
} cpr_level_info;

int cpr_num_levels(const cpr_handle *h);
int cpr_get_level_info(const cpr_handle *h, int level, cpr_level_info *info);

/* Any pointer may be NULL to skip it.  rowptr: n+1, col/val: nnz, color/cf: n
 * (cf: 1 = C, 0 = F), prow: n+1, pcol/pval: nnz_p. */
int cpr_copy_level(const cpr_handle *h, int level, int32_t *rowptr, int32_t *col, double *val,
                   int32_t *color, int32_t *cf, int32_t *prow, int32_t *pcol, double *pval);

/* w: 3*nb decoupling weights (Pi_P^T row weights). */
int cpr_copy_weights(const cpr_handle *h, double *w);

/* bcolor: nb block colors; lu: 9*nnzb factor blocks in A's pattern (L_ij below
 * the diagonal in (color, index) order, U_ij above it, U_ii^-1 on it).  In
 * FP32-preconditioner mode the factorization itself runs in FP32 and lu
 * receives those factors widened to FP64. */
int cpr_copy_bilu(const cpr_handle *h, int32_t *bcolor, double *lu, int *nbcolors);

/* ------------------------------------------------------------------------
 * Measurement hooks (diagnostics).
 * ---------------------------------------------------------------------- */

/* Number of kernels this library has launched in this process so far. */
uint64_t cpr_launch_count(void);

/* A cap on the device memory this library holds, over all handles and devices
 * of the process (bytes; 0 = no cap, the default).  An allocation that would
 * pass it fails as a failed device allocation does: CPR_ERR_OOM from the call
 * that needed it, with the handle left as CPR_ERR_OOM leaves it.  Lets a
 * caller that shares the GPU bound the library's share of it.  Not in the
 * paper. */
void cpr_set_memory_limit(uint64_t bytes);

/* Device bytes the library holds now, over all handles and devices. */
uint64_t cpr_memory_in_use(void);

/* Kernel families that cpr_profile brackets with CUDA events on the handle's
 * stream during cpr_solve. */
#define CPR_PROF_SPMV 0      /* one outer BSR SpMV launch, w = A z or r = b - A x */
#define CPR_PROF_VCYCLE 1    /* one whole V-cycle application (all its launches) */
#define CPR_PROF_BILU 2      /* one whole BILU(0) forward+backward application */
#define CPR_PROF_CGS 3       /* one CGS orthogonalisation (dots, reduction, update) */
#define CPR_PROF_RESID2 4    /* one second-residual launch (Alg. 1, second residual) */
#define CPR_PROF_SMOOTH0 5   /* one multi-color GS color launch on the finest pressure level */
#define CPR_PROF_NFAMILIES 6

#define CPR_PROF_ALL ((1 << CPR_PROF_NFAMILIES) - 1)

/* mask != 0: time the families whose bits (1 << family) are set during later
 * solves, each bracketed region with two event records on the handle's stream
 * (inside the step graphs an event node costs a few microseconds, so nested
 * families -- the level-0 sweeps inside the V-cycle -- are best timed in
 * separate passes); 0: stop.  Both reset the accumulators. */
int cpr_profile(cpr_handle *h, int mask);

/* Accumulated bracket count and device milliseconds of one family. */
int cpr_profile_read(const cpr_handle *h, int family, long *count, double *ms);

/*
 * Device time of the parts of one B application, each captured `reps` times
 * into a CUDA graph of its own and timed with CUDA events on the handle's
 * stream (best of three graph launches; microseconds per repetition):
 *   us[0] one V-cycle (Alg. 6 on every level, Alg. 1's B_P),
 *   us[1] one BILU(0) forward + backward application,
 *   us[2] the coarsest level's dense solve,
 *   us[3 + 5 l + q] level l < levels-1: q = 0 pre-smoothing sweep over its
 *         colors, 1 residual, 2 restriction, 3 prolongation, 4 post-smoothing.
 * The parts run on whatever the work vectors hold, so call this between
 * solves only (every B application rewrites those vectors before reading
 * them).  n_us must be at least 3 + 5 * (levels - 1).  Returns the count of
 * values written, or CPR_ERR_INVALID / CPR_ERR_CUDA.  No counterpart in the
 * paper: a measurement hook.
 */
int cpr_profile_vcycle_levels(cpr_handle *h, int reps, double *us, int n_us);

/* ------------------------------------------------------------------------
 * V-cycle schedule and its autotuner (not in the paper: how the kernels of
 * Alg. 6's sweeps and the transfers map onto the GPU).  The results do not
 * depend on the schedule beyond rounding order: every schedule gives the same
 * hierarchy, and B's applications agree with the FP64 definition to rounding.
 * ---------------------------------------------------------------------- */

typedef struct {
    int lanes_a;   /* lanes per row of the smoothing and residual kernels (A_l): 1, 2, 4, .., 32 */
    int lanes_p;   /* lanes per row of the prolongation kernel (P_l) */
    int lanes_r;   /* lanes per row of the restriction kernel (R_l) */
    int block;     /* threads per CTA of these kernels: 128, 256 or 512 */
} cpr_schedule;

/* The schedule of level `level` (0 <= level < levels - 1). */
int cpr_get_schedule(const cpr_handle *h, int level, cpr_schedule *s);

/* Impose a schedule on one level of the current B (CPR_ERR_INVALID for values
 * outside the sets above).  Kept until the next setup. */
int cpr_set_schedule(cpr_handle *h, int level, const cpr_schedule *s);

/* Time, on the device, each candidate schedule of every level of the current
 * hierarchy -- lanes per row for the smoothing/residual, restriction and
 * prolongation kernels in turn, then the CTA size -- each part captured `reps`
 * times into a CUDA graph of its own and run on the handle's stream, and keep
 * the fastest.  The choices apply at once (the Arnoldi step graphs are
 * recaptured) and are remembered by each level's (rows, nonzeros), so later
 * setups that build levels of the same sizes use them too.  before_us and
 * after_us (may be NULL) receive one whole B_P application's in-graph time
 * with the schedule before and after.  Call between solves: the timed parts
 * overwrite the work vectors.  Allocates only what the graph timing needs. */
int cpr_autotune(cpr_handle *h, int reps, double *before_us, double *after_us);

#ifdef __cplusplus
}
#endif
#endif /* CPR_B300_H */
