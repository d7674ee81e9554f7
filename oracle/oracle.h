/*
 * FP64 CPU oracle of the CPR-preconditioned FGMRES solve phase.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no code with
 * the CUDA library: no headers, helpers, tables or kernels.
 *
 * Conventions: 3x3 BSR blocks are stored row-major (9 doubles per block),
 * column indices are sorted within each row and every row holds its diagonal.
 * All arrays are caller-owned host arrays unless a function returns an o_csr*,
 * which the caller releases with o_csr_free().
 */
#ifndef CPR_ORACLE_H
#define CPR_ORACLE_H
#include <stdint.h>

#define O_OK 0
#define O_ERR_INVALID (-1)
#define O_ERR_SINGULAR (-4)
#define O_ERR_BREAKDOWN (-5)
#define O_NOT_CONVERGED 1

typedef struct {
    double theta_color;   /* Eq. 5.1 threshold for the smoother's coloring (0.05) */
    double theta_amg;     /* classical strength threshold for coarsening (0.25) */
    int mu;               /* adaptive-setup threshold of Alg. 3 (30) */
    int restart;          /* FGMRES restart length m (30) */
    int max_restarts;     /* restart cycles (MaxIt of Alg. 2) (100) */
    int precond_fp32;     /* ignored: the oracle computes in FP64 */
    int decouple;         /* 0: Pi_P^T is injection, 1: ABF weights w_i = D_i^-T e_1 */
    int pre, post;        /* smoothing sweeps of the V-cycle (1, 1) */
    int coarse_max;       /* coarsest level size for the dense LU (256) */
    int max_levels;       /* (20) */
    uint64_t seed;        /* hash seed of coloring and C/F splitting */
    int bilu_order;       /* 0: multicolor BILU(0) in (JP color, index) order;
                             1: natural order, the level-scheduled BILU of Sec. 6 (0) */
    int reuse_refresh;    /* 1: a B kept by Alg. 3 takes A^(k) for its second residual;
                             0: it keeps the copy of A it was built from (0) */
    int resetup;          /* when Alg. 3 rebuilds B and the pattern is unchanged: 0 full setup;
                             1 numeric only, keeping the last setup's levels, strength sets,
                             C/F splits and colorings (0) */
    int amg;              /* first stage: 0 classical AMG V-cycle; 1 the paper's
                             UA-AMG, double pairwise aggregation and the nonlinear AMLI-cycle
                             (Sec. 6) (0) */
    int amli_iters;       /* amg = 1: GCR steps of each coarse correction (2) */
    int coloring;         /* smoother coloring: 0 JP on S u S^T; 1 the paper's
                             VerticesSplitting/Grouping, Alg. 4-5 (0) */
    int agg_match;        /* amg = 1 matching: 0 greedy by (m_i, i); 1 handshake rounds, the
                             parallel form; 2 handshake rounds, then every node left alone that
                             has a candidate joins its best candidate's pair (0) */
    int coloring_rows;    /* coloring = 1 applies to levels of at most this many rows; larger
                             levels take JP (4096; 0 = every level) */
} o_opts;

typedef struct {
    int iters, restarts, setup_called, setup_count, levels, converged;
    double rel_res;
} o_stats;

typedef struct o_csr o_csr;
typedef struct o_handle o_handle;

/* ---- opaque CSR results ---- */
int  o_csr_n(const o_csr *c);
int  o_csr_ncol(const o_csr *c);
int  o_csr_nnz(const o_csr *c);
void o_csr_copy(const o_csr *c, int *rowptr, int *col, double *val);
void o_csr_free(o_csr *c);

/* ---- primitives (scalar CSR unless noted) ---- */
void   o_bsr3_spmv(int nb, const int *rowptr, const int *col, const double *val,
                   const double *x, double *y);
o_csr *o_strength_color(int n, const int *rowptr, const int *col, const double *val, double theta);
o_csr *o_sym_union(int n, const int *rowptr, const int *col);
int    o_jp_color(int n, const int *rowptr, const int *col, uint64_t seed, int salt, int level,
                  int *color);
uint32_t o_hash(uint64_t seed, int salt, int level, int i);
uint32_t o_fmix32(uint32_t h);   /* the finalizer itself, for checking against published values */
o_csr *o_strength_rs(int n, const int *rowptr, const int *col, const double *val, double theta);
int    o_pmis(int n, const int *srowptr, const int *scol, uint64_t seed, int salt, int level,
              int *cf);
o_csr *o_interp_direct(int n, const int *rowptr, const int *col, const double *val,
                       const int *srowptr, const int *scol, const int *cf);
o_csr *o_transpose(int n, int ncol, const int *rowptr, const int *col, const double *val);
o_csr *o_spgemm(int n, int ncolA, const int *arow, const int *acol, const double *aval,
                int ncolB, const int *brow, const int *bcol, const double *bval);
void   o_mcgs_sweep(int n, const int *rowptr, const int *col, const double *val,
                    const int *color, int ncolors, const double *b, double *x, int descending);
int    o_dense_lu_solve(int n, const double *a, const double *b, double *x);
int    o_decouple(int nb, const int *rowptr, const int *col, const double *val, int mode,
                  double *w, double *apval);
int    o_bilu0(int nb, const int *rowptr, const int *col, const double *val, uint64_t seed,
               int *bcolor, double *lu);
int    o_bilu0_natural(int nb, const int *rowptr, const int *col, const double *val, double *lu);
int    o_natural_levels(int nb, const int *rowptr, const int *col, int *level);
int    o_vertices_grouping(int n, const int *rowptr, const int *col, const double *val,
                           double theta, int *color);
int    o_aggregate(int n, const int *rowptr, const int *col, const double *val, double beta,
                   int passes, int match, int *agg);
void   o_bilu0_solve(int nb, const int *rowptr, const int *col, const double *lu,
                     const int *bcolor, int nbcolors, const double *r, double *z);
int    o_fgmres_identity(int nb, const int *rowptr, const int *col, const double *val,
                         const double *b, double *x, double rtol, int m, int max_restarts,
                         o_stats *st, double *hist);

/* Threads the library's parallel loops run on (1 unless compiled with OpenMP). */
int  o_threads(void);

/* ---- the solver (Alg. 2 with Alg. 3 deciding setup) ---- */
void o_default_opts(o_opts *o);
int  o_setup(o_handle **h, int nb, const int *rowptr, const int *col, const double *val,
             const o_opts *opt);
int  o_update(o_handle *h, int nb, const int *rowptr, const int *col, const double *val);
int  o_solve(o_handle *h, const double *b, double *x, double rtol, o_stats *st);
/* FGMRES on block rows [r0, r1) of a block-diagonal A (one system of a batch),
 * preconditioned by the handle's B restricted to those rows; does not count as
 * the handle's solve for Alg. 3. */
int  o_solve_rows(o_handle *h, int r0, int r1, const double *b, double *x, double rtol, o_stats *st);
void o_destroy(o_handle *h);

/* ---- inspection ---- */
int  o_num_levels(const o_handle *h);
void o_level_info(const o_handle *h, int l, int *n, int *nnz, int *ncolors, int *nc, int *nnzP);
void o_level_get(const o_handle *h, int l, int *rowptr, int *col, double *val, int *color,
                 int *cf, int *prow, int *pcol, double *pval);
void o_get_weights(const o_handle *h, double *w);
int  o_bilu_ncolors(const o_handle *h);
void o_bilu_get(const o_handle *h, int *bcolor, double *lu);
void o_cpr_apply(o_handle *h, const double *v, double *z);
void o_vcycle(o_handle *h, const double *b, double *x);
void o_bilu_apply(o_handle *h, const double *r, double *z);
int  o_last_iters(const o_handle *h);

#endif
