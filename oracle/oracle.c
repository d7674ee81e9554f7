/*
 * FP64 CPU oracle of the CPR-preconditioned FGMRES solve phase with adaptive
 * setup (Alg. 1-3), multi-color Gauss-Seidel over the strong-connection matrix
 * (Eq. 5.1, Alg. 6) inside a classical AMG V-cycle, and multicolor BILU(0).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the CUDA product path, with which it
 * shares no code.
 *
 * Written to be checked against the paper by eye: one step per function, loops
 * in the order the definitions state, no blocking and no fusion.  Built with
 * -ffp-contract=off so that every a*b+c is rounded twice, exactly as written.
 *
 * Readings of points the paper leaves open (each is named where it is used):
 *  R1 decoupling: Pi_P^T r takes w_i . r_i with w_i = D_i^-T e_1 (ABF) or e_1.
 *  R2 Eq. 5.1 sums |a_ik| over the whole row, diagonal included; the coloring
 *     graph is S united with its transpose.
 *  R3 colors: Jones-Plassmann with key (degree, hash, index) replaces the
 *     sequential greedy Alg. 4-5; each selected vertex takes the smallest
 *     color its colored neighbours leave free.
 *  R4 rows of one color are relaxed Jacobi-style (all read the iterate at the
 *     start of the color), so weakly coupled same-color rows stay deterministic.
 *  R5 V(1,1): pre-smoothing colors ascending, post-smoothing descending,
 *     starting from zero; classical strength, PMIS, direct interpolation,
 *     R = P^T, Galerkin R A P, dense LU on the coarsest level.
 *  R6 second stage: block ILU(0) in (color, index) order of a coloring of the
 *     block graph at theta = 0.
 *  R7 It of Alg. 3 is the number of inner (Arnoldi) steps of the last solve;
 *     a reused B keeps its own copy of A for the second residual of Alg. 1.
 *  Hash: MurmurHash3's 32-bit finalizer (fmix32), a published mixing function.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXLEV 32

/*
 * OMP_FOR marks loops whose iterations are independent: rows of one SpMV, the
 * rows of one color of a multi-color sweep or BILU(0) solve, and element-wise
 * vector updates.  Built with -fopenmp (the CPU baseline's multi-threaded
 * form) they run across threads; every iteration still does its own
 * arithmetic in the same order, so results are bit-identical to the
 * single-threaded build.  Dot products stay serial for the same reason.
 */
#ifdef _OPENMP
#include <omp.h>
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OMP_FOR
#endif

/* Threads the marked loops use: OpenMP's count in the multi-threaded build, 1 otherwise. */
int o_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

struct o_csr {
    int n, ncol, nnz;
    int *rowptr, *col;
    double *val; /* NULL for a pattern */
};

typedef struct {
    o_csr A;       /* level matrix A_l */
    int *color;    /* Eq. 5.1 coloring of A_l (not on the coarsest level) */
    int ncolors;
    int *cf;       /* 1 = C point, 0 = F point */
    int nc;        /* number of C points = size of level l+1 */
    o_csr P, R;    /* interpolation (n_l x n_{l+1}) and R = P^T */
    o_csr S;       /* classical strength set the interpolation used (kept for resetup = 1) */
    double *x, *b, *r, *tmp; /* V-cycle work vectors */
    double *gv, *gw, *gres;  /* amg = 1: the GCR vectors of a coarse correction on this level */
} level_t;

struct o_handle {
    o_opts opt;
    int nb, nnzb;
    int *rowptr, *col;
    double *val;   /* outer operator A^(k) */
    double *pval;  /* the copy of A inside B (the second residual of Alg. 1), frozen with B while Alg. 3 reuses it */
    double *w;     /* decoupling weights w_i = D_i^-T e_1, 3 per block row */
    int nlev;
    level_t lev[MAXLEV];
    double *clu;   /* coarsest level: dense LU, row-major, with row pivots */
    int *cpiv;
    int *bcolor;   /* BILU(0) block colors (JP at theta = 0 on the block graph) */
    int nbcolors;
    double *lu;    /* L blocks (unit diagonal implied), U blocks, U_ii^-1 at the diagonal */
    double *work1, *work2, *work3, *rp, *ep; /* CPR apply work vectors */
    long last_iters; /* It of Alg. 3: the inner steps of the previous solve; -1 = none since the last setup */
    int setup_count, setup_called, updates;
};

/* ------------------------------------------------------------------ helpers */

static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n ? n : 1, sz);
    if (!p) abort();
    return p;
}

static o_csr csr_alloc(int n, int ncol, int nnz, int with_val) {
    o_csr c;
    c.n = n;
    c.ncol = ncol;
    c.nnz = nnz;
    c.rowptr = xcalloc((size_t)n + 1, sizeof(int));
    c.col = xcalloc((size_t)nnz, sizeof(int));
    c.val = with_val ? xcalloc((size_t)nnz, sizeof(double)) : NULL;
    return c;
}

static void csr_release(o_csr *c) {
    free(c->rowptr);
    free(c->col);
    free(c->val);
    memset(c, 0, sizeof(*c));
}

static o_csr *csr_box(o_csr c) {
    o_csr *p = xcalloc(1, sizeof(o_csr));
    *p = c;
    return p;
}

static o_csr csr_view(int n, int ncol, const int *rowptr, const int *col, const double *val) {
    o_csr c;
    c.n = n;
    c.ncol = ncol;
    c.nnz = rowptr[n];
    c.rowptr = (int *)rowptr;
    c.col = (int *)col;
    c.val = (double *)val;
    return c;
}

int o_csr_n(const o_csr *c) { return c->n; }
int o_csr_ncol(const o_csr *c) { return c->ncol; }
int o_csr_nnz(const o_csr *c) { return c->nnz; }
void o_csr_copy(const o_csr *c, int *rowptr, int *col, double *val) {
    memcpy(rowptr, c->rowptr, sizeof(int) * ((size_t)c->n + 1));
    memcpy(col, c->col, sizeof(int) * (size_t)c->nnz);
    if (val && c->val) memcpy(val, c->val, sizeof(double) * (size_t)c->nnz);
}
void o_csr_free(o_csr *c) {
    if (!c) return;
    csr_release(c);
    free(c);
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static double dot(int n, const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* MurmurHash3 32-bit finalizer. */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

uint32_t o_fmix32(uint32_t h) { return fmix32(h); }

/* Per-vertex hash weight: salt 0 = smoother coloring, 1 = PMIS, 2 = BILU coloring. */
uint32_t o_hash(uint64_t seed, int salt, int level, int i) {
    uint32_t s32 = (uint32_t)(seed ^ (seed >> 32));
    uint32_t base = fmix32(s32 + 1000003u * (uint32_t)salt + (uint32_t)level);
    return fmix32((uint32_t)i ^ base);
}

/* Lexicographic comparison of keys (a, h, i): nonzero iff key 1 > key 2. */
static int key_greater(long a1, uint32_t h1, int i1, long a2, uint32_t h2, int i2) {
    if (a1 != a2) return a1 > a2;
    if (h1 != h2) return h1 > h2;
    return i1 > i2;
}

/* ------------------------------------------------------- 3x3 block algebra */

/* c = a * b */
static void mat3_mul(const double *a, const double *b, double *c) {
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double t = 0.0;
            for (int k = 0; k < 3; k++) t += a[3 * r + k] * b[3 * k + s];
            c[3 * r + s] = t;
        }
}

/* Inverse by the adjugate; returns 0 if the block is singular. */
static int mat3_inv(const double *a, double *inv) {
    double c00 = a[4] * a[8] - a[5] * a[7];
    double c01 = a[5] * a[6] - a[3] * a[8];
    double c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (det == 0.0 || !isfinite(det)) return 0;
    inv[0] = c00 / det;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    return 1;
}

/* ------------------------------------------------------------- 3x3 BSR SpMV */

/* y = A x for a 3x3 BSR matrix (Eq. 2.8 layout). */
void o_bsr3_spmv(int nb, const int *rowptr, const int *col, const double *val,
                 const double *x, double *y) {
    OMP_FOR
    for (int i = 0; i < nb; i++) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const double *blk = val + 9 * (size_t)p;
            const double *xj = x + 3 * (size_t)col[p];
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) s[r] += blk[3 * r + c] * xj[c];
        }
        y[3 * i] = s[0];
        y[3 * i + 1] = s[1];
        y[3 * i + 2] = s[2];
    }
}

static void bsr3_resid(int nb, const int *rowptr, const int *col, const double *val,
                       const double *b, const double *x, double *r) {
    o_bsr3_spmv(nb, rowptr, col, val, x, r);
    OMP_FOR
    for (int i = 0; i < 3 * nb; i++) r[i] = b[i] - r[i];
}

/* -------------------------------------------------------------- decoupling */

/*
 * Pressure decoupling and the pressure matrix (Eq. 3.1; mode 1 takes ABF weights in
 * place of the paper's plain injection).
 * mode 1: w_i = D_i^-T e_1, i.e. the first row of D_i^-1 by the adjugate:
 *   w_i = (C00, C10, C20) / det(D_i),  det = D00 C00 + D10 C10 + D20 C20.
 * mode 0: w_i = e_1 (plain injection).
 * A_P[i][j] = w_i . (column 0 of block A_ij), on the full block pattern.
 */
int o_decouple(int nb, const int *rowptr, const int *col, const double *val, int mode,
               double *w, double *apval) {
    for (int i = 0; i < nb; i++) {
        if (mode == 0) {
            w[3 * i] = 1.0;
            w[3 * i + 1] = 0.0;
            w[3 * i + 2] = 0.0;
            continue;
        }
        const double *d = NULL;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (col[p] == i) d = val + 9 * (size_t)p;
        if (!d) return O_ERR_INVALID;
        double c00 = d[4] * d[8] - d[5] * d[7];
        double c10 = d[2] * d[7] - d[1] * d[8];
        double c20 = d[1] * d[5] - d[2] * d[4];
        double det = (d[0] * c00 + d[3] * c10) + d[6] * c20;
        if (det == 0.0 || !isfinite(det)) return O_ERR_SINGULAR;
        w[3 * i] = c00 / det;
        w[3 * i + 1] = c10 / det;
        w[3 * i + 2] = c20 / det;
    }
    for (int i = 0; i < nb; i++)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const double *a = val + 9 * (size_t)p;
            apval[p] = (w[3 * i] * a[0] + w[3 * i + 1] * a[3]) + w[3 * i + 2] * a[6];
        }
    return O_OK;
}

/* ------------------------------------------------- strength and coloring */

/* Eq. 5.1: j in S_i iff j != i and |a_ij| > theta * sum_k |a_ik|, the sum over the
 * whole row, the diagonal included. */
static o_csr strength_color(const o_csr *A, double theta) {
    int n = A->n;
    o_csr S = csr_alloc(n, n, A->nnz, 0);
    int nnz = 0;
    for (int i = 0; i < n; i++) {
        double rowsum = 0.0;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) rowsum += fabs(A->val[p]);
        double t = theta * rowsum;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
            int j = A->col[p];
            if (j != i && fabs(A->val[p]) > t) S.col[nnz++] = j;
        }
        S.rowptr[i + 1] = nnz;
    }
    S.nnz = nnz;
    return S;
}

o_csr *o_strength_color(int n, const int *rowptr, const int *col, const double *val,
                        double theta) {
    o_csr A = csr_view(n, n, rowptr, col, val);
    return csr_box(strength_color(&A, theta));
}

/* Transpose by counting; scanning source rows in ascending order leaves each
 * row of the result sorted. */
static o_csr transpose(const o_csr *A) {
    o_csr T = csr_alloc(A->ncol, A->n, A->nnz, A->val != NULL);
    for (int p = 0; p < A->nnz; p++) T.rowptr[A->col[p] + 1]++;
    for (int j = 0; j < A->ncol; j++) T.rowptr[j + 1] += T.rowptr[j];
    int *next = xcalloc((size_t)A->ncol, sizeof(int));
    for (int j = 0; j < A->ncol; j++) next[j] = T.rowptr[j];
    for (int i = 0; i < A->n; i++)
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
            int q = next[A->col[p]]++;
            T.col[q] = i;
            if (A->val) T.val[q] = A->val[p];
        }
    free(next);
    return T;
}

o_csr *o_transpose(int n, int ncol, const int *rowptr, const int *col, const double *val) {
    o_csr A = csr_view(n, ncol, rowptr, col, val);
    return csr_box(transpose(&A));
}

/* Pattern of S united with S^T (the undirected graph the colorings use), sorted rows. */
static o_csr sym_union(const o_csr *S) {
    o_csr T = transpose(S);
    int n = S->n;
    o_csr G = csr_alloc(n, n, S->nnz + T.nnz, 0);
    int nnz = 0;
    for (int i = 0; i < n; i++) {
        int p = S->rowptr[i], pe = S->rowptr[i + 1];
        int q = T.rowptr[i], qe = T.rowptr[i + 1];
        while (p < pe || q < qe) {
            int a = p < pe ? S->col[p] : n;
            int b = q < qe ? T.col[q] : n;
            int c = a < b ? a : b;
            if (a == c) p++;
            if (b == c) q++;
            G.col[nnz++] = c;
        }
        G.rowptr[i + 1] = nnz;
    }
    G.nnz = nnz;
    csr_release(&T);
    return G;
}

o_csr *o_sym_union(int n, const int *rowptr, const int *col) {
    o_csr S = csr_view(n, n, rowptr, col, NULL);
    return csr_box(sym_union(&S));
}

/*
 * Jones-Plassmann coloring of an undirected graph G, standing in for the sequential
 * Alg. 4-5.
 * key(i) = (deg_G(i), hash(i), i).  Each round, from the round-start state,
 * every uncolored vertex whose key beats all uncolored neighbours is selected;
 * each selected vertex takes the smallest color not held by a neighbour.
 * Returns the number of colors.
 */
static int jp_color(const o_csr *G, uint64_t seed, int salt, int level, int *color) {
    int n = G->n;
    uint32_t *h = xcalloc((size_t)n, sizeof(uint32_t));
    char *sel = xcalloc((size_t)n, 1);
    char *used = xcalloc((size_t)n + 2, 1);
    for (int i = 0; i < n; i++) {
        color[i] = -1;
        h[i] = o_hash(seed, salt, level, i);
    }
    int left = n, ncolors = 0;
    while (left > 0) {
        for (int i = 0; i < n; i++) {
            sel[i] = 0;
            if (color[i] >= 0) continue;
            int best = 1;
            long di = G->rowptr[i + 1] - G->rowptr[i];
            for (int p = G->rowptr[i]; p < G->rowptr[i + 1] && best; p++) {
                int j = G->col[p];
                if (j == i || color[j] >= 0) continue;
                long dj = G->rowptr[j + 1] - G->rowptr[j];
                if (!key_greater(di, h[i], i, dj, h[j], j)) best = 0;
            }
            sel[i] = (char)best;
        }
        for (int i = 0; i < n; i++) {
            if (!sel[i]) continue;
            int deg = G->rowptr[i + 1] - G->rowptr[i];
            for (int p = G->rowptr[i]; p < G->rowptr[i + 1]; p++) {
                int c = color[G->col[p]];
                if (c >= 0 && c <= deg) used[c] = 1;
            }
            int c = 0;
            while (used[c]) c++;
            for (int p = G->rowptr[i]; p < G->rowptr[i + 1]; p++) {
                int cj = color[G->col[p]];
                if (cj >= 0 && cj <= deg) used[cj] = 0;
            }
            color[i] = c;
            if (c + 1 > ncolors) ncolors = c + 1;
            left--;
        }
    }
    free(h);
    free(sel);
    free(used);
    return ncolors;
}

int o_jp_color(int n, const int *rowptr, const int *col, uint64_t seed, int salt, int level,
               int *color) {
    o_csr G = csr_view(n, n, rowptr, col, NULL);
    return jp_color(&G, seed, salt, level, color);
}

/* ------------------------------------------------------------ coarsening */

/*
 * Classical (Ruge-Stueben) strength: with s = sign(a_ii) (+1 when a_ii >= 0),
 * j in S_i iff j != i and -s a_ij >= theta * max_{k != i}(-s a_ik), provided
 * that maximum is positive (otherwise S_i is empty).
 */
static o_csr strength_rs(const o_csr *A, double theta) {
    int n = A->n;
    o_csr S = csr_alloc(n, n, A->nnz, 0);
    int nnz = 0;
    for (int i = 0; i < n; i++) {
        double aii = 0.0;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++)
            if (A->col[p] == i) aii = A->val[p];
        double s = aii < 0.0 ? -1.0 : 1.0;
        double m = 0.0;
        int have = 0;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
            if (A->col[p] == i) continue;
            double v = -s * A->val[p];
            if (!have || v > m) m = v;
            have = 1;
        }
        if (have && m > 0.0) {
            double t = theta * m;
            for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
                int j = A->col[p];
                if (j != i && -s * A->val[p] >= t) S.col[nnz++] = j;
            }
        }
        S.rowptr[i + 1] = nnz;
    }
    S.nnz = nnz;
    return S;
}

o_csr *o_strength_rs(int n, const int *rowptr, const int *col, const double *val,
                     double theta) {
    o_csr A = csr_view(n, n, rowptr, col, val);
    return csr_box(strength_rs(&A, theta));
}

/*
 * PMIS C/F splitting on the strength graph S (S_i = points i depends on).
 * lambda_i = |S^T_i| (how many points depend on i); key = (lambda, hash, index).
 * A point with S_i and S^T_i both empty is F from the start.  Each round, from
 * the round-start state, an undecided point whose key beats every undecided
 * point of S_i u S^T_i becomes C; then every undecided point with a C point in
 * S_i becomes F.  cf: 1 = C, 0 = F.  Returns the number of C points.
 */
static int pmis(const o_csr *S, uint64_t seed, int salt, int level, int *cf) {
    int n = S->n;
    o_csr T = transpose(S);
    uint32_t *h = xcalloc((size_t)n, sizeof(uint32_t));
    char *newc = xcalloc((size_t)n, 1);
    int undecided = 0;
    for (int i = 0; i < n; i++) {
        h[i] = o_hash(seed, salt, level, i);
        int si = S->rowptr[i + 1] - S->rowptr[i];
        int ti = T.rowptr[i + 1] - T.rowptr[i];
        cf[i] = (si == 0 && ti == 0) ? 0 : -1;
        if (cf[i] < 0) undecided++;
    }
    while (undecided > 0) {
        for (int i = 0; i < n; i++) {
            newc[i] = 0;
            if (cf[i] != -1) continue;
            long li = T.rowptr[i + 1] - T.rowptr[i];
            int best = 1;
            for (int pass = 0; pass < 2 && best; pass++) {
                const o_csr *M = pass == 0 ? S : &T;
                for (int p = M->rowptr[i]; p < M->rowptr[i + 1] && best; p++) {
                    int j = M->col[p];
                    if (cf[j] != -1) continue;
                    long lj = T.rowptr[j + 1] - T.rowptr[j];
                    if (!key_greater(li, h[i], i, lj, h[j], j)) best = 0;
                }
            }
            newc[i] = (char)best;
        }
        for (int i = 0; i < n; i++)
            if (newc[i]) {
                cf[i] = 1;
                undecided--;
            }
        for (int i = 0; i < n; i++) {
            if (cf[i] != -1) continue;
            for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++)
                if (cf[S->col[p]] == 1) {
                    cf[i] = 0;
                    undecided--;
                    break;
                }
        }
    }
    int nc = 0;
    for (int i = 0; i < n; i++) nc += cf[i] == 1;
    csr_release(&T);
    free(h);
    free(newc);
    return nc;
}

int o_pmis(int n, const int *srowptr, const int *scol, uint64_t seed, int salt, int level,
           int *cf) {
    o_csr S = csr_view(n, n, srowptr, scol, NULL);
    return pmis(&S, seed, salt, level, cf);
}

/*
 * Direct interpolation (Stueben) with separate scaling of negative and
 * positive couplings.  C point i: P_i = e_{cidx(i)}.  F point i with
 * C_i = S_i n C (sorted): with s = sign(a_ii) and a~ = s a,
 *   alpha = sum_{k != i} min(a~_ik, 0) / sum_{k in C_i} min(a~_ik, 0),
 *   beta  = sum_{k != i} max(a~_ik, 0) / sum_{k in C_i} max(a~_ik, 0),
 *   d = a~_ii, or a~_ii + sum_{k != i} max(a~_ik, 0) when C_i has no positive
 *   entry (the positive part is lumped into the diagonal),
 *   w_ij = -alpha a~_ij / d  (a~_ij < 0),   -beta a~_ij / d  (otherwise).
 * An F point with C_i empty gets an empty row.
 */
static o_csr interp_direct(const o_csr *A, const o_csr *S, const int *cf) {
    int n = A->n;
    int *cidx = xcalloc((size_t)n, sizeof(int));
    int nc = 0;
    for (int i = 0; i < n; i++) cidx[i] = cf[i] == 1 ? nc++ : -1;
    int nnz = 0;
    for (int i = 0; i < n; i++) {
        if (cf[i] == 1) {
            nnz++;
            continue;
        }
        for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++) nnz += cf[S->col[p]] == 1;
    }
    o_csr P = csr_alloc(n, nc, nnz, 1);
    int q = 0;
    for (int i = 0; i < n; i++) {
        if (cf[i] == 1) {
            P.col[q] = cidx[i];
            P.val[q] = 1.0;
            q++;
            P.rowptr[i + 1] = q;
            continue;
        }
        double aii = 0.0;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++)
            if (A->col[p] == i) aii = A->val[p];
        double s = aii < 0.0 ? -1.0 : 1.0;
        double sum_n_neg = 0.0, sum_n_pos = 0.0;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
            if (A->col[p] == i) continue;
            double v = s * A->val[p];
            if (v < 0.0) sum_n_neg += v;
            else sum_n_pos += v;
        }
        /* a~_ik for k in C_i: walk S_i and A's row together (both sorted) */
        double sum_c_neg = 0.0, sum_c_pos = 0.0;
        int pa = A->rowptr[i];
        for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++) {
            int j = S->col[p];
            if (cf[j] != 1) continue;
            while (A->col[pa] != j) pa++;
            double v = s * A->val[pa];
            if (v < 0.0) sum_c_neg += v;
            else sum_c_pos += v;
        }
        double d = s * aii;
        double alpha = 0.0, beta = 0.0;
        if (sum_c_neg != 0.0) alpha = sum_n_neg / sum_c_neg;
        if (sum_c_pos != 0.0) beta = sum_n_pos / sum_c_pos;
        else d = d + sum_n_pos;
        pa = A->rowptr[i];
        for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++) {
            int j = S->col[p];
            if (cf[j] != 1) continue;
            while (A->col[pa] != j) pa++;
            double v = s * A->val[pa];
            double f = v < 0.0 ? -alpha : -beta;
            P.col[q] = cidx[j];
            P.val[q] = (f * v) / d;
            q++;
        }
        P.rowptr[i + 1] = q;
    }
    free(cidx);
    return P;
}

o_csr *o_interp_direct(int n, const int *rowptr, const int *col, const double *val,
                       const int *srowptr, const int *scol, const int *cf) {
    o_csr A = csr_view(n, n, rowptr, col, val);
    o_csr S = csr_view(n, n, srowptr, scol, NULL);
    return csr_box(interp_direct(&A, &S, cf));
}

/*
 * C = A B, Gustavson's row-by-row product with a dense accumulator: for each
 * row i, for k in A_i ascending, for j in B_k ascending, acc[j] += a_ik b_kj.
 * The pattern is the structural product (explicit zeros kept), sorted.
 */
static o_csr spgemm(const o_csr *A, const o_csr *B) {
    int n = A->n, m = B->ncol;
    int *mark = xcalloc((size_t)m, sizeof(int));
    double *acc = xcalloc((size_t)m, sizeof(double));
    for (int j = 0; j < m; j++) mark[j] = -1;
    long nnz = 0;
    for (int i = 0; i < n; i++)
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
            int k = A->col[p];
            for (int q = B->rowptr[k]; q < B->rowptr[k + 1]; q++)
                if (mark[B->col[q]] != i) {
                    mark[B->col[q]] = i;
                    nnz++;
                }
        }
    o_csr C = csr_alloc(n, m, (int)nnz, 1);
    for (int j = 0; j < m; j++) mark[j] = -1;
    int c = 0;
    for (int i = 0; i < n; i++) {
        int start = c;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
            int k = A->col[p];
            for (int q = B->rowptr[k]; q < B->rowptr[k + 1]; q++) {
                int j = B->col[q];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    C.col[c++] = j;
                }
                acc[j] = acc[j] + A->val[p] * B->val[q];
            }
        }
        qsort(C.col + start, (size_t)(c - start), sizeof(int), cmp_int);
        for (int q = start; q < c; q++) C.val[q] = acc[C.col[q]];
        C.rowptr[i + 1] = c;
    }
    free(mark);
    free(acc);
    return C;
}

o_csr *o_spgemm(int n, int ncolA, const int *arow, const int *acol, const double *aval,
                int ncolB, const int *brow, const int *bcol, const double *bval) {
    o_csr A = csr_view(n, ncolA, arow, acol, aval);
    o_csr B = csr_view(ncolA, ncolB, brow, bcol, bval);
    return csr_box(spgemm(&A, &B));
}

/* ----------------------------------------------------------- dense LU */

/* LU with partial pivoting (largest |a|, lowest row index on ties), in place. */
static int dense_lu(int n, double *a, int *piv) {
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(a[(size_t)i * n + k]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        piv[k] = p;
        if (best == 0.0) return O_ERR_SINGULAR;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        for (int i = k + 1; i < n; i++) {
            double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
            a[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    return O_OK;
}

static void dense_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x) {
    for (int i = 0; i < n; i++) x[i] = b[i];
    for (int k = 0; k < n; k++) {
        double t = x[k];
        x[k] = x[piv[k]];
        x[piv[k]] = t;
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < i; j++) x[i] -= lu[(size_t)i * n + j] * x[j];
    for (int i = n - 1; i >= 0; i--) {
        for (int j = i + 1; j < n; j++) x[i] -= lu[(size_t)i * n + j] * x[j];
        x[i] /= lu[(size_t)i * n + i];
    }
}

int o_dense_lu_solve(int n, const double *a, const double *b, double *x) {
    double *lu = xcalloc((size_t)n * n, sizeof(double));
    int *piv = xcalloc((size_t)n, sizeof(int));
    memcpy(lu, a, sizeof(double) * (size_t)n * n);
    int rc = dense_lu(n, lu, piv);
    if (rc == O_OK) dense_lu_solve(n, lu, piv, b, x);
    free(lu);
    free(piv);
    return rc;
}

/* ------------------------------------------------- multi-color Gauss-Seidel */

/*
 * One sweep of PGS-SCM (Alg. 6): colors in order (ascending, or descending
 * when `descending`), each row i of the color taking
 *   x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii
 * with every x_j read as of the start of the color.
 */
static void mcgs_sweep(const o_csr *A, const int *color, int ncolors, const double *b,
                       double *x, int descending, double *tmp) {
    for (int t = 0; t < ncolors; t++) {
        int c = descending ? ncolors - 1 - t : t;
        OMP_FOR
        for (int i = 0; i < A->n; i++) {
            if (color[i] != c) continue;
            double s = b[i], d = 0.0;
            for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++) {
                int j = A->col[p];
                if (j == i) d = A->val[p];
                else s -= A->val[p] * x[j];
            }
            tmp[i] = s / d;
        }
        OMP_FOR
        for (int i = 0; i < A->n; i++)
            if (color[i] == c) x[i] = tmp[i];
    }
}

void o_mcgs_sweep(int n, const int *rowptr, const int *col, const double *val, const int *color,
                  int ncolors, const double *b, double *x, int descending) {
    o_csr A = csr_view(n, n, rowptr, col, val);
    double *tmp = xcalloc((size_t)n, sizeof(double));
    mcgs_sweep(&A, color, ncolors, b, x, descending, tmp);
    free(tmp);
}

/* ------------------------ Alg. 4-5: VerticesSplitting / VerticesGrouping (f1) */

/*
 * One call of VerticesSplitting (Alg. 4) on the vertices with inV set, over
 * the strong-connection matrix S (Eq. 5.1, rows as computed, not
 * symmetrised), with these readings of its loosely defined parts:
 *  - "any take" picks, among the candidates with the largest |S_i|, the one
 *    of lowest index;
 *  - the candidates are the second-circle set W^ restricted to V when that
 *    is not empty, else V;
 *  - a vertex's color is undetermined while it is in V;
 *  - S^_i = (union of S_k over k in S_i) minus (S_i and i), restricted to V;
 *  - W-bar takes only the members of S_i that are still in V.
 * The vertices put in W get `c`; the others of V are left with inV set for
 * the next call.  Returns the size of W.
 */
static int vertices_splitting(const o_csr *S, char *inV, int *color, int c, char *inW, char *inHat) {
    int n = S->n, nW = 0, left = 0;
    for (int i = 0; i < n; i++) {
        inW[i] = 0;
        inHat[i] = 0;
        left += inV[i];
    }
    char *inBar = xcalloc((size_t)n, 1);   /* W-bar: out of V for this call, kept for the next */
    int nhat = 0;
    while (left > 0) {
        int best = -1, bdeg = -1;
        for (int pass = nhat > 0 ? 0 : 1; pass < 2 && best < 0; pass++)
            for (int i = 0; i < n; i++) {
                if (!inV[i] || inBar[i] || inW[i] || (pass == 0 && !inHat[i])) continue;
                int d = S->rowptr[i + 1] - S->rowptr[i];
                if (d > bdeg) {
                    best = i;
                    bdeg = d;
                }
            }
        int i = best;
        int free_of_w = 1;
        for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++)
            if (inW[S->col[p]]) free_of_w = 0;
        if (inHat[i]) {
            inHat[i] = 0;
            nhat--;
        }
        left--;
        if (free_of_w) {
            inW[i] = 1;
            color[i] = c;
            nW++;
            for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++) {
                int j = S->col[p];
                if (!inV[j] || inBar[j] || inW[j]) continue;
                inBar[j] = 1;
                left--;
                if (inHat[j]) {
                    inHat[j] = 0;
                    nhat--;
                }
            }
            /* the second circle of i */
            for (int p = S->rowptr[i]; p < S->rowptr[i + 1]; p++) {
                int k = S->col[p];
                for (int q = S->rowptr[k]; q < S->rowptr[k + 1]; q++) {
                    int j = S->col[q];
                    if (j == i || !inV[j] || inBar[j] || inW[j] || inHat[j]) continue;
                    int in_si = 0;
                    for (int t = S->rowptr[i]; t < S->rowptr[i + 1]; t++)
                        if (S->col[t] == j) in_si = 1;
                    if (in_si) continue;
                    inHat[j] = 1;
                    nhat++;
                }
            }
        } else {
            inBar[i] = 1;
        }
    }
    /* V for the next call: W-bar */
    for (int i = 0; i < n; i++) inV[i] = inBar[i];
    free(inBar);
    return nW;
}

/* VerticesGrouping (Alg. 5): repeated splitting until every vertex has a group. */
static int vertices_grouping(const o_csr *S, int *color) {
    int n = S->n, c = 0, left = n;
    char *inV = xcalloc((size_t)n, 1), *inW = xcalloc((size_t)n, 1), *inHat = xcalloc((size_t)n, 1);
    for (int i = 0; i < n; i++) {
        inV[i] = 1;
        color[i] = -1;
    }
    while (left > 0) {
        left -= vertices_splitting(S, inV, color, c, inW, inHat);
        c++;
    }
    for (int i = 0; i < n; i++)
        if (color[i] < 0) abort();   /* every vertex leaves V through W or W-bar */
    free(inV);
    free(inW);
    free(inHat);
    return c;
}

int o_vertices_grouping(int n, const int *rowptr, const int *col, const double *val, double theta,
                        int *color) {
    o_csr A = csr_view(n, n, rowptr, col, val);
    o_csr S = strength_color(&A, theta);
    int c = vertices_grouping(&S, color);
    csr_release(&S);
    return c;
}

/* --------------------------------------- UA-AMG: pairwise aggregation (f2) */

/* A binary min-heap of (key, node) pairs with lazy deletion. */
typedef struct {
    long *key;
    int *node;
    int size, cap;
} heap_t;

static void heap_push(heap_t *q, long key, int node) {
    if (q->size == q->cap) {
        q->cap = q->cap ? 2 * q->cap : 64;
        q->key = realloc(q->key, sizeof(long) * (size_t)q->cap);
        q->node = realloc(q->node, sizeof(int) * (size_t)q->cap);
        if (!q->key || !q->node) abort();
    }
    int c = q->size++;
    while (c > 0) {
        int p = (c - 1) / 2;
        if (q->key[p] < key || (q->key[p] == key && q->node[p] < node)) break;
        q->key[c] = q->key[p];
        q->node[c] = q->node[p];
        c = p;
    }
    q->key[c] = key;
    q->node[c] = node;
}

static void heap_pop(heap_t *q, long *key, int *node) {
    *key = q->key[0];
    *node = q->node[0];
    long k = q->key[--q->size];
    int v = q->node[q->size];
    int c = 0;
    for (;;) {
        int l = 2 * c + 1, r = l + 1, m = c;
        long mk = k;
        int mv = v;
        if (l < q->size && (q->key[l] < mk || (q->key[l] == mk && q->node[l] < mv))) {
            m = l;
            mk = q->key[l];
            mv = q->node[l];
        }
        if (r < q->size && (q->key[r] < mk || (q->key[r] == mk && q->node[r] < mv))) m = r;
        if (m == c) break;
        q->key[c] = q->key[m];
        q->node[c] = q->node[m];
        c = m;
    }
    if (q->size) {
        q->key[c] = k;
        q->node[c] = v;
    }
}

/*
 * One pass of pairwise matching (the pairwise aggregation Sec. 6
 * names as NPAIR, taken on the symmetrised couplings c_ij = (a_ij + a_ji) / 2
 * so that a nonsymmetric A is matched as its symmetric part).
 *  - j != i is a strong neighbour of i when c_ij < 0 and
 *    -c_ij >= beta * max_{k != i} (-c_ik).
 *  - m_i = the number of unmatched nodes that have i as a strong neighbour.
 *  - The unmatched node i of smallest (m_i, i) is matched with its unmatched
 *    strong neighbour j of smallest (c_ij, j), or stays alone if it has none.
 *    Both leave the pool, and each of their strong neighbours' m drops by one.
 * agg[i] = aggregate index, numbered in the order the aggregates form.
 * Returns the number of aggregates.
 */
/*
 * Handshake rounds (agg_match = 1: the parallel reading of the matching).
 * Candidates are symmetric: j is a candidate of i when either is a
 * strong neighbour of the other.  Each edge has one key for both ends,
 * (c_ij, smaller hash, larger hash), unique per edge since the hash is a
 * bijection of the index.  In a round every
 * unmatched node points to its unmatched candidate of smallest key; mutual
 * pointers pair up; an unmatched node with no unmatched candidate stays
 * alone.  The smallest remaining edge is always mutual, so every round pairs
 * or settles at least one node.  Aggregates are numbered by their smallest
 * node.  With `attach` (agg_match = 2) a node left alone joins the pair of
 * its best candidate, if it has one (see below): rounds alone leave many
 * singletons on heterogeneous media, and they pile up level after level
 * until coarsening stalls, which the greedy matching does not do.
 */
static int handshake_match(int n, const int *srow, const int *scol, const double *sval, uint32_t hb,
                           int attach, int *agg) {
    /* the symmetric candidate lists with their couplings */
    int *crow = xcalloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; i++)
        for (int t = srow[i]; t < srow[i + 1]; t++) {
            crow[i + 1]++;
            crow[scol[t] + 1]++;
        }
    for (int i = 0; i < n; i++) crow[i + 1] += crow[i];
    int *cc = xcalloc((size_t)crow[n] + 1, sizeof(int)), *fill = xcalloc((size_t)n, sizeof(int));
    double *cv = xcalloc((size_t)crow[n] + 1, sizeof(double));
    for (int i = 0; i < n; i++)
        for (int t = srow[i]; t < srow[i + 1]; t++) {
            int j = scol[t];
            cc[crow[i] + fill[i]] = j;
            cv[crow[i] + fill[i]++] = sval[t];
            cc[crow[j] + fill[j]] = i;
            cv[crow[j] + fill[j]++] = sval[t];
        }
    int *mate = xcalloc((size_t)n, sizeof(int)), *ptr = xcalloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; i++) mate[i] = -2;   /* -2 unmatched, -1 alone, else the partner */
    int left = n;
    while (left > 0) {
        for (int i = 0; i < n; i++) {
            ptr[i] = -1;
            if (mate[i] != -2) continue;
            double bc = 0.0;
            uint32_t blo = 0, bhi = 0;
            int bj = -1;
            for (int t = crow[i]; t < crow[i + 1]; t++) {
                int j = cc[t];
                if (mate[j] != -2 || j == i) continue;
                uint32_t hi_ = fmix32((uint32_t)i ^ hb), hj = fmix32((uint32_t)j ^ hb);
                uint32_t lo = hi_ < hj ? hi_ : hj, hi = hi_ < hj ? hj : hi_;
                int better = bj < 0 || cv[t] < bc ||
                             (cv[t] == bc && (lo < blo || (lo == blo && (hi < bhi || (hi == bhi && j < bj)))));
                if (better) {
                    bj = j;
                    bc = cv[t];
                    blo = lo;
                    bhi = hi;
                }
            }
            ptr[i] = bj;
        }
        for (int i = 0; i < n; i++) {
            if (mate[i] != -2) continue;
            if (ptr[i] < 0) {
                mate[i] = -1;
                left--;
            } else if (ptr[ptr[i]] == i && i < ptr[i]) {
                mate[i] = ptr[i];
                mate[ptr[i]] = i;
                left -= 2;
            }
        }
    }
    int na = 0;
    for (int i = 0; i < n; i++) agg[i] = -1;
    if (attach) {
        /* agg_match = 2: a node left alone that has a candidate joins the pair
           of its candidate of smallest edge key (every candidate of a node left
           alone is paired: an unmatched candidate would still have been one,
           and the two would have pointed somewhere).  A pair may take several
           such nodes.  Pairs and the nodes with no candidate at all are
           numbered by their smallest node; a joining node takes its host
           pair's number. */
        int *host = xcalloc((size_t)n, sizeof(int));
        for (int i = 0; i < n; i++) {
            host[i] = -1;
            if (mate[i] != -1) continue;
            double bc = 0.0;
            uint32_t blo = 0, bhi = 0;
            int bj = -1;
            for (int t = crow[i]; t < crow[i + 1]; t++) {
                int j = cc[t];
                if (j == i) continue;
                uint32_t hi_ = fmix32((uint32_t)i ^ hb), hj = fmix32((uint32_t)j ^ hb);
                uint32_t lo = hi_ < hj ? hi_ : hj, hi = hi_ < hj ? hj : hi_;
                int better = bj < 0 || cv[t] < bc ||
                             (cv[t] == bc && (lo < blo || (lo == blo && (hi < bhi || (hi == bhi && j < bj)))));
                if (better) {
                    bj = j;
                    bc = cv[t];
                    blo = lo;
                    bhi = hi;
                }
            }
            host[i] = bj;
        }
        for (int i = 0; i < n; i++) {
            if (host[i] >= 0 || agg[i] >= 0) continue;
            agg[i] = na;
            if (mate[i] >= 0) agg[mate[i]] = na;
            na++;
        }
        for (int i = 0; i < n; i++)
            if (host[i] >= 0) agg[i] = agg[host[i]];
        free(host);
    } else {
        for (int i = 0; i < n; i++) {
            if (agg[i] >= 0) continue;
            agg[i] = na;
            if (mate[i] >= 0) agg[mate[i]] = na;
            na++;
        }
    }
    free(crow);
    free(cc);
    free(fill);
    free(cv);
    free(mate);
    free(ptr);
    return na;
}

static int pairwise_pass(const o_csr *A, double beta, int match, uint32_t hb, int *agg) {
    int n = A->n;
    o_csr T = transpose(A);
    /* S with its couplings: row i holds the strong neighbours of i */
    int *srow = xcalloc((size_t)n + 1, sizeof(int));
    int cap = A->nnz + T.nnz + 1;
    int *scol = xcalloc((size_t)cap, sizeof(int));
    double *sval = xcalloc((size_t)cap, sizeof(double));
    int *ccol = xcalloc((size_t)n + 1, sizeof(int));
    double *cval = xcalloc((size_t)n + 1, sizeof(double));
    int nnz = 0;
    for (int i = 0; i < n; i++) {
        /* merge row i of A and of A^T: the couplings of i, off the diagonal */
        int p = A->rowptr[i], pe = A->rowptr[i + 1], q = T.rowptr[i], qe = T.rowptr[i + 1], nc = 0;
        double maxneg = 0.0;
        while (p < pe || q < qe) {
            int a = p < pe ? A->col[p] : n, b = q < qe ? T.col[q] : n;
            int j = a < b ? a : b;
            double c = 0.0;
            if (a == j) c += A->val[p++];
            if (b == j) c += T.val[q++];
            if (j == i) continue;
            c = 0.5 * c;
            ccol[nc] = j;
            cval[nc++] = c;
            if (-c > maxneg) maxneg = -c;
        }
        for (int t = 0; t < nc; t++)
            if (cval[t] < 0.0 && maxneg > 0.0 && -cval[t] >= beta * maxneg) {
                scol[nnz] = ccol[t];
                sval[nnz++] = cval[t];
            }
        srow[i + 1] = nnz;
    }
    if (match == 1 || match == 2) {
        int na = handshake_match(n, srow, scol, sval, hb, match == 2, agg);
        free(ccol);
        free(cval);
        free(srow);
        free(scol);
        free(sval);
        csr_release(&T);
        return na;
    }
    int *m = xcalloc((size_t)n, sizeof(int));
    for (int k = 0; k < nnz; k++) m[scol[k]]++;
    char *done = xcalloc((size_t)n, 1);
    heap_t h = {0};
    for (int i = 0; i < n; i++) heap_push(&h, m[i], i);
    int na = 0;
    while (h.size) {
        long key;
        int i;
        heap_pop(&h, &key, &i);
        if (done[i] || key != m[i]) continue;   /* a stale entry */
        int j = -1;
        double cj = 0.0;
        for (int t = srow[i]; t < srow[i + 1]; t++) {
            int k = scol[t];
            if (done[k]) continue;
            if (j < 0 || sval[t] < cj || (sval[t] == cj && k < j)) {
                j = k;
                cj = sval[t];
            }
        }
        int pair[2] = {i, j};
        for (int u = 0; u < 2 && pair[u] >= 0; u++) {
            int v = pair[u];
            done[v] = 1;
            agg[v] = na;
            for (int t = srow[v]; t < srow[v + 1]; t++) {
                int k = scol[t];
                if (done[k]) continue;
                m[k]--;
                heap_push(&h, m[k], k);
            }
        }
        na++;
    }
    free(h.key);
    free(h.node);
    free(done);
    free(m);
    free(ccol);
    free(cval);
    free(srow);
    free(scol);
    free(sval);
    csr_release(&T);
    return na;
}

/* Unsmoothed aggregation's P (n x nc): row i is the unit row of aggregate agg[i]. */
static o_csr agg_to_p(int n, int nc, const int *agg) {
    o_csr P = csr_alloc(n, nc, n, 1);
    for (int i = 0; i < n; i++) {
        P.col[i] = agg[i];
        P.val[i] = 1.0;
        P.rowptr[i + 1] = i + 1;
    }
    return P;
}

/*
 * Double pairwise aggregation: a pass on A, then a pass on the pair
 * operator P1^T A P1, so aggregates hold at most four nodes.  agg[i] = the
 * final aggregate of node i; returns their number.
 */
static int aggregate_double(const o_csr *A, double beta, int match, uint32_t hb, int *agg) {
    int n = A->n;
    int *a1 = xcalloc((size_t)n, sizeof(int));
    int n1 = pairwise_pass(A, beta, match, hb, a1);
    o_csr P1 = agg_to_p(n, n1, a1);
    o_csr R1 = transpose(&P1);
    o_csr AP = spgemm(A, &P1);
    o_csr A1 = spgemm(&R1, &AP);
    int *a2 = xcalloc((size_t)n1, sizeof(int));
    int n2 = pairwise_pass(&A1, beta, match, hb ^ 0x9e3779b9u, a2);
    for (int i = 0; i < n; i++) agg[i] = a2[a1[i]];
    free(a1);
    free(a2);
    csr_release(&P1);
    csr_release(&R1);
    csr_release(&AP);
    csr_release(&A1);
    return n2;
}

int o_aggregate(int n, const int *rowptr, const int *col, const double *val, double beta, int passes,
                int match, int *agg) {
    o_csr A = csr_view(n, n, rowptr, col, val);
    uint32_t hb = fmix32(3u * 1000003u);
    return passes == 1 ? pairwise_pass(&A, beta, match, hb, agg) : aggregate_double(&A, beta, match, hb, agg);
}

/* ----------------------------------------------------------------- BILU(0) */

/* Positions of rows in (color, index) order; order[t] = row at position t. */
static void color_order(int n, const int *color, int ncolors, int *order, int *pos) {
    int t = 0;
    for (int c = 0; c < ncolors; c++)
        for (int i = 0; i < n; i++)
            if (color[i] == c) {
                pos[i] = t;
                order[t++] = i;
            }
}

/* Block coloring for BILU(0): JP on the off-diagonal block graph at theta = 0. */
static int bilu_coloring(int nb, const int *rowptr, const int *col, uint64_t seed, int *bcolor) {
    o_csr S = csr_alloc(nb, nb, rowptr[nb], 0);
    int nnz = 0;
    for (int i = 0; i < nb; i++) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (col[p] != i) S.col[nnz++] = col[p];
        S.rowptr[i + 1] = nnz;
    }
    S.nnz = nnz;
    o_csr G = sym_union(&S);
    int nc = jp_color(&G, seed, 2, 0, bcolor);
    csr_release(&S);
    csr_release(&G);
    return nc;
}

static int find_col(const int *col, int lo, int hi, int j) {
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < 0 || col[lo] != j) ? -1 : lo;
}

/*
 * Block ILU(0) in (color, index) order, row by row: for row i and
 * each k before i in that order (ascending), L_ik = A_ik U_kk^-1, then
 * A_ij -= L_ik U_kj for every j after k in row k that is also in row i's
 * pattern.  The factor array holds L_ik and U_ij in A's pattern and U_ii^-1 at
 * the diagonal positions.
 */
static int bilu0_factor(int nb, const int *rowptr, const int *col, const double *val,
                        const int *bcolor, int nbcolors, double *lu) {
    int *order = xcalloc((size_t)nb, sizeof(int));
    int *pos = xcalloc((size_t)nb, sizeof(int));
    int *diag = xcalloc((size_t)nb, sizeof(int));
    color_order(nb, bcolor, nbcolors, order, pos);
    memcpy(lu, val, sizeof(double) * 9 * (size_t)rowptr[nb]);
    int rc = O_OK;
    for (int i = 0; i < nb; i++) {
        diag[i] = find_col(col, rowptr[i], rowptr[i + 1], i);
        if (diag[i] < 0) rc = O_ERR_INVALID;
    }
    int maxlen = 0;
    for (int i = 0; i < nb; i++)
        if (rowptr[i + 1] - rowptr[i] > maxlen) maxlen = rowptr[i + 1] - rowptr[i];
    int *lower = xcalloc((size_t)maxlen + 1, sizeof(int));
    for (int t = 0; t < nb && rc == O_OK; t++) {
        int i = order[t];
        /* entries of row i that come before i, sorted by position */
        int nl = 0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (pos[col[p]] < t) lower[nl++] = p;
        for (int a = 1; a < nl; a++)
            for (int b = a; b > 0 && pos[col[lower[b - 1]]] > pos[col[lower[b]]]; b--) {
                int x = lower[b];
                lower[b] = lower[b - 1];
                lower[b - 1] = x;
            }
        for (int a = 0; a < nl; a++) {
            int p = lower[a];
            int k = col[p];
            double L[9];
            mat3_mul(lu + 9 * (size_t)p, lu + 9 * (size_t)diag[k], L);
            memcpy(lu + 9 * (size_t)p, L, sizeof(L));
            for (int q = rowptr[k]; q < rowptr[k + 1]; q++) {
                int j = col[q];
                if (pos[j] <= pos[k]) continue;
                int r = find_col(col, rowptr[i], rowptr[i + 1], j);
                if (r < 0) continue;
                double LU[9];
                mat3_mul(L, lu + 9 * (size_t)q, LU);
                for (int e = 0; e < 9; e++) lu[9 * (size_t)r + e] -= LU[e];
            }
        }
        double inv[9];
        if (!mat3_inv(lu + 9 * (size_t)diag[i], inv)) {
            rc = O_ERR_SINGULAR;
            break;
        }
        memcpy(lu + 9 * (size_t)diag[i], inv, sizeof(inv));
    }
    free(lower);
    free(order);
    free(pos);
    free(diag);
    return rc;
}

/* Row t (position in (color, index) order) of the forward substitution. */
static void bilu_fwd_row(int t, const int *order, const int *pos, const int *rowptr, const int *col,
                         const double *lu, const double *r, double *y) {
    int i = order[t];
    double s[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int j = col[p];
        if (pos[j] >= t) continue;
        const double *L = lu + 9 * (size_t)p;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s[a] -= L[3 * a + b] * y[3 * j + b];
    }
    y[3 * i] = s[0];
    y[3 * i + 1] = s[1];
    y[3 * i + 2] = s[2];
}

/* Row t of the backward substitution. */
static void bilu_bwd_row(int t, const int *order, const int *pos, const int *rowptr, const int *col,
                         const double *lu, const double *y, double *z) {
    int i = order[t];
    double s[3] = {y[3 * i], y[3 * i + 1], y[3 * i + 2]};
    const double *Dinv = NULL;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int j = col[p];
        if (j == i) {
            Dinv = lu + 9 * (size_t)p;
            continue;
        }
        if (pos[j] < t) continue;
        const double *U = lu + 9 * (size_t)p;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s[a] -= U[3 * a + b] * z[3 * j + b];
    }
    for (int a = 0; a < 3; a++)
        z[3 * i + a] = (Dinv[3 * a] * s[0] + Dinv[3 * a + 1] * s[1]) + Dinv[3 * a + 2] * s[2];
}

/* Solve (L U) z = r: forward then backward substitution in (color, index)
 * order.  With a proper coloring (more than one color) the rows of one color
 * never reference each other, so each color's rows are independent; with one
 * color (the natural order) the rows run strictly in sequence. */
void o_bilu0_solve(int nb, const int *rowptr, const int *col, const double *lu,
                   const int *bcolor, int nbcolors, const double *r, double *z) {
    int *order = xcalloc((size_t)nb, sizeof(int));
    int *pos = xcalloc((size_t)nb, sizeof(int));
    color_order(nb, bcolor, nbcolors, order, pos);
    double *y = xcalloc(3 * (size_t)nb, sizeof(double));
    if (nbcolors > 1) {
        int *off = xcalloc((size_t)nbcolors + 1, sizeof(int));
        for (int i = 0; i < nb; i++) off[bcolor[i] + 1]++;
        for (int c = 0; c < nbcolors; c++) off[c + 1] += off[c];
        for (int c = 0; c < nbcolors; c++) {
            OMP_FOR
            for (int t = off[c]; t < off[c + 1]; t++) bilu_fwd_row(t, order, pos, rowptr, col, lu, r, y);
        }
        for (int c = nbcolors - 1; c >= 0; c--) {
            OMP_FOR
            for (int t = off[c]; t < off[c + 1]; t++) bilu_bwd_row(t, order, pos, rowptr, col, lu, y, z);
        }
        free(off);
    } else {
        for (int t = 0; t < nb; t++) bilu_fwd_row(t, order, pos, rowptr, col, lu, r, y);
        for (int t = nb - 1; t >= 0; t--) bilu_bwd_row(t, order, pos, rowptr, col, lu, y, z);
    }
    free(y);
    free(order);
    free(pos);
}

int o_bilu0(int nb, const int *rowptr, const int *col, const double *val, uint64_t seed,
            int *bcolor, double *lu) {
    int nc = bilu_coloring(nb, rowptr, col, seed, bcolor);
    int rc = bilu0_factor(nb, rowptr, col, val, bcolor, nc, lu);
    return rc == O_OK ? nc : rc;
}

/*
 * Natural-order block ILU(0), the factorization level scheduling runs in
 * parallel (Sec. 6's second stage): with every block row in one color the
 * (color, index) order above is the index order, so the lower part of row i is
 * its blocks j < i, eliminated in ascending j.  Returns 1 (one color) or an
 * error code.
 */
int o_bilu0_natural(int nb, const int *rowptr, const int *col, const double *val, double *lu) {
    int *one = xcalloc((size_t)nb, sizeof(int));
    int rc = bilu0_factor(nb, rowptr, col, val, one, 1, lu);
    free(one);
    return rc == O_OK ? 1 : rc;
}

/*
 * Level sets of the natural-order block triangular solves: level(i) is 0 when
 * block row i has no neighbour j < i in the symmetrised block pattern, else
 * 1 + the largest level among those neighbours.  Rows of one level are never
 * adjacent, and every neighbour j < i of i lies in a lower level.  Returns the
 * number of levels.
 */
int o_natural_levels(int nb, const int *rowptr, const int *col, int *level) {
    o_csr A = csr_view(nb, nb, rowptr, col, NULL);
    o_csr G = sym_union(&A);
    int nlev = 0;
    for (int i = 0; i < nb; i++) {
        int lv = 0;
        for (int p = G.rowptr[i]; p < G.rowptr[i + 1]; p++) {
            int j = G.col[p];
            if (j < i && level[j] + 1 > lv) lv = level[j] + 1;
        }
        level[i] = lv;
        if (lv + 1 > nlev) nlev = lv + 1;
    }
    csr_release(&G);
    return nlev;
}

/* ------------------------------------------------------------- hierarchy */

void o_default_opts(o_opts *o) {
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
    o->bilu_order = 0;
    o->reuse_refresh = 0;
    o->resetup = 0;
    o->amg = 0;
    o->amli_iters = 2;
    o->coloring = 0;
    o->agg_match = 0;
    o->coloring_rows = 4096;
}

static void free_setup(o_handle *h) {
    for (int l = 0; l < h->nlev; l++) {
        level_t *L = &h->lev[l];
        csr_release(&L->A);
        csr_release(&L->P);
        csr_release(&L->R);
        csr_release(&L->S);
        free(L->color);
        free(L->cf);
        free(L->x);
        free(L->b);
        free(L->r);
        free(L->tmp);
        free(L->gv);
        free(L->gw);
        free(L->gres);
        memset(L, 0, sizeof(*L));
    }
    h->nlev = 0;
    free(h->clu);
    free(h->cpiv);
    free(h->bcolor);
    free(h->lu);
    free(h->w);
    free(h->pval);
    h->clu = NULL;
    h->cpiv = NULL;
    h->bcolor = NULL;
    h->lu = NULL;
    h->w = NULL;
    h->pval = NULL;
}

/* Zero diagonals make the smoother undefined (no silent regularisation). */
static int check_diag(const o_csr *A) {
    for (int i = 0; i < A->n; i++) {
        double d = 0.0;
        for (int p = A->rowptr[i]; p < A->rowptr[i + 1]; p++)
            if (A->col[p] == i) d = A->val[p];
        if (d == 0.0 || !isfinite(d)) return O_ERR_SINGULAR;
    }
    return O_OK;
}

/* Build B from the current A (Alg. 1's preconditioner, Sec. 3.1, Alg. 6). */
/*
 * Build B from the handle's A.  numeric = 0: the full setup.  numeric = 1 (the
 * numeric-only resetup of resetup = 1): the discrete structure of the last
 * setup is kept -- the number of levels, each level's classical strength set,
 * C/F split and smoother coloring, and the BILU(0) block coloring -- and
 * every value is recomputed from A: decoupling weights and A_P, direct
 * interpolation over the kept strength sets and C/F splits, R = P^T, the
 * Galerkin products, the coarsest LU and the BILU(0) factors.  With the same
 * pattern the products have the same patterns, so the structure fits.
 */
static int build_preconditioner(o_handle *h, int numeric) {
    int knlev = h->nlev, knbc = h->nbcolors;
    o_csr kS[MAXLEV];
    int *kcf[MAXLEV], knc[MAXLEV], *kcolor[MAXLEV], kncol[MAXLEV];
    int *kbcolor = NULL;
    if (numeric) {
        for (int l = 0; l < knlev; l++) {
            level_t *L = &h->lev[l];
            kS[l] = L->S;
            kcf[l] = L->cf;
            knc[l] = L->nc;
            kcolor[l] = L->color;
            kncol[l] = L->ncolors;
            memset(&L->S, 0, sizeof(L->S));
            L->cf = NULL;
            L->color = NULL;
        }
        kbcolor = h->bcolor;
        h->bcolor = NULL;
    }
    free_setup(h);
    const o_opts *o = &h->opt;
    int nb = h->nb, nnzb = h->nnzb;
    h->pval = xcalloc(9 * (size_t)nnzb, sizeof(double));
    memcpy(h->pval, h->val, sizeof(double) * 9 * (size_t)nnzb);
    h->w = xcalloc(3 * (size_t)nb, sizeof(double));
    /* level 0: the pressure matrix A_P */
    o_csr A0 = csr_alloc(nb, nb, nnzb, 1);
    memcpy(A0.rowptr, h->rowptr, sizeof(int) * ((size_t)nb + 1));
    memcpy(A0.col, h->col, sizeof(int) * (size_t)nnzb);
    int rc = o_decouple(nb, h->rowptr, h->col, h->val, o->decouple, h->w, A0.val);
    if (rc != O_OK) {
        csr_release(&A0);
        return rc;
    }
    h->lev[0].A = A0;
    int l = 0;
    for (;;) {
        level_t *L = &h->lev[l];
        h->nlev = l + 1;
        int n = L->A.n;
        rc = check_diag(&L->A);
        if (rc != O_OK) return rc;
        L->x = xcalloc((size_t)n, sizeof(double));
        L->b = xcalloc((size_t)n, sizeof(double));
        L->r = xcalloc((size_t)n, sizeof(double));
        L->tmp = xcalloc((size_t)n, sizeof(double));
        int nc;
        if (numeric) {
            if (l == knlev - 1) break;   /* the kept coarsest level */
            L->S = kS[l];
            L->cf = kcf[l];
            nc = knc[l];
            kS[l].rowptr = NULL;
            kcf[l] = NULL;
        } else {
            if (n <= o->coarse_max || l + 1 >= o->max_levels || l + 1 >= MAXLEV) break;
            L->cf = xcalloc((size_t)n, sizeof(int));
            if (o->amg == 1) {
                /* UA-AMG: cf holds each node's aggregate */
                uint32_t s32 = (uint32_t)(o->seed ^ (o->seed >> 32));
                nc = aggregate_double(&L->A, o->theta_amg, o->agg_match,
                                      fmix32(s32 + 3u * 1000003u + (uint32_t)l), L->cf);
            } else {
                L->S = strength_rs(&L->A, o->theta_amg);
                nc = pmis(&L->S, o->seed, 1, l, L->cf);
            }
            if (nc == 0 || (double)nc > 0.95 * (double)n) {
                csr_release(&L->S);
                free(L->cf);
                L->cf = NULL;
                break;
            }
        }
        L->nc = nc;
        if (o->amg == 1) L->P = agg_to_p(n, nc, L->cf);
        else L->P = interp_direct(&L->A, &L->S, L->cf);
        L->R = transpose(&L->P);
        o_csr AP = spgemm(&L->A, &L->P);
        h->lev[l + 1].A = spgemm(&L->R, &AP);
        csr_release(&AP);
        if (numeric) {
            L->color = kcolor[l];
            L->ncolors = kncol[l];
            kcolor[l] = NULL;
        } else {
            /* the smoother's coloring (Eq. 5.1): JP standing in for Alg. 4-5, or Alg. 4-5 */
            o_csr Sc = strength_color(&L->A, o->theta_color);
            L->color = xcalloc((size_t)n, sizeof(int));
            if (o->coloring == 1 && (o->coloring_rows <= 0 || n <= o->coloring_rows)) {
                L->ncolors = vertices_grouping(&Sc, L->color);
            } else {
                o_csr G = sym_union(&Sc);
                L->ncolors = jp_color(&G, o->seed, 0, l, L->color);
                csr_release(&G);
            }
            csr_release(&Sc);
        }
        l++;
    }
    if (numeric)
        for (int k = 0; k < knlev; k++) {   /* the kept structure not taken over (the coarsest level's) */
            if (kS[k].rowptr) csr_release(&kS[k]);
            free(kcf[k]);
            free(kcolor[k]);
        }
    /* amg = 1: the coarse corrections onto levels 1 .. nlev-2 run GCR there */
    if (o->amg == 1)
        for (int k = 1; k < h->nlev - 1; k++) {
            size_t nk = (size_t)h->lev[k].A.n, m = (size_t)(o->amli_iters > 0 ? o->amli_iters : 1);
            h->lev[k].gv = xcalloc(m * nk, sizeof(double));
            h->lev[k].gw = xcalloc(m * nk, sizeof(double));
            h->lev[k].gres = xcalloc(nk, sizeof(double));
        }
    /* coarsest level: dense LU */
    level_t *C = &h->lev[h->nlev - 1];
    int n = C->A.n;
    h->clu = xcalloc((size_t)n * n, sizeof(double));
    h->cpiv = xcalloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; i++)
        for (int p = C->A.rowptr[i]; p < C->A.rowptr[i + 1]; p++)
            h->clu[(size_t)i * n + C->A.col[p]] = C->A.val[p];
    rc = dense_lu(n, h->clu, h->cpiv);
    if (rc != O_OK) return rc;
    /* second stage */
    if (numeric) {
        h->bcolor = kbcolor;
        h->nbcolors = knbc;
    } else {
        h->bcolor = xcalloc((size_t)nb, sizeof(int));
        /* natural order: one color, so the (color, index) order is the index order */
        h->nbcolors = o->bilu_order ? 1 : bilu_coloring(nb, h->rowptr, h->col, o->seed, h->bcolor);
    }
    h->lu = xcalloc(9 * (size_t)nnzb, sizeof(double));
    rc = bilu0_factor(nb, h->rowptr, h->col, h->pval, h->bcolor, h->nbcolors, h->lu);
    return rc;
}

/* V(pre, post) cycle for A_l e = b from zero: pre-smoothing colors ascending,
 * post-smoothing descending. */
static void vcycle(o_handle *h, int l, const double *b, double *x) {
    level_t *L = &h->lev[l];
    int n = L->A.n;
    if (l == h->nlev - 1) {
        dense_lu_solve(n, h->clu, h->cpiv, b, x);
        return;
    }
    OMP_FOR
    for (int i = 0; i < n; i++) x[i] = 0.0;
    for (int s = 0; s < h->opt.pre; s++) mcgs_sweep(&L->A, L->color, L->ncolors, b, x, 0, L->tmp);
    /* r = b - A x, b_c = R r */
    OMP_FOR
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int p = L->A.rowptr[i]; p < L->A.rowptr[i + 1]; p++)
            s -= L->A.val[p] * x[L->A.col[p]];
        L->r[i] = s;
    }
    level_t *Lc = &h->lev[l + 1];
    OMP_FOR
    for (int I = 0; I < L->R.n; I++) {
        double s = 0.0;
        for (int p = L->R.rowptr[I]; p < L->R.rowptr[I + 1]; p++)
            s += L->R.val[p] * L->r[L->R.col[p]];
        Lc->b[I] = s;
    }
    vcycle(h, l + 1, Lc->b, Lc->x);
    /* x += P x_c */
    OMP_FOR
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = L->P.rowptr[i]; p < L->P.rowptr[i + 1]; p++)
            s += L->P.val[p] * Lc->x[L->P.col[p]];
        x[i] += s;
    }
    for (int s = 0; s < h->opt.post; s++)
        mcgs_sweep(&L->A, L->color, L->ncolors, b, x, 1, L->tmp);
}

static void kcycle(o_handle *h, int l, const double *b, double *x);

/*
 * The coarse correction of the nonlinear AMLI-cycle (Sec. 6): amli_iters
 * steps of flexible GCR on A_k e = r from e = 0, each step preconditioned by
 * the cycle of level k.  Step t takes v_t = cycle(res), w_t = A_k v_t,
 * makes w_t orthogonal to the earlier w_s (v_t follows), then
 * alpha_t = (w_t, res) / (w_t, w_t), e += alpha_t v_t, res -= alpha_t w_t.
 */
static void amli_coarse(o_handle *h, int k, const double *r, double *e) {
    level_t *L = &h->lev[k];
    int n = L->A.n, m = h->opt.amli_iters > 0 ? h->opt.amli_iters : 1;
    double *res = L->gres;
    for (int i = 0; i < n; i++) {
        e[i] = 0.0;
        res[i] = r[i];
    }
    for (int t = 0; t < m; t++) {
        double *v = L->gv + (size_t)t * n, *w = L->gw + (size_t)t * n;
        kcycle(h, k, res, v);
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int p = L->A.rowptr[i]; p < L->A.rowptr[i + 1]; p++) s += L->A.val[p] * v[L->A.col[p]];
            w[i] = s;
        }
        for (int u = 0; u < t; u++) {
            const double *vu = L->gv + (size_t)u * n, *wu = L->gw + (size_t)u * n;
            double den = dot(n, wu, wu);
            if (den == 0.0) continue;
            double beta = dot(n, w, wu) / den;
            for (int i = 0; i < n; i++) {
                w[i] -= beta * wu[i];
                v[i] -= beta * vu[i];
            }
        }
        double ww = dot(n, w, w);
        if (ww == 0.0) break;
        double alpha = dot(n, w, res) / ww;
        for (int i = 0; i < n; i++) {
            e[i] += alpha * v[i];
            res[i] -= alpha * w[i];
        }
    }
}

/*
 * The nonlinear AMLI-cycle for A_l e = b from zero (amg = 1): the V-cycle's
 * smoothing and transfers, with the coarse problem solved exactly on the
 * coarsest level and by amli_coarse elsewhere.
 */
static void kcycle(o_handle *h, int l, const double *b, double *x) {
    level_t *L = &h->lev[l];
    int n = L->A.n;
    if (l == h->nlev - 1) {
        dense_lu_solve(n, h->clu, h->cpiv, b, x);
        return;
    }
    OMP_FOR
    for (int i = 0; i < n; i++) x[i] = 0.0;
    for (int s = 0; s < h->opt.pre; s++) mcgs_sweep(&L->A, L->color, L->ncolors, b, x, 0, L->tmp);
    OMP_FOR
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int p = L->A.rowptr[i]; p < L->A.rowptr[i + 1]; p++)
            s -= L->A.val[p] * x[L->A.col[p]];
        L->r[i] = s;
    }
    level_t *Lc = &h->lev[l + 1];
    OMP_FOR
    for (int I = 0; I < L->R.n; I++) {
        double s = 0.0;
        for (int p = L->R.rowptr[I]; p < L->R.rowptr[I + 1]; p++)
            s += L->R.val[p] * L->r[L->R.col[p]];
        Lc->b[I] = s;
    }
    if (l + 1 == h->nlev - 1) dense_lu_solve(Lc->A.n, h->clu, h->cpiv, Lc->b, Lc->x);
    else amli_coarse(h, l + 1, Lc->b, Lc->x);
    OMP_FOR
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = L->P.rowptr[i]; p < L->P.rowptr[i + 1]; p++)
            s += L->P.val[p] * Lc->x[L->P.col[p]];
        x[i] += s;
    }
    for (int s = 0; s < h->opt.post; s++)
        mcgs_sweep(&L->A, L->color, L->ncolors, b, x, 1, L->tmp);
}

/* B_P: the V-cycle (amg = 0) or the nonlinear AMLI-cycle (amg = 1). */
static void pressure_cycle(o_handle *h, const double *b, double *x) {
    if (h->opt.amg == 1) kcycle(h, 0, b, x);
    else vcycle(h, 0, b, x);
}

/*
 * One CPR application z = B v (Alg. 1 from x = 0, Eq. 3.1):
 *   r_P = Pi_P^T v (decoupled restriction), e_P = B_P r_P (AMG V-cycle),
 *   z = Pi_P e_P, r = v - A z, z += R r (BILU(0)).
 */
static void cpr_apply(o_handle *h, const double *v, double *z) {
    int nb = h->nb;
    OMP_FOR
    for (int i = 0; i < nb; i++)
        h->rp[i] = (h->w[3 * i] * v[3 * i] + h->w[3 * i + 1] * v[3 * i + 1]) +
                   h->w[3 * i + 2] * v[3 * i + 2];
    pressure_cycle(h, h->rp, h->ep);
    OMP_FOR
    for (int i = 0; i < nb; i++) {
        z[3 * i] = h->ep[i];
        z[3 * i + 1] = 0.0;
        z[3 * i + 2] = 0.0;
    }
    bsr3_resid(nb, h->rowptr, h->col, h->pval, v, z, h->work1);
    o_bilu0_solve(nb, h->rowptr, h->col, h->lu, h->bcolor, h->nbcolors, h->work1, h->work2);
    OMP_FOR
    for (int i = 0; i < 3 * nb; i++) z[i] += h->work2[i];
}

void o_cpr_apply(o_handle *h, const double *v, double *z) { cpr_apply(h, v, z); }
void o_vcycle(o_handle *h, const double *b, double *x) { pressure_cycle(h, b, x); }
void o_bilu_apply(o_handle *h, const double *r, double *z) {
    o_bilu0_solve(h->nb, h->rowptr, h->col, h->lu, h->bcolor, h->nbcolors, r, z);
}

/* ----------------------------------------------------------------- FGMRES */

typedef void (*precond_fn)(void *ctx, const double *v, double *z);

typedef struct {
    int nb;
    const int *rowptr, *col;
    const double *val;
} op_ctx;

static void identity_pc(void *ctx, const double *v, double *z) {
    int n = 3 * ((op_ctx *)ctx)->nb;
    memcpy(z, v, sizeof(double) * (size_t)n);
}

static void cpr_pc(void *ctx, const double *v, double *z) { cpr_apply((o_handle *)ctx, v, z); }

/*
 * Right-preconditioned flexible GMRES(m) following Alg. 2: Arnoldi with
 * classical Gram-Schmidt (all h_ij from the same vector), Givens rotations on
 * the Hessenberg matrix, stop when the estimated residual |g_{j+1}| falls
 * below rtol*||r_0|| (r_0 of the initial guess) or when h_{j+1,j} = 0; after
 * each cycle x += Z y and the true residual decides whether to restart.
 * Z keeps the preconditioned vectors (flexible variant).  `hist`, when not
 * NULL, receives the estimated relative residual after every inner step.
 */
static int fgmres(int nb, const int *rowptr, const int *col, const double *val, precond_fn pc,
                  void *pctx, const double *b, double *x, double rtol, int m, int max_restarts,
                  o_stats *st, double *hist) {
    int n = 3 * nb;
    double *V = xcalloc((size_t)(m + 1) * n, sizeof(double));
    double *Z = xcalloc((size_t)m * n, sizeof(double));
    double *H = xcalloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = xcalloc((size_t)m, sizeof(double));
    double *sn = xcalloc((size_t)m, sizeof(double));
    double *g = xcalloc((size_t)m + 1, sizeof(double));
    double *y = xcalloc((size_t)m, sizeof(double));
    double *r = xcalloc((size_t)n, sizeof(double));
    double *w = xcalloc((size_t)n, sizeof(double));
    int rc = O_NOT_CONVERGED, iters = 0, cycles = 0;
    bsr3_resid(nb, rowptr, col, val, b, x, r);
    double norm0 = sqrt(dot(n, r, r));
    double rnorm = norm0;
    if (!isfinite(norm0)) {
        rc = O_ERR_BREAKDOWN;
        goto done;
    }
    if (norm0 == 0.0) {
        rc = O_OK;
        goto done;
    }
    for (cycles = 0; cycles < max_restarts; cycles++) {
        double beta = rnorm;
        OMP_FOR
        for (int i = 0; i < n; i++) V[i] = r[i] / beta;
        for (int i = 0; i <= m; i++) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            pc(pctx, vj, zj);
            o_bsr3_spmv(nb, rowptr, col, val, zj, w);
            for (int i = 0; i <= j; i++) H[i * m + j] = dot(n, w, V + (size_t)i * n);
            /* w -= sum_i h_ij v_i, each entry taking i in ascending order */
            OMP_FOR
            for (int q = 0; q < n; q++)
                for (int i = 0; i <= j; i++) w[q] -= H[i * m + j] * V[(size_t)i * n + q];
            double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            iters++;
            k = j + 1;
            if (!isfinite(hn)) {
                rc = O_ERR_BREAKDOWN;
                goto done;
            }
            /* apply the previous rotations to column j, then a new one */
            for (int i = 0; i < j; i++) {
                double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[j * m + j], c = H[(j + 1) * m + j];
            double den = sqrt(a * a + c * c);
            cs[j] = den == 0.0 ? 1.0 : a / den;
            sn[j] = den == 0.0 ? 0.0 : c / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (hist) hist[iters - 1] = fabs(g[j + 1]) / norm0;
            if (hn == 0.0) break;
            OMP_FOR
            for (int q = 0; q < n; q++) V[(size_t)(j + 1) * n + q] = w[q] / hn;
            if (fabs(g[j + 1]) / norm0 < rtol) break;
        }
        /* y = H_k^-1 g (upper triangular), x += Z y */
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int q = i + 1; q < k; q++) s -= H[i * m + q] * y[q];
            y[i] = s / H[i * m + i];
        }
        OMP_FOR
        for (int q = 0; q < n; q++)
            for (int i = 0; i < k; i++) x[q] += y[i] * Z[(size_t)i * n + q];
        bsr3_resid(nb, rowptr, col, val, b, x, r);
        rnorm = sqrt(dot(n, r, r));
        if (!isfinite(rnorm)) {
            rc = O_ERR_BREAKDOWN;
            break;
        }
        if (rnorm / norm0 < rtol) {
            rc = O_OK;
            cycles++;
            break;
        }
    }
done:
    if (st) {
        st->iters = iters;
        st->restarts = cycles;
        st->converged = rc == O_OK;
        st->rel_res = norm0 > 0.0 ? rnorm / norm0 : 0.0;
    }
    free(V);
    free(Z);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(r);
    free(w);
    return rc;
}

int o_fgmres_identity(int nb, const int *rowptr, const int *col, const double *val,
                      const double *b, double *x, double rtol, int m, int max_restarts,
                      o_stats *st, double *hist) {
    op_ctx ctx = {nb, rowptr, col, val};
    return fgmres(nb, rowptr, col, val, identity_pc, &ctx, b, x, rtol, m, max_restarts, st, hist);
}

/*
 * FGMRES (Alg. 2) on one system of a block-diagonal concatenation: block rows
 * [r0, r1) of the handle's A, which must couple to no block row outside the
 * range, preconditioned by the handle's B restricted to those rows.  B is
 * applied to the vector that equals v on the range and zero elsewhere; with
 * a block-diagonal A every level, interpolation and factor of B is block
 * diagonal too, so the other systems' rows stay exactly zero and the range
 * gets what a batch of such systems gives that system.  b and x hold
 * 3 (r1 - r0) values.  Restart length and restarts are the handle's.
 */
typedef struct {
    o_handle *h;
    int r0, r1;
    double *vfull, *zfull;
} rows_ctx;

static void rows_pc(void *ctx, const double *v, double *z) {
    rows_ctx *c = (rows_ctx *)ctx;
    int n = 3 * c->h->nb, m = 3 * (c->r1 - c->r0);
    for (int i = 0; i < n; i++) c->vfull[i] = 0.0;
    memcpy(c->vfull + 3 * (size_t)c->r0, v, sizeof(double) * (size_t)m);
    cpr_apply(c->h, c->vfull, c->zfull);
    memcpy(z, c->zfull + 3 * (size_t)c->r0, sizeof(double) * (size_t)m);
}

int o_solve_rows(o_handle *h, int r0, int r1, const double *b, double *x, double rtol, o_stats *st) {
    if (r0 < 0 || r1 > h->nb || r0 >= r1) return O_ERR_INVALID;
    int ns = r1 - r0, base = h->rowptr[r0];
    int *rp = xcalloc((size_t)ns + 1, sizeof(int));
    int *cl = xcalloc((size_t)(h->rowptr[r1] - base) + 1, sizeof(int));
    for (int i = 0; i <= ns; i++) rp[i] = h->rowptr[r0 + i] - base;
    for (int p = base; p < h->rowptr[r1]; p++) {
        if (h->col[p] < r0 || h->col[p] >= r1) {
            free(rp);
            free(cl);
            return O_ERR_INVALID;
        }
        cl[p - base] = h->col[p] - r0;
    }
    rows_ctx ctx = {h, r0, r1, xcalloc(3 * (size_t)h->nb, sizeof(double)),
                    xcalloc(3 * (size_t)h->nb, sizeof(double))};
    int rc = fgmres(ns, rp, cl, h->val + 9 * (size_t)base, rows_pc, &ctx, b, x, rtol, h->opt.restart,
                    h->opt.max_restarts, st, NULL);
    if (st) {
        st->setup_called = h->setup_called;
        st->setup_count = h->setup_count;
        st->levels = h->nlev;
    }
    free(rp);
    free(cl);
    free(ctx.vfull);
    free(ctx.zfull);
    return rc;
}

/* ------------------------------------------------------------------- API */

static int check_bsr(int nb, const int *rowptr, const int *col) {
    if (nb <= 0 || rowptr[0] != 0) return O_ERR_INVALID;
    for (int i = 0; i < nb; i++) {
        if (rowptr[i + 1] < rowptr[i]) return O_ERR_INVALID;
        int has_diag = 0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            if (col[p] < 0 || col[p] >= nb) return O_ERR_INVALID;
            if (p > rowptr[i] && col[p] <= col[p - 1]) return O_ERR_INVALID;
            has_diag |= col[p] == i;
        }
        if (!has_diag) return O_ERR_INVALID;
    }
    return O_OK;
}

static void alloc_work(o_handle *h) {
    size_t n = 3 * (size_t)h->nb;
    h->work1 = xcalloc(n, sizeof(double));
    h->work2 = xcalloc(n, sizeof(double));
    h->work3 = xcalloc(n, sizeof(double));
    h->rp = xcalloc((size_t)h->nb, sizeof(double));
    h->ep = xcalloc((size_t)h->nb, sizeof(double));
}

static void free_matrix(o_handle *h) {
    free(h->rowptr);
    free(h->col);
    free(h->val);
    free(h->work1);
    free(h->work2);
    free(h->work3);
    free(h->rp);
    free(h->ep);
    h->rowptr = h->col = NULL;
    h->val = h->work1 = h->work2 = h->work3 = h->rp = h->ep = NULL;
}

static int load_matrix(o_handle *h, int nb, const int *rowptr, const int *col,
                       const double *val) {
    int rc = check_bsr(nb, rowptr, col);
    if (rc != O_OK) return rc;
    free_matrix(h);
    h->nb = nb;
    h->nnzb = rowptr[nb];
    h->rowptr = xcalloc((size_t)nb + 1, sizeof(int));
    h->col = xcalloc((size_t)h->nnzb, sizeof(int));
    h->val = xcalloc(9 * (size_t)h->nnzb, sizeof(double));
    memcpy(h->rowptr, rowptr, sizeof(int) * ((size_t)nb + 1));
    memcpy(h->col, col, sizeof(int) * (size_t)h->nnzb);
    memcpy(h->val, val, sizeof(double) * 9 * (size_t)h->nnzb);
    alloc_work(h);
    return O_OK;
}

int o_setup(o_handle **out, int nb, const int *rowptr, const int *col, const double *val,
            const o_opts *opt) {
    o_handle *h = xcalloc(1, sizeof(o_handle));
    if (opt) h->opt = *opt;
    else o_default_opts(&h->opt);
    int rc = load_matrix(h, nb, rowptr, col, val);
    if (rc == O_OK) rc = build_preconditioner(h, 0);
    if (rc != O_OK) {
        o_destroy(h);
        *out = NULL;
        return rc;
    }
    h->setup_count = 1;
    h->setup_called = 1;
    h->updates = 1;
    h->last_iters = -1;
    *out = h;
    return O_OK;
}

/*
 * A new Jacobian A^(k) (Alg. 3): the previous B is reused iff k > 1, a solve
 * has run since the last setup, It^(k-1) <= mu and the size and pattern are
 * unchanged (Remark 4.2); otherwise B is rebuilt from A^(k).
 */
int o_update(o_handle *h, int nb, const int *rowptr, const int *col, const double *val) {
    int same = nb == h->nb && rowptr[nb] == h->nnzb &&
               memcmp(rowptr, h->rowptr, sizeof(int) * ((size_t)nb + 1)) == 0 &&
               memcmp(col, h->col, sizeof(int) * (size_t)h->nnzb) == 0;
    int rc;
    if (same) {
        memcpy(h->val, val, sizeof(double) * 9 * (size_t)h->nnzb);
    } else {
        rc = load_matrix(h, nb, rowptr, col, val);
        if (rc != O_OK) return rc;
    }
    h->updates++;
    int reuse = same && h->updates > 1 && h->last_iters >= 0 && h->last_iters <= h->opt.mu;
    h->setup_called = !reuse;
    if (reuse) {
        /* reuse_refresh: the second residual's copy of A becomes A^(k) */
        if (h->opt.reuse_refresh) memcpy(h->pval, h->val, sizeof(double) * 9 * (size_t)h->nnzb);
        return O_OK;
    }
    /* resetup = 1: with the pattern unchanged, only the values are rebuilt */
    rc = build_preconditioner(h, h->opt.resetup && same && h->nlev > 0);
    if (rc != O_OK) return rc;
    h->setup_count++;
    h->last_iters = -1;
    return O_OK;
}

int o_solve(o_handle *h, const double *b, double *x, double rtol, o_stats *st) {
    o_stats s;
    memset(&s, 0, sizeof(s));
    int rc = fgmres(h->nb, h->rowptr, h->col, h->val, cpr_pc, h, b, x, rtol, h->opt.restart,
                    h->opt.max_restarts, &s, NULL);
    h->last_iters = s.iters;
    s.setup_called = h->setup_called;
    s.setup_count = h->setup_count;
    s.levels = h->nlev;
    if (st) *st = s;
    return rc;
}

void o_destroy(o_handle *h) {
    if (!h) return;
    free_setup(h);
    free_matrix(h);
    free(h);
}

/* ------------------------------------------------------------ inspection */

int o_num_levels(const o_handle *h) { return h->nlev; }
int o_last_iters(const o_handle *h) { return (int)h->last_iters; }

void o_level_info(const o_handle *h, int l, int *n, int *nnz, int *ncolors, int *nc, int *nnzP) {
    const level_t *L = &h->lev[l];
    *n = L->A.n;
    *nnz = L->A.nnz;
    *ncolors = L->ncolors;
    *nc = L->cf ? L->nc : 0;
    *nnzP = L->cf ? L->P.nnz : 0;
}

void o_level_get(const o_handle *h, int l, int *rowptr, int *col, double *val, int *color,
                 int *cf, int *prow, int *pcol, double *pval) {
    const level_t *L = &h->lev[l];
    o_csr_copy(&L->A, rowptr, col, val);
    if (L->color && color) memcpy(color, L->color, sizeof(int) * (size_t)L->A.n);
    if (L->cf && cf) memcpy(cf, L->cf, sizeof(int) * (size_t)L->A.n);
    if (L->cf && prow) o_csr_copy(&L->P, prow, pcol, pval);
}

void o_get_weights(const o_handle *h, double *w) {
    memcpy(w, h->w, sizeof(double) * 3 * (size_t)h->nb);
}

int o_bilu_ncolors(const o_handle *h) { return h->nbcolors; }

void o_bilu_get(const o_handle *h, int *bcolor, double *lu) {
    memcpy(bcolor, h->bcolor, sizeof(int) * (size_t)h->nb);
    memcpy(lu, h->lu, sizeof(double) * 9 * (size_t)h->nnzb);
}
