// Device setup of the CPR preconditioner B (the setup behind Alg. 1, Sec. 3.1):
// pressure decoupling, the AMG hierarchy (classical strength, PMIS C/F split,
// direct interpolation, R = P^T, Galerkin R A P) with the Eq. 5.1 coloring of
// every smoothed level (Jones-Plassmann with hashed keys), the dense coarsest
// solve, and the multicolor block ILU(0) second stage.
//
// Every floating-point operation whose result decides a discrete outcome
// (strength, interpolation weights, coarse matrices) is written with explicit
// round-to-nearest intrinsics in a fixed order (the ascending-column order of
// the plain definitions), so colors, C/F splits and sparsity patterns are
// reproducible bit for bit.  Discrete rounds (JP, PMIS) are round-synchronous:
// every decision of a round reads the state at the start of the round.
#include <algorithm>
#include <climits>
#include <cmath>

#include "cpr_internal.cuh"

namespace cpr {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ bool key_greater(int a1, uint32_t h1, int i1, int a2, uint32_t h2,
                                            int i2) {
    if (a1 != a2) return a1 > a2;
    if (h1 != h2) return h1 > h2;
    return i1 > i2;
}

// Lower bound of j in col[lo, hi); the caller checks col[result] == j.
__device__ __forceinline__ int find_col(const int *col, int lo, int hi, int j) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// ------------------------------------------------------------- validation

__global__ void k_validate_bsr(const int *rowptr, const int *col, int nb, int nnzb, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int a = rowptr[i], b = rowptr[i + 1];
    if ((i == 0 && a != 0) || (i == nb - 1 && b != nnzb) || b < a || a < 0 || b > nnzb) {
        set_err(err, CPR_ERR_INVALID);
        return;
    }
    int prev = -1;
    bool diag = false;
    for (int p = a; p < b; p++) {
        int c = col[p];
        if (c < 0 || c >= nb || c <= prev) {
            set_err(err, CPR_ERR_INVALID);
            return;
        }
        prev = c;
        diag |= c == i;
    }
    if (!diag) set_err(err, CPR_ERR_INVALID);
}

__global__ void k_diagpos(int n, const int *rowptr, const int *col, int *diag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = rowptr[i + 1];
    int p = find_col(col, rowptr[i], e, i);
    diag[i] = (p < e && col[p] == i) ? p : -1;
}

// ------------------------------------------------------------- decoupling

// w_i = D_i^-T e_1 = (C00, C10, C20) / det(D_i) by the adjugate, or e_1 (mode 0).
__global__ void k_decouple(int nb, const int *diag, const double *val, int mode, double *w,
                           int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    if (mode == 0) {
        w[3 * i] = 1.0;
        w[3 * i + 1] = 0.0;
        w[3 * i + 2] = 0.0;
        return;
    }
    const double *d = val + 9 * (size_t)diag[i];
    double c00 = __dsub_rn(__dmul_rn(d[4], d[8]), __dmul_rn(d[5], d[7]));
    double c10 = __dsub_rn(__dmul_rn(d[2], d[7]), __dmul_rn(d[1], d[8]));
    double c20 = __dsub_rn(__dmul_rn(d[1], d[5]), __dmul_rn(d[2], d[4]));
    double det = __dadd_rn(__dadd_rn(__dmul_rn(d[0], c00), __dmul_rn(d[3], c10)), __dmul_rn(d[6], c20));
    if (det == 0.0 || !isfinite(det)) {
        set_err(err, CPR_ERR_SINGULAR);
        det = 1.0;
    }
    w[3 * i] = __ddiv_rn(c00, det);
    w[3 * i + 1] = __ddiv_rn(c10, det);
    w[3 * i + 2] = __ddiv_rn(c20, det);
}

// A_P[i][j] = w_i . A_ij e_1 on the block pattern; also the column-0 slices of A.
__global__ void k_pressure_matrix(int nb, const int *rowptr, const double *val, const double *w,
                                  double *apval, double *pcol0) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    double w0 = w[3 * i], w1 = w[3 * i + 1], w2 = w[3 * i + 2];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        const double *a = val + 9 * (size_t)p;
        apval[p] = __dadd_rn(__dadd_rn(__dmul_rn(w0, a[0]), __dmul_rn(w1, a[3])), __dmul_rn(w2, a[6]));
        pcol0[3 * (size_t)p] = a[0];
        pcol0[3 * (size_t)p + 1] = a[3];
        pcol0[3 * (size_t)p + 2] = a[6];
    }
}

// -------------------------------------------------------- strength (Eq. 5.1)

// j in S_i iff j != i and |a_ij| > theta * sum_k |a_ik| (sum over the whole row).
// srowptr == nullptr: count pass (out = counts); otherwise fill pass (out = columns).
__global__ void k_strength51(int n, const int *rowptr, const int *col, const double *val,
                             double theta, const int *srowptr, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rowptr[i], b = rowptr[i + 1];
    double rowsum = 0.0;
    for (int p = a; p < b; p++) rowsum = __dadd_rn(rowsum, fabs(val[p]));
    double t = __dmul_rn(theta, rowsum);
    int q = srowptr ? srowptr[i] : 0, c = 0;
    for (int p = a; p < b; p++) {
        int j = col[p];
        if (j != i && fabs(val[p]) > t) {
            if (srowptr) out[q + c] = j;
            c++;
        }
    }
    if (!srowptr) out[i] = c;
}

// Classical strength: with s = sign(a_ii), j in S_i iff -s a_ij >= theta max_{k!=i}(-s a_ik) > 0.
__global__ void k_strength_rs(int n, const int *rowptr, const int *col, const double *val,
                              double theta, const int *srowptr, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rowptr[i], b = rowptr[i + 1];
    double aii = 0.0;
    for (int p = a; p < b; p++)
        if (col[p] == i) aii = val[p];
    double s = aii < 0.0 ? -1.0 : 1.0;
    double m = 0.0;
    bool have = false;
    for (int p = a; p < b; p++) {
        if (col[p] == i) continue;
        double v = -s * val[p];
        if (!have || v > m) m = v;
        have = true;
    }
    int q = srowptr ? srowptr[i] : 0, c = 0;
    if (have && m > 0.0) {
        double t = __dmul_rn(theta, m);
        for (int p = a; p < b; p++) {
            int j = col[p];
            if (j != i && -s * val[p] >= t) {
                if (srowptr) out[q + c] = j;
                c++;
            }
        }
    }
    if (!srowptr) out[i] = c;
}

// Off-diagonal block pattern (the BILU graph at theta = 0).
__global__ void k_offdiag_pattern(int n, const int *rowptr, const int *col, const int *srowptr,
                                  int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = srowptr ? srowptr[i] : 0, c = 0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
        if (col[p] != i) {
            if (srowptr) out[q + c] = col[p];
            c++;
        }
    if (!srowptr) out[i] = c;
}

// --------------------------------------------------------------- transpose

__global__ void k_count_cols(long nnz, const int *col, int *cnt) {
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < nnz; p += (long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[p]], 1);
}

__global__ void k_scatter_t(int n, const int *rowptr, const int *col, const double *val,
                            int *cursor, int *tcol, double *tval) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int q = atomicAdd(&cursor[col[p]], 1);
        tcol[q] = i;
        if (val) tval[q] = val[p];
    }
}

// Sort each row by column (insertion sort; rows of transposes are short).
__global__ void k_sort_rows(int n, const int *rowptr, int *col, double *val) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rowptr[i], b = rowptr[i + 1];
    for (int p = a + 1; p < b; p++) {
        int c = col[p];
        double v = val ? val[p] : 0.0;
        int q = p - 1;
        while (q >= a && col[q] > c) {
            col[q + 1] = col[q];
            if (val) val[q + 1] = val[q];
            q--;
        }
        col[q + 1] = c;
        if (val) val[q + 1] = v;
    }
}

// ------------------------------------------------------------------ union

// Pattern of S united with T = S^T (both sorted): count (urow == nullptr) or fill.
__global__ void k_union(int n, const int *sr, const int *sc, const int *tr, const int *tc,
                        const int *urow, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = sr[i], pe = sr[i + 1], q = tr[i], qe = tr[i + 1];
    int o = urow ? urow[i] : 0, c = 0;
    while (p < pe || q < qe) {
        int a = p < pe ? sc[p] : INT_MAX;
        int b = q < qe ? tc[q] : INT_MAX;
        int m = a < b ? a : b;
        if (a == m) p++;
        if (b == m) q++;
        if (urow) out[o + c] = m;
        c++;
    }
    if (!urow) out[i] = c;
}

// ------------------------------------------------------------ Jones-Plassmann

constexpr unsigned long long kUncolored = ~0ull;

// One JP round r.  A vertex uncolored at the start of the round (never colored,
// or colored in this very round by someone else) whose key (degree, hash,
// index) beats every neighbour uncolored at the start of the round takes the
// smallest color not held by a neighbour colored in an earlier round.  state
// packs (round << 32 | color) into one 64-bit word, written in one store.
__global__ void k_jp_round(int n, const int *grow, const int *gcol, uint32_t hbase,
                           unsigned long long *state, unsigned r, int *remaining, int *maxcolor) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (state[i] != kUncolored) return;
    int a = grow[i], b = grow[i + 1];
    int di = b - a;
    uint32_t hi = fmix32((uint32_t)i ^ hbase);
    volatile unsigned long long *vs = state;
    for (int p = a; p < b; p++) {
        int j = gcol[p];
        if (j == i) continue;
        unsigned long long sj = vs[j];
        bool unc = sj == kUncolored || (unsigned)(sj >> 32) == r;
        if (!unc) continue;
        int dj = grow[j + 1] - grow[j];
        if (!key_greater(di, hi, i, dj, fmix32((uint32_t)j ^ hbase), j)) return;
    }
    int c = 0;
    for (int base = 0;; base += 64) {
        unsigned long long mask = 0;
        for (int p = a; p < b; p++) {
            unsigned long long sj = vs[gcol[p]];
            if (sj == kUncolored || (unsigned)(sj >> 32) >= r) continue;
            int cj = (int)(unsigned)sj;
            if (cj >= base && cj < base + 64) mask |= 1ull << (cj - base);
        }
        if (mask != ~0ull) {
            c = base + __ffsll((long long)~mask) - 1;
            break;
        }
    }
    state[i] = ((unsigned long long)r << 32) | (unsigned)c;
    atomicSub(remaining, 1);
    atomicMax(maxcolor, c);
}

__global__ void k_state_to_color(int n, const unsigned long long *state, int *color) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) color[i] = (int)(unsigned)state[i];
}

// ---------------------------------------------------------------------- PMIS

__global__ void k_pmis_init(int n, const int *sr, const int *tr, int *cf, int *undecided) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool isolated = sr[i + 1] == sr[i] && tr[i + 1] == tr[i];
    cf[i] = isolated ? 0 : -1;
    if (!isolated) atomicAdd(undecided, 1);
}

// An undecided point whose key (lambda = |S^T_i|, hash, index) beats every
// undecided point of S_i u S^T_i is selected (cf is not written in this pass).
__global__ void k_pmis_select(int n, const int *sr, const int *sc, const int *tr, const int *tc,
                              uint32_t hbase, const int *cf, int *sel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sel[i] = 0;
    if (cf[i] != -1) return;
    int li = tr[i + 1] - tr[i];
    uint32_t hi = fmix32((uint32_t)i ^ hbase);
    for (int pass = 0; pass < 2; pass++) {
        const int *R = pass ? tr : sr;
        const int *Cc = pass ? tc : sc;
        for (int p = R[i]; p < R[i + 1]; p++) {
            int j = Cc[p];
            if (cf[j] != -1) continue;
            int lj = tr[j + 1] - tr[j];
            if (!key_greater(li, hi, i, lj, fmix32((uint32_t)j ^ hbase), j)) return;
        }
    }
    sel[i] = 1;
}

// Selected points become C; undecided points with a C point in S_i become F.
__global__ void k_pmis_commit(int n, const int *sr, const int *sc, int *cf, const int *sel,
                              int *undecided) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (sel[i]) {
        cf[i] = 1;
        atomicSub(undecided, 1);
        return;
    }
    if (cf[i] != -1) return;
    volatile int *vcf = cf;
    for (int p = sr[i]; p < sr[i + 1]; p++) {
        int j = sc[p];
        if (sel[j] || vcf[j] == 1) {
            cf[i] = 0;
            atomicSub(undecided, 1);
            return;
        }
    }
}

__global__ void k_is_c(int n, const int *cf, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cf[i] == 1;
}

// ------------------------------------------------------ direct interpolation

__global__ void k_interp_count(int n, const int *sr, const int *sc, const int *cf, int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == 1) {
        cnt[i] = 1;
        return;
    }
    int c = 0;
    for (int p = sr[i]; p < sr[i + 1]; p++) c += cf[sc[p]] == 1;
    cnt[i] = c;
}

// Stueben's direct interpolation with separate negative/positive scaling and
// lumping of the positive part into the diagonal when C_i has no positive entry.
__global__ void k_interp_fill(int n, const int *ar, const int *ac, const double *av,
                              const int *sr, const int *sc, const int *cf, const int *cidx,
                              const int *pr, int *pc, double *pv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = pr[i];
    if (cf[i] == 1) {
        pc[q] = cidx[i];
        pv[q] = 1.0;
        return;
    }
    int a = ar[i], b = ar[i + 1];
    double aii = 0.0;
    for (int p = a; p < b; p++)
        if (ac[p] == i) aii = av[p];
    double s = aii < 0.0 ? -1.0 : 1.0;
    double sum_n_neg = 0.0, sum_n_pos = 0.0;
    for (int p = a; p < b; p++) {
        if (ac[p] == i) continue;
        double v = __dmul_rn(s, av[p]);
        if (v < 0.0) sum_n_neg = __dadd_rn(sum_n_neg, v);
        else sum_n_pos = __dadd_rn(sum_n_pos, v);
    }
    double sum_c_neg = 0.0, sum_c_pos = 0.0;
    int pa = a;
    for (int p = sr[i]; p < sr[i + 1]; p++) {
        int j = sc[p];
        if (cf[j] != 1) continue;
        while (ac[pa] != j) pa++;
        double v = __dmul_rn(s, av[pa]);
        if (v < 0.0) sum_c_neg = __dadd_rn(sum_c_neg, v);
        else sum_c_pos = __dadd_rn(sum_c_pos, v);
    }
    double d = __dmul_rn(s, aii);
    double alpha = 0.0, beta = 0.0;
    if (sum_c_neg != 0.0) alpha = __ddiv_rn(sum_n_neg, sum_c_neg);
    if (sum_c_pos != 0.0) beta = __ddiv_rn(sum_n_pos, sum_c_pos);
    else d = __dadd_rn(d, sum_n_pos);
    pa = a;
    for (int p = sr[i]; p < sr[i + 1]; p++) {
        int j = sc[p];
        if (cf[j] != 1) continue;
        while (ac[pa] != j) pa++;
        double v = __dmul_rn(s, av[pa]);
        double f = v < 0.0 ? -alpha : -beta;
        pc[q] = cidx[j];
        pv[q] = __ddiv_rn(__dmul_rn(f, v), d);
        q++;
    }
}

// -------------------------------------------------------------------- SpGEMM

__global__ void k_spgemm_count(int n, const int *ar, const int *ac, const int *br, int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long c = 0;
    for (int p = ar[i]; p < ar[i + 1]; p++) {
        int k = ac[p];
        c += br[k + 1] - br[k];
    }
    cnt[i] = (int)min(c, (long)INT_MAX / 4);
}

__global__ void k_spgemm_fill(int n, const int *ar, const int *ac, const int *br, const int *bc,
                              const int *off, int *cand) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = off[i];
    for (int p = ar[i]; p < ar[i + 1]; p++) {
        int k = ac[p];
        for (int q = br[k]; q < br[k + 1]; q++) cand[o++] = bc[q];
    }
}

constexpr int kSortCap = 1024;
constexpr int kSortWarps = 4;

// One warp per row: sort the row's candidate columns and keep each once
// (bitonic sort in shared memory, or repeated minimum selection for rows
// longer than kSortCap).  Unique columns go to uout at the row's offset.
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_unique(int n, const int *off,
                                                                 const int *cand, int *uout,
                                                                 int *ucnt) {
    __shared__ int sbuf[kSortWarps][kSortCap];
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    int row = blockIdx.x * kSortWarps + wl;
    if (row >= n) return;
    int a = off[row], L = off[row + 1] - a;
    const int *d = cand + a;
    int *o = uout + a;
    int *buf = sbuf[wl];
    unsigned lt = (1u << lane) - 1u;
    int cnt = 0;
    if (L <= kSortCap) {
        int P = 1;
        while (P < L) P <<= 1;
        for (int k = lane; k < P; k += 32) buf[k] = k < L ? d[k] : INT_MAX;
        __syncwarp();
        for (int size = 2; size <= P; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < P / 2; t += 32) {
                    int x = (t / stride) * 2 * stride + (t % stride);
                    int y = x + stride;
                    bool up = (x & size) == 0;
                    int u = buf[x], v = buf[y];
                    if ((u > v) == up) {
                        buf[x] = v;
                        buf[y] = u;
                    }
                }
                __syncwarp();
            }
        for (int base = 0; base < L; base += 32) {
            int k = base + lane;
            int v = k < L ? buf[k] : INT_MAX;
            bool keep = k < L && (k == 0 || buf[k - 1] != v);
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            if (keep) o[cnt + __popc(mask & lt)] = v;
            cnt += __popc(mask);
        }
    } else {
        long last = -1;
        for (;;) {
            int m = INT_MAX;
            for (int k = lane; k < L; k += 32) {
                int v = d[k];
                if (v > last && v < m) m = v;
            }
            for (int sh = 16; sh > 0; sh >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, sh));
            if (m == INT_MAX) break;
            if (lane == 0) o[cnt] = m;
            cnt++;
            last = m;
        }
    }
    if (lane == 0) ucnt[row] = cnt;
}

__global__ void k_gather_unique(int n, const int *off, const int *uout, const int *crow,
                                int *ccol) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = off[i], c = crow[i], L = crow[i + 1] - c;
    for (int k = 0; k < L; k++) ccol[c + k] = uout[a + k];
}

// C = A B values, one warp per row, lanes over the row's entries: for entry
// (i, J) the products a_ik b_kJ are added in ascending k, as Gustavson's
// row-by-row accumulation adds them.
__global__ void k_spgemm_numeric(int n, const int *ar, const int *ac, const double *av,
                                 const int *br, const int *bc, const double *bv, const int *cr,
                                 const int *cc, double *cv) {
    int lane = threadIdx.x & 31;
    long row = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    int a = ar[row], b = ar[row + 1];
    for (int e = cr[row] + lane; e < cr[row + 1]; e += 32) {
        int J = cc[e];
        double acc = 0.0;
        for (int p = a; p < b; p++) {
            int k = ac[p];
            int lo = br[k], hi = br[k + 1];
            int q = find_col(bc, lo, hi, J);
            if (q < hi && bc[q] == J) acc = __dadd_rn(acc, __dmul_rn(av[p], bv[q]));
        }
        cv[e] = acc;
    }
}

// -------------------------------------------------------- level helpers

__global__ void k_check_diag(int n, const int *diag, const double *val, double *dinv, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = diag[i];
    double d = p >= 0 ? val[p] : 0.0;
    if (d == 0.0 || !isfinite(d)) {
        set_err(err, CPR_ERR_SINGULAR);
        d = 1.0;
    }
    dinv[i] = 1.0 / d;
}

__global__ void k_color_hist(int n, const int *color, int *hist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&hist[color[i]], 1);
}

__global__ void k_flag_color(int n, const int *color, int c, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = color[i] == c;
}

__global__ void k_scatter_color(int n, const int *color, int c, const int *pos, int base,
                                int *rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && color[i] == c) rows[base + pos[i]] = i;
}

__global__ void k_iperm(int n, const int *order, int *iperm) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) iperm[order[t]] = t;
}

// Row lengths of the renumbered copy: row t is natural row order[t] (order ==
// nullptr: identity), without its diagonal entry when skip_diag.
__global__ void k_perm_count(int n, const int *order, const int *rowptr, const int *col,
                             bool skip_diag, int *cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int i = order ? order[t] : t;
    int c = rowptr[i + 1] - rowptr[i];
    if (skip_diag)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) c -= col[p] == i;
    cnt[t] = c;
}

// Fill the renumbered copy; columns mapped through icol (nullptr: unchanged);
// entries keep the natural (ascending-column) order of their row.
__global__ void k_perm_fill(int n, const int *order, const int *rowptr, const int *col,
                            const double *val, bool skip_diag, const int *icol, const int *nrow,
                            int *ncol, double *nval) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int i = order ? order[t] : t;
    int q = nrow[t];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int j = col[p];
        if (skip_diag && j == i) continue;
        ncol[q] = icol ? icol[j] : j;
        nval[q] = val[p];
        q++;
    }
}

__global__ void k_perm_diag(int n, const int *order, const int *rowptr, const int *col,
                            const double *val, double *diag, double *dinv) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int i = order[t];
    double d = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
        if (col[p] == i) d = val[p];
    diag[t] = d;
    dinv[t] = 1.0 / d;
}

__global__ void k_csr_to_dense(int n, const int *rowptr, const int *col, const double *val,
                               double *a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) a[(size_t)i * n + col[p]] = val[p];
}

// Dense LU with partial pivoting (largest |a|, lowest index on ties) of the
// coarsest matrix, then its inverse column by column, stored column-major
// (inv[j*n + i] = (A^-1)_ij).  One CTA.
__global__ void __launch_bounds__(1024) k_dense_lu_inverse(int n, double *a, int *piv,
                                                           double *inv, int *err) {
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int pivot_row;
    int tid = threadIdx.x, nt = blockDim.x;
    for (int k = 0; k < n; k++) {
        double best = -1.0;
        int bi = INT_MAX;
        for (int i = k + tid; i < n; i += nt) {
            double v = fabs(a[(size_t)i * n + k]);
            if (v > best || (v == best && i < bi)) {
                best = v;
                bi = i;
            }
        }
        for (int sh = 16; sh > 0; sh >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, sh);
            int oi = __shfl_xor_sync(0xffffffffu, bi, sh);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if ((tid & 31) == 0) {
            sv[tid >> 5] = best;
            si[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double bv = sv[0];
            int bidx = si[0];
            for (int w = 1; w < (nt + 31) / 32; w++)
                if (sv[w] > bv || (sv[w] == bv && si[w] < bidx)) {
                    bv = sv[w];
                    bidx = si[w];
                }
            if (!(bv > 0.0)) {
                set_err(err, CPR_ERR_SINGULAR);
                bidx = k;
            }
            pivot_row = bidx;
            piv[k] = bidx;
        }
        __syncthreads();
        int p = pivot_row;
        if (p != k)
            for (int j = tid; j < n; j += nt) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        __syncthreads();
        double pk = a[(size_t)k * n + k];
        if (pk == 0.0) pk = 1.0;
        for (int i = k + 1 + tid; i < n; i += nt) a[(size_t)i * n + k] /= pk;
        __syncthreads();
        int m = n - k - 1;
        for (long e = tid; e < (long)m * m; e += nt) {
            int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
            a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
        }
        __syncthreads();
    }
    for (int j = tid; j < n; j += nt) {
        double *x = inv + (size_t)j * n;
        for (int i = 0; i < n; i++) x[i] = i == j ? 1.0 : 0.0;
        for (int k = 0; k < n; k++) {
            int p = piv[k];
            double t = x[k];
            x[k] = x[p];
            x[p] = t;
        }
        for (int i = 0; i < n; i++) {
            double s = x[i];
            for (int q = 0; q < i; q++) s -= a[(size_t)i * n + q] * x[q];
            x[i] = s;
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = x[i];
            for (int q = i + 1; q < n; q++) s -= a[(size_t)i * n + q] * x[q];
            double d = a[(size_t)i * n + i];
            x[i] = s / (d == 0.0 ? 1.0 : d);
        }
    }
}

// out (row-major) = in^T, n x n.
__global__ void k_transpose_dense(int n, const double *in, double *out) {
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    int i = (int)(e / n), j = (int)(e % n);
    out[e] = in[(size_t)j * n + i];
}

// ------------------------------------------------------------------ BILU(0)

__device__ __forceinline__ void mat3_mul_rn(const double *a, const double *b, double *c) {
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double t = 0.0;
            for (int k = 0; k < 3; k++) t = __dadd_rn(t, __dmul_rn(a[3 * r + k], b[3 * k + s]));
            c[3 * r + s] = t;
        }
}

__device__ __forceinline__ bool mat3_inv_rn(const double *a, double *inv) {
    double c00 = __dsub_rn(__dmul_rn(a[4], a[8]), __dmul_rn(a[5], a[7]));
    double c01 = __dsub_rn(__dmul_rn(a[5], a[6]), __dmul_rn(a[3], a[8]));
    double c02 = __dsub_rn(__dmul_rn(a[3], a[7]), __dmul_rn(a[4], a[6]));
    double det = __dadd_rn(__dadd_rn(__dmul_rn(a[0], c00), __dmul_rn(a[1], c01)), __dmul_rn(a[2], c02));
    if (det == 0.0 || !isfinite(det)) return false;
    inv[0] = __ddiv_rn(c00, det);
    inv[1] = __ddiv_rn(__dsub_rn(__dmul_rn(a[2], a[7]), __dmul_rn(a[1], a[8])), det);
    inv[2] = __ddiv_rn(__dsub_rn(__dmul_rn(a[1], a[5]), __dmul_rn(a[2], a[4])), det);
    inv[3] = __ddiv_rn(c01, det);
    inv[4] = __ddiv_rn(__dsub_rn(__dmul_rn(a[0], a[8]), __dmul_rn(a[2], a[6])), det);
    inv[5] = __ddiv_rn(__dsub_rn(__dmul_rn(a[2], a[3]), __dmul_rn(a[0], a[5])), det);
    inv[6] = __ddiv_rn(c02, det);
    inv[7] = __ddiv_rn(__dsub_rn(__dmul_rn(a[1], a[6]), __dmul_rn(a[0], a[7])), det);
    inv[8] = __ddiv_rn(__dsub_rn(__dmul_rn(a[0], a[4]), __dmul_rn(a[1], a[3])), det);
    return true;
}

// Factor the block rows of one color; rows of lower colors are final.  For
// row i, the entries k before i in (color, index) order are eliminated in that
// order: L_ik = A_ik U_kk^-1, then A_ij -= L_ik U_kj for j after k in row k
// that lies in row i's pattern.  Same-color rows are never adjacent (the
// block coloring is at theta = 0), so "after k" means "higher color than k".
__global__ void k_bilu_factor_color(const int *rows, int cnt, const int *rowptr, const int *col,
                                    const int *color, const int *diag, double *lu, int *err) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    int i = rows[t];
    int a = rowptr[i], b = rowptr[i + 1];
    int ci = color[i];
    int last_c = -1, last_k = -1;
    for (;;) {
        int best = -1, bc = INT_MAX, bk = INT_MAX;
        for (int p = a; p < b; p++) {
            int k = col[p];
            int ck = color[k];
            if (ck >= ci) continue;
            bool after_last = ck > last_c || (ck == last_c && k > last_k);
            bool before_best = ck < bc || (ck == bc && k < bk);
            if (after_last && before_best) {
                best = p;
                bc = ck;
                bk = k;
            }
        }
        if (best < 0) break;
        int k = bk;
        double L[9];
        mat3_mul_rn(lu + 9 * (size_t)best, lu + 9 * (size_t)diag[k], L);
        for (int e = 0; e < 9; e++) lu[9 * (size_t)best + e] = L[e];
        for (int q = rowptr[k]; q < rowptr[k + 1]; q++) {
            int j = col[q];
            if (j == k || color[j] <= color[k]) continue;
            int r = find_col(col, a, b, j);
            if (r >= b || col[r] != j) continue;
            double P[9];
            mat3_mul_rn(L, lu + 9 * (size_t)q, P);
            for (int e = 0; e < 9; e++) lu[9 * (size_t)r + e] = __dsub_rn(lu[9 * (size_t)r + e], P[e]);
        }
        last_c = bc;
        last_k = bk;
    }
    double inv[9];
    double *D = lu + 9 * (size_t)diag[i];
    if (!mat3_inv_rn(D, inv)) {
        set_err(err, CPR_ERR_SINGULAR);
        return;
    }
    for (int e = 0; e < 9; e++) D[e] = inv[e];
}

// Split the factor array into L (lower colors), U (higher colors) and D^-1.
__global__ void k_bilu_split_count(int nb, const int *rowptr, const int *col, const int *color,
                                   int *lcnt, int *ucnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int l = 0, u = 0, ci = color[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int j = col[p];
        if (j == i) continue;
        if (color[j] < ci) l++;
        else u++;
    }
    lcnt[i] = l;
    ucnt[i] = u;
}

__global__ void k_bilu_split_fill(int nb, const int *rowptr, const int *col, const int *color,
                                  const double *lu, const int *lr, int *lc, double *lv,
                                  const int *ur, int *uc, double *uv, double *dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int ql = lr[i], qu = ur[i], ci = color[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        int j = col[p];
        const double *src = lu + 9 * (size_t)p;
        double *dst;
        if (j == i) {
            dst = dinv + 9 * (size_t)i;
        } else if (color[j] < ci) {
            lc[ql] = j;
            dst = lv + 9 * (size_t)ql++;
        } else {
            uc[qu] = j;
            dst = uv + 9 * (size_t)qu++;
        }
        for (int e = 0; e < 9; e++) dst[e] = src[e];
    }
}

__global__ void k_d2f(long n, const double *a, float *b) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ------------------------------------------------------------ host helpers

struct Graph {
    int n = 0, nnz = 0;
    DVec<int> rowptr, col;
};

void check_err(cpr_handle *h, const char *what) {
    int e = read_int(h->err.p, h->stream);
    if (e != 0) {
        CK(cudaMemsetAsync(h->err.p, 0, sizeof(int), h->stream));
        fail(e, what);
    }
}

// A pattern CSR from a count pass and a fill pass over rows.
template <class CountFill>
Graph build_pattern(int n, cudaStream_t s, CountFill cf) {
    Graph g;
    g.n = n;
    DVec<int> cnt;
    cnt.alloc(n, s);
    cf(nullptr, cnt.p);
    g.rowptr.alloc(n + 1, s);
    exclusive_scan(cnt.p, g.rowptr.p, n, s);
    g.nnz = read_int(g.rowptr.p + n, s);
    g.col.alloc(std::max(g.nnz, 1), s);
    cf(g.rowptr.p, g.col.p);
    return g;
}

// Transpose (pattern, or with values when val != nullptr); rows of the result sorted.
void transpose(int n, int ncol, int nnz, const int *rowptr, const int *col, const double *val,
               DVec<int> &trow, DVec<int> &tcol, DVec<double> *tval, cudaStream_t s) {
    DVec<int> cnt, cursor;
    cnt.alloc(std::max(ncol, 1), s);
    cnt.zero();
    if (nnz) {
        k_count_cols<<<grid_for(nnz, kBlock, 148 * 32), kBlock, 0, s>>>(nnz, col, cnt.p);
        CK_LAUNCH();
    }
    trow.alloc(ncol + 1, s);
    exclusive_scan(cnt.p, trow.p, ncol, s);
    cursor.alloc(std::max(ncol, 1), s);
    if (ncol) CK(cudaMemcpyAsync(cursor.p, trow.p, sizeof(int) * ncol, cudaMemcpyDeviceToDevice, s));
    tcol.alloc(std::max(nnz, 1), s);
    if (tval) tval->alloc(std::max(nnz, 1), s);
    k_scatter_t<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, rowptr, col, val, cursor.p, tcol.p,
                                                      tval ? tval->p : nullptr);
    CK_LAUNCH();
    if (ncol) {
        k_sort_rows<<<grid_for(ncol, kBlock), kBlock, 0, s>>>(ncol, trow.p, tcol.p, tval ? tval->p : nullptr);
        CK_LAUNCH();
    }
}

Graph sym_union(const Graph &S, cudaStream_t s) {
    DVec<int> trow, tcol;
    transpose(S.n, S.n, S.nnz, S.rowptr.p, S.col.p, nullptr, trow, tcol, nullptr, s);
    int n = S.n;
    return build_pattern(n, s, [&](const int *urow, int *out) {
        k_union<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, trow.p, tcol.p, urow, out);
        CK_LAUNCH();
    });
}

// Jones-Plassmann coloring of graph G; returns the number of colors.
int jp_color(cpr_handle *h, const Graph &G, int salt, int level, DVec<int> &color) {
    cudaStream_t s = h->stream;
    int n = G.n;
    DVec<unsigned long long> state;
    state.alloc(n, s);
    CK(cudaMemsetAsync(state.p, 0xff, sizeof(unsigned long long) * n, s));
    DVec<int> counters;  // remaining, max color
    counters.alloc(2, s);
    int init[2] = {n, 0};
    CK(cudaMemcpyAsync(counters.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
    uint32_t hb = hash_base(h->opt.seed, salt, level);
    unsigned r = 0;
    for (;;) {
        for (int k = 0; k < 4; k++, r++) {
            k_jp_round<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, G.rowptr.p, G.col.p, hb, state.p, r,
                                                             counters.p, counters.p + 1);
            CK_LAUNCH();
        }
        if (read_int(counters.p, s) == 0) break;
        if (r > (unsigned)n + 8) fail(CPR_ERR_CUDA, "coloring did not terminate");
    }
    color.alloc(n, s);
    k_state_to_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, state.p, color.p);
    CK_LAUNCH();
    return read_int(counters.p + 1, s) + 1;
}

// Rows grouped by color, index-ascending within a color.
void rows_by_color(cpr_handle *h, int n, const int *color, int ncolors, std::vector<int> &off,
                   DVec<int> &rows) {
    cudaStream_t s = h->stream;
    DVec<int> hist, flag, pos;
    hist.alloc(ncolors, s);
    hist.zero();
    k_color_hist<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, color, hist.p);
    CK_LAUNCH();
    std::vector<int> hh(ncolors);
    CK(cudaMemcpyAsync(hh.data(), hist.p, sizeof(int) * ncolors, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    off.assign(ncolors + 1, 0);
    for (int c = 0; c < ncolors; c++) off[c + 1] = off[c] + hh[c];
    rows.alloc(n, s);
    flag.alloc(n, s);
    pos.alloc(n + 1, s);
    for (int c = 0; c < ncolors; c++) {
        k_flag_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, color, c, flag.p);
        CK_LAUNCH();
        exclusive_scan(flag.p, pos.p, n, s);
        k_scatter_color<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, color, c, pos.p, off[c], rows.p);
        CK_LAUNCH();
    }
}

// C = A B (structural pattern, sorted; values in Gustavson order).
void spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
    int n = A.n;
    DVec<int> cnt, off, cand, uout, ucnt;
    cnt.alloc(n, s);
    k_spgemm_count<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, B.rowptr.p, cnt.p);
    CK_LAUNCH();
    off.alloc(n + 1, s);
    exclusive_scan(cnt.p, off.p, n, s);
    int total = read_int(off.p + n, s);
    if (total < 0) fail(CPR_ERR_OOM, "Galerkin product too large");
    cand.alloc(std::max(total, 1), s);
    uout.alloc(std::max(total, 1), s);
    k_spgemm_fill<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, A.rowptr.p, A.col.p, B.rowptr.p, B.col.p,
                                                        off.p, cand.p);
    CK_LAUNCH();
    ucnt.alloc(n, s);
    k_sort_unique<<<(n + kSortWarps - 1) / kSortWarps, kSortWarps * 32, 0, s>>>(n, off.p, cand.p,
                                                                                uout.p, ucnt.p);
    CK_LAUNCH();
    cand.release();
    C.n = n;
    C.ncol = B.ncol;
    C.rowptr.alloc(n + 1, s);
    exclusive_scan(ucnt.p, C.rowptr.p, n, s);
    C.nnz = read_int(C.rowptr.p + n, s);
    C.col.alloc(std::max(C.nnz, 1), s);
    C.val.alloc(std::max(C.nnz, 1), s);
    k_gather_unique<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, off.p, uout.p, C.rowptr.p, C.col.p);
    CK_LAUNCH();
    long threads = (long)n * 32;
    k_spgemm_numeric<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        n, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p, C.rowptr.p, C.col.p, C.val.p);
    CK_LAUNCH();
}

void to_f32(const DVec<double> &a, DVec<float> &b, cudaStream_t s) {
    b.alloc(std::max<size_t>(a.n, 1), s);
    if (a.n) {
        k_d2f<<<grid_for((long)a.n, kBlock, 148 * 16), kBlock, 0, s>>>((long)a.n, a.p, b.p);
        CK_LAUNCH();
    }
}

// dst = src with rows taken in `order` and columns mapped through icol.
void perm_csr(const DCsr &src, const int *order, const int *icol, int ncol, bool skip_diag, DCsr &dst,
              cudaStream_t s) {
    int n = src.n;
    DVec<int> cnt;
    cnt.alloc(std::max(n, 1), s);
    k_perm_count<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, order, src.rowptr.p, src.col.p, skip_diag, cnt.p);
    CK_LAUNCH();
    dst.n = n;
    dst.ncol = ncol;
    dst.rowptr.alloc(n + 1, s);
    exclusive_scan(cnt.p, dst.rowptr.p, n, s);
    dst.nnz = read_int(dst.rowptr.p + n, s);
    dst.col.alloc(std::max(dst.nnz, 1), s);
    dst.val.alloc(std::max(dst.nnz, 1), s);
    k_perm_fill<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, order, src.rowptr.p, src.col.p, src.val.p, skip_diag,
                                                      icol, dst.rowptr.p, dst.col.p, dst.val.p);
    CK_LAUNCH();
}

// Lanes per row for a row length: the power of two >= the mean length, 4..32.
int lanes_for(long nnz, int n) {
    double avg = n ? (double)nnz / n : 1.0;
    int g = 4;
    while (g < 32 && g < avg) g <<= 1;
    return g;
}

void copy_ints(DVec<int> &dst, const int *src, size_t n, cudaStream_t s) {
    dst.alloc(std::max<size_t>(n, 1), s);
    if (n) CK(cudaMemcpyAsync(dst.p, src, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
}

}  // namespace

// ================================================================== public

void validate_bsr(const int *rowptr, const int *col, int nb, int nnzb, int *derr, cudaStream_t s) {
    k_validate_bsr<<<grid_for(nb, kBlock), kBlock, 0, s>>>(rowptr, col, nb, nnzb, derr);
    CK_LAUNCH();
}

void free_preconditioner(cpr_handle *h) {
    h->lev.clear();
    h->pcol0.release();
    h->pcol0_32.release();
    h->w.release();
    h->w32.release();
    h->cinv.release();
    h->bilu = Bilu{};
    h->cn = 0;
    h->have_B = false;
}

// Build B from the handle's current A (Sec. 3.1; the setup lines of Alg. 6 per level).
void build_preconditioner(cpr_handle *h) {
    free_preconditioner(h);
    cudaStream_t s = h->stream;
    const cpr_opts &o = h->opt;
    int nb = h->nb, nnzb = h->nnzb;
    bool f32 = o.precond_fp32 != 0;

    // ---- decoupling and the pressure matrix A_P (level 0) ----
    DVec<int> bdiag;
    bdiag.alloc(nb, s);
    k_diagpos<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->col.p, bdiag.p);
    CK_LAUNCH();
    h->w.alloc(3 * (size_t)nb, s);
    k_decouple<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, bdiag.p, h->val.p, o.decouple, h->w.p, h->err.p);
    CK_LAUNCH();
    check_err(h, "singular diagonal block in the decoupling");
    h->lev.emplace_back();
    {
        Level &L0 = h->lev[0];
        L0.A.n = L0.A.ncol = nb;
        L0.A.nnz = nnzb;
        copy_ints(L0.A.rowptr, h->rowptr.p, nb + 1, s);
        copy_ints(L0.A.col, h->col.p, nnzb, s);
        L0.A.val.alloc(nnzb, s);
        h->pcol0.alloc(3 * (size_t)nnzb, s);
        k_pressure_matrix<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->val.p, h->w.p,
                                                                 L0.A.val.p, h->pcol0.p);
        CK_LAUNCH();
    }

    // ---- the AMG hierarchy ----
    for (int l = 0;; l++) {
        int n = h->lev[l].A.n;
        {
            Level &L = h->lev[l];
            DVec<int> diag;
            diag.alloc(n, s);
            k_diagpos<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p, diag.p);
            CK_LAUNCH();
            DVec<double> dtmp;
            dtmp.alloc(n, s);
            k_check_diag<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, diag.p, L.A.val.p, dtmp.p, h->err.p);
            CK_LAUNCH();
            check_err(h, "zero diagonal on an AMG level");
        }
        if (n <= o.coarse_max || l + 1 >= o.max_levels) break;
        Level &L = h->lev[l];
        // classical strength and PMIS
        Graph S = build_pattern(n, s, [&](const int *srow, int *out) {
            k_strength_rs<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p, L.A.val.p,
                                                                o.theta_amg, srow, out);
            CK_LAUNCH();
        });
        DVec<int> trow, tcol;
        transpose(n, n, S.nnz, S.rowptr.p, S.col.p, nullptr, trow, tcol, nullptr, s);
        L.cf.alloc(n, s);
        DVec<int> sel, und;
        sel.alloc(n, s);
        und.alloc(1, s);
        und.zero();
        k_pmis_init<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, trow.p, L.cf.p, und.p);
        CK_LAUNCH();
        uint32_t hb = hash_base(o.seed, 1, l);
        int rounds = 0;
        while (read_int(und.p, s) > 0) {
            for (int k = 0; k < 3; k++, rounds++) {
                k_pmis_select<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, trow.p,
                                                                    tcol.p, hb, L.cf.p, sel.p);
                CK_LAUNCH();
                k_pmis_commit<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, L.cf.p,
                                                                    sel.p, und.p);
                CK_LAUNCH();
            }
            if (rounds > n + 8) fail(CPR_ERR_CUDA, "C/F splitting did not terminate");
        }
        DVec<int> flag, cidx;
        flag.alloc(n, s);
        cidx.alloc(n + 1, s);
        k_is_c<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.cf.p, flag.p);
        CK_LAUNCH();
        exclusive_scan(flag.p, cidx.p, n, s);
        int nc = read_int(cidx.p + n, s);
        if (nc == 0 || (double)nc > 0.95 * (double)n) {
            L.cf.release();
            break;
        }
        L.nc = nc;
        // direct interpolation P and R = P^T
        {
            DVec<int> cnt;
            cnt.alloc(n, s);
            k_interp_count<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, S.rowptr.p, S.col.p, L.cf.p, cnt.p);
            CK_LAUNCH();
            L.P.n = n;
            L.P.ncol = nc;
            L.P.rowptr.alloc(n + 1, s);
            exclusive_scan(cnt.p, L.P.rowptr.p, n, s);
            L.P.nnz = read_int(L.P.rowptr.p + n, s);
            L.P.col.alloc(std::max(L.P.nnz, 1), s);
            L.P.val.alloc(std::max(L.P.nnz, 1), s);
            k_interp_fill<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p, L.A.val.p,
                                                                S.rowptr.p, S.col.p, L.cf.p, cidx.p,
                                                                L.P.rowptr.p, L.P.col.p, L.P.val.p);
            CK_LAUNCH();
            L.R.n = nc;
            L.R.ncol = n;
            L.R.nnz = L.P.nnz;
            transpose(n, nc, L.P.nnz, L.P.rowptr.p, L.P.col.p, L.P.val.p, L.R.rowptr, L.R.col, &L.R.val, s);
        }
        // Galerkin coarse matrix A_{l+1} = R (A P)
        DCsr AP, Ac;
        spgemm(L.A, L.P, AP, s);
        spgemm(L.R, AP, Ac, s);
        AP = DCsr{};
        // the smoother's coloring: Eq. 5.1 strength, symmetrised, JP
        {
            Graph Sc = build_pattern(n, s, [&](const int *srow, int *out) {
                k_strength51<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, L.A.rowptr.p, L.A.col.p,
                                                                   L.A.val.p, o.theta_color, srow, out);
                CK_LAUNCH();
            });
            Graph G = sym_union(Sc, s);
            L.ncolors = jp_color(h, G, 0, l, L.color);
            rows_by_color(h, n, L.color.p, L.ncolors, L.color_off, L.rows_by_color);
        }
        h->lev.emplace_back();
        h->lev[l + 1].A = std::move(Ac);
    }

    // ---- coarsest level: dense inverse ----
    {
        Level &C = h->lev.back();
        int n = C.A.n;
        if (n > kMaxCoarse) fail(CPR_ERR_INVALID, "coarsest level larger than the dense-solve limit");
        h->cn = n;
        DVec<double> a;
        DVec<int> piv;
        a.alloc((size_t)n * n, s);
        a.zero();
        piv.alloc(n, s);
        h->cinv.alloc((size_t)n * n, s);
        k_csr_to_dense<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, C.A.rowptr.p, C.A.col.p, C.A.val.p, a.p);
        CK_LAUNCH();
        DVec<double> colmajor;
        colmajor.alloc((size_t)n * n, s);
        k_dense_lu_inverse<<<1, 1024, 0, s>>>(n, a.p, piv.p, colmajor.p, h->err.p);
        CK_LAUNCH();
        check_err(h, "singular coarsest matrix");
        k_transpose_dense<<<grid_for((long)n * n, kBlock), kBlock, 0, s>>>(n, colmajor.p, h->cinv.p);
        CK_LAUNCH();
    }

    // ---- second stage: multicolor BILU(0) ----
    {
        Bilu &B = h->bilu;
        Graph S = build_pattern(nb, s, [&](const int *srow, int *out) {
            k_offdiag_pattern<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->col.p, srow, out);
            CK_LAUNCH();
        });
        Graph G = sym_union(S, s);
        B.ncolors = jp_color(h, G, 2, 0, B.color);
        rows_by_color(h, nb, B.color.p, B.ncolors, B.color_off, B.rows_by_color);
        B.lu.alloc(9 * (size_t)nnzb, s);
        CK(cudaMemcpyAsync(B.lu.p, h->val.p, sizeof(double) * 9 * (size_t)nnzb, cudaMemcpyDeviceToDevice, s));
        for (int c = 0; c < B.ncolors; c++) {
            int cnt = B.color_off[c + 1] - B.color_off[c];
            if (!cnt) continue;
            k_bilu_factor_color<<<grid_for(cnt, 128), 128, 0, s>>>(B.rows_by_color.p + B.color_off[c], cnt,
                                                                  h->rowptr.p, h->col.p, B.color.p,
                                                                  bdiag.p, B.lu.p, h->err.p);
            CK_LAUNCH();
        }
        check_err(h, "singular pivot block in BILU(0)");
        DVec<int> lcnt, ucnt;
        lcnt.alloc(nb, s);
        ucnt.alloc(nb, s);
        k_bilu_split_count<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->col.p, B.color.p,
                                                                  lcnt.p, ucnt.p);
        CK_LAUNCH();
        B.Lrowptr.alloc(nb + 1, s);
        B.Urowptr.alloc(nb + 1, s);
        exclusive_scan(lcnt.p, B.Lrowptr.p, nb, s);
        exclusive_scan(ucnt.p, B.Urowptr.p, nb, s);
        int nl = read_int(B.Lrowptr.p + nb, s), nu = read_int(B.Urowptr.p + nb, s);
        B.Lcol.alloc(std::max(nl, 1), s);
        B.Ucol.alloc(std::max(nu, 1), s);
        B.Lval.alloc(9 * (size_t)std::max(nl, 1), s);
        B.Uval.alloc(9 * (size_t)std::max(nu, 1), s);
        B.Dinv.alloc(9 * (size_t)nb, s);
        k_bilu_split_fill<<<grid_for(nb, kBlock), kBlock, 0, s>>>(nb, h->rowptr.p, h->col.p, B.color.p,
                                                                 B.lu.p, B.Lrowptr.p, B.Lcol.p, B.Lval.p,
                                                                 B.Urowptr.p, B.Ucol.p, B.Uval.p, B.Dinv.p);
        CK_LAUNCH();
    }

    // ---- solve copies in color order, FP32 shadows, work vectors ----
    int L = (int)h->lev.size();
    for (int l = 0; l < L; l++) {
        Level &Lv = h->lev[l];
        int n = Lv.A.n;
        bool coarsest = l == L - 1;
        if (!coarsest) {
            Lv.iperm.alloc(n, s);
            k_iperm<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, Lv.rows_by_color.p, Lv.iperm.p);
            CK_LAUNCH();
        }
    }
    for (int l = 0; l < L - 1; l++) {
        Level &Lv = h->lev[l];
        Level &Nx = h->lev[l + 1];
        int n = Lv.A.n;
        const int *next_iperm = (l + 1 == L - 1) ? nullptr : Nx.iperm.p;
        const int *next_order = (l + 1 == L - 1) ? nullptr : Nx.rows_by_color.p;
        perm_csr(Lv.A, Lv.rows_by_color.p, Lv.iperm.p, n, true, Lv.Ao, s);
        perm_csr(Lv.P, Lv.rows_by_color.p, next_iperm, Lv.P.ncol, false, Lv.Pp, s);
        perm_csr(Lv.R, next_order, Lv.iperm.p, n, false, Lv.Rp, s);
        Lv.diag.alloc(n, s);
        Lv.dinv.alloc(n, s);
        k_perm_diag<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, Lv.rows_by_color.p, Lv.A.rowptr.p, Lv.A.col.p,
                                                          Lv.A.val.p, Lv.diag.p, Lv.dinv.p);
        CK_LAUNCH();
        Lv.gA = lanes_for(Lv.Ao.nnz, n);
        Lv.gP = lanes_for(Lv.Pp.nnz, n);
        Lv.gR = lanes_for(Lv.Rp.nnz, Lv.Rp.n);
    }
    if (f32) {
        to_f32(h->pcol0, h->pcol0_32, s);
        to_f32(h->w, h->w32, s);
        to_f32(h->bilu.Lval, h->bilu.Lval32, s);
        to_f32(h->bilu.Uval, h->bilu.Uval32, s);
        to_f32(h->bilu.Dinv, h->bilu.Dinv32, s);
    }
    for (int l = 0; l < L; l++) {
        Level &Lv = h->lev[l];
        int n = Lv.A.n;
        Lv.x.alloc(n, s);
        Lv.b.alloc(n, s);
        Lv.r.alloc(n, s);
        Lv.s0.alloc(n, s);
        Lv.s1.alloc(n, s);
        if (f32) {
            if (l < L - 1) {
                to_f32(Lv.Ao.val, Lv.Aoval32, s);
                to_f32(Lv.diag, Lv.diag32, s);
                to_f32(Lv.dinv, Lv.dinv32, s);
                to_f32(Lv.Pp.val, Lv.Ppval32, s);
                to_f32(Lv.Rp.val, Lv.Rpval32, s);
            }
            Lv.x32.alloc(n, s);
            Lv.b32.alloc(n, s);
            Lv.r32.alloc(n, s);
            Lv.s0_32.alloc(n, s);
            Lv.s1_32.alloc(n, s);
        }
    }
    CK(cudaStreamSynchronize(s));
    h->have_B = true;
    h->epoch++;
}

}  // namespace cpr
