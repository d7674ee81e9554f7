// Batched solves (C ABI): many independent systems of uneven size share one
// handle.  Their BSR matrices are concatenated into one block-diagonal matrix,
// so the preconditioner's setup and every preconditioner kernel run once over
// all systems; FGMRES runs per system in lockstep (solve.cu, fgmres_batch).
#include <chrono>

#include "cpr_internal.cuh"

using namespace cpr;

namespace {

__global__ void k_offset_rows(int n, const int *src, int *dst, int add) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + add;
}

__global__ void k_add(long n, int *a, int add) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) a[i] += add;
}

// Concatenate the systems into one block-diagonal BSR on the device.
void concat(int nsys, const cpr_bsr3 *A, cudaStream_t s, DVec<int> &rp, DVec<int> &cl, DVec<double> &v,
            std::vector<int> &boff, int &nb, int &nnzb) {
    boff.assign(nsys + 1, 0);
    std::vector<long> poff(nsys + 1, 0);
    for (int k = 0; k < nsys; k++) {
        if (A[k].nb < 1 || A[k].nnzb < A[k].nb || !A[k].rowptr || !A[k].col || !A[k].val)
            fail(CPR_ERR_INVALID, "bad matrix descriptor in the batch");
        boff[k + 1] = boff[k] + A[k].nb;
        poff[k + 1] = poff[k] + A[k].nnzb;
    }
    if (poff[nsys] > (long)INT32_MAX / 9) fail(CPR_ERR_INVALID, "batch too large");
    nb = boff[nsys];
    nnzb = (int)poff[nsys];
    rp.alloc(nb + 1, s);
    cl.alloc(nnzb, s);
    v.alloc(9 * (size_t)nnzb, s);
    DVec<int> tmp;
    int maxnb = 0;
    for (int k = 0; k < nsys; k++) maxnb = std::max(maxnb, A[k].nb);
    tmp.alloc(maxnb + 1, s);
    for (int k = 0; k < nsys; k++) {
        CK(cudaMemcpyAsync(tmp.p, A[k].rowptr, sizeof(int) * (A[k].nb + 1), cudaMemcpyDefault, s));
        k_offset_rows<<<grid_for(A[k].nb + 1, 256), 256, 0, s>>>(A[k].nb + (k == nsys - 1 ? 1 : 0), tmp.p,
                                                                rp.p + boff[k], (int)poff[k]);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(cl.p + poff[k], A[k].col, sizeof(int) * A[k].nnzb, cudaMemcpyDefault, s));
        k_add<<<grid_for(A[k].nnzb, 256, 148 * 8), 256, 0, s>>>(A[k].nnzb, cl.p + poff[k], boff[k]);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(v.p + 9 * poff[k], A[k].val, sizeof(double) * 9 * A[k].nnzb, cudaMemcpyDefault, s));
    }
    CK(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

int cpr_batch_setup(cpr_handle **out, int nsys, const cpr_bsr3 *A, const cpr_opts *opts) {
    if (!out || nsys < 1 || !A) return CPR_ERR_INVALID;
    *out = nullptr;
    cudaStream_t s = opts && opts->stream ? (cudaStream_t)opts->stream : nullptr;
    DVec<int> rp, cl;
    DVec<double> v;
    std::vector<int> boff;
    int nb = 0, nnzb = 0;
    int rc = guarded([&] {
        concat(nsys, A, s, rp, cl, v, boff, nb, nnzb);
        return CPR_OK;
    });
    if (rc != CPR_OK) return rc;
    cpr_bsr3 all{nb, nnzb, rp.p, cl.p, v.p};
    cpr_handle *h = nullptr;
    rc = cpr_setup(&h, &all, opts);
    if (rc != CPR_OK) return rc;
    rc = guarded([&] {
        h->batch = new BatchInfo();
        h->batch->nsys = nsys;
        h->batch->boff = boff;
        batch_prepare(h);
        return CPR_OK;
    });
    if (rc != CPR_OK) {
        cpr_destroy(h);
        return rc;
    }
    *out = h;
    return CPR_OK;
}

int cpr_batch_update(cpr_handle *h, const cpr_bsr3 *A) {
    if (!h || !h->batch || !A) return CPR_ERR_INVALID;
    return guarded([&] {
        DeviceGuard dg(h->device);
        BatchInfo &B = *h->batch;
        DVec<int> rp, cl;
        DVec<double> v;
        std::vector<int> boff;
        int nb = 0, nnzb = 0;
        concat(B.nsys, A, h->stream, rp, cl, v, boff, nb, nnzb);
        if (boff != B.boff) fail(CPR_ERR_INVALID, "the batch's system sizes changed");
        cpr_bsr3 all{nb, nnzb, rp.p, cl.p, v.p};
        return cpr_update(h, &all);
    });
}

int cpr_batch_solve(cpr_handle *h, const double *const *b, double *const *x, double rtol, cpr_stats *st) {
    if (!h || !h->batch || !b || !x || !(rtol > 0.0)) return CPR_ERR_INVALID;
    BatchInfo &B = *h->batch;
    return guarded([&] {
        DeviceGuard dg(h->device);
        auto t0 = std::chrono::steady_clock::now();
        cudaStream_t s = h->stream;
        for (int k = 0; k < B.nsys; k++) {
            if (!b[k] || !x[k]) fail(CPR_ERR_INVALID, "null vector in the batch");
            size_t bytes = sizeof(double) * 3 * (size_t)(B.boff[k + 1] - B.boff[k]);
            CK(cudaMemcpyAsync(B.b.p + 3 * (size_t)B.boff[k], b[k], bytes, cudaMemcpyDefault, s));
            CK(cudaMemcpyAsync(B.x.p + 3 * (size_t)B.boff[k], x[k], bytes, cudaMemcpyDefault, s));
        }
        int rc = fgmres_batch(h, rtol, st);
        for (int k = 0; k < B.nsys; k++) {
            size_t bytes = sizeof(double) * 3 * (size_t)(B.boff[k + 1] - B.boff[k]);
            CK(cudaMemcpyAsync(x[k], B.x.p + 3 * (size_t)B.boff[k], bytes, cudaMemcpyDefault, s));
        }
        CK(cudaStreamSynchronize(s));
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (st)
            for (int k = 0; k < B.nsys; k++) {
                st[k].setup_called = h->setup_called;
                st[k].setup_count = h->setup_count;
                st[k].levels = (int)h->lev.size();
                st[k].setup_ms = h->setup_called ? h->setup_ms : 0.0;
                st[k].solve_ms = ms;
            }
        return rc;
    });
}

int cpr_batch_size(const cpr_handle *h) { return h && h->batch ? h->batch->nsys : 0; }

}  // extern "C"
