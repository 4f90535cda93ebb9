// incremental.cu -- host set-up of the incremental residual.
//
// Algorithm 1 forms the full residual r = b - A x once per iteration, after
// the static updates, to pick the dynamic block; in Section 3.1's cost count
// this O(mn) product dominates an iteration, and the paper leaves a cheaper
// evaluation open.  The incremental mode keeps r up to date instead: every
// change x_c += v of an iteration is logged by the scatter that makes it, and
// r -= A_{:,c} v is applied through a column-major (CSC) copy of A.  This
// file builds that copy and the log at the first incremental solve of a
// handle:
//   csc_ptr [n+1], csc_row [nnz]  rows of each column, ascending
//   csc_val [nnz], csc_val32      FP64 values and their FP32 rounding (the
//                                 mixed-precision inner loop)
//   ilog_col, ilog_val [cap]      the change log, cap = max(2^16,
//                                 4 x the largest block's nonzeros + the
//                                 dynamic block's entry capacity): three
//                                 static updates and one dynamic update fit;
//                                 more (n_static > 3) overflow it, which only
//                                 makes that iteration's residual exact.
// The copy costs 16 bytes per nonzero plus 4 per column and is built on the
// host from the device's CSR (one transfer each way).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {

rorbk_status ensure_incremental(rorbk_ctx *h) {
    if (h->csc_ptr && h->ilog_col) return RORBK_OK;
    if (h->format != RORBK_FORMAT_CSR)
        return fail(h, RORBK_ERR_UNSUPPORTED, "the incremental residual is built for sparse (CSR) systems");
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    std::vector<int> rp(m + 1), col(nnz);
    std::vector<double> val(nnz);
    rorbk_status st;
    if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "incremental residual set-up"))) return st;
    cudaError_t e = cudaMemcpy(rp.data(), h->rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(col.data(), h->col, nnz * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(val.data(), h->val, nnz * sizeof(double), cudaMemcpyDeviceToHost);
    if ((st = cuda_check(h, e, "incremental residual set-up"))) return st;
    // counting sort of the entries by column; rows stay ascending in a column
    std::vector<int> cp(n + 1, 0), crow(nnz);
    std::vector<double> cval(nnz);
    std::vector<float> cval32(nnz);
    for (int64_t p = 0; p < nnz; ++p) ++cp[col[p] + 1];
    for (int64_t c = 0; c < n; ++c) cp[c + 1] += cp[c];
    std::vector<int> next(cp.begin(), cp.end() - 1);
    for (int64_t i = 0; i < m; ++i)
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const int q = next[col[p]]++;
            crow[q] = (int)i;
            cval[q] = val[p];
            cval32[q] = (float)val[p];
        }
    int64_t maxblk = 0;
    for (int64_t t = 0; t < h->k; ++t)
        maxblk = std::max<int64_t>(maxblk, rp[h->h_off[t + 1]] - rp[h->h_off[t]]);
    const int64_t cap = std::min<int64_t>(std::max<int64_t>(1 << 16, 4 * maxblk + h->dyn.ecap), INT32_MAX / 2);
    h->csc_ptr = (int *)dev_alloc(h, (n + 1) * sizeof(int));
    h->csc_row = (int *)dev_alloc(h, nnz * sizeof(int));
    h->csc_val = (double *)dev_alloc(h, nnz * sizeof(double));
    h->csc_val32 = (float *)dev_alloc(h, nnz * sizeof(float));
    h->ilog_col = (int *)dev_alloc(h, cap * sizeof(int));
    h->ilog_val = (double *)dev_alloc(h, cap * sizeof(double));
    if (!h->csc_ptr || !h->csc_row || !h->csc_val || !h->csc_val32 || !h->ilog_col || !h->ilog_val) {
        h->csc_ptr = nullptr;   // the allocations made stay on the handle's list
        h->ilog_col = nullptr;
        return fail(h, RORBK_ERR_OOM, "incremental residual set-up: out of device memory");
    }
    h->ilog_cap = (int)cap;
    e = cudaMemcpy(h->csc_ptr, cp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(h->csc_row, crow.data(), nnz * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(h->csc_val, cval.data(), nnz * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz) e = cudaMemcpy(h->csc_val32, cval32.data(), nnz * sizeof(float), cudaMemcpyHostToDevice);
    if ((st = cuda_check(h, e, "incremental residual set-up"))) {
        h->csc_ptr = nullptr;
        h->ilog_col = nullptr;
        return st;
    }
    return RORBK_OK;
}

}  // namespace rorbk
