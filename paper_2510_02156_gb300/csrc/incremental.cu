// incremental.cu -- set-up of the incremental residual.
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
// device (build_csc: a counting placement and merge rounds per column).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {
namespace {

// The largest number of nonzeros in one block of the partition.
__global__ void k_max_block_nnz(const int *__restrict__ rowptr, const int *__restrict__ off, int k,
                                int *__restrict__ out) {
    int v = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x)
        v = max(v, rowptr[off[t + 1]] - rowptr[off[t]]);
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

}  // namespace

rorbk_status ensure_incremental(rorbk_ctx *h) {
    const int version = h->values_version ? *h->values_version : 0;
    if (h->csc_ptr && h->ilog_col) {
        if (h->csc_version == version) return RORBK_OK;
        // the shared set-up took new values since this copy was formed
        rorbk_status st = build_csc(h, nullptr, h->csc_ptr, h->csc_row, h->csc_val, h->csc_val32);
        if (!st) h->csc_version = version;
        return st;
    }
    if (h->format != RORBK_FORMAT_CSR)
        return fail(h, RORBK_ERR_UNSUPPORTED, "the incremental residual is built for sparse (CSR) systems");
    const int64_t n = h->n, nnz = h->nnz;
    rorbk_status st;
    cudaStream_t s = h->stream;
    if ((st = cuda_check(h, cudaStreamSynchronize(s), "incremental residual set-up"))) return st;
    int *dmax = nullptr;
    if ((st = cuda_check(h, cudaMalloc(&dmax, sizeof(int)), "incremental residual set-up"))) return st;
    cudaMemsetAsync(dmax, 0, sizeof(int), s);
    k_max_block_nnz<<<std::max(1, std::min(h->num_sms, (h->k + 255) / 256)), 256, 0, s>>>(
        h->rowptr, h->off, h->k, dmax);
    int maxblk = 0;
    st = cuda_check(h, cudaMemcpyAsync(&maxblk, dmax, sizeof(int), cudaMemcpyDeviceToHost, s),
                    "incremental residual set-up");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "incremental residual set-up");
    cudaFree(dmax);
    if (st) return st;
    const int64_t cap = std::min<int64_t>(std::max<int64_t>(1 << 16, 4LL * maxblk + h->dyn.ecap), INT32_MAX / 2);
    int *cp = (int *)dev_alloc(h, (n + 1) * sizeof(int));
    int *crow = (int *)dev_alloc(h, std::max<int64_t>(1, nnz) * sizeof(int));
    double *cval = (double *)dev_alloc(h, std::max<int64_t>(1, nnz) * sizeof(double));
    float *cval32 = (float *)dev_alloc(h, std::max<int64_t>(1, nnz) * sizeof(float));
    int *lcol = (int *)dev_alloc(h, cap * sizeof(int));
    double *lval = (double *)dev_alloc(h, cap * sizeof(double));
    if (!cp || !crow || !cval || !cval32 || !lcol || !lval)   // the allocations made stay on the handle's list
        return fail(h, RORBK_ERR_OOM, "incremental residual set-up: out of device memory");
    if ((st = build_csc(h, nullptr, cp, crow, cval, cval32))) return st;
    h->csc_ptr = cp;
    h->csc_row = crow;
    h->csc_val = cval;
    h->csc_val32 = cval32;
    h->ilog_col = lcol;
    h->ilog_val = lval;
    h->ilog_cap = (int)cap;
    h->csc_version = version;
    return RORBK_OK;
}

}  // namespace rorbk
