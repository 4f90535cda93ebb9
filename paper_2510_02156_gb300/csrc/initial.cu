// initial.cu -- the initial solution of Algorithm 2 (Appendix).
//
// x0 = (<b, b~> / ||b~||^2) y with y the sum of a set of rows of A and
// b~ = A y: x0 lies in range(A^T) and ||b - A x0|| <= ||b|| (the Remark after
// Algorithm 2).  The set is the rows of one static block t: its column-sorted
// copy gives every column's entries in ascending row order, so y_c is one
// chain of additions over the block's rows, the order of the definition.
// b~ comes from the residual kernel (b~ = -(0 - A y), each row one fused
// chain in stored order); the two inner products are block partial sums
// added by the last block in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {
namespace {

// y_c = sum of A's entries in column c over block t's rows (ascending).
__global__ void k_init_rowsum(const int *__restrict__ rowptr, const int *__restrict__ off,
                              const int *__restrict__ bt_col, const double *__restrict__ bt_val,
                              const int *__restrict__ bt_seg, const int *__restrict__ nseg, int t,
                              double *__restrict__ y) {
    const int p0 = rowptr[off[t]], pend = rowptr[off[t + 1]];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nseg[t]; g += gridDim.x * blockDim.x) {
        int q = bt_seg[p0 + g];
        const int c = bt_col[q];
        double s = 0.0;
        for (; q < pend && bt_col[q] == c; ++q) s = __dadd_rn(s, bt_val[q]);
        y[c] = s;
    }
}

// <b, b~> and ||b~||^2 with b~ = -r; the last block forms alpha = <b,b~>/||b~||^2
// (NaN when ||b~|| = 0) in out[0] and ||b~||^2 in out[1].
__global__ void __launch_bounds__(256) k_init_dots(const double *__restrict__ b,
                                                   const double *__restrict__ r, int m,
                                                   double *partials, unsigned *ticket,
                                                   double *out) {
    __shared__ double red[32];
    __shared__ int is_last;
    double bb = 0.0, tt = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double v = -r[i];
        bb = __fma_rn(b[i], v, bb);
        tt = __fma_rn(v, v, tt);
    }
    bb = block_sum(bb, red);
    tt = block_sum(tt, red);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = bb;
        partials[2 * blockIdx.x + 1] = tt;
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double sb = 0.0, st = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
        sb += partials[2 * q];
        st += partials[2 * q + 1];
    }
    sb = block_sum(sb, red);
    st = block_sum(st, red);
    if (threadIdx.x == 0) {
        out[0] = st > 0.0 ? sb / st : __longlong_as_double(0x7ff8000000000000LL);
        out[1] = st;
        *ticket = 0u;
    }
}

__global__ void k_init_scale(const double *__restrict__ alpha, const double *__restrict__ y,
                             double *__restrict__ x0, int n) {
    const double a = *alpha;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        x0[c] = __dmul_rn(a, y[c]);
}

}  // namespace
}  // namespace rorbk

extern "C" rorbk_status rorbk_initial_solution(rorbk_handle h, int64_t block, const double *b,
                                               double *x0) {
    using namespace rorbk;
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!b || !x0 || block < 0 || block >= h->k)
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_initial_solution: null pointer or block out of range");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    const int m = (int)h->m, n = (int)h->n;
    double *y = h->xb;                    // workspace: y, then 0 in bb, b~ via r
    cudaMemsetAsync(y, 0, (size_t)n * sizeof(double), s);
    cudaMemsetAsync(h->bb, 0, (size_t)m * sizeof(double), s);
    const int gs = std::max(1, std::min(4 * h->num_sms, (n + 255) / 256));
    k_init_rowsum<<<gs, 256, 0, s>>>(h->rowptr, h->off, h->bt.col, h->bt.val, h->bt.seg,
                                      h->bt.seg_ptr, (int)block, y);
    launch_residual_only(h, h->bb, y, h->r);
    const int gd = std::max(1, std::min(2 * h->num_sms, (m + 255) / 256));
    double *out = h->partials + 2 * gd;   // after the block partials
    k_init_dots<<<gd, 256, 0, s>>>(b, h->r, m, h->partials, &h->ctl->ticket, out);
    k_init_scale<<<gs, 256, 0, s>>>(out, y, x0, n);
    double res[2] = {0.0, 0.0};
    rorbk_status st = cuda_check(h, cudaGetLastError(), "rorbk_initial_solution");
    if (!st) st = cuda_check(h, cudaMemcpyAsync(res, out, sizeof(res), cudaMemcpyDeviceToHost, s),
                             "rorbk_initial_solution");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_initial_solution");
    cudaSetDevice(cur);
    if (st) return st;
    if (!(res[1] > 0.0))
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_initial_solution: A y = 0 for this block's row sum");
    return RORBK_OK;
}
