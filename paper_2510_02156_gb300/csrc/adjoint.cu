// adjoint.cu -- what the differentiable solve needs beyond Algorithm 1.
//
// The paper solves A x = b and never differentiates the solution.  For a
// square, non-singular A and a loss L(x), x = A^{-1} b gives
//     dL/db = g,   where A^T g = dL/dx   (the adjoint system),
//     dL/dA = -g x^T,
// and for a sparse A only the stored entries are parameters, so the gradient
// with respect to the stored value a_ij is -g_i x_j.  The adjoint system is
// solved by ROR-BK itself: rorbk_setup_adjoint builds a handle from a
// handle's own copy of A, rorbk_adjoint_solve solves the adjoint system on it,
// and rorbk_value_grad evaluates -g_i x_j over A's stored pattern.
//
// Column equilibration.  Kaczmarz-type methods are invariant to scaling the
// rows of a system but not its columns, and A's row scaling becomes a column
// scaling of A^T: a system whose rows span four decades gives an adjoint on
// which ROR-BK stalls.  The adjoint handle therefore holds
//     At~ = A^T C^{-1},   C = diag(c_i),  c_i = ||A_i||_2  (1 for a zero row),
// the transpose of A with its rows normalised, and rorbk_adjoint_solve solves
// At~ h = y and returns g = C^{-1} h.  Since At~ h = A^T g, the residual that
// the solve tests is the adjoint system's own residual; the iterate is a
// diagonal change of variables, so the solution is unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {
namespace {

// c_i = ||A_i||_2 from ||A_i||^2 (1 for a zero row).
__global__ void k_row_scale(const double *__restrict__ rn, int m, double *__restrict__ c) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        c[i] = rn[i] > 0.0 ? __dsqrt_rn(rn[i]) : 1.0;
}

// g_i = h_i / c_i (the adjoint solution from the equilibrated iterate).
__global__ void k_unscale(double *__restrict__ g, const double *__restrict__ c, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        g[i] = __ddiv_rn(g[i], c[i]);
}

// dvals[p] = -(g_i x_j) for every stored entry p = (i, j) of A, in A's CSR
// order.  One thread per row.
__global__ void k_value_grad(const int *__restrict__ rowptr, const int *__restrict__ col, int m,
                             const double *__restrict__ g, const double *__restrict__ x,
                             double *__restrict__ dvals) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double gi = g[i];
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) dvals[p] = -__dmul_rn(gi, x[col[p]]);
    }
}

}  // namespace
}  // namespace rorbk

extern "C" rorbk_status rorbk_setup_adjoint(rorbk_handle h, const rorbk_partition *part,
                                            double lambda, const rorbk_options *opt,
                                            rorbk_handle *out) {
    using namespace rorbk;
    if (!out) return RORBK_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h || !part) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_setup_adjoint: null handle or partition");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    rorbk_status st;
    cudaStream_t s = h->stream;
    // At~ on the device: c_i = ||A_i||_2 from the row norms of the set-up (each
    // a fused chain over the row in stored order), then the column-major copy
    // of A with a_ij / c_i: row j of At~ lists the rows i of A that hold
    // column j, ascending.
    int *tp = nullptr, *tcol = nullptr;
    double *t64 = nullptr, *c = nullptr;
    cudaError_t e = cudaMalloc(&tp, (n + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&tcol, std::max<int64_t>(1, nnz) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&t64, std::max<int64_t>(1, nnz) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c, m * sizeof(double));
    auto release = [&]() {
        cudaStreamSynchronize(s);
        cudaFree(tp);
        cudaFree(tcol);
        cudaFree(t64);
        cudaFree(c);
        cudaSetDevice(cur);
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(h, RORBK_ERR_OOM, "rorbk_setup_adjoint: copy of A");
    }
    k_row_scale<<<std::max(1, std::min(8 * h->num_sms, (int)((m + 255) / 256))), 256, 0, s>>>(h->rn, (int)m, c);
    if ((st = build_csc(h, c, tp, tcol, t64, nullptr))) { release(); return st; }
    rorbk_matrix At;
    At.format = RORBK_FORMAT_CSR;
    At.dtype = RORBK_F64;
    At.m = n;
    At.n = m;
    At.nnz = nnz;
    At.row_ptr = tp;
    At.col_idx = tcol;
    At.values = t64;
    At.ld = 0;
    At.on_device = 1;
    At.reserved_ = 0;
    rorbk_options o;
    rorbk_default_options(&o);
    if (opt) o = *opt;
    else o.stream = (void *)h->stream;
    st = rorbk_setup(&At, part, lambda, &o, out);
    if (st == RORBK_OK) {
        rorbk_ctx *a = *out;
        a->adj_scale = (double *)dev_alloc(a, (size_t)m * sizeof(double));
        cudaError_t e2 = a->adj_scale ? cudaMemcpy(a->adj_scale, c, m * sizeof(double), cudaMemcpyDeviceToDevice)
                                      : cudaErrorMemoryAllocation;
        if (e2 != cudaSuccess) {
            st = a->adj_scale ? cuda_check(a, e2, "rorbk_setup_adjoint: scale")
                              : fail(a, RORBK_ERR_OOM, "rorbk_setup_adjoint: scale");
            record_setup_error(a->err);
            rorbk_free(a);
            *out = nullptr;
        }
    }
    release();
    return st;
}

extern "C" rorbk_status rorbk_adjoint_solve(rorbk_handle adj, const double *y, double *g,
                                            double tol, int64_t maxit, const rorbk_options *opt,
                                            rorbk_result *res) {
    using namespace rorbk;
    if (!adj) return RORBK_ERR_INVALID_ARG;
    if (!adj->adj_scale)
        return fail(adj, RORBK_ERR_INVALID_ARG,
                    "rorbk_adjoint_solve: the handle was not made by rorbk_setup_adjoint");
    rorbk_status st = rorbk_solve(adj, y, nullptr, g, tol, maxit, opt, res);
    if (st < 0) return st;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(adj->device);
    cudaStream_t s = (opt && opt->stream) ? (cudaStream_t)opt->stream : adj->stream;
    const int m = (int)adj->m;
    const int grid = std::max(1, std::min(4 * adj->num_sms, (m + 255) / 256));
    k_unscale<<<grid, 256, 0, s>>>(g, adj->adj_scale, m);
    rorbk_status st2 = cuda_check(adj, cudaGetLastError(), "rorbk_adjoint_solve");
    if (st2 == RORBK_OK) st2 = cuda_check(adj, cudaStreamSynchronize(s), "rorbk_adjoint_solve");
    cudaSetDevice(cur);
    return st2 != RORBK_OK ? st2 : st;
}

extern "C" rorbk_status rorbk_value_grad(rorbk_handle h, const double *g, const double *x,
                                         double *dvals) {
    using namespace rorbk;
    if (!h || !g || !x || (!dvals && h->nnz > 0))
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_value_grad: null pointer");
    if (h->nnz == 0) return RORBK_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    const int m = (int)h->m;
    const int grid = std::max(1, std::min(4 * h->num_sms, (m + 255) / 256));
    k_value_grad<<<grid, 256, 0, h->stream>>>(h->rowptr, h->col, m, g, x, dvals);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "rorbk_value_grad");
    cudaSetDevice(cur);
    return st;
}
