// fabgmres.cu -- Algorithm 3 (Appendix): flexible AB-GMRES with ROR-BK as the
// right preconditioner.
//
// x = x0, r0 = b - A x, beta = ||r0||, v_1 = r0 / beta.  Outer step j:
// z_j = ROR-BK on A z = v_j from z = 0 until ||v_j - A z|| <= eta ||v_j|| or
// lmax iterations (rorbk_solve on this handle; the Philox counter runs on
// across the inner solves); w = A z_j; modified Gram-Schmidt against
// v_1..v_j; h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; Givens rotations keep
// min ||beta e1 - H y|| triangular and |g_{j+1}| is its residual norm.  Stops
// when |g_{j+1}| <= tol ||b||, at breakdown or after maxit outer steps; then
// y from the triangle and x += Z y.  Inner products are block partial sums
// added by the last block in a fixed order; the small Hessenberg work runs in
// one thread; the host only reads the residual estimate between outer steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {
namespace {

constexpr int kFgBlocks = 256;

// out = <a, b> (one fused chain per thread, block sums, the last block adds
// the block partials in order).
__global__ void __launch_bounds__(256) k_fg_dot(const double *__restrict__ a,
                                                const double *__restrict__ b, int m,
                                                double *partials, unsigned *ticket, double *out) {
    __shared__ double red[32];
    __shared__ int is_last;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        s = __fma_rn(a[i], b[i], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double t = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) t += partials[q];
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
        *out = t;
        *ticket = 0u;
    }
}

__global__ void k_fg_axpy(double *__restrict__ w, const double *__restrict__ v,
                          const double *__restrict__ h, int m) {
    const double c = -*h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        w[i] = __fma_rn(c, v[i], w[i]);
}

// dst = src / sqrt(*sq) (a normalisation; sq is a squared norm), when > 0.
__global__ void k_fg_normalise(double *__restrict__ dst, const double *__restrict__ src,
                               const double *__restrict__ sq, int m) {
    const double d = sqrt(*sq);
    if (!(d > 0.0)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        dst[i] = __ddiv_rn(src[i], d);
}

__global__ void k_fg_neg(double *__restrict__ w, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        w[i] = -w[i];
}

// Column j of H: h_ij (i <= j) in hcol[0..j], ||w||^2 in *hsq.  Stores it,
// applies the earlier rotations, forms rotation j, updates g; est = |g_{j+1}|.
__global__ void k_fg_givens(double *H, int ld, double *cs, double *sn, double *g, int j,
                            const double *__restrict__ hcol, const double *__restrict__ hsq,
                            double bnorm, double *est) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int i = 0; i <= j; ++i) H[i * ld + j] = hcol[i];
    const double hn = sqrt(*hsq);
    H[(j + 1) * ld + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double a0 = H[i * ld + j], a1 = H[(i + 1) * ld + j];
        H[i * ld + j] = __dadd_rn(__dmul_rn(cs[i], a0), __dmul_rn(sn[i], a1));
        H[(i + 1) * ld + j] = __dadd_rn(__dmul_rn(-sn[i], a0), __dmul_rn(cs[i], a1));
    }
    const double a0 = H[j * ld + j], a1 = H[(j + 1) * ld + j];
    const double d = sqrt(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)));
    cs[j] = __ddiv_rn(a0, d);
    sn[j] = __ddiv_rn(a1, d);
    H[j * ld + j] = d;
    H[(j + 1) * ld + j] = 0.0;
    g[j + 1] = __dmul_rn(-sn[j], g[j]);
    g[j] = __dmul_rn(cs[j], g[j]);
    est[0] = __ddiv_rn(fabs(g[j + 1]), bnorm);
    est[1] = hn;
}

__global__ void k_fg_triangle(const double *H, int ld, const double *g, double *y, int J) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int i = J - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < J; ++l) s = __fma_rn(-H[i * ld + l], y[l], s);
        y[i] = __ddiv_rn(s, H[i * ld + i]);
    }
}

__global__ void k_fg_combine(double *__restrict__ x, const double *__restrict__ Z,
                             const double *__restrict__ y, int J, int n) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double u = 0.0;
        for (int j = 0; j < J; ++j) u = __fma_rn(y[j], Z[(long long)j * n + c], u);
        x[c] = __dadd_rn(x[c], u);
    }
}

struct DevBuf {
    std::vector<void *> p;
    ~DevBuf() { for (void *q : p) cudaFree(q); }
    template <typename T>
    T *get(size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return (T *)q;
    }
};

}  // namespace
}  // namespace rorbk

extern "C" rorbk_status rorbk_fabgmres(rorbk_handle h, const double *b, const double *x0, double *x,
                                       double tol, int64_t maxit, double eta, int64_t lmax,
                                       const rorbk_options *opt_in, rorbk_result *res) {
    using namespace rorbk;
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!b || !x || maxit < 1 || maxit > 4096 || lmax < 0 || !(eta >= 0) || !(tol >= 0))
        return fail(h, RORBK_ERR_INVALID_ARG,
                    "rorbk_fabgmres: b, x, 1 <= maxit <= 4096, lmax >= 0, eta >= 0, tol >= 0");
    rorbk_options opt;
    rorbk_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.host_loop || opt.trace || opt.dist_mode != RORBK_DIST_PAPER)
        return fail(h, RORBK_ERR_UNSUPPORTED, "rorbk_fabgmres: graph-launched inner solves, paper draws, no trace");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaStream_t s = opt.stream ? (cudaStream_t)opt.stream : h->stream;
    opt.stream = (void *)s;
    const cudaStream_t saved_stream = h->stream;
    h->stream = s;                                // every launch of this call on s
    const int m = (int)h->m, n = (int)h->n, M = (int)maxit;
    DevBuf buf;
    double *V = buf.get<double>((size_t)(M + 1) * m);
    double *Z = buf.get<double>((size_t)M * n);
    double *W = buf.get<double>(m);
    double *zero = buf.get<double>(m);
    double *H = buf.get<double>((size_t)(M + 1) * M);
    double *cs = buf.get<double>(M), *sn = buf.get<double>(M), *g = buf.get<double>(M + 1);
    double *y = buf.get<double>(M), *hcol = buf.get<double>(M + 1);
    double *sc = buf.get<double>(8);              // bnorm^2, beta^2, ||w||^2, est, hn
    double *partials = buf.get<double>(kFgBlocks);
    unsigned *ticket = buf.get<unsigned>(1);
    auto done = [&](rorbk_status st) {
        h->stream = saved_stream;
        cudaSetDevice(cur);
        return st;
    };
    if (!V || !Z || !W || !zero || !H || !cs || !sn || !g || !y || !hcol || !sc || !partials || !ticket)
        return done(fail(h, RORBK_ERR_OOM, "rorbk_fabgmres: Krylov basis"));
    cudaMemsetAsync(zero, 0, (size_t)m * sizeof(double), s);
    cudaMemsetAsync(H, 0, (size_t)(M + 1) * M * sizeof(double), s);
    cudaMemsetAsync(g, 0, (size_t)(M + 1) * sizeof(double), s);
    cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
    if (x0) cudaMemcpyAsync(x, x0, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), s);
    const int gv = std::max(1, std::min(4 * h->num_sms, (std::max(m, n) + 255) / 256));
    const int gd = std::max(1, std::min(kFgBlocks, (m + 255) / 256));
    auto dot = [&](const double *a, const double *bb, double *out) {
        k_fg_dot<<<gd, 256, 0, s>>>(a, bb, m, partials, ticket, out);
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    dot(b, b, sc + 0);
    launch_residual_only(h, b, x, W);             // r0 = b - A x0
    dot(W, W, sc + 1);
    k_fg_normalise<<<gv, 256, 0, s>>>(V, W, sc + 1, m);
    double host_sc[2] = {0.0, 0.0};
    rorbk_status st = cuda_check(h, cudaMemcpyAsync(host_sc, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "rorbk_fabgmres");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_fabgmres");
    if (st) return done(st);
    const double bnorm = sqrt(host_sc[0]), beta = sqrt(host_sc[1]);
    int64_t inner = 0;
    int J = 0;
    double est = 0.0, inner_res = 0.0;
    rorbk_status inner_st = RORBK_OK;
    if (bnorm > 0.0 && beta > 0.0) {
        cudaMemcpyAsync(g, &beta, sizeof(double), cudaMemcpyHostToDevice, s);
        for (int j = 0; j < M; ++j) {
            rorbk_options oi = opt;
            oi.start_iter = opt.start_iter + inner;
            rorbk_result ri;
            const rorbk_status si = rorbk_solve(h, V + (size_t)j * m, nullptr, Z + (size_t)j * n, eta,
                                                lmax, &oi, &ri);
            if (si < 0) return done(si);
            if (si == RORBK_NOT_CONVERGED) inner_st = si;
            inner += ri.iters;
            launch_residual_only(h, zero, Z + (size_t)j * n, W);   // W = -A z_j
            k_fg_neg<<<gv, 256, 0, s>>>(W, m);
            for (int i = 0; i <= j; ++i) {
                dot(W, V + (size_t)i * m, hcol + i);
                k_fg_axpy<<<gv, 256, 0, s>>>(W, V + (size_t)i * m, hcol + i, m);
            }
            dot(W, W, sc + 2);
            k_fg_normalise<<<gv, 256, 0, s>>>(V + (size_t)(j + 1) * m, W, sc + 2, m);
            k_fg_givens<<<1, 1, 0, s>>>(H, M, cs, sn, g, j, hcol, sc + 2, bnorm, sc + 3);
            double e2[2];
            st = cuda_check(h, cudaMemcpyAsync(e2, sc + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "rorbk_fabgmres");
            if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_fabgmres");
            if (st) return done(st);
            J = j + 1;
            est = e2[0];
            if (est <= tol || !(e2[1] > 0.0)) break;
        }
        k_fg_triangle<<<1, 1, 0, s>>>(H, M, g, y, J);
        k_fg_combine<<<gv, 256, 0, s>>>(x, Z, y, J, n);
    }
    launch_residual_only(h, b, x, W);
    dot(W, W, sc + 4);
    cudaEventRecord(e1, s);
    double rr = 0.0;
    st = cuda_check(h, cudaMemcpyAsync(&rr, sc + 4, sizeof(double), cudaMemcpyDeviceToHost, s), "rorbk_fabgmres");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_fabgmres");
    float ms = 0.f;
    if (!st) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return done(st);
    inner_res = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    const bool conv = inner_res <= tol;
    if (res) {
        res->iters = J;
        res->refinements = inner;
        res->rrn = inner_res;
        res->converged = conv;
        res->status = conv ? RORBK_OK : RORBK_NOT_CONVERGED;
        res->time_ms = ms;
    }
    (void)est;
    (void)inner_st;
    return done(conv ? RORBK_OK : RORBK_NOT_CONVERGED);
}
