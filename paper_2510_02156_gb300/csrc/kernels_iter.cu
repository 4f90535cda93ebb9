// kernels_iter.cu -- the ROR-BK iteration (Algorithm 1's loop body).
//
//   k_begin        ||b||, x0, loop state; sets the loop condition
//   k_static       l = 1..n_static: draw tau (Philox), r_tau = b_tau - A_tau x,
//                  y = W_tau r_tau, x += A_tau^T y   (one block of threads)
//   k_residual     r = b - A x over nnz-balanced row tiles, ||r||^2, the
//                  convergence test, and the first radix histogram of |r|
//   k_topk_hist2   second 11-bit radix histogram inside the selected bin
//   k_topk_collect the rows above the 22-bit threshold and the candidates on it
//   k_dynamic      exact top-K, G = A_I A_I^T + mu I on the coupled rows,
//                  Cholesky, two triangular solves, x += A_I^T y; ends the
//                  iteration and sets the loop condition
//
// Compute type T is double (the plain method) or float (the inner solve of
// the mixed-precision form).  In FP64 every product and sum uses the
// non-contracted __dmul_rn/__dadd_rn in the order of the oracle's
// definitions (row dots in stored order; A^T y per column over ascending rows;
// Gram entries over ascending columns; column-oriented triangular solves), so
// the iterates reproduce the FP64 definition exactly.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {

template <typename T> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
};

// Matrix and operator pointers for one compute type.
template <typename T>
struct Mat {
    const int *rowptr, *col;
    const T *val;
    const int *off;
    const double *cdf;
    int m, n, k, K;
    // static operators
    const int *s_ptr;
    const uint16_t *s_idx;
    const long long *w_ptr;
    const T *w_ss, *w_diag;
    const int *s_pos;
    // block transpose
    const int *bt_col;
    const uint16_t *bt_row;
    const T *bt_val;
    const int *bt_seg, *nseg;
    // residual tiles
    const int *tile_row0;
    int ntiles;
    double mu;
    const float *val32;         // FP32-stored values, when the system is FP32
};

template <typename T>
Mat<T> make_mat(rorbk_ctx *h);
template <>
Mat<double> make_mat<double>(rorbk_ctx *h) {
    return Mat<double>{h->rowptr, h->col, h->val, h->off, h->cdf, (int)h->m, (int)h->n, h->k, h->K,
                       h->ops.s_ptr, h->ops.s_idx, h->ops.w_ptr, h->ops.w_ss, h->ops.w_diag,
                       h->ops.s_pos, h->bt.col, h->bt.row, h->bt.val, h->bt.seg, h->bt.seg_ptr,
                       h->tile_row0, h->ntiles, h->mu, h->val32};
}
template <>
Mat<float> make_mat<float>(rorbk_ctx *h) {
    return Mat<float>{h->rowptr, h->col, h->val32, h->off, h->cdf, (int)h->m, (int)h->n, h->k, h->K,
                      h->ops.s_ptr, h->ops.s_idx, h->ops.w_ptr, h->ops.w_ss32, h->ops.w_diag32,
                      h->ops.s_pos, h->bt.col, h->bt.row, h->bt.val32, h->bt.seg, h->bt.seg_ptr,
                      h->tile_row0, h->ntiles, h->mu, h->val32};
}

// ------------------------------------------------------------------ begin
// ||b|| (deterministic: fixed grid, fixed trees), x = x0 or 0, loop state.
// Launched with one block; sets the WHILE condition to (||b|| > 0 && maxit > 0).
__global__ void k_begin(const double *__restrict__ b, int m, const double *__restrict__ x0,
                        double *__restrict__ x, int n, Ctl *ctl, int use_cond,
                        cudaGraphConditionalHandle hcond) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += b[i] * b[i];
    s = block_sum(s, red);
    __shared__ double bn;
    if (threadIdx.x == 0) bn = sqrt(s);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x)
        x[c] = (bn == 0.0 || x0 == nullptr || !ctl->has_x0) ? 0.0 : x0[c];
    if (threadIdx.x == 0) {
        ctl->bnorm = bn;
        ctl->iter = 0;
        ctl->rr = 0.0;
        ctl->rrn = bn == 0.0 ? 0.0 : 1.0;
        ctl->done = bn == 0.0;
        ctl->status = 0;
        ctl->ticket = 0;
        ctl->n_in = 0;
        ctl->n_eq = 0;
        if (use_cond) cudaGraphSetConditional(hcond, (bn > 0.0 && ctl->maxit > 0) ? 1u : 0u);
    }
}

// ----------------------------------------------------------------- static
// One block of threads runs the n_static sampled updates of an iteration in
// sequence (Algorithm 1, the inner loop over l).  force_tau >= 0 replaces the
// draw by that block (single-step API).  Uses the stored W_tau (Section 3.1).
template <typename T>
__global__ void __launch_bounds__(1024) k_static(Mat<T> A, const T *__restrict__ b, T *x,
                                                 Ctl *ctl, int force_tau) {
    __shared__ T rloc[kMaxBlockRows];
    __shared__ T y[kMaxBlockRows];
    __shared__ int tau_s;
    if (force_tau < 0 && ctl->done) return;
    const long long it = ctl->iter_base + ctl->iter;
    const int nst = force_tau >= 0 ? 1 : ctl->n_static;
    for (int l = 0; l < nst; ++l) {
        if (threadIdx.x == 0) {
            int tau = force_tau >= 0 ? force_tau
                                     : sample_block(A.cdf, A.k, ctl->seed, ctl->sysid,
                                                    (uint64_t)it, (uint64_t)l);
            tau_s = tau;
            if (force_tau < 0 && ctl->tr_tau && ctl->iter < ctl->trace_cap)
                ctl->tr_tau[ctl->iter * nst + l] = tau;
        }
        __syncthreads();
        const int tau = tau_s;
        const int r0 = A.off[tau], s = A.off[tau + 1] - r0;
        for (int a = threadIdx.x; a < s; a += blockDim.x) {
            const int i = r0 + a;
            T acc = T(0);
            for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
                acc = Ar<T>::add(acc, Ar<T>::mul(A.val[p], x[A.col[p]]));
            rloc[a] = Ar<T>::sub(b[i], acc);
        }
        __syncthreads();
        const int sb = A.s_ptr[tau], nS = A.s_ptr[tau + 1] - sb;
        const T *W = A.w_ss + A.w_ptr[tau];
        for (int a = threadIdx.x; a < s; a += blockDim.x) {
            const int i = r0 + a;
            const int pos = A.s_pos[i];
            if (pos < 0) {
                y[a] = Ar<T>::mul(A.w_diag[i], rloc[a]);
            } else {
                const T *Wr = W + (long long)pos * nS;
                T acc = T(0);
                for (int q = 0; q < nS; ++q)
                    acc = Ar<T>::add(acc, Ar<T>::mul(Wr[q], rloc[A.s_idx[sb + q]]));
                y[a] = acc;
            }
        }
        __syncthreads();
        const int p0 = A.rowptr[r0], pend = A.rowptr[r0 + s];
        const int ns = A.nseg[tau];
        for (int g = threadIdx.x; g < ns; g += blockDim.x) {
            int q = A.bt_seg[p0 + g];
            const int c = A.bt_col[q];
            T acc = T(0);
            for (; q < pend && A.bt_col[q] == c; ++q)
                acc = Ar<T>::add(acc, Ar<T>::mul(A.bt_val[q], y[A.bt_row[q]]));
            x[c] = Ar<T>::add(x[c], acc);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- residual
// Select the radix bin holding the need-th largest key: the largest bin b with
// sum_{j >= b} h[j] >= need.  One block; h in global memory.  Returns b and
// the count strictly above it; zeroes h.
__device__ void select_bin(unsigned *h, int need, int *bin_out, int *above_out) {
    __shared__ int sc[33];
    __shared__ int res_bin, res_above;
    // suffix sums through an exclusive scan of the reversed histogram
    const int per = kHistBins / blockDim.x;     // blockDim divides kHistBins
    int base = kHistBins - 1 - threadIdx.x * per;
    int cnt[8];
    int tot = 0;
    for (int u = 0; u < per; ++u) { cnt[u] = (int)h[base - u]; tot += cnt[u]; }
    int total;
    int pre = block_exclusive_scan(tot, sc, &total);   // keys in bins above this chunk
    if (threadIdx.x == 0) { res_bin = 0; res_above = 0; }
    __syncthreads();
    int run = pre;
    for (int u = 0; u < per; ++u) {
        if (run < need && run + cnt[u] >= need) { res_bin = base - u; res_above = run; }
        run += cnt[u];
    }
    __syncthreads();
    for (int u = 0; u < per; ++u) h[base - u] = 0u;
    *bin_out = res_bin;
    *above_out = res_above;
}

// r = b - A x for the tiles of rows [tile_row0[t], tile_row0[t+1]).  Tiles
// hold at most kTileNnz nonzeros (or a single longer row).  Products go to
// shared memory and each row is summed in stored order by one thread.
// finalize: 1 = convergence test + first radix level (iteration), 2 = ||r||^2
// only (single-step API).
template <typename V, typename T>
__device__ __forceinline__ const V *stored_values(const Mat<T> &A);
template <>
__device__ __forceinline__ const double *stored_values<double, double>(const Mat<double> &A) { return A.val; }
template <>
__device__ __forceinline__ const float *stored_values<float, double>(const Mat<double> &A) { return A.val32; }
template <>
__device__ __forceinline__ const float *stored_values<float, float>(const Mat<float> &A) { return A.val; }

// V is the stored value type (an FP32-stored system is read as FP32 and
// widened exactly in registers).
template <typename T, typename V>
__global__ void __launch_bounds__(256) k_residual(Mat<T> A, const T *__restrict__ b,
                                                  const T *__restrict__ x, T *__restrict__ r,
                                                  double *partials, unsigned *hist1, Ctl *ctl,
                                                  int finalize) {
    __shared__ T prod[kTileNnz];
    __shared__ unsigned hist[kHistBins];
    __shared__ double red[32];
    __shared__ int is_last;
    if (finalize == 1 && ctl->done) return;
    const V *__restrict__ val = stored_values<V, T>(A);
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    double rr = 0.0;
    __syncthreads();
    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const int row0 = A.tile_row0[t], row1 = A.tile_row0[t + 1];
        const int p0 = A.rowptr[row0], p1 = A.rowptr[row1];
        if (p1 - p0 <= kTileNnz) {
            for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x)
                prod[p - p0] = Ar<T>::mul((T)val[p], x[A.col[p]]);
            __syncthreads();
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                const int q1 = A.rowptr[i + 1] - p0;
                T s = T(0);
                for (int q = A.rowptr[i] - p0; q < q1; ++q) s = Ar<T>::add(s, prod[q]);
                const T ri = Ar<T>::sub(b[i], s);
                r[i] = ri;
                rr += (double)ri * (double)ri;
                atomicAdd(&hist[(unsigned)(abs_key(ri) >> 52)], 1u);
            }
            __syncthreads();
        } else {                                    // one long row, chunked
            T s = T(0);
            for (int c0 = p0; c0 < p1; c0 += kTileNnz) {
                const int c1 = min(p1, c0 + kTileNnz);
                for (int p = c0 + threadIdx.x; p < c1; p += blockDim.x)
                    prod[p - c0] = Ar<T>::mul((T)val[p], x[A.col[p]]);
                __syncthreads();
                if (threadIdx.x == 0)
                    for (int q = 0; q < c1 - c0; ++q) s = Ar<T>::add(s, prod[q]);
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const T ri = Ar<T>::sub(b[row0], s);
                r[row0] = ri;
                rr += (double)ri * (double)ri;
                atomicAdd(&hist[(unsigned)(abs_key(ri) >> 52)], 1u);
            }
        }
    }
    __syncthreads();
    if (finalize == 1)
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
            if (hist[i]) atomicAdd(&hist1[i], hist[i]);
    rr = block_sum(rr, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = rr;
        __threadfence();
        unsigned tk = atomicAdd(&ctl->ticket, 1u);
        is_last = tk == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += partials[i];
    tot = block_sum(tot, red);
    __shared__ int stop;
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->rr = tot;
        stop = 0;
        if (finalize == 1) {
            const double rrn = sqrt(tot) / ctl->bnorm;
            ctl->rrn = rrn;
            if (ctl->tr_rrn && ctl->iter < ctl->trace_cap) ctl->tr_rrn[ctl->iter] = rrn;
            if (!isfinite(rrn)) { set_status(&ctl->status, kDevNumeric); ctl->done = 1; }
            else if (rrn <= ctl->tol) ctl->done = 1;
            stop = ctl->done;
            ctl->n_in = 0;
            ctl->n_eq = 0;
        }
    }
    __syncthreads();
    if (finalize == 1) {
        int bin, above;
        if (!stop) {
            select_bin(hist1, A.K, &bin, &above);
            if (threadIdx.x == 0) { ctl->sel1 = bin; ctl->above1 = above; }
        } else {
            for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist1[i] = 0u;
        }
    }
}

// First radix level over a given r (single-step top-K).
template <typename T>
__global__ void __launch_bounds__(256) k_topk_hist1(const T *__restrict__ r, int m, int K,
                                                    unsigned *hist1, Ctl *ctl) {
    __shared__ unsigned hist[kHistBins];
    __shared__ int is_last;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        atomicAdd(&hist[(unsigned)(abs_key(r[i]) >> 52)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
        if (hist[i]) atomicAdd(&hist1[i], hist[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    int bin, above;
    select_bin(hist1, K, &bin, &above);
    if (threadIdx.x == 0) {
        ctl->sel1 = bin;
        ctl->above1 = above;
        ctl->ticket = 0;
        ctl->n_in = 0;
        ctl->n_eq = 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_topk_hist2(const T *__restrict__ r, int m, int K,
                                                    unsigned *hist2, Ctl *ctl, int check_done) {
    __shared__ unsigned hist[kHistBins];
    __shared__ int is_last;
    if (check_done && ctl->done) return;
    const unsigned sel1 = (unsigned)ctl->sel1;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        unsigned long long key = abs_key(r[i]);
        if ((unsigned)(key >> 52) == sel1) atomicAdd(&hist[(unsigned)(key >> 41) & 2047u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
        if (hist[i]) atomicAdd(&hist2[i], hist[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    int bin, above;
    select_bin(hist2, K - ctl->above1, &bin, &above);
    if (threadIdx.x == 0) {
        ctl->prefix = (int)((sel1 << 11) | (unsigned)bin);
        ctl->above = ctl->above1 + above;
        ctl->ticket = 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_topk_collect(const T *__restrict__ r, int m,
                                                      int *in_list, int *eq_list, Ctl *ctl,
                                                      int check_done) {
    if (check_done && ctl->done) return;
    const unsigned long long P = (unsigned long long)(unsigned)ctl->prefix;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        unsigned long long pre = abs_key(r[i]) >> 41;
        if (pre > P) {
            in_list[atomicAdd(&ctl->n_in, 1)] = i;
        } else if (pre == P) {
            int pos = atomicAdd(&ctl->n_eq, 1);
            if (pos < kEqCap) eq_list[pos] = i;
        }
    }
}

// ------------------------------------------------------------ exact top-K
// Completes the top-K set in one block of threads: the n_in rows above the
// 22-bit threshold plus the best (need) of the candidates on it, ordered by
// |r| descending and row ascending.  If more than kEqCap candidates share the
// threshold prefix, the block resolves the remaining 41 key bits itself by
// scanning r.  Writes I ascending to sI.  Shared scratch: keys and idx
// arrays of kEqCap entries.
template <typename T>
__device__ void finalize_topk(const T *__restrict__ r, int m, int K, const int *in_list,
                              const int *eq_list, Ctl *ctl, int *sI,
                              unsigned long long *skey, int *sidx) {
    __shared__ int sc[33];
    __shared__ int s_need, s_nin, s_neq, s_fill;
    __shared__ unsigned long long s_pref;
    __shared__ int s_shift;
    __shared__ unsigned shist[kHistBins];
    if (threadIdx.x == 0) {
        s_nin = ctl->n_in;
        s_neq = ctl->n_eq;
        s_need = K - s_nin;
    }
    __syncthreads();
    const int nin = s_nin, need = s_need, neq = s_neq;
    for (int a = threadIdx.x; a < nin; a += blockDim.x) sI[a] = in_list[a];
    if (need > 0 && neq <= kEqCap) {
        const int np = next_pow2(neq);
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            if (e < neq) { int i = eq_list[e]; skey[e] = abs_key(r[i]); sidx[e] = i; }
            else { skey[e] = 0ull; sidx[e] = 0x7fffffff; }
        }
        __syncthreads();
        block_bitonic_sort_desc(skey, sidx, np);
        for (int a = threadIdx.x; a < need; a += blockDim.x) sI[nin + a] = sidx[a];
        __syncthreads();
    } else if (need > 0) {
        // Rare: huge tie groups.  Resolve the remaining bits by radix passes
        // over all of r inside this block, then take ties by ascending row.
        if (threadIdx.x == 0) {
            s_pref = (unsigned long long)(unsigned)ctl->prefix;
            s_shift = 41;
            s_fill = nin;
        }
        __syncthreads();
        int want = need;
        while (s_shift > 0) {
            const int digit_bits = s_shift >= 11 ? 11 : s_shift;
            const int nshift = s_shift - digit_bits;
            for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) shist[i] = 0u;
            __syncthreads();
            const unsigned long long pref = s_pref;
            const int sh = s_shift;
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                unsigned long long key = abs_key(r[i]);
                if ((key >> sh) == pref)
                    atomicAdd(&shist[(unsigned)((key >> nshift) & ((1ull << digit_bits) - 1))], 1u);
            }
            __syncthreads();
            // largest digit with suffix >= want (sequential: rare path)
            __shared__ int s_dig, s_above;
            if (threadIdx.x == 0) {
                int run = 0, dig = 0, above = 0;
                for (int d = (1 << digit_bits) - 1; d >= 0; --d) {
                    if (run < want && run + (int)shist[d] >= want) { dig = d; above = run; break; }
                    run += (int)shist[d];
                }
                s_dig = dig;
                s_above = above;
            }
            __syncthreads();
            // rows strictly above the chosen digit are in
            const int dig = s_dig;
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                unsigned long long key = abs_key(r[i]);
                if ((key >> sh) == pref &&
                    (int)((key >> nshift) & ((1ull << digit_bits) - 1)) > dig)
                    sI[atomicAdd(&s_fill, 1)] = i;
            }
            want -= s_above;
            __syncthreads();
            if (threadIdx.x == 0) {
                s_pref = (pref << digit_bits) | (unsigned long long)dig;
                s_shift = nshift;
            }
            __syncthreads();
        }
        // ties: key == s_pref exactly; take the lowest rows in order
        const unsigned long long T0 = s_pref;
        int taken = 0;
        for (int base = 0; base < m && taken < want; base += blockDim.x) {
            int i = base + threadIdx.x;
            int f = (i < m && abs_key(r[i]) == T0) ? 1 : 0;
            int total;
            int pre = block_exclusive_scan(f, sc, &total);
            if (f && taken + pre < want) sI[s_fill + taken + pre] = i;
            taken += total;
        }
        __syncthreads();
    }
    __syncthreads();
    // ascending order
    const int np = next_pow2(K);
    for (int a = threadIdx.x; a < np; a += blockDim.x)
        skey[a] = a < K ? (unsigned long long)(unsigned)sI[a] : ~0ull;
    __syncthreads();
    block_bitonic_sort(skey, np);
    for (int a = threadIdx.x; a < K; a += blockDim.x) sI[a] = (int)skey[a];
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) k_topk_final(const T *__restrict__ r, int m, int K,
                                                    const int *in_list, const int *eq_list,
                                                    Ctl *ctl, int *I_out) {
    extern __shared__ unsigned long long dsm_u64[];
    unsigned long long *skey = dsm_u64;
    int *sidx = (int *)(skey + kEqCap);
    int *sI = sidx + kEqCap;
    finalize_topk<T>(r, m, K, in_list, eq_list, ctl, sI, skey, sidx);
    for (int a = threadIdx.x; a < K; a += blockDim.x) I_out[a] = sI[a];
}

// ----------------------------------------------------------------- dynamic
// Dynamic block of Algorithm 1: x += A_I^T (A_I A_I^T + mu I)^{-1} r_I with
// r_I read from the full residual.  One block of 512 threads.  The K rows'
// nonzeros are gathered (in row order) and sorted by (column, position); the
// distinct-column segments give the coupled rows S and the deterministic
// scatter.  The Gram is diagonal outside S; on S it is factored densely.
struct DynScratch {
    unsigned long long *keys;   // fallback (global) when E > kSortCapSmem
    int *ecol;
    double *eval;
    uint16_t *erow;
    double *g;                  // fallback (global) when |S| > kCholSmemMax
    long long ecap;
};

template <typename T>
__global__ void __launch_bounds__(512) k_dynamic(Mat<T> A, const T *__restrict__ r, T *x,
                                                 const int *in_list, const int *eq_list,
                                                 const int *I_given, DynScratch ds, Ctl *ctl,
                                                 int use_cond, cudaGraphConditionalHandle hcond,
                                                 int count_iter) {
    extern __shared__ unsigned long long dsm_u64[];
    __shared__ int sc[33];
    __shared__ int s_E, s_nS, s_bad;
    const int K = A.K;
    const int tid = threadIdx.x;
    // shared layout (sizes for K <= kMaxDynRows)
    unsigned long long *ukeys = dsm_u64;                                   // kSortCapSmem
    int *ucol = (int *)(ukeys + kSortCapSmem);                             // kSortCapSmem
    double *uval = (double *)(ucol + kSortCapSmem);                        // kSortCapSmem
    uint16_t *urow = (uint16_t *)(uval + kSortCapSmem);                    // kSortCapSmem
    double *gss = (double *)(urow + kSortCapSmem);                         // kCholSmemMax^2
    double *gdiag = gss + kCholSmemMax * kCholSmemMax;                     // K
    double *z = gdiag + kMaxDynRows;                                       // K
    double *y = z + kMaxDynRows;                                           // K
    int *sI = (int *)(y + kMaxDynRows);                                    // K
    int *estart = sI + kMaxDynRows;                                        // K+1
    int16_t *spos = (int16_t *)(estart + kMaxDynRows + 1);                 // K
    int16_t *sidx = spos + kMaxDynRows;                                    // K
    unsigned char *flag = (unsigned char *)(sidx + kMaxDynRows);           // K

    const bool skip = ctl->done;
    if (!skip) {
        if (I_given) {
            for (int a = tid; a < K; a += blockDim.x) sI[a] = I_given[a];
            __syncthreads();
        } else {
            finalize_topk<T>(r, A.m, K, in_list, eq_list, ctl, sI, ukeys, (int *)uval);
            if (ctl->tr_I && ctl->iter < ctl->trace_cap)
                for (int a = tid; a < K; a += blockDim.x) ctl->tr_I[ctl->iter * K + a] = sI[a];
        }
        // row extents and entry offsets
        int len = 0;
        for (int base = 0, carry = 0; base < K; base += blockDim.x) {
            int a = base + tid;
            len = a < K ? A.rowptr[sI[a] + 1] - A.rowptr[sI[a]] : 0;
            int total;
            int pre = block_exclusive_scan(len, sc, &total);
            if (a < K) { estart[a] = carry + pre; flag[a] = 0; }
            carry += total;
            if (base + (int)blockDim.x >= K && tid == 0) { estart[K] = carry; s_E = carry; }
        }
        if (tid == 0) s_bad = 0;
        __syncthreads();
        const int E = s_E;
        const bool big = E > kSortCapSmem;
        unsigned long long *keys = big ? ds.keys : ukeys;
        int *ecol = big ? ds.ecol : ucol;
        double *eval = big ? ds.eval : uval;
        uint16_t *erow = big ? ds.erow : urow;
        if (big && E > ds.ecap) { if (tid == 0) set_status(&ctl->status, kDevBounds); }
        else {
            // gather (row order), Gram diagonal, sort keys
            for (int a = tid; a < K; a += blockDim.x) {
                const int i = sI[a];
                int e = estart[a];
                double g = 0.0;
                for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p, ++e) {
                    const double v = (double)A.val[p];
                    ecol[e] = A.col[p];
                    eval[e] = v;
                    erow[e] = (uint16_t)a;
                    g = __dadd_rn(g, __dmul_rn(v, v));
                }
                gdiag[a] = __dadd_rn(g, A.mu);
            }
            const int np = next_pow2(max(E, 1));
            __syncthreads();
            for (int e = tid; e < np; e += blockDim.x)
                keys[e] = e < E ? (((unsigned long long)(unsigned)ecol[e]) << 32) | (unsigned)e : ~0ull;
            __syncthreads();
            block_bitonic_sort(keys, np);
            // coupled rows: members of a segment of length >= 2
            for (int q = tid; q < E; q += blockDim.x) {
                const unsigned c = (unsigned)(keys[q] >> 32);
                if (q > 0 && (unsigned)(keys[q - 1] >> 32) == c) {
                    flag[erow[(unsigned)keys[q]]] = 1;
                    flag[erow[(unsigned)keys[q - 1]]] = 1;
                }
            }
            __syncthreads();
            int cnt = 0;
            for (int base = 0; base < K; base += blockDim.x) {
                int a = base + tid;
                int f = a < K ? flag[a] : 0;
                int total;
                int pre = block_exclusive_scan(f, sc, &total);
                if (a < K) {
                    spos[a] = f ? (int16_t)(cnt + pre) : (int16_t)-1;
                    if (f) sidx[cnt + pre] = (int16_t)a;
                }
                cnt += total;
            }
            if (tid == 0) s_nS = cnt;
            __syncthreads();
            const int nS = s_nS;
            double *G = nS > kCholSmemMax ? ds.g : gss;
            // Gram on S (lower triangle, ascending-column merges)
            const long long pairs = (long long)nS * (nS + 1) / 2;
            for (long long idx = tid; idx < pairs; idx += blockDim.x) {
                int i = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
                while ((long long)(i + 1) * (i + 2) / 2 <= idx) ++i;
                while ((long long)i * (i + 1) / 2 > idx) --i;
                const int j = (int)(idx - (long long)i * (i + 1) / 2);
                const int a = sidx[i], bb = sidx[j];
                G[(long long)i * nS + j] =
                    i == j ? gdiag[a]
                           : row_merge_dot<double>(ecol, eval, estart[a], estart[a + 1], estart[bb],
                                                   estart[bb + 1]);
            }
            __syncthreads();
            block_cholesky(G, nS, nS, &s_bad);
            // uncoupled rows: y = (r / L_aa) / L_aa; coupled: z = r_S
            for (int a = tid; a < K; a += blockDim.x) {
                const double ra = (double)r[sI[a]];
                if (spos[a] < 0) {
                    const double l = sqrt(gdiag[a]);
                    if (!(gdiag[a] > 0.0)) s_bad = 1;
                    y[a] = (ra / l) / l;
                } else {
                    z[spos[a]] = ra;
                }
            }
            __syncthreads();
            for (int j = 0; j < nS; ++j) {                 // forward, column order
                if (tid == 0) z[j] = z[j] / G[(long long)j * nS + j];
                __syncthreads();
                const double zj = z[j];
                for (int i = j + 1 + tid; i < nS; i += blockDim.x) {
                    const double lij = G[(long long)i * nS + j];
                    if (lij != 0.0) z[i] = __dsub_rn(z[i], __dmul_rn(lij, zj));
                }
                __syncthreads();
            }
            for (int j = nS - 1; j >= 0; --j) {            // backward, column order
                if (tid == 0) z[j] = z[j] / G[(long long)j * nS + j];
                __syncthreads();
                const double zj = z[j];
                for (int i = tid; i < j; i += blockDim.x) {
                    const double lji = G[(long long)j * nS + i];
                    if (lji != 0.0) z[i] = __dsub_rn(z[i], __dmul_rn(lji, zj));
                }
                __syncthreads();
            }
            for (int q = tid; q < nS; q += blockDim.x) y[sidx[q]] = z[q];
            __syncthreads();
            // x += A_I^T y: one thread per distinct column, rows ascending
            for (int q = tid; q < E; q += blockDim.x) {
                const unsigned c = (unsigned)(keys[q] >> 32);
                if (q > 0 && (unsigned)(keys[q - 1] >> 32) == c) continue;
                T acc = T(0);
                for (int u = q; u < E && (unsigned)(keys[u] >> 32) == c; ++u) {
                    const unsigned e = (unsigned)keys[u];
                    acc = Ar<T>::add(acc, Ar<T>::mul((T)eval[e], (T)y[erow[e]]));
                }
                x[c] = Ar<T>::add(x[c], acc);
            }
            __syncthreads();
            if (tid == 0 && s_bad) set_status(&ctl->status, kDevNotSpd);
        }
    }
    if (!count_iter) return;
    // end of iteration: trace x, advance, loop condition
    if (ctl->tr_x && ctl->iter < ctl->trace_cap && sizeof(T) == sizeof(double))
        for (int c = tid; c < A.n; c += blockDim.x)
            ctl->tr_x[ctl->iter * (long long)A.n + c] = (double)x[c];
    __syncthreads();
    if (tid == 0) {
        const long long it = ctl->iter + 1;
        ctl->iter = it;
        const bool go = !ctl->done && ctl->status == 0 && it < ctl->maxit;
        if (use_cond) cudaGraphSetConditional(hcond, go ? 1u : 0u);
    }
}

// Sampler probe (single-step API).
__global__ void k_sample_probe(const double *cdf, int k, uint64_t seed, uint64_t sysid,
                               long long it, long long l, long long *out) {
    *out = sample_block(cdf, k, seed, sysid, (uint64_t)it, (uint64_t)l);
}

// ------------------------------------------------------------- launchers
static size_t dyn_smem_bytes() {
    return (size_t)kSortCapSmem * (8 + 4 + 8 + 2) + (size_t)kCholSmemMax * kCholSmemMax * 8 +
           (size_t)kMaxDynRows * (8 * 3 + 4 + 4 + 2 + 2 + 1) + 8 + 64;
}
static size_t topk_final_smem_bytes() { return (size_t)kEqCap * (8 + 4) + (size_t)kMaxDynRows * 4; }

static DynScratch dyn_scratch(rorbk_ctx *h) {
    return DynScratch{h->dyn_keys, h->dyn_ecol, h->dyn_eval, h->dyn_erow, h->dyn_g, h->dyn_ecap};
}

static int grid_stream(rorbk_ctx *h, int m) {
    return std::max(1, std::min(4 * h->num_sms, (m + 255) / 256));
}

void configure_kernels() {
    cudaFuncSetAttribute(k_dynamic<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)dyn_smem_bytes());
    cudaFuncSetAttribute(k_dynamic<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)dyn_smem_bytes());
    cudaFuncSetAttribute(k_topk_final<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)topk_final_smem_bytes());
    cudaFuncSetAttribute(k_topk_final<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)topk_final_smem_bytes());
}

void launch_begin(rorbk_ctx *h, const double *b, const double *x0, double *x, int use_cond,
                  unsigned long long hcond) {
    k_begin<<<1, 1024, 0, h->stream>>>(b, (int)h->m, x0, x, (int)h->n, h->ctl, use_cond,
                                       (cudaGraphConditionalHandle)hcond);
}

template <typename T>
void launch_iteration_t(rorbk_ctx *h, const T *b, T *x, T *r, Ctl *ctl, int use_cond,
                        unsigned long long hcond) {
    Mat<T> A = make_mat<T>(h);
    k_static<T><<<1, 1024, 0, h->stream>>>(A, b, x, ctl, -1);
    if (sizeof(T) == sizeof(float) || h->vdtype == RORBK_F32)
        k_residual<T, float><<<h->grid_res, 256, 0, h->stream>>>(A, b, x, r, h->partials, h->hist1, ctl, 1);
    else
        k_residual<T, double><<<h->grid_res, 256, 0, h->stream>>>(A, b, x, r, h->partials, h->hist1, ctl, 1);
    const int g = grid_stream(h, (int)h->m);
    k_topk_hist2<T><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->K, h->hist2, ctl, 1);
    k_topk_collect<T><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->in_list, h->eq_list, ctl, 1);
    k_dynamic<T><<<1, 512, dyn_smem_bytes(), h->stream>>>(A, r, x, h->in_list, h->eq_list, nullptr,
                                                          dyn_scratch(h), ctl, use_cond,
                                                          (cudaGraphConditionalHandle)hcond, 1);
}

void launch_iteration(rorbk_ctx *h, const double *b, double *x, double *r, int use_cond,
                      unsigned long long hcond) {
    launch_iteration_t<double>(h, b, x, r, h->ctl, use_cond, hcond);
}

void launch_static_forced(rorbk_ctx *h, int tau, const double *b, double *x) {
    k_static<double><<<1, 1024, 0, h->stream>>>(make_mat<double>(h), b, x, h->ctl, tau);
}

void launch_residual_only(rorbk_ctx *h, const double *b, const double *x, double *r) {
    if (h->vdtype == RORBK_F32)
        k_residual<double, float><<<h->grid_res, 256, 0, h->stream>>>(make_mat<double>(h), b, x, r,
                                                                      h->partials, h->hist1, h->ctl, 2);
    else
        k_residual<double, double><<<h->grid_res, 256, 0, h->stream>>>(make_mat<double>(h), b, x, r,
                                                                       h->partials, h->hist1, h->ctl, 2);
}

void launch_topk_only(rorbk_ctx *h, const double *r, int *I) {
    const int g = grid_stream(h, (int)h->m);
    k_topk_hist1<double><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->K, h->hist1, h->ctl);
    k_topk_hist2<double><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->K, h->hist2, h->ctl, 0);
    k_topk_collect<double><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->in_list, h->eq_list, h->ctl, 0);
    k_topk_final<double><<<1, 512, topk_final_smem_bytes(), h->stream>>>(
        r, (int)h->m, h->K, h->in_list, h->eq_list, h->ctl, I);
}

void launch_dynamic_given(rorbk_ctx *h, const int *I, const double *r, double *x) {
    k_dynamic<double><<<1, 512, dyn_smem_bytes(), h->stream>>>(
        make_mat<double>(h), r, x, h->in_list, h->eq_list, I, dyn_scratch(h), h->ctl, 0, 0, 0);
}

void launch_sample_probe(rorbk_ctx *h, uint64_t seed, uint64_t sysid, int64_t it, int64_t l,
                         long long *out) {
    k_sample_probe<<<1, 1, 0, h->stream>>>(h->cdf, h->k, seed, sysid, it, l, out);
}

}  // namespace rorbk
