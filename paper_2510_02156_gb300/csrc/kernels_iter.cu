// kernels_iter.cu -- the ROR-BK iteration (Algorithm 1's loop body).
//
//   k_begin        ||b||, x0, loop state; sets the loop condition
//   k_static       l = 1..n_static: draw tau (Philox; formed ahead by the
//                  previous k_dyn_mark when it can be), r_tau = b_tau - A_tau x,
//                  y = W_tau r_tau, x += A_tau^T y   (one block of threads)
//   k_residual     r = b - A x over nnz-balanced row tiles, ||r||^2, the
//                  convergence test, and the first radix histogram of |r|
//   k_topk_hist2   second 11-bit radix histogram inside the selected bin
//   k_topk_collect rows above the 22-bit threshold and the candidates on it;
//                  the last block completes the exact top-K set
//   k_dyn_mark     gathers A_I, marks shared columns, Gram diagonal; the last
//                  block factors G = A_I A_I^T + mu I on the coupled rows and
//                  solves for y, the first block done forms the next draws
//   k_dyn_scatter  x += A_I^T y; ends the iteration, sets the loop condition
//
// Compute type T is double (the plain method) or float (the inner solve of
// the mixed-precision form).  In FP64 every multiply-add is one fused
// multiply-add and every sum runs in the oracle's order (row dots in stored
// order; A^T y per column over ascending rows; Gram entries over ascending
// columns; column-ordered triangular solves), so the iterates reproduce the
// FP64 definition exactly.  FP64 arithmetic on this part has a long latency,
// so chains are kept short: the Cholesky of the coupled rows runs per
// connected component (one warp each), or, for components above 32 rows,
// along its elimination tree (all columns of one tree level at once); both
// perform the same operations on every entry in the same order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"
#include "topk_key.cuh"

namespace rorbk {

template <typename T> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};
template <typename T> __device__ __forceinline__ T as(double v);
template <> __device__ __forceinline__ double as<double>(double v) { return v; }
template <> __device__ __forceinline__ float as<float>(double v) { return (float)v; }
template <typename T> __device__ __forceinline__ T wide(float v);
template <> __device__ __forceinline__ double wide<double>(float v) { return widen(v); }
template <> __device__ __forceinline__ float wide<float>(float v) { return v; }
template <typename T> __device__ __forceinline__ T wide(double v) { return (T)v; }

// VEC values of T in one aligned load (16 bytes at most).
template <typename T, int VEC>
struct VecT {
    T v[VEC];
};
// STREAM: a value read once (evict-first in L1 and L2, ld.global.cs), so that
// the gathered X stays resident in L2 while A, B and R stream past it.
template <typename T, int VEC, bool STREAM = false>
__device__ __forceinline__ VecT<T, VEC> vload(const T *p) {
    VecT<T, VEC> r;
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        const float4 q = STREAM ? __ldcs(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
        r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 q = STREAM ? __ldcs(reinterpret_cast<const float2 *>(p)) : __ldg(reinterpret_cast<const float2 *>(p));
        r.v[0] = q.x; r.v[1] = q.y;
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        const double2 q = STREAM ? __ldcs(reinterpret_cast<const double2 *>(p)) : __ldg(reinterpret_cast<const double2 *>(p));
        r.v[0] = q.x; r.v[1] = q.y;
    } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) r.v[u] = STREAM ? __ldcs(p + u) : __ldg(p + u);
    }
    return r;
}

// The radix key of |v| in the top-K passes: the FP64 bit pattern of |v|, for
// an FP32 value formed with integer operations (topk_key.cuh).
__device__ __forceinline__ unsigned long long topk_key(double v) { return abs_key(v); }
__device__ __forceinline__ unsigned long long topk_key(float v) { return topk_key_f32_bits(__float_as_uint(v)); }

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
    const uint16_t *bperm;
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
    // SELL-32 copy of A (the residual)
    int nslices;
    const long long *sptr;
    const int *slen, *srow, *srlen, *scol;
    const double *sval;
    const float *sval32;
    // the s >= n form (Lemma 1, Section 3.1): block t's V_t at wood + wood_ptr[t]
    // (n x n row-major) when wood_ptr != nullptr and wood_ptr[t] >= 0
    const long long *wood_ptr;
    const T *wood;
    const double *rn;           // ||A_i||^2 of the values this instance reads
    const uint16_t *bt_off;     // CSR offset in its block of each block-transpose entry
    const int *blk_nz;          // [k+1] first entry of block t: rowptr[off[t]]
};

template <typename T>
Mat<T> make_mat(rorbk_ctx *h);
template <>
Mat<double> make_mat<double>(rorbk_ctx *h) {
    return Mat<double>{h->rowptr, h->col, h->val, h->off, h->cdf, (int)h->m, (int)h->n, h->k, h->K,
                       h->ops.s_ptr, h->ops.s_idx, h->ops.w_ptr, h->ops.w_ss, h->ops.w_diag,
                       h->ops.s_pos, h->ops.bperm, h->bt.col, h->bt.row, h->bt.val, h->bt.seg, h->bt.seg_ptr,
                       h->tile_row0, h->ntiles, h->mu, h->val32, h->sell.nslices, h->sell.ptr,
                       h->sell.len, h->sell.row, h->sell.rlen, h->sell.col, h->sell.val,
                       h->sell.val32, h->wood_ptr, h->wood_ss, h->rn, h->bt.off16, h->blk_nz};
}
template <>
Mat<float> make_mat<float>(rorbk_ctx *h) {
    return Mat<float>{h->rowptr, h->col, h->val32, h->off, h->cdf, (int)h->m, (int)h->n, h->k, h->K,
                      h->ops.s_ptr, h->ops.s_idx, h->ops.w_ptr, h->ops.w_ss32, h->ops.w_diag32,
                      h->ops.s_pos, h->ops.bperm, h->bt.col, h->bt.row, h->bt.val32, h->bt.seg, h->bt.seg_ptr,
                      h->tile_row0, h->ntiles, h->mu, h->val32, h->sell.nslices, h->sell.ptr,
                      h->sell.len, h->sell.row, h->sell.rlen, h->sell.col, h->sell.val,
                      h->sell.val32, h->wood_ptr, h->wood_ss32, h->rn32, h->bt.off16, h->blk_nz};
}

// -------------------------------------------------------- several columns
// The kernels of the iteration also run one solve per right-hand side of a
// block of nr columns (rorbk_multi_create): grid dimension y is the column,
// each column has its own loop state (ctl + column) and dynamic-block
// workspace (dyn_col), x and b are row-major n x nr and m x nr (entry c of
// column j at c * ld + j), and the residual columns are stored one after the
// other in the SELL copy's row order (position p holds row perm[p], -1 for a
// padding lane).  One column (ld = 1, perm = nullptr) is the plain solve.
struct Cols {
    int ld;               // distance between consecutive entries of x and of b
    long long rs;         // distance between the residual columns
    int mpos;             // residual positions per column (m, or the SELL length)
    const int *perm;      // SELL position -> row (nullptr: positions are rows)
    const int *iperm;     // row -> SELL position
    unsigned *grp;        // [0] column ticket of the group, [1] 1 while any column runs
};
static inline Cols one_col(int m) { return Cols{1, 0, m, nullptr, nullptr, nullptr}; }
// MC (several columns) is a template flag of every kernel that takes Cols, so
// the one-column instances compile without the column arithmetic.
template <bool MC>
__device__ __forceinline__ int rpos(const Cols &cl, int i) { return MC && cl.iperm ? cl.iperm[i] : i; }

// Called once per column and launch by one thread, after that column's loop
// state is final: the last column to arrive sets the WHILE condition to
// "some column has not halted" and records it for a host-driven loop.
__device__ void group_condition(const Ctl *ctl0, int nr, unsigned *grp, int use_cond,
                                cudaGraphConditionalHandle hcond) {
    __threadfence();
    if (atomicAdd(&grp[0], 1u) != (unsigned)nr - 1u) return;
    __threadfence();
    int any = 0;
    for (int j = 0; j < nr; ++j) any |= !((volatile const Ctl *)ctl0)[j].halt;
    grp[1] = (unsigned)any;
    grp[0] = 0u;
    if (use_cond) cudaGraphSetConditional(hcond, any ? 1u : 0u);
}

// ---------------------------------------------------- incremental residual
// Appends (c, v) for an update x_c += v to the iteration's change log.  The
// calling lanes of a warp take consecutive slots from one atomic; entries past
// the capacity set log_full, which makes the next residual exact.
__device__ __forceinline__ void inc_log(Ctl *ctl, int c, double v) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&ctl->nlog, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    const int idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < ctl->log_cap) {
        ctl->log_col[idx] = c;
        ctl->log_val[idx] = v;
    } else {
        ctl->log_full = 1;
    }
}

// ------------------------------------------------------------------ begin
// ||b||, x = x0 or 0, loop state.  One block; sets the WHILE condition.
__global__ void k_begin(const double *__restrict__ b, int m, const double *__restrict__ x0,
                        double *__restrict__ x, int n, Ctl *ctl, int use_cond,
                        cudaGraphConditionalHandle hcond) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s = __fma_rn(b[i], b[i], s);
    s = block_sum(s, red);
    __shared__ double bn;
    if (threadIdx.x == 0) bn = sqrt(s);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x)
        x[c] = (bn == 0.0 || x0 == nullptr || !ctl->has_x0) ? 0.0 : x0[c];
    if (threadIdx.x == 0) {
        const bool finite = isfinite(bn);
        ctl->bnorm = bn;
        ctl->iter = 0;
        ctl->rr = 0.0;
        ctl->rrn = bn == 0.0 ? 0.0 : 1.0;
        ctl->done = bn == 0.0;
        ctl->halt = !(finite && bn > 0.0 && ctl->maxit > 0);
        ctl->status = finite ? 0 : kDevNumeric;      // NaN or Inf in b
        ctl->ticket = 0;
        ctl->n_in = 0;
        ctl->n_eq = 0;
        ctl->outer = 0;
        ctl->inc_full = 1;         // the first residual of a solve is exact
        ctl->inc_count = 0;
        ctl->nlog = 0;
        ctl->log_full = 0;
        if (use_cond) cudaGraphSetConditional(hcond, ctl->halt ? 0u : 1u);
    }
}

// ----------------------------------------------------------------- static
// One block of threads runs the n_static sampled updates of an iteration in
// sequence (Algorithm 1, the inner loop over l); the draws do not depend on
// x and are taken up front.  Uses the stored W_tau (Section 3.1).
//
// Data movement: the CSR range of a sampled block and its column-sorted copy
// (columns, local rows, values) do not depend on x, so they are brought into
// shared memory by TMA bulk copies two blocks ahead (two stages, one mbarrier
// each), while the current update runs.  Each update then needs two
// dependent global round trips only: the gather of x at the block's columns
// and the update of x.  Blocks larger than a stage (long or dense rows) take
// the direct path (each row read from global memory by its thread), with the
// same arithmetic.
// force_tau >= 0 replaces the draw by that block (single-step API, direct
// path only).
constexpr int kStageCap = 3072;      // entries of one block held by a stage
constexpr int kStageC = kStageCap + 16;
constexpr long long kWaitTries = 1LL << 24;

template <typename T>
__host__ __device__ constexpr size_t static_stage_bytes() {
    return (size_t)kStageC * (2 * sizeof(T) + 4 + 4 + 2 + 2);
}
template <typename T>
__host__ __device__ constexpr size_t static_smem_bytes() {
    return 64 + 2 * static_stage_bytes<T>() + (size_t)kStageC * sizeof(T);
}

template <typename T>
struct Stage {
    T *val, *btval;
    int *col, *btcol;
    uint16_t *btrow, *btoff;
};
template <typename T>
__device__ __forceinline__ Stage<T> stage_at(unsigned char *base) {
    Stage<T> st;
    st.val = (T *)base;
    st.btval = st.val + kStageC;
    st.col = (int *)(st.btval + kStageC);
    st.btcol = st.col + kStageC;
    st.btrow = (uint16_t *)(st.btcol + kStageC);
    st.btoff = st.btrow + kStageC;
    return st;
}

// Issues the bulk copies of the block whose entries are [p0, pend) into a
// stage (thread 0).  Returns the aligned first entry a0, or -1 when the block
// does not fit a stage.
template <typename T>
__device__ int stage_issue(const Mat<T> &A, int p0, int pend, Stage<T> st, unsigned long long *bar) {
    if (pend <= p0) return -2;                        // no nonzeros: nothing to stage
    const int a0 = p0 & ~7, a1 = (pend + 7) & ~7;     // 16-byte aligned for every array
    const int n = a1 - a0;
    if (n > kStageC) return -1;
    const unsigned bytes = (unsigned)n * (2u * sizeof(T) + 4u + 4u + 2u + 2u);
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bytes);
    bulk_g2s(st.val, A.val + a0, n * sizeof(T), bar);
    bulk_g2s(st.btval, A.bt_val + a0, n * sizeof(T), bar);
    bulk_g2s(st.col, A.col + a0, n * 4, bar);
    bulk_g2s(st.btcol, A.bt_col + a0, n * 4, bar);
    bulk_g2s(st.btrow, A.bt_row + a0, n * 2, bar);
    bulk_g2s(st.btoff, A.bt_off + a0, n * 2, bar);
    return a0;
}

// The s >= n form of a static update (Lemma 1, Section 3.1), called by every
// thread of k_static once r_tau is in rloc: g = A_tau^T r_tau (each column
// over its rows ascending, 0 for the columns the block does not hold) into y,
// then x_c += sum over d ascending of V_cd g_d for every column c.
template <typename T>
__device__ __forceinline__ void static_update_wood(int n, int ns, const int *bt_seg, const int *bt_col,
                                                const uint16_t *bt_row, const T *bt_val, const T *V,
                                                int p0, int pend, const T *rloc, T *y, T *x, Ctl *ctl,
                                                bool lg, int ld) {
    const int a = threadIdx.x;
    for (int c = a; c < n; c += blockDim.x) y[c] = T(0);
    __syncthreads();
    for (int gq = a; gq < ns; gq += blockDim.x) {
        int q = bt_seg[p0 + gq];
        const int c = bt_col[q];
        T acc3 = T(0);
        for (; q < pend && bt_col[q] == c; ++q) acc3 = Ar<T>::fma(bt_val[q], rloc[bt_row[q]], acc3);
        y[c] = acc3;
    }
    __syncthreads();
    for (int c = a; c < n; c += blockDim.x) {
        const T *Vr = V + (long long)c * n;
        T acc4 = T(0);
        for (int d = 0; d < n; ++d) acc4 = Ar<T>::fma(Vr[d], y[d], acc4);
        x[(long long)c * ld] = Ar<T>::add(x[(long long)c * ld], acc4);
        if (lg) inc_log(ctl, c, (double)acc4);
    }
    __syncthreads();
}

// The draws of one iteration by the whole block.  Thread l < nst forms the
// target u_l * cdf[k-1] as sample_block does; every thread then counts, for
// every draw, the entries of its share of the running sum (nondecreasing) that
// do not exceed the target, and tau_l = min(count, k - 1): the first t with
// cdf[t] > target, which sample_block's binary search finds.  One coalesced
// pass over the cdf replaces a chain of log2(k) dependent loads.
template <int kHeld>                                  // entries held per thread (k <= kHeld * blockDim in one go)
__device__ __forceinline__ void sample_blocks_block(const double *cdf, int k, uint64_t seed, uint64_t sysid,
                                                    uint64_t it, int nst, double *s_target, int *s_cnt,
                                                    int *taus) {
    const int a = threadIdx.x;
    double cv[kHeld];
#pragma unroll
    for (int u = 0; u < kHeld; ++u) {
        const int t = a + u * (int)blockDim.x;
        cv[u] = t < k ? cdf[t] : 0.0;
    }
    if (a < nst) {
        uint64_t w[4];
        philox4x64_10(it, (uint64_t)a, 0, 0, seed, sysid, w);
        const double u = (double)(w[0] >> 11) * 0x1.0p-53;
        s_target[a] = u * cdf[k - 1];
        s_cnt[a] = 0;
    }
    __syncthreads();
    for (int l = 0; l < nst; ++l) {
        const double tg = s_target[l];
        int c = 0;
#pragma unroll
        for (int u = 0; u < kHeld; ++u) c += (a + u * (int)blockDim.x < k) && cv[u] <= tg;
        for (int t = a + kHeld * (int)blockDim.x; t < k; t += blockDim.x) c += cdf[t] <= tg;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((a & 31) == 0 && c) atomicAdd(&s_cnt[l], c);
    }
    __syncthreads();
    if (a < nst) taus[a] = min(s_cnt[a], k - 1);
    __syncthreads();
}

// Per-row data of a static block that does not depend on x: thread a takes
// the a-th longest row la of block tau.
template <typename T>
struct StaticRow {
    int la, q0, q1, pos;
    T bi, wd;
};

// LOG: the incremental residual's variant, which logs every change of x.
// WOOD: the variant for handles with blocks in the s >= n form (the other
// instances compile without that branch).
// Every x-independent load of an update is issued ahead of the x-dependent
// chain: the blocks' ranges for all draws at the start, the next block's row
// order during the current gather, its per-row data during the current dot
// products; the gather of x and the old values of the scatter come from
// shared memory when the block is staged.
template <typename T, bool LOG = false, bool WOOD = false, bool MC = false>
__global__ void __launch_bounds__(1024, 1) k_static(Mat<T> A, const T *__restrict__ b, T *x,
                                                 Ctl *ctl, int force_tau, int use_stages,
                                                 int l_begin, int ld_) {
    extern __shared__ unsigned long long dsm_u64[];
    __shared__ T rloc[kMaxBlockRows];
    __shared__ T y[kMaxBlockRows];
    __shared__ int taus[64];
    __shared__ int s_r0[64], s_s[64], s_p0[64], s_pend[64], s_sb[64], s_nS[64];
    __shared__ long long s_wb[64];
    __shared__ double s_target[64];
    __shared__ int s_cnt[64];
    __shared__ int s_a0[2];
    __shared__ int s_fail;
    if constexpr (MC) {                               // column blockIdx.y of a block of columns
        ctl += blockIdx.y;
        x += blockIdx.y;
        b += blockIdx.y;
    }
    const int ld = MC ? ld_ : 1;
    if (force_tau < 0 && (ctl->done || ctl->halt)) return;
    const bool lg = LOG && force_tau < 0;            // log x's changes
    const int nst = force_tau >= 0 ? 1 : ctl->n_static;
    const int a = threadIdx.x;
    unsigned long long *bar = dsm_u64;                // two mbarriers
    unsigned char *sbase = (unsigned char *)(dsm_u64 + 8);
    T *sx = (T *)(sbase + 2 * static_stage_bytes<T>());
    const long long cnt = ctl->iter_base + ctl->iter;
    // the draws and ranges formed ahead by the previous iteration's top-K pass
    const bool planned = force_tau < 0 && nst <= kPreDraws && ctl->pre_it == cnt + 1;
    if (force_tau >= 0) {
        if (a == 0) taus[0] = force_tau;
        __syncthreads();
    } else if (planned) {
        if (a < nst) {
            taus[a] = ctl->pre_tau[a];
            s_r0[a] = ctl->pre_r0[a];
            s_s[a] = ctl->pre_s[a];
            s_sb[a] = ctl->pre_sb[a];
            s_nS[a] = ctl->pre_nS[a];
            s_wb[a] = ctl->pre_wb[a];
            s_p0[a] = ctl->pre_p0[a];
            s_pend[a] = ctl->pre_pend[a];
        }
    } else {
        sample_blocks_block<4>(ctl->scdf ? ctl->scdf : A.cdf, A.k, ctl->seed, ctl->sysid, (uint64_t)cnt, nst,
                               s_target, s_cnt, taus);
    }
    if (force_tau < 0 && a < nst && ctl->tr_tau && ctl->iter < ctl->trace_cap)
        ctl->tr_tau[ctl->iter * nst + a] = taus[a];
    // the blocks' ranges and operator offsets, for every draw at once
    if (!planned && a < nst) {
        const int tau = taus[a];
        const int r0 = A.off[tau], r1 = A.off[tau + 1];
        s_r0[a] = r0;
        s_s[a] = r1 - r0;
        s_sb[a] = A.s_ptr[tau];
        s_nS[a] = A.s_ptr[tau + 1] - A.s_ptr[tau];
        s_wb[a] = A.w_ptr[tau];
        s_p0[a] = A.blk_nz[tau];
        s_pend[a] = A.blk_nz[tau + 1];
    }
    const bool inject = ctl->fault == RORBK_FAULT_WAIT_LIMIT && force_tau < 0;
    if (a == 0) {
        s_fail = 0;
        s_a0[0] = s_a0[1] = -1;
        if (use_stages) { mbar_init(&bar[0], 1); mbar_init(&bar[1], 1); }
        if (inject) mbar_init(&bar[2], 1);           // a barrier that nothing completes
    }
    __syncthreads();
    if (use_stages && a == 0) {
        if (nst > 0) s_a0[0] = stage_issue<T>(A, s_p0[0], s_pend[0], stage_at<T>(sbase), &bar[0]);
        if (nst > 1)
            s_a0[1] = stage_issue<T>(A, s_p0[1], s_pend[1], stage_at<T>(sbase + static_stage_bytes<T>()), &bar[1]);
    }
    // the first update's per-row data
    StaticRow<T> cur{0, 0, 0, -1, T(0), T(0)};
    if (l_begin < nst && a < s_s[l_begin]) {
        const int r0 = s_r0[l_begin];
        cur.la = A.bperm[r0 + a];
        cur.q0 = A.rowptr[r0 + cur.la];
        cur.q1 = A.rowptr[r0 + cur.la + 1];
        cur.bi = b[(long long)(r0 + cur.la) * ld];
        cur.pos = A.s_pos[r0 + cur.la];
        cur.wd = A.w_diag[r0 + cur.la];
    }
    unsigned phase[2] = {0u, 0u};
    for (int l = l_begin; l < nst; ++l) {
        const int tau = taus[l];
        const int sidx = l & 1;
        const int s = s_s[l];
        const int p0 = s_p0[l], pend = s_pend[l];
        const int sb = s_sb[l], nS = s_nS[l];        // W_tau on the coupled rows
        const long long wb = s_wb[l];
        const bool has_next = l + 1 < nst;
        const int r0n = has_next ? s_r0[l + 1] : 0, sn = has_next ? s_s[l + 1] : 0;
        // the next block's row order, in flight during this update
        int la_next = 0;
        if (has_next && a < sn) la_next = A.bperm[r0n + a];
        __syncthreads();                              // s_a0 of this stage published
        const int a0 = use_stages ? s_a0[sidx] : -1;
        const bool staged = a0 >= 0;
        if (staged) {
            // fault injection: the wait gives up as if the copies never landed
            const bool ok = inject ? mbar_wait_bounded(&bar[2], 0u, 1)
                                   : mbar_wait_bounded(&bar[sidx], phase[sidx], kWaitTries);
            if (!ok) atomicOr(&s_fail, 1);
            phase[sidx] ^= 1u;
        }
        __syncthreads();
        if (s_fail) {
            if (a == 0) {
                set_status(&ctl->status, kDevTimeout);
                ctl->done = 1;
                // drain whatever is still in flight before the block exits
                mbar_wait_bounded(&bar[sidx], phase[sidx] ^ 1u, kWaitTries);
                if (s_a0[sidx ^ 1] >= 0) mbar_wait_bounded(&bar[sidx ^ 1], phase[sidx ^ 1], kWaitTries);
            }
            return;
        }
        const int la = cur.la;
        T acc = T(0);
        if (staged) {
            const Stage<T> st = stage_at<T>(sbase + sidx * static_stage_bytes<T>());
            // x at the block's columns: four loads in flight per thread
            for (int p = p0 + a; p < pend; p += 4 * (int)blockDim.x) {
                T v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = p + u * (int)blockDim.x;
                    v[u] = q < pend ? x[(long long)st.col[q - a0] * ld] : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = p + u * (int)blockDim.x;
                    if (q < pend) sx[q - p0] = v[u];
                }
            }
            __syncthreads();
            for (int p = cur.q0; p < cur.q1; ++p) acc = Ar<T>::fma(st.val[p - a0], sx[p - p0], acc);
        } else {
            // a block too large for a stage: every thread runs its own row
            // straight from global memory (loads unrolled ahead of the chain),
            // so the rows proceed side by side however long they are
#pragma unroll 8
            for (int p = cur.q0; p < cur.q1; ++p) acc = Ar<T>::fma(A.val[p], x[(long long)A.col[p] * ld], acc);
        }
        // the next block's per-row data, in flight during the solve below
        StaticRow<T> nxt{0, 0, 0, -1, T(0), T(0)};
        if (has_next && a < sn) {
            nxt.la = la_next;
            nxt.q0 = A.rowptr[r0n + la_next];
            nxt.q1 = A.rowptr[r0n + la_next + 1];
            nxt.bi = b[(long long)(r0n + la_next) * ld];
            nxt.pos = A.s_pos[r0n + la_next];
            nxt.wd = A.w_diag[r0n + la_next];
        }
        if (a < s) rloc[la] = Ar<T>::sub(cur.bi, acc);
        __syncthreads();
        const long long wp = WOOD ? A.wood_ptr[tau] : -1;
        if (WOOD && wp >= 0) {
            static_update_wood<T>(A.n, A.nseg[tau], A.bt_seg, A.bt_col, A.bt_row, A.bt_val, A.wood + wp, p0,
                                  pend, rloc, y, x, ctl, lg, ld);
            if (use_stages && a == 0) s_a0[sidx] = l + 2 < nst ? stage_issue<T>(A, s_p0[l + 2], s_pend[l + 2], stage_at<T>(sbase + sidx * static_stage_bytes<T>()), &bar[sidx]) : -1;
            cur = nxt;
            continue;
        }
        if (a < s) {
            if (cur.pos < 0) {
                y[la] = Ar<T>::fma(cur.wd, rloc[la], T(0));
            } else {
                // the loads of W's row and of the row indices do not depend on
                // the chain: unrolled, they are in flight ahead of it
                const T *Wr = A.w_ss + wb + (long long)cur.pos * nS;
                T acc2 = T(0);
#pragma unroll 8
                for (int q = 0; q < nS; ++q) acc2 = Ar<T>::fma(Wr[q], rloc[A.s_idx[sb + q]], acc2);
                y[la] = acc2;
            }
        }
        __syncthreads();
        if (staged) {
            // x's old value of every column comes from the gather above (x
            // has not changed since); the sum over its rows is unchanged
            const Stage<T> st = stage_at<T>(sbase + sidx * static_stage_bytes<T>());
            for (int q = p0 + a; q < pend; q += blockDim.x) {
                const int c = st.btcol[q - a0];
                if (q > p0 && st.btcol[q - 1 - a0] == c) continue;
                T acc3 = T(0);
                for (int u = q; u < pend && st.btcol[u - a0] == c; ++u)
                    acc3 = Ar<T>::fma(st.btval[u - a0], y[st.btrow[u - a0]], acc3);
                x[(long long)c * ld] = Ar<T>::add(sx[st.btoff[q - a0]], acc3);
                if (lg) inc_log(ctl, c, (double)acc3);
            }
        } else {
            const int ns = A.nseg[tau];
            for (int g = a; g < ns; g += blockDim.x) {
                int q = A.bt_seg[p0 + g];
                const int c = A.bt_col[q];
                T acc3 = T(0);
                for (; q < pend && A.bt_col[q] == c; ++q)
                    acc3 = Ar<T>::fma(A.bt_val[q], y[A.bt_row[q]], acc3);
                x[(long long)c * ld] = Ar<T>::add(x[(long long)c * ld], acc3);
                if (lg) inc_log(ctl, c, (double)acc3);
            }
        }
        __syncthreads();
        // this stage is free again: bring in block l + 2
        if (use_stages && a == 0) s_a0[sidx] = l + 2 < nst ? stage_issue<T>(A, s_p0[l + 2], s_pend[l + 2], stage_at<T>(sbase + sidx * static_stage_bytes<T>()), &bar[sidx]) : -1;
        cur = nxt;
    }
    // incremental residual: this iteration's residual is exact after a full
    // log or every inc_refresh iterations
    if (lg && a == 0 && !ctl->inc_full)
        if (ctl->log_full || ++ctl->inc_count >= ctl->inc_refresh) ctl->inc_full = 1;
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

template <typename V, typename T>
__device__ __forceinline__ const V *sell_values(const Mat<T> &A);
template <>
__device__ __forceinline__ const double *sell_values<double, double>(const Mat<double> &A) { return A.sval; }
template <>
__device__ __forceinline__ const float *sell_values<float, double>(const Mat<double> &A) { return A.sval32; }
template <>
__device__ __forceinline__ const float *sell_values<float, float>(const Mat<float> &A) { return A.sval32; }

// Warp-aggregated shared-memory histogram increment.
__device__ __forceinline__ void hist_add(unsigned *hist, unsigned bin, bool active) {
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const unsigned peers = __match_any_sync(mask, bin);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&hist[bin], (unsigned)__popc(peers));
}

// r = b - A x on the SELL-32 copy of A: one warp per slice of 32 rows of
// (nearly) equal length, one lane per row, so every fused multiply-add
// instruction carries a full warp of rows; each row is one chain in stored
// column order.  Longest slices come first.  V is the stored value type (an
// FP32-stored system is read as FP32 and widened exactly).
// finalize: 1 = convergence test + first radix level (iteration), 2 = ||r||^2
// only (single-step API).  DN: A is dense, so entry j of a row is in column j
// and the column indices are not read (x_j is the same for the warp's lanes).
constexpr int kDnAhead = 8;      // dense residual: 16-byte loads per lane in flight

// (a dense A: three blocks per SM, so that each lane keeps kDnAhead loads in
// flight without spilling)
template <typename T, typename V, bool DN = false>
__global__ void __launch_bounds__(256, DN ? 3 : 4) k_residual(Mat<T> A, const T *__restrict__ b,
                                                  const T *__restrict__ x, T *__restrict__ r,
                                                  double *partials, unsigned *hist1, Ctl *ctl,
                                                  int finalize) {
    __shared__ unsigned hist[kHistBins];
    __shared__ double red[32];
    __shared__ int is_last;
    if ((finalize == 1 || finalize == 3) && (ctl->done || ctl->halt)) return;
    if (finalize == 1 && ctl->inc && !ctl->inc_full) return;   // r came from the change log
    const V *__restrict__ val = sell_values<V, T>(A);
    const int lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    double rr = 0.0;
    __syncthreads();
    // One resident wave of blocks; slices (longest first) are dealt to the
    // warps in snake order, warps of consecutive ids sitting on different SMs,
    // so every warp gets a mix of long and short slices.
    const int W = gridDim.x * nwb;
    const int g = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    for (int rnd = 0;; ++rnd) {
        const int sl = rnd * W + ((rnd & 1) ? W - 1 - g : g);
        if (sl >= A.nslices) break;
        const long long base = A.sptr[sl] + lane;
        const int L = A.slen[sl];
        const int slot = sl * 32 + lane;
        const int row = A.srow[slot], len = A.srlen[slot];
        T acc = T(0);
        if constexpr (DN) {
            // a dense A: entry j of lane l is at 32 VW (j / VW) + VW l + j % VW
            // of the slice, so each load brings VW consecutive entries of the
            // lane's own row (16 bytes); kDnAhead such loads are in flight while
            // the chain runs over the previous ones, columns ascending as ever
            constexpr int VW = 16 / sizeof(V);
            const V *vb = val + A.sptr[sl] + VW * lane;
            VecT<V, VW> vq[kDnAhead];
#pragma unroll
            for (int q = 0; q < kDnAhead; ++q)
                if (q * VW < len) vq[q] = vload<V, VW, true>(vb + 32LL * VW * q);
            for (int q0 = 0; q0 * VW < L; q0 += kDnAhead) {
                VecT<V, VW> vc[kDnAhead];
#pragma unroll
                for (int q = 0; q < kDnAhead; ++q) vc[q] = vq[q];
#pragma unroll
                for (int q = 0; q < kDnAhead; ++q)
                    if ((q0 + kDnAhead + q) * VW < len)
                        vq[q] = vload<V, VW, true>(vb + 32LL * VW * (q0 + kDnAhead + q));
#pragma unroll
                for (int q = 0; q < kDnAhead; ++q)
#pragma unroll
                    for (int u = 0; u < VW; ++u) {
                        const int j = (q0 + q) * VW + u;
                        if (j < len) acc = Ar<T>::fma(wide<T>(vc[q].v[u]), x[j], acc);
                    }
            }
        } else {
        // software pipeline, 8 deep: the x gathers of chunk k and the index /
        // value loads of chunk k+1 are in flight while chunk k's chain runs
        int cn[8];
        V vn[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool in = u < len;
            const long long d = base + 32LL * u;
            cn[u] = in ? A.scol[d] : 0;
            vn[u] = in ? val[d] : V(0);
        }
        for (int c0 = 0; c0 < L; c0 += 8) {
            T xv[8];
            V vc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                xv[u] = c0 + u < len ? x[cn[u]] : T(0);
                vc[u] = vn[u];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = c0 + 8 + u;
                const bool in = j < len;
                const long long d = base + 32LL * j;
                cn[u] = in ? A.scol[d] : 0;
                vn[u] = in ? val[d] : V(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c0 + u < len) acc = Ar<T>::fma(wide<T>(vc[u]), xv[u], acc);
        }
        }
        const bool act = row >= 0;
        unsigned bin = 0;
        if (act) {
            const T ri = Ar<T>::sub(b[row], acc);
            r[row] = ri;
            rr = __fma_rn((double)ri, (double)ri, rr);
            bin = (unsigned)(abs_key(ri) >> 52);
        }
        if (finalize == 1) hist_add(hist, bin, act);
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
        if (finalize == 1 || finalize == 3) {
            const double rrn = sqrt(tot) / ctl->bnorm;
            ctl->rrn = rrn;
            if (finalize == 1 && ctl->tr_rrn && ctl->iter < ctl->trace_cap) ctl->tr_rrn[ctl->iter] = rrn;
            if (!isfinite(rrn)) { set_status(&ctl->status, kDevNumeric); ctl->done = 1; }
            else if (rrn <= ctl->tol) ctl->done = 1;
            stop = ctl->done;
            ctl->n_in = 0;
            ctl->n_eq = 0;
        }
        if (finalize == 1 && ctl->inc) {   // the log so far is folded into this r
            ctl->nlog = 0;
            ctl->log_full = 0;
            ctl->inc_full = 0;
            ctl->inc_count = 0;
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

// Incremental residual, first kernel: r -= A dx from the iteration's change log,
// through the CSC copy of A.  A group of kIncLanes lanes takes one logged
// column and subtracts a_ic * dx_c from r_i for its entries (atomic adds, so
// the order of the additions into r_i varies from run to run).  Does nothing
// when this iteration's residual is exact.
constexpr int kIncLanes = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_inc_apply(const int *__restrict__ cptr,
                                                   const int *__restrict__ crow,
                                                   const T *__restrict__ cval, T *r, Ctl *ctl) {
    if (ctl->done || ctl->halt || ctl->inc_full) return;
    const int nlog = min(ctl->nlog, ctl->log_cap);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = t % kIncLanes, ng = gridDim.x * blockDim.x / kIncLanes;
    for (int e = t / kIncLanes; e < nlog; e += ng) {
        const int c = ctl->log_col[e];
        const T d = (T)ctl->log_val[e];
        const int p1 = cptr[c + 1];
        for (int p = cptr[c] + sub; p < p1; p += kIncLanes) atomicAdd(&r[crow[p]], -(cval[p] * d));
    }
}

// Incremental residual, second kernel: ||r||^2, the first radix level of the top-K
// select and the stopping test on the updated r.  A relative residual at or
// below the tolerance (or not finite) is not trusted: it sets inc_full, and
// the exact residual kernel that follows decides in the same iteration.
template <typename T>
__global__ void __launch_bounds__(256) k_inc_finish(const T *__restrict__ r, int m, int K,
                                                    double *partials, unsigned *hist1, Ctl *ctl) {
    __shared__ unsigned hist[kHistBins];
    __shared__ double red[32];
    __shared__ int is_last, stop;
    if (ctl->done || ctl->halt || ctl->inc_full) return;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    double rr = 0.0;
    for (int i0 = blockIdx.x * blockDim.x; i0 < m; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool act = i < m;
        unsigned bin = 0;
        if (act) {
            const T ri = r[i];
            rr = __fma_rn((double)ri, (double)ri, rr);
            bin = (unsigned)(topk_key(ri) >> 52);
        }
        hist_add(hist, bin, act);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
        if (hist[i]) atomicAdd(&hist1[i], hist[i]);
    rr = block_sum(rr, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = rr;
        __threadfence();
        is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += partials[i];
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->n_in = 0;
        ctl->n_eq = 0;
        ctl->nlog = 0;
        const double rrn = sqrt(tot) / ctl->bnorm;
        stop = !(rrn > ctl->tol);
        if (stop) {
            ctl->inc_full = 1;
        } else {
            ctl->rr = tot;
            ctl->rrn = rrn;
            if (ctl->tr_rrn && ctl->iter < ctl->trace_cap) ctl->tr_rrn[ctl->iter] = rrn;
        }
    }
    __syncthreads();
    if (!stop) {
        int bin, above;
        select_bin(hist1, K, &bin, &above);
        if (threadIdx.x == 0) { ctl->sel1 = bin; ctl->above1 = above; }
    } else {
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist1[i] = 0u;
    }
}

// The top-K passes over r are grid-stride loops whose iterations are
// independent: each thread loads kScanU values before it uses any, so that
// several loads are in flight per thread instead of one.
constexpr int kScanU = 8;

// First radix level over a given r (single-step top-K, and the iteration of
// a block of columns, whose residual pass leaves it out: check_done).
template <typename T, bool MC = false>
__global__ void __launch_bounds__(256) k_topk_hist1(const T *__restrict__ r, int m, int K,
                                                    unsigned *hist1, Ctl *ctl, Cols cl,
                                                    int check_done) {
    __shared__ unsigned hist[kHistBins];
    __shared__ int is_last;
    if constexpr (MC) {
        ctl += blockIdx.y;
        r += blockIdx.y * cl.rs;
        hist1 += blockIdx.y * kHistBins;
    }
    if (check_done && (ctl->done || ctl->halt)) return;
    const int mp = MC ? cl.mpos : m;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    // warp-aggregated: the keys of a residual crowd into few exponent bins
    for (int i0 = blockIdx.x * blockDim.x * kScanU; i0 < mp; i0 += gridDim.x * blockDim.x * kScanU) {
        T v[kScanU];
        bool act[kScanU];
#pragma unroll
        for (int u = 0; u < kScanU; ++u) {
            const int i = i0 + u * blockDim.x + threadIdx.x;
            act[u] = i < mp && (!MC || !cl.perm || cl.perm[i] >= 0);
            v[u] = i < mp ? r[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kScanU; ++u) hist_add(hist, act[u] ? (unsigned)(topk_key(v[u]) >> 52) : 0u, act[u]);
    }
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

template <typename T, bool MC = false>
__global__ void __launch_bounds__(256) k_topk_hist2(const T *__restrict__ r, int m, int K,
                                                    unsigned *hist2, Ctl *ctl, int check_done,
                                                    Cols cl) {
    __shared__ unsigned hist[kHistBins];
    __shared__ int is_last;
    if constexpr (MC) {
        ctl += blockIdx.y;
        r += blockIdx.y * cl.rs;
        hist2 += blockIdx.y * kHistBins;
    }
    if (check_done && (ctl->done || ctl->halt)) return;

    const unsigned sel1 = (unsigned)ctl->sel1;
    const int mp = MC ? cl.mpos : m;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int i0 = blockIdx.x * blockDim.x * kScanU; i0 < mp; i0 += gridDim.x * blockDim.x * kScanU) {
        T v[kScanU];
        bool act[kScanU];
#pragma unroll
        for (int u = 0; u < kScanU; ++u) {
            // padding positions of a column block hold exact zeros; their
            // count is taken off the zero bin below instead of reading perm
            const int i = i0 + u * blockDim.x + threadIdx.x;
            act[u] = i < mp;
            v[u] = i < mp ? r[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kScanU; ++u) {
            const unsigned long long key = topk_key(v[u]);
            if (act[u] && (unsigned)(key >> 52) == sel1) atomicAdd(&hist[(unsigned)(key >> 41) & 2047u], 1u);
        }
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
    if (MC && cl.perm && sel1 == 0u && threadIdx.x == 0) hist2[0] -= (unsigned)(mp - m);   // padding zeros
    __syncthreads();
    select_bin(hist2, K - ctl->above1, &bin, &above);
    if (threadIdx.x == 0) {
        ctl->prefix = (int)((sel1 << 11) | (unsigned)bin);
        ctl->above = ctl->above1 + above;
        ctl->ticket = 0;
    }
}

// ------------------------------------------------------------ exact top-K
// Small sorts in one block by rank: the key at position q goes to the number
// of keys that precede it (smaller keys, or equal keys at lower positions), so
// the result is the ascending order with equal keys in their input order.  It
// takes one barrier and n comparisons per key (every lane reads the same key:
// a shared-memory broadcast); up to kRankSortMax keys that costs less than
// the log2(n)(log2(n)+1)/2 barrier-separated steps of a bitonic network.
constexpr int kRankSortMax = 256;
template <typename K>
__device__ void block_rank_sort(const K *keys, K *out, int n) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const K k = keys[q];
        int rank = 0;
        for (int u = 0; u < n; ++u) {
            const K v = keys[u];
            rank += (v < k) | ((v == k) & (u < q));
        }
        out[rank] = k;
    }
    __syncthreads();
}

// Completes the top-K set in one block of threads: the n_in rows above the
// 22-bit threshold plus the best (need) of the candidates on it, ordered by
// |r| descending and row ascending.  If more than kEqCap candidates share the
// threshold prefix, the block resolves the remaining 41 key bits itself by
// scanning r.  Writes I ascending to sI.  Shared scratch: keys and idx
// arrays of kEqCap entries.
// The lists hold rows; r is read at rpos(cl, row).
template <typename T, bool MC>
__device__ void finalize_topk(const T *__restrict__ r, int m, int K, const int *in_list,
                              const int *eq_list, Ctl *ctl, int *sI,
                              unsigned long long *skey, int *sidx, const Cols &cl) {
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
    if (need > 0 && neq <= kRankSortMax) {
        // the need first candidates in top-K order (larger key, then lower
        // row), each placed by its rank
        for (int e = threadIdx.x; e < neq; e += blockDim.x) {
            const int i = eq_list[e];
            skey[e] = topk_key(r[rpos<MC>(cl, i)]);
            sidx[e] = i;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < neq; e += blockDim.x) {
            const unsigned long long ke = skey[e];
            const int ie = sidx[e];
            int rank = 0;
            for (int u = 0; u < neq; ++u) rank += topk_before(skey[u], sidx[u], ke, ie);
            if (rank < need) sI[nin + rank] = ie;
        }
        __syncthreads();
    } else if (need > 0 && neq <= kEqCap) {
        const int np = next_pow2(neq);
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            if (e < neq) { int i = eq_list[e]; skey[e] = topk_key(r[rpos<MC>(cl, i)]); sidx[e] = i; }
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
                unsigned long long key = topk_key(r[rpos<MC>(cl, i)]);
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
                unsigned long long key = topk_key(r[rpos<MC>(cl, i)]);
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
            int f = (i < m && topk_key(r[rpos<MC>(cl, i)]) == T0) ? 1 : 0;
            int total;
            int pre = block_exclusive_scan(f, sc, &total);
            if (f && taken + pre < want) sI[s_fill + taken + pre] = i;
            taken += total;
        }
        __syncthreads();
    }
    __syncthreads();
    // ascending order
    if (K <= 2 * kRankSortMax) {
        int *tmp = (int *)skey;                       // the rows are distinct
        block_rank_sort<int>(sI, tmp, K);
        for (int a = threadIdx.x; a < K; a += blockDim.x) sI[a] = tmp[a];
        __syncthreads();
        return;
    }
    const int np = next_pow2(K);
    for (int a = threadIdx.x; a < np; a += blockDim.x)
        skey[a] = a < K ? (unsigned long long)(unsigned)sI[a] : ~0ull;
    __syncthreads();
    block_bitonic_sort(skey, np);
    for (int a = threadIdx.x; a < K; a += blockDim.x) sI[a] = (int)skey[a];
    __syncthreads();
}

// --------------------------------------------------------- dynamic block
// Buffers of the dynamic-block update (Algorithm 1, the residual top-K block):
// I and its gathered nonzeros, the column owner/count marks, the Gram
// diagonal, y, and global fallbacks for sizes above the shared-memory caps.
struct Dyn {
    int *I;                     // [K] ascending rows
    int *estart;                // [K+1] entry offsets of the rows of I
    double *gdiag;              // [K] ||A_i||^2 + mu
    double *y;                  // [K] (A_I A_I^T + mu I)^{-1} r_I
    int *ecol;                  // [ecap] gathered nonzeros, row order
    double *eval;
    uint16_t *erow;
    long long ecap;
    unsigned long long *owner;  // [n] (epoch << 32 | entry) of the first entry seen in a column
    unsigned *shared;           // [n] epoch in which the column was found shared inside I
    int *segpos;                // [n] position of a shared column in the sorted shared list
    unsigned *epoch;            // dynamic-update counter (never reset; 0 = never)
    unsigned long long *raw;    // [2 ecap] shared entries as found (with repeats)
    unsigned long long *skeys;  // [pow2 >= 2 ecap] shared entries sorted by (column, entry)
    unsigned long long *pkeys;  // [pcap] Gram contributions (fallback)
    long long pcap;
    double *g;                  // [K(K+1)/2] packed Gram fallback
    int K, n;                   // sizes of one column's buffers (a block of columns
    long long skcap;            // keeps its columns' buffers one after the other)
};

// The buffers of column jc of a block of columns.
__device__ __forceinline__ Dyn dyn_col(Dyn D, int jc) {
    if (jc == 0) return D;
    const long long K = D.K, n = D.n;
    D.I += jc * K;
    D.estart += jc * (K + 1);
    D.gdiag += jc * K;
    D.y += jc * K;
    D.ecol += jc * D.ecap;
    D.eval += jc * D.ecap;
    D.erow += jc * D.ecap;
    D.owner += jc * n;
    D.shared += jc * n;
    D.segpos += jc * n;
    D.epoch += jc;
    D.raw += jc * 2 * D.ecap;
    D.skeys += jc * D.skcap;
    D.pkeys += jc * D.pcap;
    D.g += jc * (K * (K + 1) / 2);
    return D;
}

__device__ __forceinline__ long long pidx(int i, int j) {     // packed lower, row-major
    return (long long)i * (i + 1) / 2 + j;
}

// Publishes I (from shared memory) and the entry offsets of its rows.
__device__ void publish_rows(const int *rowptr, const int *sI, int K, Dyn D, Ctl *ctl,
                             int trace) {
    __shared__ int sc[33];
    int carry = 0;
    for (int base = 0; base < K; base += blockDim.x) {
        const int a = base + threadIdx.x;
        const int len = a < K ? rowptr[sI[a] + 1] - rowptr[sI[a]] : 0;
        int total;
        const int pre = block_exclusive_scan(len, sc, &total);
        if (a < K) {
            D.I[a] = sI[a];
            D.estart[a] = carry + pre;
            if (trace && ctl->tr_I && ctl->iter < ctl->trace_cap)
                ctl->tr_I[ctl->iter * K + a] = sI[a];
        }
        carry += total;
    }
    if (threadIdx.x == 0) {
        D.estart[K] = carry;
        ctl->dynE = carry;
        ctl->dyn_nraw = 0;
        *D.epoch = *D.epoch + 1u;
    }
}

// Rows above the 22-bit threshold and the candidates on it; the last block
// completes the exact top-K set and publishes it.
template <typename T, bool MC = false>
__global__ void __launch_bounds__(512) k_topk_collect(const T *__restrict__ r, int m, int K,
                                                      const int *rowptr, int *in_list,
                                                      int *eq_list, Dyn D, Ctl *ctl,
                                                      int check_done, Cols cl) {
    extern __shared__ unsigned long long dsm_u64[];
    __shared__ int is_last;
    if constexpr (MC) {
        ctl += blockIdx.y;
        r += blockIdx.y * cl.rs;
        in_list += (long long)blockIdx.y * K;
        eq_list += (long long)blockIdx.y * kEqCap;
        D = dyn_col(D, blockIdx.y);
    }
    if (check_done && (ctl->done || ctl->halt)) return;
    const unsigned long long P = (unsigned long long)(unsigned)ctl->prefix;
    const int mp = MC ? cl.mpos : m;
    for (int p0 = blockIdx.x * blockDim.x * kScanU; p0 < mp; p0 += gridDim.x * blockDim.x * kScanU) {
        T v[kScanU];
        int row[kScanU];
#pragma unroll
        for (int u = 0; u < kScanU; ++u) {
            const int p = p0 + u * blockDim.x + threadIdx.x;
            row[u] = p < mp ? p : -1;
            v[u] = p < mp ? r[p] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kScanU; ++u) {
            if (row[u] < 0) continue;
            const unsigned long long pre = topk_key(v[u]) >> 41;
            if (pre < P) continue;
            const int i = MC && cl.perm ? cl.perm[row[u]] : row[u];   // the row at this position
            if (i < 0) continue;
            if (pre > P) {
                in_list[atomicAdd(&ctl->n_in, 1)] = i;
            } else {
                int pos = atomicAdd(&ctl->n_eq, 1);
                if (pos < kEqCap) eq_list[pos] = i;
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    unsigned long long *skey = dsm_u64;
    int *sidx = (int *)(skey + kEqCap);
    int *sI = sidx + kEqCap;
    finalize_topk<T, MC>(r, m, K, in_list, eq_list, ctl, sI, skey, sidx, cl);
    publish_rows(rowptr, sI, K, D, ctl, 1);
    if (threadIdx.x == 0) ctl->ticket = 0;
}

// Single-step API: a given ascending I, checked before any row is read (an
// entry outside [0, m) or a set that is not strictly ascending records
// kDevBounds, and the kernels after this one do nothing).
__global__ void __launch_bounds__(512) k_dyn_set_rows(const int *rowptr, const int *I, int K, int m,
                                                      Dyn D, Ctl *ctl) {
    __shared__ int sI[kMaxDynRows];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < K; a += blockDim.x) {
        const int i = I[a];
        sI[a] = i;
        if (i < 0 || i >= m || (a > 0 && I[a - 1] >= i)) bad = 1;
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) { set_status(&ctl->status, kDevBounds); ctl->done = 1; }
        return;
    }
    publish_rows(rowptr, sI, K, D, ctl, 0);
}

// ---- factorisation of the coupled rows --------------------------------
// RC (the mixed form's inner solve, which applies the factor in FP32 and needs
// no bit-exact factor): the diagonal holds 1 / L_jj, from CUDA's rsqrt, and
// every division by L_jj becomes a multiplication, so the serial chain of a
// column takes one rsqrt instead of a square root and a division per entry.
// The FP64 form (RC = false) keeps L_jj and IEEE square roots and divisions.
template <bool RC>
__device__ __forceinline__ double chol_diag(double d) { return RC ? rsqrt(d) : sqrt(d); }
template <bool RC>
__device__ __forceinline__ double chol_div(double v, double dg) { return RC ? v * dg : v / dg; }

// Right-looking packed Cholesky (zero multipliers skipped: the same numbers
// as the dense algorithm).  One block of threads.
template <bool RC>
__device__ void packed_cholesky(double *G, int nS, int *bad) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < nS; ++j) {
        if (threadIdx.x == 0) {
            double d = G[pidx(j, j)];
            if (!(d > 0.0)) { *bad = 1; d = 1.0; }
            G[pidx(j, j)] = chol_diag<RC>(d);
        }
        __syncthreads();
        const double l = G[pidx(j, j)];
        int any = 0;
        for (int i = j + 1 + threadIdx.x; i < nS; i += blockDim.x) {
            const double v = G[pidx(i, j)];
            if (v != 0.0) { G[pidx(i, j)] = chol_div<RC>(v, l); any = 1; }
        }
        if (!__syncthreads_or(any)) continue;
        for (int a = j + 1 + wid; a < nS; a += nw) {
            const double la = G[pidx(a, j)];
            if (la == 0.0) continue;
            for (int b = j + 1 + lane; b <= a; b += 32) {
                const double lb = G[pidx(b, j)];
                if (lb != 0.0) G[pidx(a, b)] = __fma_rn(-la, lb, G[pidx(a, b)]);
            }
        }
        __syncthreads();
    }
}

// Elimination tree of the coupled rows (nS <= kSymMax) from the Gram's
// nonzero pattern, as bitsets: col[j] = rows i > j where L_ij may be
// nonzero, row[i] = columns j < i where L_ij may be nonzero; level[j] = height
// of j above the leaves; columns sorted by level.  Returns the cost estimates
// (cycles) of the level-scheduled and the column-by-column factorisations.
constexpr int kSymMax = 256;
constexpr int kSymW = kSymMax / 32;

struct Sym {
    unsigned *col, *row;        // [kSymMax * kSymW]
    int16_t *level, *order, *lvl_off;   // [kSymMax], [kSymMax], [kSymMax + 1]
    int *eoff;                  // [kSymMax + 1] first off-diagonal entry of order[q]
};

__device__ __forceinline__ int bit_count(const unsigned *w) {
    int c = 0;
#pragma unroll
    for (int q = 0; q < kSymW; ++q) c += __popc(w[q]);
    return c;
}

__device__ void symbolic(const double *G, int nS, Sym S, int *s_nlev, int *s_use_levels) {
    __shared__ int s_cnt[kSymMax + 1];
    __shared__ long long s_cost_lvl, s_cost_col;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int q = tid; q < kSymMax * kSymW; q += blockDim.x) { S.col[q] = 0u; S.row[q] = 0u; }
    for (int j = tid; j < kSymMax; j += blockDim.x) { S.level[j] = 0; s_cnt[j] = 0; }
    if (tid == 0) s_cnt[kSymMax] = 0;
    __syncthreads();
    for (int q = tid; q < nS * (nS - 1) / 2; q += blockDim.x) {   // entry (i, j), j < i, packed by rows
        int i = (int)((sqrtf(8.0f * (float)q + 1.0f) + 1.0f) * 0.5f);
        while (i * (i - 1) / 2 > q) --i;
        while ((i + 1) * i / 2 <= q) ++i;
        const int j = q - i * (i - 1) / 2;
        if (G[pidx(i, j)] != 0.0) atomicOr(&S.col[j * kSymW + (i >> 5)], 1u << (i & 31));
    }
    __syncthreads();
    if (nS <= 64 && tid < 32) {
        // one warp, every column's structure in registers: lane l holds
        // columns l and l + 32 as 64-bit row masks (rows below the diagonal)
        // and their levels.  Column j's parent p is its first row; p takes
        // j's other rows (fill) and a level above j's.
        unsigned long long m0 = 0ull, m1 = 0ull;
        int lv0 = 0, lv1 = 0;
        if (lane < nS) m0 = ((unsigned long long)S.col[lane * kSymW + 1] << 32) | S.col[lane * kSymW];
        if (lane + 32 < nS)
            m1 = ((unsigned long long)S.col[(lane + 32) * kSymW + 1] << 32) | S.col[(lane + 32) * kSymW];
        for (int j = 0; j < nS; ++j) {
            const bool hi = j >= 32;                  // uniform across the warp
            const unsigned long long mj = __shfl_sync(0xffffffffu, hi ? m1 : m0, j & 31);
            const int lvj = __shfl_sync(0xffffffffu, hi ? lv1 : lv0, j & 31);
            if (mj) {
                const int p = __ffsll((long long)mj) - 1;
                const unsigned long long add = mj & ~(1ull << p);
                if ((p & 31) == lane) {
                    if (p < 32) { m0 |= add; lv0 = max(lv0, lvj + 1); }
                    else { m1 |= add; lv1 = max(lv1, lvj + 1); }
                }
            }
        }
        if (lane < nS) {
            S.col[lane * kSymW] = (unsigned)m0;
            S.col[lane * kSymW + 1] = (unsigned)(m0 >> 32);
            S.level[lane] = (int16_t)lv0;
        }
        if (lane + 32 < nS) {
            S.col[(lane + 32) * kSymW] = (unsigned)m1;
            S.col[(lane + 32) * kSymW + 1] = (unsigned)(m1 >> 32);
            S.level[lane + 32] = (int16_t)lv1;
        }
    } else if (tid < 32) {              // one warp: elimination tree and fill
        for (int j = 0; j < nS; ++j) {
            const unsigned w = lane < kSymW ? S.col[j * kSymW + lane] : 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, w != 0u);
            if (bal) {
                const int fw = __ffs(bal) - 1;
                const unsigned wf = __shfl_sync(0xffffffffu, w, fw);
                const int p = fw * 32 + __ffs(wf) - 1;
                if (lane < kSymW) {
                    unsigned add = w;
                    if (lane == (p >> 5)) add &= ~(1u << (p & 31));
                    S.col[p * kSymW + lane] |= add;
                }
                if (lane == 0) S.level[p] = (int16_t)max((int)S.level[p], (int)S.level[j] + 1);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // row structures (transpose) and level counts
    for (int q = tid; q < nS * kSymW; q += blockDim.x) {
        const int j = q / kSymW, wd = q % kSymW;
        unsigned w = S.col[q];
        while (w) {
            const int bitp = __ffs(w) - 1;
            w &= w - 1;
            const int i = wd * 32 + bitp;
            atomicOr(&S.row[i * kSymW + (j >> 5)], 1u << (j & 31));
        }
    }
    for (int j = tid; j < nS; j += blockDim.x) atomicAdd(&s_cnt[S.level[j]], 1);
    __syncthreads();
    if (tid == 0) {                     // levels are below nS
        int nl = 0, acc = 0;
        for (int L = 0; L < nS; ++L) {
            if (s_cnt[L]) nl = L + 1;
            const int c = s_cnt[L];
            S.lvl_off[L] = (int16_t)acc;
            acc += c;
            s_cnt[L] = 0;
        }
        for (int L = nS; L <= kSymMax; ++L) S.lvl_off[L] = (int16_t)acc;
        *s_nlev = nl;
        s_cost_lvl = 0;
        s_cost_col = 0;
    }
    __syncthreads();
    for (int j = tid; j < nS; j += blockDim.x) {
        const int L = S.level[j];
        S.order[S.lvl_off[L] + atomicAdd(&s_cnt[L], 1)] = (int16_t)j;
    }
    __syncthreads();
    {   // off-diagonal entries of each column, in level order
        __shared__ int sc2[33];
        int carry = 0;
        for (int base = 0; base < nS; base += blockDim.x) {
            const int q = base + tid;
            const int c = q < nS ? bit_count(S.col + S.order[q] * kSymW) : 0;
            int total;
            const int pre = block_exclusive_scan(c, sc2, &total);
            if (q < nS) S.eoff[q] = carry + pre;
            carry += total;
        }
        if (tid == 0) S.eoff[nS] = carry;
        __syncthreads();
    }
    // cost model (cycles): FP64 fma ~70, sqrt/div ~500 each, barrier ~100;
    // one warp per level
    {
        const int warp = tid >> 5, nwarps = blockDim.x >> 5;
        long long lvl = 0;
        for (int L = warp; L < *s_nlev; L += nwarps) {
            int mr = 0, mc = 0;
            for (int q = S.lvl_off[L] + lane; q < S.lvl_off[L + 1]; q += 32) {
                const int j = S.order[q];
                mr = max(mr, bit_count(S.row + j * kSymW));
                mc = max(mc, bit_count(S.col + j * kSymW));
            }
            for (int o = 16; o > 0; o >>= 1) {
                mr = max(mr, __shfl_xor_sync(0xffffffffu, mr, o));
                mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
            }
            lvl += (long long)(2 * mr + mc) * 90 + 2300;
        }
        if (lane == 0 && lvl) atomicAdd((unsigned long long *)&s_cost_lvl, (unsigned long long)lvl);
    }
    __syncthreads();
    if (tid == 0) {
        s_cost_col = (long long)nS * (1300 + 2 * 800);
        *s_use_levels = s_cost_lvl < s_cost_col;
    }
    __syncthreads();
}

// Left-looking Cholesky by tree levels: every column of a level at once.
// Entry (a, b) receives its updates L_aj L_bj over the columns j of row b in
// ascending order (the right-looking order).  Diagonals first (one thread per
// column: L_bb = sqrt(.)), then the off-diagonals (one thread per entry:
// L_ab = (.) / L_bb), so every FP64 instruction carries as many columns or
// entries as the level has.
__device__ __forceinline__ int kth_bit(const unsigned *w, int k) {
    for (int wd = 0; wd < kSymW; ++wd) {
        const int c = __popc(w[wd]);
        if (k < c) return wd * 32 + (int)__fns(w[wd], 0, k + 1);
        k -= c;
    }
    return -1;
}

template <bool RC>
__device__ void level_cholesky(double *G, int nS, Sym S, int nlev, int *bad) {
    for (int L = 0; L < nlev; ++L) {
        const int q0 = S.lvl_off[L], q1 = S.lvl_off[L + 1];
        for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const int b = S.order[q];
            const unsigned *rb = S.row + b * kSymW;
            double v = G[pidx(b, b)];
            for (int wd = 0; wd < kSymW; ++wd)
                for (unsigned w = rb[wd]; w; w &= w - 1) {
                    const int j = wd * 32 + __ffs(w) - 1;
                    const double lbj = G[pidx(b, j)];
                    v = __fma_rn(-lbj, lbj, v);
                }
            if (!(v > 0.0)) { *bad = 1; v = 1.0; }
            G[pidx(b, b)] = chol_diag<RC>(v);
        }
        __syncthreads();
        const int e0 = S.eoff[q0], e1 = S.eoff[q1];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            int lo = q0, hi = q1;                       // last q with eoff[q] <= e
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (S.eoff[mid] <= e) lo = mid; else hi = mid;
            }
            const int b = S.order[lo];
            const int a = kth_bit(S.col + b * kSymW, e - S.eoff[lo]);
            const unsigned *rb = S.row + b * kSymW;
            double v = G[pidx(a, b)];
            for (int wd = 0; wd < kSymW; ++wd)
                for (unsigned w = rb[wd]; w; w &= w - 1) {
                    const int j = wd * 32 + __ffs(w) - 1;
                    v = __fma_rn(-G[pidx(a, j)], G[pidx(b, j)], v);
                }
            G[pidx(a, b)] = chol_div<RC>(v, G[pidx(b, b)]);
        }
        __syncthreads();
    }
}

// z <- L^{-T} L^{-1} z on the coupled rows, by tree levels (forward:
// ascending levels, row sums over ascending columns; backward: descending
// levels, sums over descending rows), one thread per row.
template <bool RC>
__device__ void level_solve(const double *G, int nS, Sym S, int nlev, double *z) {
    for (int L = 0; L < nlev; ++L) {
        for (int q = S.lvl_off[L] + threadIdx.x; q < S.lvl_off[L + 1]; q += blockDim.x) {
            const int b = S.order[q];
            double v = z[b];
            const unsigned *rb = S.row + b * kSymW;
            for (int wd = 0; wd < kSymW; ++wd)
                for (unsigned w = rb[wd]; w; w &= w - 1) {
                    const int j = wd * 32 + __ffs(w) - 1;
                    v = __fma_rn(-G[pidx(b, j)], z[j], v);
                }
            z[b] = chol_div<RC>(v, G[pidx(b, b)]);
        }
        __syncthreads();
    }
    for (int L = nlev - 1; L >= 0; --L) {
        for (int q = S.lvl_off[L] + threadIdx.x; q < S.lvl_off[L + 1]; q += blockDim.x) {
            const int b = S.order[q];
            double v = z[b];
            const unsigned *cb = S.col + b * kSymW;
            for (int wd = kSymW - 1; wd >= 0; --wd)
                for (unsigned w = cb[wd]; w; ) {
                    const int hb = 31 - __clz(w);
                    w &= ~(1u << hb);
                    const int c = wd * 32 + hb;
                    v = __fma_rn(-G[pidx(c, b)], z[c], v);
                }
            z[b] = chol_div<RC>(v, G[pidx(b, b)]);
        }
        __syncthreads();
    }
}

// Column-by-column solves (right-looking order) with zero columns skipped.
template <bool RC>
__device__ void column_solve(const double *G, int nS, double *z, unsigned char *cz,
                             unsigned char *rz) {
    const int tid = threadIdx.x;
    for (int i = tid; i < nS; i += blockDim.x)
        for (int j = 0; j < i; ++j)
            if (G[pidx(i, j)] != 0.0) { cz[j] = 1; rz[i] = 1; }
    __syncthreads();
    for (int j = 0; j < nS; ++j) {                       // forward
        if (tid == 0) z[j] = chol_div<RC>(z[j], G[pidx(j, j)]);
        if (!cz[j]) continue;
        __syncthreads();
        const double zj = z[j];
        for (int i = j + 1 + tid; i < nS; i += blockDim.x) {
            const double lij = G[pidx(i, j)];
            if (lij != 0.0) z[i] = __fma_rn(-lij, zj, z[i]);
        }
        __syncthreads();
    }
    __syncthreads();
    for (int j = nS - 1; j >= 0; --j) {                  // backward
        if (tid == 0) z[j] = chol_div<RC>(z[j], G[pidx(j, j)]);
        if (!rz[j]) continue;
        __syncthreads();
        const double zj = z[j];
        for (int i = tid; i < j; i += blockDim.x) {
            const double lji = G[pidx(j, i)];
            if (lji != 0.0) z[i] = __fma_rn(-lji, zj, z[i]);
        }
        __syncthreads();
    }
    __syncthreads();
}

// ---- the factor by connected components of the coupled rows ------------------
// Rows of S that are not linked through shared columns, directly or through
// other rows, form independent diagonal blocks of G: their factors and solves
// never touch one another, and every entry of L and z receives, in the same
// ascending order, the updates of the whole-matrix right-looking factor and
// column solves (packed_cholesky, column_solve; zero multipliers skipped as
// there).  The components come from union-find over the Gram's nonzero pairs
// (roots hooked to the smaller root, then pointer jumping), their members
// listed ascending; one warp factors and solves each.  Returns false, with G
// and z untouched, when a component has more than kCompMax rows or the
// union-find did not settle; the caller then takes the other paths.
constexpr int kCompMax = 32;
template <bool RC>
__device__ bool component_factor(double *G, int nS, const unsigned long long *pkeys, int npk,
                                 const int16_t *spos, double *z, int *bad) {
    __shared__ int par[kSymMax], cid[kSymMax], csz[kSymMax], cst[kSymMax + 1], memb[kSymMax];
    __shared__ int sc[33];
    __shared__ int s_changed, s_max, s_nc;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int q = tid; q < nS; q += blockDim.x) { par[q] = q; csz[q] = 0; }
    if (tid == 0) { s_changed = 1; s_max = 0; }
    __syncthreads();
    for (int rnd = 0; rnd < 64 && s_changed; ++rnd) {
        __syncthreads();
        if (tid == 0) s_changed = 0;
        __syncthreads();
        for (int q = tid; q < npk; q += blockDim.x) {
            const unsigned long long pr = pkeys[q] >> 44;
            if (q > 0 && (pkeys[q - 1] >> 44) == pr) continue;   // one visit per row pair
            int u = spos[(int)(pr >> 10)], v = spos[(int)(pr & 1023)];
            while (par[u] != u) u = par[u];                   // par[x] <= x: the walk ends
            while (par[v] != v) v = par[v];
            if (u != v) {
                atomicMin(&par[max(u, v)], min(u, v));
                s_changed = 1;
            }
        }
        __syncthreads();
        for (int q = tid; q < nS; q += blockDim.x) {
            int r = par[q];
            while (par[r] != r) r = par[r];
            par[q] = r;
        }
        __syncthreads();
    }
    if (s_changed) return false;
    // components numbered by their roots, sizes, members ascending
    const int isroot = tid < nS && par[tid] == tid;
    int nc;
    const int pre = nS <= (int)blockDim.x ? block_exclusive_scan(isroot, sc, &nc) : 0;
    if (nS > (int)blockDim.x) return false;                   // not reached: nS <= kSymMax
    if (isroot) cid[tid] = pre;
    __syncthreads();
    for (int q = tid; q < nS; q += blockDim.x) atomicAdd(&csz[cid[par[q]]], 1);
    __syncthreads();
    const int size = tid < nc ? csz[tid] : 0;
    int tot;
    const int st = block_exclusive_scan(size, sc, &tot);
    if (tid < nc) cst[tid] = st;
    if (tid == 0) { cst[nc] = tot; s_nc = nc; }
    if (size) atomicMax(&s_max, size);
    __syncthreads();
    if (s_max > kCompMax) return false;
    for (int q = tid; q < nS; q += blockDim.x) {
        const int root = par[q];
        int rank = 0;
        for (int u = 0; u < q; ++u) rank += par[u] == root;
        memb[cst[cid[root]] + rank] = q;
    }
    __syncthreads();
    // one warp per component: right-looking factor, then the two solves
    for (int c = wid; c < s_nc; c += nw) {
        const int *M = memb + cst[c];
        const int n = cst[c + 1] - cst[c];
        for (int j = 0; j < n; ++j) {
            const int mj = M[j];
            if (lane == 0) {
                double d = G[pidx(mj, mj)];
                if (!(d > 0.0)) { *bad = 1; d = 1.0; }
                G[pidx(mj, mj)] = chol_diag<RC>(d);
            }
            __syncwarp();
            const double l = G[pidx(mj, mj)];
            int any = 0;
            for (int i = j + 1 + lane; i < n; i += 32) {
                const double v = G[pidx(M[i], mj)];
                if (v != 0.0) { G[pidx(M[i], mj)] = chol_div<RC>(v, l); any = 1; }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            __syncwarp();
            const int t = n - j - 1;                          // trailing rows j+1 .. n-1
            for (int e = lane; e < t * (t + 1) / 2; e += 32) {
                int ai = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);   // e = ai (ai + 1) / 2 + bi
                while (ai * (ai + 1) / 2 > e) --ai;
                while ((ai + 1) * (ai + 2) / 2 <= e) ++ai;
                const int bi = e - ai * (ai + 1) / 2;
                const int a = M[j + 1 + ai], b = M[j + 1 + bi];
                const double la = G[pidx(a, mj)];
                if (la == 0.0) continue;
                const double lb = G[pidx(b, mj)];
                if (lb != 0.0) G[pidx(a, b)] = __fma_rn(-la, lb, G[pidx(a, b)]);
            }
            __syncwarp();
        }
        for (int j = 0; j < n; ++j) {                        // forward
            const int mj = M[j];
            if (lane == 0) z[mj] = chol_div<RC>(z[mj], G[pidx(mj, mj)]);
            __syncwarp();
            const double zj = z[mj];
            for (int i = j + 1 + lane; i < n; i += 32) {
                const double lij = G[pidx(M[i], mj)];
                if (lij != 0.0) z[M[i]] = __fma_rn(-lij, zj, z[M[i]]);
            }
            __syncwarp();
        }
        for (int j = n - 1; j >= 0; --j) {                   // backward
            const int mj = M[j];
            if (lane == 0) z[mj] = chol_div<RC>(z[mj], G[pidx(mj, mj)]);
            __syncwarp();
            const double zj = z[mj];
            for (int i = lane; i < j; i += 32) {
                const double lji = G[pidx(mj, M[i])];
                if (lji != 0.0) z[M[i]] = __fma_rn(-lji, zj, z[M[i]]);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    return true;
}

// The factor step of the dynamic update, run by the last block of
// k_dyn_mark: coupled rows S (rows sharing a column inside I), the Gram on S
// from the shared columns only (each entry summed over ascending columns), its
// Cholesky, and y = (A_I A_I^T + mu I)^{-1} r_I by two triangular solves
// (y_a = (r_a / L_aa) / L_aa outside S).
template <typename T, bool MC>
__device__ void dyn_factor(const T *__restrict__ r, int K, Dyn D, Ctl *ctl,
                           unsigned long long *dsm, const Cols &cl) {
    constexpr bool RC = sizeof(T) == sizeof(float);   // the mixed form's inner solve
    __shared__ int s_nsh, s_npk, s_nS, s_bad, s_fill, s_fill2, s_nlev, s_uselev;
    __shared__ int sc[33];
    unsigned long long *sk = dsm;                                   // kShCap
    unsigned long long *pk = sk + kShCap;                           // kPairCap
    double *z = (double *)(pk + kPairCap);                          // kMaxDynRows
    double *Gs = z + kMaxDynRows;                                   // kGPack
    Sym S;
    S.col = (unsigned *)(Gs + kGPack);                              // kSymMax * kSymW
    S.row = S.col + kSymMax * kSymW;                                // kSymMax * kSymW
    S.level = (int16_t *)(S.row + kSymMax * kSymW);                 // kSymMax
    S.order = S.level + kSymMax;                                    // kSymMax
    S.lvl_off = S.order + kSymMax;                                  // kSymMax + 1
    S.eoff = (int *)(S.lvl_off + kSymMax + 2);                      // kSymMax + 1
    int16_t *spos = (int16_t *)(S.eoff + kSymMax + 2);              // kMaxDynRows
    int16_t *sidx = spos + kMaxDynRows;                             // kMaxDynRows
    unsigned char *flag = (unsigned char *)(sidx + kMaxDynRows);    // kMaxDynRows
    unsigned char *cz = flag + kMaxDynRows;
    unsigned char *rz = cz + kMaxDynRows;
    const int tid = threadIdx.x;
    const int E = ctl->dynE;
    const int nraw = ctl->dyn_nraw;
    for (int a = tid; a < K; a += blockDim.x) { flag[a] = 0; cz[a] = 0; rz[a] = 0; }
    if (tid == 0) { s_nsh = 0; s_npk = 0; s_bad = 0; s_fill = 0; s_fill2 = 0; }
    if (nraw > 2 * D.ecap || nraw >= (1 << 22)) {   // positions are packed in 22 bits
        if (tid == 0) set_status(&ctl->status, kDevBounds);
        return;
    }
    // shared entries (found with repeats by the grid pass): sort, drop repeats
    unsigned long long *keys = nraw <= kShCap ? sk : D.skeys;
    if (nraw <= kRankSortMax) {
        unsigned long long *tmp = (unsigned long long *)Gs;   // free until the Gram
        for (int q = tid; q < nraw; q += blockDim.x) tmp[q] = D.raw[q];
        __syncthreads();
        block_rank_sort<unsigned long long>(tmp, keys, nraw);
    } else {
        const int np = next_pow2(max(nraw, 1));
        for (int q = tid; q < np; q += blockDim.x) keys[q] = q < nraw ? D.raw[q] : ~0ull;
        __syncthreads();
        block_bitonic_sort(keys, np);
    }
    int nsh_run = 0;
    for (int base = 0; base < nraw; base += blockDim.x) {
        const int q = base + tid;
        unsigned long long kq = 0ull;
        int keep = 0;
        if (q < nraw) { kq = keys[q]; keep = q == 0 || keys[q - 1] != kq; }
        int total;
        const int pre = block_exclusive_scan(keep, sc, &total);
        if (keep) {
            keys[nsh_run + pre] = kq;                // stable compaction (target <= source)
            flag[D.erow[(unsigned)kq]] = 1;
        }
        nsh_run += total;
    }
    const int nsh = nsh_run;
    __syncthreads();
    // segments: shared-list position per column, Gram contributions
    // (pair (a_hi, a_lo) of rows, positions of both entries): 10+10+22+22 bits
    for (int q = tid; q < nsh; q += blockDim.x) {
        const unsigned c = (unsigned)(keys[q] >> 32);
        if (q > 0 && (unsigned)(keys[q - 1] >> 32) == c) continue;
        D.segpos[c] = q;
        int qe = q + 1;
        while (qe < nsh && (unsigned)(keys[qe] >> 32) == c) ++qe;
        const int L = qe - q;
        atomicAdd(&s_npk, L * (L - 1) / 2);
    }
    __syncthreads();
    const int npk = s_npk;
    unsigned long long *pkeys = npk <= kPairCap ? pk : D.pkeys;
    if (npk > kPairCap && npk > D.pcap) {
        if (tid == 0) set_status(&ctl->status, kDevBounds);
        return;
    }
    for (int q = tid; q < nsh; q += blockDim.x) {
        const unsigned c = (unsigned)(keys[q] >> 32);
        if (q > 0 && (unsigned)(keys[q - 1] >> 32) == c) continue;
        int qe = q + 1;
        while (qe < nsh && (unsigned)(keys[qe] >> 32) == c) ++qe;
        for (int u = q; u < qe; ++u)
            for (int w = u + 1; w < qe; ++w) {
                const unsigned a_lo = D.erow[(unsigned)keys[u]], a_hi = D.erow[(unsigned)keys[w]];
                pkeys[atomicAdd(&s_fill2, 1)] = ((unsigned long long)a_hi << 54) |
                                                ((unsigned long long)a_lo << 44) |
                                                ((unsigned long long)u << 22) | (unsigned long long)w;
            }
    }
    __syncthreads();
    if (npk <= kRankSortMax) {
        unsigned long long *tmp = (unsigned long long *)Gs;   // free until the Gram
        for (int q = tid; q < npk; q += blockDim.x) tmp[q] = pkeys[q];
        __syncthreads();
        block_rank_sort<unsigned long long>(tmp, pkeys, npk);
    } else {
        const int npp = next_pow2(max(npk, 1));
        for (int q = npk + tid; q < npp; q += blockDim.x) pkeys[q] = ~0ull;
        __syncthreads();
        block_bitonic_sort(pkeys, npp);
    }
    // coupled set S in ascending row order
    int cnt = 0;
    for (int base = 0; base < K; base += blockDim.x) {
        const int a = base + tid;
        const int f = a < K ? flag[a] : 0;
        int total;
        const int pre = block_exclusive_scan(f, sc, &total);
        if (a < K) {
            spos[a] = f ? (int16_t)(cnt + pre) : (int16_t)-1;
            if (f) sidx[cnt + pre] = (int16_t)a;
        }
        cnt += total;
    }
    if (tid == 0) s_nS = cnt;
    __syncthreads();
    const int nS = s_nS;
    double *G = nS <= kSPackedMax ? Gs : D.g;
    for (long long q = tid; q < (long long)nS * (nS + 1) / 2; q += blockDim.x) G[q] = 0.0;
    __syncthreads();
    for (int i = tid; i < nS; i += blockDim.x) G[pidx(i, i)] = D.gdiag[sidx[i]];
    // off-diagonal Gram entries: fused sums over the pair's shared columns, ascending
    for (int q = tid; q < npk; q += blockDim.x) {
        const unsigned long long pr = pkeys[q] >> 44;
        if (q > 0 && (pkeys[q - 1] >> 44) == pr) continue;
        double acc = 0.0;
        for (int u = q; u < npk && (pkeys[u] >> 44) == pr; ++u) {
            const unsigned qa = (unsigned)((pkeys[u] >> 22) & 0x3FFFFF), qb = (unsigned)(pkeys[u] & 0x3FFFFF);
            acc = __fma_rn(D.eval[(unsigned)keys[qb]], D.eval[(unsigned)keys[qa]], acc);
        }
        const int a_hi = (int)(pr >> 10), a_lo = (int)(pr & 1023);
        G[pidx(spos[a_hi], spos[a_lo])] = acc;
    }
    __syncthreads();
    for (int q = tid; q < nS; q += blockDim.x) z[q] = (double)r[rpos<MC>(cl, D.I[sidx[q]])];
    __syncthreads();
    bool by_comp = false;
    if (nS > 0 && nS <= kSymMax) by_comp = component_factor<RC>(G, nS, pkeys, npk, spos, z, &s_bad);
    if (by_comp) {
        if (tid == 0) s_uselev = 0;
    } else if (nS > 0) {
        if (nS <= kSymMax) symbolic(G, nS, S, &s_nlev, &s_uselev);
        else if (tid == 0) s_uselev = 0;
        __syncthreads();
        if (s_uselev) {
            level_cholesky<RC>(G, nS, S, s_nlev, &s_bad);
            level_solve<RC>(G, nS, S, s_nlev, z);
        } else {
            packed_cholesky<RC>(G, nS, &s_bad);
            column_solve<RC>(G, nS, z, cz, rz);
        }
    }
    for (int q = tid; q < nS; q += blockDim.x) D.y[sidx[q]] = z[q];
    if (keys != D.skeys)
        for (int q = tid; q < nsh; q += blockDim.x) D.skeys[q] = keys[q];
    if (tid == 0) {
        ctl->dyn_nsh = nsh;
        ctl->dyn_nS = nS;
        ctl->dyn_npair = npk;
        if (ctl->tr_dyn && ctl->iter < ctl->trace_cap) {
            int *t = ctl->tr_dyn + 4 * ctl->iter;
            t[0] = E; t[1] = nsh; t[2] = nS; t[3] = nS > 0 && nS <= kSymMax && s_uselev ? s_nlev : -1;
        }
        if (s_bad) set_status(&ctl->status, kDevNotSpd);
    }
}

// Gathers the nonzeros of A_I (row order), marks each column's lowest entry
// and entry count, forms ||A_i||^2 + mu; the last block factors.
// What the dynamic update needs to form the next iteration's draws ahead of
// them (cdf == nullptr: not formed).
struct Plan {
    const double *cdf;
    int k;
    const int *off, *s_ptr, *blk_nz;
    const long long *w_ptr;
};

// The next iteration's draws and their blocks' ranges, which depend on
// neither x nor r, formed by one block of the dynamic update while its last
// block factors (so that the next sampled updates start at once).  The
// residual-weighted draws are formed by k_static itself.
__device__ void plan_next(const Plan &pl, Ctl *ctl) {
    if (ctl->weighted || ctl->n_static > kPreDraws) return;
    __shared__ int taus[64], s_cnt[64];
    __shared__ double s_target[64];
    const int nst = ctl->n_static;
    const long long next = ctl->iter_base + ctl->iter + 1;
    sample_blocks_block<8>(pl.cdf, pl.k, ctl->seed, ctl->sysid, (uint64_t)next, nst, s_target, s_cnt, taus);
    const int a = threadIdx.x;
    if (a < nst) {
        const int tau = taus[a];
        ctl->pre_tau[a] = tau;
        ctl->pre_r0[a] = pl.off[tau];
        ctl->pre_s[a] = pl.off[tau + 1] - pl.off[tau];
        ctl->pre_sb[a] = pl.s_ptr[tau];
        ctl->pre_nS[a] = pl.s_ptr[tau + 1] - pl.s_ptr[tau];
        ctl->pre_wb[a] = pl.w_ptr[tau];
        ctl->pre_p0[a] = pl.blk_nz[tau];
        ctl->pre_pend[a] = pl.blk_nz[tau + 1];
    }
    __syncthreads();
    if (a == 0) {
        __threadfence();
        ctl->pre_it = next + 1;
    }
}

template <typename T, bool MC = false>
__global__ void __launch_bounds__(512, 1) k_dyn_mark(Mat<T> A, const T *__restrict__ r, Dyn D,
                                                  Ctl *ctl, int check_done, Cols cl, Plan pl) {
    extern __shared__ unsigned long long dsm_u64[];
    __shared__ int is_last;
    __shared__ unsigned s_tk;
    if constexpr (MC) {
        ctl += blockIdx.y;
        r += blockIdx.y * cl.rs;
        D = dyn_col(D, blockIdx.y);
    }
    if ((check_done && (ctl->done || ctl->halt)) || ctl->status) return;
    const int K = A.K;
    const int E = ctl->dynE;
    if (E > D.ecap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(&ctl->status, kDevBounds);
        return;
    }
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    const unsigned ep = *D.epoch;
    // ||A_i||^2 + mu, and y_a = (r_a / l) / l with l = sqrt(.) (the value for a
    // row outside the coupled set; the factor step overwrites coupled rows).
    // Rows go to different blocks so that their chains run on different SMs.
    for (int a = blockIdx.x + gridDim.x * threadIdx.x; a < K; a += gs) {
        const int i = D.I[a];
        double g = A.rn[i];                          // the row's fused chain, formed at set-up
        g = __dadd_rn(g, A.mu);
        D.gdiag[a] = g;
        if (!(g > 0.0)) { set_status(&ctl->status, kDevNotSpd); g = 1.0; }
        if constexpr (sizeof(T) == sizeof(float)) {    // mixed form: rsqrt, products
            const double il = rsqrt(g);
            D.y[a] = ((double)r[rpos<MC>(cl, i)] * il) * il;
        } else {
            const double l = sqrt(g);
            D.y[a] = ((double)r[rpos<MC>(cl, i)] / l) / l;
        }
    }
    for (int e = gt; e < E; e += gs) {
        int lo = 0, hi = K;                          // last a with estart[a] <= e
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (D.estart[mid] <= e) lo = mid; else hi = mid;
        }
        const int p = A.rowptr[D.I[lo]] + (e - D.estart[lo]);
        const int c = A.col[p];
        D.ecol[e] = c;
        D.eval[e] = (double)A.val[p];
        D.erow[e] = (uint16_t)lo;
        // first entry of a column this epoch owns it; any later entry marks the
        // column shared and records itself and the owner
        const unsigned long long mine = ((unsigned long long)ep << 32) | (unsigned)e;
        unsigned long long old = D.owner[c];
        for (;;) {
            if ((unsigned)(old >> 32) == ep) {
                D.shared[c] = ep;
                const int pos = atomicAdd(&ctl->dyn_nraw, 2);
                if (pos + 1 < 2 * D.ecap) {
                    D.raw[pos] = ((unsigned long long)(unsigned)c << 32) | (old & 0xffffffffull);
                    D.raw[pos + 1] = ((unsigned long long)(unsigned)c << 32) | (unsigned)e;
                }
                break;
            }
            const unsigned long long prev = atomicCAS(&D.owner[c], old, mine);
            if (prev == old) break;
            old = prev;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_tk = atomicAdd(&ctl->ticket, 1u);
        is_last = s_tk == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) {
        // the first block done plans the next draws while the last one factors
        if (s_tk == 0 && pl.cdf) plan_next(pl, ctl);
        return;
    }
    __threadfence();
    dyn_factor<T, MC>(r, K, D, ctl, dsm_u64, cl);
    if (threadIdx.x == 0) ctl->ticket = 0;
}

// End of an iteration: trace x, advance, loop condition (one block).
// A block of columns (grp != nullptr) sets the condition from all columns.
template <typename T>
__device__ void end_iteration(const T *x, int n, Ctl *ctl, int use_cond,
                              cudaGraphConditionalHandle hcond, int ld = 1,
                              unsigned *grp = nullptr) {
    if (ctl->tr_x && !ctl->halt && ctl->iter < ctl->trace_cap && sizeof(T) == sizeof(double))
        for (int c = threadIdx.x; c < n; c += blockDim.x)
            ctl->tr_x[ctl->iter * (long long)n + c] = (double)x[(long long)c * ld];
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ctl->halt) {
            const long long it = ctl->iter + 1;
            ctl->iter = it;
            if (ctl->done || ctl->status != 0 || it >= ctl->maxit) ctl->halt = 1;
        }
        if (grp) group_condition(ctl - blockIdx.y, gridDim.y, grp, use_cond, hcond);
        else if (use_cond) cudaGraphSetConditional(hcond, ctl->halt ? 0u : 1u);
    }
}

// x += A_I^T y: a column used by one row of I takes its single product; a
// shared column is summed over its rows in ascending order by the entry that
// owns it.  The last block clears the column marks and ends the iteration.
template <typename T, bool LOG = false, bool MC = false>
__global__ void __launch_bounds__(512) k_dyn_scatter(T *x, int n, Dyn D, Ctl *ctl, int count_iter,
                                                     int use_cond,
                                                     cudaGraphConditionalHandle hcond, Cols cl) {
    __shared__ int is_last;
    if constexpr (MC) {
        ctl += blockIdx.y;
        x += blockIdx.y;
        D = dyn_col(D, blockIdx.y);
    }
    const int ld = MC ? cl.ld : 1;
    unsigned *grp = MC ? cl.grp : nullptr;
    if (ctl->done || ctl->status || ctl->halt) {
        if (count_iter && blockIdx.x == 0) end_iteration<T>(x, n, ctl, use_cond, hcond, ld, grp);
        return;
    }
    const int E = ctl->dynE, nsh = ctl->dyn_nsh;
    const bool lg = LOG && count_iter;               // log x's changes
    const unsigned ep = *D.epoch;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (int e = gt; e < E; e += gs) {
        const int c = D.ecol[e];
        if (D.shared[c] != ep) {
            const T d = Ar<T>::fma(as<T>(D.eval[e]), as<T>(D.y[D.erow[e]]), T(0));
            x[(long long)c * ld] = Ar<T>::add(x[(long long)c * ld], d);
            if (lg) inc_log(ctl, c, (double)d);
        } else if ((unsigned)D.skeys[D.segpos[c]] == (unsigned)e) {
            T acc = T(0);
            for (int u = D.segpos[c]; u < nsh && (int)(D.skeys[u] >> 32) == c; ++u) {
                const unsigned e2 = (unsigned)D.skeys[u];
                acc = Ar<T>::fma(as<T>(D.eval[e2]), as<T>(D.y[D.erow[e2]]), acc);
            }
            x[(long long)c * ld] = Ar<T>::add(x[(long long)c * ld], acc);
            if (lg) inc_log(ctl, c, (double)acc);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) ctl->ticket = 0;
    __syncthreads();
    if (count_iter) end_iteration<T>(x, n, ctl, use_cond, hcond, ld, grp);
}

// ---- residual-weighted draws (not in the paper) -----------------------------
// Block t's weight is Pbar_t * rho_t, rho_t = sum of r_i^2 over its rows (one
// fused chain, rows ascending); the running sum is formed in chunks of
// kWChunk blocks (each chunk from zero, the chunk totals in order, each entry
// offset by the totals before its chunk).  The next static draws use it, or
// P's running sum if every weight is zero.
constexpr int kWChunk = 64;

__global__ void __launch_bounds__(256) k_wweights(const double *__restrict__ r,
                                                  const int *__restrict__ off, int k,
                                                  const double *__restrict__ pbar,
                                                  double *__restrict__ w, Ctl *ctl) {
    if (ctl->done || ctl->halt) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll 8
        for (int i = off[t]; i < off[t + 1]; ++i) s = __fma_rn(r[i], r[i], s);
        w[t] = __dmul_rn(pbar[t], s);
    }
}

__global__ void __launch_bounds__(1024) k_wcdf(const double *__restrict__ w, int k,
                                               double *__restrict__ wcdf,
                                               const double *__restrict__ cdf, Ctl *ctl) {
    __shared__ double tot[1024];
    if (ctl->done || ctl->halt) return;
    const int nc = (k + kWChunk - 1) / kWChunk;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int t1 = min(k, (c + 1) * kWChunk);
        double s = 0.0;
        for (int t = c * kWChunk; t < t1; ++t) {
            s = __dadd_rn(s, w[t]);
            wcdf[t] = s;
        }
        tot[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {                       // chunk offsets, in chunk order
        double off = 0.0;
        for (int c = 0; c < nc; ++c) {
            const double sc = tot[c];
            tot[c] = off;
            off = __dadd_rn(off, sc);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int t1 = min(k, (c + 1) * kWChunk);
        for (int t = c * kWChunk; t < t1; ++t) wcdf[t] = __dadd_rn(tot[c], wcdf[t]);
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl->scdf = wcdf[k - 1] > 0.0 ? wcdf : cdf;
}

// ---- the static updates of a dense A --------------------------------------
// A block of a dense A (s rows of n entries) is far larger than a stage, and
// one block of threads reading it row by row runs short of loads in flight.
// Each of the first kDenseStatic updates of an iteration therefore runs as
// three grid launches with the arithmetic of k_static's direct path: the
// block's residual (one lane per row, the row's chain in column order),
// y = W_tau r_tau, and x += A_tau^T y (one thread per column segment, rows
// ascending).  Every launch draws the same tau from the Philox stream.
constexpr int kDenseStatic = 3;

// The block's residual r_tau = b_tau - A_tau x, tiled for load parallelism:
// grid block g takes rows 32g..32g+31 of the block.  Its 256 threads copy a
// tile of those rows' next kSdCols columns (coalesced along the columns) into
// shared memory, transposed, while lane a of warp 0 runs row a's chain
// acc = fma(a_aj, x_j, acc) over the previous tile, columns ascending -- the
// operations of k_static's direct path in the same order.
constexpr int kSdCols = 256;     // = blockDim: thread t copies column t of each row

template <typename T>
__host__ __device__ constexpr size_t sd_rows_smem() { return ((size_t)kSdCols * 33 + kSdCols) * sizeof(T); }

template <typename T>
__global__ void __launch_bounds__(256) k_sd_rows_tiled(Mat<T> A, const T *__restrict__ b,
                                                      const T *__restrict__ x, T *rloc, Ctl *ctl,
                                                      int l) {
    extern __shared__ unsigned long long sd_dsm[];
    T *tile = (T *)sd_dsm;                        // [kSdCols][33]: column-major tile
    T *xs = tile + kSdCols * 33;                  // [kSdCols]
    __shared__ long long rbase[32];
    if (ctl->done || ctl->halt || l >= ctl->n_static) return;
    const long long it = ctl->iter_base + ctl->iter;
    const int tau = sample_block(ctl->scdf ? ctl->scdf : A.cdf, A.k, ctl->seed, ctl->sysid, (uint64_t)it, (uint64_t)l);
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctl->tr_tau && ctl->iter < ctl->trace_cap)
        ctl->tr_tau[ctl->iter * ctl->n_static + l] = tau;
    const int r0 = A.off[tau], s = A.off[tau + 1] - r0;
    const int row0 = blockIdx.x * 32;
    if (row0 >= s) return;
    const int rows = min(32, s - row0), n = A.n, tid = threadIdx.x;
    if (tid < 32) rbase[tid] = tid < rows ? (long long)A.rowptr[r0 + row0 + tid] : 0;
    __syncthreads();
    T pre[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) pre[u] = (u < rows && tid < n) ? A.val[rbase[u] + tid] : T(0);
    T acc = T(0);
    for (int c0 = 0; c0 < n; c0 += kSdCols) {
#pragma unroll
        for (int u = 0; u < 32; ++u) tile[tid * 33 + u] = pre[u];
        xs[tid] = c0 + tid < n ? x[c0 + tid] : T(0);
        __syncthreads();
        const int c1 = c0 + kSdCols;
        if (c1 < n) {                             // next tile in flight during the chain
#pragma unroll
            for (int u = 0; u < 32; ++u) pre[u] = (u < rows && c1 + tid < n) ? A.val[rbase[u] + c1 + tid] : T(0);
        }
        if (tid < rows) {
            const int jn = min(kSdCols, n - c0);
            for (int j = 0; j < jn; ++j) acc = Ar<T>::fma(tile[j * 33 + tid], xs[j], acc);
        }
        __syncthreads();
    }
    if (tid < rows) rloc[row0 + tid] = Ar<T>::sub(b[r0 + row0 + tid], acc);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_sd_apply(Mat<T> A, const T *__restrict__ rloc, T *y,
                                                   Ctl *ctl, int l) {
    if (ctl->done || ctl->halt || l >= ctl->n_static) return;
    const long long it = ctl->iter_base + ctl->iter;
    const int tau = sample_block(ctl->scdf ? ctl->scdf : A.cdf, A.k, ctl->seed, ctl->sysid, (uint64_t)it, (uint64_t)l);
    if (A.wood_ptr && A.wood_ptr[tau] >= 0) return;   // the s >= n form needs no W r
    const int r0 = A.off[tau], s = A.off[tau + 1] - r0;
    const int a = threadIdx.x;
    if (a >= s) return;
    const int pos = A.s_pos[r0 + a];
    if (pos < 0) {
        y[a] = Ar<T>::fma(A.w_diag[r0 + a], rloc[a], T(0));
    } else {
        const int sb = A.s_ptr[tau], nS = A.s_ptr[tau + 1] - sb;
        const T *Wr = A.w_ss + A.w_ptr[tau] + (long long)pos * nS;
        T acc2 = T(0);
#pragma unroll 8
        for (int q = 0; q < nS; ++q) acc2 = Ar<T>::fma(Wr[q], rloc[A.s_idx[sb + q]], acc2);
        y[a] = acc2;
    }
}

// x_c += sum over the block's rows a (ascending) of a_ac y_a: in a dense
// block every column holds every row, so the column-sorted copy's segment of
// column c is the rows in ascending order, and A itself (row-major) gives the
// same chain with loads coalesced across the threads' columns.  For a block in
// the s >= n form it forms g_c = sum over the rows of a_ac r_a into y instead
// (k_sd_wood applies V).
template <typename T>
__global__ void __launch_bounds__(256) k_sd_scatter(Mat<T> A, const T *__restrict__ rl, T *y, T *x,
                                                    Ctl *ctl, int l) {
    __shared__ long long rbase[kMaxBlockRows];
    if (ctl->done || ctl->halt || l >= ctl->n_static) return;
    const long long it = ctl->iter_base + ctl->iter;
    const int tau = sample_block(ctl->scdf ? ctl->scdf : A.cdf, A.k, ctl->seed, ctl->sysid, (uint64_t)it, (uint64_t)l);
    const int r0 = A.off[tau], s = A.off[tau + 1] - r0;
    for (int a = threadIdx.x; a < s; a += blockDim.x) rbase[a] = A.rowptr[r0 + a];
    __syncthreads();
    const bool wood = A.wood_ptr && A.wood_ptr[tau] >= 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.n; c += gridDim.x * blockDim.x) {
        T acc3 = T(0);
        if (wood) {
            for (int a = 0; a < s; ++a) acc3 = Ar<T>::fma(A.val[rbase[a] + c], rl[a], acc3);
            y[c] = acc3;
        } else {
            for (int a = 0; a < s; ++a) acc3 = Ar<T>::fma(A.val[rbase[a] + c], y[a], acc3);
            x[c] = Ar<T>::add(x[c], acc3);
        }
    }
}

// The s >= n form of a dense block: x_c += sum over d ascending of V_cd g_d,
// one thread per column (g from k_sd_scatter).
template <typename T>
__global__ void __launch_bounds__(256) k_sd_wood(Mat<T> A, const T *__restrict__ g, T *x, Ctl *ctl, int l) {
    if (ctl->done || ctl->halt || l >= ctl->n_static) return;
    const long long it = ctl->iter_base + ctl->iter;
    const int tau = sample_block(ctl->scdf ? ctl->scdf : A.cdf, A.k, ctl->seed, ctl->sysid, (uint64_t)it, (uint64_t)l);
    const long long wp = A.wood_ptr[tau];
    if (wp < 0) return;
    const T *V = A.wood + wp;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.n; c += gridDim.x * blockDim.x) {
        const T *Vr = V + (long long)c * A.n;
        T acc = T(0);
        for (int d = 0; d < A.n; ++d) acc = Ar<T>::fma(Vr[d], g[d], acc);
        x[c] = Ar<T>::add(x[c], acc);
    }
}

// ---- the dynamic update of a dense A -------------------------------------
// Every row of I holds every column, so all of I is coupled and the Gram is
// dense: G = A_I A_I^T + mu I (packed lower, D.g), each entry one fused chain
// over ascending columns as in the definition; one block factors it and
// solves (the same right-looking Cholesky and column-oriented solves as the
// sparse coupled set); x += A_I^T y, each column summed over ascending rows
// of I, then added.
constexpr int kGT = 16;         // Gram tile: kGT x kGT entries per block
constexpr int kGC = 64;         // columns staged per step

__global__ void __launch_bounds__(kGT * kGT) k_dyn_dense_gram(const double *__restrict__ val, int n,
                                                              int K, double mu, Dyn D, Ctl *ctl) {
    __shared__ double sa[kGT][kGC + 1], sb[kGT][kGC + 1];
    if (ctl->done || ctl->status || ctl->halt) return;
    int t = blockIdx.x, ti = 0;                 // tile (ti, tj), tj <= ti
    while (t > ti) { t -= ti + 1; ++ti; }
    const int tj = t, tid = threadIdx.x;
    const int ta = tid / kGT, tb = tid % kGT;
    const int a = ti * kGT + ta, b = tj * kGT + tb;
    double acc = 0.0;
    for (int c0 = 0; c0 < n; c0 += kGC) {
        const int w = min(kGC, n - c0);
        for (int q = tid; q < kGT * kGC; q += blockDim.x) {
            const int rr = q / kGC, cc = q % kGC;
            const int ra = ti * kGT + rr, rb = tj * kGT + rr;
            sa[rr][cc] = (ra < K && cc < w) ? val[(long long)D.I[ra] * n + c0 + cc] : 0.0;
            sb[rr][cc] = (rb < K && cc < w) ? val[(long long)D.I[rb] * n + c0 + cc] : 0.0;
        }
        __syncthreads();
        if (a < K && b <= a)
            for (int cc = 0; cc < w; ++cc) acc = __fma_rn(sa[ta][cc], sb[tb][cc], acc);
        __syncthreads();
    }
    if (a < K && b <= a) D.g[pidx(a, b)] = a == b ? __dadd_rn(acc, mu) : acc;
}

// ---- the dynamic Gram of a dense A on the tensor cores (mixed precision) --
// G = A_I A_I^T + mu I from the FP32 copy of A: TF32 products accumulated in
// FP32 by tcgen05.mma, in kTcRows x kTcRows tiles of the lower triangle.  Grid
// block (t, s) takes tile t and the s-th share of the column chunks (kTcCols
// columns each).  Per chunk it stages the tile's rows in shared memory as core
// matrices (see umma_desc), one thread issues the chunk's MMAs into a TMEM
// accumulator and commits them to an mbarrier, and the block waits before it
// stages the next chunk.  The accumulator is written as an FP32 partial tile;
// k_dyn_gram_reduce adds a tile's partials in split order in FP64, adds mu on
// the diagonal and writes the packed G that the FP64 Cholesky reads.
constexpr int kTcRows = 128;                             // tile edge: M = N = 128
constexpr int kTcCols = 128;                             // columns per chunk: 16 MMAs of K = 8
constexpr unsigned kTcOperand = kTcRows * kTcCols * 4;   // bytes of one operand chunk
constexpr unsigned kTcKStride = 128;                     // core matrices adjacent along K
constexpr unsigned kTcRowStride = (kTcCols / 4) * 128;   // adjacent 8-row groups

size_t gram_tc_smem() { return 2 * (size_t)kTcOperand + 1024; }

// Rows r0.. r0+127 of A_I, columns c0.. c0+127, into core-matrix order: slot q
// holds 4 consecutive values of row 8 (q / 256) + q % 8 at column group
// (q / 8) % 32, so a warp reads 8 rows x 64 contiguous bytes and writes 512
// contiguous bytes of shared memory.  Rows >= K and columns >= n are zero.
__device__ __forceinline__ void tc_stage(unsigned char *dst, const float *__restrict__ v32,
                                         const int *__restrict__ I, int K, long long n, int r0,
                                         long long c0, bool vec) {
    for (int q = threadIdx.x; q < kTcRows * kTcCols / 4; q += blockDim.x) {
        const int r8 = q & 7, kg = (q >> 3) & 31, g = q >> 8;
        const int row = r0 + g * 8 + r8;
        const long long col = c0 + kg * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < K) {
            const float *src = v32 + (long long)I[row] * n + col;
            if (vec && col + 3 < n) {
                v = *reinterpret_cast<const float4 *>(src);
            } else {
                if (col < n) v.x = src[0];
                if (col + 1 < n) v.y = src[1];
                if (col + 2 < n) v.z = src[2];
                if (col + 3 < n) v.w = src[3];
            }
        }
        *reinterpret_cast<float4 *>(dst + g * kTcRowStride + kg * kTcKStride + r8 * 16) = v;
    }
}

__global__ void __launch_bounds__(128) k_dyn_gram_tc(const float *__restrict__ v32, int n, int K, int S,
                                                     int vec, Dyn D, float *__restrict__ part, Ctl *ctl) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ unsigned long long bar;
    __shared__ unsigned tslot;
    __shared__ int s_fail;
    if (ctl->done || ctl->status || ctl->halt) return;
    const int t = blockIdx.x, s = blockIdx.y;
    int ti = 0, tj = t;
    while (tj > ti) { tj -= ti + 1; ++ti; }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sa = tc_smem, *sb = tc_smem + kTcOperand;
    const bool diag = ti == tj;
    const int nchunks = (n + kTcCols - 1) / kTcCols;
    const int per = (nchunks + S - 1) / S, ch0 = s * per, ch1 = min(nchunks, ch0 + per);
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_fail = 0;
    }
    if (warp == 0) tmem_alloc(&tslot, kTcRows);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const unsigned tmem = tslot;
    const unsigned idesc = idesc_tf32_f32(kTcRows, kTcRows);
    unsigned phase = 0;
    for (int c = ch0; c < ch1; ++c) {
        tc_stage(sa, v32, D.I, K, n, ti * kTcRows, (long long)c * kTcCols, vec != 0);
        if (!diag) tc_stage(sb, v32, D.I, K, n, tj * kTcRows, (long long)c * kTcCols, vec != 0);
        fence_proxy_async_smem();
        __syncthreads();
        tc_fence_after_sync();
        if (tid == 0) {
            const unsigned a0 = smem_u32(sa), b0 = smem_u32(diag ? sa : sb);
            for (int k = 0; k < kTcCols / 8; ++k)      // K = 8 TF32 values = 2 core matrices
                mma_tf32(tmem, umma_desc(a0 + 256u * k, kTcKStride, kTcRowStride),
                         umma_desc(b0 + 256u * k, kTcKStride, kTcRowStride), idesc,
                         (c > ch0 || k > 0) ? 1u : 0u);
            mma_commit(&bar);
        }
        if (!mbar_wait_bounded(&bar, phase, kWaitTries)) atomicOr(&s_fail, 1);
        phase ^= 1u;
        __syncthreads();                               // the chunk's operands are free again
        if (s_fail) break;
    }
    if (s_fail && tid == 0) mbar_wait_bounded(&bar, phase ^ 1u, kWaitTries);   // the MMAs in flight
    tc_fence_after_sync();
    if (!s_fail) {
        float *P = part + ((long long)t * S + s) * kTcRows * kTcRows + (long long)(warp * 32 + lane) * kTcRows;
        for (int c0 = 0; c0 < kTcRows; c0 += 32) {
            unsigned v[32];
            if (ch1 > ch0) {
                tmem_ld_32cols(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4 *>(P + c0 + j) = make_float4(
                    __uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                    __uint_as_float(v[j + 3]));
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTcRows);
    if (s_fail && tid == 0) set_status(&ctl->status, kDevTimeout);
}

// Packed entry q = a (a + 1) / 2 + b of G: the S partials of its tile, added
// in split order in FP64, plus mu on the diagonal.
__global__ void __launch_bounds__(256) k_dyn_gram_reduce(const float *__restrict__ part, int K, int S,
                                                         double mu, Dyn D, Ctl *ctl) {
    if (ctl->done || ctl->status || ctl->halt) return;
    const long long total = (long long)K * (K + 1) / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        int a = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
        while ((long long)a * (a + 1) / 2 > q) --a;
        while ((long long)(a + 1) * (a + 2) / 2 <= q) ++a;
        const int b = (int)(q - (long long)a * (a + 1) / 2);
        const int ti = a / kTcRows, tj = b / kTcRows, t = ti * (ti + 1) / 2 + tj;
        const float *P = part + (long long)t * S * kTcRows * kTcRows + (long long)(a % kTcRows) * kTcRows +
                         (b % kTcRows);
        double g = 0.0;
        for (int s2 = 0; s2 < S; ++s2) g += (double)P[(long long)s2 * kTcRows * kTcRows];
        D.g[q] = a == b ? g + mu : g;
    }
}

// Blocked factor of the dense Gram: panels of kPW columns.  The panel kernel
// factors the panel's columns, right-looking inside the panel, and carries the
// forward solve for them (z is the panel's extra column); the trailing kernel
// (many blocks) applies the panel's columns to every later entry, in
// ascending column order; the backward solve runs last in one block.  Every
// entry sees the operations of the one-block right-looking factor and
// column-oriented solves in the same order (zero multipliers skipped alike).
constexpr int kPW = 32;

// ---- the dynamic block in the n x n form (K >= n; Lemma 1) ----------------
// G = A_I^T A_I + mu I, h = A_I^T r_I, y = G^{-1} h by the blocked Cholesky and
// its solves (size n, z starting at h), then x_c += y_c.  The rows of I are
// first laid out as a dense K x n array (dw; unstored entries zero), so the
// column sums run over the rows in ascending order as in the definition.
__global__ void __launch_bounds__(256) k_dynw_rows(const int *__restrict__ rowptr, const int *__restrict__ col,
                                                   const double *__restrict__ val, int n, int K, Dyn D,
                                                   double *dw, Ctl *ctl) {
    if (ctl->done || ctl->status || ctl->halt) return;
    const int lane = threadIdx.x & 31;
    for (int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < K; a += (gridDim.x * blockDim.x) >> 5) {
        const int row = D.I[a];
        for (int p = rowptr[row] + lane; p < rowptr[row + 1]; p += 32) dw[(long long)a * n + col[p]] = val[p];
    }
}

// Packed lower entry q = c (c + 1) / 2 + d of G = A_I^T A_I + mu I: one fused
// chain over the K rows ascending, then mu on the diagonal.
__global__ void __launch_bounds__(256) k_dynw_gram(const double *__restrict__ dw, int n, int K, double mu, Dyn D,
                                                   Ctl *ctl) {
    if (ctl->done || ctl->status || ctl->halt) return;
    const long long total = (long long)n * (n + 1) / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        int c = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
        while ((long long)c * (c + 1) / 2 > q) --c;
        while ((long long)(c + 1) * (c + 2) / 2 <= q) ++c;
        const int d = (int)(q - (long long)c * (c + 1) / 2);
        double g = 0.0;
        for (int a = 0; a < K; ++a) g = __fma_rn(dw[(long long)a * n + c], dw[(long long)a * n + d], g);
        D.g[q] = c == d ? __dadd_rn(g, mu) : g;
    }
}

// h_c = sum over the K rows ascending of a_{I_a c} r_{I_a} (one fused chain).
template <typename T>
__global__ void __launch_bounds__(256) k_dynw_rhs(const double *__restrict__ dw, const T *__restrict__ r, int n,
                                                  int K, Dyn D, double *hz, Ctl *ctl) {
    if (ctl->done || ctl->status || ctl->halt) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double g = 0.0;
        for (int a = 0; a < K; ++a) g = __fma_rn(dw[(long long)a * n + c], (double)r[D.I[a]], g);
        hz[c] = g;
    }
}

// Panel j0 with its rows spread over the grid.  Every grid block factors the
// w x w diagonal block and forward-solves its part of z in shared memory (the
// same operations in every block), with warps 1..7; lane t of warp 0 of block
// g takes row i = w + 32g + t below the diagonal block and keeps its w
// entries of L and its z entry in registers, in step with the diagonal block:
// at column jj the row's entry is divided by L_jj,jj and then applied to the
// row's later entries and to z_i.  Every entry therefore receives the
// operations of the one-block right-looking factor in the same order, while
// the divisions of a column run side by side.  The last block to finish
// (ticket) writes the diagonal block back, after every block has read it.
template <typename T>
__global__ void __launch_bounds__(256) k_dchol_panel_rows(const T *__restrict__ r, int K, int j0, Dyn D,
                                                          Ctl *ctl, const double *__restrict__ z0) {
    __shared__ double Ld[kPW][kPW + 1];
    __shared__ double zd[kPW];
    __shared__ int s_bad, is_last;
    if (ctl->done || ctl->status || ctl->halt) return;
    const int w = min(kPW, K - j0), nr = K - j0, tid = threadIdx.x;
    const int dt = tid - 32, dn = blockDim.x - 32;   // diagonal-block threads (warps 1..)
    for (int q = tid; q < w * w; q += blockDim.x) {
        const int i = q / w, jj = q % w;
        Ld[i][jj] = i >= jj ? D.g[pidx(j0 + i, j0 + jj)] : 0.0;
    }
    // z starts as r_I (or as z0, the n x n form's A_I^T r_I)
    for (int i = tid; i < w; i += blockDim.x)
        zd[i] = j0 == 0 ? (z0 ? z0[i] : (double)r[D.I[i]]) : D.y[j0 + i];
    // this block's rows below the diagonal block: read before anything is written
    const int i = w + blockIdx.x * 32 + tid;
    const bool own = tid < 32 && i < nr;
    double Lr[kPW];
#pragma unroll
    for (int jj = 0; jj < kPW; ++jj) Lr[jj] = (own && jj < w) ? D.g[pidx(j0 + i, j0 + jj)] : 0.0;
    double zi = own ? (j0 == 0 ? (z0 ? z0[i] : (double)r[D.I[i]]) : D.y[j0 + i]) : 0.0;
    if (tid == 0) s_bad = 0;
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < kPW; ++jj) {
        if (jj >= w) break;
        if (tid == 32) {
            double d = Ld[jj][jj];
            if (!(d > 0.0)) { s_bad = 1; d = 1.0; }
            Ld[jj][jj] = sqrt(d);
        }
        __syncthreads();
        const double l = Ld[jj][jj];
        double v = 0.0;
        if (dt >= 0) {
            for (int q = jj + 1 + dt; q < w; q += dn) {
                const double u = Ld[q][jj];
                if (u != 0.0) Ld[q][jj] = u / l;
            }
            if (dt == dn - 1) zd[jj] = zd[jj] / l;
        } else if (own) {
            v = Lr[jj];
            if (v != 0.0) v = v / l;
            Lr[jj] = v;
        }
        __syncthreads();
        const double wj = zd[jj];
        if (dt >= 0) {
            for (int q = dt; q < (w - jj - 1) * w; q += dn) {
                const int jj2 = jj + 1 + q / w, a = q % w;
                if (a < jj2) continue;
                const double la = Ld[a][jj], lb = Ld[jj2][jj];
                if (la != 0.0 && lb != 0.0) Ld[a][jj2] = __fma_rn(-la, lb, Ld[a][jj2]);
            }
            for (int q = jj + 1 + dt; q < w; q += dn) {
                const double lij = Ld[q][jj];
                if (lij != 0.0) zd[q] = __fma_rn(-lij, wj, zd[q]);
            }
        } else if (own) {
#pragma unroll
            for (int j2 = jj + 1; j2 < kPW; ++j2) {
                const double bb = Ld[j2][jj];
                if (j2 < w && v != 0.0 && bb != 0.0) Lr[j2] = __fma_rn(-v, bb, Lr[j2]);
            }
            if (v != 0.0) zi = __fma_rn(-v, wj, zi);
        }
        __syncthreads();
    }
    if (own) {
#pragma unroll
        for (int jj = 0; jj < kPW; ++jj)
            if (jj < w) D.g[pidx(j0 + i, j0 + jj)] = Lr[jj];
        D.y[j0 + i] = zi;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    for (int q = tid; q < w * w; q += blockDim.x) {
        const int a2 = q / w, jj = q % w;
        if (a2 >= jj) D.g[pidx(j0 + a2, j0 + jj)] = Ld[a2][jj];
    }
    for (int a2 = tid; a2 < w; a2 += blockDim.x) D.y[j0 + a2] = zd[a2];
    if (tid == 0) {
        ctl->ticket = 0;
        if (s_bad) set_status(&ctl->status, kDevNotSpd);
    }
}

// G[a][b] -= L[a][j] L[b][j] for the panel's columns j (ascending), over the
// trailing entries j1 <= b <= a < K, in 16 x 16 tiles.
__global__ void __launch_bounds__(256) k_dchol_trail(int K, int j0, Dyn D, Ctl *ctl) {
    __shared__ double La[16][kPW + 1], Lb[16][kPW + 1];
    if (ctl->done || ctl->status || ctl->halt) return;
    const int w = min(kPW, K - j0), j1 = j0 + w;
    int t = blockIdx.x, ti = 0;
    while (t > ti) { t -= ti + 1; ++ti; }
    const int tj = t, tid = threadIdx.x;
    for (int q = tid; q < 16 * w; q += blockDim.x) {
        const int rr = q / w, jj = q % w;
        const int a = j1 + ti * 16 + rr, b = j1 + tj * 16 + rr;
        La[rr][jj] = a < K ? D.g[pidx(a, j0 + jj)] : 0.0;
        Lb[rr][jj] = b < K ? D.g[pidx(b, j0 + jj)] : 0.0;
    }
    __syncthreads();
    const int ta = tid / 16, tb = tid % 16;
    const int a = j1 + ti * 16 + ta, b = j1 + tj * 16 + tb;
    if (a >= K || b > a) return;
    double g = D.g[pidx(a, b)];
    for (int jj = 0; jj < w; ++jj) {
        const double la = La[ta][jj], lb = Lb[tb][jj];
        if (la != 0.0 && lb != 0.0) g = __fma_rn(-la, lb, g);
    }
    D.g[pidx(a, b)] = g;
}

// y = L^{-T} w (column-oriented, columns descending; row j of L is contiguous).
__global__ void __launch_bounds__(1024) k_dchol_back(int K, Dyn D, Ctl *ctl) {
    __shared__ double z[kMaxDynRows];
    if (ctl->done || ctl->status || ctl->halt) return;
    const int tid = threadIdx.x;
    for (int q = tid; q < K; q += blockDim.x) z[q] = D.y[q];
    __syncthreads();
    for (int j = K - 1; j >= 0; --j) {
        if (tid == 0) z[j] = z[j] / D.g[pidx(j, j)];
        __syncthreads();
        const double zj = z[j];
        for (int i = tid; i < j; i += blockDim.x) {
            const double lji = D.g[pidx(j, i)];
            if (lji != 0.0) z[i] = __fma_rn(-lji, zj, z[i]);
        }
        __syncthreads();
    }
    for (int q = tid; q < K; q += blockDim.x) D.y[q] = z[q];
}

template <typename T>
__device__ __forceinline__ T dense_value(const double *v64, const float *v32, long long p);
template <>
__device__ __forceinline__ double dense_value<double>(const double *v64, const float *, long long p) {
    return v64[p];
}
template <>
__device__ __forceinline__ float dense_value<float>(const double *, const float *v32, long long p) {
    return v32[p];
}

template <typename T>
__global__ void __launch_bounds__(256) k_dyn_dense_scatter(const double *__restrict__ v64,
                                                           const float *__restrict__ v32, T *x, int n,
                                                           int K, Dyn D, Ctl *ctl, int count_iter,
                                                           int use_cond,
                                                           cudaGraphConditionalHandle hcond, int wood) {
    __shared__ int is_last;
    if (ctl->done || ctl->status || ctl->halt) {
        if (count_iter && blockIdx.x == 0) end_iteration<T>(x, n, ctl, use_cond, hcond);
        return;
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        if (wood) {                           // the n x n form: x_c += y_c
            x[c] = Ar<T>::add(x[c], as<T>(D.y[c]));
            continue;
        }
        T acc = T(0);
        for (int a = 0; a < K; ++a)
            acc = Ar<T>::fma(dense_value<T>(v64, v32, (long long)D.I[a] * n + c), as<T>(D.y[a]), acc);
        x[c] = Ar<T>::add(x[c], acc);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) ctl->ticket = 0;
    __syncthreads();
    if (count_iter) end_iteration<T>(x, n, ctl, use_cond, hcond);
}

// Sampler probe (single-step API).
__global__ void k_sample_probe(const double *cdf, int k, uint64_t seed, uint64_t sysid,
                               long long it, long long l, long long *out) {
    *out = sample_block(cdf, k, seed, sysid, (uint64_t)it, (uint64_t)l);
}

// -------------------------------------------------- mixed precision
// Iterative refinement around the FP32 form of the iteration (the loop state
// of the FP64 outer loop is `out`, of the FP32 inner solve `in`):
//   r = b - A x in FP64 (k_residual, finalize 3: the convergence test only);
//   k_inner_prep: b32 = fl32(r), d32 = 0, the inner loop state;
//   inner ROR-BK iterations on A d = b32 in FP32 until ||b32 - A d|| <=
//     inner_tol ||b32|| or the inner cap (the block Gram Cholesky stays FP64);
//   k_outer_update: x += d in FP64.
// The Philox counter runs on across refinements (inner iteration t of the
// refinement that starts after T inner iterations in total uses counter
// start_iter + T + t).
__global__ void __launch_bounds__(256) k_inner_prep(const double *__restrict__ r64, int m,
                                                    float *__restrict__ b32, float *__restrict__ d32,
                                                    int n, double *partials, Ctl *out, Ctl *in,
                                                    int use_cond, cudaGraphConditionalHandle hcond) {
    __shared__ double red[32];
    __shared__ int is_last;
    if (out->done || out->status || out->halt) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hcond, 0u);
        return;
    }
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const float v = (float)r64[i];
        b32[i] = v;
        acc = __fma_rn((double)v, (double)v, acc);
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) d32[c] = 0.f;
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc;
        __threadfence();
        is_last = atomicAdd(&out->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += partials[i];
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) {
        out->ticket = 0;
        const double bn = sqrt(tot);
        const long long left = out->maxit - out->iter;
        in->bnorm = bn;
        in->iter = 0;
        in->maxit = left < out->inner_maxit ? left : out->inner_maxit;
        in->iter_base = out->iter_base + out->iter;
        in->seed = out->seed;
        in->sysid = out->sysid;
        in->n_static = out->n_static;
        in->tol = out->inner_tol;
        in->rr = 0.0;
        in->rrn = 1.0;
        in->done = bn == 0.0;
        in->halt = !(bn > 0.0 && in->maxit > 0);
        in->status = 0;
        in->ticket = 0;
        in->pre_it = 0;
        in->n_in = 0;
        in->n_eq = 0;
        in->trace_cap = 0;
        in->tr_tau = nullptr;
        in->tr_rrn = nullptr;
        in->tr_I = nullptr;
        in->tr_x = nullptr;
        in->tr_dyn = nullptr;
        in->inc = out->inc;            // incremental residual: same log, exact first residual
        in->inc_refresh = out->inc_refresh;
        in->inc_full = 1;
        in->inc_count = 0;
        in->nlog = 0;
        in->log_full = 0;
        in->log_cap = out->log_cap;
        in->log_col = out->log_col;
        in->log_val = out->log_val;
        in->fault = out->fault;
        if (use_cond) cudaGraphSetConditional(hcond, in->halt ? 0u : 1u);
    }
}

__global__ void __launch_bounds__(256) k_outer_update(double *__restrict__ x, const float *__restrict__ d32,
                                                      int n, Ctl *out, Ctl *in, int use_cond,
                                                      cudaGraphConditionalHandle hcond) {
    __shared__ int is_last;
    const bool active = !(out->done || out->status || out->halt);
    if (active)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
            x[c] = __dadd_rn(x[c], (double)d32[c]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&out->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    out->ticket = 0;
    if (active) {
        out->iter += in->iter;
        out->outer += 1;
        if (in->status) set_status(&out->status, in->status);
        if (in->iter == 0 || out->iter >= out->maxit) out->halt = 1;
    }
    if (out->done || out->status) out->halt = 1;
    if (use_cond) cudaGraphSetConditional(hcond, out->halt ? 0u : 1u);
}

// ------------------------------------------------- a block of right-hand sides
// rorbk_multi_create: nr right-hand sides of one system, each solved exactly
// as rorbk_solve would solve it alone (its own draws, top-K set, dynamic
// update and stopping test), with X (n x nr) and B (m x nr) row-major.  The
// residual R = B - A X is one pass over A for all columns (k_mres): each
// gather of x brings a whole row of X (nr contiguous values) instead of one
// value per 32-byte sector, so A is read once for nr columns.  Its columns are
// written in the SELL copy's row order (position p = 32 s + l holds row
// sell.row[p]), coalesced through a per-warp staging tile.  The other steps run
// the one-column kernels with one grid row (blockIdx.y) per column.

// Loads that keep their line in L2 ahead of streamed data: an L2 eviction
// policy made with createpolicy (evict_last for the whole access) passed as
// a cache hint on the load.  The block residual gathers rows of X this way, so
// X stays resident in L2 while A, B and R stream past it (evict-first).
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
template <typename T, int VEC>
__device__ __forceinline__ VecT<T, VEC> vload_keep(const T *p, unsigned long long pol) {
    VecT<T, VEC> r;
    if constexpr (sizeof(T) == 4 && VEC == 4) {
        asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
                     : "l"(p), "l"(pol));
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                     : "=f"(r.v[0]), "=f"(r.v[1]) : "l"(p), "l"(pol));
    } else if constexpr (sizeof(T) == 8 && VEC == 2) {
        asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                     : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(p), "l"(pol));
    } else {
        r = vload<T, VEC>(p);
    }
    return r;
}

// k_begin for a block of columns: ||b_j||, x_j = x0_j or 0, loop state; the
// last column sets the WHILE condition.  Grid (1, nr).
__global__ void k_mr_begin(const double *__restrict__ b, int m, const double *__restrict__ x0,
                           double *__restrict__ x, int n, Ctl *ctl0, int nr, unsigned *grp,
                           int use_cond, cudaGraphConditionalHandle hcond) {
    __shared__ double red[32];
    __shared__ double bn;
    const int jc = blockIdx.y;
    Ctl *ctl = ctl0 + jc;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double v = b[(long long)i * nr + jc];
        s = __fma_rn(v, v, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) bn = sqrt(s);
    __syncthreads();
    const bool zero = bn == 0.0 || x0 == nullptr || !ctl->has_x0;
    for (int c = threadIdx.x; c < n; c += blockDim.x)
        x[(long long)c * nr + jc] = zero ? 0.0 : x0[(long long)c * nr + jc];
    if (threadIdx.x == 0) {
        const bool finite = isfinite(bn);
        ctl->bnorm = bn;
        ctl->iter = 0;
        ctl->rr = 0.0;
        ctl->rrn = bn == 0.0 ? 0.0 : 1.0;
        ctl->done = bn == 0.0;
        ctl->halt = !(finite && bn > 0.0 && ctl->maxit > 0);
        ctl->status = finite ? 0 : kDevNumeric;
        ctl->ticket = 0;
        ctl->n_in = 0;
        ctl->n_eq = 0;
        ctl->outer = 0;
        group_condition(ctl0, nr, grp, use_cond, hcond);
    }
}

// R = B - A X for NR columns over the SELL-32 copy of A.  A warp takes a
// slice of 32 rows.  Its lanes load the slice's column indices and values
// coalesced (lane l for row l, the next entries in flight during the current
// ones).  For entry j, lane l then works on VEC consecutive columns
// (l % LPR) * VEC .. + VEC-1 of rows g * RPS + l / LPR (g = 0 .. LPR-1),
// taking each row's index and value by a warp shuffle, so one 16-byte load
// brings a lane's VEC values of a row of X and the LPR lanes of a row read the
// whole row (NR contiguous values) -- a handful of load instructions per
// entry of the slice for all NR columns.  Each (row, column) is one chain over
// the row's entries in stored order: the arithmetic of k_residual, column by
// column.  Entry j is present for the first cnt_j rows (lengths fall within a
// slice).  The sums of squares per column are formed per lane (FP32 inner
// residual: per slice in FP32, then in FP64), per block in warp order and over
// the blocks in block order by the last block, which runs the stopping test of
// every column still running (finalize 1: the iteration's, 3: the outer
// residual of the mixed form's refinement, 2: ||r_j||^2 only).
template <typename T>
struct SqAcc;
template <>
struct SqAcc<double> {
    using type = double;
    static __device__ __forceinline__ double add(double s, double r) { return __fma_rn(r, r, s); }
};
template <>
struct SqAcc<float> {
    using type = float;
    static __device__ __forceinline__ float add(float s, float r) { return __fmaf_rn(r, r, s); }
};

constexpr int kMrWarps = 8;

// The FP32 block residual of an iteration also forms the first radix level
// of every column's top-K (the exponent histogram of the |r| keys, which
// k_topk_hist1 forms for one column): an FP32 value's key exponent is 0 (for
// 0) or one of kF32Exp values from kF32Exp0 on, so a column needs kF32Bins
// shared-memory bins instead of kHistBins.
constexpr int kF32Exp0 = 874;        // FP64 exponent of the smallest FP32 subnormal
constexpr int kF32Exp = 1151 - kF32Exp0 + 1;
constexpr int kF32Bins = kF32Exp + 2;   // + zero, + Inf/NaN

template <typename T, int NR>
__host__ __device__ constexpr size_t mres_smem_bytes() {
    return (size_t)kMrWarps * 32 * (NR + 1) * sizeof(T) +
           (sizeof(T) == 4 ? (size_t)NR * kF32Bins * sizeof(unsigned) : 0);
}

__device__ __forceinline__ int f32_bin(unsigned e) {    // e: FP64 exponent of an FP32 |r|
    return e == 0u ? 0 : (e >= (unsigned)kF32Exp0 && e < (unsigned)(kF32Exp0 + kF32Exp)) ? (int)e - kF32Exp0 + 1
                                                                                      : kF32Bins - 1;
}
__device__ __forceinline__ unsigned f32_bin_exp(int bin) {
    return bin == 0 ? 0u : bin == kF32Bins - 1 ? 2047u : (unsigned)(bin - 1 + kF32Exp0);
}

// select_bin for one warp over the histogram of an FP32 residual's keys,
// whose nonzero bins are among the kF32Bins FP32 exponents: the largest bin b
// with sum_{j >= b} h[j] >= need and the count strictly above it.  Lane l
// holds compressed bins kF32Bins - 1 - kSelPer l - u (u < kSelPer, descending
// keys) in registers; zeroes them in h.
constexpr int kSelPer = (kF32Bins + 31) / 32;
__device__ void warp_select_bin_f32(unsigned *h, int need, int *bin_out, int *above_out) {
    const int lane = threadIdx.x & 31;
    int c[kSelPer];
    int tot = 0;
#pragma unroll
    for (int u = 0; u < kSelPer; ++u) {
        const int q = kF32Bins - 1 - kSelPer * lane - u;
        c[u] = q >= 0 ? (int)h[f32_bin_exp(q)] : 0;
        tot += c[u];
    }
    int pre = tot;                                  // inclusive scan, lanes in order
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    pre -= tot;                                     // keys in bins above this lane's
    int bin = 0, above = 0, found = 0, run = pre;
#pragma unroll
    for (int u = 0; u < kSelPer; ++u) {
        if (!found && run < need && run + c[u] >= need) {
            bin = (int)f32_bin_exp(kF32Bins - 1 - kSelPer * lane - u);
            above = run;
            found = 1;
        }
        run += c[u];
    }
    const unsigned who = __ballot_sync(0xffffffffu, found);
    const int src = who ? __ffs(who) - 1 : 0;
    bin = __shfl_sync(0xffffffffu, bin, src);
    above = __shfl_sync(0xffffffffu, above, src);
#pragma unroll
    for (int u = 0; u < kSelPer; ++u) {
        const int q = kF32Bins - 1 - kSelPer * lane - u;
        if (q >= 0) h[f32_bin_exp(q)] = 0u;
    }
    *bin_out = who ? bin : 0;
    *above_out = who ? above : 0;
}

// Resident blocks per SM the register budget is set for.  Two (128
// registers): a budget of 80 for three blocks fits the FP32 16-column chains
// without spilling but keeps fewer loads in flight per thread, and measured
// slower on GB300 (0.27 against 0.17 ms at 2^20 rows).
template <typename T, typename V, int NR>
constexpr int mres_min_blocks() { return 2; }

template <typename T, typename V, int NR>
__global__ void __launch_bounds__(kMrWarps * 32, (mres_min_blocks<T, V, NR>()))
    k_mres(Mat<T> A, const T *__restrict__ B, const T *__restrict__ X, T *__restrict__ R,
           long long rs, double *partials, unsigned *tick, Ctl *ctl0, int finalize,
           unsigned *hist1) {
    constexpr int VEC = (int)(16 / sizeof(T)) < NR ? (int)(16 / sizeof(T)) : NR;   // columns per lane
    constexpr int LPR = NR / VEC;           // lanes per row
    constexpr int RPS = 32 / LPR;           // rows per step; LPR steps cover the slice
    // entries whose gathers are issued together (two where the registers allow)
    constexpr int JS = NR * sizeof(T) <= 64 ? 2 : 1;
    extern __shared__ unsigned long long dsm_u64[];
    __shared__ double red[kMrWarps][NR];
    __shared__ int is_last;
    T *stage = (T *)dsm_u64 + (threadIdx.x >> 5) * 32 * (NR + 1);
    // the first top-K level of every column (FP32 iteration residuals)
    constexpr bool F32 = sizeof(T) == 4;
    unsigned *hsh = (unsigned *)((T *)dsm_u64 + kMrWarps * 32 * (NR + 1));
    const bool h1 = F32 && finalize == 1;
    if (h1)
        for (int q = threadIdx.x; q < NR * kF32Bins; q += blockDim.x) hsh[q] = 0u;
    __syncthreads();
    const V *__restrict__ val = sell_values<V, T>(A);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lc = lane % LPR, rsub = lane / LPR;
    const int c0 = lc * VEC;                // this lane's first column
    const unsigned long long keep = l2_keep_policy();
    // slices (longest first) are taken from a queue, one per warp at a time,
    // so every warp stays busy until the queue is empty
    unsigned *queue = tick + 1;
    double rr[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) rr[v] = 0.0;
    for (;;) {
        int sl = 0;
        if (lane == 0) sl = (int)atomicAdd(queue, 1u);
        sl = __shfl_sync(0xffffffffu, sl, 0);
        if (sl >= A.nslices) break;
        const long long base = A.sptr[sl] + lane;
        const int L = A.slen[sl];
        const int mylen = A.srlen[sl * 32 + lane];      // lane l holds row l's length
        T acc[LPR][VEC];
#pragma unroll
        for (int g = 0; g < LPR; ++g)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[g][v] = T(0);
        // JS entries of the lane's row in registers, the next JS in flight
        int cc[JS];
        V ac[JS];
#pragma unroll
        for (int u = 0; u < JS; ++u) {
            cc[u] = u < L ? __ldcs(A.scol + base + 32LL * u) : 0;
            ac[u] = u < L ? __ldcs(val + base + 32LL * u) : V(0);
        }
        for (int j0 = 0; j0 < L; j0 += JS) {
            int cn[JS];
            V an[JS];
            int cnt[JS];
#pragma unroll
            for (int u = 0; u < JS; ++u) {
                const int j = j0 + JS + u;
                cn[u] = j < L ? __ldcs(A.scol + base + 32LL * j) : 0;
                an[u] = j < L ? __ldcs(val + base + 32LL * j) : V(0);
                cnt[u] = __popc(__ballot_sync(0xffffffffu, j0 + u < mylen));
            }
            VecT<T, VEC> xg[JS][LPR];
            V ag[JS][LPR];
#pragma unroll
            for (int u = 0; u < JS; ++u)
#pragma unroll
                for (int g = 0; g < LPR; ++g) {
                    const int q = g * RPS + rsub;
                    const int c = __shfl_sync(0xffffffffu, cc[u], q);
                    ag[u][g] = __shfl_sync(0xffffffffu, ac[u], q);
                    if (q < cnt[u]) xg[u][g] = vload_keep<T, VEC>(X + (long long)c * NR + c0, keep);
                }
#pragma unroll
            for (int u = 0; u < JS; ++u)
#pragma unroll
                for (int g = 0; g < LPR; ++g) {
                    if (g * RPS + rsub < cnt[u]) {
                        const T w = wide<T>(ag[u][g]);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[g][v] = Ar<T>::fma(w, xg[u][g].v[v], acc[g][v]);
                    }
                }
#pragma unroll
            for (int u = 0; u < JS; ++u) {
                cc[u] = cn[u];
                ac[u] = an[u];
            }
        }
        typename SqAcc<T>::type sq[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) sq[v] = 0;
#pragma unroll
        for (int g = 0; g < LPR; ++g) {
            const int q = g * RPS + rsub;
            const int row = A.srow[sl * 32 + q];
            VecT<T, VEC> bv;
#pragma unroll
            for (int v = 0; v < VEC; ++v) bv.v[v] = T(0);
            if (row >= 0) bv = vload<T, VEC, true>(B + (long long)row * NR + c0);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                T ri = T(0);
                if (row >= 0) {
                    ri = Ar<T>::sub(bv.v[v], acc[g][v]);
                    sq[v] = SqAcc<T>::add(sq[v], ri);
                    if (h1) atomicAdd(&hsh[(c0 + v) * kF32Bins + f32_bin((unsigned)(abs_key(ri) >> 52))], 1u);
                }
                stage[q * (NR + 1) + c0 + v] = ri;
            }
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) rr[v] += (double)sq[v];
        __syncwarp();
#pragma unroll 4
        for (int c2 = 0; c2 < NR; ++c2) __stcs(R + c2 * rs + (long long)sl * 32 + lane, stage[lane * (NR + 1) + c2]);
        __syncwarp();
    }
    // sums of squares: lanes of one column group, then warps, then blocks
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
#pragma unroll
        for (int o = LPR; o < 32; o <<= 1) rr[v] += __shfl_xor_sync(0xffffffffu, rr[v], o);
    }
    if (lane < LPR)
#pragma unroll
        for (int v = 0; v < VEC; ++v) red[wid][c0 + v] = rr[v];
    __syncthreads();
    if (threadIdx.x < NR) {
        double t = 0.0;
        for (int w = 0; w < kMrWarps; ++w) t += red[w][threadIdx.x];
        partials[(long long)blockIdx.x * NR + threadIdx.x] = t;
    }
    if (h1)
        for (int q = threadIdx.x; q < NR * kF32Bins; q += blockDim.x)
            if (hsh[q]) atomicAdd(&hist1[(q / kF32Bins) * kHistBins + f32_bin_exp(q % kF32Bins)], hsh[q]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(tick, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x < NR) {
        double tot = 0.0;
        for (int b2 = 0; b2 < (int)gridDim.x; ++b2) tot += partials[(long long)b2 * NR + threadIdx.x];
        Ctl *ctl = ctl0 + threadIdx.x;
        if (finalize == 2) {                     // single-step: ||r_j||^2 only
            ctl->rr = tot;
        } else if (!(ctl->done || ctl->halt)) {
            ctl->rr = tot;
            const double rrn = sqrt(tot) / ctl->bnorm;
            ctl->rrn = rrn;
            if (finalize == 1 && ctl->tr_rrn && ctl->iter < ctl->trace_cap) ctl->tr_rrn[ctl->iter] = rrn;
            if (!isfinite(rrn)) { set_status(&ctl->status, kDevNumeric); ctl->done = 1; }
            else if (rrn <= ctl->tol) ctl->done = 1;
            ctl->n_in = 0;
            ctl->n_eq = 0;
        }
    }
    __syncthreads();
    if (h1) {   // every column's first radix level: warp w takes columns w, w + 8, ...
        __threadfence();
        for (int c = wid; c < NR; c += kMrWarps) {
            Ctl *ctl = ctl0 + c;
            int bin = 0, above = 0;
            warp_select_bin_f32(hist1 + (long long)c * kHistBins, A.K, &bin, &above);
            if (lane == 0 && !(ctl->done || ctl->halt)) { ctl->sel1 = bin; ctl->above1 = above; }
        }
    }
    if (threadIdx.x == 0) {
        *tick = 0u;
        *queue = 0u;
    }
}

// Residual columns from the SELL order to the caller's m x nr row-major layout.
template <typename T>
__global__ void __launch_bounds__(256) k_mr_unpermute(const T *__restrict__ Rs, long long mpos,
                                                      const int *__restrict__ perm, int nr,
                                                      T *__restrict__ Rout) {
    const long long tot = mpos * nr;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / nr;
        const int j = (int)(e - p * nr);
        const int i = perm[p];
        if (i >= 0) Rout[(long long)i * nr + j] = Rs[j * mpos + p];
    }
}

// The mixed form's refinement set-up for a block of columns: column j's
// b32 = fl32(r) (r read in SELL order, written to its row), d = 0, and its
// inner loop state; a column whose outer loop has stopped runs no inner
// iteration.  Grid (g, nr); the last block of each column finishes it and the
// last column sets the inner WHILE condition.
__global__ void __launch_bounds__(256) k_mr_inner_prep(const double *__restrict__ r64, long long rs,
                                                       const int *__restrict__ perm, int mpos,
                                                       float *__restrict__ b32, float *__restrict__ d32,
                                                       int n, int nr, double *partials, Ctl *out0,
                                                       Ctl *in0, unsigned *grp, int use_cond,
                                                       cudaGraphConditionalHandle hcond) {
    __shared__ double red[32];
    __shared__ int is_last;
    const int jc = blockIdx.y;
    Ctl *out = out0 + jc, *in = in0 + jc;
    const bool active = !(out->done || out->status || out->halt);
    double acc = 0.0;
    if (active) {
        const double *r = r64 + jc * rs;
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < mpos; p += gridDim.x * blockDim.x) {
            const int i = perm[p];
            if (i < 0) continue;
            const float v = (float)r[p];
            b32[(long long)i * nr + jc] = v;
            acc = __fma_rn((double)v, (double)v, acc);
        }
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
            d32[(long long)c * nr + jc] = 0.f;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[(long long)jc * gridDim.x + blockIdx.x] = acc;
        __threadfence();
        is_last = atomicAdd(&out->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot = 0.0;
    for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += partials[(long long)jc * gridDim.x + i];
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) {
        out->ticket = 0;
        if (active) {
            const double bn = sqrt(tot);
            const long long left = out->maxit - out->iter;
            in->bnorm = bn;
            in->iter = 0;
            in->maxit = left < out->inner_maxit ? left : out->inner_maxit;
            in->iter_base = out->iter_base + out->iter;
            in->seed = out->seed;
            in->sysid = out->sysid;
            in->n_static = out->n_static;
            in->tol = out->inner_tol;
            in->rr = 0.0;
            in->rrn = 1.0;
            in->done = bn == 0.0;
            in->halt = !(bn > 0.0 && in->maxit > 0);
            in->status = 0;
        } else {
            in->done = 1;
            in->halt = 1;
        }
        in->ticket = 0;
        in->pre_it = 0;
        in->n_in = 0;
        in->n_eq = 0;
        in->trace_cap = 0;
        in->tr_tau = nullptr;
        in->tr_rrn = nullptr;
        in->tr_I = nullptr;
        in->tr_x = nullptr;
        in->tr_dyn = nullptr;
        in->inc = 0;
        in->fault = out->fault;
        group_condition(in0, nr, grp + 2, use_cond, hcond);
    }
}

// x_j += d_j in FP64 for every column whose outer loop runs, then each
// column's refinement bookkeeping (as k_outer_update); the last column sets
// the outer WHILE condition.  Grid (g, nr).
__global__ void __launch_bounds__(256) k_mr_outer_update(double *__restrict__ x, const float *__restrict__ d32,
                                                         int n, int nr, Ctl *out0, Ctl *in0, unsigned *grp,
                                                         int use_cond, cudaGraphConditionalHandle hcond) {
    __shared__ int is_last;
    const int jc = blockIdx.y;
    Ctl *out = out0 + jc, *in = in0 + jc;
    const bool active = !(out->done || out->status || out->halt);
    if (active)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
            const long long q = (long long)c * nr + jc;
            x[q] = __dadd_rn(x[q], (double)d32[q]);
        }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&out->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    out->ticket = 0;
    if (active) {
        out->iter += in->iter;
        out->outer += 1;
        if (in->status) set_status(&out->status, in->status);
        if (in->iter == 0 || out->iter >= out->maxit) out->halt = 1;
    }
    if (out->done || out->status) out->halt = 1;
    group_condition(out0, nr, grp, use_cond, hcond);
}

// ------------------------------------------------------------- launchers
static size_t collect_smem_bytes() { return (size_t)kEqCap * (8 + 4) + (size_t)kMaxDynRows * 4; }
static size_t factor_smem_bytes() {
    return (size_t)(kShCap + kPairCap) * 8 + (size_t)kMaxDynRows * 8 + (size_t)kGPack * 8 +
           (size_t)2 * kSymMax * kSymW * 4 + (size_t)(3 * kSymMax + 2) * 2 + (size_t)(kSymMax + 2) * 4 +
           (size_t)kMaxDynRows * (2 + 2 + 1 + 1 + 1) + 64;
}

static Dyn dyn_bufs(rorbk_ctx *h) {
    return Dyn{h->dyn.I, h->dyn.estart, h->dyn.gdiag, h->dyn.y, h->dyn.ecol, h->dyn.eval,
               h->dyn.erow, h->dyn.ecap, h->dyn.owner, h->dyn.shared, h->dyn.segpos,
               h->dyn.epoch, h->dyn.raw, h->dyn.skeys, h->dyn.pkeys, h->dyn.pcap, h->dyn.g,
               h->K, (int)h->n, h->dyn.skcap};
}

// The sparse path's plan of the next draws (the dense path samples its own).
static Plan plan_of(rorbk_ctx *h) {
    if (h->format != RORBK_FORMAT_CSR) return Plan{};
    return Plan{h->cdf, h->k, h->off, h->ops.s_ptr, h->blk_nz, h->ops.w_ptr};
}

static int grid_stream(rorbk_ctx *h, int m) {
    return std::max(1, std::min(4 * h->num_sms, (m + 255) / 256));
}

// Launch shapes that leave every result unchanged, per column of a block
// (rorbk_autotune / rorbk_set_tuning; 0: the defaults below).  The top-K
// counts, the dynamic update's arithmetic and the scatters do not depend on
// the grid; the block residual's grid changes only the order in which its
// per-block sums of squares are added.
static int tuned(int v, int def) { return v > 0 ? v : std::max(1, def); }
int grid_topk(rorbk_ctx *h) {
    const int nr = std::max(1, h->nr);
    const long long mp = h->nr ? h->mr.mpos : h->m;
    return tuned(h->tune.topk, std::min<long long>(4 * h->num_sms / nr, (mp + 255) / 256));
}
int grid_collect(rorbk_ctx *h) { return tuned(h->tune.collect, grid_topk(h) / 2); }
int grid_mark(rorbk_ctx *h) { return tuned(h->tune.mark, h->num_sms / std::max(1, h->nr)); }
int grid_scatter(rorbk_ctx *h) { return tuned(h->tune.scatter, 2 * h->num_sms / std::max(1, h->nr)); }

int residual_grid(rorbk_ctx *h) {
    int per_sm = 0, per_sm32 = 0;
    if (h->format == RORBK_FORMAT_DENSE) {
        if (h->vdtype == RORBK_F32)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual<double, float, true>, 256, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual<double, double, true>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_residual<float, float, true>, 256, 0);
    } else {
        if (h->vdtype == RORBK_F32)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual<double, float>, 256, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual<double, double>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_residual<float, float>, 256, 0);
    }
    return std::max(1, std::min(per_sm, per_sm32 > 0 ? per_sm32 : per_sm)) * h->num_sms;
}

template <int NR>
static void configure_mres() {
    cudaFuncSetAttribute(k_mres<double, double, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)mres_smem_bytes<double, NR>());
    cudaFuncSetAttribute(k_mres<double, float, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)mres_smem_bytes<double, NR>());
    cudaFuncSetAttribute(k_mres<float, float, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)mres_smem_bytes<float, NR>());
}

// Resident blocks per SM of the FP32 (fp32 != 0) or the FP64 instances.
template <int NR>
static int mres_blocks_per_sm(int fp32) {
    int a = 0, b = 0, c = 0;
    if (fp32) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_mres<float, float, NR>, kMrWarps * 32,
                                                      mres_smem_bytes<float, NR>());
        return std::max(1, c);
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mres<double, double, NR>, kMrWarps * 32,
                                                  mres_smem_bytes<double, NR>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mres<double, float, NR>, kMrWarps * 32,
                                                  mres_smem_bytes<double, NR>());
    return std::max(1, std::min(a, b));
}

// One resident wave of the column-block residual for nr columns (slices are
// handed out by a queue, so every resident warp takes part).
int mres_grid(rorbk_ctx *h, int nr, int fp32) {
    int per_sm = 1;
    switch (nr) {
        case 2: per_sm = mres_blocks_per_sm<2>(fp32); break;
        case 4: per_sm = mres_blocks_per_sm<4>(fp32); break;
        case 8: per_sm = mres_blocks_per_sm<8>(fp32); break;
        case 16: per_sm = mres_blocks_per_sm<16>(fp32); break;
        default: per_sm = mres_blocks_per_sm<32>(fp32); break;
    }
    return per_sm * h->num_sms;
}

void configure_kernels() {
    cudaFuncSetAttribute(k_static<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<double>());
    cudaFuncSetAttribute(k_static<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<float>());
    cudaFuncSetAttribute(k_static<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<double>());
    cudaFuncSetAttribute(k_static<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<float>());
    cudaFuncSetAttribute(k_static<double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<double>());
    cudaFuncSetAttribute(k_static<float, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<float>());
    cudaFuncSetAttribute(k_static<double, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<double>());
    cudaFuncSetAttribute(k_static<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<float>());
    cudaFuncSetAttribute(k_topk_collect<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)collect_smem_bytes());
    cudaFuncSetAttribute(k_topk_collect<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)collect_smem_bytes());
    cudaFuncSetAttribute(k_dyn_mark<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem_bytes());
    cudaFuncSetAttribute(k_dyn_mark<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem_bytes());
    cudaFuncSetAttribute(k_dyn_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem());
    cudaFuncSetAttribute(k_sd_rows_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sd_rows_smem<double>());
    cudaFuncSetAttribute(k_sd_rows_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sd_rows_smem<float>());
    // the column-block instances
    cudaFuncSetAttribute(k_static<double, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<double>());
    cudaFuncSetAttribute(k_static<float, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)static_smem_bytes<float>());
    cudaFuncSetAttribute(k_topk_collect<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)collect_smem_bytes());
    cudaFuncSetAttribute(k_topk_collect<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)collect_smem_bytes());
    cudaFuncSetAttribute(k_dyn_mark<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem_bytes());
    cudaFuncSetAttribute(k_dyn_mark<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)factor_smem_bytes());
    configure_mres<2>();
    configure_mres<4>();
    configure_mres<8>();
    configure_mres<16>();
    configure_mres<32>();
}

void launch_begin(rorbk_ctx *h, const double *b, const double *x0, double *x, int use_cond,
                  unsigned long long hcond) {
    if (h->nr) {
        k_mr_begin<<<dim3(1, h->nr), 1024, 0, h->stream>>>(b, (int)h->m, x0, x, (int)h->n, h->ctl, h->nr,
                                                           h->mr.grp, use_cond, (cudaGraphConditionalHandle)hcond);
        return;
    }
    k_begin<<<1, 1024, 0, h->stream>>>(b, (int)h->m, x0, x, (int)h->n, h->ctl, use_cond,
                                       (cudaGraphConditionalHandle)hcond);
}

void launch_dense_gram(rorbk_ctx *h, Ctl *ctl, int tensor_cores) {
    const int K = h->K;
    if (tensor_cores) {
        const int tiles = h->gram_tiles, S = h->gram_splits;
        const int vec = (h->n % 4 == 0) && ((reinterpret_cast<uintptr_t>(h->val32) & 15) == 0);
        k_dyn_gram_tc<<<dim3(tiles, S), 128, gram_tc_smem(), h->stream>>>(h->val32, (int)h->n, K, S, vec,
                                                                       dyn_bufs(h), h->gram_part, ctl);
        const long long np = (long long)K * (K + 1) / 2;
        k_dyn_gram_reduce<<<(int)std::min<long long>(4LL * h->num_sms, (np + 255) / 256), 256, 0, h->stream>>>(
            h->gram_part, K, S, h->mu, dyn_bufs(h), ctl);
    } else {
        const int T16 = (K + kGT - 1) / kGT;
        k_dyn_dense_gram<<<T16 * (T16 + 1) / 2, kGT * kGT, 0, h->stream>>>(h->val, (int)h->n, K, h->mu,
                                                                          dyn_bufs(h), ctl);
    }
}

template <typename T>
static void launch_dynamic_tail(rorbk_ctx *h, const T *r, T *x, Ctl *ctl, int check_done,
                                int count_iter, int use_cond, unsigned long long hcond, int inc = 0) {
    if (h->K >= h->n) {
        // the n x n form (Lemma 1): dense rows of I, G = A_I^T A_I + mu I,
        // h = A_I^T r_I, blocked Cholesky of size n starting z at h, x += y
        const int K = h->K, n = (int)h->n;
        double *dw = h->dynw, *hz = h->dynw + (long long)K * n;
        cudaMemsetAsync(dw, 0, (size_t)K * n * sizeof(double), h->stream);
        k_dynw_rows<<<std::max(1, std::min(4 * h->num_sms, (K * 32 + 255) / 256)), 256, 0, h->stream>>>(
            h->rowptr, h->col, h->val, n, K, dyn_bufs(h), dw, ctl);
        const long long np = (long long)n * (n + 1) / 2;
        k_dynw_gram<<<(int)std::max<long long>(1, std::min<long long>(8LL * h->num_sms, (np + 255) / 256)), 256, 0,
                      h->stream>>>(dw, n, K, h->mu, dyn_bufs(h), ctl);
        k_dynw_rhs<T><<<std::max(1, (n + 63) / 64), 64, 0, h->stream>>>(dw, r, n, K, dyn_bufs(h), hz, ctl);
        for (int j0 = 0; j0 < n; j0 += kPW) {
            const int below = n - j0 - std::min(kPW, n - j0);
            k_dchol_panel_rows<T><<<std::max(1, (below + 31) / 32), 256, 0, h->stream>>>(r, n, j0, dyn_bufs(h),
                                                                                       ctl, hz);
            const int rest = n - std::min(n, j0 + kPW), tt = (rest + 15) / 16;
            if (rest > 0) k_dchol_trail<<<tt * (tt + 1) / 2, 256, 0, h->stream>>>(n, j0, dyn_bufs(h), ctl);
        }
        k_dchol_back<<<1, 1024, 0, h->stream>>>(n, dyn_bufs(h), ctl);
        const int g = std::max(1, std::min(8 * h->num_sms, (n + 63) / 64));
        k_dyn_dense_scatter<T><<<g, 64, 0, h->stream>>>(h->val, h->val32, x, n, K, dyn_bufs(h), ctl, count_iter,
                                                          use_cond, (cudaGraphConditionalHandle)hcond, 1);
        return;
    }
    if (h->format == RORBK_FORMAT_DENSE) {
        const int K = h->K;
        // mixed precision: the TF32 tensor-core Gram (FP32 partials added in FP64)
        launch_dense_gram(h, ctl, sizeof(T) == sizeof(float) && h->gram_part);
        for (int j0 = 0; j0 < K; j0 += kPW) {
            const int below = K - j0 - std::min(kPW, K - j0);
            k_dchol_panel_rows<T><<<std::max(1, (below + 31) / 32), 256, 0, h->stream>>>(r, K, j0,
                                                                                       dyn_bufs(h), ctl,
                                                                                       nullptr);
            const int rest = K - std::min(K, j0 + kPW), tt = (rest + 15) / 16;
            if (rest > 0) k_dchol_trail<<<tt * (tt + 1) / 2, 256, 0, h->stream>>>(K, j0, dyn_bufs(h), ctl);
        }
        k_dchol_back<<<1, 1024, 0, h->stream>>>(K, dyn_bufs(h), ctl);
        const int g = std::max(1, std::min(8 * h->num_sms, (int)((h->n + 63) / 64)));
        k_dyn_dense_scatter<T><<<g, 64, 0, h->stream>>>(h->val, h->val32, x, (int)h->n, K, dyn_bufs(h),
                                                          ctl, count_iter, use_cond,
                                                          (cudaGraphConditionalHandle)hcond, 0);
        return;
    }
    Mat<T> A = make_mat<T>(h);
    k_dyn_mark<T><<<grid_mark(h), 512, factor_smem_bytes(), h->stream>>>(A, r, dyn_bufs(h), ctl,
                                                                        check_done, one_col((int)h->m),
                                                                        count_iter ? plan_of(h) : Plan{});
    (inc ? k_dyn_scatter<T, true> : k_dyn_scatter<T, false>)<<<grid_scatter(h), 512, 0, h->stream>>>(
        x, (int)h->n, dyn_bufs(h), ctl, count_iter, use_cond, (cudaGraphConditionalHandle)hcond,
        one_col((int)h->m));
}

template <typename T>
static const T *csc_values(const rorbk_ctx *h);
template <>
const double *csc_values<double>(const rorbk_ctx *h) { return h->csc_val; }
template <>
const float *csc_values<float>(const rorbk_ctx *h) { return h->csc_val32; }

// The residual kernel for this handle's format (the dense instance reads no
// column indices).
template <typename T, typename V>
static void residual_launch(rorbk_ctx *h, const Mat<T> &A, const T *b, const T *x, T *r, Ctl *ctl,
                            int finalize) {
    if (h->format == RORBK_FORMAT_DENSE)
        k_residual<T, V, true><<<h->grid_res, 256, 0, h->stream>>>(A, b, x, r, h->partials, h->hist1, ctl,
                                                                   finalize);
    else
        k_residual<T, V, false><<<h->grid_res, 256, 0, h->stream>>>(A, b, x, r, h->partials, h->hist1, ctl,
                                                                    finalize);
}

template <typename T>
void launch_iteration_t(rorbk_ctx *h, const T *b, T *x, T *r, Ctl *ctl, int use_cond,
                        unsigned long long hcond, int weighted = 0, int inc = 0) {
    Mat<T> A = make_mat<T>(h);
    if (h->format == RORBK_FORMAT_DENSE) {
        T *rl = (T *)h->sd_scratch, *yy = rl + kMaxBlockRows;
        const int gr = (h->smax + 31) / 32;
        // column-parallel passes in blocks of 64 threads: more SMs share the
        // FP64 chains of a narrow system
        const int gs = std::max(1, std::min(8 * h->num_sms, (int)((h->n + 63) / 64)));
        for (int l = 0; l < kDenseStatic; ++l) {
            k_sd_rows_tiled<T><<<gr, kSdCols, sd_rows_smem<T>(), h->stream>>>(A, b, x, rl, ctl, l);
            k_sd_apply<T><<<1, 1024, 0, h->stream>>>(A, rl, yy, ctl, l);
            k_sd_scatter<T><<<gs, 64, 0, h->stream>>>(A, rl, yy, x, ctl, l);
            if (h->n_wood) k_sd_wood<T><<<gs, 64, 0, h->stream>>>(A, yy, x, ctl, l);
        }
        // updates beyond kDenseStatic (n_static > 3), if any
        (h->n_wood ? k_static<T, false, true> : k_static<T, false, false>)<<<1, 1024, static_smem_bytes<T>(),
                                                                              h->stream>>>(A, b, x, ctl, -1, 0,
                                                                                           kDenseStatic, 1);
    } else {
        const bool wd = h->n_wood > 0;
        (inc ? (wd ? k_static<T, true, true> : k_static<T, true, false>)
             : (wd ? k_static<T, false, true> : k_static<T, false, false>))<<<1, 1024, static_smem_bytes<T>(),
                                                                               h->stream>>>(A, b, x, ctl, -1, 1, 0, 1);
    }
    if (inc) {   // r from the change log; the exact kernel below runs only when asked to
        k_inc_apply<T><<<4 * h->num_sms, 256, 0, h->stream>>>(h->csc_ptr, h->csc_row, csc_values<T>(h),
                                                              r, ctl);
        k_inc_finish<T><<<grid_stream(h, (int)h->m), 256, 0, h->stream>>>(r, (int)h->m, h->K, h->partials,
                                                                         h->hist1, ctl);
    }
    if constexpr (sizeof(T) == sizeof(float)) {
        residual_launch<T, float>(h, A, b, x, r, ctl, 1);
    } else {
        if (h->vdtype == RORBK_F32)
            residual_launch<T, float>(h, A, b, x, r, ctl, 1);
        else
            residual_launch<T, double>(h, A, b, x, r, ctl, 1);
    }
    if constexpr (sizeof(T) == sizeof(double))
        if (weighted) launch_weights(h, r);      // the draws of the next iteration
    k_topk_hist2<T><<<grid_topk(h), 256, 0, h->stream>>>(r, (int)h->m, h->K, h->hist2, ctl, 1, one_col((int)h->m));
    k_topk_collect<T><<<grid_collect(h), 512, collect_smem_bytes(), h->stream>>>(
        r, (int)h->m, h->K, h->rowptr, h->in_list, h->eq_list, dyn_bufs(h), ctl, 1, one_col((int)h->m));
    launch_dynamic_tail<T>(h, r, x, ctl, 1, 1, use_cond, hcond, inc);
}

// R = B - A X for the handle's nr columns (finalize as k_residual's).
template <typename T, typename V>
static void mres_launch(rorbk_ctx *h, const Mat<T> &A, const T *B, const T *X, T *R, Ctl *ctl, int finalize) {
    const int wave = sizeof(T) == 4 ? h->mr.grid32 : h->mr.grid;
    const dim3 grid(h->tune.residual > 0 ? std::min(h->tune.residual, wave) : wave), block(kMrWarps * 32);
    const long long rs = h->mr.mpos;
    unsigned *tick = h->mr.grp + 4;
    switch (h->nr) {
        case 2: k_mres<T, V, 2><<<grid, block, mres_smem_bytes<T, 2>(), h->stream>>>(A, B, X, R, rs, h->partials, tick, ctl, finalize, h->hist1); break;
        case 4: k_mres<T, V, 4><<<grid, block, mres_smem_bytes<T, 4>(), h->stream>>>(A, B, X, R, rs, h->partials, tick, ctl, finalize, h->hist1); break;
        case 8: k_mres<T, V, 8><<<grid, block, mres_smem_bytes<T, 8>(), h->stream>>>(A, B, X, R, rs, h->partials, tick, ctl, finalize, h->hist1); break;
        case 16: k_mres<T, V, 16><<<grid, block, mres_smem_bytes<T, 16>(), h->stream>>>(A, B, X, R, rs, h->partials, tick, ctl, finalize, h->hist1); break;
        default: k_mres<T, V, 32><<<grid, block, mres_smem_bytes<T, 32>(), h->stream>>>(A, B, X, R, rs, h->partials, tick, ctl, finalize, h->hist1); break;
    }
}

// One iteration for every column of a column-block handle: the sampled
// updates (one block of threads per column), the residual of all columns in
// one pass over A, the three top-K levels and the dynamic update (one grid
// row per column).  grp: the ticket/flag pair of the loop being run.
template <typename T>
static void launch_mr_iteration_t(rorbk_ctx *h, const T *b, T *x, T *r, Ctl *ctl, int use_cond,
                                  unsigned long long hcond, unsigned *grp) {
    Mat<T> A = make_mat<T>(h);
    const int nr = h->nr, m = (int)h->m, K = h->K;
    const Cols cl{nr, h->mr.mpos, (int)h->mr.mpos, h->sell.row, h->mr.iperm, grp};
    cudaStream_t st = h->stream;
    k_static<T, false, false, true><<<dim3(1, nr), 1024, static_smem_bytes<T>(), st>>>(A, b, x, ctl, -1, 1, 0, nr);
    if constexpr (sizeof(T) == sizeof(float)) {
        mres_launch<T, float>(h, A, b, x, r, ctl, 1);
    } else {
        if (h->vdtype == RORBK_F32) mres_launch<T, float>(h, A, b, x, r, ctl, 1);
        else mres_launch<T, double>(h, A, b, x, r, ctl, 1);
    }
    const int g = grid_topk(h);
    // the FP32 block residual formed the first radix level itself
    if constexpr (sizeof(T) == sizeof(double))
        k_topk_hist1<T, true><<<dim3(g, nr), 256, 0, st>>>(r, m, K, h->hist1, ctl, cl, 1);
    k_topk_hist2<T, true><<<dim3(g, nr), 256, 0, st>>>(r, m, K, h->hist2, ctl, 1, cl);
    k_topk_collect<T, true><<<dim3(grid_collect(h), nr), 512, collect_smem_bytes(), st>>>(
        r, m, K, h->rowptr, h->in_list, h->eq_list, dyn_bufs(h), ctl, 1, cl);
    k_dyn_mark<T, true><<<dim3(grid_mark(h), nr), 512, factor_smem_bytes(), st>>>(
        A, r, dyn_bufs(h), ctl, 1, cl, plan_of(h));
    k_dyn_scatter<T, false, true><<<dim3(grid_scatter(h), nr), 512, 0, st>>>(
        x, (int)h->n, dyn_bufs(h), ctl, 1, use_cond, (cudaGraphConditionalHandle)hcond, cl);
}

void launch_residual_multi(rorbk_ctx *h, int fp32, const void *B, const void *X, void *R) {
    const int g = std::max(1, std::min(8 * h->num_sms, (int)((h->mr.mpos * h->nr + 255) / 256)));
    if (fp32) {
        mres_launch<float, float>(h, make_mat<float>(h), (const float *)B, (const float *)X, h->r32, h->ctl, 2);
        if (R) k_mr_unpermute<float><<<g, 256, 0, h->stream>>>(h->r32, h->mr.mpos, h->sell.row, h->nr, (float *)R);
    } else {
        if (h->vdtype == RORBK_F32)
            mres_launch<double, float>(h, make_mat<double>(h), (const double *)B, (const double *)X, h->r, h->ctl, 2);
        else
            mres_launch<double, double>(h, make_mat<double>(h), (const double *)B, (const double *)X, h->r, h->ctl, 2);
        if (R) k_mr_unpermute<double><<<g, 256, 0, h->stream>>>(h->r, h->mr.mpos, h->sell.row, h->nr, (double *)R);
    }
}

void launch_weights(rorbk_ctx *h, const double *r) {
    k_wweights<<<std::max(1, std::min(4 * h->num_sms, (h->k + 255) / 256)), 256, 0, h->stream>>>(
        r, h->off, h->k, h->pbar, h->wgt, h->ctl);
    k_wcdf<<<1, 1024, 0, h->stream>>>(h->wgt, h->k, h->wcdf, h->cdf, h->ctl);
}

void launch_iteration(rorbk_ctx *h, const double *b, double *x, double *r, int use_cond,
                      unsigned long long hcond, int weighted, int inc) {
    if (h->nr) launch_mr_iteration_t<double>(h, b, x, r, h->ctl, use_cond, hcond, h->mr.grp);
    else launch_iteration_t<double>(h, b, x, r, h->ctl, use_cond, hcond, weighted, inc);
}

void launch_mixed_outer(rorbk_ctx *h, int use_cond, unsigned long long hcond_inner) {
    Mat<double> A = make_mat<double>(h);
    if (h->nr) {
        if (h->vdtype == RORBK_F32) mres_launch<double, float>(h, A, h->bb, h->xb, h->r, h->ctl, 3);
        else mres_launch<double, double>(h, A, h->bb, h->xb, h->r, h->ctl, 3);
        const int g = std::max(1, std::min(4 * h->num_sms / h->nr, (int)((std::max<long long>(h->mr.mpos, h->n) + 255) / 256)));
        k_mr_inner_prep<<<dim3(g, h->nr), 256, 0, h->stream>>>(
            h->r, h->mr.mpos, h->sell.row, (int)h->mr.mpos, h->b32, h->d32, (int)h->n, h->nr, h->partials,
            h->ctl, h->ctl_in, h->mr.grp, use_cond, (cudaGraphConditionalHandle)hcond_inner);
        return;
    }
    if (h->vdtype == RORBK_F32)
        residual_launch<double, float>(h, A, h->bb, h->xb, h->r, h->ctl, 3);
    else
        residual_launch<double, double>(h, A, h->bb, h->xb, h->r, h->ctl, 3);
    const int g = grid_stream(h, (int)std::max(h->m, h->n));
    k_inner_prep<<<g, 256, 0, h->stream>>>(h->r, (int)h->m, h->b32, h->d32, (int)h->n, h->partials,
                                           h->ctl, h->ctl_in, use_cond,
                                           (cudaGraphConditionalHandle)hcond_inner);
}

void launch_mixed_inner(rorbk_ctx *h, int use_cond, unsigned long long hcond_inner, int inc) {
    if (h->nr) launch_mr_iteration_t<float>(h, h->b32, h->d32, h->r32, h->ctl_in, use_cond, hcond_inner, h->mr.grp + 2);
    else launch_iteration_t<float>(h, h->b32, h->d32, h->r32, h->ctl_in, use_cond, hcond_inner, 0, inc);
}

void launch_mixed_update(rorbk_ctx *h, int use_cond, unsigned long long hcond_outer) {
    if (h->nr) {
        const int g = std::max(1, std::min(4 * h->num_sms / h->nr, (int)((h->n + 255) / 256)));
        k_mr_outer_update<<<dim3(g, h->nr), 256, 0, h->stream>>>(h->xb, h->d32, (int)h->n, h->nr, h->ctl, h->ctl_in,
                                                                h->mr.grp, use_cond, (cudaGraphConditionalHandle)hcond_outer);
        return;
    }
    const int g = grid_stream(h, (int)h->n);
    k_outer_update<<<g, 256, 0, h->stream>>>(h->xb, h->d32, (int)h->n, h->ctl, h->ctl_in, use_cond,
                                             (cudaGraphConditionalHandle)hcond_outer);
}

void launch_static_forced(rorbk_ctx *h, int tau, const double *b, double *x) {
    (h->n_wood ? k_static<double, false, true> : k_static<double, false, false>)<<<
        1, 1024, static_smem_bytes<double>(), h->stream>>>(make_mat<double>(h), b, x,
                                                                          h->ctl, tau, 0, 0, 1);
}

void launch_residual_only(rorbk_ctx *h, const double *b, const double *x, double *r) {
    if (h->vdtype == RORBK_F32)
        residual_launch<double, float>(h, make_mat<double>(h), b, x, r, h->ctl, 2);
    else
        residual_launch<double, double>(h, make_mat<double>(h), b, x, r, h->ctl, 2);
}

void launch_residual32_only(rorbk_ctx *h, const float *b, const float *x, float *r) {
    residual_launch<float, float>(h, make_mat<float>(h), b, x, r, h->ctl, 2);
}

void launch_topk_only(rorbk_ctx *h, const double *r, int *I) {
    const int g = grid_stream(h, (int)h->m);
    const Cols one = one_col((int)h->m);
    k_topk_hist1<double><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->K, h->hist1, h->ctl, one, 0);
    k_topk_hist2<double><<<g, 256, 0, h->stream>>>(r, (int)h->m, h->K, h->hist2, h->ctl, 0, one);
    k_topk_collect<double><<<std::max(1, g / 2), 512, collect_smem_bytes(), h->stream>>>(
        r, (int)h->m, h->K, h->rowptr, h->in_list, h->eq_list, dyn_bufs(h), h->ctl, 0, one);
    cudaMemcpyAsync(I, h->dyn.I, h->K * sizeof(int), cudaMemcpyDeviceToDevice, h->stream);
}

void launch_dynamic_given(rorbk_ctx *h, const int *I, const double *r, double *x) {
    k_dyn_set_rows<<<1, 512, 0, h->stream>>>(h->rowptr, I, h->K, (int)h->m, dyn_bufs(h), h->ctl);
    launch_dynamic_tail<double>(h, r, x, h->ctl, 0, 0, 0, 0);
}

void launch_sample_probe(rorbk_ctx *h, uint64_t seed, uint64_t sysid, int64_t it, int64_t l,
                         long long *out) {
    k_sample_probe<<<1, 1, 0, h->stream>>>(h->cdf, h->k, seed, sysid, it, l, out);
}

}  // namespace rorbk
