// internal.cuh -- device helpers and the handle layout shared by the CUDA
// translation units of the ROR-BK library.  Nothing here is part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/rorbk.h"

namespace rorbk {

// ---------------------------------------------------------------- limits
constexpr int kMaxBlockRows = 1024;     // static block rows (one thread per row)
constexpr int kGraphUnroll = 4;         // default iterations per graph WHILE-body execution
constexpr int kMaxGraphUnroll = 16;
constexpr int kMaxDynRows = 1024;       // K = floor(m/k)
constexpr int kTileRows = 256;          // residual tile: rows ...
constexpr int kTileNnz = 2048;          // ... and nonzeros per tile
constexpr int kHistBins = 2048;         // 11-bit radix digits of |r| keys
constexpr int kEqCap = 4096;            // top-K candidates sorted in one CTA
constexpr int kSortCapSmem = 4096;      // entries sorted in shared memory
constexpr int kShCap = 2048;            // dynamic block: shared-column entries in smem
constexpr int kPairCap = 2048;          // dynamic block: Gram contributions in smem
constexpr int kSPackedMax = 176;        // dynamic block: coupled rows factored in smem
constexpr int kGPack = kSPackedMax * (kSPackedMax + 1) / 2;

// device error codes (ctl->status)
constexpr int kDevOk = 0;
constexpr int kDevNotSpd = 1;
constexpr int kDevBounds = 2;
constexpr int kDevNumeric = 3;
constexpr int kDevTimeout = 4;   // a bounded device wait gave up

// ----------------------------------------------------- device-side state
// Loop state of one solve, kept in device memory so that the whole iteration
// loop runs without the host.
struct Ctl {
    long long iter;        // iterations completed in this solve
    long long maxit;
    long long iter_base;   // Philox counter of iteration 0 (start_iter)
    unsigned long long seed, sysid;
    double tol, bnorm, rr, rrn;
    int done;              // set when rrn <= tol (or ||b|| = 0)
    int status;            // kDev* error word (first error wins)
    int n_static;
    unsigned ticket;       // last-block election of grid-wide kernels
    // radix select of the top-K keys
    int sel1, above1, prefix, above, n_in, n_eq;
    // trace (device pointers, FP64 mode)
    long long trace_cap;
    long long *tr_tau;
    double *tr_rrn;
    int *tr_I;
    double *tr_x;
    int *tr_dyn;
    // mixed precision outer loop
    long long outer, inner_maxit, inner_total;
    double inner_tol, outer_rrn;
    int outer_done;
    int has_x0;
    // dynamic block bookkeeping
    int dynE, dyn_nsh, dyn_nS, dyn_npair, dyn_nraw, pad3_;
    int halt;              // no further iteration runs (converged, error or maxit)
    int weighted;          // residual-weighted draws (RORBK_DIST_RESIDUAL_WEIGHTED)
    // incremental residual (RORBK_RESIDUAL_INCREMENTAL): the scatters log
    // (column, increment) pairs, r -= A dx is applied from the log, and an
    // exact residual is formed when inc_full is set (first iteration, every
    // inc_refresh iterations, a full log, or to confirm convergence)
    int inc, inc_full, inc_count, inc_refresh;
    int nlog, log_full, log_cap, pad4_;
    int *log_col;          // [log_cap] changed columns
    double *log_val;       // [log_cap] their increments
    const double *scdf;    // the running sum the static draws use (P's, or the weighted one)
    int fault;             // RORBK_FAULT_* injected by the host (tests of the failure paths)
    // the next iteration's draws and their blocks' ranges, formed ahead by the
    // top-K pass (pre_it = that iteration's Philox counter + 1; 0: none)
    long long pre_it;
    int pre_tau[8], pre_r0[8], pre_s[8], pre_p0[8], pre_pend[8], pre_sb[8], pre_nS[8];
    long long pre_wb[8];
};
constexpr int kPreDraws = 8;           // draws per iteration formed ahead (n_static <= 8)

// Sparse operator of one static block t (Section 3.1's stored inverse
// W_t = (A_t A_t^T + mu I)^{-1}).  Rows of the block that share no column
// with another row of the block ("uncoupled") make W_t diagonal there:
// W_ii = 1 / L_ii^2; the coupled rows S_t carry a dense |S_t| x |S_t| block.
struct StaticOps {
    int *s_ptr = nullptr;       // [k+1] offsets into s_idx
    uint16_t *s_idx = nullptr;  // coupled local rows, ascending
    uint16_t *bperm = nullptr;  // [m] local rows of each block, longest first
    long long *w_ptr = nullptr; // [k+1] offsets into w_ss
    double *w_ss = nullptr;     // dense W on S_t, row-major
    double *w_diag = nullptr;   // [m] W_ii for uncoupled rows
    int *s_pos = nullptr;       // [m] position of a row in its S_t, or -1
    float *w_ss32 = nullptr, *w_diag32 = nullptr;  // FP32 copies (mixed)
};

// Per-block column-sorted copy of the block's nonzeros, used for the
// deterministic scatter x += A_t^T y.  Entries of block t occupy the same
// positions as the block's CSR range, sorted by (column, row).
struct BlockT {
    int *col = nullptr;
    uint16_t *row = nullptr;    // local row in the block
    double *val = nullptr;
    float *val32 = nullptr;
    uint16_t *off16 = nullptr;  // CSR offset in the block of each entry (blocks of at
                                // most 65,536 entries; the staged static update)
    int *seg = nullptr;         // segment (distinct column) start positions
    int *seg_ptr = nullptr;     // [k] segment count of block t; its segments
                                // start at seg[row_ptr[off[t]] ...]
};

// Device memory owned jointly by a handle and its clones (rorbk_clone): the
// set-up data.  Freed when the last of them is freed.
struct DevBlocks {
    int device = 0;
    std::vector<void *> p;
    ~DevBlocks() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        for (void *q : p) cudaFree(q);
        cudaSetDevice(cur);
    }
};

}  // namespace rorbk

struct rorbk_ctx {
    int device = 0;
    cudaStream_t stream = 0;
    std::string err;
    int64_t m = 0, n = 0, nnz = 0;
    int format = RORBK_FORMAT_CSR, vdtype = RORBK_F64;
    int k = 0, K = 0, smax = 0;
    double mu = 0;
    int precision_built = 0;
    int num_sms = 0;
    int64_t bytes = 0;
    std::vector<void *> allocs;                       // memory this handle alone owns
    std::shared_ptr<rorbk::DevBlocks> shared_setup;   // set-up memory shared with clones
    int maxrow = 0;                                   // longest row of A
    // matrix (CSR)
    int *rowptr = nullptr, *col = nullptr;
    double *val = nullptr;      // FP64 values (exact widening if given FP32)
    float *val32 = nullptr;     // FP32 values (mixed precision)
    // partition
    std::vector<int64_t> h_off;
    int *off = nullptr;
    int *blk_nz = nullptr;      // [k+1] first entry of each block, rowptr[off[t]]
    // proposal
    double *cdf = nullptr, *crowsum = nullptr;
    double *pbar = nullptr;             // [k] Pbar_t (the weights before the running sum)
    double *rn = nullptr, *rn32 = nullptr;   // [m] ||A_i||^2 from the FP64 values / the FP32 copy
    rorbk::StaticOps ops;
    rorbk::BlockT bt;
    // residual tiles (single-step residual on CSR) and the SELL-32 copy of A
    int ntiles = 0;
    int *tile_row0 = nullptr;
    int grid_res = 0;
    struct {
        int nslices = 0;
        long long *ptr = nullptr;   // [nslices+1] first entry of slice s
        int *len = nullptr;         // [nslices] entries per lane (the slice's longest row)
        int *row = nullptr;         // [nslices*32] row of each lane (-1: empty lane)
        int *rlen = nullptr;        // [nslices*32] nonzeros of that row
        int *col = nullptr;         // [entries] column-major inside a slice
        float *val32 = nullptr;     // FP32-stored values (FP32 systems and the mixed path)
        double *val = nullptr;      // FP64 values (FP64 systems)
    } sell;
    // adjoint handles (rorbk_setup_adjoint): the row norms c_i of the primal A
    double *adj_scale = nullptr;
    // workspace
    double *r = nullptr, *xb = nullptr, *bb = nullptr, *x64 = nullptr;
    double *sd_scratch = nullptr;   // [2 kMaxBlockRows] r_tau and y of the dense static updates
    double *wgt = nullptr, *wcdf = nullptr;   // [k] residual-weighted draws: weights, running sum
    // incremental residual: CSC copy of A (built at the first such solve) and
    // the log of (column, increment) pairs
    // the s >= n form (Lemma 1, Section 3.1): V_t = (A_t^T A_t + mu I)^{-1} of
    // the blocks with at least n rows (wood_ptr[t] >= 0, n x n row-major), and
    // for K >= n the dynamic block's rows as a dense K x n array plus A_I^T r_I
    long long *wood_ptr = nullptr;
    double *wood_ss = nullptr;
    float *wood_ss32 = nullptr;
    int n_wood = 0;
    double *dynw = nullptr;          // [K n + n]
    // mixed-precision dense dynamic Gram on the tensor cores: FP32 partial
    // tiles [gram_tiles][gram_splits][128][128]
    float *gram_part = nullptr;
    int gram_tiles = 0, gram_splits = 0;
    // values_version counts rorbk_update_values calls on the set-up this handle
    // shares (clones share the counter); csc_version is the count the handle's
    // own CSC copy was formed at
    std::shared_ptr<int> values_version;
    int csc_version = 0;
    int *csc_ptr = nullptr, *csc_row = nullptr;
    double *csc_val = nullptr;
    float *csc_val32 = nullptr;
    int *ilog_col = nullptr;
    double *ilog_val = nullptr;
    int ilog_cap = 0;
    cudaGraphExec_t exec_fp64_inc = nullptr, exec_mixed_inc = nullptr;
    cudaGraphExec_t exec_fp64_w = nullptr;   // the FP64 loop with residual-weighted draws
    float *r32 = nullptr, *b32 = nullptr, *d32 = nullptr;
    double *partials = nullptr;
    unsigned *hist1 = nullptr, *hist2 = nullptr;
    int *in_list = nullptr, *eq_list = nullptr;
    struct {
        int *I = nullptr, *estart = nullptr;
        double *gdiag = nullptr, *y = nullptr;
        int *ecol = nullptr;
        double *eval = nullptr;
        uint16_t *erow = nullptr;
        long long ecap = 0;
        unsigned long long *owner = nullptr;
        unsigned *shared = nullptr, *epoch = nullptr;
        int *segpos = nullptr;
        unsigned long long *raw = nullptr, *skeys = nullptr, *pkeys = nullptr;
        long long pcap = 0, skcap = 0;
        double *g = nullptr;
    } dyn;
    // a block of nr right-hand sides (rorbk_multi_create; 0: one right-hand
    // side): x, b are row-major n x nr and m x nr, r and r32 hold nr columns in
    // the SELL copy's row order, the loop state and the dynamic-block buffers
    // are nr one-column sets side by side
    int nr = 0;
    struct {
        int *iperm = nullptr;       // [m] SELL position of each row
        unsigned *grp = nullptr;    // [8] loop tickets and "some column runs" flags, residual ticket
        long long mpos = 0;         // SELL positions (32 per slice)
        int grid = 0, grid32 = 0;   // blocks of the column-block residual (FP64, FP32)
        std::vector<rorbk_result> last;   // per-column results of the last solve
    } mr;
    // launch shapes that do not change results (rorbk_autotune; 0: default)
    struct Tune {
        int topk = 0, collect = 0, mark = 0, scatter = 0, residual = 0;
        int unroll = 0;   // iterations per WHILE-body execution of the graphs
    } tune;
    rorbk::Ctl *ctl = nullptr;
    rorbk::Ctl *ctl_in = nullptr;       // inner (FP32) loop state of the mixed form
    // graphs
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr, cap_stream3 = nullptr;
    cudaGraphExec_t exec_fp64 = nullptr, exec_mixed = nullptr;
    std::vector<void *> tmp;
};

namespace rorbk {

// host helpers implemented in rorbk.cu
rorbk_status fail(rorbk_ctx *h, rorbk_status st, const std::string &msg);
rorbk_status cuda_check(rorbk_ctx *h, cudaError_t e, const char *what);
// incremental residual: CSC copy of A and the change log, built once (incremental.cu)
rorbk_status ensure_incremental(rorbk_ctx *h);
constexpr int kIncRefreshDefault = 50;
// what rorbk_last_error(NULL) reports: the last failure on this thread that
// left no handle
void record_setup_error(const std::string &msg);
void *dev_alloc(rorbk_ctx *h, size_t bytes);

// setup (kernels_setup.cu)
// refresh: new values of the same pattern; reuses every buffer (rorbk_update_values)
rorbk_status build_setup(rorbk_ctx *h, const std::vector<int> &host_row_ptr, bool refresh = false);
// Column-major copy of A built on the device: cp [n+1], crow [nnz] (rows
// ascending in each column), cval [nnz] = a_ij / scale[i] (scale == NULL: a_ij)
// and, if cval32 != NULL, its FP32 rounding.
rorbk_status build_csc(rorbk_ctx *h, const double *scale, int *cp, int *crow, double *cval, float *cval32);
void widen_values(rorbk_ctx *h, int dtype);   // FP32 <-> FP64 value copies
void fill_dense_columns(rorbk_ctx *h);        // column indices of a dense A held as CSR

// iteration launches (kernels_iter.cu); all enqueue on h->stream
void configure_kernels();
int residual_grid(rorbk_ctx *h);   // one resident wave of the residual kernel
int mres_grid(rorbk_ctx *h, int nr, int fp32);   // one resident wave of the column-block residual
// the tunable grids (per column), defaults where h->tune holds 0
int grid_topk(rorbk_ctx *h);
int grid_collect(rorbk_ctx *h);
int grid_mark(rorbk_ctx *h);
int grid_scatter(rorbk_ctx *h);
void launch_begin(rorbk_ctx *h, const double *b, const double *x0, double *x, int use_cond,
                  unsigned long long hcond);
void launch_iteration(rorbk_ctx *h, const double *b, double *x, double *r, int use_cond,
                      unsigned long long hcond, int weighted = 0, int inc = 0);
void launch_mixed_inner(rorbk_ctx *h, int use_cond, unsigned long long hcond_inner, int inc = 0);
void launch_weights(rorbk_ctx *h, const double *r);   // residual-weighted running sum from r
void launch_static_forced(rorbk_ctx *h, int tau, const double *b, double *x);
void launch_mixed_outer(rorbk_ctx *h, int use_cond, unsigned long long hcond_inner);
void launch_mixed_update(rorbk_ctx *h, int use_cond, unsigned long long hcond_outer);
void launch_residual_only(rorbk_ctx *h, const double *b, const double *x, double *r);
void launch_topk_only(rorbk_ctx *h, const double *r, int *I);
void launch_residual32_only(rorbk_ctx *h, const float *b, const float *x, float *r);
// a block of right-hand sides: R = B - A X for all columns (FP32 or FP64), into
// the handle's residual buffer, and to R (m x nr row-major) if R != nullptr
void launch_residual_multi(rorbk_ctx *h, int fp32, const void *B, const void *X, void *R);
void launch_dynamic_given(rorbk_ctx *h, const int *I, const double *r, double *x);
void launch_dense_gram(rorbk_ctx *h, Ctl *ctl, int tensor_cores);   // dense A: G of the rows dyn.I into dyn.g
void launch_sample_probe(rorbk_ctx *h, uint64_t seed, uint64_t sysid, int64_t it, int64_t l,
                         long long *out);

}  // namespace rorbk
