// rorbk.cu -- the C ABI declared in include/rorbk.h: handle life cycle,
// argument checks, device memory, the graph-captured iteration loop and the
// single-step entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {

static thread_local std::string g_setup_error;

void record_setup_error(const std::string &msg) { g_setup_error = msg; }

rorbk_status fail(rorbk_ctx *h, rorbk_status st, const std::string &msg) {
    if (h) h->err = msg;
    g_setup_error = msg;
    return st;
}

rorbk_status cuda_check(rorbk_ctx *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return RORBK_OK;
    cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? RORBK_ERR_OOM : RORBK_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

void *dev_alloc(rorbk_ctx *h, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    h->allocs.push_back(p);
    h->bytes += (int64_t)bytes;
    return p;
}

static rorbk_status device_status(rorbk_ctx *h, int code) {
    switch (code) {
        case kDevOk: return RORBK_OK;
        case kDevNotSpd: return fail(h, RORBK_ERR_NOT_SPD, "a block Gram is not positive definite");
        case kDevBounds: return fail(h, RORBK_ERR_BOUNDS, "a device index or scratch bound was exceeded");
        case kDevNumeric: return fail(h, RORBK_ERR_NUMERIC, "the residual is not finite");
        case kDevTimeout: return fail(h, RORBK_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up (asynchronous copy not completed)");
        default: return fail(h, RORBK_ERR_CUDA, "unknown device status");
    }
}

// Greedy residual tiles: consecutive rows, at most kTileRows rows and
// kTileNnz nonzeros, a longer row alone.
static void build_tiles(const std::vector<int> &rp, int m, std::vector<int> &tiles) {
    tiles.clear();
    int r = 0;
    while (r < m) {
        tiles.push_back(r);
        int nz = rp[r + 1] - rp[r];
        if (nz > kTileNnz) { ++r; continue; }
        int rows = 1, acc = nz;
        ++r;
        while (r < m && rows < kTileRows && acc + (rp[r + 1] - rp[r]) <= kTileNnz) {
            acc += rp[r + 1] - rp[r];
            ++rows;
            ++r;
        }
    }
    tiles.push_back(m);
}

// Starts capturing on cs: into a new graph, or appended to `parent` as a new
// independent component.
static cudaError_t begin_capture(cudaStream_t cs, cudaGraph_t parent) {
    if (!parent) return cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    return cudaStreamBeginCaptureToGraph(cs, parent, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
}

// Iterations per execution of a WHILE body.  Every iteration kernel returns at
// once when its loop has halted, and the last one sets the condition from the
// loop state, so a body of u iterations runs the same iterations as u
// executions of a body of one; it saves the conditional node's turnaround on
// u - 1 of every u iterations.
static int graph_unroll(const rorbk_ctx *h) { return h->tune.unroll > 0 ? h->tune.unroll : kGraphUnroll; }

// Destroys the handle's instantiated graphs; the next solve captures them again
// (after a change of launch shapes).
static void drop_graphs(rorbk_ctx *h) {
    cudaGraphExec_t *g[5] = {&h->exec_fp64, &h->exec_mixed, &h->exec_fp64_w, &h->exec_fp64_inc,
                             &h->exec_mixed_inc};
    bool any = false;
    for (auto *e : g) any = any || *e;
    if (!any) return;
    cudaStreamSynchronize(h->stream);
    for (auto *e : g)
        if (*e) { cudaGraphExecDestroy(*e); *e = nullptr; }
}

// Capture: k_begin, then WHILE(cond) { graph_unroll(h) iterations }.  With
// parent == NULL the graph is instantiated into h->exec_fp64, else it is
// appended to parent.
static rorbk_status build_graph_fp64(rorbk_ctx *h, cudaGraph_t parent = nullptr, int weighted = 0,
                                     int inc = 0) {
    rorbk_status st;
    cudaStream_t saved = h->stream;
    cudaStream_t cs = h->cap_stream, cs2 = h->cap_stream2;
    if ((st = cuda_check(h, begin_capture(cs, parent), "capture")))
        return st;
    cudaGraph_t graph = nullptr;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle hcond = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hcond, graph, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        h->stream = cs;
        launch_begin(h, h->bb, h->xb, h->xb, 1, (unsigned long long)hcond);
        if (weighted) {                 // the first draws' weights: r = b - A x0
            launch_residual_only(h, h->bb, h->xb, h->r);
            launch_weights(h, h->r);
        }
        e = cudaGetLastError();
    }
    cudaGraphNode_t wnode = nullptr;
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hcond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &cp);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            h->stream = cs2;
            for (int u = graph_unroll(h); u > 0; --u)
                launch_iteration(h, h->bb, h->xb, h->r, 1, (unsigned long long)hcond, weighted, inc);
            cudaError_t e2 = cudaGetLastError();
            cudaGraph_t body_out = nullptr;
            e = cudaStreamEndCapture(cs2, &body_out);
            if (e == cudaSuccess) e = e2;
        }
    }
    h->stream = saved;
    cudaGraph_t g_out = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(cs, &g_out);
    if (e == cudaSuccess) e = e3;
    if (!parent) {
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(weighted ? &h->exec_fp64_w : (inc ? &h->exec_fp64_inc : &h->exec_fp64),
                                     g_out, 0);
        if (g_out) cudaGraphDestroy(g_out);
    }
    return cuda_check(h, e, "building the iteration graph");
}

// Adds a WHILE node at the capture position of stream cs; returns its body.
static cudaError_t add_while(cudaStream_t cs, cudaGraphConditionalHandle *hc, cudaGraph_t *body) {
    cudaGraph_t graph = nullptr;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = *hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    e = cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &cp);
    if (e != cudaSuccess) return e;
    *body = cp.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
}

static cudaError_t new_handle(cudaStream_t cs, cudaGraphConditionalHandle *hc) {
    cudaGraph_t graph = nullptr;
    cudaStreamCaptureStatus cst;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    return cudaGraphConditionalHandleCreate(hc, graph, 0, cudaGraphCondAssignDefault);
}

// Capture: k_begin, then WHILE(outer) { FP64 residual + inner set-up,
// WHILE(inner) { graph_unroll(h) FP32 iterations }, x += d }.
static rorbk_status build_graph_mixed(rorbk_ctx *h, cudaGraph_t parent = nullptr, int inc = 0) {
    cudaStream_t saved = h->stream;
    cudaStream_t cs = h->cap_stream, cs2 = h->cap_stream2, cs3 = h->cap_stream3;
    cudaGraphConditionalHandle hout = 0, hin = 0;
    cudaGraph_t body1 = nullptr, body2 = nullptr, tmp = nullptr;
    cudaError_t e = begin_capture(cs, parent);
    if (e != cudaSuccess) return cuda_check(h, e, "capture");
    e = new_handle(cs, &hout);
    if (e == cudaSuccess) {
        h->stream = cs;
        launch_begin(h, h->bb, h->xb, h->xb, 1, (unsigned long long)hout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = add_while(cs, &hout, &body1);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs2, body1, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = new_handle(cs2, &hin);
        if (e == cudaSuccess) {
            h->stream = cs2;
            launch_mixed_outer(h, 1, (unsigned long long)hin);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = add_while(cs2, &hin, &body2);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs3, body2, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            h->stream = cs3;
            for (int u = graph_unroll(h); u > 0; --u)
                launch_mixed_inner(h, 1, (unsigned long long)hin, inc);
            cudaError_t e2 = cudaGetLastError();
            e = cudaStreamEndCapture(cs3, &tmp);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) {
            h->stream = cs2;
            launch_mixed_update(h, 1, (unsigned long long)hout);
            e = cudaGetLastError();
        }
        cudaError_t e3 = cudaStreamEndCapture(cs2, &tmp);
        if (e == cudaSuccess) e = e3;
    }
    h->stream = saved;
    cudaGraph_t g_out = nullptr;
    cudaError_t e4 = cudaStreamEndCapture(cs, &g_out);
    if (e == cudaSuccess) e = e4;
    if (!parent) {
        if (e == cudaSuccess) e = cudaGraphInstantiate(inc ? &h->exec_mixed_inc : &h->exec_mixed, g_out, 0);
        if (g_out) cudaGraphDestroy(g_out);
    }
    return cuda_check(h, e, "building the mixed-precision graph");
}

// Per-solve device state of a handle: vectors, reduction scratch, top-K
// lists, the dynamic-block workspace and the loop state.  Set-up data (A and
// its copies, the partition, the proposal, the static operators) is not part
// of it, so clones share that and own only this.
static rorbk_status alloc_workspace(rorbk_ctx *h) {
    const int64_t m = h->m, n = h->n;
    // a column-block handle keeps nr of every per-solve buffer, side by side;
    // its residual columns span the SELL copy's positions
    const int64_t nr = std::max(1, h->nr), mr = h->nr ? h->mr.mpos : m;
    cudaStream_t s = h->stream;
    h->r = (double *)dev_alloc(h, nr * mr * sizeof(double));
    h->xb = (double *)dev_alloc(h, nr * n * sizeof(double));
    h->bb = (double *)dev_alloc(h, nr * m * sizeof(double));
    h->partials = (double *)dev_alloc(h, nr * std::max(std::max(h->grid_res, std::max(h->mr.grid, h->mr.grid32)),
                                                       4 * h->num_sms) * sizeof(double) + 64);
    h->sd_scratch = (double *)dev_alloc(h, 2 * kMaxBlockRows * sizeof(double));
    h->wgt = (double *)dev_alloc(h, h->k * sizeof(double));
    h->wcdf = (double *)dev_alloc(h, h->k * sizeof(double));
    h->hist1 = (unsigned *)dev_alloc(h, nr * kHistBins * sizeof(unsigned));
    h->hist2 = (unsigned *)dev_alloc(h, nr * kHistBins * sizeof(unsigned));
    h->in_list = (int *)dev_alloc(h, nr * std::max(1, h->K) * sizeof(int));
    h->eq_list = (int *)dev_alloc(h, nr * kEqCap * sizeof(int));
    h->ctl = (Ctl *)dev_alloc(h, nr * sizeof(Ctl));
    h->ctl_in = (Ctl *)dev_alloc(h, nr * sizeof(Ctl));
    {
        auto &D = h->dyn;
        D.ecap = std::max<int64_t>(1, (int64_t)h->K * h->maxrow);
        int64_t np2 = 1;
        while (np2 < 2 * D.ecap) np2 <<= 1;
        D.pcap = 1;
        while (D.pcap < std::max<int64_t>(16 * D.ecap, 1 << 16)) D.pcap <<= 1;
        D.I = (int *)dev_alloc(h, nr * h->K * sizeof(int));
        D.estart = (int *)dev_alloc(h, nr * (h->K + 1) * sizeof(int));
        D.gdiag = (double *)dev_alloc(h, nr * h->K * sizeof(double));
        D.y = (double *)dev_alloc(h, nr * h->K * sizeof(double));
        D.ecol = (int *)dev_alloc(h, nr * D.ecap * sizeof(int));
        D.eval = (double *)dev_alloc(h, nr * D.ecap * sizeof(double));
        D.erow = (uint16_t *)dev_alloc(h, nr * D.ecap * sizeof(uint16_t));
        D.owner = (unsigned long long *)dev_alloc(h, nr * n * sizeof(unsigned long long));
        D.shared = (unsigned *)dev_alloc(h, nr * n * sizeof(unsigned));
        D.epoch = (unsigned *)dev_alloc(h, nr * sizeof(unsigned));
        D.segpos = (int *)dev_alloc(h, nr * n * sizeof(int));
        D.raw = (unsigned long long *)dev_alloc(h, nr * 2 * D.ecap * sizeof(unsigned long long));
        D.skcap = np2;
        D.skeys = (unsigned long long *)dev_alloc(h, nr * np2 * sizeof(unsigned long long));
        D.pkeys = (unsigned long long *)dev_alloc(h, nr * D.pcap * sizeof(unsigned long long));
        D.g = (double *)dev_alloc(h, nr * ((size_t)h->K * (h->K + 1) / 2) * sizeof(double));
        if (!D.I || !D.estart || !D.gdiag || !D.y || !D.ecol || !D.eval || !D.erow || !D.owner ||
            !D.shared || !D.epoch || !D.segpos || !D.raw || !D.skeys || !D.pkeys || !D.g)
            return fail(h, RORBK_ERR_OOM, "dynamic-block workspace");
        cudaMemsetAsync(D.owner, 0, nr * n * sizeof(unsigned long long), s);   // epoch 0: never
        cudaMemsetAsync(D.shared, 0, nr * n * sizeof(unsigned), s);
        cudaMemsetAsync(D.epoch, 0, nr * sizeof(unsigned), s);
    }
    if (h->K >= n) {   // the dynamic block in the n x n form: its rows as a dense K x n array, A_I^T r_I
        h->dynw = (double *)dev_alloc(h, ((size_t)h->K * n + n) * sizeof(double));
        if (!h->dynw) return fail(h, RORBK_ERR_OOM, "n x n dynamic workspace");
    }
    if (h->precision_built) {
        h->r32 = (float *)dev_alloc(h, nr * mr * sizeof(float));
        h->b32 = (float *)dev_alloc(h, nr * m * sizeof(float));
        h->d32 = (float *)dev_alloc(h, nr * n * sizeof(float));
        if (!h->r32 || !h->b32 || !h->d32) return fail(h, RORBK_ERR_OOM, "mixed workspace");
        if (h->format == RORBK_FORMAT_DENSE) {
            // tensor-core dynamic Gram: 128 x 128 lower tiles, the column chunks
            // split so that about two blocks per SM run
            const int64_t T = (h->K + 127) / 128, chunks = (n + 127) / 128;
            h->gram_tiles = (int)(T * (T + 1) / 2);
            h->gram_splits = (int)std::max<int64_t>(
                1, std::min<int64_t>(chunks, (2 * h->num_sms + h->gram_tiles - 1) / h->gram_tiles));
            h->gram_part = (float *)dev_alloc(h, (size_t)h->gram_tiles * h->gram_splits * 128 * 128 * sizeof(float));
            if (!h->gram_part) return fail(h, RORBK_ERR_OOM, "tensor-core Gram workspace");
        }
    }
    if (!h->r || !h->xb || !h->bb || !h->partials || !h->sd_scratch || !h->wgt || !h->wcdf ||
        !h->hist1 || !h->hist2 || !h->in_list ||
        !h->eq_list || !h->ctl || !h->ctl_in)
        return fail(h, RORBK_ERR_OOM, "workspace");
    cudaMemsetAsync(h->hist1, 0, nr * kHistBins * sizeof(unsigned), s);
    cudaMemsetAsync(h->hist2, 0, nr * kHistBins * sizeof(unsigned), s);
    cudaMemsetAsync(h->ctl, 0, nr * sizeof(Ctl), s);
    cudaMemsetAsync(h->ctl_in, 0, nr * sizeof(Ctl), s);
    return cuda_check(h, cudaGetLastError(), "workspace");
}

static rorbk_options defaults() {
    rorbk_options o;
    rorbk_default_options(&o);
    return o;
}

}  // namespace rorbk

namespace rorbk {
namespace {
// Counts the entries that are NaN or Inf.
__global__ void k_count_nonfinite_f64(const double *__restrict__ v, long long nn, int *out) {
    int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
        c += !isfinite(v[i]);
    if (c) atomicAdd(out, c);
}
__global__ void k_count_nonfinite_f32(const float *__restrict__ v, long long nn, int *out) {
    int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
        c += !isfinite(v[i]);
    if (c) atomicAdd(out, c);
}
}  // namespace
}  // namespace rorbk

using namespace rorbk;

extern "C" {

void rorbk_default_options(rorbk_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->n_static = 3;
    opt->precision = RORBK_PREC_FP64;
    opt->inner_tol = 1e-4;
    opt->inner_maxit = 2000000;
    opt->host_loop = 0;
    opt->poll = 64;
}

const char *rorbk_last_error(rorbk_handle h) {
    static const char none[] = "";
    if (!h) return g_setup_error.c_str();   // the last failure on this thread
    return h->err.empty() ? none : h->err.c_str();
}

void rorbk_free(rorbk_handle h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->exec_fp64) cudaGraphExecDestroy(h->exec_fp64);
    if (h->exec_mixed) cudaGraphExecDestroy(h->exec_mixed);
    if (h->exec_fp64_w) cudaGraphExecDestroy(h->exec_fp64_w);
    if (h->exec_fp64_inc) cudaGraphExecDestroy(h->exec_fp64_inc);
    if (h->exec_mixed_inc) cudaGraphExecDestroy(h->exec_mixed_inc);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
    if (h->cap_stream3) cudaStreamDestroy(h->cap_stream3);
    for (void *p : h->allocs) cudaFree(p);
    cudaSetDevice(cur);
    delete h;
}

rorbk_status rorbk_setup(const rorbk_matrix *A, const rorbk_partition *part, double lambda,
                         const rorbk_options *opt_in, rorbk_handle *out) {
    if (!out) return RORBK_ERR_INVALID_ARG;
    *out = nullptr;
    if (!A || !part) return RORBK_ERR_INVALID_ARG;
    rorbk_options opt = opt_in ? *opt_in : defaults();
    if (A->format != RORBK_FORMAT_CSR && A->format != RORBK_FORMAT_DENSE) return RORBK_ERR_UNSUPPORTED;
    if (A->dtype != RORBK_F64 && A->dtype != RORBK_F32) return RORBK_ERR_INVALID_ARG;
    const bool dense = A->format == RORBK_FORMAT_DENSE;
    if (A->m < 1 || A->n < 1 || A->m >= (1LL << 31) || A->n >= (1LL << 31)) return RORBK_ERR_INVALID_ARG;
    if (dense) {
        // every entry is stored: the matrix is held as CSR with all m*n entries
        if (!A->values || A->ld < A->n || A->m * A->n >= (1LL << 31)) return RORBK_ERR_INVALID_ARG;
    } else if (A->nnz < 0 || A->nnz >= (1LL << 31) || !A->row_ptr ||
               (A->nnz > 0 && (!A->col_idx || !A->values))) {
        return RORBK_ERR_INVALID_ARG;
    }
    const int64_t m = A->m, n = A->n, nnz = dense ? A->m * A->n : A->nnz;
    const int k = part->num_blocks;
    if (k < 1 || k > m || k > 65536) return RORBK_ERR_INVALID_ARG;

    rorbk_ctx *h = new rorbk_ctx();
    rorbk_status st;
    h->values_version = std::make_shared<int>(0);
    cudaGetDevice(&h->device);
    h->stream = (cudaStream_t)opt.stream;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    h->m = m; h->n = n; h->nnz = nnz; h->k = k;
    h->format = A->format; h->vdtype = A->dtype;
    h->K = (int)(m / k);
    h->precision_built = opt.precision == RORBK_PREC_MIXED ? 1 : 0;
    auto bail = [&](rorbk_status s) {
        std::string e = h->err.empty() ? std::string("setup failed") : h->err;
        rorbk_free(h);
        g_setup_error = e;
        *out = nullptr;
        return s;
    };

    // partition (Algorithm 1's contiguous blocks)
    h->h_off.resize(k + 1);
    if (part->offsets) {
        for (int t = 0; t <= k; ++t) h->h_off[t] = part->offsets[t];
        if (h->h_off[0] != 0 || h->h_off[k] != m) return bail(RORBK_ERR_INVALID_ARG);
        for (int t = 0; t < k; ++t)
            if (h->h_off[t + 1] <= h->h_off[t]) return bail(RORBK_ERR_INVALID_ARG);
    } else {
        const int64_t q = m / k, rem = m % k;
        for (int t = 0; t <= k; ++t) h->h_off[t] = t * q + std::min<int64_t>(t, rem);
    }
    for (int t = 0; t < k; ++t) h->smax = std::max<int>(h->smax, (int)(h->h_off[t + 1] - h->h_off[t]));
    if (h->smax > kMaxBlockRows || h->K > kMaxDynRows) return bail(RORBK_ERR_UNSUPPORTED);
    h->mu = lambda < 0 ? 1e-6 * (double)(m / k) : lambda;

    if ((st = cuda_check(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "stream")))
        return bail(st);
    if ((st = cuda_check(h, cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking), "stream")))
        return bail(st);
    if ((st = cuda_check(h, cudaStreamCreateWithFlags(&h->cap_stream3, cudaStreamNonBlocking), "stream")))
        return bail(st);
    configure_kernels();

    // copy A (CSR) and a host view of row_ptr for the tiling
    std::vector<int> hrp(m + 1);
    const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (dense) {
        for (int64_t i = 0; i <= m; ++i) hrp[i] = (int)(i * n);
    } else if (A->on_device) {
        if ((st = cuda_check(h, cudaMemcpy(hrp.data(), A->row_ptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost), "row_ptr")))
            return bail(st);
    } else {
        memcpy(hrp.data(), A->row_ptr, (m + 1) * sizeof(int));
    }
    if (hrp[0] != 0 || hrp[m] != nnz) return bail(fail(h, RORBK_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[m] = nnz"));
    for (int64_t i = 0; i < m; ++i)
        if (hrp[i + 1] < hrp[i]) return bail(fail(h, RORBK_ERR_INVALID_ARG, "row_ptr must be non-decreasing"));
    int maxrow = 0;
    for (int64_t i = 0; i < m; ++i) maxrow = std::max(maxrow, hrp[i + 1] - hrp[i]);

    h->rowptr = (int *)dev_alloc(h, (m + 1) * sizeof(int));
    // +16 entries: the static kernel's bulk copies round block ranges up to
    // 16-byte boundaries
    h->col = (int *)dev_alloc(h, (nnz + 16) * sizeof(int));
    h->val = (double *)dev_alloc(h, (nnz + 16) * sizeof(double));
    h->off = (int *)dev_alloc(h, (k + 1) * sizeof(int));
    h->cdf = (double *)dev_alloc(h, k * sizeof(double));
    h->crowsum = (double *)dev_alloc(h, k * sizeof(double));
    h->pbar = (double *)dev_alloc(h, k * sizeof(double));
    if (!h->rowptr || !h->col || !h->val || !h->off || !h->cdf || !h->crowsum || !h->pbar)
        return bail(fail(h, RORBK_ERR_OOM, "matrix"));
    cudaStream_t s = h->stream;
    // rows of a dense A are copied from its leading dimension into n-entry rows
    const size_t esz = A->dtype == RORBK_F64 ? sizeof(double) : sizeof(float);
    auto copy_values = [&](void *dst) {
        if (!nnz) return;
        if (dense) cudaMemcpy2DAsync(dst, n * esz, A->values, A->ld * esz, n * esz, m, kind, s);
        else cudaMemcpyAsync(dst, A->values, nnz * esz, kind, s);
    };
    if (dense) {
        cudaMemcpyAsync(h->rowptr, hrp.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
        fill_dense_columns(h);
    } else {
        cudaMemcpyAsync(h->rowptr, A->row_ptr, (m + 1) * sizeof(int), kind, s);
        if (nnz) cudaMemcpyAsync(h->col, A->col_idx, nnz * sizeof(int), kind, s);
    }
    if (A->dtype == RORBK_F64) {
        copy_values(h->val);
        if (h->precision_built) {
            h->val32 = (float *)dev_alloc(h, (nnz + 16) * sizeof(float));
            if (!h->val32) return bail(fail(h, RORBK_ERR_OOM, "fp32 values"));
        }
    } else {
        h->val32 = (float *)dev_alloc(h, (nnz + 16) * sizeof(float));
        if (!h->val32) return bail(fail(h, RORBK_ERR_OOM, "fp32 values"));
        copy_values(h->val32);
    }
    {
        std::vector<int> off32(k + 1);
        for (int t = 0; t <= k; ++t) off32[t] = (int)h->h_off[t];
        cudaMemcpyAsync(h->off, off32.data(), (k + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
        if ((st = cuda_check(h, cudaStreamSynchronize(s), "copy A"))) return bail(st);
    }
    widen_values(h, A->dtype);
    if ((st = cuda_check(h, cudaGetLastError(), "value copies"))) return bail(st);

    // residual tiles
    std::vector<int> tiles;
    build_tiles(hrp, (int)m, tiles);
    h->ntiles = (int)tiles.size() - 1;
    h->tile_row0 = (int *)dev_alloc(h, tiles.size() * sizeof(int));
    h->grid_res = residual_grid(h);
    h->maxrow = maxrow;
    if (!h->tile_row0) return bail(fail(h, RORBK_ERR_OOM, "workspace"));
    cudaMemcpyAsync(h->tile_row0, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if ((st = alloc_workspace(h))) return bail(st);

    if ((st = build_setup(h, hrp))) return bail(st);
    *out = h;
    return RORBK_OK;
}


rorbk_status rorbk_update_values(rorbk_handle h, const void *values, int32_t dtype, int32_t on_device) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!values) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_update_values: values");
    if (dtype != h->vdtype) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_update_values: dtype must be the handle's value type");
    if (h->adj_scale)
        return fail(h, RORBK_ERR_UNSUPPORTED, "rorbk_update_values: an adjoint handle follows its primal; set up a new one");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    const size_t esz = dtype == RORBK_F64 ? sizeof(double) : sizeof(float);
    const long long nnz = h->nnz;
    rorbk_status st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_update_values");
    // the new values in scratch first, checked before the handle is touched
    void *tmp = nullptr;
    int *bad = nullptr;
    if (!st && nnz) {
        cudaError_t e = cudaMalloc(&tmp, nnz * esz + sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaSetDevice(cur);
            return fail(h, RORBK_ERR_OOM, "rorbk_update_values: scratch");
        }
        bad = (int *)((char *)tmp + nnz * esz);
        cudaMemsetAsync(bad, 0, sizeof(int), s);
        cudaMemcpyAsync(tmp, values, nnz * esz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        const int g = (int)std::max(1LL, std::min<long long>(8LL * h->num_sms, (nnz + 255) / 256));
        if (dtype == RORBK_F64) k_count_nonfinite_f64<<<g, 256, 0, s>>>((const double *)tmp, nnz, bad);
        else k_count_nonfinite_f32<<<g, 256, 0, s>>>((const float *)tmp, nnz, bad);
        int hb = 0;
        st = cuda_check(h, cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s), "rorbk_update_values");
        if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_update_values");
        if (!st && hb) st = fail(h, RORBK_ERR_NUMERIC, "rorbk_update_values: the values hold NaN or Inf");
        if (!st) {
            cudaMemcpyAsync(dtype == RORBK_F64 ? (void *)h->val : (void *)h->val32, tmp, nnz * esz,
                            cudaMemcpyDeviceToDevice, s);
            widen_values(h, dtype);
            st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_update_values");
        }
        cudaFree(tmp);
    }
    if (!st) st = build_setup(h, std::vector<int>(), true);
    if (!st && h->values_version) ++*h->values_version;
    // this handle's own column-major copy now; those of handles sharing the
    // set-up at their next incremental solve
    if (!st && h->csc_ptr) {
        st = build_csc(h, nullptr, h->csc_ptr, h->csc_row, h->csc_val, h->csc_val32);
        if (!st) h->csc_version = *h->values_version;
    }
    cudaSetDevice(cur);
    return st;
}

// Checks a solve's arguments (h, options) and enqueues on s the copies of b
// and x0 into the handle's workspace and the initial loop state.
static rorbk_status solve_prepare(rorbk_handle h, const double *b, const double *x0, bool b_host,
                                  double tol, int64_t maxit, const rorbk_options &opt,
                                  cudaStream_t s) {
    if (!b || maxit < 0 || !(tol >= 0)) return fail(h, RORBK_ERR_INVALID_ARG, "solve: b, tol >= 0, maxit >= 0");
    if (opt.n_static < 0 || opt.n_static > 64) return fail(h, RORBK_ERR_INVALID_ARG, "n_static");
    const bool mixed = opt.precision == RORBK_PREC_MIXED;
    if (opt.precision != RORBK_PREC_FP64 && !mixed)
        return fail(h, RORBK_ERR_INVALID_ARG, "unknown precision mode");
    if (mixed && !h->precision_built)
        return fail(h, RORBK_ERR_UNSUPPORTED,
                    "mixed precision needs a handle set up with precision = RORBK_PREC_MIXED");
    if (mixed && (!(opt.inner_tol > 0) || opt.inner_maxit < 1))
        return fail(h, RORBK_ERR_INVALID_ARG, "inner_tol > 0 and inner_maxit >= 1");
    if (opt.dist_mode != RORBK_DIST_PAPER && opt.dist_mode != RORBK_DIST_RESIDUAL_WEIGHTED)
        return fail(h, RORBK_ERR_INVALID_ARG, "unknown dist_mode");
    if (mixed && opt.dist_mode == RORBK_DIST_RESIDUAL_WEIGHTED)
        return fail(h, RORBK_ERR_UNSUPPORTED, "residual-weighted draws are available in FP64 precision");
    if (opt.residual_mode != RORBK_RESIDUAL_EXACT && opt.residual_mode != RORBK_RESIDUAL_INCREMENTAL)
        return fail(h, RORBK_ERR_INVALID_ARG, "unknown residual_mode");
    const bool inc = opt.residual_mode == RORBK_RESIDUAL_INCREMENTAL;
    if (inc && opt.dist_mode == RORBK_DIST_RESIDUAL_WEIGHTED)
        return fail(h, RORBK_ERR_UNSUPPORTED, "the incremental residual is not combined with residual-weighted draws");
    if (inc && opt.refresh < 0) return fail(h, RORBK_ERR_INVALID_ARG, "refresh >= 0");
    if (opt.fault_inject != RORBK_FAULT_NONE && opt.fault_inject != RORBK_FAULT_WAIT_LIMIT)
        return fail(h, RORBK_ERR_INVALID_ARG, "unknown fault_inject");
    if (inc && h->K >= h->n)
        return fail(h, RORBK_ERR_UNSUPPORTED,
                    "the incremental residual does not log the n x n form of the dynamic update (K >= n)");
    if (h->nr && (inc || opt.dist_mode != RORBK_DIST_PAPER))
        return fail(h, RORBK_ERR_UNSUPPORTED,
                    "a block of right-hand sides is solved with the paper's draws and the exact residual");
    if (inc) {
        rorbk_status st = ensure_incremental(h);
        if (st) return st;
    }
    const int64_t m = h->m, n = h->n, nr = std::max(1, h->nr);
    cudaMemcpyAsync(h->bb, b, nr * m * sizeof(double), b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    if (x0) cudaMemcpyAsync(h->xb, x0, nr * n * sizeof(double), b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    Ctl c;
    memset(&c, 0, sizeof(c));
    c.maxit = maxit;
    c.iter_base = opt.start_iter;
    c.seed = opt.seed;
    c.sysid = opt.system_id;
    c.tol = tol;
    c.n_static = opt.n_static;
    c.has_x0 = x0 != nullptr;
    c.inner_tol = opt.inner_tol;
    c.inner_maxit = opt.inner_maxit;
    c.weighted = opt.dist_mode == RORBK_DIST_RESIDUAL_WEIGHTED;
    c.scdf = nullptr;                   // P's running sum until weights replace it
    c.inc = inc;
    c.inc_refresh = opt.refresh > 0 ? opt.refresh : kIncRefreshDefault;
    c.log_cap = inc ? h->ilog_cap : 0;
    c.log_col = inc ? h->ilog_col : nullptr;
    c.log_val = inc ? h->ilog_val : nullptr;
    c.fault = opt.fault_inject;
    // one loop state per column; a block of columns reads opt->trace as an
    // array of nr records, one per column
    std::vector<Ctl> cs(nr, c);
    if (opt.trace && !mixed)
        for (int64_t j = 0; j < nr; ++j) {
            const rorbk_trace &t = opt.trace[j];
            cs[j].trace_cap = t.capacity;
            cs[j].tr_tau = (long long *)t.tau;
            cs[j].tr_rrn = t.rrn;
            cs[j].tr_I = t.I;
            cs[j].tr_x = t.x;
            cs[j].tr_dyn = t.dyn;
        }
    // the pageable source is copied before cudaMemcpyAsync returns
    return cuda_check(h, cudaMemcpyAsync(h->ctl, cs.data(), nr * sizeof(Ctl), cudaMemcpyHostToDevice, s),
                      "solve prologue");
}

// Enqueues on s the copy of the solution out of the workspace and of the
// final loop state into *c.
// (*c holds one loop state per column: nr of them for a block of columns.)
static cudaError_t solve_collect(rorbk_handle h, double *x, bool x_host, cudaStream_t s, Ctl *c) {
    const int64_t nr = std::max(1, h->nr);
    cudaError_t e = cudaMemcpyAsync(x, h->xb, nr * h->n * sizeof(double),
                                    x_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, h->ctl, nr * sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    return e;
}

// Status and result of a finished solve from its final loop state.
static rorbk_status solve_result(rorbk_handle h, const Ctl &c, bool mixed, float ms,
                                 rorbk_result *res) {
    const rorbk_status st = c.status ? device_status(h, c.status) : (c.done ? RORBK_OK : RORBK_NOT_CONVERGED);
    if (res) {
        res->iters = c.iter;
        res->rrn = c.rrn;
        res->converged = c.done && c.status == 0;
        res->status = st;
        res->refinements = mixed ? c.outer : 0;
        res->time_ms = ms;
    }
    return st;
}

// A block of columns: every column's result kept in h->mr.last (and written
// to res[0 .. nr-1] when res_cols is set); the status is the first error of
// any column, else NOT_CONVERGED if one stopped at maxit, else OK.  *agg gets
// the block's summary: the largest iteration count and RRN, converged if all
// columns converged.
static rorbk_status solve_results_cols(rorbk_handle h, const Ctl *cs, bool mixed, float ms,
                                       rorbk_result *res_cols, rorbk_result *agg) {
    const int nr = h->nr;
    h->mr.last.assign(nr, rorbk_result{});
    rorbk_status worst = RORBK_OK;
    rorbk_result a{};
    a.converged = 1;
    for (int j = 0; j < nr; ++j) {
        const rorbk_status sj = solve_result(h, cs[j], mixed, ms, &h->mr.last[j]);
        if (sj < 0 && worst >= 0) worst = sj;
        else if (sj == RORBK_NOT_CONVERGED && worst == RORBK_OK) worst = sj;
        a.iters = std::max<int64_t>(a.iters, h->mr.last[j].iters);
        a.rrn = std::max(a.rrn, h->mr.last[j].rrn);
        a.converged &= h->mr.last[j].converged;
        a.refinements = std::max<int64_t>(a.refinements, h->mr.last[j].refinements);
    }
    a.status = worst;
    a.time_ms = ms;
    if (res_cols) std::copy(h->mr.last.begin(), h->mr.last.end(), res_cols);
    if (agg) *agg = a;
    return worst;
}

// The loop flag the host polls: the handle's own stop flag, or for a block of
// columns the group's "some column runs" flag (inverted on read).
static const int *halt_flag(rorbk_handle h, bool inner) {
    if (h->nr) return (const int *)(h->mr.grp + (inner ? 3 : 1));
    return inner ? &h->ctl_in->halt : &h->ctl->halt;
}
static cudaError_t read_halt(rorbk_handle h, bool inner, int *halt, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(halt, halt_flag(h, inner), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h->nr) *halt = !*halt;
    return e;
}

static rorbk_status solve_impl(rorbk_handle h, const double *b, const double *x0, bool b_host,
                               double *x, bool x_host, double tol, int64_t maxit,
                               const rorbk_options *opt_in, rorbk_result *res) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!x) return fail(h, RORBK_ERR_INVALID_ARG, "solve: x");
    rorbk_options opt = opt_in ? *opt_in : defaults();
    cudaSetDevice(h->device);
    cudaStream_t s = opt.stream ? (cudaStream_t)opt.stream : h->stream;
    rorbk_status st;
    if ((st = solve_prepare(h, b, x0, b_host, tol, maxit, opt, s))) return st;
    const bool mixed = opt.precision == RORBK_PREC_MIXED;
    std::vector<Ctl> cs(std::max(1, h->nr));
    Ctl &c = cs[0];
    const int weighted = opt.dist_mode == RORBK_DIST_RESIDUAL_WEIGHTED;
    const int inc = opt.residual_mode == RORBK_RESIDUAL_INCREMENTAL;
    cudaGraphExec_t *exec = mixed ? (inc ? &h->exec_mixed_inc : &h->exec_mixed)
                                  : (weighted ? &h->exec_fp64_w : (inc ? &h->exec_fp64_inc : &h->exec_fp64));
    if (!opt.host_loop && !*exec) {
        if ((st = cuda_check(h, cudaStreamSynchronize(s), "solve prologue"))) return st;
        if ((st = mixed ? build_graph_mixed(h, nullptr, inc) : build_graph_fp64(h, nullptr, weighted, inc)))
            return st;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t e = cudaSuccess;
    if (!opt.host_loop) {
        e = cudaGraphLaunch(*exec, s);
    } else {
        // host-driven: batches of `poll` iterations, stop flags read between them
        const int poll = std::max(1, opt.poll);
        cudaStream_t saved = h->stream;
        h->stream = s;
        launch_begin(h, h->bb, h->xb, h->xb, 0, 0);
        int halt = 0;
        if (!mixed) {
            if (weighted) {
                launch_residual_only(h, h->bb, h->xb, h->r);
                launch_weights(h, h->r);
            }
            int64_t launched = 0;
            if (h->nr) e = read_halt(h, false, &halt, s);
            while (e == cudaSuccess && !halt && launched < maxit) {
                for (int q = 0; q < poll && launched < maxit; ++q, ++launched)
                    launch_iteration(h, h->bb, h->xb, h->r, 0, 0, weighted, inc);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = read_halt(h, false, &halt, s);
            }
        } else {
            if (e == cudaSuccess) e = read_halt(h, false, &halt, s);
            while (e == cudaSuccess && !halt) {
                launch_mixed_outer(h, 0, 0);
                int ihalt = 0;
                e = cudaGetLastError();
                if (e == cudaSuccess) e = read_halt(h, true, &ihalt, s);
                int odone = 0;
                if (e == cudaSuccess && !h->nr) e = cudaMemcpy(&odone, &h->ctl->done, sizeof(int), cudaMemcpyDeviceToHost);
                while (e == cudaSuccess && !ihalt && !odone) {
                    for (int q = 0; q < poll; ++q) launch_mixed_inner(h, 0, 0, inc);
                    e = cudaGetLastError();
                    if (e == cudaSuccess) e = read_halt(h, true, &ihalt, s);
                }
                if (e == cudaSuccess) launch_mixed_update(h, 0, 0);
                if (e == cudaSuccess) e = read_halt(h, false, &halt, s);
            }
        }
        h->stream = saved;
    }
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = solve_collect(h, x, x_host, s, cs.data());
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((st = cuda_check(h, e, "solve"))) return st;
    if (h->nr) return solve_results_cols(h, cs.data(), mixed, ms, res, nullptr);
    return solve_result(h, c, mixed, ms, res);
}

rorbk_status rorbk_solve(rorbk_handle h, const double *b, const double *x0, double *x, double tol,
                         int64_t maxit, const rorbk_options *opt, rorbk_result *res) {
    if (h && h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "a block of right-hand sides: use rorbk_solve_multi");
    return solve_impl(h, b, x0, false, x, false, tol, maxit, opt, res);
}

rorbk_status rorbk_solve_host(rorbk_handle h, const double *b_host, const double *x0_host,
                              double *x_host, double tol, int64_t maxit, const rorbk_options *opt,
                              rorbk_result *res) {
    if (h && h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "a block of right-hand sides: use rorbk_solve_multi");
    return solve_impl(h, b_host, x0_host, true, x_host, true, tol, maxit, opt, res);
}

rorbk_status rorbk_solve_multi(rorbk_handle h, const double *B, const double *X0, double *X, double tol,
                               int64_t maxit, const rorbk_options *opt, rorbk_result *res) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_solve_multi: the handle is not a block of right-hand sides");
    return solve_impl(h, B, X0, false, X, false, tol, maxit, opt, res);
}

rorbk_status rorbk_solve_multi_host(rorbk_handle h, const double *B_host, const double *X0_host,
                                    double *X_host, double tol, int64_t maxit, const rorbk_options *opt,
                                    rorbk_result *res) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_solve_multi_host: the handle is not a block of right-hand sides");
    return solve_impl(h, B_host, X0_host, true, X_host, true, tol, maxit, opt, res);
}

rorbk_status rorbk_residual_multi(rorbk_handle h, int32_t precision, const void *B, const void *X,
                                  void *R, double *rr_host) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_residual_multi: not a block of right-hand sides");
    if (!B || !X) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_residual_multi: NULL B or X");
    if (precision != RORBK_PREC_FP64 && precision != RORBK_PREC_MIXED)
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_residual_multi: unknown precision");
    const bool fp32 = precision == RORBK_PREC_MIXED;
    if (fp32 && !h->precision_built)
        return fail(h, RORBK_ERR_UNSUPPORTED, "rorbk_residual_multi: the FP32 residual needs a mixed-precision handle");
    cudaSetDevice(h->device);
    launch_residual_multi(h, fp32, B, X, R);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "rorbk_residual_multi");
    if (st || !rr_host) return st;
    std::vector<Ctl> cs(h->nr);
    st = cuda_check(h, cudaMemcpyAsync(cs.data(), h->ctl, h->nr * sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream),
                    "rorbk_residual_multi");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "rorbk_residual_multi");
    if (!st)
        for (int j = 0; j < h->nr; ++j) rr_host[j] = cs[j].rr;
    return st;
}

}  // extern "C"

static void tuning_out(const rorbk_ctx *h, double us0, double us1, rorbk_tuning *t) {
    t->topk_blocks = grid_topk((rorbk_ctx *)h);
    t->collect_blocks = grid_collect((rorbk_ctx *)h);
    t->dyn_mark_blocks = grid_mark((rorbk_ctx *)h);
    t->dyn_scatter_blocks = grid_scatter((rorbk_ctx *)h);
    t->residual_blocks = h->tune.residual;
    t->graph_unroll = graph_unroll(h);
    t->us_default = us0;
    t->us_tuned = us1;
}

extern "C" {

rorbk_status rorbk_set_tuning(rorbk_handle h, const rorbk_tuning *t) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    drop_graphs(h);
    if (!t) { h->tune = rorbk_ctx::Tune(); return RORBK_OK; }
    if (t->topk_blocks < 0 || t->collect_blocks < 0 || t->dyn_mark_blocks < 0 || t->dyn_scatter_blocks < 0 ||
        t->residual_blocks < 0)
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_set_tuning: negative block count");
    if (t->graph_unroll < 0 || t->graph_unroll > kMaxGraphUnroll)
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_set_tuning: graph_unroll outside 0..16");
    h->tune.topk = t->topk_blocks;
    h->tune.collect = t->collect_blocks;
    h->tune.mark = t->dyn_mark_blocks;
    h->tune.scatter = t->dyn_scatter_blocks;
    h->tune.residual = t->residual_blocks;
    h->tune.unroll = t->graph_unroll;
    return RORBK_OK;
}

rorbk_status rorbk_autotune(rorbk_handle h, const double *b, int32_t precision, int64_t iters,
                            const char *cache_file, rorbk_tuning *out) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!b || iters < 1) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_autotune: b and iters >= 1");
    if (precision != RORBK_PREC_FP64 && precision != RORBK_PREC_MIXED)
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_autotune: unknown precision");
    const int nr = std::max(1, h->nr);
    char key[256];
    snprintf(key, sizeof(key), "m=%lld nnz=%lld k=%d nr=%d prec=%d sms=%d", (long long)h->m, (long long)h->nnz,
             h->k, nr, precision, h->num_sms);
    if (cache_file) {   // an earlier choice for this shape of problem
        FILE *f = fopen(cache_file, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof(line), f)) {
                if (strncmp(line, key, strlen(key)) != 0 || line[strlen(key)] != ' ') continue;
                int v[6];
                double us0 = 0, us1 = 0;
                if (sscanf(line + strlen(key),
                           " topk=%d collect=%d mark=%d scatter=%d residual=%d unroll=%d us=%lf,%lf", &v[0],
                           &v[1], &v[2], &v[3], &v[4], &v[5], &us0, &us1) == 8 &&
                    v[5] >= 0 && v[5] <= kMaxGraphUnroll) {
                    fclose(f);
                    cudaSetDevice(h->device);
                    drop_graphs(h);
                    h->tune.topk = v[0];
                    h->tune.collect = v[1];
                    h->tune.mark = v[2];
                    h->tune.scatter = v[3];
                    h->tune.residual = v[4];
                    h->tune.unroll = v[5];
                    if (out) tuning_out(h, us0, us1, out);
                    return RORBK_OK;
                }
            }
            fclose(f);
        }
    }
    cudaSetDevice(h->device);
    drop_graphs(h);
    const size_t xbytes = (size_t)nr * h->n * sizeof(double);
    double *x0 = nullptr, *x = nullptr;
    if (cudaMalloc(&x0, xbytes) != cudaSuccess || cudaMalloc(&x, xbytes) != cudaSuccess) {
        cudaGetLastError();
        if (x0) cudaFree(x0);
        return fail(h, RORBK_ERR_OOM, "rorbk_autotune: scratch x");
    }
    rorbk_options o;
    rorbk_default_options(&o);
    o.precision = precision;
    o.inner_tol = 1e-30;                      // the mixed form: inner iterations only
    o.stream = h->stream;
    std::vector<rorbk_result> res(nr);
    // the starting state: iters iterations from 0
    rorbk_status st = solve_impl(h, b, nullptr, false, x0, false, 0.0, iters, &o, res.data());
    if (st < 0) { cudaFree(x0); cudaFree(x); return st; }
    o.start_iter = iters;
    o.host_loop = 1;
    o.poll = (int32_t)std::min<int64_t>(iters, 1 << 20);
    auto time_it = [&](double *us) -> rorbk_status {
        double best = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            rorbk_status s2 = solve_impl(h, b, x0, false, x, false, 0.0, iters, &o, res.data());
            if (s2 < 0) return s2;
            best = std::min(best, res[0].time_ms * 1e3 / (double)iters);
        }
        *us = best;
        return RORBK_OK;
    };
    const auto saved = h->tune;
    h->tune = rorbk_ctx::Tune();
    double us0 = 0, cur = 0;
    st = time_it(&us0);
    cur = us0;
    // coordinate descent: each shape over 1/4 .. 4 x its default
    int *fields[5] = {&h->tune.topk, &h->tune.collect, &h->tune.mark, &h->tune.scatter, &h->tune.residual};
    const int defs[5] = {grid_topk(h), grid_collect(h), grid_mark(h), grid_scatter(h),
                         h->nr ? (precision == RORBK_PREC_MIXED ? h->mr.grid32 : h->mr.grid) : 0};
    static const double mult[4] = {0.25, 0.5, 2.0, 4.0};
    for (int f = 0; f < 5 && st == RORBK_OK; ++f) {
        if (defs[f] <= 0) continue;
        int best_v = *fields[f];
        for (double mlt : mult) {
            int v = std::max(1, (int)(defs[f] * mlt));
            if (f == 4) v = std::min(v, defs[f]);   // the residual: at most one resident wave
            if (v == defs[f]) continue;
            *fields[f] = v;
            double us = 0;
            if ((st = time_it(&us))) break;
            if (us < 0.98 * cur) { cur = us; best_v = v; }
        }
        *fields[f] = best_v;
    }
    // the graph's unroll, timed on graph-launched iterations (each candidate
    // captured afresh)
    if (st == RORBK_OK) {
        o.host_loop = 0;
        double gbest = 1e300;
        int ubest = kGraphUnroll;
        // the default first: another count is kept only if it is 2% faster
        for (int u : {kGraphUnroll, 1, 2, 8}) {
            if (u == kGraphUnroll && gbest < 1e300) continue;
            h->tune.unroll = u;
            drop_graphs(h);
            double us = 0;
            if ((st = time_it(&us))) break;
            if (us < 0.98 * gbest) { gbest = us; ubest = u; }
        }
        h->tune.unroll = ubest;
        drop_graphs(h);
    }
    cudaFree(x0);
    cudaFree(x);
    if (st) { h->tune = saved; return st; }
    if (cache_file) {
        FILE *f = fopen(cache_file, "a");
        if (f) {
            fprintf(f, "%s topk=%d collect=%d mark=%d scatter=%d residual=%d unroll=%d us=%.3f,%.3f\n", key,
                    h->tune.topk, h->tune.collect, h->tune.mark, h->tune.scatter, h->tune.residual,
                    h->tune.unroll, us0, cur);
            fclose(f);
        }
    }
    if (out) tuning_out(h, us0, cur, out);
    return RORBK_OK;
}

rorbk_status rorbk_multi_results(rorbk_handle h, rorbk_result *res) {
    if (!h || !res) return RORBK_ERR_INVALID_ARG;
    if (!h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_multi_results: not a block of right-hand sides");
    if ((int)h->mr.last.size() != h->nr) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_multi_results: no solve yet");
    std::copy(h->mr.last.begin(), h->mr.last.end(), res);
    return RORBK_OK;
}

}  // extern "C"

// A handle sharing src's set-up with its own per-solve workspace: one
// right-hand side (nr = 0, rorbk_clone) or a block of nr (rorbk_multi_create).
static rorbk_status clone_impl(rorbk_handle src, int nr, rorbk_handle *out) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(src->device);
    rorbk_status st = cuda_check(src, cudaStreamSynchronize(src->stream), "rorbk_clone");
    if (st) { cudaSetDevice(cur); return st; }
    if (!src->shared_setup) {   // the source's memory becomes jointly owned
        src->shared_setup = std::make_shared<DevBlocks>();
        src->shared_setup->device = src->device;
        src->shared_setup->p.swap(src->allocs);
    }
    rorbk_ctx *c = new rorbk_ctx(*src);
    c->err.clear();
    c->allocs.clear();
    c->tmp.clear();
    c->bytes = 0;
    c->nr = 0;                  // one right-hand side (rorbk_multi_create makes blocks)
    c->mr = decltype(c->mr)();
    c->exec_fp64 = c->exec_mixed = c->exec_fp64_w = c->exec_fp64_inc = c->exec_mixed_inc = nullptr;
    // the incremental residual's CSC copy and log belong to the handle that
    // built them: a clone builds its own at its first incremental solve
    c->csc_ptr = c->csc_row = nullptr;
    c->csc_val = nullptr;
    c->csc_val32 = nullptr;
    c->ilog_col = nullptr;
    c->ilog_val = nullptr;
    c->ilog_cap = 0;
    c->cap_stream = c->cap_stream2 = c->cap_stream3 = nullptr;
    auto bail = [&](rorbk_status e) {
        record_setup_error(c->err.empty() ? std::string("rorbk_clone failed") : c->err);
        rorbk_free(c);
        cudaSetDevice(cur);
        return e;
    };
    if (nr) {
        // the residual columns live in the SELL copy's row order: the
        // position of every row, the group tickets, one resident wave
        c->nr = nr;
        c->mr.mpos = (long long)src->sell.nslices * 32;
        c->mr.grid = mres_grid(c, nr, 0);
        c->mr.grid32 = mres_grid(c, nr, 1);
        std::vector<int> row((size_t)c->mr.mpos), ipos((size_t)c->m, -1);
        if ((st = cuda_check(c, cudaMemcpy(row.data(), src->sell.row, row.size() * sizeof(int),
                                           cudaMemcpyDeviceToHost), "rorbk_multi_create")))
            return bail(st);
        for (long long p = 0; p < c->mr.mpos; ++p)
            if (row[p] >= 0) ipos[row[p]] = (int)p;
        c->mr.iperm = (int *)dev_alloc(c, ipos.size() * sizeof(int));
        c->mr.grp = (unsigned *)dev_alloc(c, 8 * sizeof(unsigned));
        if (!c->mr.iperm || !c->mr.grp) return bail(fail(c, RORBK_ERR_OOM, "rorbk_multi_create"));
        cudaMemcpy(c->mr.iperm, ipos.data(), ipos.size() * sizeof(int), cudaMemcpyHostToDevice);
        if ((st = cuda_check(c, cudaMemset(c->mr.grp, 0, 8 * sizeof(unsigned)), "rorbk_multi_create")))
            return bail(st);
    }
    if ((st = cuda_check(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream")))
        return bail(st);
    if ((st = cuda_check(c, cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking), "stream")))
        return bail(st);
    if ((st = cuda_check(c, cudaStreamCreateWithFlags(&c->cap_stream3, cudaStreamNonBlocking), "stream")))
        return bail(st);
    if ((st = alloc_workspace(c))) return bail(st);
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "rorbk_clone"))) return bail(st);
    *out = c;
    cudaSetDevice(cur);
    return RORBK_OK;
}

extern "C" {

rorbk_status rorbk_clone(rorbk_handle src, rorbk_handle *out) {
    if (!out) return RORBK_ERR_INVALID_ARG;
    *out = nullptr;
    if (!src) return RORBK_ERR_INVALID_ARG;
    return clone_impl(src, 0, out);
}

rorbk_status rorbk_multi_create(rorbk_handle src, int32_t nr, rorbk_handle *out) {
    if (!out) return RORBK_ERR_INVALID_ARG;
    *out = nullptr;
    if (!src) return RORBK_ERR_INVALID_ARG;
    if (nr != 2 && nr != 4 && nr != 8 && nr != 16 && nr != 32)
        return fail(src, RORBK_ERR_INVALID_ARG, "rorbk_multi_create: nr must be 2, 4, 8, 16 or 32");
    if (src->nr) return fail(src, RORBK_ERR_INVALID_ARG, "rorbk_multi_create: the source is already a block");
    if (src->format != RORBK_FORMAT_CSR || src->n_wood || src->K >= src->n || !src->sell.nslices)
        return fail(src, RORBK_ERR_UNSUPPORTED,
                    "rorbk_multi_create: sparse (CSR) systems whose blocks and dynamic block have "
                    "fewer rows than A has columns");
    return clone_impl(src, nr, out);
}

rorbk_status rorbk_weighted_cdf(rorbk_handle h, const double *r, double *cdf_host) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!r || !cdf_host) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_weighted_cdf: NULL r or cdf_host");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    cudaMemsetAsync(&h->ctl->done, 0, sizeof(int), s);
    cudaMemsetAsync(&h->ctl->halt, 0, sizeof(int), s);
    launch_weights(h, r);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "rorbk_weighted_cdf");
    if (!st)
        st = cuda_check(h, cudaMemcpyAsync(cdf_host, h->wcdf, (size_t)h->k * sizeof(double),
                                           cudaMemcpyDeviceToHost, s), "rorbk_weighted_cdf");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_weighted_cdf");
    cudaSetDevice(cur);
    return st;
}

rorbk_status rorbk_dense_gram(rorbk_handle h, const int32_t *I, double *G, int32_t precision) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    if (!I || !G) return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_dense_gram: NULL I or G");
    if (h->format != RORBK_FORMAT_DENSE)
        return fail(h, RORBK_ERR_UNSUPPORTED, "rorbk_dense_gram: dense handles only");
    if (precision != RORBK_PREC_FP64 && precision != RORBK_PREC_MIXED)
        return fail(h, RORBK_ERR_INVALID_ARG, "rorbk_dense_gram: unknown precision");
    if (precision == RORBK_PREC_MIXED && !h->gram_part)
        return fail(h, RORBK_ERR_UNSUPPORTED,
                    "rorbk_dense_gram: the tensor-core Gram needs a handle set up with precision = MIXED");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    cudaMemsetAsync(&h->ctl->status, 0, sizeof(int), s);
    cudaMemsetAsync(&h->ctl->done, 0, sizeof(int), s);
    cudaMemsetAsync(&h->ctl->halt, 0, sizeof(int), s);
    cudaMemcpyAsync(h->dyn.I, I, (size_t)h->K * sizeof(int), cudaMemcpyDeviceToDevice, s);
    launch_dense_gram(h, h->ctl, precision == RORBK_PREC_MIXED);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "rorbk_dense_gram");
    if (!st)
        st = cuda_check(h, cudaMemcpyAsync(G, h->dyn.g, (size_t)h->K * (h->K + 1) / 2 * sizeof(double),
                                           cudaMemcpyDeviceToDevice, s),
                        "rorbk_dense_gram");
    int code = 0;
    if (!st) st = cuda_check(h, cudaMemcpyAsync(&code, &h->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s),
                             "rorbk_dense_gram");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "rorbk_dense_gram");
    if (!st && code) st = device_status(h, code);
    cudaSetDevice(cur);
    return st;
}

}  // extern "C"

struct rorbk_batch_ctx {
    int device = 0;
    int precision = RORBK_PREC_FP64;
    std::vector<rorbk_handle> hs;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

rorbk_status rorbk_batch_create(const rorbk_handle *hs, int32_t count, int32_t precision,
                                rorbk_batch *out) {
    if (!out) return RORBK_ERR_INVALID_ARG;
    *out = nullptr;
    auto reject = [](const char *msg) {
        record_setup_error(msg);
        return RORBK_ERR_INVALID_ARG;
    };
    if (!hs || count < 1) return reject("rorbk_batch_create: no handles");
    if (precision != RORBK_PREC_FP64 && precision != RORBK_PREC_MIXED)
        return reject("rorbk_batch_create: unknown precision mode");
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) return reject("rorbk_batch_create: NULL handle");
        if (hs[i]->device != hs[0]->device) return reject("rorbk_batch_create: handles on different devices");
        if (precision == RORBK_PREC_MIXED && !hs[i]->precision_built)
            return reject("rorbk_batch_create: mixed precision needs handles set up for it");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return reject("rorbk_batch_create: a handle appears twice (clone it instead)");
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(hs[0]->device);
    rorbk_batch_ctx *bt = new rorbk_batch_ctx();
    bt->device = hs[0]->device;
    bt->precision = precision;
    bt->hs.assign(hs, hs + count);
    cudaGraph_t parent = nullptr;
    rorbk_status st = cuda_check(hs[0], cudaGraphCreate(&parent, 0), "rorbk_batch_create");
    for (int i = 0; i < count && st == RORBK_OK; ++i) {
        rorbk_ctx *h = hs[i];
        st = cuda_check(h, cudaStreamSynchronize(h->stream), "rorbk_batch_create");
        if (st == RORBK_OK)
            st = precision == RORBK_PREC_MIXED ? build_graph_mixed(h, parent) : build_graph_fp64(h, parent);
        if (st) record_setup_error(h->err);
    }
    if (st == RORBK_OK) {
        st = cuda_check(hs[0], cudaGraphInstantiate(&bt->exec, parent, 0), "rorbk_batch_create");
        if (st) record_setup_error(hs[0]->err);
    }
    if (parent) cudaGraphDestroy(parent);
    cudaSetDevice(cur);
    if (st) {
        rorbk_batch_free(bt);
        return st;
    }
    *out = bt;
    return RORBK_OK;
}

rorbk_status rorbk_batch_solve(rorbk_batch bt, const double *const *b, const double *const *x0,
                               double *const *x, double tol, int64_t maxit,
                               const rorbk_options *opt_in, const uint64_t *system_ids,
                               rorbk_result *res) {
    auto reject = [](rorbk_status e, const char *msg) {
        record_setup_error(msg);
        return e;
    };
    if (!bt || !b || !x) return reject(RORBK_ERR_INVALID_ARG, "rorbk_batch_solve: NULL batch, b or x");
    rorbk_options opt = opt_in ? *opt_in : defaults();
    if (opt.precision != bt->precision)
        return reject(RORBK_ERR_INVALID_ARG, "rorbk_batch_solve: precision differs from the batch's");
    if (opt.host_loop || opt.trace || opt.dist_mode != RORBK_DIST_PAPER ||
        opt.residual_mode != RORBK_RESIDUAL_EXACT)
        return reject(RORBK_ERR_UNSUPPORTED,
                      "rorbk_batch_solve: no host loop, trace, residual-weighted draws or incremental "
                      "residual in a batch");
    const int count = (int)bt->hs.size();
    for (int i = 0; i < count; ++i)
        if (!b[i] || !x[i]) return reject(RORBK_ERR_INVALID_ARG, "rorbk_batch_solve: NULL b[i] or x[i]");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(bt->device);
    cudaStream_t s = opt.stream ? (cudaStream_t)opt.stream : bt->hs[0]->stream;
    rorbk_status st = RORBK_OK;
    for (int i = 0; i < count && st == RORBK_OK; ++i) {
        rorbk_options oi = opt;
        if (system_ids) oi.system_id = system_ids[i];
        st = solve_prepare(bt->hs[i], b[i], x0 ? x0[i] : nullptr, false, tol, maxit, oi, s);
        if (st) record_setup_error(bt->hs[i]->err);
    }
    if (st) { cudaSetDevice(cur); return st; }
    std::vector<std::vector<Ctl>> cs(count);
    for (int i = 0; i < count; ++i) cs[i].resize(std::max(1, bt->hs[i]->nr));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t e = cudaGraphLaunch(bt->exec, s);
    cudaEventRecord(e1, s);
    for (int i = 0; i < count && e == cudaSuccess; ++i) e = solve_collect(bt->hs[i], x[i], false, s, cs[i].data());
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        st = cuda_check(bt->hs[0], e, "rorbk_batch_solve");
        record_setup_error(bt->hs[0]->err);
        cudaSetDevice(cur);
        return st;
    }
    const bool mixed = opt.precision == RORBK_PREC_MIXED;
    rorbk_status worst = RORBK_OK;
    for (int i = 0; i < count; ++i) {
        const rorbk_status si = bt->hs[i]->nr
                                    ? solve_results_cols(bt->hs[i], cs[i].data(), mixed, ms, nullptr, res ? res + i : nullptr)
                                    : solve_result(bt->hs[i], cs[i][0], mixed, ms, res ? res + i : nullptr);
        if (si < 0 && worst >= 0) worst = si;
        else if (si == RORBK_NOT_CONVERGED && worst == RORBK_OK) worst = si;
    }
    cudaSetDevice(cur);
    return worst;
}

void rorbk_batch_free(rorbk_batch bt) {
    if (!bt) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(bt->device);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    cudaSetDevice(cur);
    delete bt;
}

rorbk_status rorbk_get_info(rorbk_handle h, rorbk_info *info) {
    if (!h || !info) return RORBK_ERR_INVALID_ARG;
    info->m = h->m; info->n = h->n; info->nnz = h->nnz;
    info->num_blocks = h->k; info->dyn_rows = h->K; info->max_block_rows = h->smax;
    info->format = h->format; info->lambda = h->mu; info->device_bytes = h->bytes;
    return RORBK_OK;
}

rorbk_status rorbk_get_proposal(rorbk_handle h, double *cdf_host, double *c_rowsum_host) {
    if (!h) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    rorbk_status st = RORBK_OK;
    if (cdf_host) st = cuda_check(h, cudaMemcpy(cdf_host, h->cdf, h->k * sizeof(double), cudaMemcpyDeviceToHost), "cdf");
    if (!st && c_rowsum_host) st = cuda_check(h, cudaMemcpy(c_rowsum_host, h->crowsum, h->k * sizeof(double), cudaMemcpyDeviceToHost), "rowsum");
    return st;
}

rorbk_status rorbk_get_static_operator(rorbk_handle h, int64_t t, double *W_host) {
    if (!h || !W_host || t < 0 || t >= h->k) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    const int r0 = (int)h->h_off[t], s = (int)(h->h_off[t + 1] - h->h_off[t]);
    if (h->n_wood) {   // a block in the s >= n form stores V_t (n x n) instead
        long long wpw = -1;
        rorbk_status st0 = cuda_check(h, cudaMemcpy(&wpw, h->wood_ptr + t, sizeof(long long), cudaMemcpyDeviceToHost), "V");
        if (st0) return st0;
        if (wpw >= 0)
            return cuda_check(h, cudaMemcpy(W_host, h->wood_ss + wpw, (size_t)h->n * h->n * sizeof(double),
                                            cudaMemcpyDeviceToHost), "V");
    }
    int sp[2];
    long long wp;
    rorbk_status st = cuda_check(h, cudaMemcpy(sp, h->ops.s_ptr + t, 2 * sizeof(int), cudaMemcpyDeviceToHost), "W");
    if (st) return st;
    st = cuda_check(h, cudaMemcpy(&wp, h->ops.w_ptr + t, sizeof(long long), cudaMemcpyDeviceToHost), "W");
    if (st) return st;
    const int nS = sp[1] - sp[0];
    std::vector<uint16_t> idx(std::max(1, nS));
    std::vector<double> wss((size_t)std::max(1, nS * nS)), wd(s);
    std::vector<int> pos(s);
    if (nS) {
        cudaMemcpy(idx.data(), h->ops.s_idx + sp[0], nS * sizeof(uint16_t), cudaMemcpyDeviceToHost);
        cudaMemcpy(wss.data(), h->ops.w_ss + wp, (size_t)nS * nS * sizeof(double), cudaMemcpyDeviceToHost);
    }
    cudaMemcpy(wd.data(), h->ops.w_diag + r0, s * sizeof(double), cudaMemcpyDeviceToHost);
    st = cuda_check(h, cudaMemcpy(pos.data(), h->ops.s_pos + r0, s * sizeof(int), cudaMemcpyDeviceToHost), "W");
    if (st) return st;
    for (int a = 0; a < s; ++a)
        for (int b2 = 0; b2 < s; ++b2) W_host[(size_t)a * s + b2] = 0.0;
    for (int a = 0; a < s; ++a)
        if (pos[a] < 0) W_host[(size_t)a * s + a] = wd[a];
    for (int i = 0; i < nS; ++i)
        for (int j = 0; j < nS; ++j) W_host[(size_t)idx[i] * s + idx[j]] = wss[(size_t)i * nS + j];
    return RORBK_OK;
}

rorbk_status rorbk_sample(rorbk_handle h, uint64_t seed, uint64_t system_id, int64_t it, int64_t l,
                          int64_t *tau_host) {
    if (!h || !tau_host) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    long long *d = (long long *)h->partials;
    launch_sample_probe(h, seed, system_id, it, l, d);
    long long v = 0;
    rorbk_status st = cuda_check(h, cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, h->stream), "sample");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "sample");
    *tau_host = v;
    return st;
}

rorbk_status rorbk_static_update(rorbk_handle h, int64_t tau, const double *b, double *x) {
    if (!h || !b || !x || tau < 0 || tau >= h->k) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    launch_static_forced(h, (int)tau, b, x);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "static update");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "static update");
    return st;
}

rorbk_status rorbk_residual(rorbk_handle h, const double *b, const double *x, double *r,
                            double *rr_host) {
    if (!h || !b || !x || !r) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    launch_residual_only(h, b, x, r);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "residual");
    if (!rr_host) return st;            // enqueue only
    Ctl c;
    if (!st) st = cuda_check(h, cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream), "residual");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "residual");
    if (!st && rr_host) *rr_host = c.rr;
    return st;
}

rorbk_status rorbk_residual32(rorbk_handle h, const float *b, const float *x, float *r,
                              double *rr_host) {
    if (!h || !b || !x || !r) return RORBK_ERR_INVALID_ARG;
    if (!h->precision_built)
        return fail(h, RORBK_ERR_UNSUPPORTED, "the FP32 residual needs a handle set up for mixed precision");
    cudaSetDevice(h->device);
    launch_residual32_only(h, b, x, r);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "residual32");
    if (!rr_host) return st;
    Ctl c;
    if (!st) st = cuda_check(h, cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream), "residual32");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "residual32");
    if (!st) *rr_host = c.rr;
    return st;
}

rorbk_status rorbk_topk(rorbk_handle h, const double *r, int32_t *I) {
    if (!h || !r || !I) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    launch_topk_only(h, r, I);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "top-K");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "top-K");
    return st;
}

rorbk_status rorbk_dynamic_update(rorbk_handle h, const int32_t *I, const double *r, double *x) {
    if (!h || !I || !r || !x) return RORBK_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaMemsetAsync(&h->ctl->status, 0, sizeof(int), h->stream);
    cudaMemsetAsync(&h->ctl->done, 0, sizeof(int), h->stream);
    cudaMemsetAsync(&h->ctl->halt, 0, sizeof(int), h->stream);
    launch_dynamic_given(h, I, r, x);
    rorbk_status st = cuda_check(h, cudaGetLastError(), "dynamic update");
    int code = 0;
    if (!st) st = cuda_check(h, cudaMemcpyAsync(&code, &h->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "dynamic update");
    if (!st) st = cuda_check(h, cudaStreamSynchronize(h->stream), "dynamic update");
    if (!st && code) st = device_status(h, code);
    return st;
}

}  // extern "C"
