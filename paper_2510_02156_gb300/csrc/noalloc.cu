// noalloc.cu -- a residual entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a
// residual: code running inside a custom allocator or a memory-pool callback,
// processes whose device memory is fully reserved up front by a framework,
// and real-time loops that forbid allocation after start-up.  For them
// rorbk_csr_residual_noalloc computes r = b - A x and ||r||^2 for a CSR
// matrix held in the caller's device memory, with the per-block partial sums
// and the completion counter kept in a file-scope __device__ array of fixed
// size instead of allocated scratch.
//
// Consequences of the static scratch:
//   - every GPU that loads the library holds kScratchBlocks doubles plus a
//     counter until the process exits (about 512 KiB);
//   - all calls on one device share it and it keeps the last call's contents;
//     every call clears the completion counter on its stream before its
//     kernel (a 4-byte cudaMemsetAsync, which allocates nothing), so calls
//     issued in stream order are independent even after a launch that never
//     finished; calls that overlap on the GPU (different streams, no
//     ordering) race on the scratch and give wrong results;
//   - the first call on each device looks up the scratch's device address
//     (cudaGetSymbolAddress) with that device current and keeps it for the
//     process; make that first call before any stream capture begins, and do
//     not call the entry point after cudaDeviceReset, which ends the context
//     the kept address belongs to.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {
namespace {

constexpr int kRowsPerBlock = 256;                 // one thread per row
constexpr int kScratchBlocks = 65536;              // => at most 2^24 rows
constexpr int kMaxDevices = 64;

struct NoallocScratch {
    double partial[kScratchBlocks];
    unsigned ticket;
    unsigned pad[63];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_lock;
NoallocScratch *g_scratch_ptr[kMaxDevices] = {};

// Same arithmetic as the handle's residual: each row is one fused
// multiply-add chain over its stored entries in order, FP32-stored values
// widened exactly.
template <typename V>
__global__ void __launch_bounds__(kRowsPerBlock)
    k_csr_residual_noalloc(int m, const int *__restrict__ row_ptr, const int *__restrict__ col,
                           const V *__restrict__ val, const double *__restrict__ b,
                           const double *__restrict__ x, double *__restrict__ r,
                           double *__restrict__ rr_out, NoallocScratch *scratch) {
    __shared__ double red[32];
    __shared__ int is_last;
    const int i = blockIdx.x * kRowsPerBlock + threadIdx.x;
    double rr = 0.0;
    if (i < m) {
        double acc = 0.0;
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) acc = __fma_rn(widen(val[p]), x[col[p]], acc);
        const double ri = __dsub_rn(b[i], acc);
        r[i] = ri;
        rr = __fma_rn(ri, ri, rr);
    }
    rr = block_sum(rr, red);
    if (threadIdx.x == 0) {
        scratch->partial[blockIdx.x] = rr;
        __threadfence();
        is_last = atomicAdd(&scratch->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) tot += scratch->partial[q];
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) {
        *rr_out = tot;
        scratch->ticket = 0u;       // ready for the next call
    }
}

NoallocScratch *scratch_for_current_device(int *dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    *dev_out = dev;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = (NoallocScratch *)p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace rorbk

extern "C" rorbk_status rorbk_csr_residual_noalloc(int64_t m, int64_t n, int64_t nnz,
                                                   const int32_t *row_ptr, const int32_t *col_idx,
                                                   const void *values, int32_t dtype,
                                                   const double *b, const double *x, double *r,
                                                   double *rr_out, void *stream) {
    using namespace rorbk;
    if (m < 1 || n < 1 || nnz < 0 || !row_ptr || (nnz > 0 && (!col_idx || !values)) || !b || !x ||
        !r || !rr_out || (dtype != RORBK_F64 && dtype != RORBK_F32))
        return fail(nullptr, RORBK_ERR_INVALID_ARG,
                    "rorbk_csr_residual_noalloc: null pointer, non-positive size or unknown dtype");
    if (m > (int64_t)kRowsPerBlock * kScratchBlocks || n >= (1LL << 31) || nnz >= (1LL << 31))
        return fail(nullptr, RORBK_ERR_INVALID_ARG,
                    "rorbk_csr_residual_noalloc: at most 16777216 rows (the fixed scratch holds "
                    "65536 per-block partial sums), n and nnz below 2^31");
    int dev = 0;
    NoallocScratch *scratch = scratch_for_current_device(&dev);
    if (!scratch)
        return fail(nullptr, RORBK_ERR_CUDA,
                    "rorbk_csr_residual_noalloc: the scratch's device address could not be found");
    const unsigned grid = (unsigned)((m + kRowsPerBlock - 1) / kRowsPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    // a launch that stopped part-way (an earlier error on the stream) may have
    // left the counter raised: clear it in stream order before this kernel
    rorbk_status st = cuda_check(nullptr, cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned), s),
                                 "rorbk_csr_residual_noalloc");
    if (st) return st;
    if (dtype == RORBK_F64)
        k_csr_residual_noalloc<double><<<grid, kRowsPerBlock, 0, s>>>(
            (int)m, row_ptr, col_idx, (const double *)values, b, x, r, rr_out, scratch);
    else
        k_csr_residual_noalloc<float><<<grid, kRowsPerBlock, 0, s>>>(
            (int)m, row_ptr, col_idx, (const float *)values, b, x, r, rr_out, scratch);
    return cuda_check(nullptr, cudaGetLastError(), "rorbk_csr_residual_noalloc");
}
