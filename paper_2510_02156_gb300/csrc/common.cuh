// common.cuh -- small device helpers for the ROR-BK kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rorbk {

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (X0,X1,X2,X3) -> (hi(M1 X2)^X1^K0, lo(M1 X2), hi(M0 X0)^X3^K1, lo(M0 X0)),
// the key advanced by the Weyl increments between rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                              uint64_t c3, uint64_t k0, uint64_t k1,
                                              uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Block draw of Algorithm 1: u from word 0 of the Philox block at counter
// (it, l, 0, 0), key (seed, sysid); tau = min{t : u * cdf[k-1] < cdf[t]}.
__device__ __forceinline__ int sample_block(const double *cdf, int k, uint64_t seed,
                                            uint64_t sysid, uint64_t it, uint64_t l) {
    uint64_t w[4];
    philox4x64_10(it, l, 0, 0, seed, sysid, w);
    double u = (double)(w[0] >> 11) * 0x1.0p-53;
    double target = u * cdf[k - 1];
    int lo = 0, hi = k;               // first t with cdf[t] > target
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    return lo < k ? lo : k - 1;
}

// Order-preserving key of |v| (non-negative doubles compare as uint64).
__device__ __forceinline__ unsigned long long abs_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long abs_key(float v) {
    return abs_key((double)v);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree for a fixed blockDim); result valid in
// thread 0.  scratch: >= 32 elements of shared memory.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *scratch) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T s = 0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        s = lane < nw ? scratch[lane] : T(0);
        s = warp_sum(s);
    }
    return s;
}

// Exclusive block scan of one int per thread; returns the prefix, *total gets
// the block total.  scratch: >= 33 ints of shared memory.
__device__ __forceinline__ int block_exclusive_scan(int v, int *scratch, int *total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        int w = lane < nw ? scratch[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) scratch[lane] = w;     // inclusive warp totals
        if (lane == nw - 1) scratch[32] = w;
    }
    __syncthreads();
    int prefix = x - v + (wid > 0 ? scratch[wid - 1] : 0);
    *total = scratch[32];
    __syncthreads();
    return prefix;
}

// Bitonic sort of n (power of two) 64-bit keys, ascending, by one block.
__device__ __forceinline__ void block_bitonic_sort(unsigned long long *keys, int n) {
    for (int kk = 2; kk <= n; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long a = keys[i], b = keys[ixj];
                    bool up = (i & kk) == 0;
                    if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// Bitonic sort of (key, idx) pairs so that larger keys come first and equal
// keys keep ascending idx (the top-K order of Algorithm 1 with ties to the
// lower row).  n is a power of two; padding uses key 0 / idx INT_MAX.
__device__ __forceinline__ bool topk_before(unsigned long long ka, int ia,
                                            unsigned long long kb, int ib) {
    return ka > kb || (ka == kb && ia < ib);
}
__device__ __forceinline__ void block_bitonic_sort_desc(unsigned long long *keys, int *idx,
                                                        int n) {
    for (int kk = 2; kk <= n; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long a = keys[i], b = keys[ixj];
                    int ia = idx[i], ib = idx[ixj];
                    bool up = (i & kk) == 0;
                    // "up" segments end with a before b in topk order
                    bool swap = up ? topk_before(b, ib, a, ia) : topk_before(a, ia, b, ib);
                    if (swap) { keys[i] = b; keys[ixj] = a; idx[i] = ib; idx[ixj] = ia; }
                }
            }
            __syncthreads();
        }
    }
}

// Exact FP32 -> FP64 widening with integer operations only (the hardware
// conversion runs on the FP64 pipe): normal numbers re-bias the exponent,
// subnormals are normalised, zeros keep their sign, Inf/NaN keep their
// payload.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
    const int lz = __clz(man | 1u) - 8;                  // leading zeros inside the 24-bit field
    const unsigned long long sub_ex = (unsigned long long)(897 - lz) << 52;
    const unsigned long long sub_man = ((unsigned long long)(man << lz) & 0x7fffffull) << 29;
    const unsigned long long norm = ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)man << 29);
    const unsigned long long special = (0x7ffull << 52) | ((unsigned long long)man << 29);
    unsigned long long d = ex == 0xffu ? special : norm;
    d = ex == 0u ? (man == 0u ? 0ull : (sub_ex | sub_man)) : d;
    return __longlong_as_double((long long)(sign | d));
}
__device__ __forceinline__ double widen(double d) { return d; }

__device__ __forceinline__ int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

__device__ __forceinline__ void set_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

// ------------------------------------------------- dense SPD helpers
// Cholesky G = L L^T of an nS x nS row-major array in place (right-looking,
// zero multipliers skipped), one block of threads.  Returns false if a pivot
// is not positive (the factorisation continues with pivot 1 so that every
// thread leaves the loop).
__device__ __forceinline__ bool block_cholesky(double *G, int ld, int nS, int *bad) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < nS; ++j) {
        if (threadIdx.x == 0) {
            double d = G[(long long)j * ld + j];
            if (!(d > 0.0)) { *bad = 1; d = 1.0; }
            G[(long long)j * ld + j] = sqrt(d);
        }
        __syncthreads();
        double l = G[(long long)j * ld + j];
        for (int i = j + 1 + threadIdx.x; i < nS; i += blockDim.x)
            G[(long long)i * ld + j] = G[(long long)i * ld + j] / l;
        __syncthreads();
        for (int a = j + 1 + wid; a < nS; a += nw) {
            double la = G[(long long)a * ld + j];
            if (la == 0.0) continue;
            for (int b = j + 1 + lane; b <= a; b += 32) {
                double lb = G[(long long)b * ld + j];
                if (lb != 0.0)
                    G[(long long)a * ld + b] = __fma_rn(-la, lb, G[(long long)a * ld + b]);
            }
        }
        __syncthreads();
    }
    for (int a = threadIdx.x; a < nS; a += blockDim.x)
        for (int b = a + 1; b < nS; ++b) G[(long long)a * ld + b] = 0.0;
    __syncthreads();
    return true;
}

// <row a, row b> over ascending columns (merge of two sorted CSR rows).
template <typename V>
__device__ __forceinline__ double row_merge_dot(const int *col, const V *val, int p, int pe,
                                                int q, int qe) {
    double s = 0.0;
    while (p < pe && q < qe) {
        int cp = col[p], cq = col[q];
        if (cp == cq) { s = __fma_rn((double)val[p], (double)val[q], s); ++p; ++q; }
        else if (cp < cq) ++p;
        else ++q;
    }
    return s;
}

// ----------------------------------------------------- TMA bulk copies
// 1-D bulk copies global -> shared completed on an mbarrier (Hopper/Blackwell
// cp.async.bulk).  Source and destination 16-byte aligned, size a multiple of
// 16 bytes.  A block that is not part of a cluster is its own cluster, so the
// shared::cluster destination is the block's own shared memory.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase: returns false after max_tries polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase,
                                                  long long max_tries) {
    for (long long t = 0; t < max_tries; ++t)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------- 5th-generation tensor cores
// tcgen05 (sm_100 family): the accumulator lives in tensor memory (TMEM,
// 512 columns x 128 lanes of 32 bits per SM), allocated by one warp; one
// thread issues the MMAs, whose operands are read from shared memory through
// 64-bit matrix descriptors; tcgen05.commit arrives on an mbarrier when the
// issued MMAs are done; each warp reads its 32 lanes back with tcgen05.ld.
//
// Operand layout used here: K-major, no swizzle, made of core matrices of 8
// rows x 16 bytes (8 x 4 FP32/TF32 values) stored contiguously (128 bytes,
// row r at 16 r).  Descriptor fields: start address >> 4 (bits 0-13), the
// byte distance between core matrices adjacent along K >> 4 (bits 16-29), the
// distance between adjacent 8-row groups >> 4 (bits 32-45), descriptor
// version 1 (bits 46-47); base offset, LBO mode and layout type (no swizzle)
// are zero.
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned k_stride,
                                                        unsigned row8_stride) {
    return (unsigned long long)((saddr >> 4) & 0x3FFFu) |
           ((unsigned long long)((k_stride >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((row8_stride >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::tf32 with an FP32 accumulator, both
// operands K-major: D format F32 (bits 4-5 = 1), A and B format TF32 (bits
// 7-9 and 10-12 = 2), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr unsigned idesc_tf32_f32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tmem_alloc(unsigned *slot, unsigned ncols) {   // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {  // the allocating warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D (+)= A B^T, M = 128 lanes of TMEM from column d_tmem on; accumulate != 0
// adds to D.
__device__ __forceinline__ void mma_tf32(unsigned d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 consecutive 32-bit columns of this warp's 32 TMEM lanes (lane = thread).
__device__ __forceinline__ void tmem_ld_32cols(unsigned taddr, unsigned (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace rorbk
