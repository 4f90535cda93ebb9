// topk_key.cuh -- the radix key of |v| in the top-K passes, for FP32 values.
//
// The top-K selection ranks rows by the bit pattern of the FP64 value |r_i|
// (for non-negative doubles that order is the numeric order).  An FP32
// residual's key is the key of (double)|v|.  Here it is formed from the
// float's bits with integer operations: the exponent re-biased from 127 to
// 1023, the 23-bit fraction moved to the top of the 52-bit one, subnormal
// floats normalised, infinity mapped to the FP64 infinity.  It equals the key
// of the converted value for every float that is not a NaN (a NaN residual
// ends the solve before any top-K pass).  The hardware conversion would run
// on the FP64 pipe, of which this part has little.
#pragma once
#include <stdint.h>

__host__ __device__ __forceinline__ unsigned long long topk_key_f32_bits(uint32_t u) {
    u &= 0x7fffffffu;
    uint32_t e = u >> 23, f = u & 0x7fffffu;
    if (e == 0xffu) return (0x7ffull << 52) | ((unsigned long long)f << 29);
    if (e == 0u) {
        if (f == 0u) return 0ull;
#ifdef __CUDA_ARCH__
        const int lz = __clz(f);
#else
        const int lz = __builtin_clz(f);
#endif
        const int sh = lz - 8;                        // brings the leading 1 to bit 23
        f = (f << sh) & 0x7fffffu;
        return ((unsigned long long)(897 - sh) << 52) | ((unsigned long long)f << 29);
    }
    return ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)f << 29);
}
