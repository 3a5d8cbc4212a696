// Split of an FP64 value into two FP32 parts by integer operations on its bit
// pattern.  GB300 issues FP64 -> FP32 conversions on the FP64 pipe, which runs
// at 1/64 of the FP32 rate; the per-event setup of the FP32 kernels splits every
// momentum component (4 per particle) this way instead.
//
//   hi = x truncated to 24 significant bits (the leading bit and the top 23
//        fraction bits of x), lo = the next 24 bits of x truncated, so that
//   x = hi + lo + r,  |r| < 2^-47 |x|,  hi and lo of the sign of x (or lo = 0).
//
// Range: |x| in FP32's normal range [2^-126, 2^128); below it hi = lo = 0
// (signed), above it hi = +-inf; lo is 0 where it would fall below 2^-126, so
// the bound on r holds for |x| >= 2^-73.  NaN gives hi = NaN.  Host and device
// compile the same integer code.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define ME_SPLIT_HD __host__ __device__ __forceinline__
#else
#define ME_SPLIT_HD inline
#endif

namespace me {

ME_SPLIT_HD uint64_t split_bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

ME_SPLIT_HD float split_float_of(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
#endif
}

ME_SPLIT_HD int split_clz32(uint32_t v)  // v != 0
{
#if defined(__CUDA_ARCH__)
    return __clz((int)v);
#else
    return __builtin_clz(v);
#endif
}

ME_SPLIT_HD void split_f32(double x, float& hi, float& lo)
{
    const uint64_t b = split_bits_of(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);            // biased FP64 exponent
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;          // 52 fraction bits
    const int ef = e - 1023 + 127;                      // biased FP32 exponent of hi
    if (e == 0x7FF) {                                   // inf or NaN
        hi = split_float_of(m ? 0x7FC00000u : (sign | 0x7F800000u));
        lo = 0.0f;
        return;
    }
    if (ef <= 0) {                                      // below FP32's normal range (or zero)
        hi = lo = split_float_of(sign);
        return;
    }
    if (ef >= 255) {                                    // above it
        hi = split_float_of(sign | 0x7F800000u);
        lo = 0.0f;
        return;
    }
    hi = split_float_of(sign | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
    // remainder: the low 29 fraction bits r, worth r * 2^(e - 1075)
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFu);
    if (r == 0) {
        lo = split_float_of(sign);
        return;
    }
    const int p = 31 - split_clz32(r);                  // position of r's leading bit (0..28)
    const int el = e - 1075 + p + 127;                  // biased FP32 exponent of lo
    if (el <= 0) {
        lo = split_float_of(sign);
        return;
    }
    const uint32_t frac = (p >= 23 ? (r >> (p - 23)) : (r << (23 - p))) & 0x7FFFFFu;
    lo = split_float_of(sign | ((uint32_t)el << 23) | frac);
}

}  // namespace me
