// bits.cuh -- exact conversions to FP64 assembled from bit patterns in the
// integer pipes (the FP64 pipe issues at 1/64 of the FP32 rate on this GPU):
// U 2^-53 for a 53-bit integer U, and t 2^e for a float t.  Both are exact,
// so they equal the FP64 conversion followed by the scaling.  The same
// functions compile as plain C++ for the host tests.
#pragma once

#include <cstdint>
#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define WOB_BITS_FN __host__ __device__ __forceinline__
#else
#define WOB_BITS_FN inline
#endif
#if !defined(__CUDA_ARCH__)
#include <cmath>
#include <cstring>
#endif

namespace wob {

WOB_BITS_FN int clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

WOB_BITS_FN double double_of_bits(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
#endif
}

WOB_BITS_FN double double_of_hilo(uint32_t hi, uint32_t lo)
{
#if defined(__CUDA_ARCH__)
    return __hiloint2double((int)hi, (int)lo);
#else
    return double_of_bits(((uint64_t)hi << 32) | lo);
#endif
}

WOB_BITS_FN uint32_t bits_of_float(float f)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t b;
    std::memcpy(&b, &f, sizeof b);
    return b;
#endif
}

// U 2^-53 for 0 <= U < 2^53, exact.  U = 1.f 2^k with k = 63 - clz(U): the
// significand is U shifted so that its leading one sits at bit 52, where
// adding it carries 1 into the exponent field; that field therefore holds
// 1023 + (k - 53) - 1 beforehand.
WOB_BITS_FN double u53_unit(uint64_t U)
{
    const int lz = clz64(U);
    const uint64_t bits = ((uint64_t)(1032 - lz) << 52) + (U << (lz - 11));
    return U != 0 ? double_of_bits(bits) : 0.0;
}

// t 2^e for a float t, exact: sign, exponent rebiased from 127 to 1023 and
// moved by e, the 23-bit significand at the top of the double's 52.  Zero,
// subnormal, infinite and NaN t and results outside the normal range take
// ldexp.
WOB_BITS_FN double scale2(float t, int e)
{
    const uint32_t b = bits_of_float(t);
    const int ef = (int)((b >> 23) & 0xFFu);
    const int ex = ef - 127 + 1023 + e;
    if (ef == 0 || ef == 255 || ex <= 0 || ex >= 2047) return t == 0.f ? 0.0 : ldexp((double)t, e);
    return double_of_hilo((b & 0x80000000u) | ((uint32_t)ex << 20) | ((b & 0x7FFFFFu) >> 3), b << 29);
}

}  // namespace wob
