// ff.cuh -- compensated FP32 arithmetic: a value is carried as an unevaluated
// sum hi + lo of two floats (about 44 significant bits).  Error-free
// transformations: Knuth's two-sum, Dekker's fast two-sum and the FMA form
// of Dekker's two-product; Dekker's (1971) correction step for the square
// root.  Every operation is written with the explicitly rounded intrinsics,
// so the compiler cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace wob {

struct ff {
    float hi, lo;
};

// a + b exactly, as s + e (Knuth).
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b exactly, as p + e.
__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const ff p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    const ff p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// sqrt(u) for a float u >= 0: the rounded root plus Dekker's correction
// (u - s^2) / (2 s), with u - s^2 exact by an FMA.
__device__ __forceinline__ ff ff_sqrt(float u)
{
    const float s = __fsqrt_rn(u);
    if (!(s > 0.f)) return {s, 0.f};
    const float e = __fmaf_rn(-s, s, u);
    return fast_two_sum(s, __fdiv_rn(e, __fmul_rn(2.f, s)));
}

}  // namespace wob
