// ff.cuh -- compensated FP32 arithmetic: a value is carried as an unevaluated
// sum hi + lo of two floats (about 44 significant bits).  Error-free
// transformations: Knuth's two-sum, Dekker's fast two-sum and the FMA form
// of Dekker's two-product; Dekker's (1971) correction step for the square
// root.  On the GPU every operation is written with the explicitly rounded
// intrinsics, so the compiler cannot contract or reassociate them.  The
// same functions compile as plain C++ (host tests, built without
// floating-point contraction), where the operations are the IEEE ones.
#pragma once

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define WOB_FF_FN __host__ __device__ __forceinline__
#else
#include <cmath>
#define WOB_FF_FN inline
#endif

namespace wob {

struct ff {
    float hi, lo;
};

// Correctly rounded single operations (round to nearest even).
WOB_FF_FN float rn_add(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
WOB_FF_FN float rn_sub(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
WOB_FF_FN float rn_mul(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
WOB_FF_FN float rn_div(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fdiv_rn(a, b);
#else
    return a / b;
#endif
}
WOB_FF_FN float rn_fma(float a, float b, float c)
{
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
WOB_FF_FN float rn_sqrt(float a)
{
#if defined(__CUDA_ARCH__)
    return __fsqrt_rn(a);
#else
    return std::sqrt(a);
#endif
}

// a + b exactly, as s + e (Knuth).
WOB_FF_FN ff two_sum(float a, float b)
{
    const float s = rn_add(a, b);
    const float bb = rn_sub(s, a);
    const float e = rn_add(rn_sub(a, rn_sub(s, bb)), rn_sub(b, bb));
    return {s, e};
}

// a + b exactly when |a| >= |b| (Dekker).
WOB_FF_FN ff fast_two_sum(float a, float b)
{
    const float s = rn_add(a, b);
    return {s, rn_sub(b, rn_sub(s, a))};
}

// a * b exactly, as p + e.
WOB_FF_FN ff two_prod(float a, float b)
{
    const float p = rn_mul(a, b);
    return {p, rn_fma(a, b, -p)};
}

WOB_FF_FN ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, rn_add(s.lo, rn_add(a.lo, b.lo)));
}

WOB_FF_FN ff ff_sub(ff a, ff b) { return ff_add(a, {-b.hi, -b.lo}); }

WOB_FF_FN ff ff_mul(ff a, ff b)
{
    const ff p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, rn_fma(a.hi, b.lo, rn_fma(a.lo, b.hi, p.lo)));
}

WOB_FF_FN ff ff_mul_f(ff a, float b)
{
    const ff p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, rn_fma(a.lo, b, p.lo));
}

// sqrt(u) for a float u >= 0: the rounded root plus Dekker's correction
// (u - s^2) / (2 s), with u - s^2 exact by an FMA.
WOB_FF_FN ff ff_sqrt(float u)
{
    const float s = rn_sqrt(u);
    if (!(s > 0.f)) return {s, 0.f};
    const float e = rn_fma(-s, s, u);
    return fast_two_sum(s, rn_div(e, rn_mul(2.f, s)));
}

// Sum of products a_i b_i of three float-float pairs, as a float-float
// (two-product and two-sum on the hi parts, the lo cross terms added to the
// error; the lo x lo products, below 2^-48 relative, are dropped).
WOB_FF_FN ff ff_dot3(const ff (&a)[3], const ff (&b)[3])
{
    ff s = two_prod(a[0].hi, b[0].hi);
    float e = rn_fma(a[0].hi, b[0].lo, rn_mul(a[0].lo, b[0].hi));
#if defined(__CUDACC__)
#pragma unroll
#endif
    for (int c = 1; c < 3; ++c) {
        const ff pc = two_prod(a[c].hi, b[c].hi);
        const ff t = two_sum(s.hi, pc.hi);
        s.hi = t.hi;
        e = rn_add(e, rn_add(t.lo, pc.lo));
        e = rn_fma(a[c].hi, b[c].lo, rn_fma(a[c].lo, b[c].hi, e));
    }
    e = rn_add(e, s.lo);
    return fast_two_sum(s.hi, e);
}

}  // namespace wob
