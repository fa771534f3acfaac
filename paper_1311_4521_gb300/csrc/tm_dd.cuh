// tm_dd.cuh -- double-float arithmetic: a value as the unevaluated sum of two
// FP32 numbers (hi + lo, |lo| <= ulp(hi)/2), about 48 significant bits.
//
// GB300 issues FP64 fused multiply-adds at 2 per SM per clock against 128
// FP32 FMAs, so FP64-accurate stencil arithmetic is cheaper as FP32 pairs
// combined by error-free transformations (Knuth's TwoSum, Dekker's
// Fast2Sum, and the exact product error of an FMA) than as FP64 operations.
// The building blocks follow the double-word algorithms of Dekker (1971)
// and of Joldes, Muller and Popescu (ACM TOMS 2017).  Every operation on the
// components goes through the __f*_rn intrinsics, which the compiler never
// contracts into FMAs (a contraction would break the error-free steps).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#ifndef TM_HD
#define TM_HD __host__ __device__ __forceinline__
#endif

namespace twm {

#if defined(__CUDA_ARCH__)
TM_HD float f_add(float a, float b) { return __fadd_rn(a, b); }
TM_HD float f_sub(float a, float b) { return __fsub_rn(a, b); }
TM_HD float f_mul(float a, float b) { return __fmul_rn(a, b); }
TM_HD float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float f_add(float a, float b) { return a + b; }
inline float f_sub(float a, float b) { return a - b; }
inline float f_mul(float a, float b) { return a * b; }
inline float f_fma(float a, float b, float c) { return fmaf(a, b, c); }
#endif

struct dd {
    float hi, lo;
    dd() = default;
    TM_HD constexpr dd(float h, float l = 0.f) : hi(h), lo(l) {}
    TM_HD explicit operator double() const { return double(hi) + double(lo); }
};

// s + e = a + b exactly (Knuth)
TM_HD dd two_sum(float a, float b)
{
    float s = f_add(a, b);
    float bb = f_sub(s, a);
    float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
    return {s, e};
}

// s + e = a + b exactly, for |a| >= |b| (Dekker)
TM_HD dd fast_two_sum(float a, float b)
{
    float s = f_add(a, b);
    return {s, f_sub(b, f_sub(s, a))};
}

// p + e = a * b exactly (FMA)
TM_HD dd two_prod(float a, float b)
{
    float p = f_mul(a, b);
    return {p, f_fma(a, b, -p)};
}

// sum of two double-floats (the "sloppy" variant: relative error ~2^-46 of
// the larger operand, enough for the stencil sums here)
TM_HD dd operator+(dd x, dd y)
{
    dd s = two_sum(x.hi, y.hi);
    float e = f_add(s.lo, f_add(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

TM_HD dd operator-(dd x) { return {-x.hi, -x.lo}; }
TM_HD dd operator-(dd x, dd y) { return x + dd{-y.hi, -y.lo}; }

// product (relative error ~2^-45)
TM_HD dd operator*(dd x, dd y)
{
    dd p = two_prod(x.hi, y.hi);
    float e = f_fma(x.hi, y.lo, f_fma(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

// quotient by one Newton correction of the FP32 quotient
TM_HD dd operator/(dd x, dd y)
{
    float q1 = x.hi / y.hi;
    dd r = x - y * dd{q1};
    float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}

TM_HD dd &operator+=(dd &a, dd b) { return a = a + b; }
TM_HD dd &operator-=(dd &a, dd b) { return a = a - b; }

TM_HD dd abs_dd(dd x) { return x.hi < 0.f ? -x : x; }

// Compensated dot-product accumulator (Ogita, Rump and Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 2005, algorithm Dot2, extended to
// double-float factors): the exact product of the high parts goes through
// TwoSum into s, every error term and the cross products of high and low
// parts are summed in FP32 into c; the result is as if computed with twice
// the working precision and normalised once at the end.
struct dot2 {
    float s = 0.f, c = 0.f;
    TM_HD void add(dd x, dd y)  // += x y
    {
        dd p = two_prod(x.hi, y.hi);
        dd t = two_sum(s, p.hi);
        s = t.hi;
        c = f_add(c, f_add(t.lo, f_fma(x.hi, y.lo, f_fma(x.lo, y.hi, p.lo))));
    }
    TM_HD void sub(dd x, dd y) { add(dd{-x.hi, -x.lo}, y); }  // -= x y
    TM_HD dd result() const { return two_sum(s, c); }
};

// nearest double-float to a double: hi = fl32(x), lo = fl32(x - hi)
TM_HD dd dd_from_double(double x)
{
    float h = float(x);
    return {h, float(x - double(h))};
}

}  // namespace twm
