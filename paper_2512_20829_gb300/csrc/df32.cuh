// Double-float ("df") arithmetic on the single-precision pipe.
//
// A df value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2; it carries about 48 significant bits, against 24 for a
// float and 53 for a double, at a fraction of the cost of double precision on
// this GPU (whose FP64 pipe runs at 1/64 of the FP32 rate).  The operations
// are composed from error-free transformations of IEEE single precision with
// round-to-nearest:
//   two_sum(a, b)       s + e = a + b exactly        (Knuth, TAOCP vol. 2, 4.2.2)
//   fast_two_sum(a, b)  the same when |a| >= |b|     (Dekker 1971)
//   two_prod(a, b)      p + e = a b exactly, e = fma(a, b, -p)
// Sums and products renormalise once at the end and carry a relative error of
// a few u^2 (u = 2^-24), or u^2 times the operands' magnitude where a sum
// cancels.  The explicitly rounded intrinsics keep the compiler from
// contracting or reassociating these sequences.
#pragma once
#include <cuda_runtime.h>

namespace fla {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_of(float h) { return {h, 0.0f}; }

// Nearest df of a double: hi the rounded value, lo the rounded remainder.
__device__ __forceinline__ df df_of(double d)
{
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(__dsub_rn(d, (double)h))};
}

__device__ __forceinline__ double df_value(df a) { return (double)a.hi + (double)a.lo; }

// The same split on the host (kernel arguments).
inline df df_host(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }

// a + b: the exact sum of the high parts, the low parts added to its error,
// and one renormalisation.  Where the sum cancels, the error term can exceed
// the sum and fast_two_sum's low part is then inexact by at most u times that
// term: the result stays within u^2 (|a| + |b|) of a + b.
__device__ __forceinline__ df operator+(df a, df b)
{
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator+(df a, float b)
{
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// a + b without the final renormalisation (|lo| up to a few ulp(hi)): for
// running sums whose value is renormalised once at the end.
__device__ __forceinline__ df add_unnorm(df a, df b)
{
    const df s = two_sum(a.hi, b.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

// y + c k in one pass: the exact product of the high parts and the cross terms
// added to the exact sum's error, one renormalisation.
__device__ __forceinline__ df df_axpy(df c, df k, df y)
{
    const df p = two_prod(c.hi, k.hi);
    const df s = two_sum(y.hi, p.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(y.lo, p.lo));
    e = __fmaf_rn(c.hi, k.lo, __fmaf_rn(c.lo, k.hi, e));
    return fast_two_sum(s.hi, e);
}

// df_axpy without the final renormalisation (|lo| up to a few ulp(hi)).
__device__ __forceinline__ df axpy_unnorm(df c, df k, df y)
{
    const df p = two_prod(c.hi, k.hi);
    const df s = two_sum(y.hi, p.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(y.lo, p.lo));
    e = __fmaf_rn(c.hi, k.lo, __fmaf_rn(c.lo, k.hi, e));
    return {s.hi, e};
}

// Compensated dot product (Ogita, Rump and Oishi 2005, "Dot2"): the running
// sum s of the rounded products of the high parts, with every rounding error
// -- of the products (two_prod) and of the additions (two_sum) -- and the
// cross terms with the low parts collected in e.  The result is as accurate
// as a sum evaluated in twice the working precision.
struct DotAcc {
    float s, e;
};

__device__ __forceinline__ DotAcc dot_first(df a, df b)
{
    const df p = two_prod(a.hi, b.hi);
    return {p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo))};
}

__device__ __forceinline__ DotAcc dot_add(DotAcc acc, df a, df b)
{
    const df p = two_prod(a.hi, b.hi);
    const df s = two_sum(acc.s, p.hi);
    float e = __fadd_rn(acc.e, __fadd_rn(s.lo, p.lo));
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return {s.hi, e};
}

// acc + b (a df term added without a product)
__device__ __forceinline__ DotAcc dot_add(DotAcc acc, df b)
{
    const df s = two_sum(acc.s, b.hi);
    return {s.hi, __fadd_rn(acc.e, __fadd_rn(s.lo, b.lo))};
}

__device__ __forceinline__ df dot_value(DotAcc acc) { return fast_two_sum(acc.s, acc.e); }

// The sum as an unrenormalised pair (s, e): |e| can reach a few ulp(s).
__device__ __forceinline__ df dot_unnorm(DotAcc acc) { return {acc.s, acc.e}; }

__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }

// a b: the exact product of the high parts plus the two cross terms (the
// lo * lo term is below the result's precision).
__device__ __forceinline__ df operator*(df a, df b)
{
    const df p = two_prod(a.hi, b.hi);
    const float e = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, p.lo));
    return fast_two_sum(p.hi, e);
}

// a b without the final renormalisation: hi is the rounded product of the
// high parts and lo collects its rounding error and the cross terms, so
// |lo| can reach a few ulp(hi); the pair still represents a b to about u^2.
// For products that feed further products or a final split, not comparisons.
__device__ __forceinline__ df mul_unnorm(df a, df b)
{
    const df p = two_prod(a.hi, b.hi);
    return {p.hi, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, p.lo))};
}

__device__ __forceinline__ df operator*(df a, float b)
{
    const df p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// 1/a by one Newton correction of the rounded reciprocal q of the high part:
// r = 1 - a q (its high-part term 1 - a.hi q is exact for q = RN(1/a.hi)),
// 1/a = q (1 + r) + O(r^2).
__device__ __forceinline__ df df_rcp(df a)
{
    const float q = __frcp_rn(a.hi);
    const float r = __fmaf_rn(-a.lo, q, __fmaf_rn(-a.hi, q, 1.0f));
    return fast_two_sum(q, __fmul_rn(q, r));
}

__device__ __forceinline__ bool df_lt(df a, float b) { return a.hi < b || (a.hi == b && a.lo < 0.0f); }
__device__ __forceinline__ bool df_gt(df a, float b) { return a.hi > b || (a.hi == b && a.lo > 0.0f); }

// floor of a df as an integer (|a| < 2^31): floor(hi), one less when hi is an
// integer and the low part is negative.
__device__ __forceinline__ int df_floor(df a)
{
    const float f = floorf(a.hi);
    int i = (int)f;
    if (f == a.hi && a.lo < 0.0f) i -= 1;
    return i;
}

}  // namespace fla
