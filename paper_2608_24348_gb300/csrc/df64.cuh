// df64.cuh -- an FP64-accurate scalar held as a pair of FP32 numbers, for kernels
// written once over a scalar type T (the dealiased convection).
//
// GB300 executes FP64 at 1/58 of its FP32 rate.  A df64 value is hi + lo with
// |lo| <= ulp(hi)/2 after every operation; products are exact in their leading
// part (TwoProd via FMA, Dekker 1971), sums are error-free in their leading part
// (TwoSum, Knuth 1969), and each result is renormalised with FastTwoSum, which
// is exact when the leading term dominates and otherwise keeps the error at the
// operands' 2^-48 scale.  Relative accuracy about 2^-48 per operation, within
// the FP32 exponent range (callers keep values there).  Every FP32 step uses the
// _rn intrinsics so the compiler never contracts or reassociates them.
#pragma once

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __device__ df64(int v) : hi((float)v), lo(0.f) {}  // small integer constants
    __device__ explicit df64(double v)
    {
        hi = __double2float_rn(v);
        lo = __double2float_rn(v - (double)hi);
    }
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df64_fast2(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return df64(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    return df64_fast2(s, __fadd_rn(t, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df64_fast2(p, e);
}

// a * b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(c.hi, p);
    const float bv = __fsub_rn(s, c.hi);
    const float t = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    return df64_fast2(s, __fadd_rn(t, __fadd_rn(c.lo, e)));
}

__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
