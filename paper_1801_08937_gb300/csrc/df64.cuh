// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// float32 numbers, giving about 44 bits of precision from float32 units.
// Addition uses the error-free two-sum of Knuth and Moller on the hi parts;
// multiplication uses the error-free product through a fused multiply-add
// (Dekker's product with FMA).  Neither renormalises: the lo part carries
// only rounding errors of the order of eps_32 times the magnitudes of the
// operands that produced it, and is itself rounded in float32, so every
// result is exact to about eps_32^2 of those magnitudes, which is the
// absolute accuracy a transform or band sum needs (after a cancellation lo
// may exceed ulp(hi); the represented value hi + lo stays as accurate).
// GB300 issues float32 at 64 times its float64 rate, so float64-accurate
// products run several times faster this way.
#pragma once
#include <cuda_runtime.h>

namespace mm {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df(s, e);
}
__device__ __forceinline__ df operator+(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return s;
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// The product is returned as (p, e) without renormalising; the dropped term
// a.lo b.lo is of the order of eps_32^2 |a| |b|.
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

__device__ __forceinline__ df shfl_down(df v, int d) {
    return df(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}

}  // namespace mm
