// Conversions between float64 and float32 as integer bit operations.
//
// On the GB300 the hardware conversions between float64 and float32 issue on
// the float64 pipe, which runs about two operations per clock per SM; kernels
// that convert every element they stream would be bound by it.  These
// helpers keep the common values on the integer pipes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

// float64 -> float32 by truncation of the significand (error below one
// float32 ulp) and float32 -> float64 (exact).  Zeros (the fourth entry of
// every pixel) take the integer path too; values outside float32's normal
// range, denormals, infinities and NaN fall back to the hardware conversion,
// which is out of line so that the rare path stays a branch instead of being
// computed for every element and selected.
static __device__ __noinline__ float d2f_hw(double x) { return (float)x; }
static __device__ __noinline__ double f2d_hw(float f) { return (double)f; }
__device__ __forceinline__ float d2f_trunc(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    if (((hi << 1) | lo) == 0u) return __uint_as_float(hi);
    const int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
    if (e <= 0 || e >= 255) return d2f_hw(x);
    return __uint_as_float((hi & 0x80000000u) | ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t u = __float_as_uint(f);
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)u, 0);
    const uint32_t e = (u >> 23) & 0xFF;
    if (e == 0u || e == 0xFFu) return f2d_hw(f);
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)),
                            (int)(u << 29));
}

}  // namespace mm
