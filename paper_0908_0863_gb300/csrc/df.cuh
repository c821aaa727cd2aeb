// Double-float arithmetic: a real number held as the unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi) / 2), about 48 significant bits, computed
// on the FP32 units.  The sum takes Knuth's two-sum of the high parts, adds
// the low parts into its error term and renormalises with a second two-sum
// (after cancellation the high sum can be smaller than that term, which a
// fast two-sum would get wrong): its error is about 2^-48 times |a| + |b|,
// what a transform's norm-wise error analysis needs.  The product forms the
// exact product of the high parts with a fused multiply-add, adds the cross
// terms and renormalises with a fast two-sum (the high product dominates).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace dda {

struct DF {
    float hi, lo;
    DF() = default;
    // the double rounded to the nearest float, plus the rounded remainder
    __host__ __device__ __forceinline__ DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
};

// The high product, rounded on its own: the device compiler never contracts
// __fmul_rn into the sum that follows it, which would count the product's
// rounding error twice.
__host__ __device__ __forceinline__ float df_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

__host__ __device__ __forceinline__ DF df_fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return DF(s, b - (s - a));
}
__host__ __device__ __forceinline__ DF df_two_sum(float a, float b) {   // any magnitudes
    const float s = a + b;
    const float v = s - a;
    return DF(s, (a - (s - v)) + (b - v));
}
__host__ __device__ __forceinline__ DF operator+(DF a, DF b) {
    const DF s = df_two_sum(a.hi, b.hi);
    return df_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__host__ __device__ __forceinline__ DF operator*(DF a, DF b) {
    const float p = df_mul(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);   // the exact error of the high product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
// a * b + c (with float and double overloads, so that the name does not
// hide the math library's inside this namespace)
__host__ __device__ __forceinline__ DF fma(DF a, DF b, DF c) { return a * b + c; }
__host__ __device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__host__ __device__ __forceinline__ double to_double(DF a) { return (double)a.hi + (double)a.lo; }

// complex double-float (16 bytes, loaded and stored as one float4)
struct __align__(16) cdf {
    DF x, y;
};

}  // namespace dda
