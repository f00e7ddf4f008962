// Double-float arithmetic on the FP32 pipe: a value is hi + lo, two FP32
// words with |lo| <= ulp(hi) / 2 after conversion (about 48 significant bits).
// Products use Dekker's exact product of the high words, the error term taken
// with one fused multiply-add (TwoProduct of Ogita, Rump and Oishi, 2005), plus
// the two cross terms; sums use Knuth's error-free two-sum.  A multiply-add
// costs 12 FP32 instructions and adds a relative error of at most about 2^-44
// of the product (the lo x lo term and the rounding of the low word), far below
// the FP32-class rounding of the mixed-precision samples it is used on.
//
// Values must lie in FP32's normal range (about 1e-38 .. 3e38); below it the
// low word degrades gracefully to an absolute error of about 1e-45.
#pragma once

#include <cuda_runtime.h>

namespace hm {

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit dfloat(int v) : hi((float)v), lo(0.0f) {}
};

// FP64 -> double-float (exact for the 48 leading bits)
__device__ __forceinline__ dfloat df_from(double x) {
    const float h = __double2float_rn(x);
    return dfloat(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_to(dfloat a) { return (double)a.hi + (double)a.lo; }

// c + a b
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);  // p + e == a.hi b.hi exactly
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = c.hi + p;        // two-sum: s + t == c.hi + p exactly
    const float bb = s - c.hi;
    const float t = (c.hi - (s - bb)) + (p - bb);
    return dfloat(s, c.lo + (t + e));
}

// a + b
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float t = (a.hi - (s - bb)) + (b.hi - bb);
    return dfloat(s, a.lo + (b.lo + t));
}

// c + a b and a + b for the arithmetic types of the templated kernels
__device__ __forceinline__ float mac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mac(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ dfloat mac(dfloat a, dfloat b, dfloat c) { return df_fma(a, b, c); }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ dfloat add(dfloat a, dfloat b) { return df_add(a, b); }

// conversions of the templated kernels: FP64 operand -> arithmetic type, and a
// sum in the arithmetic type -> the accumulation type
template <class T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ float from_f64<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ dfloat from_f64<dfloat>(double x) { return df_from(x); }
__device__ __forceinline__ float widen(float a, float) { return a; }
__device__ __forceinline__ double widen(float a, double) { return (double)a; }
__device__ __forceinline__ double widen(double a, double) { return a; }
__device__ __forceinline__ double widen(dfloat a, double) { return df_to(a); }

}  // namespace hm
