// Float-float ("double-single") arithmetic for the demag convolution (Sec. III,
// Eq. 14) when it must accumulate at FP64-class precision on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| at most
// half an ulp of hi: about 48 significant bits.  The error-free steps are
// Knuth's TwoSum, Dekker's FastTwoSum and the FMA form of Dekker's TwoProduct
// (Dekker, Numer. Math. 18, 1971); addition is the short form of the
// double-double add of Hida, Li and Bailey (ARITH-15, 2001), whose error is at
// most a few units of 2^-48 (|a| + |b|), the norm-wise bound an FFT's error
// analysis rests on.  Every step goes through the round-to-nearest intrinsics
// so that the compiler cannot contract a product into the following sum, which
// would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"

namespace mmc {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ff(float v) : hi(v), lo(0.f) {}
  __host__ __device__ constexpr ff(int v) : hi((float)v), lo((float)((long long)v - (long long)(float)v)) {}
  // the double split into its leading 24 bits and the rounded rest
  __host__ __device__ constexpr ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// complex float-float value; 16 bytes like double2, so the FP64 plans' buffer
// sizes and shared-memory layouts carry over unchanged
struct __align__(16) ff2 {
  ff x, y;
};
template <> struct Cx<ff> { using T = ff2; };

// a + b exactly as s + e (Knuth)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}

// a + b exactly as s + e when |a| >= |b| (Dekker)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }

__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

// product: hi * hi exactly as p + e by one FMA, plus the cross terms
// (lo * lo is below the format's precision)
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

// quotient by one correction step (long division on the leading parts)
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - ff(q1) * b;
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return ff_fast_two_sum(q1, q2);
}

}  // namespace mmc
