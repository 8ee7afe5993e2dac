// Double-float ("double-word") arithmetic: a value is the unevaluated sum of
// two float32 numbers, hi + lo with |lo| <= ulp(hi) / 2, i.e. 48 significant
// bits, computed with float32 operations only.  GB300 runs float64 at 1/64 of
// its float32 rate, so float64-class element arithmetic (the residual's
// internal force) runs faster this way.
//
// Building blocks (error-free transformations): Knuth's two-sum, the fast
// two-sum for |a| >= |b|, and the exact product through FMA.  Addition and
// multiplication follow the accurate double-word algorithms of Joldes, Muller
// and Popescu (ACM TOMS 44(2), 2017: "DWPlusDW" with relative error below
// 3u^2, "DWTimesDW" with the FMA, below 5u^2, u = 2^-24).  Every float32
// operation uses the _rn intrinsics, which the compiler never contracts into
// FMAs (a contraction would break the error-free transformations).
#pragma once

#include <cuda_runtime.h>

namespace tl {

struct dfl {
  float hi, lo;
  __host__ __device__ dfl() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ dfl(int x) : hi((float)x), lo(0.0f) {}
  __host__ __device__ dfl(float x) : hi(x), lo(0.0f) {}
  __host__ __device__ dfl(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ dfl(float h, float l, int) : hi(h), lo(l) {}   // raw pair
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e, 0);
}

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {   // |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dfl(s, e, 0);
}

__device__ __forceinline__ dfl operator+(dfl x, dfl y) {
  const dfl s = df_two_sum(x.hi, y.hi);
  const dfl t = df_two_sum(x.lo, y.lo);
  dfl v = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo, 0); }
__device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }

__device__ __forceinline__ dfl operator*(dfl x, dfl y) {
  const float ph = __fmul_rn(x.hi, y.hi);
  float pl = __fmaf_rn(x.hi, y.hi, -ph);
  const float tl = __fmaf_rn(x.lo, y.lo, __fmul_rn(x.hi, y.lo));
  pl = __fadd_rn(pl, __fmaf_rn(x.lo, y.hi, tl));
  return df_fast_two_sum(ph, pl);
}

// Division by one Newton correction of the float32 quotient (used only for a
// few reciprocals per quadrature point of the Mooney-Rivlin law).
__device__ __forceinline__ dfl operator/(dfl x, dfl y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const dfl r = x - y * dfl(q1);
  const float q2 = __fdiv_rn(r.hi, y.hi);
  return df_fast_two_sum(q1, q2);
}

__device__ __forceinline__ dfl& operator+=(dfl& x, dfl y) { return x = x + y; }
__device__ __forceinline__ dfl& operator-=(dfl& x, dfl y) { return x = x - y; }
__device__ __forceinline__ dfl& operator*=(dfl& x, dfl y) { return x = x * y; }

__device__ __forceinline__ bool operator>(dfl x, dfl y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
__device__ __forceinline__ bool operator<(dfl x, dfl y) { return y > x; }

}  // namespace tl
