// dd.cuh -- double-double arithmetic for the one-time geometry construction.
//
// A value is hi + lo with |lo| <= ulp(hi)/2 (about 32 significant digits).
// Error-free transformations: Knuth's TwoSum, Dekker's Fast-TwoSum, and the
// FMA form of TwoProd; products and sums follow the standard double-double
// algorithms built on them.  Only the geometry uses this: the curl-form metric
// differentiates node positions twice, so it is evaluated well beyond FP64
// and rounded once.
#pragma once
#include <cuda_runtime.h>

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_make(double a) { return dd{a, 0.0}; }

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  const double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}

__device__ __forceinline__ dd dd_fast_two_sum(double a, double b) {  // |a| >= |b|
  const double s = a + b;
  const double e = b - (s - a);
  return dd{s, e};
}

__device__ __forceinline__ dd dd_two_prod(double a, double b) {
  const double p = a * b;
  return dd{p, fma(a, b, -p)};
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = dd_two_sum(x.hi, y.hi);
  const dd t = dd_two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = dd_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const double p = x.hi * y.hi;
  double e = fma(x.hi, y.hi, -p);
  e = fma(x.hi, y.lo, e);
  e = fma(x.lo, y.hi, e);
  return dd_fast_two_sum(p, e);
}

__device__ __forceinline__ dd dd_mul_d(dd x, double b) { return dd_mul(x, dd_make(b)); }

__device__ __forceinline__ dd dd_div_d(dd a, double b) {
  const double q1 = a.hi / b;
  const dd r = dd_sub(a, dd_two_prod(q1, b));
  const double q2 = r.hi / b;
  return dd_fast_two_sum(q1, q2);
}

// sin(pi t) for t in [-4, 4]: reduce by the nearest multiple of 1/2, then the
// Taylor series of sin or cos of x = pi u, |x| <= pi/4, in nested (Horner)
// form; 15 terms leave a truncation error below 1e-33.
__device__ __forceinline__ dd dd_sinpi(dd t) {
  const dd PI = dd{3.141592653589793116e+00, 1.224646799147353207e-16};
  const double k = rint(2.0 * t.hi);
  const dd u = dd_sub(t, dd_make(0.5 * k));  // exact multiple of 1/2
  const dd x = dd_mul(PI, u);
  const dd x2 = dd_mul(x, x);
  int q = ((int)k) & 3;
  dd s = dd_make(1.0);
  if (q == 0 || q == 2) {
    for (int n = 15; n >= 1; n--)
      s = dd_sub(dd_make(1.0), dd_div_d(dd_mul(x2, s), (double)((2 * n) * (2 * n + 1))));
    s = dd_mul(x, s);
  } else {
    for (int n = 15; n >= 1; n--)
      s = dd_sub(dd_make(1.0), dd_div_d(dd_mul(x2, s), (double)((2 * n - 1) * (2 * n))));
  }
  return (q >= 2) ? dd_neg(s) : s;
}
