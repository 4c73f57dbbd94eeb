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
// Exact reciprocals 1/((2n)(2n+1)) (sine steps) and 1/((2n-1)(2n)) (cosine steps),
// n = 1..15, split into double-double (hi, lo): the rational value rounded to
// double, then the remainder rounded to double.  Index 0 is unused.
static __constant__ double2 k_dd_rsin[16] = {
    {0.0, 0.0},
    {0x1.5555555555555p-3, 0x1.5555555555555p-57},
    {0x1.999999999999ap-5, -0x1.999999999999ap-59},
    {0x1.8618618618618p-6, 0x1.8618618618618p-60},
    {0x1.c71c71c71c71cp-7, 0x1.c71c71c71c71cp-61},
    {0x1.29e4129e4129ep-7, 0x1.04a7904a7904ap-61},
    {0x1.a41a41a41a41ap-8, 0x1.0690690690690p-62},
    {0x1.3813813813814p-8, -0x1.fb1fb1fb1fb20p-62},
    {0x1.e1e1e1e1e1e1ep-9, 0x1.e1e1e1e1e1e1ep-65},
    {0x1.7f405fd017f40p-9, 0x1.7f405fd017f40p-63},
    {0x1.3813813813814p-9, -0x1.fb1fb1fb1fb20p-63},
    {0x1.03091b51f5e1ap-9, 0x1.3bb3194be3ab0p-63},
    {0x1.b4e81b4e81b4fp-10, -0x1.f92c5f92c5f93p-64},
    {0x1.756cac201756dp-10, -0x1.4f7fa2a4d4f80p-64},
    {0x1.42d6625d51f87p-10, -0x1.064e2febd299ep-66},
    {0x1.19e0119e0119ep-10, 0x1.19e0119e0119ep-70}};
static __constant__ double2 k_dd_rcos[16] = {
    {0.0, 0.0},
    {0x1.0000000000000p-1, 0x0.0p+0},
    {0x1.5555555555555p-4, 0x1.5555555555555p-58},
    {0x1.1111111111111p-5, 0x1.1111111111111p-61},
    {0x1.2492492492492p-6, 0x1.2492492492492p-60},
    {0x1.6c16c16c16c17p-7, -0x1.f49f49f49f49fp-62},
    {0x1.f07c1f07c1f08p-8, -0x1.f07c1f07c1f08p-63},
    {0x1.6816816816817p-8, -0x1.fa5fa5fa5fa60p-62},
    {0x1.1111111111111p-8, 0x1.1111111111111p-64},
    {0x1.ac5701ac5701bp-9, -0x1.d47f29d47f29dp-64},
    {0x1.58ed2308158edp-9, 0x1.1840ac7691841p-64},
    {0x1.1bb4a4046ed29p-9, 0x1.1bb4a4046ed29p-69},
    {0x1.dae6076b981dbp-10, -0x1.9f89467e251a0p-66},
    {0x1.934c67f9b2ce6p-10, 0x1.934c67f9b2ce6p-70},
    {0x1.5ac056b015ac0p-10, 0x1.5ac056b015ac0p-64},
    {0x1.2d50a012d50a0p-10, 0x1.2d50a012d50a0p-66}};

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
      s = dd_sub(dd_make(1.0), dd_mul(dd_mul(x2, s), dd{k_dd_rsin[n].x, k_dd_rsin[n].y}));
    s = dd_mul(x, s);
  } else {
    for (int n = 15; n >= 1; n--)
      s = dd_sub(dd_make(1.0), dd_mul(dd_mul(x2, s), dd{k_dd_rcos[n].x, k_dd_rcos[n].y}));
  }
  return (q >= 2) ? dd_neg(s) : s;
}
