// Double-double arithmetic (an unevaluated sum hi + lo of two binary64 numbers,
// about 106 significant bits), written from the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA form of TwoProduct.
//
// The set-up of the path runs in this arithmetic next to the scaling centre: the
// algorithmic condensation amplifies rounding errors of the coefficient matrices by
// about four orders of magnitude through its first pivot -xi0 E0 / (2h) (xi0 = 1e-3),
// which in plain binary64 would move receiver traces by ~1e-10 relative.  Results
// are rounded to binary64 (the hi part) before the time loop uses them.
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define DD_HD __host__ __device__ __forceinline__
#else
#define DD_HD inline
#endif

struct dd {
  double hi, lo;
};

DD_HD dd dd_make(double a) { return dd{a, 0.0}; }

// s + e = a + b exactly (Knuth's TwoSum, no magnitude precondition)
DD_HD dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker's FastTwoSum)
DD_HD dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd{s, e};
}

// p + e = a * b exactly (needs a fused multiply-add)
DD_HD dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd{p, e};
}

DD_HD dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  double e = s.lo + t.hi;
  dd u = fast_two_sum(s.hi, e);
  e = u.lo + t.lo;
  return fast_two_sum(u.hi, e);
}

DD_HD dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
DD_HD dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

DD_HD dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  double e = p.lo + (x.hi * y.lo + x.lo * y.hi);
  return fast_two_sum(p.hi, e);
}

DD_HD dd dd_mul_d(dd x, double y) {
  dd p = two_prod(x.hi, y);
  double e = p.lo + x.lo * y;
  return fast_two_sum(p.hi, e);
}

// acc + x * y
DD_HD dd dd_fma(dd acc, dd x, dd y) { return dd_add(acc, dd_mul(x, y)); }

// x / y by long division with two correction steps
DD_HD dd dd_div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = dd_sub(x, dd_mul_d(y, q1));
  double q2 = r.hi / y.hi;
  r = dd_sub(r, dd_mul_d(y, q2));
  double q3 = r.hi / y.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, dd_make(q3));
}

DD_HD double dd_abs_hi(dd x) { return fabs(x.hi); }
DD_HD double dd_to_d(dd x) { return x.hi + x.lo; }
