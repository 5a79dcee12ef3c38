// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) (about 48 significant bits, relative error ~2^-46 per operation).
//
// Built from the error-free transformations of Knuth (two-sum: the exact rounding error of an
// addition) and Dekker (two-product, here the FMA form p = a*b, e = fma(a, b, -p)), following
// Dekker, "A floating-point technique for extending the available precision" (1971), and the
// double-double algorithms of Hida, Li & Bailey (QD library, 2001) transposed to FP32 pairs.
//
// Why: on this GPU the FP32 pipe issues 64 operations for every FP64 one, so sums that need
// FP64-class accuracy run several times faster as double-float FP32 code than as FP64 code.
//
// The additions and multiplications inside the error-free transformations must not be
// contracted into FMAs or reassociated: device code uses the _rn intrinsics (never contracted);
// host code (used only by the CPU tests) must be compiled with -ffp-contract=off.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define DF_FN __host__ __device__ __forceinline__
#else
#define DF_FN inline
#endif

namespace dfl {

struct df {
  float hi, lo;
};

DF_FN float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DF_FN float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DF_FN float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DF_FN float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly (Knuth)
DF_FN df two_sum(float a, float b) {
  const float s = add_rn(a, b);
  const float bb = sub_rn(s, a);
  const float e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly, requires |a| >= |b| or a == 0 (Dekker)
DF_FN df quick_two_sum(float a, float b) {
  const float s = add_rn(a, b);
  return {s, sub_rn(b, sub_rn(s, a))};
}
// p + e = a * b exactly (FMA form)
DF_FN df two_prod(float a, float b) {
  const float p = mul_rn(a, b);
  return {p, fma_rn(a, b, -p)};
}

DF_FN df from_double(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}
DF_FN double to_double(df a) { return (double)a.hi + (double)a.lo; }
DF_FN df from_float(float f) { return {f, 0.0f}; }

DF_FN df neg(df a) { return {-a.hi, -a.lo}; }

// a + b; error bounded by ~2^-45 (|a| + |b|) ("sloppy" addition of the QD library)
DF_FN df add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = add_rn(s.lo, add_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}
DF_FN df sub(df a, df b) { return add(a, neg(b)); }
DF_FN df add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = add_rn(s.lo, a.lo);
  return quick_two_sum(s.hi, s.lo);
}

DF_FN df mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fma_rn(a.hi, b.lo, fma_rn(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}
DF_FN df mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fma_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
DF_FN df sqr(df a) {
  df p = two_prod(a.hi, a.hi);
  p.lo = fma_rn(a.hi + a.hi, a.lo, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// Accumulator for long sums: hi carries the running sum, lo collects every rounding error (two-
// sum of each addition) and the low-order parts of the terms; normalised only when read.
struct acc {
  float hi = 0.0f, lo = 0.0f;
  DF_FN void add(df t) {
    const df s = two_sum(hi, t.hi);
    hi = s.hi;
    lo = add_rn(lo, add_rn(s.lo, t.lo));
  }
  DF_FN void add_f(float t) {
    const df s = two_sum(hi, t);
    hi = s.hi;
    lo = add_rn(lo, s.lo);
  }
  // += a * b exactly up to the low-order products
  DF_FN void add_prod(df a, df b) {
    const df p = two_prod(a.hi, b.hi);
    const float e = fma_rn(a.hi, b.lo, fma_rn(a.lo, b.hi, p.lo));
    const df s = two_sum(hi, p.hi);
    hi = s.hi;
    lo = add_rn(lo, add_rn(s.lo, e));
  }
  // += a * b with b an exact FP32 value
  DF_FN void add_prod_f(df a, float b) {
    const df p = two_prod(a.hi, b);
    const float e = fma_rn(a.lo, b, p.lo);
    const df s = two_sum(hi, p.hi);
    hi = s.hi;
    lo = add_rn(lo, add_rn(s.lo, e));
  }
  DF_FN df value() const { return quick_two_sum(hi, lo); }
};

// a - b with both operands double-float
DF_FN df diff(df a, df b) {
  const df s = two_sum(a.hi, -b.hi);
  return quick_two_sum(s.hi, add_rn(s.lo, sub_rn(a.lo, b.lo)));
}

// a0 b0 + a1 b1 + a2 b2: exact leading products, low-order cross terms in FP32
DF_FN df dot3(df a0, df a1, df a2, df b0, df b1, df b2) {
  const df p0 = two_prod(a0.hi, b0.hi), p1 = two_prod(a1.hi, b1.hi), p2 = two_prod(a2.hi, b2.hi);
  float e = fma_rn(a0.hi, b0.lo, fma_rn(a0.lo, b0.hi, p0.lo));
  e = fma_rn(a1.hi, b1.lo, fma_rn(a1.lo, b1.hi, add_rn(e, p1.lo)));
  e = fma_rn(a2.hi, b2.lo, fma_rn(a2.lo, b2.hi, add_rn(e, p2.lo)));
  const df s = two_sum(p0.hi, p1.hi);
  const df t = two_sum(s.hi, p2.hi);
  return quick_two_sum(t.hi, add_rn(add_rn(s.lo, t.lo), e));
}

// 1 / sqrt(a) for a > 0: FP32 seed y, then one Newton step y + y (1 - a y^2) / 2 with the
// residual 1 - a y^2 formed in double-float (quadratic convergence: ~2^-46 from a ~2^-22 seed).
DF_FN df rsqrt(df a) {
#ifdef __CUDA_ARCH__
  const float y = rsqrtf(a.hi);
#else
  const float y = 1.0f / std::sqrt(a.hi);
#endif
  const df ay2 = mul_f(mul_f(a, y), y);          // a y^2 ~ 1
  const df r = add_f(neg(ay2), 1.0f);            // 1 - a y^2, small
  const float corr = mul_rn(mul_rn(0.5f, y), r.hi);
  return quick_two_sum(y, corr);
}

// sqrt(a) for a >= 0 (Karp & Markstein): x = a y with y ~ 1/sqrt(a), then x + y (a - x^2) / 2.
DF_FN df sqrt(df a) {
  if (a.hi <= 0.0f) return {0.0f, 0.0f};
#ifdef __CUDA_ARCH__
  const float y = rsqrtf(a.hi);
#else
  const float y = 1.0f / std::sqrt(a.hi);
#endif
  const float x = mul_rn(a.hi, y);
  const df r = sub(a, two_prod(x, x));           // a - x^2, exact product
  return quick_two_sum(x, mul_rn(mul_rn(0.5f, y), r.hi));
}

// a / b: q1 = a.hi / b.hi, then one correction from the remainder a - q1 b formed in double-float.
DF_FN df div(df a, df b) {
  const float q1 = a.hi / b.hi;
  const df r = sub(a, mul_f(b, q1));
  const float q2 = r.hi / b.hi;
  return quick_two_sum(q1, q2);
}

}  // namespace dfl
