// The digit arithmetic of the tensor-core kernels with FP64-class accuracy (tc.cuh), kept apart
// from the PTX so that the CPU tests can compile it with a host compiler (as the double-float
// header): digit splitting of FP64 table values on the host, of double-float values in the kernels,
// and the recombination of the six exact FP32 diagonal sums. Host builds must not contract or
// reassociate floating-point operations (-ffp-contract=off).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "dfloat.cuh"

#ifdef __CUDACC__
#define TC_FN __host__ __device__ __forceinline__
#else
#define TC_FN inline
#endif

namespace shbim {
namespace tc {

constexpr int kDig = 6;          // digits per value

// digits of x 2^(42 - e), |x| < 2^e: d_0..d_4 balanced base 2^7, d_5 the rest (host)
inline void digits_host(double x, int e, int d[kDig]) {
  long long X = std::llrint(std::ldexp(x, 42 - e));
  for (int j = 0; j < kDig - 1; ++j) {
    const long long dj = ((X + 64) & 127) - 64;
    d[j] = (int)dj;
    X = (X - dj) / 128;
  }
  d[kDig - 1] = (int)X;
}

// bfloat16 bits of a small integer (|v| <= 256 is exact: the low 16 bits of the float are zero)
inline uint16_t bf16_int(int v) {
  const float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

// Six balanced base-2^7 digits of y = yh + yl (|yh| < 128, |yl| <= ulp(yh) / 2), top first:
// d5 = rint(y), then the digits of the remainder times 128, and so on. The top three come from yh
// alone (every remainder exact); yl joins through one two-sum at the scale of d2; the last two come
// from an FP32 remainder whose rounding (< 2^-25 of d2's unit) stays far below d0's half unit.
// Bounds: |d5| <= 128, |d4|, |d3| <= 64, |d2| <= 72, |d1|, |d0| <= 65.
TC_FN void digits6(float yh, float yl, float (&d)[kDig]) {
  float t = yh;
  d[5] = rintf(t);
  t = (t - d[5]) * 128.f;
  d[4] = rintf(t);
  t = (t - d[4]) * 128.f;
  d[3] = rintf(t);
  t = (t - d[3]) * 128.f;
  const dfl::df u = dfl::two_sum(t, yl * 2097152.f);   // yl at the scale of d2 (2^21)
  d[2] = rintf(u.hi);
  float r = ((u.hi - d[2]) + u.lo) * 128.f;
  d[1] = rintf(r);
  r = (r - d[1]) * 128.f;
  d[0] = rintf(r);
}

// Largest |digit| by position (row operand after digits6; table operand after digits_host) and the
// worst case of diagonal sum s (products with j_a + j_b = s + 5) over K products: every tensor-core
// kernel asserts at compile time that this stays below 2^24 at its longest K, so that the FP32
// accumulation in tensor memory is exact.
constexpr int kRowDigitMax[kDig] = {65, 65, 72, 64, 64, 128};
constexpr int kTabDigitMax[kDig] = {64, 64, 64, 64, 64, 128};
constexpr long long diag_sum_bound(int K, int s) {
  long long w = 0;
  for (int ja = 0; ja < kDig; ++ja) {
    const int jb = s + kDig - 1 - ja;
    if (jb >= 0 && jb < kDig) w += (long long)kRowDigitMax[ja] * kTabDigitMax[jb];
  }
  return w * K;
}
constexpr bool diag_sums_exact(int K) {
  for (int s = 0; s < kDig; ++s)
    if (diag_sum_bound(K, s) >= (1LL << 24)) return false;
  return true;
}

// sum_s acc_s 2^(7 (s - 5)) as a double-float from the six exact FP32 diagonal sums
// (|acc_s| < 2^24): the three top terms are exact in FP32 and joined by two-sums; the three lowest
// (weights 2^-21 and below) are summed in plain FP32, rounding below 2^-21 units of the top term.
TC_FN dfl::df combine6(float a5, float a4, float a3, float a2, float a1, float a0) {
  const float low = fmaf(a0, 0x1p-35f, fmaf(a1, 0x1p-28f, a2 * 0x1p-21f));
  const dfl::df s1 = dfl::two_sum(a5, a4 * 0x1p-7f);
  const dfl::df s2 = dfl::two_sum(s1.hi, a3 * 0x1p-14f);
  return dfl::quick_two_sum(s2.hi, (s1.lo + s2.lo) + low);
}

}  // namespace tc
}  // namespace shbim
