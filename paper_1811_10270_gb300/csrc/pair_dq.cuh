// Kernel terms of the FP64-class all-pairs sums with exactly representable coordinate differences.
//
// Positions relative to the source drop's centre are split as v = vq + vl, vq a multiple of a
// power-of-two quantum 2^-Q and vl = v - vq (|vl| <= 2^-Q-1) rounded to FP32. The host picks Q so that
// every |vq| and every difference |x0q - xq| stays below 2^(24-Q): the difference of the quantised
// parts is then an integer multiple of 2^-Q below 2^24 quanta, exact in FP32, and
//   d = x0 - x = dh + dl,   dh = x0q - xq exactly,   dl = x0l - xl (error ~2^-24 |dl| <= 2^-Q-24).
// What the general double-float difference spends on two-sums (about a third of a Laplace term) is
// gone. The rest is error-free arithmetic (Knuth's two-sum, the FMA two-product):
//   r^2 = R + delta with R = fl(dh.dh) and delta collecting the product and addition errors and
//         (2 dh + dl).dl, to ~2^-46 r^2;
//   1/r = y + c: y = rsqrt(R) (FP32 seed, ~2^-22), rho = 1 - (R + delta) y^2 formed exactly up to
//         ~2^-46 (1 - R y2 is exact by Sterbenz's lemma since R y2 ~ 1), c = y rho (1/2 + 3 rho/8);
// and every product with a strength or a normal keeps its leading two-product and first-order cross
// terms. The FP32 remainders hold the positions to ~2^-(Q+23) absolute (the general double-float form:
// ~2^-47 of the offset), so a term is good to ~2^-(Q+23)/r relative: ~2^-42 for pairs of drops at least
// 2^(19-Q) apart, the only ones the all-pairs kernel gives this form (pairs.cu).
//
// Staged source records (float4): Laplace a = (xq, yq, zq, xl), b = (yl, zl, s, s_lo); Stokes as the
// double-float form's records with the quantised positions (pair_df.cuh). Th, Tl are the target's
// quantised offset from the source drop's centre and its remainder; N0 its normal (double-float).
#pragma once

#include "dfloat.cuh"

namespace shbim {

struct DqGeo {
  float dh[3], dl[3];  // d = dh + dl
  float y, c;          // 1/r = y + c
  float y2, y2e;       // y^2 = y2 + y2e exactly
};

// FP32 reciprocal square root seed (~2^-22 relative): the approximate instruction alone; its input, a
// squared distance between different drops' nodes, is never subnormal
__device__ __forceinline__ float dq_rsqrt_seed(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void dq_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void dq_geo(const float Th[3], const float Tl[3], float xq, float yq, float zq,
                                       float xl, float yl, float zl, DqGeo& g) {
  g.dh[0] = __fsub_rn(Th[0], xq);
  g.dh[1] = __fsub_rn(Th[1], yq);
  g.dh[2] = __fsub_rn(Th[2], zq);
  g.dl[0] = __fsub_rn(Tl[0], xl);
  g.dl[1] = __fsub_rn(Tl[1], yl);
  g.dl[2] = __fsub_rn(Tl[2], zl);
  float p[3], e[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p[k] = __fmul_rn(g.dh[k], g.dh[k]);
    e[k] = __fmaf_rn(g.dh[k], g.dh[k], -p[k]);
  }
  float s1, e1, R, e2;
  dq_two_sum(p[0], p[1], s1, e1);
  dq_two_sum(s1, p[2], R, e2);
  // (dh + dl)^2 - dh^2 = (2 dh + dl) dl
  float t = __fmul_rn(__fmaf_rn(2.0f, g.dh[0], g.dl[0]), g.dl[0]);
  t = __fmaf_rn(__fmaf_rn(2.0f, g.dh[1], g.dl[1]), g.dl[1], t);
  t = __fmaf_rn(__fmaf_rn(2.0f, g.dh[2], g.dl[2]), g.dl[2], t);
  const float delta = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e[0], e[1])), __fadd_rn(e[2], t));
  const float y = dq_rsqrt_seed(R);
  const float y2 = __fmul_rn(y, y), y2e = __fmaf_rn(y, y, -y2);
  const float P = __fmul_rn(R, y2), Pe = __fmaf_rn(R, y2, -P);
  float rho = __fsub_rn(__fsub_rn(1.0f, P), Pe);
  rho = __fmaf_rn(-R, y2e, rho);
  rho = __fmaf_rn(-delta, y2, rho);
  g.y = y;
  g.c = __fmul_rn(y, __fmul_rn(rho, __fmaf_rn(0.375f, rho, 0.5f)));
  g.y2 = y2;
  g.y2e = y2e;
}

// (vh + vl) . d with the leading products exact: returns an unevaluated pair h + l
__device__ __forceinline__ dfl::df dq_dot(const DqGeo& g, float vh0, float vl0, float vh1, float vl1, float vh2,
                                          float vl2) {
  const float q0 = __fmul_rn(g.dh[0], vh0), q1 = __fmul_rn(g.dh[1], vh1), q2 = __fmul_rn(g.dh[2], vh2);
  float l = __fmaf_rn(g.dh[0], vh0, -q0);
  l = __fadd_rn(l, __fmaf_rn(g.dh[1], vh1, -q1));
  l = __fadd_rn(l, __fmaf_rn(g.dh[2], vh2, -q2));
  float s1, f1, h, f2;
  dq_two_sum(q0, q1, s1, f1);
  dq_two_sum(s1, q2, h, f2);
  l = __fadd_rn(l, __fadd_rn(f1, f2));
  l = __fmaf_rn(g.dl[0], vh0, __fmaf_rn(g.dh[0], vl0, l));
  l = __fmaf_rn(g.dl[1], vh1, __fmaf_rn(g.dh[1], vl1, l));
  l = __fmaf_rn(g.dl[2], vh2, __fmaf_rn(g.dh[2], vl2, l));
  return {h, l};
}

// a b for unevaluated pairs: leading product exact, first-order cross terms
__device__ __forceinline__ dfl::df dq_mul(dfl::df a, dfl::df b) {
  const float h = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -h);
  return {h, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e))};
}

// 1/r^3 = (y + c)^3 = y^3 + 3 y^2 c + ..., y^3 from the exact y^2
__device__ __forceinline__ dfl::df dq_ri3(const DqGeo& g) {
  const float h = __fmul_rn(g.y2, g.y);
  float l = __fmaf_rn(g.y2, g.y, -h);
  l = __fmaf_rn(g.y2e, g.y, l);
  l = __fmaf_rn(3.0f * g.y2, g.c, l);
  return {h, l};
}

// 1/r^2 = y^2 + 2 y c + ...
__device__ __forceinline__ dfl::df dq_ri2(const DqGeo& g) {
  return {g.y2, __fmaf_rn(2.0f * g.y, g.c, g.y2e)};
}

// d_k t for one component
__device__ __forceinline__ dfl::df dq_comp(const DqGeo& g, int k, dfl::df t) {
  const float h = __fmul_rn(g.dh[k], t.hi);
  const float e = __fmaf_rn(g.dh[k], t.hi, -h);
  return {h, __fmaf_rn(g.dh[k], t.lo, __fmaf_rn(g.dl[k], t.hi, e))};
}

template <int KIND>
__device__ __forceinline__ void dq_term(const float Th[3], const float Tl[3], const dfl::df N0[3], float4 a,
                                        float4 b, float4 c, float4 d, float4 e, float4 gg, dfl::acc* A) {
  using dfl::df;
  DqGeo g;
  dq_geo(Th, Tl, a.x, a.y, a.z, a.w, b.x, b.y, g);
  const df ri{g.y, g.c};
  if (KIND == 1) {
    A[0].add(dq_mul(df{b.z, b.w}, ri));
  } else if (KIND == 0) {
    const df dn = dq_dot(g, N0[0].hi, N0[0].lo, N0[1].hi, N0[1].lo, N0[2].hi, N0[2].lo);
    A[0].add(dq_mul(dq_mul(df{b.z, b.w}, dq_ri3(g)), dn));
  } else if (KIND == 4) {
    // stresslet on u alone: d (d.u)(d.n) / r^5
    const df hu = dq_dot(g, d.x, d.y, d.z, d.w, e.x, e.y);
    const df hn = dq_dot(g, e.z, e.w, gg.x, gg.y, gg.z, gg.w);
    const df tt = dq_mul(dq_mul(hu, hn), dq_mul(dq_ri3(g), dq_ri2(g)));
    A[0].add(dq_comp(g, 0, tt));
    A[1].add(dq_comp(g, 1, tt));
    A[2].add(dq_comp(g, 2, tt));
  } else {
    // KIND 2: Stokeslet on f and stresslet on u; KIND 3: Stokeslet alone
    const df fx{b.z, b.w}, fy{c.x, c.y}, fz{c.z, c.w};
    const df hf = dq_dot(g, fx.hi, fx.lo, fy.hi, fy.lo, fz.hi, fz.lo);
    const df ri3 = dq_ri3(g);
    df tt;
    if (KIND == 3) {
      tt = dq_mul(ri3, hf);
    } else {
      const df hu = dq_dot(g, d.x, d.y, d.z, d.w, e.x, e.y);
      const df hn = dq_dot(g, e.z, e.w, gg.x, gg.y, gg.z, gg.w);
      // hf + (d.u)(d.n)/r^2, then times 1/r^3
      const df s = dq_mul(dq_mul(hu, hn), dq_ri2(g));
      float sh, se;
      dq_two_sum(hf.hi, s.hi, sh, se);
      tt = dq_mul(ri3, df{sh, __fadd_rn(se, __fadd_rn(hf.lo, s.lo))});
    }
    A[0].add(dq_mul(fx, ri));
    A[0].add(dq_comp(g, 0, tt));
    A[1].add(dq_mul(fy, ri));
    A[1].add(dq_comp(g, 1, tt));
    A[2].add(dq_mul(fz, ri));
    A[2].add(dq_comp(g, 2, tt));
  }
}

}  // namespace shbim
