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
//         rho is the seed's error plus delta/R, which the remainders make up to ~2^-19 (far pairs);
// and every product with a strength or a normal keeps its leading two-product and first-order cross
// terms. The FP32 remainders hold the positions to ~2^-(Q+23) absolute (the general double-float form:
// ~2^-47 of the offset), so a term is good to ~2^-(Q+23)/r relative: ~2^-42 for pairs of drops at least
// 2^(19-Q) apart, the only ones the all-pairs kernel gives this form (pairs.cu).
//
// The arithmetic below is host-compilable (the error-free operations of dfloat.cuh; the host build,
// used only by the CPU tests, must not contract them into FMAs); the kernel term that reads staged
// records is device code.
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
DF_FN float dq_rsqrt_seed(float x) {
#ifdef __CUDA_ARCH__
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / std::sqrt(x);
#endif
}

DF_FN void dq_two_sum(float a, float b, float& s, float& e) {
  s = dfl::add_rn(a, b);
  const float bb = dfl::sub_rn(s, a);
  e = dfl::add_rn(dfl::sub_rn(a, dfl::sub_rn(s, bb)), dfl::sub_rn(b, bb));
}

DF_FN void dq_geo(const float Th[3], const float Tl[3], float xq, float yq, float zq,
                                       float xl, float yl, float zl, DqGeo& g) {
  g.dh[0] = dfl::sub_rn(Th[0], xq);
  g.dh[1] = dfl::sub_rn(Th[1], yq);
  g.dh[2] = dfl::sub_rn(Th[2], zq);
  g.dl[0] = dfl::sub_rn(Tl[0], xl);
  g.dl[1] = dfl::sub_rn(Tl[1], yl);
  g.dl[2] = dfl::sub_rn(Tl[2], zl);
  float p[3], e[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p[k] = dfl::mul_rn(g.dh[k], g.dh[k]);
    e[k] = dfl::fma_rn(g.dh[k], g.dh[k], -p[k]);
  }
  float s1, e1, R, e2;
  dq_two_sum(p[0], p[1], s1, e1);
  dq_two_sum(s1, p[2], R, e2);
  // (dh + dl)^2 - dh^2 = (2 dh + dl) dl
  float t = dfl::mul_rn(dfl::fma_rn(2.0f, g.dh[0], g.dl[0]), g.dl[0]);
  t = dfl::fma_rn(dfl::fma_rn(2.0f, g.dh[1], g.dl[1]), g.dl[1], t);
  t = dfl::fma_rn(dfl::fma_rn(2.0f, g.dh[2], g.dl[2]), g.dl[2], t);
  const float delta = dfl::add_rn(dfl::add_rn(dfl::add_rn(e1, e2), dfl::add_rn(e[0], e[1])), dfl::add_rn(e[2], t));
  const float y = dq_rsqrt_seed(R);
  const float y2 = dfl::mul_rn(y, y), y2e = dfl::fma_rn(y, y, -y2);
  const float P = dfl::mul_rn(R, y2), Pe = dfl::fma_rn(R, y2, -P);
  float rho = dfl::sub_rn(dfl::sub_rn(1.0f, P), Pe);
  rho = dfl::fma_rn(-R, y2e, rho);
  rho = dfl::fma_rn(-delta, y2, rho);
  g.y = y;
  g.c = dfl::mul_rn(y, dfl::mul_rn(rho, dfl::fma_rn(0.375f, rho, 0.5f)));
  g.y2 = y2;
  g.y2e = y2e;
}

// (vh + vl) . d with the leading products exact: returns an unevaluated pair h + l
DF_FN dfl::df dq_dot(const DqGeo& g, float vh0, float vl0, float vh1, float vl1, float vh2,
                                          float vl2) {
  const float q0 = dfl::mul_rn(g.dh[0], vh0), q1 = dfl::mul_rn(g.dh[1], vh1), q2 = dfl::mul_rn(g.dh[2], vh2);
  float l = dfl::fma_rn(g.dh[0], vh0, -q0);
  l = dfl::add_rn(l, dfl::fma_rn(g.dh[1], vh1, -q1));
  l = dfl::add_rn(l, dfl::fma_rn(g.dh[2], vh2, -q2));
  float s1, f1, h, f2;
  dq_two_sum(q0, q1, s1, f1);
  dq_two_sum(s1, q2, h, f2);
  l = dfl::add_rn(l, dfl::add_rn(f1, f2));
  l = dfl::fma_rn(g.dl[0], vh0, dfl::fma_rn(g.dh[0], vl0, l));
  l = dfl::fma_rn(g.dl[1], vh1, dfl::fma_rn(g.dh[1], vl1, l));
  l = dfl::fma_rn(g.dl[2], vh2, dfl::fma_rn(g.dh[2], vl2, l));
  return {h, l};
}

// a b for unevaluated pairs: leading product exact, first-order cross terms
DF_FN dfl::df dq_mul(dfl::df a, dfl::df b) {
  const float h = dfl::mul_rn(a.hi, b.hi);
  const float e = dfl::fma_rn(a.hi, b.hi, -h);
  return {h, dfl::fma_rn(a.hi, b.lo, dfl::fma_rn(a.lo, b.hi, e))};
}

// Powers of 1/r = y + c. c/y = rho/2 carries delta/R, up to ~2^-19 far from the source drop (the
// remainders' cross term (2 dh + dl).dl), so an unevaluated (y, c) holds only ~44 bits and its powers
// lose more: the pair is renormalised first (Dekker's fast two-sum, |y| >= |c|), y' + c' with
// |c'| <= ulp(y')/2, and the powers are taken from y' with the exact square y'^2 = s + se.
struct DqPow {
  float y, c, s, se;
};

DF_FN DqPow dq_pow(const DqGeo& g) {
  DqPow w;
  w.y = dfl::add_rn(g.y, g.c);
  w.c = dfl::sub_rn(g.c, dfl::sub_rn(w.y, g.y));
  w.s = dfl::mul_rn(w.y, w.y);
  w.se = dfl::fma_rn(w.y, w.y, -w.s);
  return w;
}

// 1/r^3 = y'^3 + 3 y'^2 c' + ... with y'^3 = (s + se) y'
DF_FN dfl::df dq_ri3(const DqPow& w) {
  const float h = dfl::mul_rn(w.s, w.y);
  float l = dfl::fma_rn(w.s, w.y, -h);
  l = dfl::fma_rn(w.se, w.y, l);
  l = dfl::fma_rn(3.0f * w.s, w.c, l);
  return {h, l};
}

// 1/r^2 = s + se + 2 y' c' + ...
DF_FN dfl::df dq_ri2(const DqPow& w) {
  return {w.s, dfl::fma_rn(2.0f * w.y, w.c, w.se)};
}

// d_k t for one component
DF_FN dfl::df dq_comp(const DqGeo& g, int k, dfl::df t) {
  const float h = dfl::mul_rn(g.dh[k], t.hi);
  const float e = dfl::fma_rn(g.dh[k], t.hi, -h);
  return {h, dfl::fma_rn(g.dh[k], t.lo, dfl::fma_rn(g.dl[k], t.hi, e))};
}

#ifdef __CUDACC__
template <int KIND>
DF_FN void dq_term(const float Th[3], const float Tl[3], const dfl::df N0[3], float4 a,
                                        float4 b, float4 c, float4 d, float4 e, float4 gg, dfl::acc* A) {
  using dfl::df;
  DqGeo g;
  dq_geo(Th, Tl, a.x, a.y, a.z, a.w, b.x, b.y, g);
  const df ri{g.y, g.c};
  if (KIND == 1) {
    A[0].add(dq_mul(df{b.z, b.w}, ri));
  } else if (KIND == 0) {
    const df dn = dq_dot(g, N0[0].hi, N0[0].lo, N0[1].hi, N0[1].lo, N0[2].hi, N0[2].lo);
    A[0].add(dq_mul(dq_mul(df{b.z, b.w}, dq_ri3(dq_pow(g))), dn));
  } else if (KIND == 4) {
    // stresslet on u alone: d (d.u)(d.n) / r^5
    const df hu = dq_dot(g, d.x, d.y, d.z, d.w, e.x, e.y);
    const df hn = dq_dot(g, e.z, e.w, gg.x, gg.y, gg.z, gg.w);
    const DqPow w = dq_pow(g);
    const df tt = dq_mul(dq_mul(hu, hn), dq_mul(dq_ri3(w), dq_ri2(w)));
    A[0].add(dq_comp(g, 0, tt));
    A[1].add(dq_comp(g, 1, tt));
    A[2].add(dq_comp(g, 2, tt));
  } else {
    // KIND 2: Stokeslet on f and stresslet on u; KIND 3: Stokeslet alone
    const df fx{b.z, b.w}, fy{c.x, c.y}, fz{c.z, c.w};
    const df hf = dq_dot(g, fx.hi, fx.lo, fy.hi, fy.lo, fz.hi, fz.lo);
    const DqPow w = dq_pow(g);
    const df ri3 = dq_ri3(w);
    df tt;
    if (KIND == 3) {
      tt = dq_mul(ri3, hf);
    } else {
      const df hu = dq_dot(g, d.x, d.y, d.z, d.w, e.x, e.y);
      const df hn = dq_dot(g, e.z, e.w, gg.x, gg.y, gg.z, gg.w);
      // hf + (d.u)(d.n)/r^2, then times 1/r^3
      const df s = dq_mul(dq_mul(hu, hn), dq_ri2(w));
      float sh, se;
      dq_two_sum(hf.hi, s.hi, sh, se);
      tt = dq_mul(ri3, df{sh, dfl::add_rn(se, dfl::add_rn(hf.lo, s.lo))});
    }
    A[0].add(dq_mul(fx, ri));
    A[0].add(dq_comp(g, 0, tt));
    A[1].add(dq_mul(fy, ri));
    A[1].add(dq_comp(g, 1, tt));
    A[2].add(dq_mul(fz, ri));
    A[2].add(dq_comp(g, 2, tt));
  }
}

#endif  // __CUDACC__

}  // namespace shbim
