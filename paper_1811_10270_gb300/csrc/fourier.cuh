// Device helpers shared by the transform kernels (header-only: no separate compilation).
#pragma once

namespace shbim {

// Fourier synthesis of V(k) = a0 + sqrt2 (sum_m a_m cos(m phi_k) + beta sum_m b_m sin(m phi_k)),
// m = 1..p, phi_k = 2 pi k / N, at the four longitudes k, N-k, N/2-k, N/2+k at once
// (N divisible by 4, 0 <= k <= N/4). With the partial sums split by the parity of m,
// cos(m(pi - phi)) = (-1)^m cos(m phi) and sin(m(pi - phi)) = -(-1)^m sin(m phi), one pass of
// 2p FMAs gives all four outputs.
__device__ __forceinline__ void synth4(const double* __restrict__ a, const double* __restrict__ b,
                                       double a0, double beta, int p, int k, int N,
                                       const double* __restrict__ tc, const double* __restrict__ ts,
                                       double* __restrict__ dst) {
  double ce = 0.0, co = 0.0, se = 0.0, so = 0.0;
  int id = 0;
  int m = 1;
  for (; m + 1 <= p; m += 2) {
    id += k;
    if (id >= N) id -= N;
    co = fma(a[m], tc[id], co);
    so = fma(b[m], ts[id], so);
    id += k;
    if (id >= N) id -= N;
    ce = fma(a[m + 1], tc[id], ce);
    se = fma(b[m + 1], ts[id], se);
  }
  if (m <= p) {
    id += k;
    if (id >= N) id -= N;
    co = fma(a[m], tc[id], co);
    so = fma(b[m], ts[id], so);
  }
  const double s2 = 1.41421356237309504880;
  const double c1 = ce + co, s1 = beta * (se + so);
  const double c2 = ce - co, s2v = beta * (so - se);
  const int h = N >> 1;
  dst[k] = a0 + s2 * (c1 + s1);
  dst[(N - k) % N] = a0 + s2 * (c1 - s1);
  dst[h - k] = a0 + s2 * (c2 + s2v);
  dst[h + k] = a0 + s2 * (c2 - s2v);
}

}  // namespace shbim
