// Host driver for tests/test_df_term_host.py: the general double-float kernel terms of pair_df.cuh on
// the host. Each input line: KIND, the target offset T (3 doubles), the source offset V (3), the
// Laplace strength s or the Stokes density f (3), u (3), the source normal n (3) and the target normal
// N0 (3), all relative to the source drop's centre. Every double is split as the library stages it
// (FP32 value and FP32 remainder). Output per line: the three accumulators (one for Laplace) as doubles.
#include <cstdio>

struct float4 {
  float x, y, z, w;
};

#include "pair_df.cuh"

static void split(double v, float* h, float* l) {
  *h = (float)v;
  *l = (float)(v - (double)*h);
}

int main() {
  int kind;
  double T[3], V[3], f[3], u[3], n[3], N[3];
  while (std::scanf("%d", &kind) == 1) {
    double* fields[6] = {T, V, f, u, n, N};
    bool ok = true;
    for (double* v : fields)
      for (int k = 0; k < 3; ++k) ok = ok && std::scanf("%lf", &v[k]) == 1;
    if (!ok) return 1;
    float Vh[3], Vl[3], fh[3], fl[3], uh[3], ul[3], nh[3], nl[3];
    dfl::df Td[3], Nd[3];
    for (int k = 0; k < 3; ++k) {
      split(V[k], &Vh[k], &Vl[k]);
      split(f[k], &fh[k], &fl[k]);
      split(u[k], &uh[k], &ul[k]);
      split(n[k], &nh[k], &nl[k]);
      split(T[k], &Td[k].hi, &Td[k].lo);
      split(N[k], &Nd[k].hi, &Nd[k].lo);
    }
    const float4 a{Vh[0], Vh[1], Vh[2], Vl[0]}, b{Vl[1], Vl[2], fh[0], fl[0]}, c{fh[1], fl[1], fh[2], fl[2]},
        d{uh[0], ul[0], uh[1], ul[1]}, e{uh[2], ul[2], nh[0], nl[0]}, g{nh[1], nl[1], nh[2], nl[2]};
    dfl::acc A[3];
    switch (kind) {
      case 0: shbim::df_term<0>(Td, Nd, a, b, c, d, e, g, A); break;
      case 1: shbim::df_term<1>(Td, Nd, a, b, c, d, e, g, A); break;
      case 2: shbim::df_term<2>(Td, Nd, a, b, c, d, e, g, A); break;
      case 3: shbim::df_term<3>(Td, Nd, a, b, c, d, e, g, A); break;
      default: shbim::df_term<4>(Td, Nd, a, b, c, d, e, g, A); break;
    }
    std::printf("%.17g %.17g %.17g\n", dfl::to_double(A[0].value()), dfl::to_double(A[1].value()),
                dfl::to_double(A[2].value()));
  }
  return 0;
}
