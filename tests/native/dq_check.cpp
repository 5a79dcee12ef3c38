// Host driver for tests/test_dq_host.py: the quantised double-float kernel terms of pair_dq.cuh on
// the host. Each input line: Q, then the target offset from the source drop's centre (3 doubles), the
// source node's offset (3 doubles), the strength s and the target normal n0 (3 doubles). The positions
// are split as the library splits them (the multiple of 2^-Q nearest to the offset, and the FP32
// remainder). Output per line: 1/r, r^2, s/r (single layer), s (d.n0)/r^3 (target-normal double
// layer) and 1/r^5 (the stresslet's power), each the double value of an unevaluated FP32 pair.
#include <cmath>
#include <cstdio>

#include "pair_dq.cuh"

using shbim::DqGeo;

static void split(double v, double qs, double qi, float* h, float* l) {
  const double q = std::rint(v * qs) * qi;
  *h = (float)q;
  *l = (float)(v - q);
}

static double val(dfl::df a) { return (double)a.hi + (double)a.lo; }

int main() {
  int Q;
  double T[3], V[3], sg, n0[3];
  while (std::scanf("%d %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf", &Q, &T[0], &T[1], &T[2], &V[0], &V[1], &V[2],
                    &sg, &n0[0], &n0[1], &n0[2]) == 11) {
    const double qs = std::ldexp(1.0, Q), qi = std::ldexp(1.0, -Q);
    float Th[3], Tl[3], Vh[3], Vl[3];
    for (int k = 0; k < 3; ++k) {
      split(T[k], qs, qi, &Th[k], &Tl[k]);
      split(V[k], qs, qi, &Vh[k], &Vl[k]);
    }
    DqGeo g;
    shbim::dq_geo(Th, Tl, Vh[0], Vh[1], Vh[2], Vl[0], Vl[1], Vl[2], g);
    const dfl::df s = dfl::from_double(sg);
    const dfl::df N[3] = {dfl::from_double(n0[0]), dfl::from_double(n0[1]), dfl::from_double(n0[2])};
    const dfl::df ri{g.y, g.c};
    // r^2 from the pieces dq_geo uses: (dh + dl).(dh + dl) with the exact dh
    double r2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double d = (double)g.dh[k] + (double)g.dl[k];
      r2 += d * d;
    }
    const dfl::df sl = shbim::dq_mul(s, ri);
    const dfl::df dn = shbim::dq_dot(g, N[0].hi, N[0].lo, N[1].hi, N[1].lo, N[2].hi, N[2].lo);
    const shbim::DqPow w = shbim::dq_pow(g);
    const dfl::df dl = shbim::dq_mul(shbim::dq_mul(s, shbim::dq_ri3(w)), dn);
    const dfl::df r5 = shbim::dq_mul(shbim::dq_ri3(w), shbim::dq_ri2(w));
    std::printf("%.17g %.17g %.17g %.17g %.17g\n", val(ri), r2, val(sl), val(dl), val(r5));
  }
  return 0;
}
