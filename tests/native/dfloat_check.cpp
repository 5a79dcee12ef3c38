// Host driver for the double-float header: reads operand pairs (as doubles, one pair per line)
// from stdin and prints, per line, the double-float results of add, mul, sqr, rsqrt, sqrt, div and
// of the accumulator (a*b summed over all lines so far), each converted to double with %.17g.
#include <cstdio>

#include "dfloat.cuh"

int main() {
  double a, b;
  dfl::acc s;
  while (std::scanf("%lf %lf", &a, &b) == 2) {
    const dfl::df x = dfl::from_double(a), y = dfl::from_double(b);
    s.add_prod(x, y);
    std::printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", dfl::to_double(dfl::add(x, y)),
                dfl::to_double(dfl::mul(x, y)), dfl::to_double(dfl::sqr(x)),
                dfl::to_double(dfl::rsqrt(dfl::mul(x, x))), dfl::to_double(dfl::sqrt(dfl::mul(x, x))),
                dfl::to_double(dfl::div(x, y)), dfl::to_double(s.value()));
  }
  return 0;
}
