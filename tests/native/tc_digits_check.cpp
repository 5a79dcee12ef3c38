// Host driver for the digit arithmetic of the tensor-core kernels (tc_digits.cuh). One request per
// line on stdin, one answer per line on stdout; floating-point values travel as hexadecimal (%a):
//   D yh yl        -> the six digits d0..d5 of digits6(yh, yl)       (FP32 operands)
//   H x e          -> the six digits d0..d5 of digits_host(x, e)     (FP64 operand)
//   C a5 .. a0     -> hi lo of combine6(a5, .., a0)                  (FP32 operands)
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tc_digits.cuh"

int main() {
  char op[4];
  char s[6][64];
  while (std::scanf("%3s", op) == 1) {
    if (op[0] == 'D') {
      if (std::scanf("%63s %63s", s[0], s[1]) != 2) return 1;
      float d[shbim::tc::kDig];
      shbim::tc::digits6(std::strtof(s[0], nullptr), std::strtof(s[1], nullptr), d);
      std::printf("%d %d %d %d %d %d\n", (int)d[0], (int)d[1], (int)d[2], (int)d[3], (int)d[4], (int)d[5]);
    } else if (op[0] == 'H') {
      int e = 0;
      if (std::scanf("%63s %d", s[0], &e) != 2) return 1;
      int d[shbim::tc::kDig];
      shbim::tc::digits_host(std::strtod(s[0], nullptr), e, d);
      std::printf("%d %d %d %d %d %d\n", d[0], d[1], d[2], d[3], d[4], d[5]);
    } else if (op[0] == 'C') {
      float a[6];
      for (int i = 0; i < 6; ++i) {
        if (std::scanf("%63s", s[i]) != 1) return 1;
        a[i] = std::strtof(s[i], nullptr);
      }
      const dfl::df r = shbim::tc::combine6(a[0], a[1], a[2], a[3], a[4], a[5]);
      std::printf("%a %a\n", (double)r.hi, (double)r.lo);
    } else {
      return 1;
    }
  }
  return 0;
}
