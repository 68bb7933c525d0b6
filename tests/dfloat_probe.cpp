// Test probe for the CPU suite: the library's double-float arithmetic
// (csrc/dfloat.cuh) compiled as plain C++ -- tests/test_dfloat.py supplies a
// stand-in <cuda_runtime.h> that maps the round-to-nearest intrinsics to IEEE
// single-precision operations -- and applied to operand pairs read from
// stdin.  Each input line "op a_hi a_lo b_hi b_lo" (op: add, mul) prints the
// result pair as "hi lo" in %a form (exact).
#include <cstdio>
#include <cstring>

#include "dfloat.cuh"

int main() {
  char op[8];
  float a_hi, a_lo, b_hi, b_lo;
  while (std::scanf("%7s %a %a %a %a", op, &a_hi, &a_lo, &b_hi, &b_lo) == 5) {
    const wlseno::dfloat a{a_hi, a_lo}, b{b_hi, b_lo};
    const wlseno::dfloat r = std::strcmp(op, "add") == 0 ? wlseno::df_add(a, b) : wlseno::df_mul(a, b);
    std::printf("%a %a\n", static_cast<double>(r.hi), static_cast<double>(r.lo));
  }
  return 0;
}
