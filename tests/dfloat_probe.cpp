// Test probe for the CPU suite: the library's double-float arithmetic
// (csrc/dfloat.cuh) compiled as plain C++ -- tests/test_dfloat.py supplies a
// stand-in <cuda_runtime.h> that maps the round-to-nearest intrinsics to IEEE
// single-precision operations -- and applied to operand pairs read from
// stdin.  Each input line "op a_hi a_lo b_hi b_lo" (op: add, mul) prints the
// result pair as "hi lo" in %a form (exact).  With the argument "split" it
// instead reads 64-bit patterns (hex) and prints, per line, whether the
// integer split df_from_double_bits gives the bits of df_from_double, and
// whether df_f64_bits_nonneg of |fl32(v)| gives the bits of its FP64 value
// ("1 1" when both agree).
#include <cstdio>
#include <cmath>
#include <cstring>

#include "dfloat.cuh"

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "split") == 0) {
    unsigned long long b;
    while (std::scanf("%llx", &b) == 1) {
      double v;
      std::memcpy(&v, &b, sizeof v);
      const wlseno::dfloat x = wlseno::df_from_double_bits(v), y = wlseno::df_from_double(v);
      const bool same = std::memcmp(&x.hi, &y.hi, 4) == 0 && std::memcmp(&x.lo, &y.lo, 4) == 0;
      const float a = std::fabs(static_cast<float>(v));
      const double ad = static_cast<double>(a);
      unsigned long long ab;
      std::memcpy(&ab, &ad, sizeof ab);
      const bool same_max = a != a || wlseno::df_f64_bits_nonneg(a) == ab;
      std::printf("%d %d\n", same ? 1 : 0, same_max ? 1 : 0);
    }
    return 0;
  }
  char op[8];
  float a_hi, a_lo, b_hi, b_lo;
  while (std::scanf("%7s %a %a %a %a", op, &a_hi, &a_lo, &b_hi, &b_lo) == 5) {
    const wlseno::dfloat a{a_hi, a_lo}, b{b_hi, b_lo};
    const wlseno::dfloat r = std::strcmp(op, "add") == 0 ? wlseno::df_add(a, b) : wlseno::df_mul(a, b);
    std::printf("%a %a\n", static_cast<double>(r.hi), static_cast<double>(r.lo));
  }
  return 0;
}
