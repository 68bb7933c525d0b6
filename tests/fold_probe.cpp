// Test probe for the CPU suite: the library's square-root-free Givens fold
// (csrc/k_recon_tpc.cuh: sqrt_free_init / fold / spread / solve, FP64)
// compiled as host C++, on weighted least-squares problems read from stdin:
// "n" then n rows of "w a_0 .. a_9 b"; prints "x x_0 .. x_9",
// "spread qmax qmin" and "est z" (the inverse estimate of the factor); with
// the argument "first" the first row of each problem is folded by
// sqrt_free_fold_first.  The probe supplies the host stand-in for the
// correctly rounded FP64 reciprocal the fold uses on the device.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>

static inline double __drcp_rn(double x) { return 1.0 / x; }

#include "k_recon_tpc.cuh"

int main(int argc, char** argv) {
  constexpr int M = 10;
  // "first": the first row of each problem is folded by sqrt_free_fold_first
  // (as the all-components kernel folds its centre row)
  const bool first = argc > 1 && std::string(argv[1]) == "first";
  int n = 0;
  while (std::scanf("%d", &n) == 1) {
    wlseno::SqrtFreeQR<double, M> f;
    wlseno::sqrt_free_init(f);
    for (int t = 0; t < n; ++t) {
      double w = 0.0, z[M + 1];
      if (std::scanf("%lf", &w) != 1) return 2;
      for (int c = 0; c <= M; ++c)
        if (std::scanf("%lf", &z[c]) != 1) return 2;
      if (first && t == 0)
        wlseno::sqrt_free_fold_first(f, z, w * w);
      else
        wlseno::sqrt_free_fold(f, z, w * w);
    }
    double qmax = 0.0, qmin = 0.0, x[M];
    wlseno::sqrt_free_spread(f, &qmax, &qmin);
    wlseno::sqrt_free_solve(f, x);
    std::printf("x");
    for (int c = 0; c < M; ++c) std::printf(" %.17g", x[c]);
    std::printf("\nspread %.17g %.17g\n", qmax, qmin);
    std::printf("est %.9g\n", static_cast<double>(wlseno::sqrt_free_inverse_estimate(f)));
  }
  return 0;
}
