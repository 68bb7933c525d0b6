// Test probe for the CPU suite: the library's closed-form characteristic
// basis (csrc/euler_basis.cuh) evaluated on the host.  stdin: per line
// "dim gamma U_0 .. U_{dim+1} n_0 .. n_{dim-1}"; stdout: the (dim+2)^2
// entries of L, then those of R, row-major.
#include <cuda_runtime.h>

#include <cstdio>

#include "euler_basis.cuh"

namespace {

template <int DIM>
bool one(double gamma) {
  constexpr int C = DIM + 2;
  double U[C], n[DIM], L[C][C], R[C][C];
  for (int c = 0; c < C; ++c)
    if (std::scanf("%lf", &U[c]) != 1) return false;
  for (int a = 0; a < DIM; ++a)
    if (std::scanf("%lf", &n[a]) != 1) return false;
  wlseno::char_basis<DIM>(U, n, gamma, L, R);
  for (int a = 0; a < C; ++a)
    for (int b = 0; b < C; ++b) std::printf("%.17g ", L[a][b]);
  for (int a = 0; a < C; ++a)
    for (int b = 0; b < C; ++b) std::printf("%.17g ", R[a][b]);
  std::printf("\n");
  return true;
}

}  // namespace

int main() {
  int dim = 0;
  double gamma = 0.0;
  while (std::scanf("%d %lf", &dim, &gamma) == 2) {
    const bool ok = dim == 1 ? one<1>(gamma) : dim == 2 ? one<2>(gamma) : false;
    if (!ok) return 2;
  }
  return 0;
}
