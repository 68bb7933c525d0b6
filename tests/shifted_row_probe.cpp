// Test probe for the CPU suite: the library's moment rows formed on the fly
// (shifted_row in csrc/monomials.cuh, FP32, as the on-the-fly kernel forms
// them) evaluated on the host.  stdin: "dim m", then per row "d_0 .. d_{dim-1}
// h_inv own_0 .. own_{m-2-dim}"; stdout: the m entries of each row.
#include <cuda_runtime.h>

#include <cstdio>

#include "monomials.cuh"

namespace {

template <int DIM, int M>
void run() {
  float d[DIM], hinv, own[M];
  for (;;) {
    for (int a = 0; a < DIM; ++a)
      if (std::scanf("%f", &d[a]) != 1) return;
    if (std::scanf("%f", &hinv) != 1) return;
    for (int k = 0; k < M - 1 - DIM; ++k)
      if (std::scanf("%f", &own[k]) != 1) return;
    float hp[5] = {1.0f, hinv, hinv * hinv, hinv * hinv * hinv, hinv * hinv * hinv * hinv};
    float row[M];
    wlseno::shifted_row<DIM, M>(d, hp, own, row);
    for (int c = 0; c < M; ++c) std::printf("%.9g ", static_cast<double>(row[c]));
    std::printf("\n");
  }
}

}  // namespace

int main() {
  int dim = 0, m = 0;
  if (std::scanf("%d %d", &dim, &m) != 2) return 2;
  if (dim == 1 && m == 3) run<1, 3>();
  else if (dim == 1 && m == 5) run<1, 5>();
  else if (dim == 2 && m == 6) run<2, 6>();
  else if (dim == 2 && m == 10) run<2, 10>();
  else if (dim == 3 && m == 10) run<3, 10>();
  else return 3;
  return 0;
}
