// Scaled Taylor monomials prod_c y_c^kappa_c / kappa_c! in the column order of
// the moment matrix: by degree, then descending power of x, then of y
// (1-D: 1, x, x^2, x^3, x^4;
//  2-D: 1, x, y, x^2, xy, y^2, x^3, x^2y, xy^2, y^3;
//  3-D: 1, x, y, z, x^2, xy, xz, y^2, yz, z^2).
#pragma once

namespace wlseno {

// Exponent of axis a in column c.
template <int DIM>
__host__ __device__ constexpr int exponent(int c, int a) {
  if (DIM == 1) {
    return c;
  } else if (DIM == 2) {
    constexpr int ex[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
    constexpr int ey[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
    return a == 0 ? ex[c] : ey[c];
  } else {
    constexpr int ex[10] = {0, 1, 0, 0, 2, 1, 1, 0, 0, 0};
    constexpr int ey[10] = {0, 0, 1, 0, 0, 1, 0, 2, 1, 0};
    constexpr int ez[10] = {0, 0, 0, 1, 0, 0, 1, 0, 1, 2};
    return a == 0 ? ex[c] : (a == 1 ? ey[c] : ez[c]);
  }
}

template <typename T, int DIM, int M>
__host__ __device__ __forceinline__ void eval_monomials(const T (&y)[DIM], T (&mono)[M]) {
  // pw[a][k] = y_a^k / k!
  T pw[DIM][5];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    pw[a][0] = T(1);
    pw[a][1] = y[a];
    pw[a][2] = y[a] * y[a] * T(0.5);
    pw[a][3] = pw[a][2] * y[a] * T(1.0 / 3.0);
    pw[a][4] = pw[a][3] * y[a] * T(0.25);
  }
#pragma unroll
  for (int c = 0; c < M; ++c) {
    T v = pw[0][exponent<DIM>(c, 0)];
#pragma unroll
    for (int a = 1; a < DIM; ++a) v *= pw[a][exponent<DIM>(c, a)];
    mono[c] = v;
  }
}

}  // namespace wlseno
