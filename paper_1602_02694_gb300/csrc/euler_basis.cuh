// Characteristic basis of the Euler equations for one facet (host and
// device): at the state us (d + 2 conserved components) and the facet's unit
// normal n, the right eigenvectors R (columns, eigenvalues u.n - c, u.n,
// [u.n,] u.n + c) of d(F(U).n)/dU and L = R^-1 in closed form, for 1-D and
// 2-D (the formulas are written out in k_euler_char.cu).
#pragma once

#include <cmath>

namespace wlseno {

// The basis of the facet with normal n at the state us (d + 2 components).
template <int DIM>
__host__ __device__ __forceinline__ void char_basis(const double (&us)[DIM + 2], const double* n, double gamma,
                                           double (&Ld)[DIM + 2][DIM + 2], double (&Rd)[DIM + 2][DIM + 2]) {
  constexpr int C = DIM + 2;
  const double rho = us[0];
  double vel[DIM], ke = 0.0, un = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    vel[a] = us[1 + a] / rho;
    ke += 0.5 * vel[a] * vel[a];
    un += vel[a] * n[a];
  }
  const double p = (gamma - 1.0) * (us[C - 1] - rho * ke);
  const double cs = sqrt(gamma * p / rho);
  const double H = (us[C - 1] + p) / rho;
  const double b1 = (gamma - 1.0) / (cs * cs), b2 = ke * b1;
  if constexpr (DIM == 1) {
    const double u = vel[0], nx = n[0];
    const double L1[3][3] = {{0.5 * (b2 + un / cs), 0.5 * (-b1 * u - nx / cs), 0.5 * b1},
                             {1.0 - b2, b1 * u, -b1},
                             {0.5 * (b2 - un / cs), 0.5 * (-b1 * u + nx / cs), 0.5 * b1}};
    const double R1[3][3] = {{1.0, 1.0, 1.0}, {u - cs * nx, u, u + cs * nx}, {H - cs * un, ke, H + cs * un}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Ld[a][b] = L1[a][b];
        Rd[a][b] = R1[a][b];
      }
  } else {
    const double u = vel[0], v = vel[1], nx = n[0], ny = n[1];
    const double ut = -u * ny + v * nx;
    const double L2[4][4] = {{0.5 * (b2 + un / cs), 0.5 * (-b1 * u - nx / cs), 0.5 * (-b1 * v - ny / cs), 0.5 * b1},
                             {1.0 - b2, b1 * u, b1 * v, -b1},
                             {-ut, -ny, nx, 0.0},
                             {0.5 * (b2 - un / cs), 0.5 * (-b1 * u + nx / cs), 0.5 * (-b1 * v + ny / cs), 0.5 * b1}};
    const double R2[4][4] = {{1.0, 1.0, 0.0, 1.0},
                             {u - cs * nx, u, -ny, u + cs * nx},
                             {v - cs * ny, v, nx, v + cs * ny},
                             {H - cs * un, ke, ut, H + cs * un}};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        Ld[a][b] = L2[a][b];
        Rd[a][b] = R2[a][b];
      }
  }
}

}  // namespace wlseno
