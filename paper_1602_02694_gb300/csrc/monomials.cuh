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

// Moments on the fly.  The row of stencil cell j is the cell average over
// tau_j of prod_a y_a^kappa_a / kappa_a! with y = (x - x_i)/h_i.  Writing
// y = w + d, w = (x - x_j)/h_i and d = (x_j - x_i)/h_i, the binomial theorem
// gives (w_a + d_a)^k / k! = sum_{b <= k} w_a^b / b! d_a^(k-b) / (k-b)!, so
//   A[kappa] = sum_{alpha <= kappa} M_j[alpha] h_i^-|alpha| d^(kappa-alpha) / (kappa-alpha)!
// with M_j[alpha] cell j's own central moments (absolute units; M_j[0] = 1,
// M_j[alpha] = 0 for |alpha| = 1 about the centroid).  own holds M_j for the
// columns of degree >= 2 in column order, hp[k] = h_i^-k.
template <int DIM>
__host__ __device__ constexpr int taylor_deg(int c) {
  int s = 0;
  for (int a = 0; a < DIM; ++a) s += exponent<DIM>(c, a);
  return s;
}

template <int DIM, int M>
__host__ __device__ __forceinline__ void shifted_row(const float (&d)[DIM], const float (&hp)[5], const float* own,
                                            float (&row)[M]) {
  float pw[DIM][5];  // d_a^k / k!
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    pw[a][0] = 1.0f;
    pw[a][1] = d[a];
    pw[a][2] = d[a] * d[a] * 0.5f;
    pw[a][3] = pw[a][2] * d[a] * (1.0f / 3.0f);
    pw[a][4] = pw[a][3] * d[a] * 0.25f;
  }
  float ms[M];  // own moments in h_i units, by column
#pragma unroll
  for (int c = 0, k = 0; c < M; ++c) {
    if (taylor_deg<DIM>(c) >= 2) ms[c] = own[k++] * hp[taylor_deg<DIM>(c)];
    else ms[c] = c == 0 ? 1.0f : 0.0f;
  }
#pragma unroll
  for (int c = 0; c < M; ++c) {
    float acc = 0.0f;
#pragma unroll
    for (int c2 = 0; c2 < M; ++c2) {
      if (taylor_deg<DIM>(c2) == 1) continue;
      bool below = true;
#pragma unroll
      for (int a = 0; a < DIM; ++a) below = below && exponent<DIM>(c2, a) <= exponent<DIM>(c, a);
      if (!below) continue;
      float term = ms[c2];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int e = exponent<DIM>(c, a) - exponent<DIM>(c2, a);
        if (e > 0) term *= pw[a][e];
      }
      acc += term;
    }
    row[c] = acc;
  }
}

}  // namespace wlseno
