// One row of the FP64 Taylor-moment matrix (Sec. 3.2; h-normalised as in
// Sec. 3.3.2), shared by the moments precompute and the balanced-stencil
// re-selection (which builds the rows of its new stencils on the fly).
//
// For stencil cell j of centre cell i:  A[kappa] = (1/|tau_j|) int_{tau_j}
//   prod_c ((x_c - x_i,c)/h_i)^kappa_c / kappa_c!  dx
// with tau_j taken at its minimum-image copy next to tau_i.  The average over
// the simplex is computed exactly with a (collapsed, Duffy) Gauss-Legendre
// product rule: 1-D x = Y0 + s (Y1 - Y0); 2-D x = Y0 + s (Y1 - Y0) +
// s t (Y2 - Y1), weight 2 s; 3-D x = Y0 + r (Y1 - Y0) + r s (Y2 - Y1) +
// r s t (Y3 - Y2), weight 6 r^2 s.  With K = 4 points per direction the rule
// is exact for the degrees used (<= 4 in 1-D, <= 3 in 2-D, <= 2 in 3-D, plus
// the Jacobian's powers).
#pragma once

#include <cmath>

#include "monomials.cuh"
#include "wlseno_internal.h"

namespace wlseno {

constexpr int kGaussK = 4;
struct GaussRule {
  double x[kGaussK];
  double w[kGaussK];
};

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_K.
inline GaussRule make_gauss_rule() {
  constexpr int K = kGaussK;
  GaussRule g;
  for (int i = 0; i < K; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (K + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int n = 2; n <= K; ++n) {
        double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = K * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    g.x[i] = 0.5 * (1.0 - z);
    g.w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) on [-1,1], halved
  }
  return g;
}

template <int DIM, int M>
__device__ __forceinline__ void moment_row(const DeviceMesh& dm, const GaussRule& g, int64_t i, int64_t j,
                                           double (&acc)[M]) {
  constexpr int K = kGaussK;
  const double* per = dm.period + 3 * dm.mesh_of[i];
  const double hinv = 1.0 / dm.h[i];
  double Y[DIM + 1][DIM];
  for (int a = 0; a < DIM; ++a) {
    const double ci = dm.centroid[i * DIM + a];
    const double cj = dm.centroid[j * DIM + a];
    const double d = cj - ci;
    double shift = 0.0;
    if (per[a] > 0.0) shift = -per[a] * nearbyint(d / per[a]);
    for (int v = 0; v <= DIM; ++v)
      Y[v][a] = (dm.coords[(j * (DIM + 1) + v) * DIM + a] + shift - ci) * hinv;
  }
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = 0.0;
  if (DIM == 1) {  // Gauss-Legendre on the segment (weights sum to 1)
    for (int qs = 0; qs < K; ++qs) {
      double y[DIM];
      for (int a = 0; a < DIM; ++a) y[a] = Y[0][a] + g.x[qs] * (Y[1][a] - Y[0][a]);
      double mono[M];
      eval_monomials<double, DIM, M>(y, mono);
#pragma unroll
      for (int c = 0; c < M; ++c) acc[c] += g.w[qs] * mono[c];
    }
  } else if (DIM == 2) {
    for (int qs = 0; qs < K; ++qs)
      for (int qt = 0; qt < K; ++qt) {
        const double s = g.x[qs], t = g.x[qt];
        const double wq = 2.0 * g.w[qs] * g.w[qt] * s;
        double y[DIM];
        for (int a = 0; a < DIM; ++a)
          y[a] = Y[0][a] + s * (Y[1][a] - Y[0][a]) + s * t * (Y[2][a] - Y[1][a]);
        double mono[M];
        eval_monomials<double, DIM, M>(y, mono);
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] += wq * mono[c];
      }
  } else {
    for (int qr = 0; qr < K; ++qr)
      for (int qs = 0; qs < K; ++qs)
        for (int qt = 0; qt < K; ++qt) {
          const double r = g.x[qr], s = g.x[qs], t = g.x[qt];
          const double wq = 6.0 * g.w[qr] * g.w[qs] * g.w[qt] * r * r * s;
          double y[DIM];
          for (int a = 0; a < DIM; ++a)
            y[a] = Y[0][a] + r * (Y[1][a] - Y[0][a]) + r * s * (Y[2][a] - Y[1][a]) +
                   r * s * t * (Y[3][a] - Y[2][a]);
          double mono[M];
          eval_monomials<double, DIM, M>(y, mono);
#pragma unroll
          for (int c = 0; c < M; ++c) acc[c] += wq * mono[c];
        }
  }
}

}  // namespace wlseno
