// FP64 Taylor-moment precompute (Sec. 3.2; h-normalised as in Sec. 3.3.2).
//
// For stencil row (i, j):  A[e][kappa] = (1/|tau_j|) int_{tau_j}
//   prod_c ((x_c - x_i,c)/h_i)^kappa_c / kappa_c!  dx
// with tau_j taken at its minimum-image copy next to tau_i.  The average over
// the simplex is computed exactly with a (collapsed, Duffy) Gauss-Legendre
// product rule: 1-D x = Y0 + s (Y1 - Y0); 2-D x = Y0 + s (Y1 - Y0) +
// s t (Y2 - Y1), weight 2 s; 3-D x = Y0 + r (Y1 - Y0) + r s (Y2 - Y1) +
// r s t (Y3 - Y2), weight 6 r^2 s.  With K = 4 points per direction the rule
// is exact for the degrees used (<= 4 in 1-D, <= 3 in 2-D, <= 2 in 3-D, plus
// the Jacobian's powers).
#include <cmath>

#include "wlseno_internal.h"
#include "monomials.cuh"

namespace wlseno {
namespace {

constexpr int K = 4;
struct GaussRule {
  double x[K];
  double w[K];
};

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_K.
GaussRule make_rule() {
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
__global__ void moments_kernel(DeviceMesh dm, GaussRule g) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= dm.nnz) return;
  // owner row i of stencil entry e (binary search on st_ptr)
  int64_t lo = 0, hi = dm.N;  // st_ptr[lo] <= e < st_ptr[hi]
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (dm.st_ptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  const int64_t i = lo;
  const int64_t j = dm.st_idx[e];
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
  double acc[M];
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
#pragma unroll
  for (int c = 0; c < M; ++c) {
    dm.A64[e * M + c] = acc[c];
    dm.A32[e * M + c] = static_cast<float>(acc[c]);
  }
}

template <int DIM, int M>
cudaError_t launch_dm(const DeviceMesh& dm, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (dm.nnz + threads - 1) / threads;
  moments_kernel<DIM, M><<<static_cast<unsigned>(blocks), threads, 0, s>>>(dm, make_rule());
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_moments(const DeviceMesh& dm, cudaStream_t s) {
  if (dm.dim == 1) {
    switch (dm.m) {
      case 3: return launch_dm<1, 3>(dm, s);
      case 5: return launch_dm<1, 5>(dm, s);
    }
  } else if (dm.dim == 2) {
    switch (dm.m) {
      case 3: return launch_dm<2, 3>(dm, s);
      case 6: return launch_dm<2, 6>(dm, s);
      case 10: return launch_dm<2, 10>(dm, s);
    }
  } else {
    switch (dm.m) {
      case 4: return launch_dm<3, 4>(dm, s);
      case 10: return launch_dm<3, 10>(dm, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace wlseno
