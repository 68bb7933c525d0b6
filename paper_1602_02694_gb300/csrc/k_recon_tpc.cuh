// WLS-ENO reconstruction, one thread per cell (Sec. 3.1.2, Sec. 3.2,
// Sec. 3.3.2): the row fold and its helpers.
//
// The weighted least-squares problem of cell i is min sum_t delta_t
// (x_t . d - b_t)^2 over its stencil rows, with x_t the moment row of cell t
// (Sec. 3.2), b_t = ubar_t - ubar_i and delta_t = w_t^2 the squared weight of
// Sec. 3.1.2 -- the problem whose rows are w_t [x_t | b_t].  The thread folds
// its rows one at a time into the triangular factor of W A = Q R by Givens
// rotations in the square-root-free form of Gentleman (1973, "Least squares
// computations by Givens transformations without square roots"; Applied
// Statistics algorithm AS 75): R = D^(1/2) U with U unit upper triangular and
// D = diag(d_k), so an incoming row (z, delta) updates, for k = 0..m-1,
//
//   d_k' = d_k + delta z_k^2,   cbar = d_k / d_k',   sbar = delta z_k / d_k',
//   z_j <- z_j - z_k u_kj,       u_kj <- u_kj + sbar z_j      (j > k),
//   delta <- delta cbar,
//
// which is the Givens rotation that annihilates the row against row k of R
// (the same Q and R), written without square roots: two multiply-adds per
// entry instead of four.  The right-hand side is column m of U, so
// R d = Q^T W b reduces to the unit-triangular U d = u_{:,m}: no divisions.
// Column k of R has squared norm n_k = sum_{i<=k} d_i u_ik^2, so the
// column-scaled diagonal of W A S (S = diag(1/||col R||), Sec. 3.3.2) is
// q_k = sqrt(d_k / n_k); its spread bounds the conditioning of W A S.
//
// d_k starts at a tiny tau instead of 0 (a prior tau u_k^2 far below the
// rounding of any real row): the first row reaching column k then needs no
// special case, and a zero row leaves D and U unchanged exactly.
#pragma once

#include <cmath>
#include <utility>

#include "monomials.cuh"
#include "wlseno_internal.h"

namespace wlseno {

// Reciprocal for the fold: FP32 uses the hardware approximation (about 1 ulp,
// inside the rounding the FP32 factorisation already carries); FP64 the
// correctly rounded reciprocal.
template <typename T>
__device__ __forceinline__ T recip_t(T x);
template <>
__device__ __forceinline__ float recip_t<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <>
__device__ __forceinline__ double recip_t<double>(double x) { return __drcp_rn(x); }

template <typename T>
__device__ __forceinline__ constexpr T fold_tau() { return sizeof(T) == 4 ? T(1e-30) : T(1e-280); }

// The square-root-free factor: d[k] and U[k][j] for j > k (column m is the
// transformed right-hand side).  Entries with j <= k are never touched.
template <typename T, int M>
struct SqrtFreeQR {
  T d[M];
  T U[M][M + 1];
};

template <typename T, int M>
__device__ __forceinline__ void sqrt_free_init(SqrtFreeQR<T, M>& f) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    f.d[k] = fold_tau<T>();
#pragma unroll
    for (int j = k + 1; j <= M; ++j) f.U[k][j] = T(0);
  }
}

// Fold the row z (z[M] = right-hand side) with weight delta into f.
//
// Of the two algebraically equal updates of U -- with x = z_j before the
// update, Gentleman's u_kj' = cbar u_kj + sbar x, or u_kj' = u_kj + sbar z_j'
// with z_j' = x - z_k u_kj -- this is the second, which saves a multiply
// per entry.  It leaves u_kj' an absolute rounding error of about
// eps |u_kj| when the incoming row dominates row k (cbar small) and the new
// entry is much smaller than the old: harmless for the solution, but where
// a few rows of far larger weight than the others carry nearly dependent
// moment rows (weights spanning 1e13, say), it can leave a moderate
// diagonal where the true factor has an entry near 0, and the conditioning
// estimates then miss the near dependence.  The FP64 kernel therefore also
// sends every cell whose weights span more than kWeightSpread to the
// pivoted path (the error stays below eps times the spread of the row
// weights otherwise).
template <typename T, int M>
__device__ __forceinline__ void sqrt_free_fold(SqrtFreeQR<T, M>& f, T (&z)[M + 1], T delta) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const T zk = z[k];
    const T t = delta * zk;
    const T dn = fma(t, zk, f.d[k]);
    const T r = recip_t<T>(dn);
    const T sbar = t * r;
    delta *= f.d[k] * r;
    f.d[k] = dn;
#pragma unroll
    for (int j = k + 1; j <= M; ++j) {
      z[j] = fma(-zk, f.U[k][j], z[j]);
      f.U[k][j] = fma(sbar, z[j], f.U[k][j]);
    }
  }
}

// The first row folded into a fresh factor (d_k = tau, U = 0), as far as row
// 0 of the factor: its z_0 = 1 (the constant column) is absorbed there,
// leaving a weight of tau delta / (tau + delta), about tau, for the rows
// below, where the full fold would put entries weighted at the scale of tau,
// far below the rounding of any row that follows.  (z_0 != 0 for every row
// of the moment matrix, whose constant column is 1.)
template <typename T, int M>
__device__ __forceinline__ void sqrt_free_fold_first(SqrtFreeQR<T, M>& f, const T (&z)[M + 1], T delta) {
  const T t = delta * z[0];
  const T dn = fma(t, z[0], f.d[0]);
  const T sbar = t * recip_t<T>(dn);
  f.d[0] = dn;
#pragma unroll
  for (int j = 1; j <= M; ++j) f.U[0][j] = sbar * z[j];  // U[0][j] was 0: z_j unchanged by row 0
}

// Spread of the row weights above which the FP64 thread-per-cell kernel
// sends a cell to the pivoted path (see sqrt_free_fold).
constexpr double kWeightSpread = 1e6;

// Spread of the column-scaled diagonal: qmax = max_k q_k^2 and qmin =
// min_k q_k^2.  A cell is ill-conditioned at threshold K when
// !(qmax <= K^2 qmin), which also catches a zero or non-finite diagonal.
// Squared column norms n_k = sum_{i<=k} d_i u_ik^2 of R.
template <typename T, int M>
__host__ __device__ __forceinline__ void sqrt_free_colnorms(const SqrtFreeQR<T, M>& f, T (&nrm)[M]) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    T n = f.d[k];
#pragma unroll
    for (int i = 0; i < k; ++i) n = fma(f.d[i] * f.U[i][k], f.U[i][k], n);
    nrm[k] = n;
  }
}

template <typename T, int M>
__device__ __forceinline__ void sqrt_free_spread(const SqrtFreeQR<T, M>& f, const T (&nrm)[M], T* qmax_out,
                                                 T* qmin_out) {
  T qmax = T(0), qmin = T(INFINITY);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    // (FP32: the hardware reciprocal, ample for a threshold test)
    const T q = sizeof(T) == 4 ? f.d[k] * recip_t<T>(nrm[k]) : f.d[k] / nrm[k];
    qmax = q > qmax ? q : qmax;
    qmin = q < qmin ? q : qmin;
  }
  *qmax_out = qmax;
  *qmin_out = qmin;
}

template <typename T, int M>
__device__ __forceinline__ void sqrt_free_spread(const SqrtFreeQR<T, M>& f, T* qmax_out, T* qmin_out) {
  T nrm[M];
  sqrt_free_colnorms(f, nrm);
  sqrt_free_spread(f, nrm, qmax_out, qmin_out);
}

// Approximate 1/sqrt for the estimate below (the hardware approximation on
// the device; the host-compiled tests use the library's sqrt).
__host__ __device__ __forceinline__ float est_rsqrt(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / std::sqrt(x);
#endif
}

// Approximate reciprocal for the estimate below (the hardware
// approximation on the device, flushing subnormals: a diagonal entry below
// the FP32 normal range gives infinity).
__host__ __device__ __forceinline__ float est_rcp(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return 1.0f / x;
#endif
}

// A second conditioning estimate, for the cells the spread misses (it only
// bounds the conditioning from below, and nearly dependent columns can leave
// every column-scaled diagonal entry moderate): the LINPACK estimate of
// ||R_B^-1|| for the column-scaled factor R_B = D^(1/2) U diag(1/sqrt(n_k))
// of W A S (Cline, Moler, Stewart and Wilkinson 1979): solve R_B^T z = e
// with e_k = +-1 chosen as the solve goes to make |z_k| grow, then
// R_B w = z, and take ||w|| / ||z|| (max norms), a lower bound on
// ||R_B^-1|| that in practice lies within a small factor of it.  With
// y_k = sqrt(d_k) z_k the first solve is y_k = e_k sqrt(n_k) -
// sum_{i<k} u_ik y_i; with w = sqrt(n) v the second is the unit-triangular
// U v = D^(-1/2) z = D^(-1) y: neither divides by U.  The squares
// z_k^2 = y_k^2 / d_k and w_k^2 = v_k^2 n_k need no square root of d or w,
// so this returns max w_k^2 and max z_k^2 (the estimate is the square root
// of their quotient).  An estimate only decides a routing threshold, so it
// runs in FP32 for either factor precision (a diagonal entry below the FP32
// range gives an infinite w: near singular).
template <typename T, int M>
__host__ __device__ __forceinline__ void sqrt_free_inverse_estimate_sq(const SqrtFreeQR<T, M>& f, const T (&nrm)[M],
                                                                       float* w2max_out, float* z2max_out) {
  float y[M], rdd[M];
  float z2max = 0.0f;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    float sk = 0.0f;
#pragma unroll
    for (int i = 0; i < k; ++i) sk = std::fma(static_cast<float>(f.U[i][k]), y[i], sk);
    const float nf = static_cast<float>(nrm[k]);
    rdd[k] = est_rcp(static_cast<float>(f.d[k]));        // 1 / d_k
    const float mag = nf * est_rsqrt(nf) + std::fabs(sk);  // sqrt(n_k) + |s_k|
    y[k] = sk > 0.0f ? -mag : mag;
    const float z2 = mag * mag * rdd[k];
    z2max = z2 > z2max ? z2 : z2max;
  }
  float v[M];
  float w2max = 0.0f;
#pragma unroll
  for (int k = M - 1; k >= 0; --k) {
    float t = y[k] * rdd[k];
#pragma unroll
    for (int c = k + 1; c < M; ++c) t = std::fma(-static_cast<float>(f.U[k][c]), v[c], t);
    v[k] = t;
    const float w2 = t * t * static_cast<float>(nrm[k]);
    w2max = w2 > w2max ? w2 : w2max;
  }
  *w2max_out = w2max;
  *z2max_out = z2max;
}

// The estimate itself (infinity where it is not a number).
template <typename T, int M>
__host__ __device__ __forceinline__ float sqrt_free_inverse_estimate(const SqrtFreeQR<T, M>& f) {
  T nrm[M];
  sqrt_free_colnorms(f, nrm);
  float w2, z2;
  sqrt_free_inverse_estimate_sq(f, nrm, &w2, &z2);
  const float e2 = w2 / z2;
  return e2 == e2 ? std::sqrt(e2) : INFINITY;
}

// Whether the estimate exceeds the bound K (or is not a number, or the
// second solve overflowed).
__host__ __device__ __forceinline__ bool inverse_estimate_exceeds(float w2max, float z2max, float K) {
  return !(w2max <= K * K * z2max) || !(w2max <= 3.0e38f);
}

// Packed position of U[k][j] (k < j < M) in a strict upper triangle.
__host__ __device__ constexpr int strict_upper_index(int M, int k, int j) {
  return k * M - k * (k + 1) / 2 + (j - k - 1);
}

// U d = u_{:,m} by back substitution (unit diagonal).
template <typename T, int M>
__device__ __forceinline__ void sqrt_free_solve(const SqrtFreeQR<T, M>& f, T (&x)[M]) {
#pragma unroll
  for (int k = M - 1; k >= 0; --k) {
    T t = f.U[k][M];
#pragma unroll
    for (int c = k + 1; c < M; ++c) t = fma(-f.U[k][c], x[c], t);
    x[k] = t;
  }
}

template <typename T>
__device__ __forceinline__ const T* tpc_points(const DeviceMesh& dm);
template <>
__device__ __forceinline__ const float* tpc_points<float>(const DeviceMesh& dm) { return dm.fpts32; }
template <>
__device__ __forceinline__ const double* tpc_points<double>(const DeviceMesh& dm) { return dm.fpts; }

// Weights (Sec. 3.1.2) of cell i: eps h^2 and the centre weight.
template <typename T, int DIM>
__device__ __forceinline__ void tpc_weights(const DeviceMesh& dm, const SchemeParams& sp,
                                            const double* WLSENO_BODY_RESTRICT ubar, int64_t i, double ui,
                                            T* eh2, T* w_centre) {
  constexpr int NF = DIM + 1;
  const double hi = dm.h[i];
  const T e = static_cast<T>(sp.eps * hi * hi);
  T bmin = T(INFINITY);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[i * NF + f];
    if (nb >= 0) {
      const T d = static_cast<T>(ubar[nb >> 2] - ui);
      bmin = fmin(bmin, d * d + e);
    }
  }
  *eh2 = e;
  *w_centre = static_cast<T>(sp.alpha_c) * e / bmin;
}

// The same weights in FP32-bulk from the FP32 pairs of ubar, eps h_i^2 and
// alpha rounded to FP32 on the host (no FP64 instruction).  The pairs of
// cell j sit at upair[j * C] (C > 1: the pairs of all components
// interleaved, upair pointing at this thread's component).
template <int DIM, int C = 1>
__device__ __forceinline__ void tpc_weights_pair(const DeviceMesh& dm, const SchemeParams& sp,
                                                 const float2* WLSENO_BODY_RESTRICT upair, int64_t i, float2 pi,
                                                 float* eh2, float* w_centre) {
  constexpr int NF = DIM + 1;
  // eps h_i^2 rounded to FP32 on the host (no FP64 arithmetic here)
  const float e = dm.hscale32 ? dm.hscale32[i].x : static_cast<float>(sp.eps * dm.h[i] * dm.h[i]);
  float bmin = INFINITY;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[i * NF + f];
    if (nb >= 0) {
      const float2 pj = upair[static_cast<int64_t>(nb >> 2) * C];
      const float d = (pj.x - pi.x) + (pj.y - pi.y);
      bmin = fminf(bmin, d * d + e);
    }
  }
  *eh2 = e;
  *w_centre = sp.alpha_c32 * e / bmin;
}

}  // namespace wlseno
