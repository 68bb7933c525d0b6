// WLS-ENO reconstruction, one thread per cell (Sec. 3.1.2, Sec. 3.2,
// Sec. 3.3.2).
//
// The thread streams its stencil rows a_j = w_j [A_j | ubar_j - ubar_i] from
// an ELL layout (row t of every cell contiguous across cells, so a warp's
// loads are coalesced) and folds each into an m x m upper-triangular factor R
// (plus the transformed right-hand side) with Givens rotations: W A = Q R.
// Column norms of W A equal those of R, so S = diag(1/||col R||) and the
// paper's QR with column pivoting of W A S is the pivoted QR of the small
// R S: W A S E = Q (R S E) = Q Q2 R2.  The pivots, R2 and hence the numerical
// rank and the basic solution are those of W A S E = Q R (Sec. 3.3.2); only
// the order of the orthogonal transformations differs.  Everything lives in
// registers: no shuffles, no shared memory.
//
// FP32-bulk: the weights, W A, the factorisations and the polynomial run in
// FP32; ubar_j - ubar_i and ubar_i + deviation in FP64.  Cells whose
// |R2_00| / |R2_rr| exceeds kappa_flag are appended to a work list; a second
// kernel recomputes them and applies one corrected-seminormal-equations
// refinement, y += (R2^T R2)^-1 (B E)^T (b - B y), with the residual and
// B^T r formed in FP64 from the FP64 weights and moments.
#pragma once

#include <cmath>
#include <utility>

#include "monomials.cuh"
#include "wlseno_internal.h"

namespace wlseno {

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void cswap(bool c, T& a, T& b) {
  const T ta = a;
  a = c ? b : a;
  b = c ? ta : b;
}

// Fold row a (a[M] = right-hand side) into the triangular factor R.
template <typename T, int M>
__device__ __forceinline__ void givens_fold(T (&R)[M][M + 1], T (&a)[M + 1]) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const T rkk = R[k][k];
    const T ak = a[k];
    const T t2 = rkk * rkk + ak * ak;
    const bool nz = t2 > T(0);
    const T inv = nz ? rsqrt_t<T>(t2) : T(0);
    const T c = nz ? rkk * inv : T(1);
    const T s = ak * inv;
    R[k][k] = t2 * inv;
#pragma unroll
    for (int j = k + 1; j <= M; ++j) {
      const T rj = R[k][j];
      const T aj = a[j];
      R[k][j] = c * rj + s * aj;
      a[j] = c * aj - s * rj;
    }
  }
}

// Pivoted QR of the small scaled factor and its solve.
template <typename T, int M>
struct SmallQR {
  T F[M][M];     // R S E after pivoting; R2 in its upper triangle at the end
  T z[M];        // (Q Q2)^T W (ubar_S - ubar_i), first M entries
  T s[M];        // S in pivoted order
  int col[M];    // original column of pivoted position k
  T y[M];        // solution in pivoted order (S-scaled unknowns)
  T r00, rlast;
  int rank;
};

template <int K, typename T, int M>
__device__ __forceinline__ void small_qr_step(SmallQR<T, M>& q, T tau_piv, T rank_tol) {
  T pn[M];
#pragma unroll
  for (int c = K; c < M; ++c) {
    T acc = T(0);
#pragma unroll
    for (int k = K; k < M; ++k) acc += q.F[k][c] * q.F[k][c];
    pn[c] = acc;
  }
  T mx = T(0);
#pragma unroll
  for (int c = K; c < M; ++c) mx = pn[c] > mx ? pn[c] : mx;
  int p = K;
  T sigma = pn[K];
#pragma unroll
  for (int c = M - 1; c >= K; --c)
    if (pn[c] >= (T(1) - tau_piv) * mx) {
      p = c;
      sigma = pn[c];
    }
#pragma unroll
  for (int c = K + 1; c < M; ++c) {
    const bool sw = c == p;
#pragma unroll
    for (int k = 0; k < M; ++k) cswap(sw, q.F[k][K], q.F[k][c]);
    cswap(sw, q.s[K], q.s[c]);
    cswap(sw, q.col[K], q.col[c]);
  }
  const T xk = q.F[K][K];
  const T nrm = sqrt(sigma);
  const T alpha = xk >= T(0) ? -nrm : nrm;
  const T vtv = T(2) * (sigma + fabs(xk) * nrm);
  const T tau = vtv > T(0) ? T(2) / vtv : T(0);
  T v[M];
#pragma unroll
  for (int k = K; k < M; ++k) v[k] = k == K ? xk - alpha : q.F[k][K];
#pragma unroll
  for (int c = K + 1; c < M; ++c) {
    T d = T(0);
#pragma unroll
    for (int k = K; k < M; ++k) d += v[k] * q.F[k][c];
    d *= tau;
#pragma unroll
    for (int k = K; k < M; ++k) q.F[k][c] -= d * v[k];
  }
  {
    T d = T(0);
#pragma unroll
    for (int k = K; k < M; ++k) d += v[k] * q.z[k];
    d *= tau;
#pragma unroll
    for (int k = K; k < M; ++k) q.z[k] -= d * v[k];
  }
  q.F[K][K] = alpha;
  if (K == 0) q.r00 = fabs(alpha);
  if (q.rank == M && !(fabs(alpha) > rank_tol * q.r00)) q.rank = K;
}

template <int K, typename T, int M>
__device__ __forceinline__ void small_backsub_step(SmallQR<T, M>& q) {
  T t = q.z[K];
#pragma unroll
  for (int c = K + 1; c < M; ++c) t -= q.F[K][c] * q.y[c];
  const T rkk = q.F[K][K];
  q.y[K] = (K < q.rank && rkk != T(0)) ? t / rkk : T(0);
  if (K == q.rank - 1) q.rlast = fabs(rkk);
}

template <typename T, int M, int... Ks>
__device__ __forceinline__ void small_qr_solve(SmallQR<T, M>& q, T tau_piv, T rank_tol,
                                               std::integer_sequence<int, Ks...>) {
  (small_qr_step<Ks, T, M>(q, tau_piv, rank_tol), ...);
  (small_backsub_step<M - 1 - Ks, T, M>(q), ...);
}

// ELL moments of the FP64 kernel (the FP32 kernel reads row records).
template <typename T>
__device__ __forceinline__ const T* ell_moments(const DeviceMesh& dm) { return dm.A64e; }

template <typename T>
__device__ __forceinline__ const T* tpc_points(const DeviceMesh& dm);
template <>
__device__ __forceinline__ const float* tpc_points<float>(const DeviceMesh& dm) { return dm.fpts32; }
template <>
__device__ __forceinline__ const double* tpc_points<double>(const DeviceMesh& dm) { return dm.fpts; }

// Weights (Sec. 3.1.2) of cell i: eps h^2 and the centre weight.
template <typename T, int DIM>
__device__ __forceinline__ void tpc_weights(const DeviceMesh& dm, const SchemeParams& sp,
                                            const double* __restrict__ ubar, int64_t i, double ui,
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

}  // namespace wlseno
