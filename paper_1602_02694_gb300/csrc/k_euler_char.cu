// Characteristic-wise WLS-ENO reconstruction for the Euler equations in 1-D
// and 2-D: the characteristic decomposition the paper applies to its Euler
// runs (Sec. 5.1.4, Sec. 5.2.4), in the per-facet form for segments and
// triangles.
//
// One thread per (cell i, facet f).  At the mean U* of the averages of i and
// of its neighbour across f, the Jacobian of F(U).n_f has the eigenvalues
// u.n - c, u.n, u.n, u.n + c with right eigenvectors R (columns)
//   (1, u - c n_x, v - c n_y, H - c u.n), (1, u, v, |u|^2/2),
//   (0, -n_y, n_x, -u n_y + v n_x),       (1, u + c n_x, v + c n_y, H + c u.n)
// and L = R^-1 in closed form (b1 = (gamma-1)/c^2, b2 = b1 |u|^2/2):
//   ((b2 + u.n/c)/2, (-b1 u - n_x/c)/2, (-b1 v - n_y/c)/2, b1/2),
//   (1 - b2, b1 u, b1 v, -b1), (-(-u n_y + v n_x), -n_y, n_x, 0),
//   ((b2 - u.n/c)/2, (-b1 u + n_x/c)/2, (-b1 v + n_y/c)/2, b1/2).
// The stencil deviations ubar_k - ubar_i are projected with L, each of the
// four characteristic fields gets its own WLS-ENO weights (Sec. 3.1.2) and
// least-squares solve (the square-root-free factor of k_recon_tpc.cuh, full
// rank), is evaluated at facet f's two Gauss points and projected back with
// R: u(x_q) = ubar_i + R dw(x_q).  The eigenvector set for -n is that for n
// up to order and sign, which leave each field's reconstruction unchanged, so
// both cells of a facet use the facet's stored (lower-indexed cell's) normal.
// In 1-D (n = +-1) the shear wave is absent: R has the columns
//   (1, u - c n, H - c u n), (1, u, u^2/2), (1, u + c n, H + c u n)
// and L the first, second and fourth rows above without their v entries.
// Output: facet values [d+2][N][(d+1)*nq], the layout of the componentwise
// path.
#include <cmath>
#include <type_traits>

#include "euler_basis.cuh"
#include "k_recon_tpc.cuh"
#include "monomials.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

template <typename T>
__device__ __forceinline__ const T* csr_moments(const DeviceMesh& dm);
template <>
__device__ __forceinline__ const float* csr_moments<float>(const DeviceMesh& dm) { return dm.A32; }
template <>
__device__ __forceinline__ const double* csr_moments<double>(const DeviceMesh& dm) { return dm.A64; }

template <typename T, int DIM, int M>
__global__ void __launch_bounds__(128)
euler_char_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ ubar,
                  double* __restrict__ fvals, unsigned long long* __restrict__ counters,
                  T flag_threshold) {
  constexpr int NF = DIM + 1, NQ = nq_of(DIM), NP = NF * NQ, C = DIM + 2;
  const int64_t N = dm.N;
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (tid >= N * NF) return;
  const int64_t i = tid / NF;
  const int f = static_cast<int>(tid % NF);
  const double gamma = sp.gamma;
  double ui[C], us[C];
  const int nb = dm.nbr[i * NF + f];
  const int64_t jf = nb >= 0 ? (nb >> 2) : i;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    ui[c] = ubar[c * N + i];
    us[c] = 0.5 * (ui[c] + ubar[c * N + jf]);
  }
  // eigenvectors at U* in the direction of the facet's stored normal
  const double* g = dm.fgeo + (i * NF + f) * 4;
  double Ld[C][C], Rd[C][C];
  char_basis<DIM>(us, g, gamma, Ld, Rd);
  T Lt[C][C];
#pragma unroll
  for (int a = 0; a < C; ++a)
#pragma unroll
    for (int b = 0; b < C; ++b) Lt[a][b] = static_cast<T>(Ld[a][b]);
  const int beg = dm.st_ptr[i];
  const int n = dm.st_ptr[i + 1] - beg;
  const double hi = dm.h[i];
  const T eh2 = static_cast<T>(sp.eps * hi * hi);
  const T* A = csr_moments<T>(dm);
  // monomials at facet f's points
  T mono[NQ][M];
  const T* P = tpc_points<T>(dm) + (i * NP + f * NQ) * DIM;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T y[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) y[a] = P[q * DIM + a];
    eval_monomials<T, DIM, M>(y, mono[q]);
  }
  T dw[NQ][C];
  bool flagged = false;
#pragma unroll 1
  for (int cf = 0; cf < C; ++cf) {
    // centre weight: the smallest beta of this field over the facet neighbours
    T bmin = T(INFINITY);
#pragma unroll
    for (int ff = 0; ff < NF; ++ff) {
      const int nb2 = dm.nbr[i * NF + ff];
      if (nb2 >= 0) {
        const int64_t k = nb2 >> 2;
        T d = T(0);
#pragma unroll
        for (int c = 0; c < C; ++c) d += Lt[cf][c] * static_cast<T>(ubar[c * N + k] - ui[c]);
        bmin = fmin(bmin, d * d + eh2);
      }
    }
    const T wc = static_cast<T>(sp.alpha_c) * eh2 / bmin;
    SqrtFreeQR<T, M> fq;
    sqrt_free_init(fq);
    for (int t = 0; t < n; ++t) {
      const int64_t k = dm.st_idx[beg + t];
      T dev = T(0);
#pragma unroll
      for (int c = 0; c < C; ++c) dev += Lt[cf][c] * static_cast<T>(ubar[c * N + k] - ui[c]);
      T z[M + 1];
      const T* a = A + static_cast<int64_t>(beg + t) * M;
#pragma unroll
      for (int m = 0; m < M; ++m) z[m] = a[m];
      z[M] = dev;
      const T w = t == 0 ? wc : eh2 * recip_t<T>(dev * dev + eh2);
      sqrt_free_fold(fq, z, w * w);
    }
    T qmax, qmin;
    sqrt_free_spread(fq, &qmax, &qmin);
    flagged = flagged || !(qmax <= flag_threshold * flag_threshold * qmin);
    T x[M];
    sqrt_free_solve(fq, x);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < M; ++m) s += x[m] * mono[q][m];
      dw[q][cf] = s;
    }
  }
  // back to the conserved variables
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T s = T(0);
#pragma unroll
      for (int cf = 0; cf < C; ++cf) s += static_cast<T>(Rd[c][cf]) * dw[q][cf];
      fvals[(c * N + i) * NP + f * NQ + q] = ui[c] + static_cast<double>(s);
    }
  if (flagged) atomicAdd(&counters[0], 1ull);
}

}  // namespace

cudaError_t launch_euler_char(const DeviceMesh& dm, const SchemeParams& sp, int precision,
                              const double* ubar, double* fvals, unsigned long long* counters,
                              cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = static_cast<unsigned>((dm.N * (dm.dim + 1) + threads - 1) / threads);
  const bool f32 = precision == WLSENO_FP32_BULK;
  const double flag = f32 ? sp.kappa_flag : 1e6;
  auto launch = [&](auto D, auto Mc) {
    constexpr int DD = decltype(D)::value, MM = decltype(Mc)::value;
    if (f32)
      euler_char_kernel<float, DD, MM><<<blocks, threads, 0, s>>>(dm, sp, ubar, fvals, counters,
                                                                  static_cast<float>(flag));
    else
      euler_char_kernel<double, DD, MM><<<blocks, threads, 0, s>>>(dm, sp, ubar, fvals, counters, flag);
  };
  using std::integral_constant;
  if (dm.dim == 1 && dm.m == 3) launch(integral_constant<int, 1>{}, integral_constant<int, 3>{});
  else if (dm.dim == 1 && dm.m == 5) launch(integral_constant<int, 1>{}, integral_constant<int, 5>{});
  else if (dm.dim == 2 && dm.m == 6) launch(integral_constant<int, 2>{}, integral_constant<int, 6>{});
  else if (dm.dim == 2 && dm.m == 10) launch(integral_constant<int, 2>{}, integral_constant<int, 10>{});
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace wlseno
