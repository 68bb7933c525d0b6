// Characteristic-wise WLS-ENO reconstruction for the 2-D Euler equations:
// the characteristic decomposition the paper applies to its Euler runs
// (Sec. 5.1.4, Sec. 5.2.4), in the per-facet form for triangles.
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
// Output: facet values [4][N][3*2], the layout of the componentwise path.
#include <cmath>

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

template <typename T, int M>
__global__ void __launch_bounds__(128)
euler_char_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ ubar,
                  double* __restrict__ fvals, unsigned long long* __restrict__ counters,
                  T flag_threshold) {
  constexpr int DIM = 2, NF = 3, NQ = 2, NP = NF * NQ, C = 4;
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
  const double nx = g[0], ny = g[1];
  const double rho = us[0], u = us[1] / rho, v = us[2] / rho;
  const double ke = 0.5 * (u * u + v * v);
  const double p = (gamma - 1.0) * (us[3] - rho * ke);
  const double cs = sqrt(gamma * p / rho);
  const double H = (us[3] + p) / rho;
  const double un = u * nx + v * ny, ut = -u * ny + v * nx;
  const double b1 = (gamma - 1.0) / (cs * cs), b2 = ke * b1;
  const double Ld[C][C] = {{0.5 * (b2 + un / cs), 0.5 * (-b1 * u - nx / cs), 0.5 * (-b1 * v - ny / cs), 0.5 * b1},
                           {1.0 - b2, b1 * u, b1 * v, -b1},
                           {-ut, -ny, nx, 0.0},
                           {0.5 * (b2 - un / cs), 0.5 * (-b1 * u + nx / cs), 0.5 * (-b1 * v + ny / cs), 0.5 * b1}};
  const double Rd[C][C] = {{1.0, 1.0, 0.0, 1.0},
                           {u - cs * nx, u, -ny, u + cs * nx},
                           {v - cs * ny, v, nx, v + cs * ny},
                           {H - cs * un, ke, ut, H + cs * un}};
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
    const T y[DIM] = {P[q * DIM], P[q * DIM + 1]};
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
  if (dm.dim != 2 || (dm.m != 6 && dm.m != 10)) return cudaErrorInvalidValue;
  const int threads = 128;
  const unsigned blocks = static_cast<unsigned>((dm.N * 3 + threads - 1) / threads);
  const bool f32 = precision == WLSENO_FP32_BULK;
  const double flag = f32 ? sp.kappa_flag : 1e6;
  if (dm.m == 6) {
    if (f32)
      euler_char_kernel<float, 6><<<blocks, threads, 0, s>>>(dm, sp, ubar, fvals, counters, static_cast<float>(flag));
    else
      euler_char_kernel<double, 6><<<blocks, threads, 0, s>>>(dm, sp, ubar, fvals, counters, flag);
  } else {
    if (f32)
      euler_char_kernel<float, 10><<<blocks, threads, 0, s>>>(dm, sp, ubar, fvals, counters, static_cast<float>(flag));
    else
      euler_char_kernel<double, 10><<<blocks, threads, 0, s>>>(dm, sp, ubar, fvals, counters, flag);
  }
  return cudaGetLastError();
}

}  // namespace wlseno
