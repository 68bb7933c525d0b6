// Compressible Euler in 2-D (conserved rho, rho u, rho v, E; gamma-law gas),
// componentwise WLS-ENO: the reconstruction kernels run once per component
// (each with its own weights, Sec. 3.1.2), then
//  * a positivity fix-up: a cell whose traces give density or pressure
//    <= 1e-12 at any facet quadrature point uses its cell averages at all its
//    facets (reading: the paper is silent; counted in counters[3]);
//  * the flux/RK-stage kernel: Lax-Friedrichs flux per facet (Sec. 1,
//    Eq. (flux)) with alpha = max over the facet's points and both sides of
//    |u.n| + c, in the lower-indexed cell's orientation (bitwise-equal in both
//    cells, so conservation is exact), FP64 accumulation of the residual and
//    the Shu-Osher combine for all four components;
//  * the largest |u| + c per mesh for the CFL step.
#include <cmath>
#include <type_traits>

#include "k_flux_cell.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

constexpr double kFloor = 1e-12;

template <int DIM>
__global__ void __launch_bounds__(256)
euler_positivity_kernel(int64_t N, double gamma, const double* __restrict__ ubar,
                        double* __restrict__ fvals, unsigned long long* __restrict__ counters) {
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  constexpr int C = DIM + 2;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  bool ok = true;
  for (int p = 0; p < NP; ++p) {
    double U[C];
    for (int c = 0; c < C; ++c) U[c] = fvals[(c * N + i) * NP + p];
    double ke = 0.0;
    for (int a = 0; a < DIM; ++a) ke += U[1 + a] * U[1 + a];
    const double rho = U[0];
    const double pr = (gamma - 1.0) * (U[C - 1] - 0.5 * ke / rho);
    ok = ok && rho > kFloor && pr > kFloor;
  }
  if (!ok) {
    for (int c = 0; c < C; ++c)
      for (int p = 0; p < NP; ++p) fvals[(c * N + i) * NP + p] = ubar[c * N + i];
    atomicAdd(&counters[3], 1ull);
  }
}

// F(U).n and the wave speed |u.n| + c of one state.
template <typename T, int DIM>
__device__ __forceinline__ void euler_state(const T (&U)[DIM + 2], const T (&n)[DIM], T gamma,
                                            T (&F)[DIM + 2], T* speed) {
  constexpr int C = DIM + 2;
  const T rho = U[0];
  const T inv = T(1) / rho;
  T un = T(0), ke = T(0);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    un += U[1 + a] * n[a];
    ke += U[1 + a] * U[1 + a];
  }
  un *= inv;
  const T p = (gamma - T(1)) * (U[C - 1] - T(0.5) * ke * inv);
  F[0] = rho * un;
#pragma unroll
  for (int a = 0; a < DIM; ++a) F[1 + a] = U[1 + a] * un + p * n[a];
  F[C - 1] = (U[C - 1] + p) * un;
  const T c2 = gamma * p * inv;
  *speed = fabs(un) + sqrt(c2 > T(0) ? c2 : T(0));
}

template <typename T, int DIM>
__global__ void __launch_bounds__(128)
euler_flux_stage_kernel(DeviceMesh dm, double gamma, const double* __restrict__ fvals,
                        const double* __restrict__ u, const double* __restrict__ u0, double a,
                        double b, const double* __restrict__ dt_mesh, int residual_only,
                        double* __restrict__ out, unsigned long long* __restrict__ counters) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
  constexpr int C = DIM + 2;
  const int64_t N = dm.N;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  const T g = static_cast<T>(gamma);
  const T wq = T(1) / T(NQ);
  double acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[i * NF + f];
    bool owner = true;
    int64_t j = i;
    int f2 = f;
    if (nb >= 0) {
      j = nb >> 2;
      f2 = nb & 3;
      owner = i < j;
    }
    const double* geo = dm.fgeo + (i * NF + f) * 4;
    T n[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) n[d] = static_cast<T>(geo[d]);
    T FL[NQ][C], FR[NQ][C], UL[NQ][C], UR[NQ][C];
    T alpha = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T Uo[C], Un[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        Uo[c] = static_cast<T>(fvals[(c * N + i) * NP + f * NQ + q]);
        Un[c] = nb >= 0 ? static_cast<T>(fvals[(c * N + j) * NP + f2 * NQ + q]) : Uo[c];
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        UL[q][c] = owner ? Uo[c] : Un[c];
        UR[q][c] = owner ? Un[c] : Uo[c];
      }
      T sL, sR;
      euler_state<T, DIM>(UL[q], n, g, FL[q], &sL);
      euler_state<T, DIM>(UR[q], n, g, FR[q], &sR);
      alpha = fmax(alpha, fmax(sL, sR));
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T fs = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        fs += wq * (T(0.5) * ((FL[q][c] + FR[q][c]) - alpha * (UR[q][c] - UL[q][c])));
      const double contrib = geo[3] * static_cast<double>(fs);
      acc[c] += owner ? contrib : -contrib;
    }
  }
  const double dt = residual_only ? 0.0 : dt_mesh[dm.mesh_of[i]];
  bool finite = true;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const double L = -acc[c] / dm.volume[i];
    const double res = residual_only ? L : a * u0[c * N + i] + b * (u[c * N + i] + dt * L);
    out[c * N + i] = res;
    finite = finite && isfinite(res);
  }
  if (!finite) report_nonfinite(dm, counters);
}

// Largest |u| + c over each mesh's cells (bits of a non-negative double).
template <int DIM>
__global__ void __launch_bounds__(256)
euler_speed_kernel(int64_t N, double gamma, const double* __restrict__ ubar,
                   const int32_t* __restrict__ mesh_of, unsigned long long* __restrict__ lmax_bits) {
  constexpr int C = DIM + 2;
  chunked_mesh_max(N, mesh_of, lmax_bits, [&](int64_t i) {
    const double rho = ubar[i];
    double ke = 0.0;
    for (int a = 0; a < DIM; ++a) ke += ubar[(1 + a) * N + i] * ubar[(1 + a) * N + i];
    const double p = (gamma - 1.0) * (ubar[(C - 1) * N + i] - 0.5 * ke / rho);
    const double c2 = gamma * p / rho;
    double s = sqrt(ke) / rho + sqrt(c2 > 0.0 ? c2 : 0.0);
    if (!(s >= 0.0)) s = INFINITY;  // a non-finite state stops the step (dt = 0)
    return static_cast<unsigned long long>(__double_as_longlong(s));
  });
}

}  // namespace

cudaError_t launch_euler_positivity(const DeviceMesh& dm, double gamma, const double* ubar,
                                    double* fvals, unsigned long long* counters, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>((dm.N + 255) / 256);
  if (dm.dim == 1)
    euler_positivity_kernel<1><<<blocks, 256, 0, s>>>(dm.N, gamma, ubar, fvals, counters);
  else if (dm.dim == 2)
    euler_positivity_kernel<2><<<blocks, 256, 0, s>>>(dm.N, gamma, ubar, fvals, counters);
  else if (dm.dim == 3)
    euler_positivity_kernel<3><<<blocks, 256, 0, s>>>(dm.N, gamma, ubar, fvals, counters);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_euler_flux_stage(const DeviceMesh& dm, double gamma, int precision,
                                    const double* fvals, const double* u, const double* u0,
                                    double a, double b, const double* dt_mesh, bool residual_only,
                                    double* out, unsigned long long* counters, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>((dm.N + 127) / 128);
  if (dm.dim < 1 || dm.dim > 3) return cudaErrorInvalidValue;
  const int ro = residual_only ? 1 : 0;
  const bool f32 = precision == WLSENO_FP32_BULK;
  auto launch = [&](auto D) {
    constexpr int DD = decltype(D)::value;
    if (f32)
      euler_flux_stage_kernel<float, DD><<<blocks, 128, 0, s>>>(dm, gamma, fvals, u, u0, a, b, dt_mesh, ro, out, counters);
    else
      euler_flux_stage_kernel<double, DD><<<blocks, 128, 0, s>>>(dm, gamma, fvals, u, u0, a, b, dt_mesh, ro, out, counters);
  };
  if (dm.dim == 1) launch(std::integral_constant<int, 1>{});
  else if (dm.dim == 2) launch(std::integral_constant<int, 2>{});
  else launch(std::integral_constant<int, 3>{});
  return cudaGetLastError();
}

cudaError_t launch_euler_speed(const DeviceMesh& dm, double gamma, const double* ubar,
                               unsigned long long* lmax_bits, int n_meshes, cudaStream_t s) {
  if (dm.dim < 1 || dm.dim > 3) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(lmax_bits, 0, sizeof(unsigned long long) * n_meshes, s);
  if (e != cudaSuccess) return e;
  const unsigned blocks = chunked_blocks(dm.N);
  if (dm.dim == 1)
    euler_speed_kernel<1><<<blocks, 256, 0, s>>>(dm.N, gamma, ubar, dm.mesh_of, lmax_bits);
  else if (dm.dim == 2)
    euler_speed_kernel<2><<<blocks, 256, 0, s>>>(dm.N, gamma, ubar, dm.mesh_of, lmax_bits);
  else
    euler_speed_kernel<3><<<blocks, 256, 0, s>>>(dm.N, gamma, ubar, dm.mesh_of, lmax_bits);
  return cudaGetLastError();
}

}  // namespace wlseno
