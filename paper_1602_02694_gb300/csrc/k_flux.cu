// Lax-Friedrichs facet flux (Sec. 1, Eq. (flux)), finite-volume residual
// (Sec. 1, Eq. (fvm), divided by |tau_i|) and one TVD-RK3 stage
// (Sec. 4.2.1, Eq. (3rd-order-Runge-Kutta)), fused in one thread-per-cell
// kernel, plus the CFL time step.
//
// Each cell gathers the facet values of its d+1 facets from itself and from
// its facet neighbours and computes every facet flux in the orientation of the
// facet's lower-indexed cell with that cell's normal and area (stored
// identically in both cells' facet records).  Both cells therefore compute the
// bitwise-same flux and use it with opposite signs: no atomics, a fixed
// summation order, and exact discrete conservation up to the final sums.
// Variants: FP64 facet values (FP64 mode, and FP32-bulk with lane-group
// shapes); FP32 facet deviations with FP64 sums (FP32-bulk without the
// state's FP32 pairs); FP32 deviations with double-float sums and stage
// (the FP32-bulk thread-per-cell path, dfloat.cuh).
#include <cmath>
#include <type_traits>

#include "dfloat.cuh"
#include "k_flux_cell.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

template <typename T, int DIM>
__global__ void __launch_bounds__(256)
flux_stage_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ fvals,
                  const double* __restrict__ u, const double* __restrict__ u0, double a, double b,
                  const double* __restrict__ dt_mesh, int residual_only, double* __restrict__ out,
                  unsigned long long* __restrict__ counters) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  flux_cell<T, DIM>(dm, sp, fvals, u, u0, a, b, dt_mesh, residual_only, out, counters, i);
}

template <int DIM>
__global__ void __launch_bounds__(256)
flux_stage_dev_kernel(DeviceMesh dm, SchemeParams sp, const float* __restrict__ fdev,
                      const double* __restrict__ u, const double* __restrict__ u0, double a, double b,
                      const double* __restrict__ dt_mesh, int residual_only, double* __restrict__ out,
                      unsigned long long* __restrict__ counters, const float2* __restrict__ pin,
                      float2* __restrict__ pout) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  flux_dev_cell<DIM>(dm, sp, fdev, u, u0, a, b, dt_mesh, residual_only, out, counters, pin, pout, i);
}

template <int DIM>
__global__ void __launch_bounds__(256)
flux_stage_df_kernel(DeviceMesh dm, int pde, float speed, const float* __restrict__ fdev,
                     const float2* __restrict__ pin, const float2* __restrict__ p0, dfloat a, dfloat b,
                     const float2* __restrict__ dt2, int residual_only, double* __restrict__ out,
                     unsigned long long* __restrict__ counters, float2* __restrict__ pout) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  flux_df_cell<DIM>(dm, pde, speed, fdev, pin, p0, a, b, dt2, residual_only, out, counters, pout, i);
}

__global__ void split_pairs_kernel(const double* __restrict__ u, float2* __restrict__ pair, int64_t n) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= n) return;
  const dfloat d = df_from_double_bits(u[k]);
  pair[k] = make_float2(d.hi, d.lo);
}

// Largest |ubar| per mesh (and the state's FP32 pairs in the same pass).
__global__ void __launch_bounds__(256)
max_abs_kernel(int64_t N, const double* __restrict__ u, const int32_t* __restrict__ mesh_of,
               unsigned long long* __restrict__ lmax_bits, float2* __restrict__ pairs) {
  chunked_mesh_max(N, mesh_of, lmax_bits, [&](int64_t i) {
    const double v = u[i];
    if (pairs) {
      const dfloat d = df_from_double_bits(v);
      pairs[i] = make_float2(d.hi, d.lo);
    }
    // |v| by clearing the sign bit (no FP64 instruction)
    return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
  });
}

__global__ void cfl_dt_kernel(int n_meshes, int pde, int dim, double adv_speed,
                              const unsigned long long* __restrict__ lmax_bits,
                              const double* __restrict__ rmin, double cfl, double dt_fixed,
                              double* __restrict__ dt_mesh, float2* __restrict__ dt2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_meshes) return;
  const double dt = cfl_dt_of(pde, dim, adv_speed, lmax_bits[k], rmin[k], cfl, dt_fixed);
  dt_mesh[k] = dt;
  if (dt2) {
    const dfloat v = df_from_double(dt);
    dt2[k] = make_float2(v.hi, v.lo);
  }
}

}  // namespace

cudaError_t launch_flux_stage_impl(const DeviceMesh& dm, const SchemeParams& sp, int precision,
                                   const double* fvals, const float* fdev, const double* u,
                                   const double* u0, double a, double b, const double* dt_mesh,
                                   bool residual_only, double* out, unsigned long long* counters,
                                   cudaStream_t s, const float2* pin, float2* pout, const float2* p0,
                                   const float2* dt2) {
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((dm.N + threads - 1) / threads);
  const int ro = residual_only ? 1 : 0;
  const bool df = fdev && pin && dm.ff32 && dm.inv_vol2 && (residual_only || dt2) &&
                  (residual_only || a == 0.0 || p0);
  double speed = 0.0;
  for (int k = 0; k < dm.dim; ++k) speed += sp.vel[k] * sp.vel[k];
  const float speedf = static_cast<float>(std::sqrt(speed));
  auto launch = [&](auto D) {
    constexpr int DD = decltype(D)::value;
    if (df)
      flux_stage_df_kernel<DD><<<blocks, threads, 0, s>>>(dm, sp.pde, speedf, fdev, pin, p0,
                                                          df_from_double(a), df_from_double(b), dt2, ro,
                                                          out, counters, residual_only ? nullptr : pout);
    else if (fdev)
      flux_stage_dev_kernel<DD><<<blocks, threads, 0, s>>>(dm, sp, fdev, u, u0, a, b, dt_mesh, ro, out, counters,
                                                           pin, residual_only ? nullptr : pout);
    else if (precision == WLSENO_FP32_BULK)
      flux_stage_kernel<float, DD><<<blocks, threads, 0, s>>>(dm, sp, fvals, u, u0, a, b, dt_mesh, ro, out, counters);
    else
      flux_stage_kernel<double, DD><<<blocks, threads, 0, s>>>(dm, sp, fvals, u, u0, a, b, dt_mesh, ro, out, counters);
  };
  if (dm.dim == 1)
    launch(std::integral_constant<int, 1>{});
  else if (dm.dim == 2)
    launch(std::integral_constant<int, 2>{});
  else
    launch(std::integral_constant<int, 3>{});
  return cudaGetLastError();
}

cudaError_t launch_split_pairs(const double* u, float2* pair, int64_t n, cudaStream_t s) {
  const int threads = 256;
  split_pairs_kernel<<<static_cast<unsigned>((n + threads - 1) / threads), threads, 0, s>>>(u, pair, n);
  return cudaGetLastError();
}

cudaError_t launch_cfl_dt_impl(const DeviceMesh& dm, const SchemeParams& sp, int n_meshes,
                               const double* u, const double* rmin, double cfl, double dt_fixed,
                               unsigned long long* lmax_bits, double* dt_mesh, cudaStream_t s,
                               int* launches, float2* dt2, float2* pairs_out) {
  double speed = 0.0;
  for (int a = 0; a < dm.dim; ++a) speed += sp.vel[a] * sp.vel[a];
  speed = std::sqrt(speed);
  *launches = 0;
  if (dt_fixed <= 0.0 && sp.pde == WLSENO_BURGERS) {
    cudaError_t e = cudaMemsetAsync(lmax_bits, 0, sizeof(unsigned long long) * n_meshes, s);
    if (e != cudaSuccess) return e;
    max_abs_kernel<<<chunked_blocks(dm.N), 256, 0, s>>>(dm.N, u, dm.mesh_of, lmax_bits, pairs_out);
    ++*launches;
    pairs_out = nullptr;  // made
  } else if (dt_fixed <= 0.0 && sp.pde == WLSENO_EULER && pairs_out && dm.dim == 2) {
    // FP32-bulk 2-D Euler: the wave speeds from the pairs it writes
    cudaError_t e = launch_euler2_speed_pairs32(dm, sp.gamma, u, lmax_bits, n_meshes, pairs_out, s);
    if (e != cudaSuccess) return e;
    ++*launches;
    pairs_out = nullptr;  // made
  } else if (dt_fixed <= 0.0 && sp.pde == WLSENO_EULER) {
    cudaError_t e = launch_euler_speed(dm, sp.gamma, u, lmax_bits, n_meshes, s);
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  if (pairs_out && sp.pde == WLSENO_EULER) {  // 2-D Euler FP32-bulk: interleaved [N][4]
    cudaError_t e = launch_euler2_split_pairs(u, pairs_out, dm.N, s);
    if (e != cudaSuccess) return e;
    ++*launches;
  } else if (pairs_out) {  // no wave-speed pass to carry them
    const int threads = 256;
    split_pairs_kernel<<<static_cast<unsigned>((dm.N + threads - 1) / threads), threads, 0, s>>>(u, pairs_out,
                                                                                               dm.N);
    ++*launches;
  }
  cfl_dt_kernel<<<(n_meshes + 127) / 128, 128, 0, s>>>(n_meshes, sp.pde, dm.dim, speed, lmax_bits,
                                                        rmin, cfl, dt_fixed, dt_mesh, dt2);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace wlseno
