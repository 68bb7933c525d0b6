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
#include "wlseno_internal.h"

namespace wlseno {
namespace {

// One facet's integrated LF flux in the orientation of its lower-indexed cell
// L (normal nrm and area of L), from the traces uL (of L) and uR at its NQ
// points.  FP64 mode evaluates it directly.  FP32-bulk mode splits it at the
// reference state u_ref = uL[0]: F(u_ref).n in FP64 plus the FP32 flux of the
// deviations u - u_ref, so the FP32 rounding is relative to the (small)
// deviations and a constant state gives an exactly constant flux.
template <typename T, int DIM, int NQ>
__device__ __forceinline__ double facet_flux(const SchemeParams& sp, const double* geo,
                                             const double (&uL)[NQ], const double (&uR)[NQ]) {
  const T wq = T(1) / T(NQ);  // equal-weight rules on every facet
  double n64[DIM];
  double nsum64 = 0.0, vn64 = 0.0, speed2 = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    n64[a] = geo[a];
    nsum64 += n64[a];
    vn64 += sp.vel[a] * n64[a];
    speed2 += sp.vel[a] * sp.vel[a];
  }
  const bool adv = sp.pde == WLSENO_ADVECTION;
  if constexpr (sizeof(T) == 8) {
    double alpha;
    if (adv) {
      alpha = sqrt(speed2);
    } else {
      double mx = 0.0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) mx = fmax(mx, fmax(fabs(uL[q]), fabs(uR[q])));
      alpha = mx * fabs(nsum64);
    }
    double fsum = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double fl, fr;
      if (adv) {
        fl = vn64 * uL[q];
        fr = vn64 * uR[q];
      } else {
        fl = 0.5 * uL[q] * uL[q] * nsum64;
        fr = 0.5 * uR[q] * uR[q] * nsum64;
      }
      fsum += wq * (0.5 * ((fl + fr) - alpha * (uR[q] - uL[q])));
    }
    return geo[3] * fsum;
  } else {
    const double uref = uL[0];
    const float ur = static_cast<float>(uref);
    const float nsum = static_cast<float>(nsum64), vn = static_cast<float>(vn64);
    float dL[NQ], dR[NQ];
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      dL[q] = static_cast<float>(uL[q] - uref);
      dR[q] = static_cast<float>(uR[q] - uref);
      mx = fmaxf(mx, fmaxf(fabsf(ur + dL[q]), fabsf(ur + dR[q])));
    }
    const float alpha = adv ? static_cast<float>(sqrt(speed2)) : mx * fabsf(nsum);
    float fsum = 0.0f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float fl, fr;
      if (adv) {
        fl = vn * dL[q];
        fr = vn * dR[q];
      } else {  // (u^2 - u_ref^2)/2 = d (u_ref + d/2)
        fl = nsum * dL[q] * (ur + 0.5f * dL[q]);
        fr = nsum * dR[q] * (ur + 0.5f * dR[q]);
      }
      fsum += wq * (0.5f * ((fl + fr) - alpha * (dR[q] - dL[q])));
    }
    const double fref = adv ? vn64 * uref : 0.5 * uref * uref * nsum64;
    return geo[3] * (fref + static_cast<double>(fsum));
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256)
flux_stage_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ fvals,
                  const double* __restrict__ u, const double* __restrict__ u0, double a, double b,
                  const double* __restrict__ dt_mesh, int residual_only, double* __restrict__ out,
                  unsigned long long* __restrict__ counters) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  double acc = 0.0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[i * NF + f];
    double uo[NQ], un[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) uo[q] = fvals[i * NP + f * NQ + q];
    bool owner = true;
    if (nb >= 0) {
      const int64_t j = nb >> 2;
      const int f2 = nb & 3;
#pragma unroll
      for (int q = 0; q < NQ; ++q) un[q] = fvals[j * NP + f2 * NQ + q];
      owner = i < j;
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) un[q] = uo[q];
    }
    double uL[NQ], uR[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      uL[q] = owner ? uo[q] : un[q];
      uR[q] = owner ? un[q] : uo[q];
    }
    const double flux = facet_flux<T, DIM, NQ>(sp, dm.fgeo + (i * NF + f) * 4, uL, uR);
    acc += owner ? flux : -flux;
  }
  const double L = -acc / dm.volume[i];
  double res;
  if (residual_only) {
    res = L;
  } else {
    const double dt = dt_mesh[dm.mesh_of[i]];
    res = a * u0[i] + b * (u[i] + dt * L);
  }
  out[i] = res;
  if (!isfinite(res)) atomicAdd(&counters[2], 1ull);
}

// FP32-bulk flux from facet deviations: the facet values arrive as FP32
// deviations from their cell averages, value = ubar_c + dev.  Each facet is
// split at its lower-indexed cell's average u_ref = ubar_L (the same for both
// cells, so both compute the bitwise-same flux; ur = fl32(u_ref)): F(u_ref).n |f| in FP64 from
// the precomputed reference coefficient, plus the FP32 flux of the deviations
// from u_ref, where the other cell's deviations are shifted by the FP32
// rounding of ubar_R - ubar_L.  FP64 work per facet: that subtraction, the
// reference flux and the accumulation.
__device__ __forceinline__ double pref64(const FacetF32& g) {
  return static_cast<double>(g.pref_hi) + static_cast<double>(g.pref_lo);
}

// The FP32 flux of the deviations dL, dR from u_ref (ur = its FP32 value):
// the facet's flux minus F(u_ref).n |f|, before the factor |f|.
template <int NQ>
__device__ __forceinline__ float facet_flux_dev_part(int pde, const FacetF32& g, float speed, float ur,
                                                     const float (&dL)[NQ], const float (&dR)[NQ]) {
  const float wq = 1.0f / NQ;
  float fsum = 0.0f;
  if (pde == WLSENO_ADVECTION) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) fsum += wq * (0.5f * (g.coef * (dL[q] + dR[q]) - speed * (dR[q] - dL[q])));
    return fsum;
  }
  float mx = 0.0f;
#pragma unroll
  for (int q = 0; q < NQ; ++q) mx = fmaxf(mx, fmaxf(fabsf(ur + dL[q]), fabsf(ur + dR[q])));
  const float alpha = mx * fabsf(g.coef);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {  // (u^2 - u_ref^2)/2 = d (u_ref + d/2)
    const float fl = g.coef * dL[q] * (ur + 0.5f * dL[q]);
    const float fr = g.coef * dR[q] * (ur + 0.5f * dR[q]);
    fsum += wq * (0.5f * ((fl + fr) - alpha * (dR[q] - dL[q])));
  }
  return fsum;
}

template <int NQ>
__device__ __forceinline__ double facet_flux_dev(int pde, const FacetF32& g, float speed, double uref,
                                                 float ur, const float (&dL)[NQ], const float (&dR)[NQ]) {
  const float fsum = facet_flux_dev_part<NQ>(pde, g, speed, ur, dL, dR);
  if (pde == WLSENO_ADVECTION) return fma(pref64(g), uref, static_cast<double>(g.area * fsum));
  return fma(pref64(g) * uref, uref, static_cast<double>(g.area * fsum));
}

template <int DIM>
__global__ void __launch_bounds__(256)
flux_stage_dev_kernel(DeviceMesh dm, SchemeParams sp, const float* __restrict__ fdev,
                      const double* __restrict__ u, const double* __restrict__ u0, double a, double b,
                      const double* __restrict__ dt_mesh, int residual_only, double* __restrict__ out,
                      unsigned long long* __restrict__ counters, const float2* __restrict__ pin,
                      float2* __restrict__ pout) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  float speed2 = 0.0f;
#pragma unroll
  for (int q = 0; q < DIM; ++q) speed2 += static_cast<float>(sp.vel[q] * sp.vel[q]);
  const float speed = sqrtf(speed2);
  const double ui = u[i];
  const float2 pi = pin ? pin[i] : make_float2(0.0f, 0.0f);
  double acc = 0.0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[i * NF + f];
    float di[NQ], dj[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) di[q] = fdev[i * NP + f * NQ + q];
    double uj = ui;
    float2 pj = pi;
    bool owner = true;
    if (nb >= 0) {
      const int64_t j = nb >> 2;
      const int f2 = nb & 3;
#pragma unroll
      for (int q = 0; q < NQ; ++q) dj[q] = fdev[j * NP + f2 * NQ + q];
      uj = u[j];
      if (pin) pj = pin[j];
      owner = i < j;
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) dj[q] = di[q];
    }
    const double uL = owner ? ui : uj;
    // ubar_R - ubar_L in FP32: from the pairs when given (no FP64 work)
    const float2 pL = owner ? pi : pj, pR = owner ? pj : pi;
    const float jump = pin ? (pR.x - pL.x) + (pR.y - pL.y) : static_cast<float>((owner ? uj : ui) - uL);
    float dL[NQ], dR[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      dL[q] = owner ? di[q] : dj[q];
      dR[q] = (owner ? dj[q] : di[q]) + jump;
    }
    const double flux = facet_flux_dev<NQ>(sp.pde, dm.ff32[i * NF + f], speed, uL,
                                                pin ? pL.x : static_cast<float>(uL), dL, dR);
    acc += owner ? flux : -flux;
  }
  const double L = -acc * dm.inv_volume[i];
  double res;
  if (residual_only) {
    res = L;
  } else {
    const double dt = dt_mesh[dm.mesh_of[i]];
    res = a * u0[i] + b * (ui + dt * L);
  }
  out[i] = res;
  if (pout) {
    const float hi = __double2float_rn(res);
    pout[i] = make_float2(hi, __double2float_rn(res - static_cast<double>(hi)));
  }
  if (!isfinite(res)) atomicAdd(&counters[2], 1ull);
}

// The same flux, residual and stage with every FP64 operation replaced by
// double-float arithmetic (dfloat.cuh) on the FP32 pairs of the states: per
// facet F(u_ref).n |f| = pref u_ref (u_ref) from the pair of the reference
// coefficient and the pair of u_ref = ubar_L, plus the exact product |f| fsum
// of the FP32 deviation flux; the facet sum, the factor 1/|tau_i| (a pair)
// and a u0 + b (u + dt L) likewise.  Both cells of a facet form its flux from
// the same operands in the same order, so it is bitwise the same in both and
// discrete conservation stays exact up to the final rounding.  FP64 is left
// with forming the pair of dt and the FP64 output (hi + lo, exact).
template <int DIM>
__global__ void __launch_bounds__(256)
flux_stage_df_kernel(DeviceMesh dm, int pde, float speed, const float* __restrict__ fdev,
                     const float2* __restrict__ pin, const float2* __restrict__ p0, dfloat a, dfloat b,
                     const float2* __restrict__ dt2, int residual_only, double* __restrict__ out,
                     unsigned long long* __restrict__ counters, float2* __restrict__ pout) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  // every load up front: the neighbours first (the other loads depend on
  // them), then this cell's data, then the neighbours' (a boundary facet reads
  // this cell's own values and discards them)
  int nb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) nb[f] = dm.nbr[i * NF + f];
  const float2 pi = pin[i];
  float di[NF][NQ];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int q = 0; q < NQ; ++q) di[f][q] = fdev[i * NP + f * NQ + q];
  FacetF32 g[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) g[f] = dm.ff32[i * NF + f];
  const float2 iv = dm.inv_vol2[i];
  float2 dtp = make_float2(0.0f, 0.0f), q0 = make_float2(0.0f, 0.0f);
  if (!residual_only) {
    dtp = dt2[dm.mesh_of[i]];
    if (a.hi != 0.0f) q0 = p0[i];
  }
  float dj[NF][NQ];
  float2 pj[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int64_t j = nb[f] >= 0 ? (nb[f] >> 2) : i;
    const int f2 = nb[f] >= 0 ? (nb[f] & 3) : f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) dj[f][q] = fdev[j * NP + f2 * NQ + q];
    pj[f] = pin[j];
  }
  dfloat acc = {0.0f, 0.0f};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const bool owner = nb[f] < 0 || i < (nb[f] >> 2);
    const float2 pL = owner ? pi : pj[f], pR = owner ? pj[f] : pi;
    const float jump = (pR.x - pL.x) + (pR.y - pL.y);  // ubar_R - ubar_L
    float dL[NQ], dR[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      dL[q] = owner ? di[f][q] : dj[f][q];
      dR[q] = (owner ? dj[f][q] : di[f][q]) + jump;
    }
    const float fsum = facet_flux_dev_part<NQ>(pde, g[f], speed, pL.x, dL, dR);
    const dfloat uref = {pL.x, pL.y};
    dfloat ref = df_mul(dfloat{g[f].pref_hi, g[f].pref_lo}, uref);
    if (pde != WLSENO_ADVECTION) ref = df_mul(ref, uref);
    const dfloat flux = df_add(ref, df_two_prod(g[f].area, fsum));
    acc = df_add(acc, owner ? flux : df_neg(flux));
  }
  dfloat res = df_neg(df_mul(acc, dfloat{iv.x, iv.y}));  // L
  if (!residual_only) {
    res = df_mul(b, df_add(dfloat{pi.x, pi.y}, df_mul(dfloat{dtp.x, dtp.y}, res)));
    if (a.hi != 0.0f) res = df_add(df_mul(a, dfloat{q0.x, q0.y}), res);
  }
  out[i] = static_cast<double>(res.hi) + static_cast<double>(res.lo);
  if (pout) pout[i] = make_float2(res.hi, res.lo);
  if (!isfinite(res.hi) || !isfinite(res.lo)) atomicAdd(&counters[2], 1ull);
}

__global__ void split_pairs_kernel(const double* __restrict__ u, float2* __restrict__ pair, int64_t n) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= n) return;
  const double v = u[k];
  const float hi = __double2float_rn(v);
  pair[k] = make_float2(hi, __double2float_rn(v - static_cast<double>(hi)));
}

// Largest |ubar| per mesh, as the bits of a non-negative double (their
// integer order is the numeric order, so atomicMax is exact and deterministic).
__global__ void max_abs_kernel(int64_t N, const double* __restrict__ u,
                               const int32_t* __restrict__ mesh_of,
                               unsigned long long* __restrict__ lmax_bits, float2* __restrict__ pairs) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (pairs && i < N) {  // the FP32 pairs of the state, in the same pass
    const double v = u[i];
    const float hi = __double2float_rn(v);
    pairs[i] = make_float2(hi, __double2float_rn(v - static_cast<double>(hi)));
  }
  const bool in = i < N;
  const int mesh = in ? mesh_of[i] : -1;
  unsigned long long bits = in ? static_cast<unsigned long long>(__double_as_longlong(fabs(u[i]))) : 0ull;
  const int lane = threadIdx.x & 31;
  const int m0 = __shfl_sync(0xffffffffu, mesh, 0);
  const bool same = __all_sync(0xffffffffu, mesh == m0 || mesh < 0);
  if (same) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      unsigned long long o = __shfl_xor_sync(0xffffffffu, bits, off);
      bits = o > bits ? o : bits;
    }
    if (lane == 0 && m0 >= 0) atomicMax(&lmax_bits[m0], bits);
  } else if (in) {
    atomicMax(&lmax_bits[mesh], bits);
  }
}

__global__ void cfl_dt_kernel(int n_meshes, int pde, int dim, double adv_speed,
                              const unsigned long long* __restrict__ lmax_bits,
                              const double* __restrict__ rmin, double cfl, double dt_fixed,
                              double* __restrict__ dt_mesh, float2* __restrict__ dt2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_meshes) return;
  double dt = dt_fixed;
  if (dt_fixed <= 0.0) {
    double lam = adv_speed;
    if (pde == WLSENO_BURGERS)
      lam = sqrt(static_cast<double>(dim)) * __longlong_as_double(static_cast<long long>(lmax_bits[k]));
    if (pde == WLSENO_EULER) lam = __longlong_as_double(static_cast<long long>(lmax_bits[k]));  // max |u| + c
    dt = lam > 0.0 ? cfl * rmin[k] / lam : 0.0;
  }
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
    const int threads = 256;
    const unsigned blocks = static_cast<unsigned>((dm.N + threads - 1) / threads);
    max_abs_kernel<<<blocks, threads, 0, s>>>(dm.N, u, dm.mesh_of, lmax_bits, pairs_out);
    ++*launches;
    pairs_out = nullptr;  // made
  } else if (dt_fixed <= 0.0 && sp.pde == WLSENO_EULER) {
    cudaError_t e = launch_euler_speed(dm, sp.gamma, u, lmax_bits, n_meshes, s);
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  if (pairs_out) {  // no wave-speed pass to carry them
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
