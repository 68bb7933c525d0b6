// Per-cell bodies of the flux / residual / RK-stage kernels (k_flux.cu) and
// of the CFL wave-speed pass, shared with the persistent step kernel
// (k_persistent.cu).  See k_flux.cu for the method.
#pragma once

#include <cmath>

#include "dfloat.cuh"
#include "wlseno_internal.h"

namespace wlseno {

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
__device__ __forceinline__ void
flux_cell(DeviceMesh dm, SchemeParams sp, const double* WLSENO_BODY_RESTRICT fvals,
                  const double* WLSENO_BODY_RESTRICT u, const double* WLSENO_BODY_RESTRICT u0, double a, double b,
                  const double* WLSENO_BODY_RESTRICT dt_mesh, int residual_only, double* WLSENO_BODY_RESTRICT out,
                  unsigned long long* WLSENO_BODY_RESTRICT counters, int64_t i) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
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
  if (!isfinite(res)) report_nonfinite(dm, counters);
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
__device__ __forceinline__ void
flux_dev_cell(DeviceMesh dm, SchemeParams sp, const float* WLSENO_BODY_RESTRICT fdev,
                      const double* WLSENO_BODY_RESTRICT u, const double* WLSENO_BODY_RESTRICT u0, double a, double b,
                      const double* WLSENO_BODY_RESTRICT dt_mesh, int residual_only, double* WLSENO_BODY_RESTRICT out,
                      unsigned long long* WLSENO_BODY_RESTRICT counters, const float2* WLSENO_BODY_RESTRICT pin,
                      float2* WLSENO_BODY_RESTRICT pout, int64_t i) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
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
  if (!isfinite(res)) report_nonfinite(dm, counters);
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
__device__ __forceinline__ void
flux_df_cell(DeviceMesh dm, int pde, float speed, const float* WLSENO_BODY_RESTRICT fdev,
                     const float2* WLSENO_BODY_RESTRICT pin, const float2* WLSENO_BODY_RESTRICT p0, dfloat a, dfloat b,
                     const float2* WLSENO_BODY_RESTRICT dt2, int residual_only, double* WLSENO_BODY_RESTRICT out,
                     unsigned long long* WLSENO_BODY_RESTRICT counters, float2* WLSENO_BODY_RESTRICT pout, int64_t i) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
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
  if (!isfinite(res.hi) || !isfinite(res.lo)) report_nonfinite(dm, counters);
}


// FP32 pair of u[i] and this cell's |ubar| folded into the per-mesh maximum
// (the bits of a non-negative double: their integer order is the numeric
// order, so atomicMax is exact and deterministic).  All lanes of the warp
// call it (cells past N pass in = false).
__device__ __forceinline__ void max_abs_cell(int64_t N, const double* WLSENO_BODY_RESTRICT u,
                                             const int32_t* WLSENO_BODY_RESTRICT mesh_of,
                                             unsigned long long* WLSENO_BODY_RESTRICT lmax_bits, float2* WLSENO_BODY_RESTRICT pairs,
                                             int64_t i, bool in) {
  if (pairs && in) {  // the FP32 pairs of the state, in the same pass
    const dfloat d = df_from_double_bits(u[i]);
    pairs[i] = make_float2(d.hi, d.lo);
  }
  const int mesh = in ? mesh_of[i] : -1;
  unsigned long long bits =
      in ? static_cast<unsigned long long>(__double_as_longlong(u[i])) & 0x7fffffffffffffffull : 0ull;  // |u_i|
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

// Per-mesh maxima of the non-negative double bit patterns value_of(i) over
// all cells, with few atomics: block b takes a contiguous chunk of cells,
// each thread keeps a running maximum for the mesh of its current cell
// (flushed with atomicMax when its cells move on to another mesh), and at the
// end the threads that finish on thread 0's mesh are combined in the block
// before one atomicMax; the others flush their own.  (Integer order of the
// bits of non-negative doubles is their numeric order: exact and
// deterministic.)  Launch with a grid of at most a few thousand blocks.
template <typename F>
__device__ __forceinline__ void chunked_mesh_max(int64_t N, const int32_t* WLSENO_BODY_RESTRICT mesh_of,
                                                 unsigned long long* lmax, F&& value_of) {
  __shared__ int m0;
  __shared__ unsigned long long red[32];
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t chunk = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
  const int64_t begin = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t end = begin + chunk < N ? begin + chunk : N;
  int cur = -1;
  unsigned long long mx = 0ull;
  // four cells per pass, their loads issued together
  constexpr int kU = 4;
  for (int64_t i0 = begin + threadIdx.x; i0 < end; i0 += kU * static_cast<int64_t>(blockDim.x)) {
    unsigned long long b[kU];
    int m[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = i0 + u * static_cast<int64_t>(blockDim.x);
      m[u] = i < end ? mesh_of[i] : -1;
      b[u] = i < end ? value_of(i) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (m[u] < 0) continue;
      if (m[u] != cur) {
        if (cur >= 0) atomicMax(&lmax[cur], mx);
        cur = m[u];
        mx = 0ull;
      }
      mx = b[u] > mx ? b[u] : mx;
    }
  }
  if (threadIdx.x == 0) m0 = cur;
  __syncthreads();
  const bool same = cur >= 0 && cur == m0;
  if (!same && cur >= 0) atomicMax(&lmax[cur], mx);
  unsigned long long v = same ? mx : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0ull;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
      v = o > v ? o : v;
    }
    if (threadIdx.x == 0 && m0 >= 0) atomicMax(&lmax[m0], v);
  }
}

// Blocks of a chunked_mesh_max launch over n cells (256 threads each).
__host__ __device__ inline unsigned chunked_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<unsigned>(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

// dt of mesh k: the fixed step when dt_fixed > 0, else cfl rmin / lambda_max
// (advection |a|, Burgers sqrt(dim) max |ubar|, Euler max(|u| + c)).
__device__ __forceinline__ double cfl_dt_of(int pde, int dim, double adv_speed, unsigned long long lmax_bits,
                                            double rmin, double cfl, double dt_fixed) {
  if (dt_fixed > 0.0) return dt_fixed;
  double lam = adv_speed;
  if (pde == WLSENO_BURGERS) lam = sqrt(static_cast<double>(dim)) * __longlong_as_double(static_cast<long long>(lmax_bits));
  if (pde == WLSENO_EULER) lam = __longlong_as_double(static_cast<long long>(lmax_bits));  // max |u| + c
  return lam > 0.0 ? cfl * rmin / lam : 0.0;
}

}  // namespace wlseno
