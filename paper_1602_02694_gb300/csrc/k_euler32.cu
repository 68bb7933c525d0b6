// FP32-bulk compressible Euler in 2-D (componentwise WLS-ENO, p = 3): the
// flux / RK-stage kernel that follows the all-components reconstruction
// (launch_recon_euler2d), and the FP32 pairs of the state it reads.
//
// Inputs per cell: the FP32 traces of the four components at its six facet
// points ([N][6] float4, written by the reconstruction and its follow-ups:
// hi + (lo + deviation) of each component, or the averages hi + lo at every
// point of a cell whose traces give density or pressure <= 1e-12, reading
// R14), and the averages as FP32 pairs interleaved [N][4] (hi + lo of each
// FP64 average, for the stage update).  A facet reads its own traces and the
// neighbour's at the same points: two 16-byte loads per point.  Per facet the
// Lax-Friedrichs flux of Sec. 1, Eq. (flux), with alpha = max over the
// facet's points and both sides of |u.n| + c, is evaluated in FP32 in the
// orientation of the facet's lower-indexed cell with that cell's normal and
// area (stored identically in both cells' facet records): both cells form it
// from the same operands in the same order, so it is bitwise the same in
// both, conservation stays exact and no atomics are needed.  The facet sums,
// the division by |tau_i| and the Shu-Osher combination (Sec. 4.2.1) run in
// double-float arithmetic (dfloat.cuh) on the FP32 pipes; the FP64 state
// written is hi + lo exactly, and the pairs of the new state are written for
// the next stage.
#include <cmath>

#include "dfloat.cuh"
#include "k_flux_cell.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

constexpr int kC = 4;  // rho, rho u, rho v, E

// The normal flux F(U).n and the wave speed |u.n| + c of a state in FP32,
// with the hardware reciprocal and reciprocal square root (about one ulp;
// the flux carries FP32 rounding relative to |F| in any case, and both cells
// of a facet evaluate it from the same operands: the same bits).
__device__ __forceinline__ float approx_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_sqrt_nonneg(float x) {  // 0 for x <= 0
  return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

__device__ __forceinline__ void euler2_state(const float (&U)[kC], float nx, float ny, float gamma,
                                             float (&F)[kC], float* speed) {
  const float rho = U[0];
  const float inv = approx_rcp(rho);
  const float un = (U[1] * nx + U[2] * ny) * inv;
  const float ke = U[1] * U[1] + U[2] * U[2];
  const float p = (gamma - 1.0f) * (U[3] - 0.5f * ke * inv);
  F[0] = rho * un;
  F[1] = U[1] * un + p * nx;
  F[2] = U[2] * un + p * ny;
  F[3] = (U[3] + p) * un;
  const float c2 = gamma * p * inv;
  *speed = fabsf(un) + approx_sqrt_nonneg(c2);
}

__global__ void __launch_bounds__(128, 6)
euler2_flux32_kernel(DeviceMesh dm, float gamma, const float4* __restrict__ tr, const float2* __restrict__ pin,
                     const float2* __restrict__ p0, dfloat a, dfloat b, const float2* __restrict__ dt2,
                     int residual_only, double* __restrict__ out, unsigned long long* __restrict__ counters,
                     float2* __restrict__ pout) {
  constexpr int NF = 3, NQ = 2, NP = 6;
  const int64_t N = dm.N;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  // every load up front: neighbours first (the other loads depend on them)
  int nb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) nb[f] = dm.nbr[i * NF + f];
  float4 To[NP];  // own traces, the four components of a point together
#pragma unroll
  for (int k = 0; k < NP; ++k) To[k] = tr[i * NP + k];
  const float4* pin4 = reinterpret_cast<const float4*>(pin);
  float2 P[kC];
  {
    const float4 v0 = pin4[2 * i], v1 = pin4[2 * i + 1];
    P[0] = make_float2(v0.x, v0.y);
    P[1] = make_float2(v0.z, v0.w);
    P[2] = make_float2(v1.x, v1.y);
    P[3] = make_float2(v1.z, v1.w);
  }
  float4 g[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) g[f] = dm.nf32[i * NF + f];
  const float2 iv = dm.inv_vol2[i];
  float2 dtp = make_float2(0.0f, 0.0f);
  float2 q0[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) q0[c] = make_float2(0.0f, 0.0f);
  if (!residual_only) {
    dtp = dt2[dm.mesh_of[i]];
    if (a.hi != 0.0f) {
      const float4* p04 = reinterpret_cast<const float4*>(p0);
      const float4 v0 = p04[2 * i], v1 = p04[2 * i + 1];
      q0[0] = make_float2(v0.x, v0.y);
      q0[1] = make_float2(v0.z, v0.w);
      q0[2] = make_float2(v1.x, v1.y);
      q0[3] = make_float2(v1.z, v1.w);
    }
  }
  // the neighbours' traces at the shared facets (the same points, in the
  // same order, as the facet's points in cell i)
  float4 Tn[NF][NQ];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int64_t j = nb[f] >= 0 ? (nb[f] >> 2) : i;
    const int f2 = nb[f] >= 0 ? (nb[f] & 3) : f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) Tn[f][q] = tr[j * NP + f2 * NQ + q];
  }
  dfloat acc[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) acc[c] = dfloat{0.0f, 0.0f};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const bool inner = nb[f] >= 0;
    const bool owner = !inner || i < (nb[f] >> 2);
    float fs[kC] = {0.0f, 0.0f, 0.0f, 0.0f};
    float UL[NQ][kC], UR[NQ][kC];
    float alpha = 0.0f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 o = To[f * NQ + q];
      const float4 t = inner ? Tn[f][q] : o;  // transmissive: u+ = u-
      const float Uo[kC] = {o.x, o.y, o.z, o.w}, Un[kC] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        UL[q][c] = owner ? Uo[c] : Un[c];
        UR[q][c] = owner ? Un[c] : Uo[c];
      }
    }
    float FL[NQ][kC], FR[NQ][kC];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float sL, sR;
      euler2_state(UL[q], g[f].x, g[f].y, gamma, FL[q], &sL);
      euler2_state(UR[q], g[f].x, g[f].y, gamma, FR[q], &sR);
      alpha = fmaxf(alpha, fmaxf(sL, sR));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int c = 0; c < kC; ++c)
        fs[c] += 0.5f * (0.5f * ((FL[q][c] + FR[q][c]) - alpha * (UR[q][c] - UL[q][c])));
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const dfloat contrib = df_two_prod(g[f].w, fs[c]);
      acc[c] = df_add(acc[c], owner ? contrib : df_neg(contrib));
    }
  }
  bool finite = true;
  float2 outp[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) {
    dfloat res = df_neg(df_mul(acc[c], dfloat{iv.x, iv.y}));  // L
    if (!residual_only) {
      res = df_mul(b, df_add(dfloat{P[c].x, P[c].y}, df_mul(dfloat{dtp.x, dtp.y}, res)));
      if (a.hi != 0.0f) res = df_add(df_mul(a, dfloat{q0[c].x, q0[c].y}), res);
    }
    out[c * N + i] = static_cast<double>(res.hi) + static_cast<double>(res.lo);
    outp[c] = make_float2(res.hi, res.lo);
    finite = finite && isfinite(res.hi) && isfinite(res.lo);
  }
  if (pout) {
    float4* po = reinterpret_cast<float4*>(pout);
    po[2 * i] = make_float4(outp[0].x, outp[0].y, outp[1].x, outp[1].y);
    po[2 * i + 1] = make_float4(outp[2].x, outp[2].y, outp[3].x, outp[3].y);
  }
  if (!finite) report_nonfinite(dm, counters);
}

// pairs[i][c] = (fl32(u[c][i]), fl32(u[c][i] - hi)) for the four components.
__global__ void euler2_split_pairs_kernel(const double* __restrict__ u, float2* __restrict__ pairs, int64_t N) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  float v[2 * kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) {
    const dfloat d = df_from_double_bits(u[c * N + i]);
    v[2 * c] = d.hi;
    v[2 * c + 1] = d.lo;
  }
  float4* po = reinterpret_cast<float4*>(pairs);
  po[2 * i] = make_float4(v[0], v[1], v[2], v[3]);
  po[2 * i + 1] = make_float4(v[4], v[5], v[6], v[7]);
}

// The FP32 pairs of the state (interleaved) and, in the same pass, the
// largest |u| + c per mesh from them in FP32 (the CFL step of the FP32-bulk
// path; FP32 relative accuracy is ample for a time step), as the bits of a
// non-negative double; a non-finite state gives infinity (dt = 0).  The
// pairs and the bits come from integer operations (dfloat.cuh): with four
// FP64 values per cell, the FP64 pipe would otherwise bound the pass.
__global__ void __launch_bounds__(256)
euler2_speed_pairs32_kernel(int64_t N, float gamma, const double* __restrict__ u,
                            const int32_t* __restrict__ mesh_of, unsigned long long* __restrict__ lmax_bits,
                            float2* __restrict__ pairs) {
  float4* po = reinterpret_cast<float4*>(pairs);
  chunked_mesh_max(N, mesh_of, lmax_bits, [&](int64_t i) {
    float v[2 * kC], U[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const dfloat d = df_from_double_bits(u[c * N + i]);
      v[2 * c] = d.hi;
      v[2 * c + 1] = d.lo;
      U[c] = d.hi;
    }
    po[2 * i] = make_float4(v[0], v[1], v[2], v[3]);
    po[2 * i + 1] = make_float4(v[4], v[5], v[6], v[7]);
    const float inv = approx_rcp(U[0]);
    const float ke = U[1] * U[1] + U[2] * U[2];
    const float p = (gamma - 1.0f) * (U[3] - 0.5f * ke * inv);
    const float c2 = gamma * p * inv;
    float s = approx_sqrt_nonneg(ke) * inv + approx_sqrt_nonneg(c2);
    if (!(s >= 0.0f) || !(s <= 3.0e38f)) s = INFINITY;
    return static_cast<unsigned long long>(df_f64_bits_nonneg(s));
  });
}

}  // namespace

cudaError_t launch_euler2_speed_pairs32(const DeviceMesh& dm, double gamma, const double* u,
                                        unsigned long long* lmax_bits, int n_meshes, float2* pairs,
                                        cudaStream_t s) {
  if (dm.dim != 2 || !pairs) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(lmax_bits, 0, sizeof(unsigned long long) * n_meshes, s);
  if (e != cudaSuccess) return e;
  euler2_speed_pairs32_kernel<<<chunked_blocks(dm.N), 256, 0, s>>>(
      dm.N, static_cast<float>(gamma), u, dm.mesh_of, lmax_bits, pairs);
  return cudaGetLastError();
}

cudaError_t launch_euler2_flux32(const DeviceMesh& dm, double gamma, const float* traces, const float2* pin,
                                 const float2* p0, double a, double b, const float2* dt2, bool residual_only,
                                 double* out, unsigned long long* counters, float2* pout, cudaStream_t s) {
  if (dm.dim != 2 || !dm.nf32 || !dm.inv_vol2 || !pin || !traces) return cudaErrorInvalidValue;
  if (!residual_only && (!dt2 || (a != 0.0 && !p0))) return cudaErrorInvalidValue;
  const unsigned blocks = static_cast<unsigned>((dm.N + 127) / 128);
  euler2_flux32_kernel<<<blocks, 128, 0, s>>>(dm, static_cast<float>(gamma),
                                              reinterpret_cast<const float4*>(traces), pin, p0,
                                              df_from_double(a), df_from_double(b), dt2, residual_only ? 1 : 0,
                                              out, counters, residual_only ? nullptr : pout);
  return cudaGetLastError();
}

cudaError_t launch_euler2_split_pairs(const double* u, float2* pairs, int64_t N, cudaStream_t s) {
  euler2_split_pairs_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, s>>>(u, pairs, N);
  return cudaGetLastError();
}

}  // namespace wlseno
