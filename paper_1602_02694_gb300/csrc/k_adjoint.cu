// Adjoint (vector-Jacobian product) of the spatial operator L and of one
// TVD-RK3 step, in FP64.  The forward operator (Sec. 1, Eqs. (fvm), (flux);
// Sec. 3.1.2, Sec. 3.3.2) is differentiated by hand:
//
//   facet traces  u_{c,f,q} = ubar_c + sum_k d_{c,k} phi_k(y_{c,f,q})
//   WLS solve     d = argmin || W (A d - (ubar_S - ubar_c)) ||  (full rank):
//                 G d = A^T W^2 b, G = A^T W^2 A = R^T R, so for a cotangent
//                 dbar: lambda = G^-1 dbar, bbar_t = w_t^2 (A_t lambda),
//                 wbar_t = 2 w_t (A_t lambda) r_t with r = b - A d
//   weights       w_t = eps h^2 / beta_t (any constant scale of W leaves d
//                 unchanged and gives the same derivative), so
//                 betabar_t = -wbar_t w_t / beta_t; beta_t = (ubar_j -
//                 ubar_c)^2 + eps h^2, and the centre's beta is the minimum
//                 over the facet neighbours (derivative to the first minimiser)
//   LF flux       d/du of 1/2 [(F(uL)+F(uR)).n - alpha (uR - uL)] including
//                 alpha's derivative at its maximiser (Burgers; first maximum)
//
// Cotangents that belong to other cells are written to per-(row, cell) slots
// and gathered through the transposed stencils: no atomics, fixed order.
#include <cmath>

#include "k_recon_tpc_kernels.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

// Cotangents of each cell's own facet traces from lambda = Lbar.
template <int DIM>
__global__ void __launch_bounds__(256)
adj_facet_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ fvals,
                 const double* __restrict__ lambda, double* __restrict__ gfv) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  const double wq = 1.0 / NQ;
  const bool adv = sp.pde == WLSENO_ADVECTION;
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[i * NF + f];
    double uo[NQ], un[NQ];
    for (int q = 0; q < NQ; ++q) uo[q] = fvals[i * NP + f * NQ + q];
    bool owner = true, boundary = nb < 0;
    int64_t j = i;
    if (!boundary) {
      j = nb >> 2;
      const int f2 = nb & 3;
      for (int q = 0; q < NQ; ++q) un[q] = fvals[j * NP + f2 * NQ + q];
      owner = i < j;
    } else {
      for (int q = 0; q < NQ; ++q) un[q] = uo[q];
    }
    double uL[NQ], uR[NQ];
    for (int q = 0; q < NQ; ++q) {
      uL[q] = owner ? uo[q] : un[q];
      uR[q] = owner ? un[q] : uo[q];
    }
    const double* geo = dm.fgeo + (i * NF + f) * 4;
    double nsum = 0.0, vn = 0.0, speed2 = 0.0;
    for (int a = 0; a < DIM; ++a) {
      nsum += geo[a];
      vn += sp.vel[a] * geo[a];
      speed2 += sp.vel[a] * sp.vel[a];
    }
    const double area = geo[3];
    // alpha and its maximiser (q, side), first maximum in the order q, L then R
    double alpha = sqrt(speed2);
    int qmax = -1, smax = 0;
    if (!adv) {
      double mx = -1.0;
      for (int q = 0; q < NQ; ++q) {
        if (fabs(uL[q]) > mx) { mx = fabs(uL[q]); qmax = q; smax = 0; }
        if (fabs(uR[q]) > mx) { mx = fabs(uR[q]); qmax = q; smax = 1; }
      }
      alpha = mx * fabs(nsum);
    }
    double jump = 0.0;
    for (int q = 0; q < NQ; ++q) jump += wq * (uR[q] - uL[q]);
    const int64_t cL = owner ? i : j;
    double Fbar = -lambda[cL] / dm.volume[cL];
    if (!boundary) {
      const int64_t cR = owner ? j : i;
      Fbar += lambda[cR] / dm.volume[cR];
    }
    for (int q = 0; q < NQ; ++q) {
      const double fpL = adv ? vn : uL[q] * nsum;
      const double fpR = adv ? vn : uR[q] * nsum;
      double dL = area * wq * 0.5 * (fpL + alpha);
      double dR = area * wq * 0.5 * (fpR - alpha);
      if (!adv && q == qmax) {
        const double da = -0.5 * area * jump * fabs(nsum);
        if (smax == 0) dL += da * (uL[q] >= 0.0 ? 1.0 : -1.0);
        else dR += da * (uR[q] >= 0.0 ? 1.0 : -1.0);
      }
      const double d_own = boundary ? dL + dR : (owner ? dL : dR);
      gfv[i * NP + f * NQ + q] = Fbar * d_own;
    }
  }
}

// Reconstruction VJP of cell c: per-row cotangents for the other cells
// (contrib[t*N + c], t >= 1), the argmin neighbour's share and c's own.
template <int DIM, int M>
__global__ void __launch_bounds__(128)
adj_recon_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ ubar,
                 const double* __restrict__ gfv, double* __restrict__ contrib,
                 double* __restrict__ selfbar, int* __restrict__ amin_cell,
                 double* __restrict__ amin_val) {
  constexpr int NF = DIM + 1;
  constexpr int NP = NF * nq_of(DIM);
  const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (c >= dm.N) return;
  const int64_t N = dm.N;
  const int n = dm.st_ptr[c + 1] - dm.st_ptr[c];
  const double uc = ubar[c];
  const double hc = dm.h[c];
  const double e = sp.eps * hc * hc;
  double bmin = INFINITY;
  int64_t kmin = -1;
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[c * NF + f];
    if (nb >= 0) {
      const double d = ubar[nb >> 2] - uc;
      const double b = d * d + e;
      if (b < bmin) {
        bmin = b;
        kmin = nb >> 2;
      }
    }
  }
  const double wc = sp.alpha_c * e / bmin;
  SqrtFreeQR<double, M> f;  // W A = Q D^(1/2) U
  tpc_fold<DIM, M>(dm, ubar, c, uc, n, e, wc, f);
  double d[M];
  sqrt_free_solve(f, d);
  // dbar from the facet-trace cotangents
  double dbar[M];
#pragma unroll
  for (int k = 0; k < M; ++k) dbar[k] = 0.0;
  double direct = 0.0;
  const double* P = dm.fpts + c * NP * DIM;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    double yy[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) yy[a] = P[p * DIM + a];
    double mono[M];
    eval_monomials<double, DIM, M>(yy, mono);
    const double g = gfv[c * NP + p];
    direct += g;
#pragma unroll
    for (int k = 0; k < M; ++k) dbar[k] += g * mono[k];
  }
  // lambda = (R^T R)^-1 dbar = U^-1 D^-1 U^-T dbar
  double v[M], lam[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    double t = dbar[k];
#pragma unroll
    for (int q = 0; q < k; ++q) t = fma(-f.U[q][k], v[q], t);
    v[k] = t;
  }
#pragma unroll
  for (int k = 0; k < M; ++k) v[k] /= f.d[k];
#pragma unroll
  for (int k = M - 1; k >= 0; --k) {
    double t = v[k];
#pragma unroll
    for (int q = k + 1; q < M; ++q) t = fma(-f.U[k][q], lam[q], t);
    lam[k] = t;
  }
  double self = direct;
  double aval = 0.0;
  for (int t = 0; t < n; ++t) {
    const int64_t j = dm.st_ell[t * N + c];
    const double dev = ubar[j] - uc;
    const double beta = t == 0 ? bmin : dev * dev + e;
    const double w = t == 0 ? wc : e / beta;
    double al = 0.0, ad = 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const double a = dm.A64e[(static_cast<int64_t>(t) * M + k) * N + c];
      al += a * lam[k];
      ad += a * d[k];
    }
    const double r = dev - ad;
    const double devbar = w * w * al;
    const double betabar = -(2.0 * w * al * r) * w / beta;
    if (t == 0) {
      if (kmin >= 0) aval = 2.0 * (ubar[kmin] - uc) * betabar;
    } else {
      const double cj = devbar + 2.0 * dev * betabar;
      contrib[t * N + c] = cj;
      self -= cj;
    }
  }
  self -= aval;
  selfbar[c] = self;
  amin_cell[c] = static_cast<int>(kmin);
  amin_val[c] = aval;
}

template <int DIM>
__global__ void __launch_bounds__(256)
adj_gather_kernel(DeviceMesh dm, const double* __restrict__ contrib,
                  const double* __restrict__ selfbar, const int* __restrict__ amin_cell,
                  const double* __restrict__ amin_val, const int64_t* __restrict__ tr_ptr,
                  const int64_t* __restrict__ tr_slot, double* __restrict__ out) {
  constexpr int NF = DIM + 1;
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= dm.N) return;
  double acc = selfbar[j];
  for (int64_t e = tr_ptr[j]; e < tr_ptr[j + 1]; ++e) acc += contrib[tr_slot[e]];
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[j * NF + f];
    if (nb >= 0 && amin_cell[nb >> 2] == j) acc += amin_val[nb >> 2];
  }
  out[j] = acc;
}

// out = ca x + cb y + cc w + cz dt_mesh z (null inputs skipped)
__global__ void adj_combine_kernel(int64_t N, const int32_t* __restrict__ mesh_of,
                                   const double* __restrict__ dt_mesh, const double* x, double ca,
                                   const double* y, double cb, const double* w, double cc,
                                   const double* z, double cz, double* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  if (x) acc += ca * x[i];
  if (y) acc += cb * y[i];
  if (w) acc += cc * w[i];
  if (z) acc += cz * dt_mesh[mesh_of[i]] * z[i];
  out[i] = acc;
}

template <int DIM, int M>
cudaError_t launch_recon_vjp(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                             const double* gfv, const AdjointWork& w, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>((dm.N + 127) / 128);
  adj_recon_kernel<DIM, M><<<blocks, 128, 0, s>>>(dm, sp, ubar, gfv, w.contrib, w.selfbar,
                                                  w.amin_cell, w.amin_val);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_operator_vjp(const DeviceMesh& dm, const SchemeParams& sp, const double* state,
                                const double* fvals, const double* lambda, const AdjointWork& w,
                                double* out, cudaStream_t s, int* launches) {
  const unsigned b256 = static_cast<unsigned>((dm.N + 255) / 256);
  *launches = 0;
  if (dm.dim == 2) adj_facet_kernel<2><<<b256, 256, 0, s>>>(dm, sp, fvals, lambda, w.gfv);
  else adj_facet_kernel<3><<<b256, 256, 0, s>>>(dm, sp, fvals, lambda, w.gfv);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (dm.dim == 2 && dm.m == 6) e = launch_recon_vjp<2, 6>(dm, sp, state, w.gfv, w, s);
  else if (dm.dim == 2 && dm.m == 10) e = launch_recon_vjp<2, 10>(dm, sp, state, w.gfv, w, s);
  else if (dm.dim == 3 && dm.m == 10) e = launch_recon_vjp<3, 10>(dm, sp, state, w.gfv, w, s);
  else return cudaErrorInvalidValue;
  ++*launches;
  if (e != cudaSuccess) return e;
  if (dm.dim == 2)
    adj_gather_kernel<2><<<b256, 256, 0, s>>>(dm, w.contrib, w.selfbar, w.amin_cell, w.amin_val,
                                             w.tr_ptr, w.tr_slot, out);
  else
    adj_gather_kernel<3><<<b256, 256, 0, s>>>(dm, w.contrib, w.selfbar, w.amin_cell, w.amin_val,
                                             w.tr_ptr, w.tr_slot, out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_adj_combine(const DeviceMesh& dm, const double* dt_mesh, const double* x,
                               double ca, const double* y, double cb, const double* w, double cc,
                               const double* z, double cz, double* out, cudaStream_t s) {
  const unsigned b256 = static_cast<unsigned>((dm.N + 255) / 256);
  adj_combine_kernel<<<b256, 256, 0, s>>>(dm.N, dm.mesh_of, dt_mesh, x, ca, y, cb, w, cc, z, cz, out);
  return cudaGetLastError();
}

}  // namespace wlseno
