// Balanced-stencil re-selection (Sec. 3.2, last paragraph), scalar equations.
//
// After a reconstruction, a cell whose reconstructed value at any of its facet
// quadrature points leaves [min, max] of its stencil's averages by more than
// margin * (max - min of the averages over its mesh) is re-solved on a new
// stencil balanced about the plane through its centroid x_i normal to the
// gradient of its reconstruction:
//   * the candidates are the cells of the enlarged ring (ceil(ring) + 1
//     vertex-sharing steps; built on the host, centre excluded, ascending);
//   * the new stencil keeps the centre and its facet neighbours and has the
//     old stencil's size n; the plus side (x_j - x_i).grad u > 0 gets
//     floor(n/2) cells and the other side floor((n-1)/2), facet neighbours
//     counting towards their side; each side is filled with its nearest
//     candidates (squared centroid distance, ties by index), and when a side
//     runs short the nearest remaining candidates of either side fill up;
//   * the rows are ordered centre first, then by cell index; their moments
//     are computed on the fly with the precompute's quadrature, the weights
//     are those of Sec. 3.1.2 and the system is solved in FP64.
// The margin is a reading of the paper's range test: smooth extrema exceed
// their stencil's range by O(h^2) of the data's range, overshoots at a jump
// by a share of the jump; the margin also keeps averages that are equal up to
// rounding (flat regions) from deciding the test.
//
// Three launches: the per-mesh range of the averages (warp-reduced atomic
// maxima of order-preserving keys of u and -u), the range test (one thread
// per cell; cells out of range go to a list), and the re-selection (one
// thread per listed cell, grid-stride over the list, whose length stays on
// the device so the sequence can be captured in a graph).  Cells whose
// gradient vanishes or whose system is ill-conditioned keep the plain result.
#include <cmath>
#include <climits>

#include "k_recon_tpc_kernels.cuh"
#include "moment_row.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

// Conditioning bound (spread of the column-scaled diagonal) above which a
// balanced system is left alone: the plain result stays.
constexpr double kBalanceBound = 1e6;

// Order-preserving map of doubles to unsigned keys, and back.
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(static_cast<long long>(b));
}

// state[1 + 2k] = max key of u over mesh k, state[2 + 2k] = max key of -u.
__global__ void range_kernel(const double* __restrict__ ubar, const int32_t* __restrict__ mesh_of,
                             int64_t N, unsigned long long* __restrict__ state) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const bool valid = i < N;
  const int mi = valid ? mesh_of[i] : -1;
  unsigned long long kp = valid ? order_key(ubar[i]) : 0ull;
  unsigned long long kn = valid ? order_key(-ubar[i]) : 0ull;
  const unsigned full = 0xffffffffu;
  const int m0 = __shfl_sync(full, mi, 0);
  if (__all_sync(full, mi == m0 || mi < 0)) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long op = __shfl_down_sync(full, kp, off);
      const unsigned long long on = __shfl_down_sync(full, kn, off);
      kp = op > kp ? op : kp;
      kn = on > kn ? on : kn;
    }
    if ((threadIdx.x & 31) == 0 && m0 >= 0) {
      atomicMax(&state[1 + 2 * m0], kp);
      atomicMax(&state[2 + 2 * m0], kn);
    }
  } else if (valid) {
    atomicMax(&state[1 + 2 * mi], kp);
    atomicMax(&state[2 + 2 * mi], kn);
  }
}

// Range test of every cell on the reconstruction's own output (facet values,
// FP32 deviations, or the coefficients evaluated at the facet points).
template <int DIM, int M>
__global__ void range_test_kernel(DeviceMesh dm, BalanceWork bw, const double* __restrict__ ubar,
                                  const double* __restrict__ coeffs, const double* __restrict__ fvals,
                                  const float* __restrict__ fdev) {
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  const double ui = ubar[i];
  double lo = ui, hi = ui;
  for (int t = dm.st_ptr[i]; t < dm.st_ptr[i + 1]; ++t) {
    const double u = ubar[dm.st_idx[t]];
    lo = fmin(lo, u);
    hi = fmax(hi, u);
  }
  const int mi = dm.mesh_of[i];
  const double gmax = key_value(bw.state[1 + 2 * mi]);
  const double gmin = -key_value(bw.state[2 + 2 * mi]);
  const double tol = bw.margin * (gmax - gmin);
  bool out = false;
  for (int pt = 0; pt < NP; ++pt) {
    double v;
    if (fvals) {
      v = fvals[i * NP + pt];
    } else if (fdev) {
      v = ui + static_cast<double>(fdev[i * NP + pt]);
    } else {
      double y[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) y[a] = dm.fpts[(i * NP + pt) * DIM + a];
      double mono[M];
      eval_monomials<double, DIM, M>(y, mono);
      v = 0.0;
#pragma unroll
      for (int c = 0; c < M; ++c) v += coeffs[i * M + c] * mono[c];
    }
    out = out || v < lo - tol || v > hi + tol;
  }
  if (out) bw.list[atomicAdd(&bw.state[0], 1ull)] = static_cast<int>(i);
}

// Sort key of a candidate: (squared distance, index).
struct Key {
  double d2;
  int j;
};
__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
  return a.d2 < b.d2 || (a.d2 == b.d2 && a.j < b.j);
}

template <int DIM, int M>
__global__ void __launch_bounds__(64)
balance_kernel(DeviceMesh dm, SchemeParams sp, BalanceWork bw, const double* __restrict__ ubar,
               double* __restrict__ coeffs, double* __restrict__ fvals, float* __restrict__ fdev,
               GaussRule g) {
  constexpr int NF = DIM + 1;
  const int64_t n_list = static_cast<int64_t>(bw.state[0]);
  for (int64_t L = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; L < n_list;
       L += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = bw.list[L];
    const double ui = ubar[i];
    const int n = dm.st_ptr[i + 1] - dm.st_ptr[i];
    double eh2, wc;
    tpc_weights<double, DIM>(dm, sp, ubar, i, ui, &eh2, &wc);
    // gradient direction: first-order coefficients of the plain reconstruction
    double gdir[DIM];
    {
      SqrtFreeQR<double, M> f;
      tpc_fold<DIM, M>(dm, ubar, i, ui, n, eh2, wc, f);
      double qmax, qmin;
      sqrt_free_spread(f, &qmax, &qmin);
      if (!(qmax <= kBalanceBound * kBalanceBound * qmin)) continue;
      double x[M];
      sqrt_free_solve(f, x);
#pragma unroll
      for (int a = 0; a < DIM; ++a) gdir[a] = x[1 + a];
    }
    bool nonzero = false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) nonzero = nonzero || gdir[a] != 0.0;
    if (!nonzero) continue;
    // facet neighbours (distinct), their sides and the side quotas
    const double* per = dm.period + 3 * dm.mesh_of[i];
    auto locate = [&](int j, bool* plus, double* d2) {
      double s = 0.0, q = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        double d = dm.centroid[static_cast<int64_t>(j) * DIM + a] - dm.centroid[i * DIM + a];
        if (per[a] > 0.0) d -= per[a] * nearbyint(d / per[a]);
        s = fma(d, gdir[a], s);
        q = fma(d, d, q);
      }
      *plus = s > 0.0;
      *d2 = q;
    };
    int face[NF];
    int n_face = 0;
    int quota[2] = {(n - 1) / 2, n / 2};  // [0]: s <= 0 side, [1]: s > 0 side
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int nb = dm.nbr[i * NF + f];
      int j = nb >= 0 ? (nb >> 2) : -1;
      for (int e = 0; e < n_face; ++e)
        if (face[e] == j) j = -1;
      if (j >= 0 && j != i) {
        face[n_face++] = j;
        bool plus;
        double d2;
        locate(j, &plus, &d2);
        --quota[plus ? 1 : 0];
      }
    }
    auto is_face = [&](int j) {
      bool r = false;
      for (int e = 0; e < n_face; ++e) r = r || face[e] == j;
      return r;
    };
    const int cb = bw.cand_ptr[i], ce = bw.cand_ptr[i + 1];
    // each side's nearest candidates: those with key <= last[side]
    Key last[2] = {{-1.0, -1}, {-1.0, -1}};
    int chosen = n_face;
    for (int sd = 1; sd >= 0; --sd) {
      for (int k = 0; k < quota[sd]; ++k) {
        Key best{INFINITY, INT_MAX};
        bool found = false;
        for (int c = cb; c < ce; ++c) {
          const int j = bw.cand_idx[c];
          if (is_face(j)) continue;
          bool plus;
          double d2;
          locate(j, &plus, &d2);
          const Key kj{d2, j};
          if ((plus ? 1 : 0) != sd || !key_less(last[sd], kj)) continue;
          if (key_less(kj, best)) {
            best = kj;
            found = true;
          }
        }
        if (!found) break;
        last[sd] = best;
        ++chosen;
      }
    }
    // top-up from the remaining candidates of either side: key <= last_t
    Key last_t{-1.0, -1};
    while (chosen < n - 1) {
      Key best{INFINITY, INT_MAX};
      bool found = false;
      for (int c = cb; c < ce; ++c) {
        const int j = bw.cand_idx[c];
        if (is_face(j)) continue;
        bool plus;
        double d2;
        locate(j, &plus, &d2);
        const Key kj{d2, j};
        if (!key_less(last[plus ? 1 : 0], kj) || !key_less(last_t, kj)) continue;
        if (key_less(kj, best)) {
          best = kj;
          found = true;
        }
      }
      if (!found) break;
      last_t = best;
      ++chosen;
    }
    // fold the new stencil: centre, then the chosen candidates by index
    SqrtFreeQR<double, M> f;
    sqrt_free_init(f);
    {
      double z[M + 1];
      double row[M];
      moment_row<DIM, M>(dm, g, i, i, row);
#pragma unroll
      for (int c = 0; c < M; ++c) z[c] = row[c];
      z[M] = 0.0;
      sqrt_free_fold(f, z, wc * wc);
    }
    for (int c = cb; c < ce; ++c) {
      const int j = bw.cand_idx[c];
      bool take = is_face(j);
      if (!take) {
        bool plus;
        double d2;
        locate(j, &plus, &d2);
        const Key kj{d2, j};
        take = !key_less(last[plus ? 1 : 0], kj) || !key_less(last_t, kj);
      }
      if (!take) continue;
      const double dev = ubar[j] - ui;
      double z[M + 1];
      double row[M];
      moment_row<DIM, M>(dm, g, i, j, row);
#pragma unroll
      for (int k = 0; k < M; ++k) z[k] = row[k];
      z[M] = dev;
      const double w = eh2 * recip_t(fma(dev, dev, eh2));
      sqrt_free_fold(f, z, w * w);
    }
    double qmax, qmin;
    sqrt_free_spread(f, &qmax, &qmin);
    if (!(qmax <= kBalanceBound * kBalanceBound * qmin)) continue;
    double x[M];
    sqrt_free_solve(f, x);
    tpc_write<double, DIM, M>(dm, i, ui, x, coeffs, fvals, fdev);
    atomicAdd(bw.count, 1ull);
  }
}

template <int DIM, int M>
cudaError_t launch_dm(const DeviceMesh& dm, const SchemeParams& sp, const BalanceWork& bw,
                      const double* ubar, const ReconOut& out, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = static_cast<unsigned>((dm.N + threads - 1) / threads);
  range_kernel<<<blocks, threads, 0, s>>>(ubar, dm.mesh_of, dm.N, bw.state);
  range_test_kernel<DIM, M><<<blocks, threads, 0, s>>>(dm, bw, ubar, out.coeffs, out.fvals, out.fdev);
  const int64_t want = (dm.N + 63) / 64;
  const unsigned bblocks = static_cast<unsigned>(want < 1216 ? want : 1216);
  balance_kernel<DIM, M><<<bblocks, 64, 0, s>>>(dm, sp, bw, ubar, out.coeffs, out.fvals, out.fdev,
                                                make_gauss_rule());
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_balance(const DeviceMesh& dm, const SchemeParams& sp, const BalanceWork& bw,
                           const double* ubar, const ReconOut& out, cudaStream_t s, int* launches) {
  *launches = 0;
  if (dm.N == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(bw.state, 0, sizeof(unsigned long long) * (1 + 2 * bw.n_meshes), s);
  if (e != cudaSuccess) return e;
  if (dm.dim == 1 && dm.m == 3) e = launch_dm<1, 3>(dm, sp, bw, ubar, out, s);
  else if (dm.dim == 1 && dm.m == 5) e = launch_dm<1, 5>(dm, sp, bw, ubar, out, s);
  else if (dm.dim == 2 && dm.m == 6) e = launch_dm<2, 6>(dm, sp, bw, ubar, out, s);
  else if (dm.dim == 2 && dm.m == 10) e = launch_dm<2, 10>(dm, sp, bw, ubar, out, s);
  else if (dm.dim == 3 && dm.m == 10) e = launch_dm<3, 10>(dm, sp, bw, ubar, out, s);
  else return cudaErrorInvalidValue;
  if (e == cudaSuccess) *launches = 3;
  return e;
}

}  // namespace wlseno
