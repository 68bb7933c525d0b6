// WLS-ENO reconstruction kernel (Sec. 3.1.2, Sec. 3.2, Sec. 3.3.2).
//
// One group of G consecutive lanes of a warp owns one cell.  The weighted,
// column-scaled system [W A S | W (ubar_S - ubar_i)] is built in registers,
// its rows are put in order of decreasing norm through shared memory, and
// lane g then holds sorted rows g, g+G, ..., g+(R-1)G.  Householder QR with
// column pivoting (columns swapped in registers) runs on the group with
// butterfly shuffles: every lane ends each reduction with the bitwise-same
// sum, so pivot and rank decisions agree across the group.  Row k of R stays
// in its owner lane; the back substitution broadcasts each unknown.
//
// Arithmetic type T is double (FP64 mode) or float (FP32-bulk mode).
// FP32-bulk keeps in FP64: ubar_j - ubar_i, the final ubar_i + deviation, and
// -- for cells whose estimate |R_00|/|R_rr| exceeds kappa_flag -- one
// refinement sweep: the residual r = W(ubar_S - ubar_i) - W A S y with the
// FP64 moments, then y += R^-1 Q^T r with the FP32 factors.
//
// Readings of the paper used here (Sec. 3.1.2, Sec. 3.3.2):
//  * weights are scaled by the constant eps h_i^2 (the least-squares solution
//    does not depend on the scale of W): w_j = eps h^2 / beta_j,
//    w_i = alpha eps h^2 / beta_i, beta_i = min over facet neighbours;
//  * the right-hand side is the deviation ubar_j - ubar_i; the constant
//    column of A is 1 in every row, so this only shifts d_0 by ubar_i;
//  * pivot = lowest-index remaining column whose trailing norm is within a
//    relative 1e-6 (FP32: 1e-4) of the largest, trailing norms recomputed at
//    every step; rank r = #{k : |R_kk| > rank_tol |R_00|}; dropped
//    coefficients are 0;
//  * rows are processed in order of decreasing norm (the solution does not
//    depend on the row order; sorted rows make Householder QR row-wise
//    backward stable when the weights spread over orders of magnitude).
#pragma once

#include <cmath>
#include <utility>

#include "monomials.cuh"
#include "wlseno_internal.h"

namespace wlseno {

constexpr unsigned kFull = 0xffffffffu;

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

template <typename T>
__device__ __forceinline__ const T* moment_array(const DeviceMesh& dm);
template <>
__device__ __forceinline__ const double* moment_array<double>(const DeviceMesh& dm) { return dm.A64; }
template <>
__device__ __forceinline__ const float* moment_array<float>(const DeviceMesh& dm) { return dm.A32; }

template <typename T>
__device__ __forceinline__ const T* facet_point_array(const DeviceMesh& dm);
template <>
__device__ __forceinline__ const double* facet_point_array<double>(const DeviceMesh& dm) { return dm.fpts; }
template <>
__device__ __forceinline__ const float* facet_point_array<float>(const DeviceMesh& dm) { return dm.fpts32; }

// Register state of one cell's factorisation, shared by the unrolled steps.
template <typename T, int M, int R>
struct QRState {
  T B[R][M];       // sorted rows of W A S; then R above the diagonal and the
                   // Householder vectors below it (column k, rows > k)
  T rhs[R];        // W (ubar_S - ubar_i), then Q^T of it
  T y[M];          // solution in pivoted column order
  T inv_s[M];      // S, in pivoted column order
  T hv[M];         // k-th entry of the k-th Householder vector
  T ht[M];         // its 2 / (v^T v)
  int col[M];      // original column at pivoted position k
  T r00, rlast;
  int rank;
};

template <typename T>
__device__ __forceinline__ void swap_if(bool c, T& a, T& b) {
  const T ta = a;
  a = c ? b : a;
  b = c ? ta : b;
}

// Step K of Householder QR with column pivoting on the group's rows.
template <int K, typename T, int M, int G, int R>
__device__ __forceinline__ void qr_step(QRState<T, M, R>& st, int g, T tau_piv, T rank_tol) {
  // trailing norms of the remaining columns
  T pn[M];
#pragma unroll
  for (int c = K; c < M; ++c) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (g + G * r >= K) s += st.B[r][c] * st.B[r][c];
    pn[c] = group_sum<G>(s);
  }
  T mx = T(0);
#pragma unroll
  for (int c = K; c < M; ++c) mx = pn[c] > mx ? pn[c] : mx;
  int p = M;
  T sigma = T(0);
#pragma unroll
  for (int c = M - 1; c >= K; --c)
    if (pn[c] >= (T(1) - tau_piv) * mx) {
      p = c;
      sigma = pn[c];
    }
  // move the pivot column to position K
#pragma unroll
  for (int c = K + 1; c < M; ++c) {
    const bool sw = c == p;
#pragma unroll
    for (int r = 0; r < R; ++r) swap_if(sw, st.B[r][K], st.B[r][c]);
    swap_if(sw, st.inv_s[K], st.inv_s[c]);
    swap_if(sw, st.col[K], st.col[c]);
  }
  const T xk = __shfl_sync(kFull, st.B[K / G][K], K % G, G);
  const T nrm = sqrt(sigma);
  const T alpha = xk >= T(0) ? -nrm : nrm;
  const T vtv = T(2) * (sigma + fabs(xk) * nrm);
  const T tau = vtv > T(0) ? T(2) / vtv : T(0);
  const T vk = xk - alpha;
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = g + G * r;
    v[r] = row > K ? st.B[r][K] : (row == K ? vk : T(0));
  }
#pragma unroll
  for (int c = K + 1; c < M; ++c) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) s += v[r] * st.B[r][c];
    s = group_sum<G>(s) * tau;
#pragma unroll
    for (int r = 0; r < R; ++r) st.B[r][c] -= s * v[r];
  }
  {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) s += v[r] * st.rhs[r];
    s = group_sum<G>(s) * tau;
#pragma unroll
    for (int r = 0; r < R; ++r) st.rhs[r] -= s * v[r];
  }
  // R_KK on the owner lane; rows > K of column K keep the Householder vector
  if (g == K % G) st.B[K / G][K] = alpha;
  st.hv[K] = vk;
  st.ht[K] = tau;
  if (K == 0) st.r00 = fabs(alpha);
  if (st.rank == M && !(fabs(alpha) > rank_tol * st.r00)) st.rank = K;
}

// Row K of the back substitution R x = z (z in the rows' owner lanes),
// keeping only the first `rank` pivots.
template <int K, typename T, int M, int G, int R>
__device__ __forceinline__ void backsub_step(QRState<T, M, R>& st, const T (&z)[R], T (&x)[M]) {
  T t = z[K / G];
#pragma unroll
  for (int c = K + 1; c < M; ++c) t -= st.B[K / G][c] * x[c];
  const T rkk = st.B[K / G][K];
  T val = (K < st.rank && rkk != T(0)) ? t / rkk : T(0);
  x[K] = __shfl_sync(kFull, val, K % G, G);
}

// Q^T z for a new right-hand side with the stored Householder vectors.
template <int K, typename T, int M, int G, int R>
__device__ __forceinline__ void apply_qt_step(const QRState<T, M, R>& st, int g, T (&z)[R]) {
  T s = T(0);
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = g + G * r;
    v[r] = row > K ? st.B[r][K] : (row == K ? st.hv[K] : T(0));
    s += v[r] * z[r];
  }
  s = group_sum<G>(s) * st.ht[K];
#pragma unroll
  for (int r = 0; r < R; ++r) z[r] -= s * v[r];
}

template <typename T, int M, int G, int R, int... Ks>
__device__ __forceinline__ void factor(QRState<T, M, R>& st, int g, T tau_piv, T rank_tol,
                                       std::integer_sequence<int, Ks...>) {
  (qr_step<Ks, T, M, G, R>(st, g, tau_piv, rank_tol), ...);
}

template <typename T, int M, int G, int R, int... Ks>
__device__ __forceinline__ void solve_r(QRState<T, M, R>& st, const T (&z)[R], T (&x)[M],
                                        std::integer_sequence<int, Ks...>) {
  (backsub_step<M - 1 - Ks, T, M, G, R>(st, z, x), ...);
}

template <typename T, int M, int G, int R, int... Ks>
__device__ __forceinline__ void apply_qt(const QRState<T, M, R>& st, int g, T (&z)[R],
                                         std::integer_sequence<int, Ks...>) {
  (apply_qt_step<Ks, T, M, G, R>(st, g, z), ...);
}

// Shared memory per cell: the G*R sorted rows (M+1 values) and their
// stencil row indices.
template <typename T, int M, int G, int R>
constexpr size_t recon_smem_per_cell() {
  return static_cast<size_t>(G * R) * ((M + 1) * sizeof(T) + sizeof(int));
}

// One cell on the lanes of one group.  `listed`: the cell came from the work
// list of the thread-per-cell kernel; in FP32-bulk it is always refined.
template <typename T, int DIM, int M, int G, int R>
__device__ __forceinline__ void group_reconstruct_cell(
    const DeviceMesh& dm, const SchemeParams& sp, const double* WLSENO_BODY_RESTRICT ubar,
    double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev,
    unsigned long long* WLSENO_BODY_RESTRICT counters, unsigned char* smem_raw, int g, int gib,
    int64_t cell, bool valid, bool listed, const TraceOut& tr = TraceOut{}, int comp = 0) {
  constexpr int NF = DIM + 1;
  constexpr int NQ = nq_of(DIM);
  constexpr int NP = NF * NQ;
  constexpr int NR = G * R;
  constexpr bool kF32 = sizeof(T) == 4;
  const T tau_piv = kF32 ? T(1e-4) : T(1e-6);
  const int64_t ci = valid ? cell : 0;
  const int beg = dm.st_ptr[ci];
  const int n = valid ? dm.st_ptr[ci + 1] - beg : 0;
  const double ui = ubar[ci];
  const double hi = dm.h[ci];
  const T eh2 = static_cast<T>(sp.eps * hi * hi);

  // beta_i: the smallest beta over the cells sharing a facet with tau_i
  T bmin = T(INFINITY);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int nb = dm.nbr[ci * NF + f];
    if (nb >= 0) {
      const T d = static_cast<T>(ubar[nb >> 2] - ui);
      bmin = fmin(bmin, d * d + eh2);
    }
  }
  const T w_centre = static_cast<T>(sp.alpha_c) * eh2 / bmin;

  // rows of [W A | W (ubar_S - ubar_i)]
  QRState<T, M, R> st;
  const T* A = moment_array<T>(dm);
  T rn[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = g + G * r;
    if (row < n) {
      const int j = dm.st_idx[beg + row];
      const T dev = static_cast<T>(ubar[j] - ui);
      const T w = row == 0 ? w_centre : eh2 / (dev * dev + eh2);
      st.rhs[r] = w * dev;
      const T* a = A + static_cast<int64_t>(beg + row) * M;
#pragma unroll
      for (int c = 0; c < M; ++c) st.B[r][c] = w * a[c];
    } else {
      st.rhs[r] = T(0);
#pragma unroll
      for (int c = 0; c < M; ++c) st.B[r][c] = T(0);
    }
  }
  // S = diag(1 / ||column of W A||)
#pragma unroll
  for (int c = 0; c < M; ++c) {
    T s2 = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) s2 += st.B[r][c] * st.B[r][c];
    s2 = group_sum<G>(s2);
    st.inv_s[c] = s2 > T(0) ? T(1) / sqrt(s2) : T(0);
    st.col[c] = c;
#pragma unroll
    for (int r = 0; r < R; ++r) st.B[r][c] *= st.inv_s[c];
  }
  // sort the rows by decreasing norm (ties: stencil order).  A non-finite
  // norm sorts like a padding row (-1): the order must stay a strict total
  // order (value, then index) so that every slot of the sorted rows and of
  // their row indices is written
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < M; ++c) s += static_cast<float>(st.B[r][c]) * static_cast<float>(st.B[r][c]);
    rn[r] = g + G * r < n && s <= 3.0e38f ? s : -1.0f;
  }
  int rank_of[R];
#pragma unroll
  for (int r = 0; r < R; ++r) rank_of[r] = 0;
#pragma unroll
  for (int r2 = 0; r2 < R; ++r2) {
#pragma unroll
    for (int l = 0; l < G; ++l) {
      const float o = __shfl_sync(kFull, rn[r2], l, G);
      const int oi = l + G * r2;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int mi = g + G * r;
        rank_of[r] += (o > rn[r] || (o == rn[r] && oi < mi)) ? 1 : 0;
      }
    }
  }
  T* srow = reinterpret_cast<T*>(smem_raw) + static_cast<size_t>(gib) * NR * (M + 1);
  int* sidx = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(smem_raw) +
                                     static_cast<size_t>(blockDim.x / G) * NR * (M + 1) * sizeof(T)) +
              gib * NR;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T* dst = srow + rank_of[r] * (M + 1);
#pragma unroll
    for (int c = 0; c < M; ++c) dst[c] = st.B[r][c];
    dst[M] = st.rhs[r];
    sidx[rank_of[r]] = g + G * r;
  }
  __syncwarp();
  int myrow[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const T* src = srow + (g + G * r) * (M + 1);
#pragma unroll
    for (int c = 0; c < M; ++c) st.B[r][c] = src[c];
    st.rhs[r] = src[M];
    myrow[r] = sidx[g + G * r];
  }

  st.r00 = T(0);
  st.rlast = T(0);
  st.rank = M;
  factor<T, M, G, R>(st, g, tau_piv, static_cast<T>(sp.rank_tol), std::make_integer_sequence<int, M>{});
  solve_r<T, M, G, R>(st, st.rhs, st.y, std::make_integer_sequence<int, M>{});
  st.rlast = st.rank > 0 ? T(1) : T(0);
  {
    // |R_rr| of the last kept pivot, for the conditioning flag
    T rl = T(0);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const T rkk = __shfl_sync(kFull, st.B[k / G][k], k % G, G);
      if (k == st.rank - 1) rl = fabs(rkk);
    }
    st.rlast = rl;
  }
  const bool flagged = valid && (listed ? kF32 : (st.rank > 0 && st.r00 > static_cast<T>(sp.kappa_flag) * st.rlast));

  // FP32-bulk: one refinement sweep with the FP64 residual on flagged cells
  T dy[M];
#pragma unroll
  for (int c = 0; c < M; ++c) dy[c] = T(0);
  if (kF32 && __any_sync(kFull, flagged)) {
    double vpos[M];
#pragma unroll
    for (int c = 0; c < M; ++c) vpos[c] = static_cast<double>(st.y[c]) * static_cast<double>(st.inv_s[c]);
    double vorig[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < M; ++k) v = st.col[k] == c ? vpos[k] : v;
      vorig[c] = v;
    }
    // the residual of the FP64 problem: FP64 weights, moments and deviations
    // (the FP32 factors only precondition the correction)
    const double eh2d = sp.eps * hi * hi;
    double bmind = INFINITY;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int nb = dm.nbr[ci * NF + f];
      if (nb >= 0) {
        const double d = ubar[nb >> 2] - ui;
        bmind = fmin(bmind, d * d + eh2d);
      }
    }
    T z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      z[r] = T(0);
      const int row = myrow[r];
      if (flagged && static_cast<unsigned>(row) < static_cast<unsigned>(n)) {
        const int j = dm.st_idx[beg + row];
        const double dev = ubar[j] - ui;
        const double w = row == 0 ? sp.alpha_c * eh2d / bmind : eh2d / (dev * dev + eh2d);
        const double* a = dm.A64 + static_cast<int64_t>(beg + row) * M;
        double fit = 0.0;
#pragma unroll
        for (int c = 0; c < M; ++c) fit += a[c] * vorig[c];
        z[r] = static_cast<T>(w * (dev - fit));
      }
    }
    apply_qt<T, M, G, R>(st, g, z, std::make_integer_sequence<int, M>{});
    solve_r<T, M, G, R>(st, z, dy, std::make_integer_sequence<int, M>{});
  }

  if (!valid) return;
  // coefficients back in the original column order: d = S y (+ S dy)
  T chi[M], clo[M];
#pragma unroll
  for (int c = 0; c < M; ++c) {
    T h = T(0), l = T(0);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const bool sel = st.col[k] == c;
      h = sel ? st.y[k] * st.inv_s[k] : h;
      l = sel ? dy[k] * st.inv_s[k] : l;
    }
    chi[c] = h;
    clo[c] = l;
  }
  if (coeffs) {
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c % G == g)
        coeffs[cell * M + c] = static_cast<double>(chi[c]) + static_cast<double>(clo[c]) + (c == 0 ? ui : 0.0);
  }
  const T* P = facet_point_array<T>(dm) + cell * NP * DIM;
  bool finite = true;
#pragma unroll
  for (int pt = 0; pt < NP; ++pt) {
    if (pt % G != g) continue;
    T yy[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) yy[a] = P[pt * DIM + a];
    T mono[M];
    eval_monomials<T, DIM, M>(yy, mono);
    T sh = T(0), sl = T(0);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      sh += chi[c] * mono[c];
      sl += clo[c] * mono[c];
    }
    if (tr.base) {
      // the component's trace, in a cell whose traces are used
      const float dv = static_cast<float>(sh) + static_cast<float>(sl);
      constexpr int TC = DIM + 2;
      if (tr.pos_ok[cell]) {
        const float2 pc = tr.upair[cell * TC + comp];
        tr.base[(cell * NP + pt) * TC + comp] = pc.x + (pc.y + dv);
      }
      finite = finite && isfinite(dv);
    } else if (fdev) {
      const float dv = static_cast<float>(sh) + static_cast<float>(sl);
      fdev[cell * NP + pt] = dv;
      finite = finite && isfinite(dv);
    } else {
      const double val = ui + static_cast<double>(sh) + static_cast<double>(sl);
      fvals[cell * NP + pt] = val;
      finite = finite && isfinite(val);
    }
  }
  if (!finite) report_nonfinite(dm, counters);
  if (g == 0) {
    if (st.rank < M) atomicAdd(&counters[1], 1ull);
    if (flagged && !listed) atomicAdd(&counters[0], 1ull);
  }
}

template <typename T, int DIM, int M, int G, int R>
__global__ void __launch_bounds__(128)
reconstruct_kernel(DeviceMesh dm, SchemeParams sp, const double* WLSENO_BODY_RESTRICT ubar,
                   double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev,
                   unsigned long long* WLSENO_BODY_RESTRICT counters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t cell = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) / G;
  group_reconstruct_cell<T, DIM, M, G, R>(dm, sp, ubar, coeffs, fvals, fdev, counters, smem_raw,
                                          threadIdx.x % G, threadIdx.x / G, cell < dm.N ? cell : 0,
                                          cell < dm.N, false);
}

// The work-listed cells of the thread-per-cell kernel (pivoted path, and in
// FP32-bulk the refinement sweep), grid-stride over the list.
// The listed cells for block `block` of `nblocks` (the kernel's body and the
// pivoted phase of the persistent step); smem_raw holds
// recon_smem_per_cell<T, M, G, R>() * (blockDim.x / G) bytes.
template <typename T, int DIM, int M, int G, int R>
__device__ __forceinline__ void reconstruct_listed(const DeviceMesh& dm, const SchemeParams& sp,
                                                   const double* WLSENO_BODY_RESTRICT ubar, double* WLSENO_BODY_RESTRICT coeffs,
                                                   double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev,
                                                   unsigned long long* WLSENO_BODY_RESTRICT counters,
                                                   const int* WLSENO_BODY_RESTRICT worklist, const int* WLSENO_BODY_RESTRICT wl_count,
                                                   unsigned char* smem_raw, int64_t block, int64_t nblocks,
                                                   const TraceOut& tr = TraceOut{}) {
  const int count = *reinterpret_cast<const volatile int*>(wl_count);
  const int gpb = blockDim.x / G;
  const int gib = threadIdx.x / G;
  for (int64_t base = block * gpb; base < count; base += nblocks * gpb) {
    __syncwarp();
    const int idx = base + gib;
    const bool valid = idx < count;
    // list entries c N + i: component c (multi-component contexts), cell i
    const int64_t tag = valid ? worklist[idx] : 0;
    const int64_t comp = tag >= dm.N ? tag / dm.N : 0;
    const int64_t cell = tag - comp * dm.N;
    constexpr int NP = (DIM + 1) * nq_of(DIM);
    const int64_t off = comp * dm.N;
    group_reconstruct_cell<T, DIM, M, G, R>(dm, sp, ubar + off, coeffs ? coeffs + off * M : nullptr,
                                            fvals ? fvals + off * NP : nullptr,
                                            fdev && !tr.base ? fdev + off * NP : nullptr, counters, smem_raw,
                                            threadIdx.x % G, gib, cell, valid, true, tr, static_cast<int>(comp));
  }
}

template <typename T, int DIM, int M, int G, int R>
__global__ void __launch_bounds__(128)
reconstruct_list_kernel(DeviceMesh dm, SchemeParams sp, const double* WLSENO_BODY_RESTRICT ubar,
                        double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev,
                        unsigned long long* WLSENO_BODY_RESTRICT counters, const int* WLSENO_BODY_RESTRICT worklist,
                        const int* WLSENO_BODY_RESTRICT wl_count, TraceOut tr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  reconstruct_listed<T, DIM, M, G, R>(dm, sp, ubar, coeffs, fvals, fdev, counters, worklist, wl_count, smem_raw,
                                      blockIdx.x, gridDim.x, tr);
}

template <typename T, int DIM, int M, int G, int R>
cudaError_t launch_reconstruct_list(const DeviceMesh& dm, const SchemeParams& sp,
                                    const double* ubar, const ReconOut& out, const int* worklist,
                                    const int* wl_count, cudaStream_t s, const TraceOut& tr = TraceOut{}) {
  constexpr int threads = 128;
  const size_t smem = recon_smem_per_cell<T, M, G, R>() * (threads / G);
  // set before every launch: the attribute belongs to the current device's
  // context, so a flag kept per process would miss a second device
  cudaError_t e = cudaFuncSetAttribute(reconstruct_list_kernel<T, DIM, M, G, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  // a few blocks per SM: the list is short (and usually empty)
  const int64_t groups = (dm.N * G + threads - 1) / threads;
  const unsigned blocks = static_cast<unsigned>(groups < 152 * 2 ? groups : 152 * 2);
  reconstruct_list_kernel<T, DIM, M, G, R><<<blocks, threads, smem, s>>>(
      dm, sp, ubar, out.coeffs, out.fvals, out.fdev, out.counters, worklist, wl_count, tr);
  return cudaGetLastError();
}

template <typename T, int DIM, int M, int G, int R>
cudaError_t launch_reconstruct_shape(const DeviceMesh& dm, const SchemeParams& sp,
                                     const double* ubar, const ReconOut& out, cudaStream_t s) {
  constexpr int threads = 128;
  const size_t smem = recon_smem_per_cell<T, M, G, R>() * (threads / G);
  // set before every launch (per device, see launch_reconstruct_list)
  cudaError_t e = cudaFuncSetAttribute(reconstruct_kernel<T, DIM, M, G, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t total = dm.N * G;
  const unsigned blocks = static_cast<unsigned>((total + threads - 1) / threads);
  reconstruct_kernel<T, DIM, M, G, R>
      <<<blocks, threads, smem, s>>>(dm, sp, ubar, out.coeffs, out.fvals, out.fdev, out.counters);
  return cudaGetLastError();
}

// Shapes compiled for every (T, DIM, M): lanes per cell G, rows per lane R.
#define WLSENO_FOR_EACH_SHAPE(X) X(8, 2) X(8, 3) X(8, 5) X(16, 3) X(16, 4)

template <typename T, int DIM, int M>
cudaError_t launch_reconstruct_tm(const DeviceMesh& dm, const SchemeParams& sp, int G, int R,
                                  const double* ubar, const ReconOut& out, cudaStream_t s) {
#define WLSENO_SHAPE_CASE(GG, RR) \
  if (G == GG && R == RR) return launch_reconstruct_shape<T, DIM, M, GG, RR>(dm, sp, ubar, out, s);
  WLSENO_FOR_EACH_SHAPE(WLSENO_SHAPE_CASE)
#undef WLSENO_SHAPE_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace wlseno
