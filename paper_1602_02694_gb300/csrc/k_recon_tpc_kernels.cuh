// Thread-per-cell reconstruction kernels (the fold is in k_recon_tpc.cuh).
//
// Main kernel: fold the stencil rows into the square-root-free factor of
// W A = Q R, solve R d = Q^T W (ubar_S - ubar_i), and estimate the
// conditioning of W A S from the column-scaled diagonal of R.  For a
// full-rank system this d is the least-squares solution the paper's QR with
// column pivoting returns (Sec. 3.3.2).  Cells whose estimate exceeds the
// flag threshold -- where pivoting and rank truncation could matter, and in
// FP32-bulk mode where a refinement is due -- go to a work list.
//
// Work-listed cells are then redone by the lane-group kernel (rows spread over
// the lanes of a group, so their loads run in parallel): the paper's path in
// full -- column scaling, QR with column pivoting, numerical rank, basic
// solution -- and, in FP32-bulk mode, one refinement sweep with the FP64
// residual (FP64 weights and moments).  It overwrites the main kernel's
// outputs for those cells.
#pragma once

#include "k_recon_tpc.cuh"
#include "k_reconstruct.cuh"

namespace wlseno {

// FP64 fold: rows read from the ELL layout, row t+1 fetched while row t is
// folded (hides the index -> ubar chain).
template <int DIM, int M>
__device__ __forceinline__ void tpc_fold(const DeviceMesh& dm, const double* __restrict__ ubar,
                                         int64_t i, double ui, int n, double eh2, double w_centre,
                                         SqrtFreeQR<double, M>& f) {
  const int64_t N = dm.N;
  const double* Ae = dm.A64e;
  sqrt_free_init(f);
  double u_next = ubar[dm.st_ell[i]];
  double a_next[M];
#pragma unroll
  for (int c = 0; c < M; ++c) a_next[c] = Ae[static_cast<int64_t>(c) * N + i];
  for (int t = 0; t < n; ++t) {
    const double dev = u_next - ui;
    double z[M + 1];
#pragma unroll
    for (int c = 0; c < M; ++c) z[c] = a_next[c];
    if (t + 1 < n) {
      u_next = ubar[dm.st_ell[(t + 1) * N + i]];
#pragma unroll
      for (int c = 0; c < M; ++c) a_next[c] = Ae[(static_cast<int64_t>(t + 1) * M + c) * N + i];
    }
    const double w = t == 0 ? w_centre : eh2 * recip_t(fma(dev, dev, eh2));
    z[M] = dev;
    sqrt_free_fold(f, z, w * w);
  }
}

constexpr int kTpcThreads = 128;  // block size of the thread-per-cell kernels

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kPending) : "memory");
}

// FP32 fold with the rows staged through shared memory.  Each thread copies
// its own rows asynchronously: the row record (moments + stencil index) four
// rows ahead, and ubar_j two rows ahead (its index read from the staged
// record), so neither the HBM latency of the records nor the record -> index
// -> ubar chain stalls the rotations, and no prefetched row occupies
// registers.  Commit groups: one per iteration t, holding ubar of row t+2 and
// the record of row t+4; waiting for all but the newest group therefore
// guarantees the record and ubar of row t and the record of row t+2.  Record
// slots cycle mod 5 and ubar slots mod 3, so a copy never lands in a slot
// whose previous row is still to be read.  Threads touch only their own
// slots: no block barrier.
template <int DIM, int M>
__device__ __forceinline__ void tpc_fold_staged(const DeviceMesh& dm, const double* __restrict__ ubar,
                                                int64_t i, double ui, int n, float eh2, float w_centre,
                                                SqrtFreeQR<float, M>& f) {
  constexpr int W4 = rec32_width(M) / 4;
  constexpr int kRec = 5, kU = 3;
  __shared__ float4 srec[kRec][W4][kTpcThreads];
  __shared__ double su[kU][kTpcThreads];
  const int tid = threadIdx.x;
  const int64_t N = dm.N;
  const float4* rec = reinterpret_cast<const float4*>(dm.rec32);
  auto fetch_rec = [&](int t, int slot) {
    const float4* src = rec + (static_cast<int64_t>(t) * N + i) * W4;
#pragma unroll
    for (int k = 0; k < W4; ++k) cp_async16(&srec[slot][k][tid], src + k);
  };
  auto fetch_u = [&](int rec_slot, int u_slot) {
    const int j = __float_as_int(reinterpret_cast<const float*>(&srec[rec_slot][M / 4][tid])[M % 4]);
    cp_async8(&su[u_slot][tid], ubar + j);
  };
  sqrt_free_init(f);
  for (int t = 0; t < 4 && t < n; ++t) fetch_rec(t, t);
  cp_async_commit();
  cp_async_wait<0>();
  for (int t = 0; t < 2 && t < n; ++t) fetch_u(t, t);
  cp_async_commit();
  cp_async_commit();  // empty: the first wait below then covers the ubar copies
  int sr = 0, sv = 0;  // slots of row t
  for (int t = 0; t < n; ++t) {
    cp_async_wait<1>();
    float z[M + 1];
#pragma unroll
    for (int k = 0; k < W4; ++k) {
      const float4 v = srec[sr][k][tid];
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * k + q < M) z[4 * k + q] = vv[q];
    }
    const double uj = su[sv][tid];
    const int sr2 = sr + 2 < kRec ? sr + 2 : sr + 2 - kRec;
    const int sr4 = sr + 4 < kRec ? sr + 4 : sr + 4 - kRec;
    const int sv2 = sv + 2 < kU ? sv + 2 : sv + 2 - kU;
    if (t + 2 < n) fetch_u(sr2, sv2);
    if (t + 4 < n) fetch_rec(t + 4, sr4);
    cp_async_commit();
    const float dev = static_cast<float>(uj - ui);
    const float w = t == 0 ? w_centre : eh2 * recip_t(fmaf(dev, dev, eh2));
    z[M] = dev;
    sqrt_free_fold(f, z, w * w);
    sr = sr + 1 < kRec ? sr + 1 : 0;
    sv = sv + 1 < kU ? sv + 1 : 0;
  }
  cp_async_wait<0>();
}

// Coefficients and facet values of cell i (FP32-bulk: the polynomial in FP32,
// ubar_i added in FP64).
template <typename T, int DIM, int M>
__device__ __forceinline__ void tpc_write(const DeviceMesh& dm, int64_t i, double ui, const T (&x)[M],
                                          double* __restrict__ coeffs, double* __restrict__ fvals) {
  constexpr int NP = (DIM + 1) * (DIM == 2 ? 2 : 3);
  if (coeffs) {
#pragma unroll
    for (int c = 0; c < M; ++c) coeffs[i * M + c] = static_cast<double>(x[c]) + (c == 0 ? ui : 0.0);
  }
  const T* P = tpc_points<T>(dm) + i * NP * DIM;
#pragma unroll
  for (int pt = 0; pt < NP; ++pt) {
    T yy[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) yy[a] = P[pt * DIM + a];
    T mono[M];
    eval_monomials<T, DIM, M>(yy, mono);
    T sh = T(0);
#pragma unroll
    for (int c = 0; c < M; ++c) sh = fma(x[c], mono[c], sh);
    fvals[i * NP + pt] = ui + static_cast<double>(sh);
  }
}

template <typename T, int DIM, int M>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1)
recon_tpc_kernel(DeviceMesh dm, SchemeParams sp, const double* __restrict__ ubar,
                 double* __restrict__ coeffs, double* __restrict__ fvals,
                 unsigned long long* __restrict__ counters, int* __restrict__ worklist,
                 int* __restrict__ wl_count, T flag_threshold) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  const int n = dm.st_ptr[i + 1] - dm.st_ptr[i];
  const double ui = ubar[i];
  T eh2, wc;
  tpc_weights<T, DIM>(dm, sp, ubar, i, ui, &eh2, &wc);
  SqrtFreeQR<T, M> f;
  if constexpr (sizeof(T) == 4)
    tpc_fold_staged<DIM, M>(dm, ubar, i, ui, n, eh2, wc, f);
  else
    tpc_fold<DIM, M>(dm, ubar, i, ui, n, eh2, wc, f);
  const bool flagged = sqrt_free_ill_conditioned(f, flag_threshold);
  T d[M];
  sqrt_free_solve(f, d);
  tpc_write<T, DIM, M>(dm, i, ui, d, coeffs, fvals);
  if (flagged) {
    if (sizeof(T) == 4) atomicAdd(&counters[0], 1ull);
    worklist[atomicAdd(wl_count, 1)] = static_cast<int>(i);
  }
}

template <typename T, int DIM, int M>
cudaError_t launch_recon_tpc(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                             const ReconOut& out, int* worklist, int* wl_count, cudaStream_t s,
                             int* launches) {
  constexpr int threads = kTpcThreads;
  const unsigned blocks = static_cast<unsigned>((dm.N + threads - 1) / threads);
  // FP32-bulk: refine above kappa_flag; FP64: take the pivoted path above 1e6
  const T threshold = sizeof(T) == 4 ? static_cast<T>(sp.kappa_flag) : T(1e6);
  *launches = 0;
  cudaError_t e = cudaMemsetAsync(wl_count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  recon_tpc_kernel<T, DIM, M><<<blocks, threads, 0, s>>>(dm, sp, ubar, out.coeffs, out.fvals,
                                                        out.counters, worklist, wl_count, threshold);
  ++*launches;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the listed cells, one lane group each: rows spread over the lanes
  if (dm.nmax <= 40)
    e = launch_reconstruct_list<T, DIM, M, 8, 5>(dm, sp, ubar, out, worklist, wl_count, s);
  else
    e = launch_reconstruct_list<T, DIM, M, 16, 4>(dm, sp, ubar, out, worklist, wl_count, s);
  ++*launches;
  return e;
}

}  // namespace wlseno
