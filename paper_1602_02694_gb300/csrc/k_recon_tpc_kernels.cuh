// Thread-per-cell reconstruction kernels (the fold is in k_recon_tpc.cuh).
//
// Main kernel: fold the stencil rows into the square-root-free factor of
// W A = Q R, solve R d = Q^T W (ubar_S - ubar_i), and estimate the
// conditioning of W A S from the column-scaled diagonal of R.  For a
// full-rank system this d is the least-squares solution the paper's QR with
// column pivoting returns (Sec. 3.3.2).  In FP32-bulk mode the rows are
// either streamed from stored records or formed on the fly from each stencil
// cell's offset and own central moments (moments mode 1).  Cells whose
// estimate exceeds the flag threshold -- where pivoting and rank truncation
// could matter, and in FP32-bulk mode where a refinement is due -- go to a
// refine record or a work list.
//
// Refine records are finished by one sweep with the FP64 residual
// (refine_kernel).  Work-listed cells are redone by the lane-group kernel
// (rows spread over the lanes of a group, so their loads run in parallel):
// the paper's path in full -- column scaling, QR with column pivoting,
// numerical rank, basic solution -- and, in FP32-bulk mode, one refinement
// sweep with the FP64 residual (FP64 weights and moments).  Both overwrite
// the main kernel's outputs for their cells.
#pragma once

#include "k_recon_tpc.cuh"
#include "k_reconstruct.cuh"

namespace wlseno {

// FP64 fold: rows read from the ELL layout, row t+1 fetched while row t is
// folded (hides the index -> ubar chain).
template <int DIM, int M>
__device__ __forceinline__ void tpc_fold(const DeviceMesh& dm, const double* WLSENO_BODY_RESTRICT ubar,
                                         int64_t i, double ui, int n, double eh2, double w_centre,
                                         SqrtFreeQR<double, M>& f, double* w_spread = nullptr) {
  const int64_t N = dm.N;
  const double* Ae = dm.A64e;
  sqrt_free_init(f);
  double wmin = INFINITY, wmax = 0.0;
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
    wmin = fmin(wmin, w);
    wmax = fmax(wmax, w);
    z[M] = dev;
    sqrt_free_fold(f, z, w * w);
  }
  if (w_spread) *w_spread = wmax / wmin;  // NaN for non-finite weights: fails the caller's <= test
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

// FP32 fold with the rows staged through shared memory.  Each cell's rows
// are copied asynchronously: the row record (moments + stencil index) kLeadR
// rows ahead, and the FP32 pair of ubar_j kLeadU rows ahead (its index read
// from the staged record), so neither the HBM latency of the records nor the
// record -> index -> ubar chain stalls the rotations, and no prefetched row
// occupies registers.  Commit groups: one per iteration t, holding ubar of row
// t+kLeadU and the record of row t+kLeadR.  Iteration t needs the groups of
// iterations t-kLeadU (ubar of row t) and t+kLeadU-kLeadR (record of row
// t+kLeadU), so all but the newest kPending groups must be complete.  Record
// slots cycle mod kLeadR+1 and ubar slots mod kLeadU+1, so a copy never lands
// in a slot whose previous row is still to be read; the row loop is unrolled
// by a common multiple of both, so every slot is a compile-time constant.
// With C > 1 the C threads of a cell share one record slot (each copies part
// of the record) and order their copies with a barrier over the cell's lanes;
// the ubar pairs stay per thread (the all-components kernel folds its stored
// rows with tpc_fold_chunked below instead).  No block barrier.
constexpr int kLeadR = 7, kLeadU = 3, kUnrollS = 8;
constexpr int kPending = (kLeadU - 1) < (kLeadR - kLeadU - 1) ? (kLeadU - 1) : (kLeadR - kLeadU - 1);
static_assert(kPending >= 0 && kLeadR > kLeadU && kLeadU >= 1, "prefetch leads");
static_assert(kUnrollS % (kLeadR + 1) == 0 && kUnrollS % (kLeadU + 1) == 0, "unroll by whole slot cycles");

// Lanes of the C threads of this thread's cell (C divides 32).
template <int C>
__device__ __forceinline__ unsigned cell_lanes() {
  const unsigned lane = threadIdx.x & 31u;
  return C == 1 ? (1u << lane) : (((1u << C) - 1u) << (lane & ~static_cast<unsigned>(C - 1)));
}

// weights(&eh2, &w_centre) computes the cell's weights; it runs after the
// first record copies are issued, so its gathers overlap them.
template <int DIM, int M, int C = 1, typename WFn>
__device__ __forceinline__ void tpc_fold_staged(const DeviceMesh& dm, const float2* WLSENO_BODY_RESTRICT upair,
                                                int64_t i, float2 pi, int n, WFn&& weights, float* eh2_out,
                                                float* wc_out, SqrtFreeQR<float, M>& f) {
  constexpr int W4 = rec32_width(M) / 4;
  constexpr int kRec = kLeadR + 1, kU = kLeadU + 1, kCells = kTpcThreads / C;
  __shared__ float4 srec[kRec][W4][kCells];
  __shared__ float2 su[kU][kTpcThreads];
  const int tid = threadIdx.x;
  const int cell = tid / C, part = tid % C;
  const unsigned lanes = cell_lanes<C>();
  const int64_t N = dm.N;
  const float4* rec = reinterpret_cast<const float4*>(dm.rec32);
  auto fetch_rec = [&](int t, int slot) {
    const float4* src = rec + (static_cast<int64_t>(t) * N + i) * W4;
#pragma unroll
    for (int k = 0; k < W4; ++k)
      if (k % C == part) cp_async16(&srec[slot][k][cell], src + k);
  };
  auto fetch_u = [&](int rec_slot, int u_slot) {
    const int j = __float_as_int(reinterpret_cast<const float*>(&srec[rec_slot][M / 4][cell])[M % 4]);
    cp_async8(&su[u_slot][tid], upair + static_cast<int64_t>(j) * C);
  };
  sqrt_free_init(f);
  for (int t = 0; t < kLeadR && t < n; ++t) fetch_rec(t, t);
  cp_async_commit();
  float eh2, w_centre;
  weights(&eh2, &w_centre);
  *eh2_out = eh2;
  *wc_out = w_centre;
  cp_async_wait<0>();
  if (C > 1) __syncwarp(lanes);
  for (int t = 0; t < kLeadU && t < n; ++t) fetch_u(t, t);
  cp_async_commit();
  // empty groups: the first waits below then cover the ubar copies
#pragma unroll
  for (int k = 0; k < kPending; ++k) cp_async_commit();
  for (int t0 = 0; t0 < n; t0 += kUnrollS) {
#pragma unroll
    for (int s = 0; s < kUnrollS; ++s) {
      const int t = t0 + s;
      if (t >= n) break;
      const int sr = s % kRec, sv = s % kU;  // slots of row t
      cp_async_wait<kPending>();
      // the cell's other lanes' record copies; every lane has also read row
      // t-1 (the slot the record copy below overwrites)
      if (C > 1) __syncwarp(lanes);
      float z[M + 1];
#pragma unroll
      for (int k = 0; k < W4; ++k) {
        const float4 v = srec[sr][k][cell];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (4 * k + q < M) z[4 * k + q] = vv[q];
      }
      const float2 pj = su[sv][tid];
      if (t + kLeadU < n) fetch_u((s + kLeadU) % kRec, (s + kLeadU) % kU);
      if (t + kLeadR < n) fetch_rec(t + kLeadR, (s + kLeadR) % kRec);
      cp_async_commit();
      const float dev = (pj.x - pi.x) + (pj.y - pi.y);  // ubar_j - ubar_i
      const float w = t == 0 ? w_centre : eh2 * recip_t(fmaf(dev, dev, eh2));
      z[M] = dev;
      sqrt_free_fold(f, z, w * w);
    }
  }
  cp_async_wait<0>();
}

// The FP32 fold of tpc_fold_staged for C > 1 lanes per cell, in chunks of
// kChunk rows: a chunk's rows are folded as one straight-line block (no
// branch between them, so the compiler can overlap one row's rotations with
// the next row's), and the copies, waits and barriers are per chunk rather
// than per row.  Records of chunks c+1 and c+2 and the ubar pairs of chunk
// c+1 are in flight while chunk c is folded: three record slots (shared by
// the cell's lanes, each lane copying part of them) and two ubar slots (per
// thread).  At the start of chunk c every copy issued so far has landed (the
// copies of chunk c-1's iteration had a whole chunk of rotations to arrive),
// and the barrier over the cell's lanes orders their reads of chunk c-1's
// record slot before the copy that reuses it.  A last partial chunk folds its
// rows one by one.
constexpr int kChunk = 4;

template <int DIM, int M, int C, typename WFn>
__device__ __forceinline__ void tpc_fold_chunked(const DeviceMesh& dm, const float2* WLSENO_BODY_RESTRICT upair,
                                                 int64_t i, float2 pi, int n, WFn&& weights, float* eh2_out,
                                                 float* wc_out, SqrtFreeQR<float, M>& f) {
  static_assert(C > 1, "records shared by a cell's lanes");
  constexpr int W4 = rec32_width(M) / 4;
  constexpr int kCells = kTpcThreads / C, kPieces = kChunk * W4;
  __shared__ float4 srec[3][kChunk][W4][kCells];
  __shared__ float2 su[2][kChunk][kTpcThreads];
  const int tid = threadIdx.x;
  const int cell = tid / C, part = tid % C;
  const unsigned lanes = cell_lanes<C>();
  const int64_t stride = dm.N * W4;  // float4s between rows t and t+1 of a cell
  const float4* rec = reinterpret_cast<const float4*>(dm.rec32) + i * W4;
  // records of the rows of chunk c below n (16-byte pieces spread over the
  // cell's lanes) into record slot c % 3
  auto fetch_rec = [&](int c) {
    const int slot = c % 3;
#pragma unroll
    for (int q0 = 0; q0 < kPieces; q0 += C) {
      const int q = q0 + part, r = q / W4, k = q % W4, t = c * kChunk + r;
      if (q < kPieces && t < n) cp_async16(&srec[slot][r][k][cell], rec + t * stride + k);
    }
  };
  // ubar pairs of the rows of chunk c below n into ubar slot c % 2 (their
  // indices from the chunk's records)
  auto fetch_u = [&](int c) {
    const int slot = c % 3, us = c % 2;
#pragma unroll
    for (int r = 0; r < kChunk; ++r) {
      if (c * kChunk + r < n) {
        const int j = __float_as_int(reinterpret_cast<const float*>(&srec[slot][r][M / 4][cell])[M % 4]);
        cp_async8(&su[us][r][tid], upair + static_cast<int64_t>(j) * C);
      }
    }
  };
  sqrt_free_init(f);
  fetch_rec(0);
  fetch_rec(1);
  cp_async_commit();
  float eh2, w_centre;
  weights(&eh2, &w_centre);
  *eh2_out = eh2;
  *wc_out = w_centre;
  // one row: deviation, weight (Sec. 3.1.2), rotations
  auto fold_row = [&](int slot, int us, int r, int t) {
    float z[M + 1];
#pragma unroll
    for (int k = 0; k < W4; ++k) {
      const float4 v = srec[slot][r][k][cell];
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * k + q < M) z[4 * k + q] = vv[q];
    }
    const float2 pj = su[us][r][tid];
    const float dev = (pj.x - pi.x) + (pj.y - pi.y);  // ubar_j - ubar_i
    const float w = t == 0 ? w_centre : eh2 * recip_t(fmaf(dev, dev, eh2));
    z[M] = dev;
    sqrt_free_fold(f, z, w * w);
  };
  // the centre row (row 0, the cell itself: ubar_j - ubar_i = 0), the first
  // row folded
  auto fold_centre = [&]() {
    float z[M + 1];
#pragma unroll
    for (int k = 0; k < W4; ++k) {
      const float4 v = srec[0][0][k][cell];
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * k + q < M) z[4 * k + q] = vv[q];
    }
    z[M] = 0.0f;
    sqrt_free_fold_first(f, z, w_centre * w_centre);
  };
  cp_async_wait<0>();
  __syncwarp(lanes);
  fetch_u(0);
  cp_async_commit();
  const int nchunks = (n + kChunk - 1) / kChunk;
  for (int c = 0; c < nchunks; ++c) {
    cp_async_wait<0>();
    __syncwarp(lanes);
    if ((c + 1) * kChunk < n) fetch_u(c + 1);
    if ((c + 2) * kChunk < n) fetch_rec(c + 2);
    cp_async_commit();
    const int slot = c % 3, us = c % 2, t0 = c * kChunk;
    if (c == 0 && kChunk <= n) {
      fold_centre();
#pragma unroll
      for (int r = 1; r < kChunk; ++r) fold_row(0, 0, r, r);
    } else if (t0 + kChunk <= n) {
#pragma unroll
      for (int r = 0; r < kChunk; ++r) fold_row(slot, us, r, t0 + r);
    } else {
      for (int r = 0; r < n - t0; ++r) fold_row(slot, us, r, t0 + r);
    }
  }
}

// The FP32 fold of tpc_fold_staged with the rows formed on the fly: the
// 16-byte geometry record (offset and index) kLeadR rows ahead, and the pair
// of ubar_j with cell j's own moments kLeadU rows ahead, through the same
// commit-group schedule (with C > 1 the geometry record and cell j's moments
// shared by the cell's lanes, the pairs per thread).
template <int DIM, int M, int C = 1, typename WFn>
__device__ __forceinline__ void tpc_fold_staged_otf(const DeviceMesh& dm, const float2* WLSENO_BODY_RESTRICT upair,
                                                    int64_t i, float2 pi, int n, WFn&& weights, float* eh2_out,
                                                    float* wc_out, SqrtFreeQR<float, M>& f) {
  constexpr int OW4 = own32_width(DIM, M) / 4;
  // the 16-byte geometry records allow a deeper lead than the stored rows
  constexpr int kLeadRo = 7, kRec = kLeadRo + 1, kU = kLeadU + 1, kUnrollO = 8;
  constexpr int kPendingO = (kLeadU - 1) < (kLeadRo - kLeadU - 1) ? (kLeadU - 1) : (kLeadRo - kLeadU - 1);
  static_assert(kUnrollO % kRec == 0 && kUnrollO % kU == 0, "unroll by whole slot cycles");
  constexpr int kCells = kTpcThreads / C;
  __shared__ float4 sgeo[kRec][kCells];
  __shared__ float4 sown[kU][OW4][kCells];
  __shared__ float2 su[kU][kTpcThreads];
  const int tid = threadIdx.x;
  const int cell = tid / C, part = tid % C;
  const unsigned lanes = cell_lanes<C>();
  const int64_t N = dm.N;
  const float4* geo = reinterpret_cast<const float4*>(dm.geo32);
  const float4* own = reinterpret_cast<const float4*>(dm.own32);
  float hp[5];
  hp[0] = 1.0f;
  hp[1] = dm.hscale32 ? dm.hscale32[i].y : static_cast<float>(1.0 / dm.h[i]);  // 1/h_i (FP32, from the host)
#pragma unroll
  for (int k = 2; k < 5; ++k) hp[k] = hp[k - 1] * hp[1];
  auto fetch_rec = [&](int t, int slot) {
    if (part == 0) cp_async16(&sgeo[slot][cell], geo + static_cast<int64_t>(t) * N + i);
  };
  auto fetch_u = [&](int rec_slot, int u_slot) {
    const int j = __float_as_int(reinterpret_cast<const float*>(&sgeo[rec_slot][cell])[DIM]);
    cp_async8(&su[u_slot][tid], upair + static_cast<int64_t>(j) * C);
#pragma unroll
    for (int k = 0; k < OW4; ++k)
      if (k % C == part) cp_async16(&sown[u_slot][k][cell], own + static_cast<int64_t>(j) * OW4 + k);
  };
  sqrt_free_init(f);
  for (int t = 0; t < kLeadRo && t < n; ++t) fetch_rec(t, t);
  cp_async_commit();
  float eh2, w_centre;
  weights(&eh2, &w_centre);
  *eh2_out = eh2;
  *wc_out = w_centre;
  cp_async_wait<0>();
  if (C > 1) __syncwarp(lanes);
  for (int t = 0; t < kLeadU && t < n; ++t) fetch_u(t, t);
  cp_async_commit();
#pragma unroll
  for (int k = 0; k < kPendingO; ++k) cp_async_commit();
  // unrolled by a common multiple of both slot counts: every slot, and so
  // every shared-memory address, is a compile-time constant
  for (int t0 = 0; t0 < n; t0 += kUnrollO) {
#pragma unroll
    for (int s = 0; s < kUnrollO; ++s) {
      const int t = t0 + s;
      if (t >= n) break;
      const int sr = s % kRec, sv = s % kU;  // slots of row t
      cp_async_wait<kPendingO>();
      if (C > 1) __syncwarp(lanes);  // as in tpc_fold_staged
      const float4 gv = sgeo[sr][cell];
      const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
      float d[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) d[a] = gg[a];
      float ow[OW4 * 4];
#pragma unroll
      for (int k = 0; k < OW4; ++k) {
        const float4 v = sown[sv][k][cell];
        ow[4 * k] = v.x;
        ow[4 * k + 1] = v.y;
        ow[4 * k + 2] = v.z;
        ow[4 * k + 3] = v.w;
      }
      const float2 pj = su[sv][tid];
      if (t + kLeadU < n) fetch_u((s + kLeadU) % kRec, (s + kLeadU) % kU);
      if (t + kLeadRo < n) fetch_rec(t + kLeadRo, (s + kLeadRo) % kRec);
      cp_async_commit();
      float z[M + 1];
      float row[M];
      shifted_row<DIM, M>(d, hp, ow, row);
#pragma unroll
      for (int c = 0; c < M; ++c) z[c] = row[c];
      const float dev = (pj.x - pi.x) + (pj.y - pi.y);  // ubar_j - ubar_i
      const float w = t == 0 ? w_centre : eh2 * recip_t(fmaf(dev, dev, eh2));
      z[M] = dev;
      sqrt_free_fold(f, z, w * w);
    }
  }
  cp_async_wait<0>();
}

// Coefficients and facet values of cell i (FP32-bulk: the polynomial in FP32,
// ubar_i added in FP64), or with fdev set the FP32 deviations ubar - ubar_i;
// dev_out (may be null) also receives the deviations.
template <typename T, int DIM, int M>
__device__ __forceinline__ void tpc_write(const DeviceMesh& dm, int64_t i, double ui, const T (&x)[M],
                                          double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals,
                                          float* WLSENO_BODY_RESTRICT fdev, T* dev_out = nullptr);

// The FP32-deviation output alone (no coefficients): with the FP64 output
// path compiled out, no FP64 instruction is predicated into the FP32 kernel.
// Copies of n floats between 8-byte aligned addresses in the widest
// accesses their count allows (each cell's point offsets and deviations
// start at a multiple of 8 bytes: n is even).
template <int NF>
__device__ __forceinline__ void load_floats(const float* WLSENO_BODY_RESTRICT src, float (&dst)[NF]) {
  static_assert(NF % 2 == 0, "even counts");
  if constexpr (NF % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NF / 4; ++k) {
      const float4 v = reinterpret_cast<const float4*>(src)[k];
      dst[4 * k] = v.x, dst[4 * k + 1] = v.y, dst[4 * k + 2] = v.z, dst[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NF / 2; ++k) {
      const float2 v = reinterpret_cast<const float2*>(src)[k];
      dst[2 * k] = v.x, dst[2 * k + 1] = v.y;
    }
  }
}
template <int NF>
__device__ __forceinline__ void store_floats(float* WLSENO_BODY_RESTRICT dst, const float (&src)[NF]) {
  static_assert(NF % 2 == 0, "even counts");
  if constexpr (NF % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NF / 4; ++k)
      reinterpret_cast<float4*>(dst)[k] = make_float4(src[4 * k], src[4 * k + 1], src[4 * k + 2], src[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < NF / 2; ++k) reinterpret_cast<float2*>(dst)[k] = make_float2(src[2 * k], src[2 * k + 1]);
  }
}

// The polynomial's deviations from ubar_i at the cell's facet points.
template <typename T, int DIM, int M>
__device__ __forceinline__ void tpc_eval_dev(const DeviceMesh& dm, int64_t i, const T (&x)[M],
                                             T (&dev)[(DIM + 1) * nq_of(DIM)]) {
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  const T* P = tpc_points<T>(dm) + i * NP * DIM;
  T pts[NP * DIM];
  if constexpr (sizeof(T) == 4) {
    // FP32 offsets of a cell: 8 (1-D), 48 (2-D) or 144 (3-D) bytes from a
    // multiple of their size
    load_floats<NP * DIM>(P, pts);
  } else {
#pragma unroll
    for (int k = 0; k < NP * DIM; ++k) pts[k] = P[k];
  }
#pragma unroll
  for (int pt = 0; pt < NP; ++pt) {
    T yy[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) yy[a] = pts[pt * DIM + a];
    T mono[M];
    eval_monomials<T, DIM, M>(yy, mono);
    T sh = T(0);
#pragma unroll
    for (int c = 0; c < M; ++c) sh = fma(x[c], mono[c], sh);
    dev[pt] = sh;
  }
}

template <typename T, int DIM, int M>
__device__ __forceinline__ void tpc_write_dev(const DeviceMesh& dm, int64_t i, const T (&x)[M],
                                              float* WLSENO_BODY_RESTRICT fdev, T* dev_out) {
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  T dev[NP];
  tpc_eval_dev<T, DIM, M>(dm, i, x, dev);
  float out[NP];
#pragma unroll
  for (int pt = 0; pt < NP; ++pt) {
    if (dev_out) dev_out[pt] = dev[pt];
    out[pt] = static_cast<float>(dev[pt]);
  }
  store_floats<NP>(fdev + i * NP, out);
}

template <typename T, int DIM, int M>
__device__ __forceinline__ void tpc_write(const DeviceMesh& dm, int64_t i, double ui, const T (&x)[M],
                                          double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals,
                                          float* WLSENO_BODY_RESTRICT fdev, T* dev_out) {
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  if (fdev && !coeffs) {
    tpc_write_dev<T, DIM, M>(dm, i, x, fdev, dev_out);
    return;
  }
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
    if (dev_out) dev_out[pt] = sh;
    if (fdev)
      fdev[i * NP + pt] = static_cast<float>(sh);
    else
      fvals[i * NP + pt] = ui + static_cast<double>(sh);
  }
}

// One thread per (cell, component): C = 1 for the scalar equations; C = 4
// for 2-D Euler in FP32-bulk (componentwise, each component its own weights,
// Sec. 3.1.2), the four threads of a cell adjacent in the warp so that they
// share every row load (geometry, moments) and their state pairs are 32
// contiguous bytes (upair interleaved [N][C]).  With C > 1 the threads of a
// cell then take the positivity decision of the Euler traces together
// (work.pos_ok): a cell whose reconstructed density or pressure is <= 1e-12
// at any facet point uses its averages at all its facets (the flux kernel
// reads the flag).  Flagged (cell, component) pairs are listed as c N + i.
// The main kernel's work for global thread gt (one cell, or one (cell,
// component) pair); also the reconstruction phase of the persistent step.
template <typename T, int DIM, int M, bool OTF = false, int C = 1>
__device__ __forceinline__ void recon_tpc_cell(const DeviceMesh& dm, const SchemeParams& sp,
                                               const double* WLSENO_BODY_RESTRICT ubar, double* WLSENO_BODY_RESTRICT coeffs,
                                               double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev,
                                               unsigned long long* WLSENO_BODY_RESTRICT counters, const TpcWork& work,
                                               T flag_threshold, T pivot_threshold, int64_t gt) {
  static_assert(C == 1 || (sizeof(T) == 4 && 32 % C == 0), "components share a warp");
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  const int64_t i = C == 1 ? gt : gt / C;
  const int comp = C == 1 ? 0 : static_cast<int>(gt - i * C);
  if (i >= dm.N) return;  // the C threads of a cell leave together
  const int n = dm.st_ptr[i + 1] - dm.st_ptr[i];
  const int64_t coff = static_cast<int64_t>(comp) * dm.N;
  ubar += coff;
  if (coeffs) coeffs += coff * M;
  if (fvals) fvals += coff * NP;
  if (fdev && C == 1) fdev += coff * NP;  // (C > 1: the traces of all components, [N][NP][C])
  T eh2, wc;
  SqrtFreeQR<T, M> f;
  float2 pi = make_float2(0.0f, 0.0f);
  double w_spread = 1.0;  // FP64: spread of the row weights
  double ui;
  if constexpr (sizeof(T) == 4) {
    const float2* up = work.upair + comp;
    pi = up[i * C];
    auto wfn = [&](float* e, float* w) { tpc_weights_pair<DIM, C>(dm, sp, up, i, pi, e, w); };
    if constexpr (OTF)
      tpc_fold_staged_otf<DIM, M, C>(dm, up, i, pi, n, wfn, &eh2, &wc, f);
    else if constexpr (C > 1)
      tpc_fold_chunked<DIM, M, C>(dm, up, i, pi, n, wfn, &eh2, &wc, f);
    else
      tpc_fold_staged<DIM, M, C>(dm, up, i, pi, n, wfn, &eh2, &wc, f);
    // needed by the FP64 outputs and the refine records only: not loaded
    // for the deviation outputs (see the refine record below)
    ui = fdev && !coeffs ? 0.0 : ubar[i];
  } else {
    ui = ubar[i];
    tpc_weights<T, DIM>(dm, sp, ubar, i, ui, &eh2, &wc);
    tpc_fold<DIM, M>(dm, ubar, i, ui, n, eh2, wc, f, &w_spread);
  }
  T qmax, qmin, nrm[M];
  sqrt_free_colnorms(f, nrm);  // shared by the two conditioning tests
  sqrt_free_spread(f, nrm, &qmax, &qmin);
  T x[M];
  sqrt_free_solve(f, x);
  if constexpr (C > 1) {
    // the C threads of the cell: each evaluates its component's traces
    // hi + (lo + dev) (Sec. 3.2 polynomial, FP32) and puts them, with its
    // average hi + lo, in shared memory; then each tests the points p =
    // lane, lane + C, ... for rho and p > 1e-12 with all components
    // (conserved rho, rho u_1 .. rho u_dim, E) and, after the cell's lanes
    // agree, writes those points' traces -- or the averages, when any point
    // fails -- to fdev as [N][NP] float4 (the components of a point together)
    T dv[NP];
    tpc_eval_dev<T, DIM, M>(dm, i, x, dv);
    __shared__ float4 spos[kTpcThreads / C][NP + 1];
    static_assert(C == 4, "one float4 per facet point");
    const int cell = threadIdx.x / C;
    float* sp_cell = reinterpret_cast<float*>(&spos[cell][0]);
#pragma unroll
    for (int pt = 0; pt < NP; ++pt) sp_cell[pt * C + comp] = pi.x + (pi.y + static_cast<float>(dv[pt]));
    sp_cell[NP * C + comp] = pi.x + (pi.y + 0.0f);
    const unsigned seg = cell_lanes<C>();
    __syncwarp(seg);
    const float gm1 = work.gamma - 1.0f;
    bool ok = true;
#pragma unroll
    for (int p0 = 0; p0 < NP; p0 += C) {
      const int pt = p0 + comp;
      if (pt < NP) {
        const float4 U = spos[cell][pt];
        const float ke = fmaf(U.z, U.z, U.y * U.y);
        const float pr = gm1 * (U.w - 0.5f * ke * recip_t(U.x));  // a threshold test
        ok = ok && U.x > 1e-12f && pr > 1e-12f;
      }
    }
    ok = __all_sync(seg, ok);
    float4* trace = reinterpret_cast<float4*>(fdev) + i * NP;
#pragma unroll
    for (int p0 = 0; p0 < NP; p0 += C) {
      const int pt = p0 + comp;
      if (pt < NP) trace[pt] = spos[cell][ok ? pt : NP];
    }
    if (comp == 0) {
      work.pos_ok[i] = ok ? 1 : 0;
      if (!ok) atomicAdd(&counters[3], 1ull);
    }
  } else {
    tpc_write<T, DIM, M>(dm, i, ui, x, coeffs, fvals, fdev);
  }
  // a cell is flagged when its spread passes the flag threshold or its
  // inverse estimate passes the pivot bound (then it always takes the
  // pivoted path); a non-finite factor fails both tests
  float w2max, z2max;
  sqrt_free_inverse_estimate_sq(f, nrm, &w2max, &z2max);
  const bool near_singular = inverse_estimate_exceeds(w2max, z2max, static_cast<float>(pivot_threshold)) ||
                             !(w_spread <= kWeightSpread);
  if (!near_singular && qmax <= flag_threshold * flag_threshold * qmin) return;
  const int tag = static_cast<int>(coff + i);  // (component, cell) of the lists
  if (sizeof(T) == 4) atomicAdd(&counters[0], 1ull);
  if (sizeof(T) == 4 && work.refine_buf && !near_singular &&
      qmax <= pivot_threshold * pivot_threshold * qmin) {
    // keep the FP32 factor for the refinement kernel: one contiguous record
    constexpr int RW = refine_record_floats(M);
    float v[RW];
    v[0] = __int_as_float(tag);
    v[1] = __int_as_float(dm.st_ptr[i]);
    v[2] = __int_as_float(n);
    v[3] = static_cast<float>(wc);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      v[4 + c] = static_cast<float>(x[c]);
      v[4 + M + c] = static_cast<float>(f.d[c]);
    }
#pragma unroll
    for (int k = 0; k < M; ++k)
#pragma unroll
      for (int j = k + 1; j < M; ++j) v[4 + 2 * M + strict_upper_index(M, k, j)] = static_cast<float>(f.U[k][j]);
    constexpr int RE = refine_record_eps(M);
    v[RE] = static_cast<float>(eh2);
    const double ui_rec = sizeof(T) == 4 && fdev && !coeffs ? ubar[i] : ui;
    v[RE + 1] = __int_as_float(__double2loint(ui_rec));
    v[RE + 2] = __int_as_float(__double2hiint(ui_rec));
#pragma unroll
    for (int c = RE + 3; c < RW; ++c) v[c] = 0.0f;
    const int slot = atomicAdd(&work.counts[1], 1);
    float4* rec = reinterpret_cast<float4*>(work.refine_buf + static_cast<int64_t>(slot) * RW);
#pragma unroll
    for (int q = 0; q < RW / 4; ++q) rec[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
    work.group_list[atomicAdd(&work.counts[0], 1)] = tag;
  }
}

// Resident blocks per SM the main kernel is compiled for: the FP32 kernels
// of up to six columns fit 64 registers with the records shared by a
// cell's lanes (C > 1: 8 blocks, 32 warps) or 80 with per-thread records
// (6 blocks, which the 36 KB of staging per block also allows); the
// ten-column fold needs 128 (4); the FP64 fold its full register file.
template <typename T, int M, int C>
constexpr int tpc_min_blocks() {
  return sizeof(T) != 4 ? 1 : C > 1 ? 8 : M <= 6 ? 6 : 4;
}

template <typename T, int DIM, int M, bool OTF = false, int C = 1>
__global__ void __launch_bounds__(128, tpc_min_blocks<T, M, C>())
recon_tpc_kernel(DeviceMesh dm, SchemeParams sp, const double* WLSENO_BODY_RESTRICT ubar,
                 double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev,
                 unsigned long long* WLSENO_BODY_RESTRICT counters, TpcWork work, T flag_threshold,
                 T pivot_threshold) {
  recon_tpc_cell<T, DIM, M, OTF, C>(dm, sp, ubar, coeffs, fvals, fdev, counters, work, flag_threshold,
                                    pivot_threshold, blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x);
}

// One corrected-seminormal-equations sweep on the refine-listed cells
// (FP32-bulk): with the FP32 factor W A = Q D^(1/2) U of the main kernel and
// its solution x, x += (U^T D U)^-1 A^T W^2 (b - A x), with the residual
// b - A x formed in FP64 from the FP64 moments and deviations (the FP32
// factor only preconditions the correction).  L lanes share a
// cell, lane l taking rows l, l+L, ..., l+(RPL-1)L (the thread-per-cell path
// serves stencils of at most L*RPL rows).  The kernel is a latency chain on
// few warps, so its dependent loads are kept to three levels: the list length
// and the first record together; then everything the record addresses (the
// stencil indices, both copies of the moment rows, the lane's facet point;
// the record carries the weights' eps h^2 and w_c and ubar_i); then ubar of the
// stencil cells.  The partial sums are combined by shuffles.  It overwrites
// the main kernel's outputs for those cells.
// The sweep for global thread gt of nthreads (whole warps): the kernel's body
// and the refinement phase of the persistent step.
// The traces of an all-components context (its work carries the
// positivity flags; fdev then holds [N][NP][C] traces), else none.
__host__ __device__ inline TraceOut trace_out(const ReconOut& out, const TpcWork& work) {
  TraceOut tr;
  if (work.pos_ok) {
    tr.base = out.fdev;
    tr.upair = work.upair;
    tr.pos_ok = work.pos_ok;
  }
  return tr;
}

template <int DIM, int M, int L, int RPL>
__device__ __forceinline__ void refine_records(const DeviceMesh& dm, const double* WLSENO_BODY_RESTRICT ubar,
                                               double* WLSENO_BODY_RESTRICT coeffs, double* WLSENO_BODY_RESTRICT fvals,
                                               float* WLSENO_BODY_RESTRICT fdev, const TpcWork& work, int64_t gt,
                                               int64_t nthreads) {
  constexpr int NP = (DIM + 1) * nq_of(DIM);
  static_assert(NP <= L && M <= L, "one facet point and one coefficient per lane");
  constexpr int kPerWarp = 32 / L;
  constexpr int RW = refine_record_floats(M);
  constexpr int RE = refine_record_eps(M);
  const int lane = threadIdx.x % L;
  const int64_t warp = gt / 32;
  const int64_t warps = nthreads / 32;
  const int64_t sub = (threadIdx.x % 32) / L;
  const int64_t last = work.capacity - 1;  // the record buffer holds `capacity` records
  float r[RW];
  auto load_record = [&](int64_t slot) {
    const float4* rec = reinterpret_cast<const float4*>(work.refine_buf + (slot < last ? slot : last) * RW);
#pragma unroll
    for (int q = 0; q < RW / 4; ++q) {
      const float4 v = rec[q];
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  };
  const int64_t first = warp * kPerWarp;
  load_record(first + sub);  // issued together with the list length
  const int count = *reinterpret_cast<const volatile int*>(work.counts + 1);
  for (int64_t base = first; base < count; base += warps * kPerWarp) {
    if (base != first) load_record(base + sub);
    const int64_t slot = base + sub;
    const bool valid = slot < count;
    // the record's tag c N + i: component c (multi-component contexts), cell i
    const int64_t tag = valid ? __float_as_int(r[0]) : 0;
    const int64_t comp = tag >= dm.N ? tag / dm.N : 0;
    const int64_t i = tag - comp * dm.N;
    const double* WLSENO_BODY_RESTRICT ubc = ubar + comp * dm.N;
    const int beg = __float_as_int(r[1]);
    const int n = valid ? __float_as_int(r[2]) : 0;
    const float wc = r[3];
    const float e = r[RE];
    const double ui = __hiloint2double(__float_as_int(r[RE + 2]), __float_as_int(r[RE + 1]));
    // every load the record addresses, stencil indices first (the longest chain)
    int64_t jrow[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int t = lane + q * L;
      jrow[q] = t < n ? dm.st_idx[beg + t] : i;
    }
    float yy[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) yy[a] = lane < NP ? dm.fpts32[(i * NP + lane) * DIM + a] : 0.0f;
    double a[RPL][M];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int t = lane + q * L;
      const double* row = dm.A64 + static_cast<int64_t>(beg + t) * M;
      if constexpr (M % 2 == 0) {  // rows of 16-byte multiples: 16-byte loads
        const double2* row2 = reinterpret_cast<const double2*>(row);
#pragma unroll
        for (int c = 0; c < M; c += 2) {
          const double2 v = t < n ? row2[c / 2] : make_double2(0.0, 0.0);
          a[q][c] = v.x;
          a[q][c + 1] = v.y;
        }
      } else {  // odd m: rows start on 8-byte boundaries only
#pragma unroll
        for (int c = 0; c < M; ++c) a[q][c] = t < n ? row[c] : 0.0;
      }
    }
    // the FP32 copy of the same rows for A^T W^2 r (no FP64 -> FP32 conversions)
    float a32[RPL][M];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int t = lane + q * L;
      const float* row = dm.A32 + static_cast<int64_t>(beg + t) * M;
      if constexpr (M % 2 == 0) {  // rows of 8-byte multiples: 8-byte loads
        const float2* row2 = reinterpret_cast<const float2*>(row);
#pragma unroll
        for (int c = 0; c < M; c += 2) {
          const float2 v = t < n ? row2[c / 2] : make_float2(0.0f, 0.0f);
          a32[q][c] = v.x;
          a32[q][c + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int c = 0; c < M; ++c) a32[q][c] = t < n ? row[c] : 0.0f;
      }
    }
    double uj[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) uj[q] = ubc[jrow[q]];
    double x[M];
#pragma unroll
    for (int c = 0; c < M; ++c) x[c] = static_cast<double>(r[4 + c]);
    // weights of the FP64 problem (Sec. 3.1.2) to FP32 relative accuracy:
    // only the residual needs FP64 (its cancellation), A^T W^2 r does not
    float g[M];
#pragma unroll
    for (int c = 0; c < M; ++c) g[c] = 0.0f;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int t = lane + q * L;
      // rows past both cells' stencils: skip their FP64 work (warp-uniform)
      if (!__any_sync(0xffffffffu, t < n)) continue;
      const double dev = uj[q] - ui;
      const float devf = static_cast<float>(dev);
      const float w = t == 0 ? wc : e / fmaf(devf, devf, e);
      double fit0 = 0.0, fit1 = 0.0;
#pragma unroll
      for (int c = 0; c < M; c += 2) {
        fit0 = fma(a[q][c], x[c], fit0);
        if (c + 1 < M) fit1 = fma(a[q][c + 1], x[c + 1], fit1);
      }
      const float wr = t < n ? w * w * static_cast<float>(dev - (fit0 + fit1)) : 0.0f;
#pragma unroll
      for (int c = 0; c < M; ++c) g[c] = fmaf(wr, a32[q][c], g[c]);
    }
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1)
#pragma unroll
      for (int c = 0; c < M; ++c) g[c] += __shfl_xor_sync(0xffffffffu, g[c], off);
    if (!valid) continue;
    // (U^T D U) delta = g with the FP32 factor
    float dl[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      float v = g[k];
#pragma unroll
      for (int q = 0; q < k; ++q) v = fmaf(-r[4 + 2 * M + strict_upper_index(M, q, k)], dl[q], v);
      dl[k] = v;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) dl[k] /= r[4 + M + k];
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
      float v = dl[k];
#pragma unroll
      for (int q = k + 1; q < M; ++q) v = fmaf(-r[4 + 2 * M + strict_upper_index(M, k, q)], dl[q], v);
      dl[k] = v;
    }
    float xh[M];
#pragma unroll
    for (int c = 0; c < M; ++c) xh[c] = r[4 + c];
    if (coeffs) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        if (c == lane)
          coeffs[(comp * dm.N + i) * M + c] = static_cast<double>(xh[c]) + static_cast<double>(dl[c]) + (c == 0 ? ui : 0.0);
    }
    if (lane < NP) {
      float mono[M];
      eval_monomials<float, DIM, M>(yy, mono);
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int c = 0; c < M; ++c) {
        sh = fmaf(xh[c], mono[c], sh);
        sl = fmaf(dl[c], mono[c], sl);
      }
      if (work.pos_ok) {
        // all-components context: the component's trace, where used
        constexpr int TC = DIM + 2;
        if (work.pos_ok[i]) {
          const float2 pc = work.upair[i * TC + comp];
          fdev[(i * NP + lane) * TC + comp] = pc.x + (pc.y + (sh + sl));
        }
      } else if (fdev)
        fdev[(comp * dm.N + i) * NP + lane] = sh + sl;
      else
        fvals[(comp * dm.N + i) * NP + lane] = ui + static_cast<double>(sh) + static_cast<double>(sl);
    }
  }
}

template <int DIM, int M, int L, int RPL>
__global__ void __launch_bounds__(64)
refine_kernel(DeviceMesh dm, const double* WLSENO_BODY_RESTRICT ubar, double* WLSENO_BODY_RESTRICT coeffs,
              double* WLSENO_BODY_RESTRICT fvals, float* WLSENO_BODY_RESTRICT fdev, TpcWork work) {
  refine_records<DIM, M, L, RPL>(dm, ubar, coeffs, fvals, fdev, work,
                                 blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                                 gridDim.x * static_cast<int64_t>(blockDim.x));
}


// The main kernel; the list lengths (work.counts[0..1]) must be zero.  C > 1:
// all components at once (FP32-bulk 2-D Euler), ubar the [C][N] state.
template <typename T, int DIM, int M, int C = 1>
cudaError_t launch_recon_tpc(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                             const ReconOut& out, const TpcWork& work, cudaStream_t s) {
  constexpr int threads = kTpcThreads;
  const unsigned blocks = static_cast<unsigned>((dm.N * C + threads - 1) / threads);
  // thresholds: refine / pivot bounds (tpc_thresholds, capi.cpp)
  const bool f32 = sizeof(T) == 4;
  double flag64 = 0.0, pivot64 = 0.0;
  tpc_thresholds(sp, f32, &flag64, &pivot64);
  const T pivot = static_cast<T>(pivot64);
  const T flag = static_cast<T>(flag64);
  if (f32 && !work.upair) return cudaErrorInvalidValue;
  if (work.capacity < dm.N * C) return cudaErrorInvalidValue;
  if (C > 1 && !work.pos_ok) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (work.otf) {
      if (!dm.geo32 || !dm.own32) return cudaErrorInvalidValue;
      recon_tpc_kernel<T, DIM, M, true, C><<<blocks, threads, 0, s>>>(
          dm, sp, ubar, out.coeffs, out.fvals, out.fdev, out.counters, work, flag, pivot);
      return cudaGetLastError();
    }
  }
  recon_tpc_kernel<T, DIM, M, false, C><<<blocks, threads, 0, s>>>(dm, sp, ubar, out.coeffs, out.fvals,
                                                                  out.fdev, out.counters, work, flag, pivot);
  return cudaGetLastError();
}

// The pivoted cells, one lane group each: rows spread over the lanes.
template <typename T, int DIM, int M>
cudaError_t launch_list(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                        const ReconOut& out, const TpcWork& work, cudaStream_t s) {
  const TraceOut tr = trace_out(out, work);
  if (dm.nmax <= 40)
    return launch_reconstruct_list<T, DIM, M, 8, 5>(dm, sp, ubar, out, work.group_list, work.counts, s, tr);
  return launch_reconstruct_list<T, DIM, M, 16, 4>(dm, sp, ubar, out, work.group_list, work.counts, s, tr);
}

// The follow-ups on the listed cells: the refinement sweep (FP32-bulk) and
// the pivoted path; *launches receives the number of kernels launched.
template <typename T, int DIM, int M>
cudaError_t launch_recon_fixup(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                               const ReconOut& out, const TpcWork& work, cudaStream_t s,
                               int* launches) {
  *launches = 0;
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (!work.refine_buf) return cudaErrorInvalidValue;
    // 16 lanes x 4 rows: every stencil the thread-per-cell path accepts (<= 64)
    constexpr int L = 16, RPL = 4, kThreads = 64;
    const int64_t want = (dm.N * L + kThreads - 1) / kThreads;
    const unsigned rblocks = static_cast<unsigned>(want < 8 * 152 ? want : 8 * 152);
    // the pivoted path on the side stream when one is given (different cells,
    // the same inputs): fork before the refinement, join after it
    const bool fork = work.side && work.fork && work.join;
    cudaStream_t sl = s;
    if (fork) {
      if ((e = cudaEventRecord(work.fork, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(work.side, work.fork, 0)) != cudaSuccess) return e;
      sl = work.side;
      if ((e = launch_list<T, DIM, M>(dm, sp, ubar, out, work, sl)) != cudaSuccess) return e;
      ++*launches;
      if ((e = cudaEventRecord(work.join, sl)) != cudaSuccess) return e;
    }
    refine_kernel<DIM, M, L, RPL>
        <<<rblocks, kThreads, 0, s>>>(dm, ubar, out.coeffs, out.fvals, out.fdev, work);
    ++*launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fork) return cudaStreamWaitEvent(s, work.join, 0);
  }
  e = launch_list<T, DIM, M>(dm, sp, ubar, out, work, s);
  ++*launches;
  return e;
}

}  // namespace wlseno
