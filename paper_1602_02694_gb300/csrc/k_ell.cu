// Copies the CSR stencils and moment rows, once after the moment precompute,
// into the layouts of the thread-per-cell kernels:
//  * ELL (FP64 kernel, adjoint): row t of cell i at t*N + i, column c of it at
//    (t*m + c)*N + i, so a warp's loads of one column are coalesced;
//  * FP32 row records (staged FP32 kernel): record (t, i) at (t*N + i)*W
//    floats, W = round_up(m + 1, 4): the m moments, the stencil index as int32
//    bits, zeros.  A warp's records are one contiguous 16-byte-aligned span,
//    moved into shared memory by 16-byte asynchronous copies.
//  * FP32-bulk only, for the moments-on-the-fly kernel: per row the offset
//    (x_j - x_i)/h_i of the stencil cell's centroid at its minimum image
//    (the image the moments use) and the stencil index, 16 bytes; per cell its
//    own central moments of degree >= 2 in absolute units (the centre row of
//    its moments times h_i^|kappa|).
// Rows past a cell's stencil (t >= n) point at the cell itself with zero
// moments; the kernels never read them.
#include "wlseno_internal.h"

namespace wlseno {
namespace {

// Total degree of Taylor column c (the column order of monomials.cuh).
__device__ int taylor_degree(int dim, int c) {
  if (dim == 1) return c;
  if (dim == 2) return c == 0 ? 0 : c < 3 ? 1 : c < 6 ? 2 : 3;
  return c == 0 ? 0 : c < 4 ? 1 : 2;
}

__global__ void ell_copy_kernel(DeviceMesh dm) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  const int64_t N = dm.N;
  const int m = dm.m;
  const int W = dm.rec_width;
  const int beg = dm.st_ptr[i];
  const int n = dm.st_ptr[i + 1] - beg;
  for (int t = 0; t < dm.nmax; ++t) {
    const bool in = t < n;
    const int32_t j = in ? dm.st_idx[beg + t] : static_cast<int32_t>(i);
    dm.st_ell[t * N + i] = j;
    float* rec = dm.rec32 + (static_cast<int64_t>(t) * N + i) * W;
    for (int c = 0; c < m; ++c) {
      const int64_t src = static_cast<int64_t>(beg + t) * m + c;
      const int64_t dst = (static_cast<int64_t>(t) * m + c) * N + i;
      dm.A64e[dst] = in ? dm.A64[src] : 0.0;
      rec[c] = in ? dm.A32[src] : 0.0f;
    }
    rec[m] = __int_as_float(j);
    for (int c = m + 1; c < W; ++c) rec[c] = 0.0f;
    if (dm.geo32) {
      const int dim = dm.dim;
      const double hinv = 1.0 / dm.h[i];
      const double* per = dm.period + 3 * dm.mesh_of[i];
      float* g = dm.geo32 + (static_cast<int64_t>(t) * N + i) * 4;
      for (int a = 0; a < 4; ++a) g[a] = 0.0f;
      if (in) {
        for (int a = 0; a < dim; ++a) {
          double d = dm.centroid[static_cast<int64_t>(j) * dim + a] - dm.centroid[i * dim + a];
          if (per[a] > 0.0) d -= per[a] * nearbyint(d / per[a]);
          g[a] = static_cast<float>(d * hinv);
        }
      }
      g[dim] = __int_as_float(j);
    }
  }
  if (dm.own32) {
    // the centre row (t = 0) about x_i in h_i units, scaled back by h_i^|kappa|
    const double hi = dm.h[i];
    float* o = dm.own32 + i * dm.own_width;
    int k = 0;
    for (int c = 0; c < m; ++c) {
      const int deg = taylor_degree(dm.dim, c);
      if (deg >= 2) o[k++] = static_cast<float>(dm.A64[static_cast<int64_t>(beg) * m + c] * pow(hi, deg));
    }
    for (; k < dm.own_width; ++k) o[k] = 0.0f;
  }
}

}  // namespace

cudaError_t launch_ell_copy(const DeviceMesh& dm, cudaStream_t s) {
  const int threads = 128;
  const unsigned blocks = static_cast<unsigned>((dm.N + threads - 1) / threads);
  ell_copy_kernel<<<blocks, threads, 0, s>>>(dm);
  return cudaGetLastError();
}

}  // namespace wlseno
