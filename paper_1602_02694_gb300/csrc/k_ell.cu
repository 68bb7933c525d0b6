// Copies the CSR stencils and moment rows, once after the moment precompute,
// into the layouts of the thread-per-cell kernels:
//  * ELL (FP64 kernel, adjoint): row t of cell i at t*N + i, column c of it at
//    (t*m + c)*N + i, so a warp's loads of one column are coalesced;
//  * FP32 row records (staged FP32 kernel): record (t, i) at (t*N + i)*W
//    floats, W = round_up(m + 1, 4): the m moments, the stencil index as int32
//    bits, zeros.  A warp's records are one contiguous 16-byte-aligned span,
//    moved into shared memory by 16-byte asynchronous copies.
// Rows past a cell's stencil (t >= n) point at the cell itself with zero
// moments; the kernels never read them.
#include "wlseno_internal.h"

namespace wlseno {
namespace {

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
