// Copies the CSR stencils and moment rows into the ELL layout of the
// thread-per-cell kernel (row t of cell i at t*N + i), once after the
// moment precompute.
#include "wlseno_internal.h"

namespace wlseno {
namespace {

__global__ void ell_copy_kernel(DeviceMesh dm) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= dm.N) return;
  const int64_t N = dm.N;
  const int m = dm.m;
  const int beg = dm.st_ptr[i];
  const int n = dm.st_ptr[i + 1] - beg;
  for (int t = 0; t < dm.nmax; ++t) {
    const bool in = t < n;
    dm.st_ell[t * N + i] = in ? dm.st_idx[beg + t] : static_cast<int32_t>(i);
    for (int c = 0; c < m; ++c) {
      const int64_t src = static_cast<int64_t>(beg + t) * m + c;
      const int64_t dst = (static_cast<int64_t>(t) * m + c) * N + i;
      dm.A64e[dst] = in ? dm.A64[src] : 0.0;
      dm.A32e[dst] = in ? dm.A32[src] : 0.0f;
    }
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
