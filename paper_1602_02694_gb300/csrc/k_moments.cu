// FP64 Taylor-moment precompute (Sec. 3.2; h-normalised as in Sec. 3.3.2):
// one thread per stencil entry (i, j) evaluates row j of cell i's moment
// matrix (moment_row.cuh: exact Gauss-Legendre product rule on the simplex)
// and stores it in FP64 and FP32.
#include "moment_row.cuh"
#include "wlseno_internal.h"

namespace wlseno {
namespace {

template <int DIM, int M>
__global__ void moments_kernel(DeviceMesh dm, GaussRule g) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= dm.nnz) return;
  // owner row i of stencil entry e (binary search on st_ptr)
  int64_t lo = 0, hi = dm.N;  // st_ptr[lo] <= e < st_ptr[hi]
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (dm.st_ptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  const int64_t i = lo;
  const int64_t j = dm.st_idx[e];
  double acc[M];
  moment_row<DIM, M>(dm, g, i, j, acc);
#pragma unroll
  for (int c = 0; c < M; ++c) {
    dm.A64[e * M + c] = acc[c];
    dm.A32[e * M + c] = static_cast<float>(acc[c]);
  }
}

template <int DIM, int M>
cudaError_t launch_dm(const DeviceMesh& dm, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (dm.nnz + threads - 1) / threads;
  moments_kernel<DIM, M><<<static_cast<unsigned>(blocks), threads, 0, s>>>(dm, make_gauss_rule());
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_moments(const DeviceMesh& dm, cudaStream_t s) {
  if (dm.dim == 1) {
    switch (dm.m) {
      case 3: return launch_dm<1, 3>(dm, s);
      case 5: return launch_dm<1, 5>(dm, s);
    }
  } else if (dm.dim == 2) {
    switch (dm.m) {
      case 3: return launch_dm<2, 3>(dm, s);
      case 6: return launch_dm<2, 6>(dm, s);
      case 10: return launch_dm<2, 10>(dm, s);
    }
  } else {
    switch (dm.m) {
      case 4: return launch_dm<3, 4>(dm, s);
      case 10: return launch_dm<3, 10>(dm, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace wlseno
