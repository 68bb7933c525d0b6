// Instantiation of the reconstruction kernel for T = double, 2-D, m = 6.
#include "k_reconstruct.cuh"

namespace wlseno {
template <>
cudaError_t launch_reconstruct_inst<double, 2, 6>(const DeviceMesh& dm, const SchemeParams& sp,
                                                   int G, int R, const double* ubar,
                                                   const ReconOut& out, cudaStream_t s) {
  return launch_reconstruct_tm<double, 2, 6>(dm, sp, G, R, ubar, out, s);
}
}  // namespace wlseno
