// Instantiation of the reconstruction kernel for T = float, 2-D, m = 10.
#include "k_reconstruct.cuh"

namespace wlseno {
template <>
cudaError_t launch_reconstruct_inst<float, 2, 10>(const DeviceMesh& dm, const SchemeParams& sp,
                                                   int G, int R, const double* ubar,
                                                   const ReconOut& out, cudaStream_t s) {
  return launch_reconstruct_tm<float, 2, 10>(dm, sp, G, R, ubar, out, s);
}
}  // namespace wlseno
