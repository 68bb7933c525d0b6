// Instantiations of the reconstruction kernels for T = double, 1-D, m = 3.
#include "k_recon_tpc_kernels.cuh"
#include "k_reconstruct.cuh"

namespace wlseno {
template <>
cudaError_t launch_reconstruct_inst<double, 1, 3>(const DeviceMesh& dm, const SchemeParams& sp,
                                                   int G, int R, const double* ubar,
                                                   const ReconOut& out, cudaStream_t s) {
  return launch_reconstruct_tm<double, 1, 3>(dm, sp, G, R, ubar, out, s);
}

template <>
cudaError_t launch_recon_tpc_inst<double, 1, 3>(const DeviceMesh& dm, const SchemeParams& sp,
                                 const double* ubar, const ReconOut& out, const TpcWork& work,
                                 cudaStream_t s) {
  return launch_recon_tpc<double, 1, 3>(dm, sp, ubar, out, work, s);
}

template <>
cudaError_t launch_recon_fixup_inst<double, 1, 3>(const DeviceMesh& dm, const SchemeParams& sp,
                                   const double* ubar, const ReconOut& out, const TpcWork& work,
                                   cudaStream_t s, int* launches) {
  return launch_recon_fixup<double, 1, 3>(dm, sp, ubar, out, work, s, launches);
}
}  // namespace wlseno
