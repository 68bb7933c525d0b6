// Instantiations of the reconstruction kernels for T = float, 2-D, m = 6.
#include "k_recon_tpc_kernels.cuh"
#include "k_reconstruct.cuh"

namespace wlseno {
template <>
cudaError_t launch_reconstruct_inst<float, 2, 6>(const DeviceMesh& dm, const SchemeParams& sp,
                                                   int G, int R, const double* ubar,
                                                   const ReconOut& out, cudaStream_t s) {
  return launch_reconstruct_tm<float, 2, 6>(dm, sp, G, R, ubar, out, s);
}

template <>
cudaError_t launch_recon_tpc_inst<float, 2, 6>(const DeviceMesh& dm, const SchemeParams& sp,
                                 const double* ubar, const ReconOut& out, const TpcWork& work,
                                 cudaStream_t s) {
  return launch_recon_tpc<float, 2, 6>(dm, sp, ubar, out, work, s);
}

template <>
cudaError_t launch_recon_fixup_inst<float, 2, 6>(const DeviceMesh& dm, const SchemeParams& sp,
                                   const double* ubar, const ReconOut& out, const TpcWork& work,
                                   cudaStream_t s, int* launches) {
  return launch_recon_fixup<float, 2, 6>(dm, sp, ubar, out, work, s, launches);
}

cudaError_t launch_recon_euler2d(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                                 const ReconOut& out, const TpcWork& work, cudaStream_t s) {
  return launch_recon_tpc<float, 2, 6, 4>(dm, sp, ubar, out, work, s);
}
}  // namespace wlseno
