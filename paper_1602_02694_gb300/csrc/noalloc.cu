// wlseno_flux_residual_static: the spatial operator L(ubar) without any
// device allocation by the call.
//
// Some callers cannot call cudaMalloc when they need a residual: code running
// while a stream is being captured (a capture may not allocate), real-time
// loops that forbid allocation after start-up, and hosts whose device memory
// is owned by their own pool allocator.  For them the facet values that
// wlseno_flux_residual keeps in context-owned scratch live here instead, in a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
#include <mutex>
#include <string>

#include "wlseno_internal.h"

namespace wlseno {
namespace {

// Facet-value scratch: n_cells * (dim+1) * quad_per_facet doubles at most
// (8 MiB: 174,762 triangles or 87,381 tetrahedra).
constexpr size_t kStaticScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double g_facet_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (current), looked up once
// per device: in host code the array's name is only a host-side stand-in.
cudaError_t scratch_on(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_facet_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace wlseno

using namespace wlseno;

extern "C" wlseno_status wlseno_flux_residual_static(wlseno_ctx* ctx, const double* ubar,
                                                     double* residual, void* stream) {
  CtxView v;
  if (!ctx || !ctx_view(ctx, &v)) return WLSENO_ERR_INVALID_ARG;
  if (v.sp.pde == WLSENO_EULER) {
    ctx_set_error(ctx, "wlseno_flux_residual_static covers the scalar equations");
    return WLSENO_ERR_INVALID_ARG;
  }
  if (!v.ready) {
    ctx_set_error(ctx, "call wlseno_build_stencils and wlseno_precompute_moments first");
    return WLSENO_ERR_STATE;
  }
  if (!ubar || !residual) {
    ctx_set_error(ctx, "null array");
    return WLSENO_ERR_INVALID_ARG;
  }
  const int np = (v.dm.dim + 1) * v.dm.nq;
  if (static_cast<size_t>(v.dm.N) * np > kStaticScratchDoubles) {
    ctx_set_error(ctx, "wlseno_flux_residual_static: " + std::to_string(v.dm.N) + " cells need " +
                           std::to_string(static_cast<size_t>(v.dm.N) * np) +
                           " facet values, more than its fixed scratch of " +
                           std::to_string(kStaticScratchDoubles));
    return WLSENO_ERR_INVALID_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != v.device && cudaSetDevice(v.device) != cudaSuccess) {
    cudaGetLastError();
    return WLSENO_ERR_CUDA;
  }
  wlseno_status st = WLSENO_OK;
  double* scratch = nullptr;
  cudaError_t e = scratch_on(v.device, &scratch);
  if (e != cudaSuccess) {
    ctx_set_error(ctx, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    st = WLSENO_ERR_CUDA;
  } else if (!device_pointer(ubar) || !device_pointer(residual)) {
    ctx_set_error(ctx, "wlseno_flux_residual_static needs device arrays (it stages nothing)");
    st = WLSENO_ERR_INVALID_ARG;
  } else {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(v.counters, 0, kCounters * sizeof(unsigned long long), s);
    for (int c = 0; c < v.n_comp && e == cudaSuccess; ++c) {
      const double* u = ubar + c * v.dm.N;
      // the same facet-value format as wlseno_flux_residual (FP32 deviations
      // in FP32-bulk thread-per-cell contexts; they take half the scratch)
      float* dev = v.dev_facets ? reinterpret_cast<float*>(scratch) : nullptr;
      ReconOut out{nullptr, dev ? nullptr : scratch, v.counters, dev};
      e = ctx_launch_reconstruct(ctx, u, out, s);
      if (e == cudaSuccess)
        e = ctx_launch_flux_residual(ctx, scratch, dev, u, residual + c * v.dm.N, s);
    }
    if (e != cudaSuccess) {
      ctx_set_error(ctx, std::string("wlseno_flux_residual_static: ") + cudaGetErrorString(e));
      cudaGetLastError();
      st = WLSENO_ERR_CUDA;
    }
  }
  if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
  return st;
}
