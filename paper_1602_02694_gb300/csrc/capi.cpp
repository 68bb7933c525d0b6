// C ABI of libwlseno: context, device buffers, host/device pointer staging
// and the entry points of include/wlseno.h.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "wlseno_internal.h"

using namespace wlseno;

// Polls of a bounded device wait before it gives up (about 64 ns apart: ~1 s).
constexpr long long kDefaultSpinCap = 1ll << 24;

struct wlseno_ctx {
  int device = 0;
  wlseno_scheme scheme{};
  SchemeParams sp{};
  bool built = false;
  bool moments_ready = false;
  HostSetup host;
  int G = 0, R = 0;
  bool otf = false;              // FP32-bulk main kernel forms its moment rows on the fly
  DeviceMesh dm{};
  std::vector<void*> allocs;     // every device allocation of the context
  size_t alloc_bytes = 0;        // their total size
  size_t alloc_limit = 0;        // WLSENO_DEVICE_BYTES_LIMIT at creation (0: none)
  int32_t* d_st_ptr = nullptr;
  int32_t* d_st_idx = nullptr;
  double* d_rmin = nullptr;
  double* d_dt = nullptr;
  float2* d_dt2 = nullptr;       // [n_meshes] double-float pairs of d_dt
  unsigned long long* d_lmax = nullptr;
  unsigned long long* d_counters = nullptr;
  double* d_fvals = nullptr;     // [N][NP]
  double* d_k1 = nullptr;        // [C][N] RK stage states
  double* d_k2 = nullptr;
  double* d_in = nullptr;        // [C][N] staging for host inputs / outputs
  double* d_out = nullptr;       // [C][N] staging for host outputs
  double* d_coef = nullptr;      // [C][N][m] staging for host coefficient output
  double* d_fv_out = nullptr;    // [C][N][NP] staging for host facet-value output
  int* d_wl = nullptr;           // [wl_cap] (component, cell) tags for the pivoted lane-group path
  int* d_wl_count = nullptr;     // [2] lengths of d_wl and of the refine records
  float* d_rbuf = nullptr;       // [wl_cap][refine_record_floats(m)] FP32-bulk refine records
  int64_t wl_cap = 0;            // N, or C N with the all-components Euler kernel
  float* d_fdev = nullptr;       // FP32-bulk facet deviations [N][NP] (scalar equations); 2-D Euler traces [N][NP][4]
  float2* d_pair = nullptr;      // [3][C][N] FP32 pairs of states: scratch, k1, k2 (FP32-bulk;
                                 // interleaved [N][C] on the all-components Euler path)
  bool euler32 = false;          // FP32-bulk 2-D Euler p = 3: all components in one kernel
  unsigned char* d_pos_ok = nullptr;  // [N] its positivity flags
  BalanceWork bal{};             // balanced-stencil re-selection (when the scheme asks for it)
  // side stream of the pivoted-path kernel, forked from and joined to the
  // caller's stream around the refinement sweep
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool mesh_dt_set = false;      // d_dt holds per-mesh steps from wlseno_set_mesh_dt
  // one captured RK step, replayed for multi-step calls
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  const double* graph_u = nullptr;
  double graph_dt = 0.0, graph_cfl = 0.0;
  int graph_shape = 0;           // shape_key of the captured step
  int64_t graph_launches = 0;
  int64_t graph_kind[WLSENO_N_KERNEL_KINDS] = {};
  // adjoint work (allocated on the first wlseno_step_adjoint)
  AdjointWork adj{};
  double* d_gbar[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t launches = 0;
  int64_t by_kind[WLSENO_N_KERNEL_KINDS] = {};
  // timing mode: event pairs recorded around launches, summed on demand
  bool timing = false;
  struct TimedLaunch {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<cudaEvent_t> event_pool;
  std::vector<TimedLaunch> timed;
  size_t events_used = 0;
  cudaStream_t last_stream = nullptr;
  double last_dt = 0.0;
  // status words (mapped pinned host memory, set by the kernels): [0]
  // non-finite results, [1] a bounded device wait gave up
  unsigned int* h_latch = nullptr;
  unsigned int* d_latch = nullptr;
  // persistent step kernel (opts.persistent): per-stage list lengths [6],
  // barrier words [3], the poll limit of its waits
  bool persistent = false;
  int* d_counts6 = nullptr;
  unsigned int* d_sync = nullptr;
  long long spin_cap = kDefaultSpinCap;
  bool persist_no_capture = false;  // the cooperative launch could not be captured
  std::string error;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

wlseno_status fail(wlseno_ctx* ctx, wlseno_status s, const std::string& msg) {
  if (ctx) ctx->error = msg;
  return s;
}

wlseno_status cuda_fail(wlseno_ctx* ctx, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(ctx, e == cudaErrorMemoryAllocation ? WLSENO_ERR_OOM : WLSENO_ERR_CUDA, msg);
}

template <typename T>
wlseno_status dalloc(wlseno_ctx* ctx, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (ctx->alloc_limit > 0 && ctx->alloc_bytes + bytes > ctx->alloc_limit)
    return fail(ctx, WLSENO_ERR_OOM,
                "device allocation of " + std::to_string(bytes) + " bytes would exceed the context's limit of " +
                    std::to_string(ctx->alloc_limit) + " (WLSENO_DEVICE_BYTES_LIMIT)");
  void* raw = nullptr;
  cudaError_t e = cudaMalloc(&raw, bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
  ctx->allocs.push_back(raw);
  ctx->alloc_bytes += bytes;
  *p = static_cast<T*>(raw);
  return WLSENO_OK;
}

template <typename T>
wlseno_status upload(wlseno_ctx* ctx, T** p, const std::vector<T>& v) {
  wlseno_status s = dalloc(ctx, p, v.size());
  if (s != WLSENO_OK) return s;
  cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
  return WLSENO_OK;
}

void free_all(wlseno_ctx* ctx) {
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->alloc_bytes = 0;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Shapes compiled into the reconstruction (lanes per cell, rows per lane):
// (1, 0) is the thread-per-cell kernel (any stencil size), the others the
// lane-group kernel holding at most lanes x rows stencil rows.
const int kShapes[][2] = {{1, 0}, {8, 2}, {8, 3}, {8, 5}, {16, 3}, {16, 4}};

bool shape_ok(int G, int R) {
  for (auto& s : kShapes)
    if (s[0] == G && s[1] == R) return true;
  return false;
}

// The thread-per-cell kernel hands ill-conditioned cells to the lane-group
// kernel, whose largest compiled shape holds 64 rows.
bool shape_fits(int G, int R, int max_n) { return G == 1 ? max_n <= 64 : G * R >= max_n; }

void choose_shape(int max_n, int* G, int* R) {
  (void)max_n;
  *G = 1;  // thread per cell: fastest on GB300 for every compiled (dim, m)
  *R = 0;
}

int points_per_cell(const wlseno_ctx* ctx) { return (ctx->dm.dim + 1) * ctx->dm.nq; }

cudaEvent_t next_event(wlseno_ctx* ctx) {
  if (ctx->events_used == ctx->event_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ctx->event_pool.push_back(e);
  }
  return ctx->event_pool[ctx->events_used++];
}

// Brackets the launches of one kernel kind: counts them and, in timing mode,
// records an event pair on the launching stream.
struct KernelScope {
  wlseno_ctx* ctx;
  int kind;
  cudaStream_t s;
  cudaEvent_t start = nullptr;
  KernelScope(wlseno_ctx* c, int k, cudaStream_t st) : ctx(c), kind(k), s(st) {
    if (ctx->timing) {
      start = next_event(ctx);
      if (start) cudaEventRecord(start, s);
    }
  }
  void done(int n_launches) {
    ctx->launches += n_launches;
    ctx->by_kind[kind] += n_launches;
    if (start) {
      cudaEvent_t stop = next_event(ctx);
      if (stop) {
        cudaEventRecord(stop, s);
        ctx->timed.push_back({kind, start, stop});
      }
    }
  }
};

void reset_kind_stats(wlseno_ctx* ctx) {
  for (auto& v : ctx->by_kind) v = 0;
  ctx->timed.clear();
  ctx->events_used = 0;
}


// fvals receives the facet values, or with fdev set (FP32-bulk) their FP32
// deviations from the cell averages instead.
// Calls f(integral_constant<dim>, integral_constant<m>) for the compiled
// (dimension, unknowns) pairs: 1-D p = 3, 5; 2-D p = 3, 4; 3-D p = 3.
template <typename F>
cudaError_t dispatch_dim_m(int dim, int m, F&& f) {
  using std::integral_constant;
  if (dim == 1 && m == 3) return f(integral_constant<int, 1>{}, integral_constant<int, 3>{});
  if (dim == 1 && m == 5) return f(integral_constant<int, 1>{}, integral_constant<int, 5>{});
  if (dim == 2 && m == 6) return f(integral_constant<int, 2>{}, integral_constant<int, 6>{});
  if (dim == 2 && m == 10) return f(integral_constant<int, 2>{}, integral_constant<int, 10>{});
  if (dim == 3 && m == 10) return f(integral_constant<int, 3>{}, integral_constant<int, 10>{});
  return cudaErrorInvalidValue;
}

// The all-components FP32-bulk Euler path is in use (thread-per-cell shape).
bool euler_fused(const wlseno_ctx* ctx) { return ctx->euler32 && ctx->G == 1; }

// FP32 pairs of a state (the scratch slot of d_pair), counted as a per-step
// preparation kernel.
cudaError_t split_state(wlseno_ctx* ctx, const double* u, float2* pair, cudaStream_t s) {
  KernelScope scope(ctx, WLSENO_KERNEL_DT, s);
  cudaError_t e = launch_split_pairs(u, pair, ctx->dm.N, s);
  scope.done(e == cudaSuccess ? 1 : 0);
  return e;
}

// pair: the FP32 pairs of ubar for the FP32-bulk thread-per-cell kernel; when
// null they are made here, in the scratch slot of d_pair.
cudaError_t reconstruct_plain(wlseno_ctx* ctx, const double* ubar, double* coeffs, double* fvals,
                              cudaStream_t s, float* fdev, const float2* pair) {
  ReconOut out{coeffs, fdev ? nullptr : fvals, ctx->d_counters, fdev};
  const DeviceMesh& dm = ctx->dm;
  const bool f32 = ctx->scheme.precision == WLSENO_FP32_BULK;
  cudaError_t e = cudaErrorInvalidValue;
  if (f32 && ctx->G == 1 && !pair) {
    if ((e = split_state(ctx, ubar, ctx->d_pair, s)) != cudaSuccess) return e;
    pair = ctx->d_pair;
  }
  // the work-list lengths start at zero (outside the timed kernel scope)
  if (ctx->G == 1 && (e = cudaMemsetAsync(ctx->d_wl_count, 0, 2 * sizeof(int), s)) != cudaSuccess)
    return e;
  KernelScope scope(ctx, WLSENO_KERNEL_RECONSTRUCT, s);
  if (ctx->G == 1) {
    TpcWork wl{ctx->d_wl,   ctx->d_wl_count, ctx->d_rbuf, pair,
               ctx->side,   ctx->ev_fork,    ctx->ev_join, ctx->otf && f32};
    wl.capacity = ctx->wl_cap;
    e = dispatch_dim_m(dm.dim, dm.m, [&](auto D, auto Mc) {
      constexpr int DD = decltype(D)::value, MM = decltype(Mc)::value;
      return f32 ? launch_recon_tpc_inst<float, DD, MM>(dm, ctx->sp, ubar, out, wl, s)
                 : launch_recon_tpc_inst<double, DD, MM>(dm, ctx->sp, ubar, out, wl, s);
    });
    scope.done(e == cudaSuccess ? 1 : 0);
    if (e != cudaSuccess) return e;
    int nl = 0;
    KernelScope fix(ctx, WLSENO_KERNEL_FIXUP, s);
    e = dispatch_dim_m(dm.dim, dm.m, [&](auto D, auto Mc) {
      constexpr int DD = decltype(D)::value, MM = decltype(Mc)::value;
      return f32 ? launch_recon_fixup_inst<float, DD, MM>(dm, ctx->sp, ubar, out, wl, s, &nl)
                 : launch_recon_fixup_inst<double, DD, MM>(dm, ctx->sp, ubar, out, wl, s, &nl);
    });
    fix.done(e == cudaSuccess ? nl : 0);
    return e;
  }
  e = dispatch_dim_m(dm.dim, dm.m, [&](auto D, auto Mc) {
    constexpr int DD = decltype(D)::value, MM = decltype(Mc)::value;
    return f32 ? launch_reconstruct_inst<float, DD, MM>(dm, ctx->sp, ctx->G, ctx->R, ubar, out, s)
               : launch_reconstruct_inst<double, DD, MM>(dm, ctx->sp, ctx->G, ctx->R, ubar, out, s);
  });
  scope.done(e == cudaSuccess ? 1 : 0);
  return e;
}

// The reconstruction followed, when the scheme asks for it, by the
// balanced-stencil re-selection of the cells out of range (counted as
// follow-up kernels).
cudaError_t reconstruct_one(wlseno_ctx* ctx, const double* ubar, double* coeffs, double* fvals,
                            cudaStream_t s, float* fdev = nullptr, const float2* pair = nullptr) {
  cudaError_t e = reconstruct_plain(ctx, ubar, coeffs, fvals, s, fdev, pair);
  if (e != cudaSuccess || !ctx->scheme.balanced) return e;
  const ReconOut out{coeffs, fdev ? nullptr : fvals, ctx->d_counters, fdev};
  int nl = 0;
  KernelScope scope(ctx, WLSENO_KERNEL_FIXUP, s);
  e = launch_balance(ctx->dm, ctx->sp, ctx->bal, ubar, out, s, &nl);
  scope.done(e == cudaSuccess ? nl : 0);
  return e;
}

cudaError_t flux_one(wlseno_ctx* ctx, const double* fvals, const double* u, const double* u0,
                     double a, double b, bool residual_only, double* out, cudaStream_t s,
                     const float* fdev = nullptr, const float2* pin = nullptr, float2* pout = nullptr,
                     const float2* p0 = nullptr) {
  KernelScope scope(ctx, WLSENO_KERNEL_FLUX, s);
  cudaError_t e = launch_flux_stage_impl(ctx->dm, ctx->sp, ctx->scheme.precision, fvals, fdev, u, u0,
                                         a, b, ctx->d_dt, residual_only, out, ctx->d_counters, s,
                                         pin, pout, p0, ctx->d_dt2);
  scope.done(e == cudaSuccess ? 1 : 0);
  return e;
}

// One RK stage (or the residual) over all components: out = a u0 + b (u + dt
// L(u)), or L(u) itself.  Euler reconstructs every component, applies the
// positivity fix-up and runs the coupled flux; scalar equations go component
// by component.
// FP32-bulk scalar path: pin holds the FP32 pairs of u (else they are made
// here), pout (may be null) receives those of out, p0 (may be null) holds
// those of u0.
cudaError_t stage_all(wlseno_ctx* ctx, const double* u, const double* u0, double a, double b,
                      bool residual_only, double* out, cudaStream_t s, const float2* pin = nullptr,
                      float2* pout = nullptr, const float2* p0 = nullptr) {
  const int64_t N = ctx->dm.N;
  const int C = ctx->scheme.n_comp;
  const int NP = (ctx->dm.dim + 1) * ctx->dm.nq;
  cudaError_t e = cudaSuccess;
  if (euler_fused(ctx)) {
    // FP32-bulk 2-D Euler: the pairs of u (interleaved), one reconstruction
    // of all components with the positivity flags, its follow-ups, the flux
    const DeviceMesh& dm = ctx->dm;
    const float2* pu = pin;
    if (!pu) {
      KernelScope sp_scope(ctx, WLSENO_KERNEL_DT, s);
      e = launch_euler2_split_pairs(u, ctx->d_pair, N, s);
      sp_scope.done(e == cudaSuccess ? 1 : 0);
      if (e != cudaSuccess) return e;
      pu = ctx->d_pair;
    }
    if ((e = cudaMemsetAsync(ctx->d_wl_count, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
    TpcWork wl{ctx->d_wl, ctx->d_wl_count, ctx->d_rbuf, pu, ctx->side, ctx->ev_fork, ctx->ev_join, ctx->otf};
    wl.capacity = ctx->wl_cap;
    wl.pos_ok = ctx->d_pos_ok;
    wl.gamma = static_cast<float>(ctx->sp.gamma);
    const ReconOut ro{nullptr, nullptr, ctx->d_counters, ctx->d_fdev};
    {
      KernelScope scope(ctx, WLSENO_KERNEL_RECONSTRUCT, s);
      e = launch_recon_euler2d(dm, ctx->sp, u, ro, wl, s);
      scope.done(e == cudaSuccess ? 1 : 0);
      if (e != cudaSuccess) return e;
    }
    {
      int nl = 0;
      KernelScope fix(ctx, WLSENO_KERNEL_FIXUP, s);
      e = launch_recon_fixup_inst<float, 2, 6>(dm, ctx->sp, u, ro, wl, s, &nl);
      fix.done(e == cudaSuccess ? nl : 0);
      if (e != cudaSuccess) return e;
    }
    KernelScope scope(ctx, WLSENO_KERNEL_FLUX, s);
    e = launch_euler2_flux32(dm, ctx->sp.gamma, ctx->d_fdev, pu, p0, a, b, ctx->d_dt2, residual_only, out,
                             ctx->d_counters, pout, s);
    scope.done(e == cudaSuccess ? 1 : 0);
    return e;
  }
  if (ctx->scheme.pde == WLSENO_EULER) {
    if (ctx->scheme.characteristic) {
      KernelScope scope(ctx, WLSENO_KERNEL_RECONSTRUCT, s);
      e = launch_euler_char(ctx->dm, ctx->sp, ctx->scheme.precision, u, ctx->d_fvals, ctx->d_counters, s);
      scope.done(e == cudaSuccess ? 1 : 0);
    } else {
      for (int c = 0; c < C && e == cudaSuccess; ++c)
        e = reconstruct_one(ctx, u + c * N, nullptr, ctx->d_fvals + c * N * NP, s);
    }
    if (e != cudaSuccess) return e;
    KernelScope scope(ctx, WLSENO_KERNEL_FLUX, s);
    e = launch_euler_positivity(ctx->dm, ctx->sp.gamma, u, ctx->d_fvals, ctx->d_counters, s);
    if (e == cudaSuccess)
      e = launch_euler_flux_stage(ctx->dm, ctx->sp.gamma, ctx->scheme.precision, ctx->d_fvals, u, u0,
                                  a, b, ctx->d_dt, residual_only, out, ctx->d_counters, s);
    scope.done(e == cudaSuccess ? 2 : 0);
    return e;
  }
  // FP32-bulk thread-per-cell: facet values travel as FP32 deviations
  float* fdev = ctx->G == 1 ? ctx->d_fdev : nullptr;
  for (int c = 0; c < C && e == cudaSuccess; ++c) {
    const float2* pc = nullptr;
    if (fdev) {
      if (pin) {
        pc = pin + c * N;
      } else if ((e = split_state(ctx, u + c * N, ctx->d_pair, s)) == cudaSuccess) {
        pc = ctx->d_pair;
      }
    }
    if (e == cudaSuccess) e = reconstruct_one(ctx, u + c * N, nullptr, ctx->d_fvals, s, fdev, pc);
    if (e == cudaSuccess)
      e = flux_one(ctx, ctx->d_fvals, u + c * N, u0 ? u0 + c * N : nullptr, a, b, residual_only,
                   out + c * N, s, fdev, pc, fdev && pout ? pout + c * N : nullptr,
                   fdev && p0 ? p0 + c * N : nullptr);
  }
  return e;
}

// One stage's reconstruction with the context's current shape, for the
// autotuner: the all-components Euler kernel with its follow-ups, or every
// component through the one-component kernels.
cudaError_t tune_recon(wlseno_ctx* ctx, const double* u, cudaStream_t s) {
  const int64_t N = ctx->dm.N;
  if (euler_fused(ctx)) {
    cudaError_t e = launch_euler2_split_pairs(u, ctx->d_pair, N, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctx->d_wl_count, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
    TpcWork wl{ctx->d_wl, ctx->d_wl_count, ctx->d_rbuf, ctx->d_pair, ctx->side, ctx->ev_fork, ctx->ev_join,
               ctx->otf};
    wl.capacity = ctx->wl_cap;
    wl.pos_ok = ctx->d_pos_ok;
    wl.gamma = static_cast<float>(ctx->sp.gamma);
    const ReconOut ro{nullptr, nullptr, ctx->d_counters, ctx->d_fdev};
    if ((e = launch_recon_euler2d(ctx->dm, ctx->sp, u, ro, wl, s)) != cudaSuccess) return e;
    int nl = 0;
    return launch_recon_fixup_inst<float, 2, 6>(ctx->dm, ctx->sp, u, ro, wl, s, &nl);
  }
  const int C = ctx->scheme.pde == WLSENO_EULER ? ctx->scheme.n_comp : 1;
  const int NP = (ctx->dm.dim + 1) * ctx->dm.nq;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < C && e == cudaSuccess; ++c)
    e = reconstruct_one(ctx, u + c * N, nullptr, ctx->d_fvals + c * N * NP, s);
  return e;
}

// The kernel variant a captured step used: shape and moments mode.
int shape_key(const wlseno_ctx* ctx) { return (ctx->G * 64 + ctx->R) * 2 + (ctx->otf ? 1 : 0); }

wlseno_status check_ready(wlseno_ctx* ctx) {
  if (!ctx) return WLSENO_ERR_INVALID_ARG;
  if (!ctx->built || !ctx->moments_ready)
    return fail(ctx, WLSENO_ERR_STATE, "call wlseno_build_stencils and wlseno_precompute_moments first");
  return WLSENO_OK;
}

// Non-finite values written by kernels the context launched earlier (seen
// once their work has reached the status word): reported once, then cleared.
wlseno_status take_nonfinite(wlseno_ctx* ctx) {
  volatile unsigned int* latch = ctx->h_latch;
  if (!latch) return WLSENO_OK;
  if (latch[1] != 0u) {
    latch[1] = 0u;
    latch[0] = 0u;  // the results of a step that gave up are not reported twice
    return fail(ctx, WLSENO_ERR_TIMEOUT,
                "a grid barrier of the persistent step kernel waited longer than its poll limit; "
                "the state of that step is incomplete");
  }
  if (latch[0] == 0u) return WLSENO_OK;
  latch[0] = 0u;
  return fail(ctx, WLSENO_ERR_NUMERIC,
              "non-finite values in the results (cell averages, facet values or residuals) of "
              "work this context ran");
}

}  // namespace

namespace wlseno {

// FP32-bulk: refine above kappa_flag, pivot above 1e5 (one FP32 refinement
// sweep contracts the error by about kappa 2^-24); FP64: pivot above 1e6.  A rank tolerance above 1e-8 lowers the pivot bound to 1e-2 /
// rank_tol, so that every cell whose rank the rule of Sec. 3.3.2 might cut
// still reaches the pivoted path (the estimates bound the conditioning from
// below; from rank_tol >= 1e-2 on every cell goes there).
void tpc_thresholds(const SchemeParams& sp, bool f32, double* flag, double* pivot) {
  const double route = sp.rank_tol > 0.0 ? 1e-2 / sp.rank_tol : 1e300;
  *pivot = std::fmin(f32 ? 1e5 : 1e6, route);
  *flag = f32 ? std::fmin(sp.kappa_flag, *pivot) : *pivot;
}

bool ctx_view(const wlseno_ctx* ctx, CtxView* out) {
  if (!ctx || !out) return false;
  out->device = ctx->device;
  out->precision = ctx->scheme.precision;
  out->n_comp = ctx->scheme.n_comp;
  out->ready = ctx->built && ctx->moments_ready;
  out->dm = ctx->dm;
  out->sp = ctx->sp;
  out->counters = ctx->d_counters;
  out->dt = ctx->d_dt;
  out->dev_facets = ctx->d_fdev != nullptr && ctx->G == 1;
  return true;
}

void ctx_set_error(wlseno_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->error = msg;
}

cudaError_t ctx_launch_reconstruct(wlseno_ctx* ctx, const double* ubar, const ReconOut& out,
                                   cudaStream_t s) {
  ctx->last_stream = s;
  return reconstruct_one(ctx, ubar, out.coeffs, out.fvals, s, out.fdev);
}

// With fdev, the pairs of ubar are the ones ctx_launch_reconstruct just made
// in the scratch slot (same ubar, same stream).
cudaError_t ctx_launch_flux_residual(wlseno_ctx* ctx, const double* fvals, const float* fdev,
                                     const double* ubar, double* residual, cudaStream_t s) {
  return flux_one(ctx, fvals, ubar, nullptr, 0.0, 1.0, true, residual, s, fdev,
                  fdev ? ctx->d_pair : nullptr);
}

}  // namespace wlseno

extern "C" {

const char* wlseno_status_string(wlseno_status s) {
  switch (s) {
    case WLSENO_OK: return "ok";
    case WLSENO_ERR_INVALID_ARG: return "invalid argument";
    case WLSENO_ERR_MESH: return "invalid mesh";
    case WLSENO_ERR_STENCIL: return "invalid stencil";
    case WLSENO_ERR_CUDA: return "CUDA error";
    case WLSENO_ERR_OOM: return "out of memory";
    case WLSENO_ERR_NUMERIC: return "non-finite value";
    case WLSENO_ERR_TIMEOUT: return "device wait timed out";
    case WLSENO_ERR_STATE: return "calls made in the wrong order";
  }
  return "unknown status";
}

const char* wlseno_last_error_message(const wlseno_ctx* ctx) {
  return ctx ? ctx->error.c_str() : "null context";
}

wlseno_status wlseno_create(wlseno_ctx** out, int device, const wlseno_scheme* scheme) {
  if (!out || !scheme) return WLSENO_ERR_INVALID_ARG;
  *out = nullptr;
  if (scheme->pde != WLSENO_ADVECTION && scheme->pde != WLSENO_BURGERS && scheme->pde != WLSENO_EULER)
    return WLSENO_ERR_INVALID_ARG;
  if (scheme->pde == WLSENO_EULER ? (scheme->n_comp < 3 || scheme->n_comp > 5) || !(scheme->gamma > 1.0)
                                  : scheme->n_comp != 1)
    return WLSENO_ERR_INVALID_ARG;
  if (scheme->precision != WLSENO_FP64 && scheme->precision != WLSENO_FP32_BULK)
    return WLSENO_ERR_INVALID_ARG;
  if (scheme->characteristic != 0 && (scheme->characteristic != 1 || scheme->pde != WLSENO_EULER))
    return WLSENO_ERR_INVALID_ARG;
  if (scheme->balanced != 0 &&
      (scheme->balanced != 1 || scheme->pde == WLSENO_EULER || !(scheme->balance_margin >= 0.0) ||
       !std::isfinite(scheme->balance_margin)))
    return WLSENO_ERR_INVALID_ARG;
  if (!(scheme->eps > 0.0) || !(scheme->alpha_c > 0.0) || !(scheme->rank_tol >= 0.0))
    return WLSENO_ERR_INVALID_ARG;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return WLSENO_ERR_CUDA;
  }
  wlseno_ctx* ctx = new (std::nothrow) wlseno_ctx();
  if (!ctx) return WLSENO_ERR_OOM;
  ctx->device = device;
  if (const char* lim = std::getenv("WLSENO_DEVICE_BYTES_LIMIT")) {
    char* end = nullptr;
    const unsigned long long v = std::strtoull(lim, &end, 10);
    if (end != lim && *end == '\0') ctx->alloc_limit = static_cast<size_t>(v);
  }
  {
    DeviceGuard guard(device);
    void* h = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&h, 2 * sizeof(unsigned int), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
      cudaGetLastError();
      if (h) cudaFreeHost(h);
      delete ctx;
      return WLSENO_ERR_CUDA;
    }
    ctx->h_latch = static_cast<unsigned int*>(h);
    ctx->d_latch = static_cast<unsigned int*>(d);
    ctx->h_latch[0] = ctx->h_latch[1] = 0u;
  }
  ctx->scheme = *scheme;
  ctx->sp.pde = scheme->pde;
  for (int a = 0; a < 3; ++a) ctx->sp.vel[a] = scheme->velocity[a];
  ctx->sp.eps = scheme->eps;
  ctx->sp.alpha_c = scheme->alpha_c;
  ctx->sp.alpha_c32 = static_cast<float>(scheme->alpha_c);
  ctx->sp.rank_tol = scheme->rank_tol;
  ctx->sp.kappa_flag = scheme->kappa_flag > 0.0 ? scheme->kappa_flag : 1e3;
  ctx->sp.gamma = scheme->gamma;
  *out = ctx;
  return WLSENO_OK;
}

void wlseno_destroy(wlseno_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx->device);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    free_all(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->h_latch) cudaFreeHost(ctx->h_latch);
  }
  delete ctx;
}

wlseno_status wlseno_build_stencils(wlseno_ctx* ctx, const wlseno_mesh* meshes, int n_meshes,
                                    const wlseno_stencil_opts* opts, int64_t* perm_out) {
  if (!ctx) return WLSENO_ERR_INVALID_ARG;
  if (opts && opts->reorder != 0 && opts->reorder != 1)
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "reorder must be 0 or 1");
  if (opts && opts->persistent != 0 && opts->persistent != 1)
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "persistent must be 0 or 1");
  // Hilbert order: permuted copies of the meshes' cell arrays
  std::vector<wlseno_mesh> reordered;
  std::vector<std::vector<int64_t>> cells_new;
  std::vector<int64_t> perm;
  if (meshes && n_meshes > 0 && opts && opts->reorder == 1) {
    reordered.assign(meshes, meshes + n_meshes);
    cells_new.resize(n_meshes);
    int64_t base = 0;
    for (int k = 0; k < n_meshes; ++k) {
      const wlseno_mesh& m = meshes[k];
      if (!m.cells || !m.vertices || m.n_cells <= 0 || m.dim < 1 || m.dim > 3)
        return fail(ctx, WLSENO_ERR_INVALID_ARG, "mesh " + std::to_string(k) + ": null arrays or bad sizes");
      std::vector<int64_t> order;
      if (!hilbert_order(m, &order))
        return fail(ctx, WLSENO_ERR_MESH, "mesh " + std::to_string(k) + ": vertex index out of range");
      const int nv = m.dim + 1;
      cells_new[k].resize(static_cast<size_t>(m.n_cells) * nv);
      for (int64_t c = 0; c < m.n_cells; ++c) {
        for (int v = 0; v < nv; ++v) cells_new[k][c * nv + v] = m.cells[order[c] * nv + v];
        perm.push_back(base + order[c]);
      }
      reordered[k].cells = cells_new[k].data();
      base += m.n_cells;
    }
    meshes = reordered.data();
  }
  DeviceGuard guard(ctx->device);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);  // it captured the old buffers
  ctx->graph_exec = nullptr;
  free_all(ctx);
  ctx->built = ctx->moments_ready = false;
  ctx->mesh_dt_set = false;
  ctx->adj = AdjointWork{};
  std::string err;
  HostSetup& H = ctx->host;
  // balanced stencils draw from the (ceil(ring) + 1)-vertex ring
  const int bal_steps =
      ctx->scheme.balanced && opts ? static_cast<int>(std::ceil(opts->ring - 1e-9)) + 1 : 0;
  ctx->bal = BalanceWork{};
  wlseno_status st = build_host_setup(meshes, n_meshes, opts, &H, &err, bal_steps);
  if (st != WLSENO_OK) return fail(ctx, st, err);
  if (ctx->scheme.pde == WLSENO_EULER && ctx->scheme.n_comp != H.dim + 2)
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "Euler needs n_comp = dim + 2 (3, 4 or 5)");
  if (ctx->scheme.characteristic && H.dim > 2)
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "characteristic-wise reconstruction is built for 1-D and 2-D meshes");
  if ((H.dim == 1 && H.m != 3 && H.m != 5) || (H.dim == 2 && H.m != 6 && H.m != 10) ||
      (H.dim == 3 && H.m != 10))
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "order p not compiled for this dimension");
  int G = opts->lanes_per_cell, R = opts->rows_per_lane;
  if (G == 0 && R == 0) {
    choose_shape(H.max_n, &G, &R);
  } else if (!shape_ok(G, R)) {
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "lanes_per_cell/rows_per_lane not compiled");
  }
  if (G == 0 || !shape_fits(G, R, H.max_n))
    return fail(ctx, WLSENO_ERR_STENCIL, "largest stencil (" + std::to_string(H.max_n) +
                                             " cells) exceeds the kernel's rows");
  if (opts->moments_mode != 0 &&
      (opts->moments_mode != 1 || G != 1 || ctx->scheme.precision != WLSENO_FP32_BULK))
    return fail(ctx, WLSENO_ERR_INVALID_ARG,
                "moments_mode 1 needs FP32-bulk precision and the thread-per-cell shape");
  if (opts->persistent &&
      (ctx->scheme.pde == WLSENO_EULER || ctx->scheme.balanced || G != 1 || !persistent_supported(H.dim, H.m)))
    return fail(ctx, WLSENO_ERR_INVALID_ARG,
                "the persistent step is built for the scalar equations on 2-D meshes (p = 3, 4), fixed "
                "stencils and the thread-per-cell shape");
  ctx->G = G;
  ctx->R = R;
  ctx->otf = opts->moments_mode == 1;
  ctx->persistent = opts->persistent == 1;
  const int64_t N = H.N;
  std::vector<int32_t> ptr32(N + 1), idx32(H.nnz);
  for (int64_t i = 0; i <= N; ++i) ptr32[i] = static_cast<int32_t>(H.row_ptr[i]);
  for (int64_t i = 0; i < H.nnz; ++i) idx32[i] = static_cast<int32_t>(H.cols[i]);
  std::vector<float> fpts32(H.fpts.begin(), H.fpts.end());
  DeviceMesh& dm = ctx->dm;
  dm = DeviceMesh{};
  dm.dim = H.dim;
  dm.p = H.p;
  dm.m = H.m;
  dm.nq = H.nq;
  dm.N = N;
  dm.nnz = H.nnz;
  double *coords, *centroid, *h, *vol, *ivol, *inr, *period, *fgeo, *fpts;
  int32_t *mesh_of, *nbr;
  float* fp32;
  std::vector<double> inv_volume(H.volume.size());
  for (size_t k = 0; k < inv_volume.size(); ++k) inv_volume[k] = 1.0 / H.volume[k];
  if ((st = upload(ctx, &ctx->d_st_ptr, ptr32)) || (st = upload(ctx, &ctx->d_st_idx, idx32)) ||
      (st = upload(ctx, &coords, H.coords)) || (st = upload(ctx, &centroid, H.centroid)) ||
      (st = upload(ctx, &h, H.h)) || (st = upload(ctx, &vol, H.volume)) ||
      (st = upload(ctx, &ivol, inv_volume)) ||
      (st = upload(ctx, &inr, H.inradius)) || (st = upload(ctx, &mesh_of, H.mesh_of)) ||
      (st = upload(ctx, &period, H.period)) || (st = upload(ctx, &nbr, H.nbr)) ||
      (st = upload(ctx, &fgeo, H.fgeo)) || (st = upload(ctx, &fpts, H.fpts)) ||
      (st = upload(ctx, &fp32, fpts32)) || (st = upload(ctx, &ctx->d_rmin, H.rmin)))
    return st;
  dm.st_ptr = ctx->d_st_ptr;
  dm.st_idx = ctx->d_st_idx;
  dm.coords = coords;
  dm.centroid = centroid;
  dm.h = h;
  dm.volume = vol;
  dm.inv_volume = ivol;
  dm.inradius = inr;
  dm.mesh_of = mesh_of;
  dm.period = period;
  dm.nbr = nbr;
  dm.fgeo = fgeo;
  dm.fpts = fpts;
  dm.fpts32 = fp32;
  dm.ff32 = nullptr;
  dm.inv_vol2 = nullptr;
  dm.nf_latch = ctx->d_latch;
  dm.nf32 = nullptr;
  dm.hscale32 = nullptr;
  if (ctx->scheme.precision == WLSENO_FP32_BULK) {
    std::vector<float2> hs(static_cast<size_t>(N));
    for (int64_t i = 0; i < N; ++i) {
      const double hh = H.h[i];
      hs[i] = make_float2(static_cast<float>(ctx->sp.eps * hh * hh), static_cast<float>(1.0 / hh));
    }
    float2* d_hs = nullptr;
    if ((st = upload(ctx, &d_hs, hs))) return st;
    dm.hscale32 = d_hs;
  }
  ctx->euler32 = ctx->scheme.precision == WLSENO_FP32_BULK && ctx->scheme.pde == WLSENO_EULER &&
                 !ctx->scheme.characteristic && H.dim == 2 && H.m == 6;
  if (ctx->euler32) {
    // FP32 owner normal and area of every (cell, facet) record, 1/|tau| pairs
    const int nf = H.dim + 1;
    std::vector<float4> nf4(static_cast<size_t>(N) * nf);
    for (size_t k = 0; k < nf4.size(); ++k) {
      const double* G = &H.fgeo[k * 4];
      nf4[k] = make_float4(static_cast<float>(G[0]), static_cast<float>(G[1]), 0.0f, static_cast<float>(G[3]));
    }
    float4* d_nf = nullptr;
    if ((st = upload(ctx, &d_nf, nf4))) return st;
    dm.nf32 = d_nf;
  }
  if (ctx->scheme.precision == WLSENO_FP32_BULK && (ctx->scheme.pde != WLSENO_EULER || ctx->euler32)) {
    const int nf = H.dim + 1;
    std::vector<FacetF32> ff(static_cast<size_t>(N) * nf);
    for (size_t k = 0; k < ff.size(); ++k) {
      const double* G = &H.fgeo[k * 4];
      double nsum = 0.0, vn = 0.0;
      for (int a = 0; a < H.dim; ++a) {
        nsum += G[a];
        vn += ctx->sp.vel[a] * G[a];
      }
      const bool adv = ctx->scheme.pde == WLSENO_ADVECTION;
      const double pref = adv ? G[3] * vn : 0.5 * G[3] * nsum;
      ff[k].pref_hi = static_cast<float>(pref);
      ff[k].pref_lo = static_cast<float>(pref - static_cast<double>(ff[k].pref_hi));
      ff[k].coef = static_cast<float>(adv ? vn : nsum);
      ff[k].area = static_cast<float>(G[3]);
    }
    FacetF32* d_ff = nullptr;
    if ((st = upload(ctx, &d_ff, ff))) return st;
    dm.ff32 = ctx->scheme.pde == WLSENO_EULER ? nullptr : d_ff;
    std::vector<float2> iv(static_cast<size_t>(N));
    for (int64_t i = 0; i < N; ++i) {
      const double v = 1.0 / H.volume[i];
      const float hi = static_cast<float>(v);
      iv[i] = make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
    }
    float2* d_iv = nullptr;
    if ((st = upload(ctx, &d_iv, iv))) return st;
    dm.inv_vol2 = d_iv;
  }
  const int C = ctx->scheme.n_comp;
  const int NP = (H.dim + 1) * H.nq;
  if ((st = dalloc(ctx, &dm.A64, H.nnz * H.m)) || (st = dalloc(ctx, &dm.A32, H.nnz * H.m)) ||
      (st = dalloc(ctx, &ctx->d_dt, H.n_meshes)) || (st = dalloc(ctx, &ctx->d_dt2, H.n_meshes)) ||
      (st = dalloc(ctx, &ctx->d_lmax, H.n_meshes)) ||
      (st = dalloc(ctx, &ctx->d_counters, kCounters)) || (st = dalloc(ctx, &ctx->d_fvals, C * N * NP)) ||
      (st = dalloc(ctx, &ctx->d_k1, C * N)) || (st = dalloc(ctx, &ctx->d_k2, C * N)))
    return st;
  dm.nmax = H.max_n;
  const size_t ell = static_cast<size_t>(H.max_n) * N;
  ctx->wl_cap = ctx->euler32 ? static_cast<int64_t>(C) * N : N;
  dm.rec_width = rec32_width(H.m);
  if ((st = dalloc(ctx, &dm.st_ell, ell)) || (st = dalloc(ctx, &dm.A64e, ell * H.m)) ||
      (st = dalloc(ctx, &dm.rec32, ell * dm.rec_width)) || (st = dalloc(ctx, &ctx->d_wl, ctx->wl_cap)) ||
      (st = dalloc(ctx, &ctx->d_wl_count, 2)))
    return st;
  dm.geo32 = dm.own32 = nullptr;
  dm.own_width = own32_width(H.dim, H.m);
  if (ctx->scheme.precision == WLSENO_FP32_BULK &&
      ((st = dalloc(ctx, &ctx->d_fdev, (ctx->euler32 ? C : 1) * N * NP)) ||
       (st = dalloc(ctx, &ctx->d_pair, 3 * C * N)) ||
       (st = dalloc(ctx, &ctx->d_rbuf, static_cast<size_t>(refine_record_floats(H.m)) * ctx->wl_cap)) ||
       (st = dalloc(ctx, &dm.geo32, ell * 4)) ||
       (st = dalloc(ctx, &dm.own32, static_cast<size_t>(N) * dm.own_width))))
    return st;
  if (ctx->euler32 && (st = dalloc(ctx, &ctx->d_pos_ok, N))) return st;
  if (ctx->persistent && ((st = dalloc(ctx, &ctx->d_counts6, 6)) || (st = dalloc(ctx, &ctx->d_sync, 4))))
    return st;
  ctx->persist_no_capture = false;
  if (ctx->scheme.balanced) {
    BalanceWork& b = ctx->bal;
    std::vector<int32_t> bp(N + 1), bi(H.bal_idx.size());
    for (int64_t i = 0; i <= N; ++i) bp[i] = static_cast<int32_t>(H.bal_ptr[i]);
    for (size_t k = 0; k < bi.size(); ++k) bi[k] = static_cast<int32_t>(H.bal_idx[k]);
    int32_t *d_bp = nullptr, *d_bi = nullptr;
    if ((st = upload(ctx, &d_bp, bp)) || (st = upload(ctx, &d_bi, bi)) ||
        (st = dalloc(ctx, &b.state, 1 + 2 * static_cast<size_t>(H.n_meshes))) ||
        (st = dalloc(ctx, &b.list, N)))
      return st;
    b.cand_ptr = d_bp;
    b.cand_idx = d_bi;
    b.count = ctx->d_counters + 4;
    b.margin = ctx->scheme.balance_margin;
    b.n_meshes = H.n_meshes;
  }
  cudaError_t e = cudaMemset(ctx->d_counters, 0, kCounters * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemset");
  if (ctx->scheme.precision == WLSENO_FP32_BULK && !ctx->side) {
    if ((e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(ctx, e, "side stream");
  }
  ctx->d_in = ctx->d_out = ctx->d_coef = ctx->d_fv_out = nullptr;
  ctx->built = true;
  if (perm_out) {
    if (perm.empty())
      for (int64_t k = 0; k < N; ++k) perm_out[k] = k;
    else
      std::memcpy(perm_out, perm.data(), sizeof(int64_t) * N);
  }
  return WLSENO_OK;
}

wlseno_status wlseno_precompute_moments(wlseno_ctx* ctx, void* stream) {
  if (!ctx) return WLSENO_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, WLSENO_ERR_STATE, "call wlseno_build_stencils first");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  KernelScope scope(ctx, WLSENO_KERNEL_MOMENTS, s);
  cudaError_t e = launch_moments(ctx->dm, s);
  if (e == cudaSuccess) e = launch_ell_copy(ctx->dm, s);
  scope.done(e == cudaSuccess ? 2 : 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "moments kernel");
  ctx->moments_ready = true;
  ctx->last_stream = s;
  return WLSENO_OK;
}

wlseno_status wlseno_reconstruct(wlseno_ctx* ctx, const double* ubar, double* coeffs,
                                 double* facet_values, void* stream) {
  wlseno_status st = check_ready(ctx);
  if (st != WLSENO_OK || (st = take_nonfinite(ctx)) != WLSENO_OK) return st;
  if (!ubar) return fail(ctx, WLSENO_ERR_INVALID_ARG, "ubar is null");
  if (ctx->scheme.characteristic && coeffs)
    return fail(ctx, WLSENO_ERR_INVALID_ARG,
                "characteristic reconstruction has no per-cell polynomial: pass coeffs = NULL");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->last_stream = s;
  const int64_t N = ctx->dm.N;
  const int C = ctx->scheme.n_comp, m = ctx->dm.m, NP = points_per_cell(ctx);
  bool host_io = false;
  const double* u = ubar;
  cudaError_t e;
  if (!is_device_pointer(ubar)) {
    if (!ctx->d_in && (st = dalloc(ctx, &ctx->d_in, C * N))) return st;
    e = cudaMemcpyAsync(ctx->d_in, ubar, sizeof(double) * C * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy ubar");
    u = ctx->d_in;
    host_io = true;
  }
  const bool coef_host = coeffs && !is_device_pointer(coeffs);
  const bool fv_host = facet_values && !is_device_pointer(facet_values);
  if (coef_host && !ctx->d_coef && (st = dalloc(ctx, &ctx->d_coef, C * N * m))) return st;
  if (fv_host && !ctx->d_fv_out && (st = dalloc(ctx, &ctx->d_fv_out, C * N * NP))) return st;
  if ((e = cudaMemsetAsync(ctx->d_counters, 0, kCounters * sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset counters");
  if (ctx->scheme.characteristic) {
    // facet values of all components at once (there is no per-cell polynomial)
    double* fv = facet_values ? (fv_host ? ctx->d_fv_out : facet_values) : ctx->d_fvals;
    KernelScope scope(ctx, WLSENO_KERNEL_RECONSTRUCT, s);
    e = launch_euler_char(ctx->dm, ctx->sp, ctx->scheme.precision, u, fv, ctx->d_counters, s);
    scope.done(e == cudaSuccess ? 1 : 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reconstruction kernel");
  }
  for (int c = 0; c < C && !ctx->scheme.characteristic; ++c) {
    double* co = coeffs ? (coef_host ? ctx->d_coef : coeffs) + c * N * m : nullptr;
    double* fv = facet_values ? (fv_host ? ctx->d_fv_out : facet_values) + c * N * NP : ctx->d_fvals;
    e = reconstruct_one(ctx, u + c * N, co, fv, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reconstruction kernel");
  }
  if (coef_host) {
    e = cudaMemcpyAsync(coeffs, ctx->d_coef, sizeof(double) * C * N * m, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy coeffs");
  }
  if (fv_host) {
    e = cudaMemcpyAsync(facet_values, ctx->d_fv_out, sizeof(double) * C * N * NP,
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy facet values");
  }
  if (host_io || coef_host || fv_host) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reconstruct");
    return take_nonfinite(ctx);
  }
  return WLSENO_OK;
}

wlseno_status wlseno_flux_residual(wlseno_ctx* ctx, const double* ubar, double* residual,
                                   void* stream) {
  wlseno_status st = check_ready(ctx);
  if (st != WLSENO_OK || (st = take_nonfinite(ctx)) != WLSENO_OK) return st;
  if (!ubar || !residual) return fail(ctx, WLSENO_ERR_INVALID_ARG, "null array");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->last_stream = s;
  const int64_t N = ctx->dm.N;
  const int C = ctx->scheme.n_comp;
  cudaError_t e;
  const double* u = ubar;
  const bool in_host = !is_device_pointer(ubar);
  const bool out_host = !is_device_pointer(residual);
  if (in_host) {
    if (!ctx->d_in && (st = dalloc(ctx, &ctx->d_in, C * N))) return st;
    e = cudaMemcpyAsync(ctx->d_in, ubar, sizeof(double) * C * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy ubar");
    u = ctx->d_in;
  }
  if (out_host && !ctx->d_out && (st = dalloc(ctx, &ctx->d_out, C * N))) return st;
  double* res = out_host ? ctx->d_out : residual;
  if ((e = cudaMemsetAsync(ctx->d_counters, 0, kCounters * sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset counters");
  if ((e = stage_all(ctx, u, nullptr, 0.0, 1.0, true, res, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "residual kernels");
  if (out_host) {
    e = cudaMemcpyAsync(residual, ctx->d_out, sizeof(double) * C * N, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy residual");
  }
  if (in_host || out_host) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "flux_residual");
    return take_nonfinite(ctx);
  }
  return WLSENO_OK;
}

wlseno_status wlseno_rk_step(wlseno_ctx* ctx, double* ubar, double dt, double cfl, int n_steps,
                             double* dt_out, void* stream) {
  wlseno_status st = check_ready(ctx);
  if (st != WLSENO_OK || (st = take_nonfinite(ctx)) != WLSENO_OK) return st;
  if (!ubar || n_steps < 0) return fail(ctx, WLSENO_ERR_INVALID_ARG, "null ubar or n_steps < 0");
  if (dt < 0.0 && !ctx->mesh_dt_set)
    return fail(ctx, WLSENO_ERR_STATE, "dt < 0 needs wlseno_set_mesh_dt first");
  if (dt == 0.0 && !(cfl > 0.0)) return fail(ctx, WLSENO_ERR_INVALID_ARG, "need dt != 0 or cfl > 0");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->last_stream = s;
  const int64_t N = ctx->dm.N;
  const int C = ctx->scheme.n_comp;
  cudaError_t e;
  const bool host = !is_device_pointer(ubar);
  double* u = ubar;
  if (host) {
    if (!ctx->d_in && (st = dalloc(ctx, &ctx->d_in, C * N))) return st;
    e = cudaMemcpyAsync(ctx->d_in, ubar, sizeof(double) * C * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy ubar");
    u = ctx->d_in;
  }
  if ((e = cudaMemsetAsync(ctx->d_counters, 0, kCounters * sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset counters");
  // one TVD-RK3 step on stream `st` (Sec. 4.2.1, Eq. (3rd-order-Runge-Kutta))
  // FP32-bulk scalar thread-per-cell path: the FP32 pairs of u for stage 1
  // are made with the time step (scratch slot of d_pair; stages 2 and 3 read
  // them as the pairs of u0)
  const bool fused = euler_fused(ctx);
  float2* pre = ctx->d_pair && ctx->G == 1 && ((C == 1 && ctx->scheme.pde != WLSENO_EULER) || fused)
                    ? ctx->d_pair : nullptr;
  const bool persist = ctx->persistent && ctx->G == 1;
  auto enqueue_step = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t err = cudaSuccess;
    if (persist) {
      // the whole step in one persistent cooperative kernel
      PersistLaunch L;
      L.dm = ctx->dm;
      L.sp = ctx->sp;
      L.fp32 = ctx->scheme.precision == WLSENO_FP32_BULK;
      L.otf = ctx->otf && L.fp32;
      L.u = u;
      L.k1 = ctx->d_k1;
      L.k2 = ctx->d_k2;
      L.pairs = ctx->d_pair;
      L.fvals = ctx->d_fvals;
      L.fdev = ctx->d_fdev;
      L.counters = ctx->d_counters;
      L.group_list = ctx->d_wl;
      L.counts = ctx->d_counts6;
      L.refine_buf = ctx->d_rbuf;
      L.capacity = ctx->wl_cap;
      L.dt_mode = dt > 0.0 ? 1 : dt == 0.0 ? 0 : 2;
      L.cfl = cfl;
      L.dt_fixed = dt > 0.0 ? dt : 0.0;
      double sp2 = 0.0;
      for (int a = 0; a < ctx->dm.dim; ++a) sp2 += ctx->sp.vel[a] * ctx->sp.vel[a];
      L.adv_speed = std::sqrt(sp2);  // as launch_cfl_dt_impl and the flux kernels take it
      L.n_meshes = ctx->host.n_meshes;
      L.rmin = ctx->d_rmin;
      L.lmax = dt == 0.0 && ctx->scheme.pde == WLSENO_BURGERS ? ctx->d_lmax : nullptr;
      L.dt_mesh = ctx->d_dt;
      L.dt2 = ctx->d_dt2;
      L.sync_words = ctx->d_sync;
      L.timeout_word = ctx->d_latch + 1;
      L.spin_cap = ctx->spin_cap;
      tpc_thresholds(ctx->sp, L.fp32, &L.flag, &L.pivot);
      KernelScope scope(ctx, WLSENO_KERNEL_STEP, st);
      err = launch_persistent_step(L, st);
      scope.done(err == cudaSuccess ? 1 : 0);
      return err;
    }
    if (dt >= 0.0) {  // dt < 0: the per-mesh steps already in d_dt
      int nl = 0;
      KernelScope scope(ctx, WLSENO_KERNEL_DT, st);
      err = launch_cfl_dt_impl(ctx->dm, ctx->sp, ctx->host.n_meshes, u, ctx->d_rmin, cfl,
                               dt > 0.0 ? dt : 0.0, ctx->d_lmax, ctx->d_dt, st, &nl, ctx->d_dt2, pre);
      scope.done(nl);
      if (err != cudaSuccess) return err;
    } else if (pre && !fused && (err = split_state(ctx, u, pre, st)) != cudaSuccess) {
      return err;
    } else if (pre && fused) {
      KernelScope scope(ctx, WLSENO_KERNEL_DT, st);
      err = launch_euler2_split_pairs(u, pre, ctx->dm.N, st);
      scope.done(err == cudaSuccess ? 1 : 0);
      if (err != cudaSuccess) return err;
    }
    // k1 = u + dt L(u);  k2 = 3/4 u + 1/4 (k1 + dt L(k1));  u <- 1/3 u + 2/3 (k2 + dt L(k2))
    double* k1 = ctx->d_k1;
    double* k2 = ctx->d_k2;
    // FP32 pairs: made for u at stage 1, written by the flux for k1 and k2
    const int64_t CN = static_cast<int64_t>(ctx->scheme.n_comp) * ctx->dm.N;
    float2* p1 = ctx->d_pair ? ctx->d_pair + CN : nullptr;
    float2* p2 = ctx->d_pair ? ctx->d_pair + 2 * CN : nullptr;
    // the pairs of u stay in the scratch slot from stage 1 on (one component)
    float2* p0 = ctx->d_pair && (ctx->scheme.n_comp == 1 || fused) ? ctx->d_pair : nullptr;
    if ((err = stage_all(ctx, u, u, 0.0, 1.0, false, k1, st, pre, p1)) != cudaSuccess ||
        (err = stage_all(ctx, k1, u, 0.75, 0.25, false, k2, st, p1, p2, p0)) != cudaSuccess ||
        (err = stage_all(ctx, k2, u, 1.0 / 3.0, 2.0 / 3.0, false, u, st, p2, nullptr, p0)) != cudaSuccess)
      return err;
    return cudaSuccess;
  };
  // Capture one step as a CUDA graph (on the context's own stream) and launch
  // it n_steps times on `s`.  Not when timing, and not when `s` is itself
  // being captured (then the launches join the caller's graph).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;
  }
  // One step replays the captured step too when that graph is already there
  // for these arguments, or when the state is staged through the context's
  // own buffer (a host array: the same device address every call).
  const bool same = ctx->graph_exec && ctx->graph_u == u && ctx->graph_dt == dt &&
                    ctx->graph_cfl == cfl && ctx->graph_shape == shape_key(ctx);
  const bool use_graph = (n_steps >= 2 || (n_steps == 1 && (host || same))) && !ctx->timing &&
                         cap == cudaStreamCaptureStatusNone && !(persist && ctx->persist_no_capture);
  if (use_graph) {
    if (!same) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
      if (!ctx->cap_stream &&
          (e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(ctx, e, "capture stream");
      const int64_t l0 = ctx->launches;
      int64_t k0[WLSENO_N_KERNEL_KINDS];
      for (int k = 0; k < WLSENO_N_KERNEL_KINDS; ++k) k0[k] = ctx->by_kind[k];
      cudaGraph_t graph = nullptr;
      if ((e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(ctx, e, "begin capture");
      cudaError_t ecap = enqueue_step(ctx->cap_stream);
      e = cudaStreamEndCapture(ctx->cap_stream, &graph);
      if (ecap != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (persist) {
          // the cooperative launch could not be captured: launch it directly
          cudaGetLastError();
          ctx->persist_no_capture = true;
          ctx->launches = l0;
          for (int k = 0; k < WLSENO_N_KERNEL_KINDS; ++k) ctx->by_kind[k] = k0[k];
          for (int step = 0; step < n_steps; ++step)
            if ((e = enqueue_step(s)) != cudaSuccess) return cuda_fail(ctx, e, "persistent step");
          goto steps_done;
        }
        return cuda_fail(ctx, ecap != cudaSuccess ? ecap : e, "capture step");
      }
      e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        ctx->graph_exec = nullptr;
        return cuda_fail(ctx, e, "instantiate step graph");
      }
      ctx->graph_launches = ctx->launches - l0;
      ctx->launches = l0;
      for (int k = 0; k < WLSENO_N_KERNEL_KINDS; ++k) {
        ctx->graph_kind[k] = ctx->by_kind[k] - k0[k];
        ctx->by_kind[k] = k0[k];
      }
      ctx->graph_u = u;
      ctx->graph_dt = dt;
      ctx->graph_cfl = cfl;
      ctx->graph_shape = shape_key(ctx);
    }
    for (int step = 0; step < n_steps; ++step) {
      if ((e = cudaGraphLaunch(ctx->graph_exec, s)) != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
      ctx->launches += ctx->graph_launches;
      for (int k = 0; k < WLSENO_N_KERNEL_KINDS; ++k) ctx->by_kind[k] += ctx->graph_kind[k];
    }
  } else {
    for (int step = 0; step < n_steps; ++step)
      if ((e = enqueue_step(s)) != cudaSuccess) return cuda_fail(ctx, e, "RK step");
  }
steps_done:
  if (dt > 0.0) ctx->mesh_dt_set = false;
  if (host) {
    e = cudaMemcpyAsync(ubar, ctx->d_in, sizeof(double) * C * N, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy ubar back");
  }
  if (dt_out) {
    double v = 0.0;
    e = cudaMemcpyAsync(&v, ctx->d_dt, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read dt");
    *dt_out = v;
    ctx->last_dt = v;
    return take_nonfinite(ctx);
  } else if (host) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rk_step");
    return take_nonfinite(ctx);
  }
  return WLSENO_OK;
}

wlseno_status wlseno_autotune(wlseno_ctx* ctx, const double* ubar, int reps, void* stream,
                              double* best_us) {
  wlseno_status st = check_ready(ctx);
  if (st != WLSENO_OK) return st;
  if (!ubar || reps <= 0) return fail(ctx, WLSENO_ERR_INVALID_ARG, "null ubar or reps <= 0");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->last_stream = s;
  const int64_t N = ctx->dm.N;
  cudaError_t e;
  const double* u = ubar;
  if (!is_device_pointer(ubar)) {
    if (!ctx->d_in && (st = dalloc(ctx, &ctx->d_in, ctx->scheme.n_comp * N))) return st;
    e = cudaMemcpyAsync(ctx->d_in, ubar, sizeof(double) * ctx->scheme.n_comp * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy ubar");
    u = ctx->d_in;
  }
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(ctx, e, "event");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, e, "event");
  }
  const int G0 = ctx->G, R0 = ctx->R;
  const bool otf0 = ctx->otf;
  int bestG = G0, bestR = R0;
  bool bestO = otf0;
  float best = -1.0f;
  // (G, R, moments on the fly): the thread-per-cell shape twice in FP32-bulk
  std::vector<std::array<int, 3>> cands;
  for (auto& sh : kShapes) {
    cands.push_back({sh[0], sh[1], 0});
    if (sh[0] == 1 && ctx->scheme.precision == WLSENO_FP32_BULK) cands.push_back({sh[0], sh[1], 1});
  }
  for (auto& sh : cands) {
    if (!shape_fits(sh[0], sh[1], ctx->host.max_n)) continue;
    if (ctx->persistent && sh[0] != 1) continue;  // the persistent step runs thread per cell
    ctx->G = sh[0];
    ctx->R = sh[1];
    ctx->otf = sh[2] != 0;
    e = tune_recon(ctx, u, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = tune_recon(ctx, u, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      ctx->G = G0;
      ctx->R = R0;
      ctx->otf = otf0;
      return cuda_fail(ctx, e, "autotune");
    }
    if (best < 0.0f || ms < best) {
      best = ms;
      bestG = sh[0];
      bestR = sh[1];
      bestO = sh[2] != 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->G = bestG;
  ctx->R = bestR;
  ctx->otf = bestO;
  if (best_us) *best_us = best < 0.0f ? 0.0 : 1e3 * best / reps;
  return WLSENO_OK;
}

wlseno_status wlseno_set_mesh_dt(wlseno_ctx* ctx, const double* dt_host) {
  if (!ctx || !dt_host) return WLSENO_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, WLSENO_ERR_STATE, "call wlseno_build_stencils first");
  for (int k = 0; k < ctx->host.n_meshes; ++k)
    if (!(dt_host[k] > 0.0)) return fail(ctx, WLSENO_ERR_INVALID_ARG, "per-mesh dt must be > 0");
  DeviceGuard guard(ctx->device);
  std::vector<float2> pairs(ctx->host.n_meshes);
  for (int k = 0; k < ctx->host.n_meshes; ++k) {
    const float hi = static_cast<float>(dt_host[k]);
    pairs[k] = make_float2(hi, static_cast<float>(dt_host[k] - static_cast<double>(hi)));
  }
  cudaError_t e = cudaMemcpy(ctx->d_dt, dt_host, sizeof(double) * ctx->host.n_meshes,
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->d_dt2, pairs.data(), sizeof(float2) * pairs.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "set mesh dt");
  ctx->mesh_dt_set = true;
  return WLSENO_OK;
}

wlseno_status wlseno_step_adjoint(wlseno_ctx* ctx, const double* ubar_n, double dt,
                                  const double* gbar_next, double* gbar_n, void* stream) {
  wlseno_status st = check_ready(ctx);
  if (st != WLSENO_OK || (st = take_nonfinite(ctx)) != WLSENO_OK) return st;
  if (!ubar_n || !gbar_next || !gbar_n) return fail(ctx, WLSENO_ERR_INVALID_ARG, "null array");
  if (dt == 0.0) return fail(ctx, WLSENO_ERR_INVALID_ARG, "the adjoint needs a fixed dt (> 0, or < 0 for per-mesh steps)");
  if (ctx->scheme.pde == WLSENO_EULER)
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "the adjoint is built for the scalar equations");
  if (ctx->scheme.precision != WLSENO_FP64)
    return fail(ctx, WLSENO_ERR_INVALID_ARG,
                "the adjoint is built for FP64 contexts (its VJP would not be the derivative of the "
                "FP32-bulk step it recomputes)");
  if (ctx->dm.dim == 1)
    return fail(ctx, WLSENO_ERR_INVALID_ARG, "the adjoint is built for 2-D and 3-D meshes");
  if (ctx->scheme.balanced)
    return fail(ctx, WLSENO_ERR_INVALID_ARG,
                "the adjoint is built for fixed stencils (balanced stencils depend on the solution)");
  if (dt < 0.0 && !ctx->mesh_dt_set)
    return fail(ctx, WLSENO_ERR_STATE, "dt < 0 needs wlseno_set_mesh_dt first");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->last_stream = s;
  const int64_t N = ctx->dm.N;
  const int NP = points_per_cell(ctx);
  cudaError_t e;
  // work arrays on first use
  if (!ctx->adj.gfv) {
    AdjointWork& w = ctx->adj;
    double* tp = nullptr;
    int64_t* tr_ptr = nullptr;
    int64_t* tr_slot = nullptr;
    if ((st = dalloc(ctx, &w.gfv, N * NP)) || (st = dalloc(ctx, &w.contrib, ctx->dm.nmax * N)) ||
        (st = dalloc(ctx, &w.selfbar, N)) || (st = dalloc(ctx, &w.amin_cell, N)) ||
        (st = dalloc(ctx, &w.amin_val, N)) || (st = upload(ctx, &tr_ptr, ctx->host.tr_ptr)) ||
        (st = upload(ctx, &tr_slot, ctx->host.tr_slot)) || (st = dalloc(ctx, &tp, 6 * N)))
      return st;
    w.tr_ptr = tr_ptr;
    w.tr_slot = tr_slot;
    for (int k = 0; k < 6; ++k) ctx->d_gbar[k] = tp + k * N;
  }
  double* t = ctx->d_gbar[0];    // J_L^T products
  double* gk2 = ctx->d_gbar[1];
  double* gk1 = ctx->d_gbar[2];
  double* u = ctx->d_gbar[3];    // staged inputs / output
  double* gnext = ctx->d_gbar[4];
  double* gout = ctx->d_gbar[5];
  const bool in_host = !is_device_pointer(ubar_n), g_host = !is_device_pointer(gbar_next);
  const bool out_host = !is_device_pointer(gbar_n);
  if (in_host) {
    if ((e = cudaMemcpyAsync(u, ubar_n, sizeof(double) * N, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "copy ubar_n");
  } else {
    u = const_cast<double*>(ubar_n);
  }
  if (g_host) {
    if ((e = cudaMemcpyAsync(gnext, gbar_next, sizeof(double) * N, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "copy gbar_next");
  } else {
    gnext = const_cast<double*>(gbar_next);
  }
  double* gres = out_host ? gout : gbar_n;
  if (dt > 0.0) {
    int nl = 0;
    KernelScope scope(ctx, WLSENO_KERNEL_DT, s);
    e = launch_cfl_dt_impl(ctx->dm, ctx->sp, ctx->host.n_meshes, u, ctx->d_rmin, 0.0, dt,
                           ctx->d_lmax, ctx->d_dt, s, &nl, ctx->d_dt2);
    scope.done(nl);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dt");
    ctx->mesh_dt_set = false;
  }
  // recompute the stages k1, k2 of the step from the checkpoint u
  double* k1 = ctx->d_k1;
  double* k2 = ctx->d_k2;
  // (the same launches as the forward step, so the stages match it bitwise)
  const int64_t CN = static_cast<int64_t>(ctx->scheme.n_comp) * ctx->dm.N;
  float2* p1 = ctx->d_pair ? ctx->d_pair + CN : nullptr;
  if ((e = stage_all(ctx, u, u, 0.0, 1.0, false, k1, s, nullptr, p1)) != cudaSuccess ||
      (e = stage_all(ctx, k1, u, 0.75, 0.25, false, k2, s, p1, nullptr)) != cudaSuccess)
    return cuda_fail(ctx, e, "adjoint: forward stages");
  auto vjp = [&](const double* state, const double* lam, double* out) -> cudaError_t {
    cudaError_t err = reconstruct_one(ctx, state, nullptr, ctx->d_fvals, s);
    if (err != cudaSuccess) return err;
    int nl = 0;
    KernelScope scope(ctx, WLSENO_KERNEL_ADJOINT, s);
    err = launch_operator_vjp(ctx->dm, ctx->sp, state, ctx->d_fvals, lam, ctx->adj, out, s, &nl);
    scope.done(nl);
    return err;
  };
  auto combine = [&](const double* x, double ca, const double* y, double cb, const double* w,
                     double cc, const double* z, double cz, double* out) -> cudaError_t {
    KernelScope scope(ctx, WLSENO_KERNEL_ADJOINT, s);
    cudaError_t err = launch_adj_combine(ctx->dm, ctx->d_dt, x, ca, y, cb, w, cc, z, cz, out, s);
    scope.done(1);
    return err;
  };
  // u' = u/3 + 2/3 (k2 + dt L(k2)):  gk2 = 2/3 (g' + dt J(k2)^T g')
  // k2 = 3/4 u + 1/4 (k1 + dt L(k1)): gk1 = 1/4 (gk2 + dt J(k1)^T gk2)
  // k1 = u + dt L(u):                 g = g'/3 + 3/4 gk2 + gk1 + dt J(u)^T gk1
  if ((e = vjp(k2, gnext, t)) != cudaSuccess ||
      (e = combine(gnext, 2.0 / 3.0, nullptr, 0.0, nullptr, 0.0, t, 2.0 / 3.0, gk2)) != cudaSuccess ||
      (e = vjp(k1, gk2, t)) != cudaSuccess ||
      (e = combine(gk2, 0.25, nullptr, 0.0, nullptr, 0.0, t, 0.25, gk1)) != cudaSuccess ||
      (e = vjp(u, gk1, t)) != cudaSuccess ||
      (e = combine(gnext, 1.0 / 3.0, gk2, 0.75, gk1, 1.0, t, 1.0, gres)) != cudaSuccess)
    return cuda_fail(ctx, e, "adjoint");
  if (out_host) {
    e = cudaMemcpyAsync(gbar_n, gout, sizeof(double) * N, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy gbar_n");
  }
  if (in_host || g_host || out_host) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint");
    return take_nonfinite(ctx);
  }
  return WLSENO_OK;
}

wlseno_status wlseno_get_info(const wlseno_ctx* ctx, wlseno_info* out) {
  if (!ctx || !out) return WLSENO_ERR_INVALID_ARG;
  if (!ctx->built) return WLSENO_ERR_STATE;
  const HostSetup& H = ctx->host;
  out->dim = H.dim;
  out->order_p = H.p;
  out->m = H.m;
  out->n_comp = ctx->scheme.n_comp;
  out->n_meshes = H.n_meshes;
  out->n_cells = H.N;
  out->stencil_nnz = H.nnz;
  out->max_stencil = H.max_n;
  out->min_stencil = H.min_n;
  out->quad_per_facet = H.nq;
  out->lanes_per_cell = ctx->G;
  out->rows_per_lane = ctx->R;
  out->moments_mode = ctx->otf ? 1 : 0;
  out->persistent = ctx->persistent ? 1 : 0;
  return WLSENO_OK;
}

wlseno_status wlseno_get_stencils(const wlseno_ctx* ctx, int64_t* row_ptr, int64_t* cols) {
  if (!ctx) return WLSENO_ERR_INVALID_ARG;
  if (!ctx->built) return WLSENO_ERR_STATE;
  if (row_ptr) std::memcpy(row_ptr, ctx->host.row_ptr.data(), sizeof(int64_t) * ctx->host.row_ptr.size());
  if (cols) std::memcpy(cols, ctx->host.cols.data(), sizeof(int64_t) * ctx->host.cols.size());
  return WLSENO_OK;
}

wlseno_status wlseno_get_geometry(const wlseno_ctx* ctx, double* centroid, double* volume,
                                  double* h, double* inradius) {
  if (!ctx) return WLSENO_ERR_INVALID_ARG;
  if (!ctx->built) return WLSENO_ERR_STATE;
  const HostSetup& H = ctx->host;
  if (centroid) std::memcpy(centroid, H.centroid.data(), sizeof(double) * H.centroid.size());
  if (volume) std::memcpy(volume, H.volume.data(), sizeof(double) * H.volume.size());
  if (h) std::memcpy(h, H.h.data(), sizeof(double) * H.h.size());
  if (inradius) std::memcpy(inradius, H.inradius.data(), sizeof(double) * H.inradius.size());
  return WLSENO_OK;
}

wlseno_status wlseno_get_diagnostics(wlseno_ctx* ctx, wlseno_diagnostics* out) {
  if (!ctx || !out) return WLSENO_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->kernel_launches = ctx->launches;
  out->last_dt = ctx->last_dt;
  for (int k = 0; k < WLSENO_N_KERNEL_KINDS; ++k) out->launches_by_kind[k] = ctx->by_kind[k];
  if (!ctx->built) return WLSENO_OK;
  DeviceGuard guard(ctx->device);
  unsigned long long c[kCounters] = {0, 0, 0, 0, 0};
  cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
  if (e == cudaSuccess) e = cudaMemcpy(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read counters");
  out->flagged_cells = static_cast<int64_t>(c[0]);
  out->rank_deficient = static_cast<int64_t>(c[1]);
  out->nonfinite = static_cast<int64_t>(c[2]);
  out->positivity_fallbacks = static_cast<int64_t>(c[3]);
  out->balanced_cells = static_cast<int64_t>(c[4]);
  for (int k = 0; k < WLSENO_N_KERNEL_KINDS; ++k) out->launches_by_kind[k] = ctx->by_kind[k];
  for (const auto& t : ctx->timed) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) out->kernel_ms[t.kind] += ms;
    else cudaGetLastError();
  }
  return WLSENO_OK;
}

wlseno_status wlseno_set_wait_limit(wlseno_ctx* ctx, int64_t max_polls) {
  if (!ctx || max_polls < 0) return WLSENO_ERR_INVALID_ARG;
  ctx->spin_cap = max_polls == 0 ? kDefaultSpinCap : static_cast<long long>(max_polls);
  return WLSENO_OK;
}

wlseno_status wlseno_set_timing(wlseno_ctx* ctx, int enable) {
  if (!ctx) return WLSENO_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  reset_kind_stats(ctx);
  return WLSENO_OK;
}

}  // extern "C"
